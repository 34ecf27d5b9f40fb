"""Learned probe count on the GPU vs the fp64 oracle (oracle/probe_mlp.py).

The network, its features and its labels are an extension (the paper has
none); these tests check the GPU kernels against the oracle's restatement
and show what the trained network gains over fixed-t probing.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import probe_mlp
from parity_util import topk_mismatches

pytestmark = pytest.mark.gpu


def _t(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t.to(dtype) if dtype is not None else t


def _split(flat, d_in, hidden):
    sizes = [("W1", (hidden, d_in)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
             ("W3", (1, hidden)), ("b3", (1,))]
    out, pos = {}, 0
    for name, shape in sizes:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[pos:pos + n], dtype=np.float64).reshape(shape)
        pos += n
    assert pos == flat.size
    return out


def _random_params(d_in, hidden, seed):
    from paper_2404_00774_gb300 import probe
    flat = probe.he_uniform_params(d_in, hidden, seed)
    rng = np.random.default_rng(seed + 1)
    p = _split(flat, d_in, hidden)
    for name in ("b1", "b2", "b3"):                 # non-zero biases exercise their gradients
        p[name][:] = rng.standard_normal(p[name].shape) * 0.1
    flat = np.concatenate([p[n].reshape(-1) for n in probe_mlp.PARAM_NAMES]).astype(np.float32)
    return flat, _split(flat, d_in, hidden)


@pytest.mark.parametrize("bf16,rtol", [(False, 2e-5), (True, 2e-2)])
def test_mlp_forward_and_gradients_match_oracle(soar, bf16, rtol):
    d_in, hidden, B = 40, 48, 70                     # ragged against the 64-wide tiles
    flat, p = _random_params(d_in, hidden, 3)
    rng = np.random.default_rng(4)
    Z = rng.standard_normal((B, d_in)).astype(np.float32)
    target = rng.standard_normal(B).astype(np.float32)
    if bf16:
        # bf16 mode multiplies bf16-rounded weights and inputs: the oracle gets
        # the same rounded values, so only the rounding of intermediate
        # operands (activations, gradients) separates the two
        flat = oracle.bf16_round(flat)
        Z = oracle.bf16_round(Z)
        p = _split(flat, d_in, hidden)
    y = soar.soar_mlp_forward(_t(flat), d_in, hidden, _t(Z), bf16).cpu().numpy()
    y_ref, _ = probe_mlp.forward(p, Z)
    scale = np.abs(y_ref).max()
    assert np.abs(y - y_ref).max() <= rtol * scale
    g, loss = soar.soar_mlp_backward(_t(flat), d_in, hidden, _t(Z), _t(target), bf16)
    g = _split(g.cpu().numpy(), d_in, hidden)
    g_ref = probe_mlp.backward(p, Z, target)
    for name in probe_mlp.PARAM_NAMES:
        err = np.abs(g[name] - g_ref[name]).max()
        assert err <= rtol * max(np.abs(g_ref[name]).max(), 1e-12), (name, err)
    assert float(loss) == pytest.approx(probe_mlp.loss(p, Z, target), rel=10 * rtol)


def test_adam_step_matches_oracle(soar):
    d_in, hidden = 10, 16
    flat, p = _random_params(d_in, hidden, 5)
    rng = np.random.default_rng(6)
    g = rng.standard_normal(flat.size).astype(np.float32)
    m = (0.1 * rng.standard_normal(flat.size)).astype(np.float32)
    v = np.abs(0.1 * rng.standard_normal(flat.size)).astype(np.float32)
    P, G, M, V = _t(flat), _t(g), _t(m), _t(v)
    soar.soar_mlp_adam(P, G, M, V, step=3, lr=1e-2)
    pd, gd = _split(flat, d_in, hidden), _split(g, d_in, hidden)
    md, vd = _split(m, d_in, hidden), _split(v, d_in, hidden)
    probe_mlp.adam_step(pd, gd, md, vd, 3, 1e-2)
    want = np.concatenate([pd[n].reshape(-1) for n in probe_mlp.PARAM_NAMES])
    np.testing.assert_allclose(P.cpu().numpy(), want, rtol=1e-5, atol=1e-6)


@pytest.fixture(scope="module")
def tiny_index(soar):
    X, Q, init = synth.workload_arrays("tiny")
    C = oracle.kmeans(X, init, 10)
    A = oracle.soar_assign(X, C, 1.0, 1)
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    yield X, Q, C, A, ix
    ix.close()


def test_probe_features_match_oracle(soar, tiny_index):
    X, Q, C, A, ix = tiny_index
    Z = soar.soar_probe_features(ix, _t(Q), top=32).cpu().numpy()
    Z_ref = probe_mlp.features(Q, C, top=32)
    np.testing.assert_allclose(Z, Z_ref, rtol=1e-5, atol=1e-6)


def test_probe_labels_match_oracle(soar, tiny_index):
    X, Q, C, A, ix = tiny_index
    truth, _ = oracle.mips_topk(Q, X, 10)
    got = soar.soar_probe_labels(ix, _t(Q), _t(truth), 0.9).cpu().numpy()
    want = oracle.probe_labels(Q, C, A, truth, 0.9)
    # a label can only move where two centroid scores tie to fp32 precision
    assert (got != want).sum() <= 1, np.nonzero(got != want)[0]
    got8 = soar.soar_probe_labels(ix, _t(Q), _t(truth), 0.5).cpu().numpy()
    want8 = oracle.probe_labels(Q, C, A, truth, 0.5)
    assert (got8 != want8).sum() <= 1


def test_probe_labels_ignore_ids_outside_the_index(soar, tiny_index):
    X, Q, C, A, ix = tiny_index
    truth, _ = oracle.mips_topk(Q[:4], X, 10)
    bad = truth.copy()
    bad[:, -1] = X.shape[0] + 5                     # never found: position "infinite"
    got = soar.soar_probe_labels(ix, _t(Q[:4]), _t(bad), 0.9).cpu().numpy()
    assert np.all(got > 0)


def test_learned_probe_count_saves_probes_at_recall_target(soar):
    from paper_2404_00774_gb300 import probe
    mix = synth.Mixture(48, 100, "anisotropic", 0.0, param_seed=41, mean_scale=0.2)
    n, c, k = 60_000, 256, 10
    X = _t(mix.sample(n, 42))
    Qtr, Qcal, Qte = (_t(mix.sample(m, s)) for m, s in [(20_000, 43), (2_000, 44), (2_000, 45)])
    C = soar.soar_train_centroids(X, c, 8, _t(synth.init_indices(n, c, 46)))
    ix = soar.soar_index_build(X, C, soar.soar_assign(X, C, 1.0, 1))
    truth = {name: soar.soar_exact_mips(X, Qs, k)[0] for name, Qs in [("tr", Qtr), ("cal", Qcal), ("te", Qte)]}
    Z = {name: soar.soar_probe_features(ix, Qs, 64) for name, Qs in [("tr", Qtr), ("cal", Qcal), ("te", Qte)]}
    labels = soar.soar_probe_labels(ix, Qtr, truth["tr"], 0.9)
    params, losses = probe.train(ix, Z["tr"], labels, hidden=64, steps=600, batch=1024, lr=2e-3, bf16=True)
    assert losses[-1] < losses[0]
    alpha = probe.calibrate_alpha(ix, params, 64, Z["cal"], Qcal, truth["cal"], k, c)
    t = soar.soar_mlp_predict_probes(params, Z["te"].shape[1], 64, Z["te"], alpha, c, True)
    ids, _ = soar.soar_search(ix, Qte, k, int(t.max()), t_per_query=t)
    rec_mlp = probe.recall(ids, truth["te"])
    # the fixed probe count that reaches the same recall on the same queries
    fixed = next(tt for tt in range(1, c + 1)
                 if probe.recall(soar.soar_search(ix, Qte, k, tt)[0], truth["te"]) >= rec_mlp - 1e-9)
    mean_t = float(t.float().mean())
    print(f"learned probe: recall {rec_mlp:.4f} with mean t {mean_t:.2f}; fixed t needs {fixed}")
    assert rec_mlp >= 0.88
    assert mean_t < fixed
    ix.close()


def test_search_learned_equals_features_predict_search_and_oracle(soar, tiny_index):
    # the one-call learned-probe search against the three calls it fuses
    # (features, prediction, search with those counts) and against the
    # oracle's IVF search with the same per-query counts
    X, Q, C, A, ix = tiny_index
    d, top, hidden, cap = X.shape[1], 32, 64, 16
    params = _t(_random_params(d + top, hidden, 51)[0])
    Qd = _t(Q)
    Z = soar.soar_probe_features(ix, Qd, top)
    y = soar.soar_mlp_forward(params, d + top, hidden, Z, bf16=True)
    alpha = float(6.0 / torch.exp(y.median()))     # counts spread around 6
    t_ref = soar.soar_mlp_predict_probes(params, d + top, hidden, Z, alpha, cap, True)
    ids, scores, t = soar.soar_search_learned(ix, Qd, 10, top, params, hidden, alpha, cap, bf16=True)
    np.testing.assert_array_equal(t.cpu().numpy(), t_ref.cpu().numpy())
    tn = t.cpu().numpy()
    assert tn.min() >= 1 and tn.max() <= cap and len(np.unique(tn)) > 2
    want_i, want_s = soar.soar_search(ix, Qd, 10, top, t_per_query=t)
    np.testing.assert_array_equal(ids.cpu().numpy(), want_i.cpu().numpy())
    np.testing.assert_array_equal(scores.cpu().numpy(), want_s.cpu().numpy())
    off, ivf = oracle.build_ivf(A, C.shape[0])
    wi, ws = oracle.ivf_search(Q, X, C, off, ivf, 10, top, t_per_query=tn)
    Xd, Qf = X.astype(np.float64), Q.astype(np.float64)
    assert topk_mismatches(ids.cpu().numpy(), wi, ws, lambda q, i: Xd[np.asarray(i, np.int64)] @ Qf[q]) == []
