"""Index persistence (soar_index_save / soar_index_load) on the GPU.

A saved and reloaded index must describe the same inverted lists (Section
2.2, with the spilled copies of Section 3.5) and answer every search bit for
bit like the index it was saved from; damaged files are rejected.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _t(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t.to(dtype) if dtype is not None else t


@pytest.fixture(scope="module")
def data():
    X, Q, init = synth.workload_arrays("tiny", nq=300)
    C = oracle.kmeans(X, init, 5)
    A = oracle.soar_assign(X, C, 1.0, 1)
    return X, Q, C, A


@pytest.mark.parametrize("mode", ["f32", "fp8"])
def test_save_load_round_trip_is_bit_exact(soar, data, tmp_path, mode):
    X, Q, C, A = data
    if mode == "f32":
        ix = soar.soar_index_build(_t(X), _t(C), _t(A))
        runs = [(10, 4, 0), (64, 9, 0), (1, 1, 0)]
        Qd = _t(Q)
    else:
        ix = soar.soar_index_build(_t(X, torch.bfloat16), _t(C), _t(A), mode=soar.SOAR_SCORE_FP8)
        runs = [(10, 4, 100)]
        Qd = _t(Q, torch.bfloat16)
    path = str(tmp_path / f"ix_{mode}.soar")
    soar.soar_index_save(ix, path)
    ix2 = soar.soar_index_load(path)
    a, b = ix.info, ix2.info
    for f in ("n", "d", "c", "spills", "mode", "dtype", "row_stride", "rows", "max_partition", "device_bytes"):
        assert getattr(a, f) == getattr(b, f), f
    assert torch.equal(ix.offsets(), ix2.offsets())
    assert torch.equal(ix.ids(), ix2.ids())
    assert torch.equal(ix.vectors(), ix2.vectors())
    off, ids = oracle.build_ivf(A, C.shape[0])
    np.testing.assert_array_equal(ix2.offsets().cpu().numpy(), off)
    np.testing.assert_array_equal(ix2.ids().cpu().numpy(), ids)
    for k, t, r in runs:
        i1, s1 = soar.soar_search(ix, Qd, k, t, rescore=r)
        i2, s2 = soar.soar_search(ix2, Qd, k, t, rescore=r)
        assert torch.equal(i1, i2) and torch.equal(s1, s2), (k, t)
    ix.close()
    ix2.close()


def test_load_rejects_damaged_files(soar, data, tmp_path):
    X, Q, C, A = data
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    path = tmp_path / "ix.soar"
    soar.soar_index_save(ix, str(path))
    ix.close()
    raw = path.read_bytes()
    for name, blob in [("truncated", raw[: len(raw) - 100]), ("trailing", raw + b"\0"),
                       ("magic", b"XXXXXXXX" + raw[8:])]:
        bad = tmp_path / f"bad_{name}.soar"
        bad.write_bytes(blob)
        with pytest.raises(soar.SoarError) as e:
            soar.soar_index_load(str(bad))
        assert e.value.status == soar.SOAR_EINVAL, name
