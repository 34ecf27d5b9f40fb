"""Mutation check of the oracle's pins (test infrastructure, run by hand:
``python tests/oracle_mutations.py [name filter ...]``).

Plants one plausible mistake at a time in oracle/*.py (a dropped term, a
flipped sign or comparison, the other tie order, an off-by-one index, a
transposed operand), runs the CPU suite (``-m "not gpu"``, without the ABI
tests, which do not touch the oracle) and reports every mistake that no test
catches.  The oracle files are restored from memory after each run and in a
``finally`` block.  Not collected by pytest."""
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SO = "oracle/soar_oracle.py"
PM = "oracle/probe_mlp.py"

M = [
    # (name, file, old, new, occurrence)
    ("topk tie to higher id", SO, "np.lexsort((ids[cand], -scores[cand]))", "np.lexsort((-ids[cand], -scores[cand]))", 0),
    ("topk strict kth", SO, "cand = np.nonzero(scores >= kth)[0]", "cand = np.nonzero(scores > kth)[0]", 0),
    ("topk pad score 0", SO, "out_s = np.full(k, -np.inf, dtype=F64)\n    if n == 0", "out_s = np.full(k, 0.0, dtype=F64)\n    if n == 0", 0),
    ("mips sign", SO, "S = Q[lo:lo + chunk] @ Xd.T", "S = -(Q[lo:lo + chunk] @ Xd.T)", 0),
    ("recall denominator", SO, "out[i] = len(f.intersection(int(v) for v in truth[i])) / k", "out[i] = len(f.intersection(int(v) for v in truth[i])) / max(k - 1, 1)", 0),
    ("recall_tol strict", SO, "np.sum(s >= kth - rel * abs(kth))", "np.sum(s > kth + rel * abs(kth))", 0),
    ("rank strict", SO, "@ q >= sv))", "@ q > sv))", 0),
    ("sqdist factor 2", SO, "D = x2[:, None] - 2.0 * (Xc @ C.T) + c2[None, :]", "D = x2[:, None] - 1.0 * (Xc @ C.T) + c2[None, :]", 0),
    ("sqdist drop c2", SO, "D = x2[:, None] - 2.0 * (Xc @ C.T) + c2[None, :]", "D = x2[:, None] - 2.0 * (Xc @ C.T)", 0),
    ("primary gap not relative", SO, "gap[lo:lo + chunk] = D.min(axis=1) - best[lo:lo + chunk]", "gap[lo:lo + chunk] = D.min(axis=1)", 0),
    ("primary tie to higher", SO, "a = np.argmin(D, axis=1)", "a = D.shape[1] - 1 - np.argmin(D[:, ::-1], axis=1)", 0),
    ("soar_loss sign", SO, "return float(rp @ rp) + lam * pen", "return float(rp @ rp) - lam * pen", 0),
    ("soar_loss unnormalised", SO, "pen = 0.0 if nr == 0.0 else float((rp @ r) / nr) ** 2", "pen = 0.0 if nr == 0.0 else float(rp @ r) ** 2", 0),
    ("assign proj sign", SO, "proj = np.einsum(\"ij,ij->i\", Xc, rhat)[:, None] - rhat @ C.T", "proj = np.einsum(\"ij,ij->i\", Xc, rhat)[:, None] + rhat @ C.T", 0),
    ("assign pen not accumulated", SO, "pen += proj * proj", "pen = proj * proj", 0),
    ("assign lambda dropped", SO, "L = D + lam * pen", "L = D + pen", 0),
    ("assign prior not excluded", SO, "L[taken] = np.inf", "L[taken] = L[taken]", 0),
    ("assign residual of primary only", SO, "r = Xc - C[prev]", "r = Xc - C[a0]", 0),
    ("assign gap not relative", SO, "gaps[lo:lo + m, j] = nxt - best", "gaps[lo:lo + m, j] = nxt", 0),
    ("spill tie to higher", SO, "aj = np.argmin(L, axis=1)", "aj = L.shape[1] - 1 - np.argmin(L[:, ::-1], axis=1)", 0),
    ("primary in assign tie higher", SO, "a0 = np.argmin(D, axis=1)", "a0 = D.shape[1] - 1 - np.argmin(D[:, ::-1], axis=1)", 0),
    ("kmeans mean off by one", SO, "C[nz] = (sums[nz] / cnt[nz, None]).astype(np.float32)", "C[nz] = (sums[nz] / (cnt[nz, None] + 1)).astype(np.float32)", 0),
    ("kmeans empty cluster", SO, "nz = cnt > 0", "nz = cnt >= 0", 0),
    ("kmeans fp32 sums", SO, "sums = np.zeros((c, d), dtype=F64)", "sums = np.zeros((c, d), dtype=np.float32)", 0),
    ("ivf member order", SO, "order = np.lexsort((pid, part))", "order = np.lexsort((-pid, part))", 0),
    ("ivf offsets shifted", SO, "offsets[1:] = np.cumsum(cnt)", "offsets[:-1] = np.cumsum(cnt)", 0),
    ("select sign", SO, "a, b = topk_desc(S[i], t)", "a, b = topk_desc(-S[i], t)", 0),
    ("ivf no dedup", SO, "mem = np.unique(mem).astype(np.int64)", "mem = mem.astype(np.int64)", 0),
    ("ivf per-query counts ignored", SO, "tq = t if t_per_query is None else int(t_per_query[i])\n        parts = top[i, :tq]", "tq = t\n        parts = top[i, :tq]", 0),
    ("pq per-query counts ignored", SO, "tq = t if t_per_query is None else int(t_per_query[i])\n        lut", "tq = t\n        lut", 0),
    ("ivf one probe short", SO, "parts = top[i, :tq]", "parts = top[i, :max(tq - 1, 1)]", 0),
    ("ivf wrong query", SO, "s = np.asarray(X[mem], dtype=F64) @ Q[i]", "s = np.asarray(X[mem], dtype=F64) @ Q[(i + 1) % nq]", 0),
    ("pq residual sign", SO, "np.asarray(X, dtype=np.float32) - np.asarray(C, dtype=np.float32)[np.asarray(part)]", "np.asarray(X, dtype=np.float32) + np.asarray(C, dtype=np.float32)[np.asarray(part)]", 0),
    ("pq encode wrong codebook", SO, "B[s])[0]", "B[(s + 1) % B.shape[0]])[0]", 0),
    ("pq codes from partition 0", SO, "part = np.repeat(np.arange(len(offsets) - 1), np.diff(offsets))", "part = np.zeros(int(offsets[-1]), dtype=np.int64)", 0),
    ("pq base dropped", SO, "base = float(Cd[p] @ Q[i])", "base = 0.0", 0),
    ("pq last copy wins", SO, "if pid not in seen:", "if True:", 0),
    ("pq lut transposed", SO, "lut = np.einsum(\"sjd,sd->sj\", Bd, Q[i].reshape(m, PQ_DIMS))", "lut = np.einsum(\"sjd,sd->sj\", Bd[:, :, ::-1], Q[i].reshape(m, PQ_DIMS))", 0),
    ("pq shortlist short", SO, "cand, _ = topk_desc(approx, rescore, mem)", "cand, _ = topk_desc(approx, max(rescore - 1, 1), mem)", 0),
    ("multilevel t/t1 swapped", SO, "return ivf_search(Q, C, C2, offsets2, ids2, t, t1)", "return ivf_search(Q, C, C2, offsets2, ids2, t1, t)", 0),
    ("multilevel drops id 0", SO, "parts = top[i][top[i] >= 0]", "parts = top[i][top[i] >= 1]", 0),
    ("multilevel no dedup", SO, "mem = np.unique(mem).astype(np.int64)", "mem = mem.astype(np.int64)", 1),
    ("positions tie", SO, "order = np.lexsort((np.arange(c), -S[i]))", "order = np.lexsort((-np.arange(c), -S[i]))", 0),
    ("positions zero based", SO, "pos[i, order] = np.arange(1, c + 1)", "pos[i, order] = np.arange(0, c)", 0),
    ("kmr strict rank", SO, "r = np.sum(S[i][None, :] >= S[i, p][:, None], axis=1)", "r = np.sum(S[i][None, :] > S[i, p][:, None], axis=1)", 0),
    ("kmr last assignment only", SO, "best = np.minimum(best, r)", "best = r", 0),
    ("kmr strict t", SO, "hits += np.sum(best[None, :] <= ts[:, None], axis=1)", "hits += np.sum(best[None, :] < ts[:, None], axis=1)", 0),
    ("datapoints one short", SO, "return sizes[top].sum(axis=1)", "return sizes[top[:, :-1]].sum(axis=1)", 0),
    ("labels floor", SO, "need = int(np.ceil(target * k - 1e-9))", "need = int(np.floor(target * k))", 0),
    ("labels max over copies", SO, "pv = pos[i][assign[truth[i]]].min(axis=1)", "pv = pos[i][assign[truth[i]]].max(axis=1)", 0),
    ("labels primary only", SO, "pv = pos[i][assign[truth[i]]].min(axis=1)", "pv = pos[i][assign[truth[i], 0]]", 0),
    ("bf16 no tie to even", SO, "u = (u + 0x7FFF + lsb) & 0xFFFF0000", "u = (u + 0x7FFF) & 0xFFFF0000", 0),
    ("fp8 subnormal exponent", SO, "e = np.maximum(e, -6.0)", "e = np.maximum(e, -7.0)", 0),
    ("fp8 mantissa bits", SO, "step = np.exp2(e - 3.0)", "step = np.exp2(e - 2.0)", 0),
    ("fp8 saturation", SO, "q = np.minimum(q, 448.0)", "q = np.minimum(q, 480.0)", 0),
    ("fp8 scale 447", SO, "amax / np.float32(448.0)", "amax / np.float32(447.0)", 0),
    ("fp8 zero row scale", SO, "np.float32(1.0)).astype(np.float32)", "np.float32(0.0)).astype(np.float32)", 0),
    ("fp8 select drop centroid scale", SO, " * qs[:, None].astype(F64) * cs[None, :].astype(F64)", " * qs[:, None].astype(F64)", 0),
    ("precision drop row scale", SO, "* xs.astype(F64) * F64(qs[i])", "* F64(qs[i])", 0),
    ("precision shortlist short", SO, "cand, _ = topk_desc(approx, rescore, mem)", "cand, _ = topk_desc(approx, max(rescore - 1, 1), mem)", 1),
    ("precision rescored by fp8", SO, "exact = np.asarray(X[cand], dtype=F64) @ Qf[i].astype(F64)", "exact = np.asarray(X[cand], dtype=F64) @ (q8[i].astype(F64) * F64(qs[i]))", 0),
    ("precision exact selection", SO, "top, _ = select_partitions_fp8(Qf, C, t)", "top, _ = select_partitions(Qf, C, t)", 0),
    ("precision no dedup", SO, "mem = np.unique(np.concatenate([ids[offsets[p]:offsets[p + 1]] for p in parts])).astype(np.int64)", "mem = np.concatenate([ids[offsets[p]:offsets[p + 1]] for p in parts]).astype(np.int64)", 0),
    ("kmr normalisation", SO, "return hits / (k * S.shape[0])", "return hits / S.shape[0]", 0),
    ("fp8 sign dropped", SO, "return (np.sign(v) * q).astype(np.float32)", "return q.astype(np.float32)", 0),
    ("fp8 codes unscaled", SO, "codes = fp8_e4m3_round((R / scale[:, None]).astype(np.float32))", "codes = fp8_e4m3_round(R.astype(np.float32))", 0),
    ("bf16 truncation", SO, "u = (u + 0x7FFF + lsb) & 0xFFFF0000", "u = u & 0xFFFF0000", 0),
    ("ivf sorted by point first", SO, "order = np.lexsort((pid, part))", "order = np.lexsort((part, pid))", 0),
    ("kmeans seeds reversed", SO, "C = np.asarray(X[np.asarray(init_idx)], dtype=np.float32).copy()", "C = np.asarray(X[np.asarray(init_idx)[::-1]], dtype=np.float32).copy()", 0),
    ("datapoints cumulative sizes", SO, "sizes = np.diff(np.asarray(offsets))", "sizes = np.asarray(offsets)[1:]", 0),
    ("forward b3 sign", PM, "y = (h2 @ p[\"W3\"].T)[:, 0] + p[\"b3\"][0]", "y = (h2 @ p[\"W3\"].T)[:, 0] - p[\"b3\"][0]", 0),
    ("backward W2 transposed", PM, "g[\"W2\"] = ga2.T @ h1", "g[\"W2\"] = h1.T @ ga2", 0),
    ("adam no v bias correction", PM, "vh = v[name] / (1 - beta2 ** step)", "vh = v[name]", 0),
    ("features drop the best", PM, "S = -np.sort(-S, axis=1)[:, :top]", "S = -np.sort(-S, axis=1)[:, 1:top + 1]", 0),
    ("features ascending", PM, "S = -np.sort(-S, axis=1)[:, :top]", "S = np.sort(S, axis=1)[:, ::-1][:, 1:top + 1] if S.shape[1] > top else -np.sort(-S, axis=1)[:, :top]", 0),
    ("features order swapped", PM, "np.concatenate([Q, S], axis=1)", "np.concatenate([S, Q], axis=1)", 0),
    ("forward relu1 dropped", PM, "h1 = np.maximum(a1, 0.0)", "h1 = a1", 0),
    ("forward W2 transposed", PM, "a2 = h1 @ p[\"W2\"].T + p[\"b2\"]", "a2 = h1 @ p[\"W2\"] + p[\"b2\"]", 0),
    ("forward b1 dropped", PM, "a1 = Z @ p[\"W1\"].T + p[\"b1\"]", "a1 = Z @ p[\"W1\"].T", 0),
    ("loss sum", PM, "np.mean((y - target) ** 2)", "np.sum((y - target) ** 2)", 0),
    ("backward factor 2", PM, "gy = 2.0 * (y - np.asarray(target, dtype=F64)) / B", "gy = (y - np.asarray(target, dtype=F64)) / B", 0),
    ("backward relu2 mask", PM, "ga2 = gh2 * (a2 > 0)", "ga2 = gh2", 0),
    ("backward b1 mean", PM, "g[\"b1\"] = ga1.sum(axis=0)", "g[\"b1\"] = ga1.mean(axis=0)", 0),
    ("adam no bias correction", PM, "mh = m[name] / (1 - beta1 ** step)", "mh = m[name]", 0),
    ("adam abs second moment", PM, "v[name] = beta2 * v[name] + (1 - beta2) * g[name] ** 2", "v[name] = beta2 * v[name] + (1 - beta2) * np.abs(g[name])", 0),
    ("adam eps inside sqrt", PM, "p[name] = p[name] - lr * mh / (np.sqrt(vh) + eps)", "p[name] = p[name] - lr * mh / np.sqrt(vh + eps)", 0),
    ("predict round", PM, "np.ceil(alpha * np.exp(y))", "np.round(alpha * np.exp(y))", 0),
    ("predict clamp 0", PM, "np.clip(np.ceil(alpha * np.exp(y)), 1, c)", "np.clip(np.ceil(alpha * np.exp(y)), 0, c)", 0),
    ("init fan_out", PM, "lim = np.sqrt(6.0 / fan_in)", "lim = np.sqrt(6.0 / fan_out)", 0),
]


def apply(src, old, new, occ):
    pos = -1
    for _ in range(occ + 1):
        pos = src.find(old, pos + 1)
        if pos < 0:
            return None
    return src[:pos] + new + src[pos + len(old):]


def main():
    only = sys.argv[1:]
    orig = {f: open(os.path.join(ROOT, f)).read() for f in (SO, PM)}
    survivors, errors = [], []
    try:
        for name, f, old, new, occ in M:
            if only and not any(o in name for o in only):
                continue
            mutated = apply(orig[f], old, new, occ)
            if mutated is None:
                errors.append(name)
                print(f"NOT APPLIED  {name}", flush=True)
                continue
            with open(os.path.join(ROOT, f), "w") as fh:
                fh.write(mutated)
            r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "not gpu", "-x", "-q",
                                "-p", "no:cacheprovider", "--deselect", "tests/test_abi_args.py",
                                "--deselect", "tests/test_abi.py"], cwd=ROOT, capture_output=True, text=True,
                               timeout=900)
            caught = r.returncode != 0
            last = [ln for ln in r.stdout.splitlines() if ln.strip()][-1:] or [""]
            print(f"{'caught  ' if caught else 'SURVIVED'}  {name}   ({last[0][:90]})", flush=True)
            if not caught:
                survivors.append(name)
            with open(os.path.join(ROOT, f), "w") as fh:
                fh.write(orig[f])
    finally:
        for f, s in orig.items():
            with open(os.path.join(ROOT, f), "w") as fh:
                fh.write(s)
    print("survivors:", survivors)
    print("not applied:", errors)


if __name__ == "__main__":
    main()
