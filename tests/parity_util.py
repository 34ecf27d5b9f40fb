"""Comparison rules between the GPU path and the fp64 oracle.

* Integer work (inverted lists, codes): bit-exact.
* Assignments: equal, except a decision whose oracle loss gap (runner-up
  minus best) is below 1e-5 of the best loss; after such a near-tie the later
  spills of that row are not compared (they depend on the earlier choice).
* Top-t / top-k lists: position by position the same id, or a different id
  whose exact score lies within 1e-4 (relative) of the oracle's score at that
  position (a tie swap); ids distinct; padding (-1) where the oracle pads.
"""
import numpy as np

ASSIGN_REL = 1e-5
TOPK_REL = 1e-4


def assign_mismatches(got, want, gaps, best, rel=ASSIGN_REL):
    """Rows whose assignment differs without an oracle near-tie excusing it."""
    got = np.asarray(got).reshape(want.shape)
    bad = []
    exempt = 0
    for i in np.nonzero((got != want).any(axis=1))[0]:
        for j in range(want.shape[1]):
            if got[i, j] == want[i, j]:
                continue
            if gaps[i, j] <= rel * max(best[i, j], 1e-30):
                exempt += 1
                break            # later columns depend on this choice
            bad.append(i)
            break
    return np.array(bad, dtype=np.int64), exempt


def rel_close(a, b, rel):
    return np.abs(a - b) <= rel * np.maximum(np.abs(b), 1e-6)


def topk_mismatches(got_ids, want_ids, want_scores, exact_score, rel=TOPK_REL):
    """Queries whose top-k differs beyond tie swaps.

    exact_score(q, ids) -> fp64 exact scores of `ids` for query q.
    """
    bad = []
    for q in range(want_ids.shape[0]):
        g, w = np.asarray(got_ids[q]), np.asarray(want_ids[q])
        if np.array_equal(g, w):
            continue
        gv = g[g >= 0]
        if len(set(gv.tolist())) != len(gv) or (g >= 0).sum() != (w >= 0).sum():
            bad.append(q)
            continue
        diff = (g != w) & (w >= 0)
        es = exact_score(q, g[diff])
        if not np.all(rel_close(es, want_scores[q][diff], rel)):
            bad.append(q)
    return bad


def score_errors(got_ids, got_scores, exact_score):
    """Max and mean |fp32 score - fp64 exact score| over the returned ids."""
    errs = []
    for q in range(got_ids.shape[0]):
        ok = got_ids[q] >= 0
        if ok.any():
            errs.append(np.abs(got_scores[q][ok] - exact_score(q, got_ids[q][ok])))
    e = np.concatenate(errs) if errs else np.zeros(1)
    return float(e.max()), float(e.mean())
