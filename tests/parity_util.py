"""Comparison of library results with the CPU oracle (shared by GPU tests).

The bar (stated by the library's design): indices equal the oracle's
exactly, ties included; scores within 1e-9 * ||u|| ||i|| of the oracle's
FP64 value (the library's own bound is about 2.3e-10 at f = 128), which is
far inside the 1e-6 relative score tolerance of the exactness target.
"""
import numpy as np

import oracle

SCORE_TOL = 1e-9


def check_against_oracle(U, I, K, idx, sc, rows=None, ref=None):
    """U, I: FP32 inputs; idx/sc: library outputs for all users (numpy);
    rows: user rows to check (default all); ref: precomputed oracle output
    for those rows."""
    rows = np.arange(U.shape[0]) if rows is None else np.asarray(rows)
    if ref is None:
        ref = oracle.topk(U[rows], I, K)
    ref_idx, ref_sc = ref
    got_idx, got_sc = idx[rows], sc[rows]
    bad = np.nonzero((got_idx != ref_idx).any(axis=1))[0]
    assert bad.size == 0, (f"{bad.size} of {rows.size} users differ from the oracle; first user {rows[bad[0]]}: "
                           f"got {got_idx[bad[0]].tolist()} want {ref_idx[bad[0]].tolist()}")
    nu = np.linalg.norm(U[rows].astype(np.float64), axis=1)[:, None]
    ni = np.linalg.norm(I.astype(np.float64), axis=1)[ref_idx]
    err = np.abs(got_sc - ref_sc)
    assert (err <= SCORE_TOL * nu * ni + 1e-300).all(), f"max score error {err.max()}"
    return err.max() if err.size else 0.0
