"""What single precision does to the pair eigenproblems by itself (the
basis of the FP32 form's stated eigenvalue errors): the Schur complements of
the 16^3 channels workload computed with single-precision Cholesky,
triangular solve and product (LAPACK/BLAS) differ from FP64 by about 1e-7 of
their largest entry and stay positive semidefinite, and the top eigenvalue of
each pair pencil built from them (eq. eig-matrix, the oracle's literal form)
lies within 3% of the FP64 value."""
import numpy as np
import scipy.linalg as sla

import amb_inputs as ai
from oracle import levels as lv, pair as op


def _schur_fp32(sb):
    k = sb.k.astype(np.float32)
    ni = sb.n_i
    L = sla.cholesky(k[:ni, :ni], lower=True)
    X = sla.solve_triangular(L, k[:ni, ni:], lower=True)
    s = k[ni:, ni:] - X.T @ X
    assert s.dtype == np.float32
    return (0.5 * (s + s.T)).astype(np.float64)


def test_fp32_schur_and_pair_pencils_channels():
    prob = ai.config(1)
    lev = lv.level_one(prob)
    lev.schur()
    lev.coarse_basis()
    s64 = [sb.s.copy() for sb in lev.subs]
    s32 = [_schur_fp32(sb) for sb in lev.subs]
    for a, b in zip(s64, s32):
        assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()
        assert np.linalg.eigvalsh(b)[0] >= -1e-6 * np.abs(b).max()
    for s, t in [(1, 5), (2, 3), (3, 7)]:
        tops = []
        for ss in (s64, s32):
            for sb, m in zip(lev.subs, ss):
                sb.s = m
            lam = np.sort(op.literal(lev, s, t)[0])[::-1]
            tops.append(lam[0])
        for sb, m in zip(lev.subs, s64):
            sb.s = m
        assert abs(tops[1] - tops[0]) <= 3e-2 * tops[0], ((s, t), tops)
