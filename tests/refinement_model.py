"""A reference model of the solver's projection by one refinement step, for
the BF16-storage parity test (test infrastructure, FP64, numpy/scipy).

The solver computes each iteration's projection (Algorithm 2 step 18 in its
one-solve form, w = M^{-1}(b_tilde - A_hat p), M = A_hat A_hat') as one step
of iterative refinement from the previous w: the residual
r0 = b_tilde - A_hat (p + q), q = A_hat' w, in FP64 with the FP64 values of A,
and a correction dw = M_c^{-1} r0 with the matrix the correction solve reads.
With M_c = M this is the exact projection, i.e. Algorithm 2 itself; with A
stored in BF16, M_c = A_bf O^2 A_bf' with A_bf = A rounded to BF16 values.
This module runs that iteration in FP64 with exact (dense Cholesky)
corrections, so that the only difference from the GPU run with BF16 storage
is the FP32 arithmetic of its correction CG.  Pinned against
oracle.alg.algorithm2 with M_c = M (tests/test_oracle_alg.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import alg, cones as C


def bf16_round(v):
    """Values rounded to the nearest BF16 value (FP32 first), ties to even,
    chosen between the two neighbouring BF16 patterns by distance."""
    f = np.asarray(v, dtype=np.float64).astype(np.float32)
    lo = (f.view(np.uint32) >> 16).astype(np.uint32)
    hi = lo + 1

    def val(t):
        return (np.asarray(t, np.uint32) << 16).view(np.float32).astype(np.float64)

    d_lo = np.abs(val(lo) - f.astype(np.float64))
    d_hi = np.abs(val(hi) - f.astype(np.float64))
    pick = np.where(d_lo < d_hi, lo, np.where(d_hi < d_lo, hi, np.where(lo % 2 == 0, lo, hi)))
    return val(pick)


def refined_iterates(A, b, c, n_orth, soc_dims=(), mu=1.0, t=9.2, L=alg.LP_SCHEDULE, iters=50,
                     correction_values=None):
    """x after each of the first `iters` iterations of Algorithm 2 with the
    projection applied as one refinement step per iteration (see above).
    correction_values: the stored values the correction solve reads (same
    pattern as A), None for A's own."""
    A = sp.csr_matrix(A, dtype=np.float64)
    m, n = A.shape
    Ac = A.copy()
    if correction_values is not None:
        Ac.data = np.asarray(correction_values, dtype=np.float64).copy()
    e = C.cone_identity(n, n_orth, soc_dims)
    x, z = e.copy(), e.copy()
    w = np.zeros(m)
    out = []
    O = chat = btil = q = factor = s = None
    for l in range(1, iters + 1):
        if l == 1 or l in L:
            O, _ = alg.conditioning_matrix(x, z, n_orth, soc_dims, t)
            Ah = A @ sp.diags(O)
            chat = O * c
            btil = b + mu * (Ah @ chat)
            s = x / O - mu * O * z
            Mc = (Ac @ sp.diags(O * O) @ Ac.T).toarray()
            factor = sla.cho_factor(Mc)
            q = Ah.T @ w
        Ah = A @ sp.diags(O)
        p = C.abs_K(s, n_orth, soc_dims)
        r0 = btil - Ah @ (p + q)
        w = w + sla.cho_solve(factor, r0)
        q = Ah.T @ w
        s = 0.5 * (s + p) - mu * chat + q
        x = O * (p + s) / 2.0
        z = (p - s) / (2.0 * mu * O)
        out.append(x.copy())
    return out
