"""Right-side triangular solve with emulated GEMMs, and the LU-based block tau_00: plain
restatements -- TEST INFRASTRUCTURE ONLY.

Sec. 3.2 of the paper: the LU-based inversion of the multiple scattering matrix spends its
time in ZGEMM and ZTRSM.  Readings used here and on the GPU:

* ``trsm_right_fp64``: the definition, X T = B for triangular T (upper or lower, with its
  diagonal or unit), solved in binary64 with a library solve on the triangle of T.
* ``trsm_right_emulated``: the blocked algorithm of the GPU path.  Block columns of width bt
  (16): for an upper T in the order 0, 1, ..., for a lower T from the last;
      X_j = (B_j - X_solved T[solved, j]) T_jj^-1,
  the update an emulated LU-mode GEMM (C - RN(A B)), the product by the block inverse an
  emulated GEMM, the block inverse binary64.
* ``lu_panel``: P D = L U by Gaussian elimination with partial pivoting (the row of largest
  |.|^2 in the column, the first on ties), L unit lower and U upper stored in one array.
* ``tau00_lu``: the block LU of ``kkr.tau00_block`` with every pivot block factored instead of
  inverted: P D = L U, M_RJ := M_RJ U^-1 L^-1 by the two solves above, the row interchanges
  applied to M_JR, M_RR -= M_RJ (P M_JR).  The Schur complement S_00 is the same as with the
  inverse, so tau_00 = S_00^-1 t_0 agrees with ``kkr.tau00_full`` to the emulation accuracy.
"""
from __future__ import annotations

import numpy as np

from . import kkr, ozaki


def _triangle(T, upper, unit):
    """The triangle of T that the solve reads (the other one zero, ones on the diagonal if unit)."""
    T = np.asarray(T, dtype=np.complex128)
    Tt = np.triu(T) if upper else np.tril(T)
    if unit:
        np.fill_diagonal(Tt, 1.0)
    return Tt


def trsm_right_fp64(T, B, upper=True, unit=False):
    """X with X T = B (binary64): X^T solves T^T X^T = B^T."""
    Tt = _triangle(T, upper, unit)
    return np.linalg.solve(Tt.T, np.asarray(B, dtype=np.complex128).T).T


def trsm_right_emulated(T, B, S, upper=True, unit=False, bt=16, gemm=None, gemm_lu=None):
    """The blocked emulated solve (module docstring); gemm(A, B, S) and gemm_lu(C, A, B, S)
    default to the Python restatement of the emulated ZGEMM."""
    gemm = gemm or (lambda A_, B_, S_: ozaki.ozaki_zgemm(A_, B_, S_))
    gemm_lu = gemm_lu or (lambda C_, A_, B_, S_: ozaki.ozaki_lu_update(C_, A_, B_, S_))
    T = np.asarray(T, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128)
    w = T.shape[0]
    nblk = (w + bt - 1) // bt
    for step in range(nblk):
        j = step if upper else nblk - 1 - step
        c0 = j * bt
        r = min(bt, w - c0)
        cols = slice(c0, c0 + r)
        solved = slice(0, c0) if upper else slice(c0 + r, w)
        if (c0 if upper else w - c0 - r) > 0:
            X[:, cols] = gemm_lu(X[:, cols], X[:, solved], T[solved, cols], S)
        Tjj_inv = np.linalg.inv(_triangle(T[cols, cols], upper, unit))
        X[:, cols] = gemm(X[:, cols], Tjj_inv, S)
    return X


def lu_panel(D):
    """(LU, perm): P D = L U with partial pivoting; LU holds L's multipliers below the
    diagonal and U on and above it; step k exchanged rows k and perm[k]."""
    A = np.array(D, dtype=np.complex128)
    w = A.shape[0]
    perm = np.zeros(w, dtype=np.int64)
    for k in range(w):
        piv = k + int(np.argmax(np.abs(A[k:, k]) ** 2))
        perm[k] = piv
        if A[piv, k] == 0:
            raise kkr.SingularError("singular pivot block")
        if piv != k:
            A[[k, piv], :] = A[[piv, k], :]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, perm


def tau00_lu(M, t0, nb, S, gemm=None, gemm_lu=None):
    """tau_00 by the LU variant of the block elimination (module docstring)."""
    gemm = gemm or (lambda A_, B_, S_: ozaki.ozaki_zgemm(A_, B_, S_))
    gemm_lu = gemm_lu or (lambda C_, A_, B_, S_: ozaki.ozaki_lu_update(C_, A_, B_, S_))
    b = t0.shape[0]
    A = np.array(M, dtype=np.complex128)
    n = A.shape[0]
    q = n
    while q > b:
        p = max(q - nb, b)
        LU, perm = lu_panel(A[p:q, p:q])
        A[p:q, p:q] = LU
        for k, pk in enumerate(perm):                   # the interchanges on M_JR, in order
            if pk != k:
                A[[p + k, p + pk], :p] = A[[p + pk, p + k], :p]
        Y = trsm_right_emulated(LU, A[:p, p:q], S, upper=True, unit=False, gemm=gemm, gemm_lu=gemm_lu)
        A[:p, p:q] = trsm_right_emulated(LU, Y, S, upper=False, unit=True, gemm=gemm, gemm_lu=gemm_lu)
        A[:p, :p] = gemm_lu(A[:p, :p], A[:p, p:q], A[p:q, :p], S)
        q = p
    return kkr.gepp_inverse(A[:b, :b]) @ t0
