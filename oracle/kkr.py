"""KKR tau_00 oracle -- TEST INFRASTRUCTURE ONLY.

Sec. 3.2 of the paper: the dominant cost of the LSMS method is the LU-based inversion of
the multiple scattering matrix at each point of the complex energy contour, done with
ZGEMM and ZTRSM.  The quantity the inversion yields for an atom is the central block of
the scattering-path matrix; with the standard KKR convention (the paper does not write
the formula) it is

    M = I - t G,   tau = M^-1 t,   tau_00 = [M^-1]_00 t_0,

with t block diagonal (one b x b block per LIZ site, site 0 the centre) and G the
structure-constant matrix with zero diagonal blocks.

Two oracles:

* ``tau00_full`` inverts M by textbook Gauss-Jordan elimination with partial pivoting in
  binary64 and takes the (0, 0) block times t_0.
* ``tau00_block`` is the block-LU algorithm of the GPU path written out.  The centre
  block (site 0, the leading b x b block) is eliminated last: panels J of width nb are
  eliminated from the trailing end of the matrix towards the front, so that what remains
  after each step is the leading r x r block R = [0, r).  Each step computes
      L_RJ = M_RJ D^-1,   M_RR <- M_RR - L_RJ M_JR,   D = M_JJ,
  with no pivoting across panels (partial pivoting only inside the inverse of each pivot
  block).  Every panel product and every Schur update is an emulated ZGEMM (or a
  binary64 matmul when S is None), and tau_00 = S_00^-1 t_0 with S_00 the Schur
  complement left in the centre block.
"""
from __future__ import annotations

import numpy as np

from . import ozaki


class SingularError(ArithmeticError):
    pass


def gepp_inverse(M: np.ndarray) -> np.ndarray:
    """Gauss-Jordan inverse with partial pivoting (largest modulus in the column)."""
    M = np.asarray(M, dtype=np.complex128)
    n = M.shape[0]
    A = np.concatenate([M.copy(), np.eye(n, dtype=np.complex128)], axis=1)
    for p in range(n):
        piv = p + int(np.argmax(np.abs(A[p:, p])))
        if A[piv, p] == 0:
            raise SingularError(f"zero pivot in column {p}")
        if piv != p:
            A[[p, piv]] = A[[piv, p]]
        A[p] = A[p] / A[p, p]
        col = A[:, p].copy()
        col[p] = 0
        A -= np.outer(col, A[p])
    return A[:, n:]


def tau00_full(M: np.ndarray, t0: np.ndarray) -> np.ndarray:
    b = t0.shape[0]
    return gepp_inverse(M)[:b, :b] @ t0


def tau00_lapack(M: np.ndarray, t0: np.ndarray) -> np.ndarray:
    """The same tau_00 = [M^-1]_00 t_0 from a library LU solve (LAPACK through numpy) of
    M X = E with E the first b columns of the identity: X = the first b columns of M^-1, at a
    third of the cost of the full inverse -- the reference at the largest sizes."""
    b = t0.shape[0]
    E = np.zeros((M.shape[0], b), dtype=np.complex128)
    E[:b] = np.eye(b)
    return np.linalg.solve(np.asarray(M, dtype=np.complex128), E)[:b] @ t0


def tau00_block(M: np.ndarray, t0: np.ndarray, nb: int, S=None, mode: str = "tri", leaf=None) -> np.ndarray:
    """Block LU eliminating from the trailing end, the centre block last (module docstring).

    leaf=None: each panel J = [p, q) is one pivot block (D = M_JJ inverted whole).
    leaf=w:    the panel is factored leaf by leaf (w x w pivot blocks, from its last leaf; the
               front leaf narrower when w does not divide the panel width): L column of the
               leaf, then its rank-w update of the rows and columns of [0, a) outside
               [0, p) x [0, p); the update of [0, p) x [0, p) by the whole panel is applied
               once afterwards.  Same block LU, fewer and deeper trailing updates."""
    b = t0.shape[0]
    A = np.array(M, dtype=np.complex128)
    n = A.shape[0]

    def mul(X, Y):
        return X @ Y if S is None else ozaki.ozaki_zgemm(X, Y, S, mode)

    def sub_mul(C, X, Y):
        return C - X @ Y if S is None else ozaki.ozaki_lu_update(C, X, Y, S, mode)

    q = n                                   # panel J = [p, q), remainder R = [0, p)
    while q > b:
        p = max(q - nb, b)
        wl = (q - p) if leaf is None else leaf
        hi = q
        while hi > p:                        # leaves [a, hi), last one first
            a = max(hi - wl, p)
            w = hi - a
            Dinv = gepp_inverse(A[a:a + w, a:a + w])
            A[:a, a:a + w] = mul(A[:a, a:a + w], Dinv)                       # L column
            if a > p:
                box = A[:p, :p].copy()
                A[:a, :a] = sub_mul(A[:a, :a], A[:a, a:a + w], A[a:a + w, :a])  # outside the box
                A[:p, :p] = box
            hi = a
        A[:p, :p] = sub_mul(A[:p, :p], A[:p, p:q], A[p:q, :p])                 # deferred update
        q = p
    return gepp_inverse(A[:b, :b]) @ t0


def kkr_build(t: np.ndarray, G: np.ndarray) -> np.ndarray:
    """M = I - blockdiag(t) G, binary64."""
    L, b, _ = t.shape
    n = L * b
    M = -np.einsum("lij,ljn->lin", t, G.reshape(L, b, n)).reshape(n, n)
    M[np.arange(n), np.arange(n)] += 1.0
    return M


def rel_err(X: np.ndarray, Y: np.ndarray) -> float:
    """Relative Frobenius error ||X - Y||_F / ||Y||_F."""
    d = np.linalg.norm(Y)
    return float(np.linalg.norm(X - Y) / d) if d else float(np.linalg.norm(X))


def contour_trace(taus, w):
    """Tr tau_00(z_i) for every energy point and the quadrature sum_i w_i Tr tau_00(z_i) (the
    site-diagonal Green's-function trace integrated along the contour, whose error per
    precision mode the paper reports, Sec. 4)."""
    tr = np.array([np.trace(np.asarray(t)) for t in taus], dtype=np.complex128)
    return tr, complex(np.sum(np.asarray(w, dtype=np.complex128) * tr))
