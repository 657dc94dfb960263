"""Ozaki-II (CRT) emulated ZGEMM: plain restatement -- TEST INFRASTRUCTURE ONLY.

The paper describes Ozaki-II (Sec. 2.2) as converting the floating-point matrices to integers,
multiplying them modulo several small pairwise-coprime moduli and reconstructing the product
with the Chinese Remainder Theorem; its precision knob is the number of moduli (10..18 in the
experiments of Sec. 3.2 and Sec. 4).  Readings used here and on the GPU:

* moduli: the N largest pairwise-coprime integers <= 256 (greedy from 256 down), so that a
  symmetric residue r in [-m/2, m/2] is an exact fp16 value and a product of two is <= 2^14;
* integer images: e_i = frexp exponent of the row maximum of op(A) over |Re|, |Im| (f_j for the
  columns of op(B)), X = trunc(x 2^(beta - e)) with beta the largest integer such that
  2k 4^beta < P / 2 (P the product of the moduli): every exact real entry of the stacked 4M
  product [Re A | Im A] [[Re B, Im B], [-Im B, Re B]] is then below P / 2 in magnitude;
* per modulus m_l: the stacked product of the symmetric residues, exact in integers;
* CRT: the unique C' with |C'| < P / 2 congruent to every product, C' = sum_l (C_l mod m_l)
  c_l mod P with c_l = (P / m_l) ((P / m_l)^-1 mod m_l), lifted to the symmetric range;
* result: C' 2^(e_i + f_j - 2 beta) rounded once to binary64 (round to nearest even).
"""
from __future__ import annotations

import math

import numpy as np

from .ozaki import round_scaled, row_exponents

MAX_MODULUS = 256


def moduli(N):
    """The N largest pairwise-coprime integers <= 256 (greedy from 256 down)."""
    out = []
    c = MAX_MODULUS
    while len(out) < N and c > 1:
        if all(math.gcd(c, m) == 1 for m in out):
            out.append(c)
        c -= 1
    if len(out) < N:
        raise ValueError("not enough moduli")
    return out


def crt_constants(ms):
    P = math.prod(ms)
    cs = []
    for m in ms:
        Mi = P // m
        cs.append(Mi * pow(Mi, -1, m))
    return P, cs


def beta_bits(k, P):
    """Largest beta with 2k 4^beta < P / 2 (so |C'| < P / 2 for |A'|, |B'| < 2^beta)."""
    beta = 0
    while 2 * k * (1 << (2 * (beta + 1))) * 2 < P:
        beta += 1
    return beta


def integer_image(x, e, beta):
    """trunc(x 2^(beta - e)) as a Python int (exact: x is a binary64 value)."""
    if x == 0.0:
        return 0
    n, d = float(x).as_integer_ratio()          # x = n / d, d a power of two
    sh = beta - e
    if sh >= 0:
        num, den = n << sh, d
    else:
        num, den = n, d << (-sh)
    q = abs(num) // den
    return q if num >= 0 else -q


def sym_residue(X, m):
    r = X % m                                  # Python: in [0, m)
    return r - m if 2 * r > m else r


def residues_left(A, beta, ms):
    """Row exponents of op(A) (m x k) and, per modulus, the m x 2k stacked residues
    [Re | Im] as int64 arrays."""
    A = np.asarray(A, dtype=np.complex128)
    m, k = A.shape
    e = row_exponents(A)
    R = np.zeros((len(ms), m, 2 * k), dtype=np.int64)
    for i in range(m):
        for l_ in range(k):
            xr = integer_image(A[i, l_].real, int(e[i]), beta)
            xi = integer_image(A[i, l_].imag, int(e[i]), beta)
            for t, mod in enumerate(ms):
                R[t, i, l_] = sym_residue(xr, mod)
                R[t, i, k + l_] = sym_residue(xi, mod)
    return e, R


def residues_right(B, beta, ms):
    """Column exponents of op(B) (k x n) and, per modulus, the 2n x 2k stacked residues: row
    2j = [Re B_j ; -Im B_j], row 2j + 1 = [Im B_j ; Re B_j] (the negation residue-wise)."""
    B = np.asarray(B, dtype=np.complex128)
    k, n = B.shape
    f = row_exponents(B.T)
    R = np.zeros((len(ms), 2 * n, 2 * k), dtype=np.int64)
    for j in range(n):
        for l_ in range(k):
            xr = integer_image(B[l_, j].real, int(f[j]), beta)
            xi = integer_image(B[l_, j].imag, int(f[j]), beta)
            for t, mod in enumerate(ms):
                rr, ri = sym_residue(xr, mod), sym_residue(xi, mod)
                R[t, 2 * j, l_], R[t, 2 * j, k + l_] = rr, -ri
                R[t, 2 * j + 1, l_], R[t, 2 * j + 1, k + l_] = ri, rr
    return f, R


def crt(res, ms, P, cs):
    """The integer C' with |C'| < P / 2 and C' = res[l] mod ms[l] for every l."""
    s = sum((int(r) % m) * c for r, m, c in zip(res, ms, cs)) % P
    return s - P if 2 * s > P else s


def ozaki2_zgemm(A, B, N):
    """op(A) op(B) by Ozaki-II with N moduli (mathematical orientation, complex128)."""
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    m, k = A.shape
    n = B.shape[1]
    ms = moduli(N)
    P, cs = crt_constants(ms)
    beta = beta_bits(k, P)
    e, RA = residues_left(A, beta, ms)
    f, RB = residues_right(B, beta, ms)
    # exact integer products per modulus (|entries| <= 2k 2^14 < 2^53: float64 matmul is exact)
    prods = [np.rint(RA[t].astype(np.float64) @ RB[t].astype(np.float64).T).astype(np.int64)
             for t in range(len(ms))]
    C = np.zeros((m, n), dtype=np.complex128)
    for i in range(m):
        for j in range(n):
            re = crt([p[i, 2 * j] for p in prods], ms, P, cs)
            im = crt([p[i, 2 * j + 1] for p in prods], ms, P, cs)
            E = int(e[i]) + int(f[j]) - 2 * beta
            C[i, j] = complex(round_scaled(re, E), round_scaled(im, E))
    return C


def exact_truncated_product(A, B, N):
    """The exact product of the integer images (what the CRT must recover), as Python ints,
    with the scale exponents: (C' re, C' im, e, f, beta)."""
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    m, k = A.shape
    n = B.shape[1]
    P, _ = crt_constants(moduli(N))
    beta = beta_bits(k, P)
    e = row_exponents(A)
    f = row_exponents(B.T)
    Ai = [[(integer_image(A[i, l].real, int(e[i]), beta), integer_image(A[i, l].imag, int(e[i]), beta))
           for l in range(k)] for i in range(m)]
    Bi = [[(integer_image(B[l, j].real, int(f[j]), beta), integer_image(B[l, j].imag, int(f[j]), beta))
           for j in range(n)] for l in range(k)]
    re = [[sum(Ai[i][l][0] * Bi[l][j][0] - Ai[i][l][1] * Bi[l][j][1] for l in range(k)) for j in range(n)]
          for i in range(m)]
    im = [[sum(Ai[i][l][0] * Bi[l][j][1] + Ai[i][l][1] * Bi[l][j][0] for l in range(k)) for j in range(n)]
          for i in range(m)]
    return re, im, e, f, beta
