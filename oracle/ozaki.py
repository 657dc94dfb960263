"""Ozaki-I emulated complex GEMM, written out step by step -- TEST INFRASTRUCTURE ONLY.

The paper (Sec. 2.2, "GEMM Emulation on Integer Matrix Multiplication Unit") states the
scheme in words: split the high-precision matrices into low-precision slices by their
significant bits with exponent alignment, multiply slice pairs in low precision, and
accumulate the pair products in higher precision.  Its precision knob is the number of
mantissa bits (31/39/47/55/63, Sec. 3.2 and Sec. 4), read here as B = 8S - 1 bits held in
S int8-sized slices.  Everything below is the reading of those sentences used by this
project; the choices the paper leaves open are listed in the module-level constants and
in the docstrings:

1. Exponent alignment.  e_i = frexp-exponent of max_l max(|Re a_il|, |Im a_il|) for each
   row i of A, f_j likewise for each column j of B, so that the scaled row lies in
   (-1, 1).  A zero row has exponent 0.
2. Integer image.  X = trunc(x * 2^(B - e)) (toward zero) with B = 8S - 1, |X| < 2^B.
3. Slices.  Balanced base-256 digits, least significant first:
   d_S = ((X + 128) mod 256) - 128, X <- (X - d_S) / 256, ..., d_1 = what remains;
   so X = sum_t d_t 256^(S-t), d_t in [-128, 127] for t >= 2, d_1 in [-128, 128].
4. Complex operands are stacked (4M form): A_s = [Re A_s | Im A_s] (m x 2k); the right
   operand has, for output column j, row 2j = [Re B_s(:,j) ; -Im B_s(:,j)] and row
   2j+1 = [Im B_s(:,j) ; Re B_s(:,j)], the -Im block being the digit-wise negation.
   Column 2j of the stacked product is Re c_ij, column 2j+1 is Im c_ij.
5. Pairs.  Triangular set {(s, t): s + t <= S + 1} (default) or the full S x S set.
   Group sums G_g = sum_{s+t=g} A_s B_t^T are exact integers.
6. Reconstruction.  Z_ij = 2^(e_i + f_j - 2B) * sum_g G_g 256^(2S - g), rounded ONCE to
   binary64 (round to nearest, ties to even).
7. Epilogues.  "store": C = Z.  "lu": C_out = C_in - Z in binary64 (one more rounding).
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

DIGIT_BITS = 8          # bits per slice (int8-sized digits)


def bits_for(S: int) -> int:
    """Total fixed-point bits B = 8S - 1 (31, 39, 47, 55, 63 for S = 4..8)."""
    return DIGIT_BITS * S - 1


# ----------------------------------------------------------------------------- step 1

def row_exponents(X: np.ndarray) -> np.ndarray:
    """frexp exponents of the per-row max over |Re| and |Im| (Sec. 2.2 exponent alignment).

    X is complex (R x K).  Returns int64 e (R,), e = 0 for an all-zero row.
    Raises ValueError on NaN or Inf (the product path reports a status code instead).
    """
    X = np.asarray(X)
    if not np.all(np.isfinite(X)):
        raise ValueError("non-finite input")
    mu = np.maximum(np.abs(X.real), np.abs(X.imag)).max(axis=1) if X.shape[1] else np.zeros(X.shape[0])
    _, e = np.frexp(mu)
    return e.astype(np.int64)


# ----------------------------------------------------------------------------- steps 2-3

def integer_image(x: np.ndarray, e: np.ndarray, S: int) -> np.ndarray:
    """X = trunc(x * 2^(B - e_row)) as exact Python ints (object array, same shape as x)."""
    B = bits_for(S)
    y = np.trunc(np.ldexp(np.asarray(x, dtype=np.float64), (B - np.asarray(e))[:, None]))
    # y holds exact integers (a power-of-two scaling is exact; trunc is exact)
    out = np.empty(y.shape, dtype=object)
    flat = out.reshape(-1)
    for i, v in enumerate(y.reshape(-1)):
        flat[i] = int(v)
    return out


def balanced_digits(Xint: np.ndarray, S: int) -> np.ndarray:
    """Balanced base-256 digits, most significant first: shape (S,) + Xint.shape, int64."""
    D = np.zeros((S,) + Xint.shape, dtype=np.int64)
    flatX = Xint.reshape(-1)
    flatD = D.reshape(S, -1)
    for i, X in enumerate(flatX):
        r = int(X)
        for t in range(S - 1, 0, -1):        # d_S ... d_2
            d = ((r + 128) % 256) - 128
            flatD[t, i] = d
            r = (r - d) // 256
        flatD[0, i] = r                      # d_1
    return D


def split_left(A: np.ndarray, S: int):
    """Exponents and stacked slices of the left operand: e (m,), D (S, m, 2k) int64."""
    e = row_exponents(A)
    Dr = balanced_digits(integer_image(A.real, e, S), S)
    Di = balanced_digits(integer_image(A.imag, e, S), S)
    return e, np.concatenate([Dr, Di], axis=2)


def split_right(B: np.ndarray, S: int):
    """Exponents and stacked slices of the right operand: f (n,), D (S, 2n, 2k) int64.

    Row 2j = [Re | -Im] digits of column j, row 2j+1 = [Im | Re]."""
    Bt = np.ascontiguousarray(B.T)                     # n x k, row j = column j of B
    f = row_exponents(Bt)
    Dr = balanced_digits(integer_image(Bt.real, f, S), S)
    Di = balanced_digits(integer_image(Bt.imag, f, S), S)
    S_, n, k = Dr.shape
    D = np.zeros((S, 2 * n, 2 * k), dtype=np.int64)
    D[:, 0::2, :k] = Dr
    D[:, 0::2, k:] = -Di
    D[:, 1::2, :k] = Di
    D[:, 1::2, k:] = Dr
    return f, D


# ----------------------------------------------------------------------------- step 5

def pair_set(S: int, mode: str = "tri"):
    """Slice pairs (s, t), 1-based.  'tri': s + t <= S + 1; 'full': all S x S."""
    if mode == "tri":
        return [(s, t) for s in range(1, S + 1) for t in range(1, S + 2 - s)]
    if mode == "full":
        return [(s, t) for s in range(1, S + 1) for t in range(1, S + 1)]
    raise ValueError(mode)


def group_sums(DA: np.ndarray, DB: np.ndarray, pairs) -> dict:
    """Exact G_g = sum_{(s,t) in pairs, s+t=g} DA[s] DB[t]^T as int64 arrays.

    The products are formed with a float64 matmul, which is exact here: every term is an
    integer of magnitude <= 2^14 and every partial sum stays below 2^53, so no rounding
    can occur in any summation order."""
    Kp = DA.shape[2]
    assert Kp * (2 ** 14) * len(pairs) < 2 ** 53
    G = {}
    for (s, t) in pairs:
        P = DA[s - 1].astype(np.float64) @ DB[t - 1].astype(np.float64).T
        g = s + t
        G[g] = G.get(g, 0) + P
    return {g: v.astype(np.int64) for g, v in G.items()}


# ----------------------------------------------------------------------------- step 6

def round_scaled(T: int, E: int) -> float:
    """RN-even of the exact value T * 2^E as a binary64 (single rounding).

    Python's int / int true division is correctly rounded, which makes this the
    definition written out (Fraction -> float)."""
    if T == 0:
        return 0.0
    if E >= 0:
        try:
            return float(T * (1 << E))
        except OverflowError:
            return math.copysign(math.inf, T)
    try:
        return T / (1 << (-E))
    except OverflowError:
        return math.copysign(math.inf, T)


def reconstruct(G: dict, e: np.ndarray, f: np.ndarray, S: int) -> np.ndarray:
    """Complex (m x n) result from the group sums (step 6), one rounding per real part."""
    B = bits_for(S)
    gs = sorted(G)
    gmax = gs[-1]
    m, n2 = G[gs[0]].shape
    # exact integer T = sum_g G_g * 256^(gmax - g); value = T * 2^(e+f-2B+8(2S-gmax))
    T = np.zeros((m, n2), dtype=object)
    for g in gs:
        T = T + G[g].astype(object) * (256 ** (gmax - g))
    out = np.empty((m, n2), dtype=np.float64)
    base = -2 * B + 8 * (2 * S - gmax)
    for i in range(m):
        for j in range(n2):
            out[i, j] = round_scaled(int(T[i, j]), int(e[i]) + int(f[j // 2]) + base)
    return out[:, 0::2] + 1j * out[:, 1::2]


# ----------------------------------------------------------------------------- whole GEMM

def ozaki_zgemm(A: np.ndarray, B: np.ndarray, S: int, mode: str = "tri") -> np.ndarray:
    """Emulated C = A B (store epilogue), steps 1-6."""
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    if m == 0 or n == 0:
        return np.zeros((m, n), dtype=np.complex128)
    if k == 0:
        return np.zeros((m, n), dtype=np.complex128)
    e, DA = split_left(A, S)
    f, DB = split_right(B, S)
    G = group_sums(DA, DB, pair_set(S, mode))
    return reconstruct(G, e, f, S)


def ozaki_lu_update(C: np.ndarray, A: np.ndarray, B: np.ndarray, S: int, mode: str = "tri") -> np.ndarray:
    """LU epilogue: C_out = C_in - Z, Z the emulated product rounded once (step 7)."""
    Z = ozaki_zgemm(A, B, S, mode)
    return (C.real - Z.real) + 1j * (C.imag - Z.imag)


def truncated_operands(A: np.ndarray, B: np.ndarray, S: int):
    """The exact rational values the slices represent: x_hat = X * 2^(e - B).

    Used by the pins: with the full pair set the emulation must equal the exact product
    of these truncated operands rounded once."""
    Bits = bits_for(S)
    e = row_exponents(A)
    f = row_exponents(np.ascontiguousarray(B.T))
    Ar = integer_image(A.real, e, S)
    Ai = integer_image(A.imag, e, S)
    Bt = np.ascontiguousarray(B.T)
    Br = integer_image(Bt.real, f, S)
    Bi = integer_image(Bt.imag, f, S)

    def q(X, ex):
        return [[Fraction(int(X[i, l])) * Fraction(2) ** (int(ex[i]) - Bits) for l in range(X.shape[1])]
                for i in range(X.shape[0])]
    return q(Ar, e), q(Ai, e), q(Br, f), q(Bi, f)


def exact_product_rounded(Ar, Ai, Br, Bi) -> np.ndarray:
    """RN(sum_l a_il b_lj) of Fraction operands (Ar[i][l], Br[j][l] layout)."""
    m, k, n = len(Ar), len(Ar[0]) if Ar else 0, len(Br)
    out = np.zeros((m, n), dtype=np.complex128)
    for i in range(m):
        for j in range(n):
            re = sum((Ar[i][l] * Br[j][l] - Ai[i][l] * Bi[j][l] for l in range(k)), Fraction(0))
            im = sum((Ar[i][l] * Bi[j][l] + Ai[i][l] * Br[j][l] for l in range(k)), Fraction(0))
            out[i, j] = complex(float(re), float(im))
    return out


def zgemm_exact(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Exact complex product of binary64 inputs, rounded once per part (tiny inputs)."""
    m, k = A.shape
    n = B.shape[1]
    out = np.zeros((m, n), dtype=np.complex128)
    for i in range(m):
        for j in range(n):
            re = Fraction(0)
            im = Fraction(0)
            for l in range(k):
                ar, ai = Fraction(A[i, l].real), Fraction(A[i, l].imag)
                br, bi = Fraction(B[l, j].real), Fraction(B[l, j].imag)
                re += ar * br - ai * bi
                im += ar * bi + ai * br
            out[i, j] = complex(float(re), float(im))
    return out


def ozaki_error_bound(A: np.ndarray, B: np.ndarray, S: int) -> np.ndarray:
    """Elementwise bound on |Z - A B| for the triangular pair set (real and imag parts).

    Two error sources: (i) truncating each operand to B bits: |x - x_hat| < 2^(e - B);
    (ii) dropping pairs with s + t > S + 1, whose digit products are bounded by
    128^2 * 256^(2S - g) * 2^(e + f - 2B) per term; plus the final rounding (half an ulp).
    Returns a real (m x n) array bounding both parts."""
    Bits = bits_for(S)
    m, k = A.shape
    n = B.shape[1]
    e = row_exponents(A).astype(np.float64)
    f = row_exponents(np.ascontiguousarray(B.T)).astype(np.float64)
    absA = np.maximum(np.abs(A.real), np.abs(A.imag))
    absB = np.maximum(np.abs(B.real), np.abs(B.imag))
    ea = np.ldexp(1.0, (e - Bits).astype(np.int64))         # per-row truncation unit
    fb = np.ldexp(1.0, (f - Bits).astype(np.int64))
    # (i): per term |x y - x^ y^| <= |x| dy + |y| dx + dx dy, 2k terms per part
    trunc = 2.0 * (absA.sum(axis=1)[:, None] * fb[None, :]
                   + ea[:, None] * absB.sum(axis=0)[None, :]
                   + k * np.outer(ea, fb))
    # (ii): dropped groups g = S+2 .. 2S with (2S + 1 - g) pairs each
    drop = 0.0
    for g in range(S + 2, 2 * S + 1):
        drop += (2 * S + 1 - g) * (128.0 ** 2) * 256.0 ** (2 * S - g)
    dropped = 2 * k * drop * np.ldexp(1.0, (e[:, None] + f[None, :] - 2 * Bits).astype(np.int64))
    ref = np.abs(A) @ np.abs(B) + trunc + dropped
    return trunc + dropped + np.spacing(ref)
