"""Slice-count selector: plain float64 restatement -- TEST INFRASTRUCTURE ONLY.

The paper finds that the emulation's accuracy depends both on the precision (the number of
mantissa bits, i.e. of slices) and on the operator, handled by tuning the precision
(Abstract; Sec. 4, error falling mode by mode), and argues for adaptive precision (Sec. 5),
but gives no rule for choosing it.  The selector built here picks, per GEMM, the smallest
slice count S in 3..10 whose predicted relative error meets a tolerance, and verifies the
result a posteriori:

* 16 features of the operands (``features``), computed from per-row / per-column
  statistics and a probe product z = op(A) (op(B) X) with random probe vectors X;
* a multilayer perceptron 16 -> 64 -> 64 -> 8 with ReLU hidden layers whose outputs are the
  predicted log10 relative Frobenius errors for S = 3..10 (``forward``);
* trained by mean-squared error on measured errors with Adam (``loss``, ``backward``,
  ``adam_step``; Kingma and Ba, "Adam: a method for stochastic optimization", ICLR 2015);
* selection (``choose``): the smallest S with prediction <= log10(tol) - margin, else 10;
* residual check (``residual_estimate``): for probe vectors x with independent zero-mean,
  unit-variance entries E||E x||^2 = ||E||_F^2, so ||D X - z|| / ||z|| estimates the
  relative Frobenius error of a computed product D without the exact product.

Parameter layout (float32 on the device, float64 here), one flat vector of 5768 values:
W1[64][16], b1[64], W2[64][64], b2[64], W3[8][64], b3[8] (row-major, W[out][in]).
"""
from __future__ import annotations

import math

import numpy as np

NF, NH, NO = 16, 64, 8
SMIN, SMAX = 3, 10
OFF_W1 = 0
OFF_B1 = OFF_W1 + NH * NF
OFF_W2 = OFF_B1 + NH
OFF_B2 = OFF_W2 + NH * NH
OFF_W3 = OFF_B2 + NH
OFF_B3 = OFF_W3 + NO * NH
NPARAMS = OFF_B3 + NO
PROBES = 4
PROBE_SCALE = math.sqrt(6.0)          # (U[0,1) - 1/2) * sqrt(6): variance 1/2 per real part


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[OFF_W1:OFF_B1].reshape(NH, NF), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(NH, NH),
            p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3].reshape(NO, NH), p[OFF_B3:NPARAMS])


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3]).astype(np.float64)


# ----------------------------------------------------------------------------- the network

def forward(p, X):
    """Y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for every row x of X (N x 16).
    Returns Y and the pre-activations (Z1, Z2) the backward pass needs."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ W3.T + b3
    return Y, Z1, Z2


def loss(p, X, T):
    """Mean squared error over all N x 8 outputs."""
    Y, _, _ = forward(p, X)
    return float(np.mean((Y - np.asarray(T, dtype=np.float64)) ** 2))


def backward(p, X, T):
    """Gradient of ``loss`` with respect to the flat parameter vector (chain rule by hand;
    the ReLU derivative at 0 is taken as 0)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    Y, Z1, Z2 = forward(p, X)
    N = X.shape[0]
    dY = 2.0 * (Y - np.asarray(T, dtype=np.float64)) / (N * NO)
    H2 = np.maximum(Z2, 0.0)
    H1 = np.maximum(Z1, 0.0)
    gW3 = dY.T @ H2
    gb3 = dY.sum(0)
    dZ2 = (dY @ W3) * (Z2 > 0)
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2) * (Z1 > 0)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(0)
    return pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1, bias-corrected moments).  Returns p, m, v."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def choose(pred, tol, margin=0.0):
    """Smallest S in SMIN..SMAX whose predicted log10 error is <= log10(tol) - margin; SMAX
    if none is."""
    lim = math.log10(tol) - margin
    for o in range(NO):
        if pred[o] <= lim:
            return SMIN + o
    return SMAX


# ----------------------------------------------------------------------------- features

def probe_vectors(n, seed):
    """The PROBES probe vectors (n x PROBES complex): real part of column p from stream 2p,
    imaginary part from stream 2p + 1 of the counter-based generator, (U - 1/2) sqrt(6)."""
    import synth
    X = np.zeros((n, PROBES), dtype=np.complex128)
    idx = np.arange(n, dtype=np.uint64)
    for p in range(PROBES):
        re = (synth.uniform(seed, 2 * p, idx) - 0.5) * PROBE_SCALE
        im = (synth.uniform(seed, 2 * p + 1, idx) - 0.5) * PROBE_SCALE
        X[:, p] = re + 1j * im
    return X


def _vector_stats(V):
    """Per row of V (rows x len complex): r = max of |Re|, |Im|; e = frexp exponent of r
    (0 for a zero row); sh = sum |v / 2^e|^2 (the row's sum of squares scaled by 4^-e, so
    that it neither overflows nor underflows); zero count."""
    r = np.maximum(np.abs(V.real), np.abs(V.imag)).max(axis=1) if V.shape[1] else np.zeros(V.shape[0])
    e = np.array([math.frexp(float(x))[1] if x > 0 else 0 for x in r], dtype=np.int64)
    Vs = np.ldexp(V.real, -e[:, None]) + 1j * np.ldexp(V.imag, -e[:, None])
    sh = (np.abs(Vs) ** 2).sum(axis=1)
    z = (V == 0).sum(axis=1)
    return r, e, sh, z


def _to_int(V):
    """Exact integer image of a complex binary64 array: (Re, Im, e) with V = (Re + i Im) 2^e,
    Re and Im object arrays of Python ints."""
    V = np.asarray(V, dtype=np.complex128)
    parts = [x.as_integer_ratio() for x in np.concatenate([V.real.ravel(), V.imag.ravel()])]
    den = max(d for _, d in parts) if parts else 1
    ints = np.array([n * (den // d) for n, d in parts], dtype=object)
    half = V.size
    e = -(den.bit_length() - 1)
    return ints[:half].reshape(V.shape), ints[half:].reshape(V.shape), e


def _int_mul(a, b):
    """Exact product of two integer images (object-array matmul of Python ints)."""
    ar, ai, ea = a
    br, bi, eb = b
    return ar @ br - ai @ bi, ar @ bi + ai @ br, ea + eb


def _int_sq(re, im):
    return int(np.sum(re * re + im * im)) if re.size else 0


def _scaled(V, s):
    """V * 2^s, exactly (ldexp of both parts)."""
    return np.ldexp(V.real, s) + 1j * np.ldexp(V.imag, s)


def _log2sum(w, e):
    """log2 of sum_i w_i 4^e_i (w_i > 0) without overflow; -inf for an empty sum."""
    if len(e) == 0:
        return -math.inf
    em = int(np.max(e))
    return 2.0 * em + math.log2(float(np.sum(np.ldexp(np.asarray(w, dtype=np.float64),
                                                      2 * (np.asarray(e, dtype=np.int64) - em)))))


def features(Aop, Bop, X, exact=False):
    """The 16 selector features of the product Aop @ Bop (m x k times k x n, complex), with
    probe vectors X (n x PROBES).  Returns (f, zs, E) where zs = (2^-EA Aop)((2^-EB Bop) X)
    is the scaled probe product the residual check reuses and E = EA + EB.  With exact=True
    the probe product is formed in exact integer arithmetic and returned as its integer
    image (see _to_int); otherwise by binary64 matrix products.

    Per row i of Aop: r_i = max(|Re|, |Im|), e_i its frexp exponent, sh_i = sum |a_il/2^e_i|^2;
    per column j of Bop likewise (f_j).  EA = max e_i, EB = max f_j over nonzero vectors.
      f0 = log2 k / 10, f1 = log2 m / 10, f2 = log2 n / 10
      crest_i = log2(r_i / 2^e_i) + log2(2k)/2 - log2(sh_i)/2 (0 when every real and
      imaginary part of the row has the same magnitude)
      f3, f4, f5 = mean, max, population std of the crest over the nonzero rows of Aop, / 8
      f6, f7, f8 = the same over the nonzero columns of Bop, / 8
      f9  = (max e_i - mean e_i) / 16 over the nonzero rows
      f10 = the same over the nonzero columns of Bop
      log2 c = log2(n ||zs||_F^2 / ||X||_F^2) / 2 + E     (estimate of log2 ||Aop Bop||_F)
      lA = log2 ||Aop||_F^2 = log2 sum_i sh_i 4^e_i, lB likewise
      f11 = (lA/2 + lB/2 - log2 c) / 16                    (cancellation)
      f12 = (log2(sum_i 4^e_i 2^lB + sum_j 4^f_j 2^lA) / 2 - log2 c) / 16
            (scale of the truncation error relative to the product)
      f13, f14 = fraction of exactly zero entries of Aop, Bop
      f15 = 1
    f11 and f12 are 0 when zs = 0 or an operand is zero; statistics over an empty set are 0."""
    Aop = np.asarray(Aop, dtype=np.complex128)
    Bop = np.asarray(Bop, dtype=np.complex128)
    m, k = Aop.shape
    n = Bop.shape[1]
    f = np.zeros(NF)
    f[0] = math.log2(max(k, 1)) / 10
    f[1] = math.log2(max(m, 1)) / 10
    f[2] = math.log2(max(n, 1)) / 10
    ra, ea, sa, za = _vector_stats(Aop)
    rb, eb, sb, zb = _vector_stats(Bop.T)

    def crest_stats(r, e, sh):
        nz = r > 0
        if not np.any(nz):
            return 0.0, 0.0, 0.0, 0.0
        c = np.log2(np.ldexp(r[nz], -e[nz])) + 0.5 * math.log2(2 * k) - 0.5 * np.log2(sh[nz])
        ee = e[nz].astype(np.float64)
        return c.mean(), c.max(), c.std(), ee.max() - ee.mean()

    ca = crest_stats(ra, ea, sa)
    cb = crest_stats(rb, eb, sb)
    f[3], f[4], f[5] = ca[0] / 8, ca[1] / 8, ca[2] / 8
    f[6], f[7], f[8] = cb[0] / 8, cb[1] / 8, cb[2] / 8
    f[9], f[10] = ca[3] / 16, cb[3] / 16
    nza, nzb = ra > 0, rb > 0
    EA = int(ea[nza].max()) if np.any(nza) else 0
    EB = int(eb[nzb].max()) if np.any(nzb) else 0
    if exact:
        zr, zi, ez = _int_mul(_to_int(Aop), _int_mul(_to_int(Bop), _to_int(X)))
        zs = (zr, zi, ez - EA - EB)
        z2 = math.ldexp(float(_int_sq(zr, zi) >> max(0, _int_sq(zr, zi).bit_length() - 60)),
                        2 * zs[2] + max(0, _int_sq(zr, zi).bit_length() - 60))
    else:
        zs = _scaled(Aop, -EA) @ (_scaled(Bop, -EB) @ X)
        z2 = float(np.sum(np.abs(zs) ** 2))
    if z2 > 0 and np.any(nza) and np.any(nzb):
        lc = 0.5 * math.log2(n * z2 / float(np.sum(np.abs(X) ** 2))) + EA + EB
        lA = _log2sum(sa[nza], ea[nza])
        lB = _log2sum(sb[nzb], eb[nzb])
        f[11] = (0.5 * lA + 0.5 * lB - lc) / 16
        ta = _log2sum(np.ones(int(nza.sum())), ea[nza]) + lB
        tb = _log2sum(np.ones(int(nzb.sum())), eb[nzb]) + lA
        hi = max(ta, tb)
        f[12] = (0.5 * (hi + math.log2(2.0 ** (ta - hi) + 2.0 ** (tb - hi))) - lc) / 16
    f[13] = float(za.sum()) / max(1, m * k)
    f[14] = float(zb.sum()) / max(1, k * n)
    f[15] = 1.0
    return f, zs, EA + EB


def residual_estimate(D, X, zs, E):
    """||2^-E D X - zs||_F / ||zs||_F for the scaled probe product zs of ``features`` (0 when
    both vanish, inf when only zs does); exact when zs is an integer image."""
    if isinstance(zs, tuple):
        zr, zi, ez = zs
        wr, wi, ew = _int_mul(_to_int(D), _to_int(X))
        ew -= E
        e0 = min(ez, ew)                               # common scale 2^e0
        dr = wr * (1 << (ew - e0)) - zr * (1 << (ez - e0))
        di = wi * (1 << (ew - e0)) - zi * (1 << (ez - e0))
        num = _int_sq(dr, di)
        den = _int_sq(zr, zi) << (2 * (ez - e0))
        if den == 0:
            return 0.0 if num == 0 else math.inf
        q = (num << 200) // den                        # num / den with 200 extra bits
        return math.sqrt(math.ldexp(float(q >> max(0, q.bit_length() - 60)), max(0, q.bit_length() - 60) - 200))
    w = _scaled(np.asarray(D, dtype=np.complex128) @ X, -E)
    num = float(np.sum(np.abs(w - zs) ** 2))
    den = float(np.sum(np.abs(zs) ** 2))
    if den == 0.0:
        return 0.0 if num == 0.0 else math.inf
    return math.sqrt(num / den)
