"""Seeded synthetic inputs for the emulated ZGEMM and the KKR tau_00 solve.

This module is shared by the oracle tests and the GPU path.  It holds no arithmetic
of the method itself (no exponent scan, no slicing, no integer products, no
reconstruction, no factorisation): only the recipes that produce input matrices.

Every random number comes from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): the i-th output of stream (seed, stream) is mix(base + (i+1)*gamma)
with gamma = 0x9E3779B97F4A7C15 and base = mix(seed * 0x100000001B3 ^ stream).
Any element can therefore be regenerated on its own, by any implementation.

Workloads (all synthetic; the paper's FeNi3 input is not available):

* ``zgemm_operands``: complex m x k / k x n matrices whose real and imaginary parts
  are U(-1, 1) * 2**round(N(0, 2)), independently per element.
* ``bcc_sites``: the first L sites of a bcc lattice (lattice constant 1) sorted by
  distance from the origin, ties broken lexicographically; site 0 is the centre.
* ``kkr_system``: block-diagonal single-site t (one b x b block per site, diagonal,
  entries 0.1 * (0.5 + U(0, 1)) * exp(i phi)) and a structure-constant stand-in
  G with zero diagonal blocks and G_ij = R_ij * exp(-r_ij / 1.5) * exp(i k r_ij),
  R_ij entries (U(-1, 1) + i U(-1, 1)) / sqrt(b), k = sqrt(E) (principal branch).
  G is rescaled so that the power-iteration estimate of ||t G||_2 is at most 0.9.
* ``contour``: a semicircle in the upper half plane with centre -0.3 Ry and radius
  1.0 Ry (so it ends at E_F = 0.7 Ry), nodes at the Gauss-Legendre points of
  theta in [asin(0.005), pi - asin(0.005)], so that Im E runs from 0.005 to 1.0.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _base(seed: int, stream: int) -> np.uint64:
    x = ((seed * 0x100000001B3) & _MASK) ^ (stream & _MASK)
    return _mix(np.array([x], dtype=np.uint64))[0]


def splitmix64(seed: int, stream: int, idx) -> np.ndarray:
    """Raw 64-bit outputs number ``idx`` (array of non-negative ints) of a stream."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = _base(seed, stream) + (idx + np.uint64(1)) * _GAMMA
    return _mix(state)


def uniform(seed: int, stream: int, idx) -> np.ndarray:
    """U[0, 1) doubles with 53 random bits."""
    return (splitmix64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, idx) -> np.ndarray:
    """N(0, 1) by Box-Muller from outputs 2*idx and 2*idx+1 of the stream."""
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = 1.0 - uniform(seed, stream, 2 * idx)          # (0, 1]
    u2 = uniform(seed, stream, 2 * idx + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------- ZGEMM operands

def scaled_uniform(seed: int, stream: int, shape, sigma: float = 2.0) -> np.ndarray:
    """U(-1, 1) * 2**round(N(0, sigma)) per element (float64, C order)."""
    n = int(np.prod(shape))
    idx = np.arange(n, dtype=np.uint64)
    u = 2.0 * uniform(seed, 2 * stream, idx) - 1.0
    e = np.rint(sigma * normal(seed, 2 * stream + 1, idx))
    return np.ldexp(u, e.astype(np.int64)).reshape(shape)


def zgemm_operands(m: int, n: int, k: int, seed: int = 20260330, sigma: float = 2.0):
    """A (m x k) and B (k x n) complex128, in the mathematical orientation (C order)."""
    A = scaled_uniform(seed, 0, (m, k), sigma) + 1j * scaled_uniform(seed, 1, (m, k), sigma)
    B = scaled_uniform(seed, 2, (k, n), sigma) + 1j * scaled_uniform(seed, 3, (k, n), sigma)
    return A, B


# ----------------------------------------------------------------------------- KKR geometry

def bcc_sites(L: int) -> np.ndarray:
    """First L bcc lattice sites (L x 3, lattice constant 1) by distance, centre first."""
    if L < 1:
        raise ValueError("L must be positive")
    R = 1
    while True:
        rng = np.arange(-R, R + 1, dtype=np.float64)
        g = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
        pts = np.concatenate([g, g + 0.5])
        r2 = (pts ** 2).sum(1)
        # every site with |r| <= R - 0.5 is inside the enumerated cube
        inside = r2 <= (R - 0.5) ** 2
        if inside.sum() >= L:
            pts = pts[inside]
            r2 = r2[inside]
            order = np.lexsort((pts[:, 2], pts[:, 1], pts[:, 0], r2))
            return pts[order[:L]].copy()
        R += 1


def shell_counts(sites: np.ndarray, tol: float = 1e-9) -> list:
    """Cumulative number of sites at the end of each distance shell."""
    r = np.sqrt((sites ** 2).sum(1))
    out = []
    for i in range(1, len(r)):
        if r[i] - r[i - 1] > tol:
            out.append(i)
    out.append(len(r))
    return out


def kkr_system(L: int, b: int, E: complex, seed: int = 20260331, atom: int = 0,
               max_norm: float = 0.9):
    """t (L x b x b), G (n x n, n = L*b) complex128 in C order, and the site positions.

    The stream numbers separate t and G draws and the atom index, so that atoms of a
    batch get independent matrices from one seed.
    """
    pos = bcc_sites(L)
    t = kkr_t(L, b, seed=seed, atom=atom)
    G = _structure_G(_random_R(L, b, seed, atom), pos, t, E, max_norm)
    return t, G, pos


def kkr_contour_G(L: int, b: int, energies, seed: int = 20260331, atom: int = 0, max_norm: float = 0.9,
                  workers: int = 1):
    """G at each energy of ``energies``, element for element what ``kkr_system(L, b, E, seed,
    atom)[1]`` returns, with the random block factors R drawn once for all energies (the
    energy enters only through exp(i k r) and the rescaling).  A generator of n x n arrays in
    the order of ``energies``; ``workers`` > 1 computes them on that many threads."""
    pos = bcc_sites(L)
    t = kkr_t(L, b, seed=seed, atom=atom)
    R = _random_R(L, b, seed, atom)
    if workers <= 1:
        for E in energies:
            yield _structure_G(R, pos, t, E, max_norm)
        return
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(workers) as ex:
        yield from ex.map(lambda E: _structure_G(R, pos, t, E, max_norm), list(energies))


def _random_R(L: int, b: int, seed: int, atom: int) -> np.ndarray:
    """R_ij entries (U(-1, 1) + i U(-1, 1)) / sqrt(b) of the structure-constant stand-in."""
    n = L * b
    st = 4 * atom
    idx = np.arange(n * n, dtype=np.uint64)
    Rr = 2.0 * uniform(seed, st + 2, idx) - 1.0
    Ri = 2.0 * uniform(seed, st + 3, idx) - 1.0
    return ((Rr + 1j * Ri) / math.sqrt(b)).reshape(n, n)


def _structure_G(R: np.ndarray, pos: np.ndarray, t: np.ndarray, E: complex, max_norm: float) -> np.ndarray:
    """G_ij = R_ij exp(-r_ij / 1.5) exp(i k r_ij) (zero diagonal blocks), rescaled so that the
    power-iteration estimate of ||t G||_2 is at most max_norm."""
    L = pos.shape[0]
    b = R.shape[0] // L
    d = np.sqrt(((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1))      # L x L
    kk = np.sqrt(complex(E))
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.exp(-d / 1.5) * np.exp(1j * kk * d)
    f[np.arange(L), np.arange(L)] = 0.0
    # the site factor f_IJ multiplies every element of block (I, J)
    G = (R.reshape(L, b, L, b) * f[:, None, :, None]).reshape(L * b, L * b)
    # power-iteration estimate of ||t G||_2, then rescale G
    tG = block_diag_times(t, G)
    nrm = _norm2_estimate(tG)
    if nrm > max_norm:
        G *= max_norm / nrm
    return G


def kkr_t(L: int, b: int, seed: int = 20260331, atom: int = 0) -> np.ndarray:
    """Single-site t of one atom: L diagonal b x b blocks, entries 0.1 (0.5 + U(0,1)) e^(i phi)."""
    st = 4 * atom
    u = uniform(seed, st, np.arange(L * b, dtype=np.uint64)).reshape(L, b)
    phi = 2 * np.pi * uniform(seed, st + 1, np.arange(L * b, dtype=np.uint64)).reshape(L, b)
    t = np.zeros((L, b, b), dtype=np.complex128)
    t[:, np.arange(b), np.arange(b)] = 0.1 * (0.5 + u) * np.exp(1j * phi)
    return t


def block_diag_times(t: np.ndarray, X: np.ndarray) -> np.ndarray:
    """blockdiag(t) @ X for t of shape (L, b, b); used only to size the inputs."""
    L, b, _ = t.shape
    return np.einsum("lij,ljn->lin", t, X.reshape(L, b, -1)).reshape(L * b, -1)


def _norm2_estimate(X: np.ndarray, iters: int = 30) -> float:
    v = np.ones(X.shape[1], dtype=np.complex128) / math.sqrt(X.shape[1])
    s = 0.0
    for _ in range(iters):
        w = X @ v
        v = np.dot(w.conj(), X).conj()                 # X^H w without a conjugated copy of X
        s = np.linalg.norm(v)
        if s == 0:
            return 0.0
        v /= s
    return math.sqrt(s)


def kkr_matrix(t: np.ndarray, G: np.ndarray) -> np.ndarray:
    """M = I - t G (complex128, C order) for inputs given directly as M."""
    n = G.shape[0]
    return np.eye(n, dtype=np.complex128) - block_diag_times(t, G)


# ----------------------------------------------------------------------------- contour

def contour(npts: int = 32, e_fermi: float = 0.7, radius: float = 1.0, im_min: float = 0.005):
    """Semicircle nodes E_z and weights w_z with sum_z w_z f(E_z) ~ integral of f along the
    path from the bottom of the contour to E_F."""
    x, w = np.polynomial.legendre.leggauss(npts)
    th0 = math.asin(im_min / radius)
    a, bnd = th0, math.pi - th0
    theta = 0.5 * (bnd - a) * x + 0.5 * (bnd + a)
    c = e_fermi - radius
    E = c + radius * np.exp(1j * theta)
    # the path runs from the bottom (theta = pi - th0) to E_F (theta = th0): dE/dtheta < 0
    dE = -1j * radius * np.exp(1j * theta) * 0.5 * (bnd - a) * w
    # order from the bottom of the contour (theta near pi) to E_F
    order = np.argsort(-theta)
    return E[order], dE[order]


def liz_sizes(natoms: int, lo: int = 27, hi: int = 169, seed: int = 20260332) -> np.ndarray:
    """LIZ site counts drawn uniformly from lo..hi inclusive."""
    u = uniform(seed, 0, np.arange(natoms, dtype=np.uint64))
    return lo + np.floor(u * (hi - lo + 1)).astype(np.int64)
