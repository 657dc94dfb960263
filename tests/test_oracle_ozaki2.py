"""Pins of the Ozaki-II (CRT) oracle: moduli, CRT constants and reconstruction, the scaling
bound, and the full product against the exact product of the integer images (CPU only)."""
import math
import random

import numpy as np
import pytest

import synth
from oracle import ozaki2 as oz2
from oracle import ozaki as oz


def test_moduli_are_the_largest_pairwise_coprime_integers():
    ms = oz2.moduli(18)
    # worked by hand: 254, 252, 250 share 2; 249, 243, 237 share 3; 245, 235 share 5 ...
    assert ms[:8] == [256, 255, 253, 251, 247, 241, 239, 233]
    assert all(math.gcd(a, b) == 1 for i, a in enumerate(ms) for b in ms[i + 1:])
    assert ms == sorted(ms, reverse=True) and max(ms) <= 256
    assert math.prod(oz2.moduli(16)) < 2 ** 128


def test_crt_constants_and_round_trip():
    ms = oz2.moduli(10)
    P, cs = oz2.crt_constants(ms)
    for l, (m, c) in enumerate(zip(ms, cs)):
        assert c % m == 1 and all(c % mj == 0 for j, mj in enumerate(ms) if j != l)
    rng = random.Random(5)
    for _ in range(500):
        x = rng.randrange(-(P // 2) + 1, P // 2)
        assert oz2.crt([x % m for m in ms], ms, P, cs) == x
        assert oz2.crt([oz2.sym_residue(x, m) for m in ms], ms, P, cs) == x
    for m in ms:
        assert all(-m / 2 <= oz2.sym_residue(x, m) <= m / 2 for x in range(-600, 600))


@pytest.mark.parametrize("k", [1, 16, 1000, 5650])
def test_beta_is_the_largest_safe_scale(k):
    P, _ = oz2.crt_constants(oz2.moduli(14))
    b = oz2.beta_bits(k, P)
    assert 2 * k * 4 ** b * 2 < P <= 2 * k * 4 ** (b + 1) * 2


def _ops(m, n, k, seed, sigma=2.0):
    A = synth.scaled_uniform(seed, 0, (m, k), sigma) + 1j * synth.scaled_uniform(seed, 1, (m, k), sigma)
    B = synth.scaled_uniform(seed + 1, 0, (k, n), sigma) + 1j * synth.scaled_uniform(seed + 1, 1, (k, n), sigma)
    return A, B


@pytest.mark.parametrize("N", [6, 10, 16])
def test_product_is_the_exact_integer_product_rounded_once(N):
    A, B = _ops(5, 4, 7, 11)
    C = oz2.ozaki2_zgemm(A, B, N)
    re, im, e, f, beta = oz2.exact_truncated_product(A, B, N)
    for i in range(5):
        for j in range(4):
            E = int(e[i]) + int(f[j]) - 2 * beta
            assert C[i, j].real == oz.round_scaled(re[i][j], E)
            assert C[i, j].imag == oz.round_scaled(im[i][j], E)


def test_error_falls_with_the_number_of_moduli():
    A, B = _ops(24, 20, 40, 13, sigma=1.0)
    ref = A @ B
    errs = [np.linalg.norm(oz2.ozaki2_zgemm(A, B, N) - ref) / np.linalg.norm(ref) for N in (6, 8, 10, 12, 14, 16)]
    assert all(b < a / 100 for a, b in zip(errs[:4], errs[1:5]))     # ~16 bits per 2 moduli
    assert errs[-1] < 1e-15


def test_identity_returns_the_truncated_right_operand():
    k = 12
    _, B = _ops(1, 9, k, 17)
    C = oz2.ozaki2_zgemm(np.eye(k, dtype=np.complex128), B, 12)
    P, _ = oz2.crt_constants(oz2.moduli(12))
    beta = oz2.beta_bits(k, P)
    f = oz.row_exponents(B.T)
    for j in range(9):
        for l in range(k):
            # identity rows have exponent 1: the row image is 2^(beta-1), so the product is the
            # truncated B entry scaled back exactly
            want = complex(oz.round_scaled(oz2.integer_image(B[l, j].real, int(f[j]), beta), int(f[j]) - beta),
                           oz.round_scaled(oz2.integer_image(B[l, j].imag, int(f[j]), beta), int(f[j]) - beta))
            assert C[l, j] == want
