"""Pins of the emulated-ZGEMM oracle against what the mathematics fixes (CPU only)."""
import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import c_oracle as co
from oracle import ozaki as oz

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand(m, n, seed, sigma=2.0):
    return synth.scaled_uniform(seed, 0, (m, n), sigma) + 1j * synth.scaled_uniform(seed, 1, (m, n), sigma)


# ----------------------------------------------------------------------------- exponents

def test_exponents_match_frexp():
    X = _rand(40, 17, 1)
    X[3] = 0.0                                   # zero row
    X[5, 2] = 2.0 ** 10                          # exact power of two as row max
    X[6] = 5e-324                                # subnormal row
    X[7, 0] = -1e300
    e = oz.row_exponents(X)
    for i in range(X.shape[0]):
        mu = max(max(abs(z.real), abs(z.imag)) for z in X[i])
        assert e[i] == (math.frexp(mu)[1] if mu else 0)
        if mu:
            assert 0.5 <= math.ldexp(mu, -int(e[i])) < 1.0


def test_exponents_reject_nonfinite():
    X = _rand(4, 4, 2)
    X[1, 1] = np.nan
    with pytest.raises(ValueError):
        oz.row_exponents(X)


def test_precision_modes_golden():
    rows = [l.split() for l in open(os.path.join(GOLD, "precision_modes.txt")) if l.strip() and l[0] != "#"]
    for bits, S in rows:
        assert oz.bits_for(int(S)) == int(bits)


# ----------------------------------------------------------------------------- slices

def test_digits_golden():
    rows = [l.split() for l in open(os.path.join(GOLD, "digits.txt")) if l.strip() and l[0] != "#"]
    for r in rows:
        x, mx, S, e, X = float(r[0]), float(r[1]), int(r[2]), int(r[3]), int(r[4])
        d = [int(v) for v in r[5:]]
        ee = oz.row_exponents(np.array([[complex(mx, 0.0)]]))[0]
        assert ee == e
        XX = oz.integer_image(np.array([[x]]), np.array([e]), S)[0, 0]
        assert XX == X
        D = oz.balanced_digits(np.array([X], dtype=object), S)[:, 0]
        assert list(D) == d


@pytest.mark.parametrize("S", [1, 2, 3, 5, 7, 8, 9, 10, 13])
def test_digit_reconstruction_invariant(S):
    A = _rand(9, 11, 3 + S)
    e = oz.row_exponents(A)
    B = oz.bits_for(S)
    for part in (A.real, A.imag):
        X = oz.integer_image(part, e, S)
        D = oz.balanced_digits(X, S)
        if S > 1:
            assert D[1:].min() >= -128 and D[1:].max() <= 127
        assert D[0].min() >= -128 and D[0].max() <= 128
        for i in range(X.shape[0]):
            for l in range(X.shape[1]):
                val = sum(int(D[t, i, l]) * 256 ** (S - 1 - t) for t in range(S))
                assert val == X[i, l]
                assert abs(X[i, l]) < 2 ** B
                exact = Fraction(float(part[i, l])) * Fraction(2) ** (B - int(e[i]))
                assert abs(exact - X[i, l]) < 1
                assert X[i, l] == int(exact)          # truncation toward zero


@pytest.mark.parametrize("S", [2, 3, 5, 7, 8])
def test_balanced_digits_are_bytes_of_the_biased_image(S):
    """The identity the split's compile-time-S path rests on: with C = 128 (1 + 256 + ... +
    256^(S-2)), the balanced digits of X below the top are the bytes of Y = X + C minus 128 and
    the top digit is floor(Y / 256^(S-1)); and a digit d (|d| <= 511) is the binary16 value
    whose bit pattern is 0x6600 + d minus 1536 (exactly, +0 for d = 0), -d the value 1536
    minus it."""
    rng = random.Random(40 + S)
    lim = 2 ** (8 * S - 1) - 1
    xs = [0, 1, -1, lim, -lim, 127, -128, 128, -129] + [rng.randint(-lim, lim) for _ in range(500)]
    D = oz.balanced_digits(np.array(xs, dtype=object), S)
    C = sum(128 * 256 ** t for t in range(S - 1))
    for i, X in enumerate(xs):
        Y = X + C
        for t in range(1, S):                       # D[t]: place S - 1 - t from the bottom
            assert int(D[t, i]) + 128 == (Y >> (8 * (S - 1 - t))) & 255
        assert int(D[0, i]) == Y >> (8 * (S - 1))
    d = np.arange(-511, 512)
    biased = (0x6600 + d).astype(np.uint16).view(np.float16)
    k = np.float16(1536)
    assert k.view(np.uint16) == 0x6600
    assert np.array_equal(((biased - k).astype(np.float16)).view(np.uint16), d.astype(np.float16).view(np.uint16))
    neg = (k - biased).astype(np.float16)
    assert np.array_equal(neg.astype(np.int64), -d)
    assert neg[d == 0].view(np.uint16)[0] == 0      # +0, as the int -> half conversion gives


def test_negated_imag_block_is_digitwise_negation():
    B = _rand(6, 5, 7)
    f, D = oz.split_right(B, 4)
    k = B.shape[0]
    assert np.array_equal(D[:, 0::2, k:], -D[:, 1::2, :k])
    assert np.array_equal(D[:, 0::2, :k], D[:, 1::2, k:])


# ----------------------------------------------------------------------------- integer GEMMs

def test_group_sums_brute_force():
    S = 4
    A = _rand(5, 3, 11)
    B = _rand(3, 4, 12)
    e, DA = oz.split_left(A, S)
    f, DB = oz.split_right(B, S)
    for mode in ("tri", "full"):
        P = oz.pair_set(S, mode)
        G = oz.group_sums(DA, DB, P)
        ref = {}
        for (s, t) in P:
            g = s + t
            ref.setdefault(g, [[0] * DB.shape[1] for _ in range(DA.shape[1])])
            for i in range(DA.shape[1]):
                for j in range(DB.shape[1]):
                    ref[g][i][j] += sum(int(DA[s - 1, i, l]) * int(DB[t - 1, j, l]) for l in range(DA.shape[2]))
        assert sorted(G) == sorted(ref)
        for g in G:
            assert G[g].tolist() == ref[g]


def test_pair_sets():
    assert len(oz.pair_set(7)) == 28
    assert all(s + t <= 8 for s, t in oz.pair_set(7))
    assert len(oz.pair_set(5, "full")) == 25


# ----------------------------------------------------------------------------- reconstruction

def test_round_scaled_is_correct_rounding():
    rng = random.Random(5)
    cases = [(1, 0), (3, -1), (-5, 2), ((1 << 53) + 1, 0), ((1 << 54) + 2, -1), ((1 << 53) + 3, -1),
             (1, -1074), (1, -1075), (3, -1076), (1, 1023), (1, 1024), ((1 << 60) - 1, -1130)]
    for _ in range(3000):
        T = rng.randrange(-(1 << rng.randrange(1, 120)), 1 << rng.randrange(1, 120))
        cases.append((T, rng.randrange(-1250, 960)))
    for T, E in cases:
        v = oz.round_scaled(T, E)
        if T == 0:
            assert v == 0.0
            continue
        exact = Fraction(T) * Fraction(2) ** E
        if math.isinf(v):
            assert abs(exact) >= Fraction(2) ** 1024 - Fraction(2) ** 970
            continue
        # v is a binary64 nearest to exact: no binary64 neighbour is strictly closer
        err = abs(Fraction(v) - exact)
        for nb in (math.nextafter(v, math.inf), math.nextafter(v, -math.inf)):
            if not math.isinf(nb):
                assert err <= abs(Fraction(nb) - exact)
        assert co.round_scaled(T, E) == v


def test_full_pairs_equal_exact_product_of_truncated_operands():
    A = _rand(4, 5, 21)
    B = _rand(5, 3, 22)
    for S in (1, 2, 3):
        Z = oz.ozaki_zgemm(A, B, S, "full")
        ref = oz.exact_product_rounded(*oz.truncated_operands(A, B, S))
        assert np.array_equal(Z, ref)


def test_identity_left_returns_truncated_right():
    S = 5
    B = _rand(6, 4, 31)
    Z = oz.ozaki_zgemm(np.eye(6, dtype=np.complex128), B, S)
    Ar, Ai, Br, Bi = oz.truncated_operands(np.eye(6, dtype=np.complex128), B, S)
    expect = np.array([[complex(float(Br[j][l]), float(Bi[j][l])) for j in range(4)] for l in range(6)])
    assert np.array_equal(Z, expect)


def test_power_of_two_outer_products_exact_at_S1():
    rng = np.random.default_rng(3)
    a = (2.0 ** rng.integers(-4, 5, size=(7, 1))) * rng.choice([-1, 1], size=(7, 1))
    b = (2.0 ** rng.integers(-4, 5, size=(1, 6))) * rng.choice([-1, 1], size=(1, 6))
    A = a.astype(np.complex128)
    B = b.astype(np.complex128) * 1j
    Z = oz.ozaki_zgemm(A, B, 1)
    # each row/column has a single entry, so it is its own row max and scales to 2^-1 exactly
    assert np.array_equal(Z, A @ B)


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5, 6, 7, 8])
def test_triangular_error_within_closed_form_bound(S):
    A = _rand(12, 10, 41)
    B = _rand(10, 9, 42)
    Z = oz.ozaki_zgemm(A, B, S)
    X = oz.zgemm_exact(A, B)
    bound = oz.ozaki_error_bound(A, B, S)
    assert np.all(np.abs(Z.real - X.real) <= bound)
    assert np.all(np.abs(Z.imag - X.imag) <= bound)


def test_error_falls_with_S_until_binary64_floor():
    A = _rand(24, 20, 51)
    B = _rand(20, 16, 52)
    X = oz.zgemm_exact(A, B)
    errs = [np.linalg.norm(oz.ozaki_zgemm(A, B, S) - X) / np.linalg.norm(X) for S in range(1, 10)]
    for S in range(1, 7):
        assert errs[S] < errs[S - 1] / 16          # about 2^-8 per slice, at least 2^-4
    assert errs[7] < 4e-16 and errs[8] < 4e-16


def test_config1_relative_error_at_S7():
    A, B = synth.zgemm_operands(512, 512, 512)
    Z = co.zgemm(A, B, 7)
    X = co.zgemm_fp64(A, B)
    assert np.linalg.norm(Z - X) / np.linalg.norm(X) <= 1e-13


def test_empty_and_degenerate_shapes():
    A = _rand(3, 0, 1).reshape(3, 0)
    B = np.zeros((0, 2), dtype=np.complex128)
    assert np.array_equal(oz.ozaki_zgemm(A, B, 3), np.zeros((3, 2)))
    Z = oz.ozaki_zgemm(np.zeros((2, 3), dtype=np.complex128), _rand(3, 2, 3), 4)
    assert np.array_equal(Z, np.zeros((2, 2)))


def test_lu_epilogue_is_one_more_rounding():
    A = _rand(5, 4, 61)
    B = _rand(4, 6, 62)
    C = _rand(5, 6, 63)
    Z = oz.ozaki_zgemm(A, B, 6)
    U = oz.ozaki_lu_update(C, A, B, 6)
    assert np.array_equal(U.real, C.real - Z.real) and np.array_equal(U.imag, C.imag - Z.imag)


# ----------------------------------------------------------------------------- C oracle

@pytest.mark.parametrize("S,mode", [(3, "tri"), (7, "tri"), (10, "tri"), (4, "full")])
def test_c_oracle_matches_python_bit_for_bit(S, mode):
    A = _rand(13, 9, 70 + S)
    B = _rand(9, 7, 80 + S)
    full = mode == "full"
    e1, D1 = oz.split_left(A, S)
    e2, D2 = co.split_left(A, S)
    f1, E1 = oz.split_right(B, S)
    f2, E2 = co.split_right(B, S)
    assert np.array_equal(e1, e2) and np.array_equal(D1, D2)
    assert np.array_equal(f1, f2) and np.array_equal(E1, E2)
    G1 = oz.group_sums(D1, E1, oz.pair_set(S, mode))
    G2 = co.group_sums(D2, E2, S, full)
    assert all(np.array_equal(G1[g], G2[g]) for g in G1)
    assert np.array_equal(oz.ozaki_zgemm(A, B, S, mode), co.zgemm(A, B, S, full))
    C = _rand(13, 7, 90)
    assert np.array_equal(oz.ozaki_lu_update(C, A, B, S, mode), co.zgemm_lu(C, A, B, S, full))
