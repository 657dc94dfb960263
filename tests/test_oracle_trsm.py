"""Pins of the ZTRSM and LU-variant oracle (oracle/trsm.py) against the mathematics: known
solutions, ignored triangles and diagonals, convergence of the emulated solve to binary64 as
S grows, the LU reconstruction, and tau_00 of the LU variant against the full inverse."""
import numpy as np
import pytest

import synth
from oracle import kkr, trsm


def _rand(m, n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))


def _tri(w, upper, seed):
    T = _rand(w, w, seed) * 0.3
    T += np.eye(w) * (2.0 + 1.0j)                     # well conditioned
    return np.triu(T) if upper else np.tril(T)


@pytest.mark.parametrize("upper", [True, False])
@pytest.mark.parametrize("unit", [True, False])
def test_fp64_solve_recovers_known_solution(upper, unit):
    w, m = 21, 13
    T = _tri(w, upper, 1)
    if unit:
        np.fill_diagonal(T, 1.0)
    X = _rand(m, w, 2)
    B = X @ T
    assert kkr.rel_err(trsm.trsm_right_fp64(T, B, upper, unit), X) < 1e-13
    # a 2 x 2 case by hand: [x1 x2] [[a, b], [0, d]] = [c1 c2] -> x1 = c1 / a, x2 = (c2 - x1 b) / d
    T2 = np.array([[2.0, 1.0j], [0.0, 4.0]])
    x = trsm.trsm_right_fp64(T2, np.array([[2.0, 1.0]]), True, False)
    assert np.allclose(x, [[1.0, (1.0 - 1.0j) / 4.0]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("upper", [True, False])
def test_other_triangle_and_unit_diagonal_are_not_read(upper):
    w, m = 37, 9
    T = _tri(w, upper, 3)
    B = _rand(m, w, 4)
    junk = np.array(T)
    mask = np.tril(np.ones((w, w)), -1) if upper else np.triu(np.ones((w, w)), 1)
    junk[mask.astype(bool)] = 1e30 + 1e30j
    for unit in (False, True):
        ref = trsm.trsm_right_emulated(T, B, 7, upper, unit)
        got = trsm.trsm_right_emulated(junk, B, 7, upper, unit)
        assert np.array_equal(got, ref)
    ones = np.array(T)
    np.fill_diagonal(ones, 1.0)
    big = np.array(T)
    np.fill_diagonal(big, 1e300)
    assert np.array_equal(trsm.trsm_right_emulated(big, B, 5, upper, True),
                          trsm.trsm_right_emulated(ones, B, 5, upper, True))


@pytest.mark.parametrize("upper", [True, False])
def test_emulated_solve_converges_to_fp64(upper):
    w, m = 37, 20                                      # ragged blocks 16 + 16 + 5
    T = _tri(w, upper, 5)
    B = _rand(m, w, 6)
    ref = trsm.trsm_right_fp64(T, B, upper, False)
    errs = [kkr.rel_err(trsm.trsm_right_emulated(T, B, S, upper, False), ref) for S in (3, 5, 7, 9)]
    assert errs[3] < 1e-14
    assert errs[0] > errs[1] > errs[2]


def test_one_block_is_a_product_with_the_block_inverse():
    w, m = 12, 7
    T = _tri(w, True, 7)
    B = _rand(m, w, 8)
    from oracle import ozaki
    got = trsm.trsm_right_emulated(T, B, 6, True, False, bt=16)
    assert np.array_equal(got, ozaki.ozaki_zgemm(B, np.linalg.inv(np.triu(T)), 6))


def test_lu_panel_reconstructs_with_forced_interchanges():
    w = 24
    D = 0.05 * _rand(w, w, 9)
    D[np.arange(w), w - 1 - np.arange(w)] += 1.0        # reversal-dominated: every column pivots
    LU, perm = trsm.lu_panel(D)
    L = np.tril(LU, -1) + np.eye(w)
    U = np.triu(LU)
    PD = np.array(D)
    for k, pk in enumerate(perm):
        PD[[k, pk]] = PD[[pk, k]]
    assert np.linalg.norm(PD - L @ U) <= 1e-14 * np.linalg.norm(D)
    assert (perm != np.arange(w)).sum() >= w // 2
    assert np.abs(L).max() <= 1.0 + 1e-12               # partial pivoting bounds the multipliers


@pytest.mark.parametrize("S", [5, 7])
def test_tau00_lu_variant_matches_full_inverse(S):
    t, G, _ = synth.kkr_system(9, 16, 0.5 + 0.05j, atom=1)
    M = kkr.kkr_build(t, G)
    full = kkr.tau00_full(M, t[0])
    lu = trsm.tau00_lu(M, t[0], 48, S)
    assert kkr.rel_err(lu, full) <= (1e-10 if S == 7 else 1e-7)
    inv = kkr.tau00_block(M, t[0], 48, S=S)
    assert kkr.rel_err(lu, inv) <= (1e-11 if S == 7 else 1e-7)
