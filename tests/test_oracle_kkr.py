"""Pins of the KKR tau_00 oracle and of the synthetic inputs (CPU only)."""
import os

import numpy as np
import pytest

import synth
from oracle import c_oracle as co
from oracle import kkr

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _system(L, b=16, E=0.5 + 0.05j, seed=20260331, atom=0):
    t, G, pos = synth.kkr_system(L, b, E, seed=seed, atom=atom)
    return t, G, kkr.kkr_build(t, G)


def test_bcc_shells_golden():
    want = [int(v) for l in open(os.path.join(GOLD, "bcc_shells.txt")) if l.strip() and l[0] != "#" for v in l.split()]
    assert synth.shell_counts(synth.bcc_sites(169)) == want
    s = synth.bcc_sites(65)
    assert np.all(s[0] == 0.0)
    r2 = (s ** 2).sum(1)
    assert np.all(np.diff(r2) >= -1e-12)
    assert set(np.round(r2[1:9], 12)) == {0.75}


def test_kkr_build_matches_dense_product():
    t, G, M = _system(9)
    L, b, _ = t.shape
    T = np.zeros((L * b, L * b), dtype=np.complex128)
    for i in range(L):
        T[i * b:(i + 1) * b, i * b:(i + 1) * b] = t[i]
    assert np.allclose(M, np.eye(L * b) - T @ G, rtol=0, atol=1e-15)
    for i in range(L):                                   # G_ii = 0 -> M_ii = I
        assert np.array_equal(M[i * b:(i + 1) * b, i * b:(i + 1) * b], np.eye(b))


def test_gepp_inverse_against_library_and_identity():
    t, G, M = _system(9)
    Mi = kkr.gepp_inverse(M)
    assert np.abs(M @ Mi - np.eye(M.shape[0])).max() < 1e-13
    assert np.allclose(Mi, np.linalg.inv(M), rtol=0, atol=1e-13)
    Mc = co.gepp_inverse(M)
    assert np.abs(M @ Mc - np.eye(M.shape[0])).max() < 1e-13


def test_gepp_detects_singular():
    A = np.ones((4, 4), dtype=np.complex128)
    with pytest.raises(kkr.SingularError):
        kkr.gepp_inverse(A)
    with pytest.raises(RuntimeError):
        co.gepp_inverse(A)


def test_tau00_full_against_library_solve():
    t, G, M = _system(15)
    ref = np.linalg.solve(M, np.eye(M.shape[0]))[:16, :16] @ t[0]
    assert kkr.rel_err(kkr.tau00_full(M, t[0]), ref) < 1e-13
    assert kkr.rel_err(co.tau00_full(M, t[0]), ref) < 1e-13


def test_tau00_lapack_against_gauss_jordan():
    """The library-solve reference used at the largest sizes agrees with the oracle's own
    Gauss-Jordan inverse (two independent computations of [M^-1]_00 t_0), also for b = 50."""
    for L, b in ((15, 16), (5, 50)):
        t, G, M = _system(L, b=b)
        assert kkr.rel_err(kkr.tau00_lapack(M, t[0]), co.tau00_full(M, t[0])) < 1e-13


@pytest.mark.parametrize("nb,leaf", [(16, None), (32, None), (48, None), (64, 16), (48, 16), (128, 16), (128, 48),
                                     (96, 64), (192, 64)])
def test_block_lu_agrees_with_full_inverse(nb, leaf):
    t, G, M = _system(15)
    ref = kkr.tau00_full(M, t[0])
    assert kkr.rel_err(kkr.tau00_block(M, t[0], nb, leaf=leaf), ref) < 1e-12
    assert kkr.rel_err(co.tau00_block(M, t[0], nb, leaf=leaf), ref) < 1e-12


def test_leafwise_panel_equals_whole_panel_in_exact_arithmetic():
    """With binary64 GEMMs the leaf-wise factorisation of a panel and the whole-panel pivot
    inverse differ only by rounding: the same block LU."""
    t, G, M = _system(9)
    a = kkr.tau00_block(M, t[0], 64, leaf=16)
    b = kkr.tau00_block(M, t[0], 64)
    assert kkr.rel_err(a, b) < 1e-13
    # ragged front leaves (a 128-wide panel in leaves of 48, 48, 32; 96 in 64 and 32)
    for nb, leaf in ((128, 48), (96, 64)):
        assert kkr.rel_err(kkr.tau00_block(M, t[0], nb, leaf=leaf), kkr.tau00_block(M, t[0], nb)) < 1e-13


def test_two_site_closed_form():
    t, G, M = _system(2)
    b = 16
    G01, G10 = G[:b, b:], G[b:, :b]
    # M = [[I, -t0 G01], [-t1 G10, I]]; Schur complement of the centre:
    S00 = np.eye(b) - (t[0] @ G01) @ (t[1] @ G10)
    ref = np.linalg.solve(S00, t[0])
    assert kkr.rel_err(kkr.tau00_full(M, t[0]), ref) < 1e-13
    assert kkr.rel_err(kkr.tau00_block(M, t[0], 16), ref) < 1e-13
    assert kkr.rel_err(kkr.tau00_block(M, t[0], 16, S=7), ref) < 1e-12


def test_degenerate_t_and_G():
    t, G, M = _system(9)
    tz = np.zeros_like(t)
    Mz = kkr.kkr_build(tz, G)
    assert np.array_equal(Mz, np.eye(Mz.shape[0]))
    assert np.array_equal(kkr.tau00_block(Mz, tz[0], 16, S=5), np.zeros((16, 16)))
    M0 = kkr.kkr_build(t, np.zeros_like(G))
    assert np.allclose(kkr.tau00_block(M0, t[0], 16, S=5), t[0], rtol=0, atol=0)


def test_emulated_block_lu_error_per_S():
    t, G, M = _system(15)
    ref = kkr.tau00_full(M, t[0])
    for nb, leaf in ((64, None), (64, 16), (128, 48)):     # whole-panel pivot blocks, and leaf by leaf
        errs = {S: kkr.rel_err(co.tau00_block(M, t[0], nb, S=S, leaf=leaf), ref) for S in (3, 4, 5, 6, 7)}
        assert errs[7] <= 1e-10
        for S in (3, 4, 5, 6):
            assert errs[S + 1] < errs[S]
        # the Python and C restatements of the algorithm agree to rounding
        py = kkr.tau00_block(M, t[0], nb, S=5, leaf=leaf)
        assert kkr.rel_err(py, co.tau00_block(M, t[0], nb, S=5, leaf=leaf)) < 1e-13


def test_config2_system_is_well_posed():
    t, G, M = _system(65)
    tG = np.eye(M.shape[0]) - M
    assert np.linalg.norm(tG, 2) <= 0.9 + 1e-9
    assert M.shape == (1040, 1040)


def test_contour_range():
    E, w = synth.contour(32)
    assert len(E) == 32
    assert np.all(E.imag > 0.005) and E.imag.max() < 1.0
    assert np.all(E.real >= -1.3 - 1e-12) and np.all(E.real <= 0.7 + 1e-12)
    # the quadrature integrates a linear function along the arc exactly
    c = 0.7 - 1.0
    th0 = np.arcsin(0.005)
    za, zb = c + np.exp(1j * (np.pi - th0)), c + np.exp(1j * th0)
    assert abs(np.sum(w * E) - (zb ** 2 - za ** 2) / 2) < 1e-12


def test_generators_are_counter_based():
    a = synth.uniform(7, 3, np.arange(10, dtype=np.uint64))
    b = synth.uniform(7, 3, np.array([4, 9], dtype=np.uint64))
    assert a[4] == b[0] and a[9] == b[1]
    assert np.all((a >= 0) & (a < 1))
    # SplitMix64 published test vector: seed state 0 -> first output 0xE220A8397B1DCDAF
    z = synth._mix(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))[0]
    assert int(z) == 0xE220A8397B1DCDAF


def test_contour_trace_of_a_polynomial_is_exact():
    """G = 0 gives tau_00 = t_0; with t_0(z) = z I the contour sum is b (z_b^2 - z_a^2) / 2,
    which the Gauss-Legendre rule integrates exactly."""
    E, w = synth.contour(32)
    b = 16
    taus = [kkr.tau00_full(np.eye(b, dtype=np.complex128), z * np.eye(b)) for z in E]
    tr, integral = kkr.contour_trace(taus, w)
    assert np.allclose(tr, b * E, rtol=0, atol=1e-14)
    th0 = np.arcsin(0.005)
    za, zb = -0.3 + np.exp(1j * (np.pi - th0)), -0.3 + np.exp(1j * th0)
    assert abs(integral - b * (zb ** 2 - za ** 2) / 2) < 1e-11


def test_contour_G_equals_the_single_energy_recipe():
    """kkr_contour_G draws the random block factors once for all energies: each G it yields is
    element for element the G of kkr_system at that energy (same seed and atom)."""
    E, _ = synth.contour(32)
    zs = [0, 7, 31]
    got = list(synth.kkr_contour_G(15, 16, [complex(E[z]) for z in zs], atom=2, workers=2))
    for z, G in zip(zs, got):
        assert np.array_equal(G, synth.kkr_system(15, 16, complex(E[z]), atom=2)[1])
