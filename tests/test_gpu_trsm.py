"""GPU parity of the emulated right-side ZTRSM and of the LU-based tau_00 variant against the
oracle (oracle/trsm.py), through the C ABI."""
import numpy as np
import pytest

import synth
from gpu_util import rand_complex
from oracle import c_oracle as co
from oracle import kkr, trsm

pytestmark = pytest.mark.gpu


def _tri(w, upper, seed):
    # off-diagonal entries of 0.1 scale: also with a unit diagonal the triangle stays well
    # conditioned (condition number below 1e4 at w = 50), so the binary64 comparison measures
    # the emulation, not the conditioning
    T = rand_complex(w, w, seed) * 0.1 + np.eye(w) * (2.0 + 1.0j)
    return np.triu(T) if upper else np.tril(T)


def _c_gemm(A, B, S):
    return co.zgemm(A, B, S)


def _c_gemm_lu(C, A, B, S):
    return co.zgemm_lu(C, A, B, S)


@pytest.mark.parametrize("uplo,diag", [("U", "N"), ("L", "U"), ("U", "U"), ("L", "N")])
def test_ztrsm_matches_oracle(ozk_mod, handle, uplo, diag):
    m, n, S = 150, 50, 7                               # blocks 16 + 16 + 16 + 2
    upper, unit = uplo == "U", diag == "U"
    T = _tri(n, upper, 11)
    # the triangle that is not read holds junk, as it does inside an LU-factored block
    T[(np.tril(np.ones((n, n)), -1) if upper else np.triu(np.ones((n, n)), 1)).astype(bool)] = 7.0 - 3.0j
    B = rand_complex(m, n, 12)
    Bd = ozk_mod.colmajor_cuda(B)
    ozk_mod.ozaki_ztrsm(handle, ozk_mod.colmajor_cuda(T), Bd, uplo=uplo, diag=diag, S=S)
    assert handle.status() == 0
    got = ozk_mod.to_numpy(Bd)
    ref = trsm.trsm_right_emulated(T, B, S, upper, unit, gemm=_c_gemm, gemm_lu=_c_gemm_lu)
    # the same blocked algorithm and emulated GEMMs; only the binary64 block inverses differ
    assert kkr.rel_err(got, ref) < 1e-13
    assert kkr.rel_err(got, trsm.trsm_right_fp64(T, B, upper, unit)) < 1e-12


def test_ztrsm_zero_diagonal_sets_singular(ozk_mod, handle):
    n = 20
    T = _tri(n, True, 13)
    T[5, 5] = 0.0
    B = ozk_mod.colmajor_cuda(rand_complex(8, n, 14))
    ozk_mod.ozaki_ztrsm(handle, ozk_mod.colmajor_cuda(T), B, uplo="U", diag="N", S=5)
    assert handle.status() & (1 << 3)


@pytest.mark.parametrize("S,nb", [(7, 64), (5, 48)])
def test_tau00_lu_variant(ozk_mod, handle, S, nb):
    t, G, _ = synth.kkr_system(27, 16, 0.5 + 0.05j, atom=2)
    M = kkr.kkr_build(t, G)
    tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
    ozk_mod.kkr_tau00_lu(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=S, nb=nb)
    assert handle.status() == 0
    got = ozk_mod.to_numpy(tau)
    full = co.tau00_full(M, t[0])
    assert kkr.rel_err(got, full) <= (1e-10 if S == 7 else 1e-7)
    ref = trsm.tau00_lu(M, t[0], nb, S, gemm=_c_gemm, gemm_lu=_c_gemm_lu)
    assert kkr.rel_err(got, ref) < 1e-12
    inv = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
    ozk_mod.kkr_tau00(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), inv, S=S, nb=nb)
    assert kkr.rel_err(got, ozk_mod.to_numpy(inv)) <= (1e-11 if S == 7 else 1e-7)


def test_tau00_lu_variant_pivots(ozk_mod, handle):
    """Pivot blocks dominated by their reversal permutation (zero diagonal): the LU needs an
    interchange at every step; tau_00 still matches the full-inverse oracle."""
    rng = np.random.default_rng(20260403)
    n, b, nb = 160, 16, 48
    M = 0.02 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    for lo, hi in ((0, 16), (16, 64), (64, 112), (112, 160)):
        for r in range(hi - lo):
            M[lo + r, hi - 1 - r] += 1.0
    np.fill_diagonal(M, 0.0)
    t0 = np.eye(b, dtype=np.complex128) * (0.3 + 0.1j)
    tau = ozk_mod.colmajor_cuda(np.zeros((b, b), dtype=np.complex128))
    ozk_mod.kkr_tau00_lu(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t0), tau, S=7, nb=nb)
    assert handle.status() == 0
    assert kkr.rel_err(ozk_mod.to_numpy(tau), co.tau00_full(M, t0)) < 1e-10
