"""GPU parity of the emulated ZGEMM (split, tensor-core group sums, reconstruction) against the
CPU oracle, through the C ABI.  Integer stages are compared bit for bit; the binary64 results
of the store and LU epilogues too (both sides round the same exact value once)."""
import numpy as np
import pytest

import synth
from gpu_util import op, rand_complex, stored
from oracle import c_oracle as co
from oracle import ozaki as oz

pytestmark = pytest.mark.gpu


def _dev(ozk, X):
    return ozk.colmajor_cuda(X)


@pytest.mark.parametrize("S", [1, 3, 7, 8, 10, 16])
@pytest.mark.parametrize("shape", [(1, 1), (33, 17), (130, 70)])
def test_split_left_bit_exact(ozk_mod, handle, S, shape):
    A = rand_complex(*shape, seed=100 + S)
    A[min(2, shape[0] - 1)] = 0.0
    e, d = ozk_mod.ozk_split_debug(handle, _dev(ozk_mod, A), 0, S)
    e_ref, d_ref = oz.split_left(A, S) if S <= 10 else co.split_left(A, S)
    assert np.array_equal(ozk_mod.to_numpy(e).astype(np.int64), e_ref)
    assert np.array_equal(ozk_mod.to_numpy(d).astype(np.int64), d_ref)


@pytest.mark.parametrize("trans", ["N", "T", "C"])
def test_split_right_bit_exact(ozk_mod, handle, trans):
    S = 5
    Bop = rand_complex(29, 41, seed=7)               # op(B) is k x n = 29 x 41
    Bst = stored(Bop, trans)
    e, d = ozk_mod.ozk_split_debug(handle, _dev(ozk_mod, Bst), 1, S, trans)
    f_ref, d_ref = co.split_right(Bop, S)
    assert np.array_equal(ozk_mod.to_numpy(e).astype(np.int64), f_ref)
    assert np.array_equal(ozk_mod.to_numpy(d).astype(np.int64), d_ref)


def test_split_subnormal_and_extreme_rows(ozk_mod, handle):
    A = rand_complex(40, 9, seed=3)
    A[0] = 5e-324
    A[1, 3] = 1e300 + 1e-300j
    A[2] = -np.ldexp(1.0, -1022)
    A[3, :] = np.ldexp(1.0, 7)
    e, d = ozk_mod.ozk_split_debug(handle, _dev(ozk_mod, A), 0, 9)
    e_ref, d_ref = co.split_left(A, 9)
    assert np.array_equal(ozk_mod.to_numpy(e).astype(np.int64), e_ref)
    assert np.array_equal(ozk_mod.to_numpy(d).astype(np.int64), d_ref)


@pytest.mark.parametrize("S,mode", [(1, 0), (4, 0), (5, 0), (7, 0), (8, 0), (9, 0), (12, 0), (3, 1), (5, 1), (8, 1)])
@pytest.mark.parametrize("mnk", [(7, 5, 3), (129, 40, 77), (256, 65, 300)])
def test_group_sums_bit_exact(ozk_mod, handle, S, mode, mnk):
    m, n, k = mnk
    A = rand_complex(m, k, seed=200 + S)
    B = rand_complex(k, n, seed=300 + S)
    G = ozk_mod.to_numpy(ozk_mod.ozk_group_sums_debug(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), S, mode))
    e, DA = co.split_left(A, S)
    f, DB = co.split_right(B, S)
    ref = co.group_sums(DA, DB, S, full=bool(mode))
    for g in sorted(ref):
        assert np.array_equal(G[g - 2], ref[g]), f"group {g}"


def test_group_sums_extreme_digits(ozk_mod, handle):
    """Constant rows: the top group accumulates the largest digit product 2^14 over a full
    exactness chunk, so its FP32 accumulator sits at the 2^24 bound."""
    S, k = 8, 512
    A = np.full((128, k), -0.9999999999999999 - 0.9999999999999999j)
    B = np.full((k, 64), -0.9999999999999999 + 0.9999999999999999j)
    G = ozk_mod.to_numpy(ozk_mod.ozk_group_sums_debug(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), S))
    e, DA = co.split_left(A, S)
    f, DB = co.split_right(B, S)
    ref = co.group_sums(DA, DB, S)
    for g in sorted(ref):
        assert np.array_equal(G[g - 2], ref[g])


@pytest.mark.parametrize("S", [5, 7])
@pytest.mark.parametrize("k", [64, 128, 200])
def test_fixed_slice_count_split_bit_exact(ozk_mod, handle, S, k):
    """S = 5 and S = 7 split with compile-time slice counts (every digit one byte of the
    biased integer image, turned into binary16 by a packed subtraction): the product of
    operands whose rows hold the extreme digits (top digit 128 from 1 - 2^-53 at the row
    maximum, alternating signs, zeros of both signs, subnormals next to normal values) is
    bit-exact against the oracle; K a multiple of 8 so that every run is 8 wide, and a ragged
    last tile at k = 200."""
    rng = np.random.default_rng(100 + S + k)
    m, n = 96, 80
    big = 0.9999999999999999
    A = rand_complex(m, k, seed=31 + S)
    B = rand_complex(k, n, seed=32 + S)
    A[0, :] = big - big * 1j
    A[1, :] = 0.0
    A[1, ::2] = -0.0 + 0.0j
    A[2, :] = 5e-324 * (1 + 1j)
    A[2, 5] = big + 0j
    A[3, :] = big * np.where(np.arange(k) % 2, 1.0, -1.0) * (1 - 1j)
    A[4, :] = rng.integers(-3, 4, k) * 2.0 ** -20 + 1j * rng.integers(-3, 4, k)
    B[:, 0] = -big + big * 1j
    B[:, 1] = 0.0
    B[:, 2] = np.ldexp(1.0, -1022) * (1 - 1j)
    B[7, 2] = -big * 1j
    B[:, 3] = big * np.where(np.arange(k) % 3, -1.0, 1.0) * (1 + 1j)
    C = ozk_mod.colmajor_cuda(np.zeros((m, n), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S)
    assert np.array_equal(ozk_mod.to_numpy(C), co.zgemm(A, B, S))
    assert handle.status() == 0


@pytest.mark.parametrize("S", [3, 5, 7, 9])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "C"), ("C", "T")])
def test_zgemm_store_bit_exact(ozk_mod, handle, S, ta, tb):
    m, n, k = 150, 70, 45
    Aop = rand_complex(m, k, seed=11 + S)
    Bop = rand_complex(k, n, seed=12 + S)
    A, B = _dev(ozk_mod, stored(Aop, ta)), _dev(ozk_mod, stored(Bop, tb))
    import torch
    C = ozk_mod.colmajor_cuda(np.zeros((m, n), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, A, B, C, S=S, transa=ta, transb=tb)
    ref = co.zgemm(Aop, Bop, S)
    assert np.array_equal(ozk_mod.to_numpy(C), ref)
    assert handle.status() == 0


def test_zgemm_lu_update_bit_exact(ozk_mod, handle):
    m, n, k, S = 300, 200, 16, 7
    A, B, C0 = rand_complex(m, k, 1), rand_complex(k, n, 2), rand_complex(m, n, 3)
    C = _dev(ozk_mod, C0)
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S, alpha=-1.0, beta=1.0)
    assert np.array_equal(ozk_mod.to_numpy(C), co.zgemm_lu(C0, A, B, S))


@pytest.mark.parametrize("S", [2, 4, 5])
@pytest.mark.parametrize("k", [16, 64, 112])
def test_zgemm_lu_update_64bit_sums_bit_exact(ozk_mod, handle, S, k):
    """S <= 5 and one exactness chunk: every exact sum fits in 64 bits and the epilogue rounds
    it from one int64 per output; the result equals the oracle's bit for bit."""
    m, n = 200, 150
    A, B, C0 = rand_complex(m, k, 51 + S), rand_complex(k, n, 52 + k), rand_complex(m, n, 53)
    C = _dev(ozk_mod, C0)
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S, alpha=-1.0, beta=1.0)
    assert np.array_equal(ozk_mod.to_numpy(C), co.zgemm_lu(C0, A, B, S))


@pytest.mark.parametrize("S,k", [(5, 64), (7, 64), (7, 112), (9, 40)])
def test_lu_update_subtraction_edge_cases(ozk_mod, handle, S, k):
    """C - RN(Z) with C built around the rounded product Z itself: C = Z (exact cancellation to
    +0), C = -Z (doubling), Z one or two ulps away (massive cancellation), C = +-0, C far above
    and far below Z (the aligned operand only a sticky bit), C of the same and of the opposite
    sign with half-ulp distances (ties of the subtraction's rounding), subnormal and infinite C.
    The epilogue's integer subtraction matches the binary64 subtraction of the oracle bit for
    bit (the rare operands take the binary64 path)."""
    m, n = 131, 77
    A, B = rand_complex(m, k, 81 + S), rand_complex(k, n, 82 + k)
    Z = co.zgemm(A, B, S)
    rng = np.random.default_rng(2026 + S)
    kind = rng.integers(0, 12, size=(m, n))
    re, im = Z.real.copy(), Z.imag.copy()

    def craft(z, kd):
        out = z.copy()
        out[kd == 0] = z[kd == 0]
        out[kd == 1] = -z[kd == 1]
        out[kd == 2] = np.nextafter(z[kd == 2], np.inf)
        out[kd == 3] = np.nextafter(np.nextafter(z[kd == 3], -np.inf), -np.inf)
        out[kd == 4] = 0.0
        out[kd == 5] = -0.0
        out[kd == 6] = z[kd == 6] * 2.0 ** 70
        out[kd == 7] = z[kd == 7] * 2.0 ** -70
        out[kd == 8] = z[kd == 8] * (1 + 2.0 ** -52) * 0.5
        out[kd == 9] = -z[kd == 9] * 3.0 * 2.0 ** -54
        out[kd == 10] = 5e-324 * (1 + (np.arange((kd == 10).sum()) % 7))
        out[kd == 11] = z[kd == 11] * 1.5
        return out

    C0 = craft(re, kind) + 1j * craft(im, (kind + 3) % 12)
    C0[0, 0] = complex(np.inf, 1.0)
    C = _dev(ozk_mod, C0)
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S, alpha=-1.0, beta=1.0)
    got, want = ozk_mod.to_numpy(C), co.zgemm_lu(C0, A, B, S)
    eq = (got.real.view(np.int64) == want.real.view(np.int64)) & (got.imag.view(np.int64) == want.imag.view(np.int64))
    assert eq.all(), np.argwhere(~eq)[:5]


def test_zgemm_64bit_sums_large_group_values(ozk_mod, handle):
    """Rows and columns of (127/255)(1 + i), whose five balanced digits are all 127: the
    five-pair group sums of the imaginary parts reach 128 * 5 * 127^2 ~ 2^23.3, past the range
    of the one-add FP32 conversion, so those warps take the hardware conversion; the other
    rows are random.  Bitwise equal to the oracle."""
    S, m, n, k = 5, 160, 48, 64
    A, B, C0 = rand_complex(m, k, 71), rand_complex(k, n, 72), rand_complex(m, n, 73)
    A[:40] = (127 / 255) * (1 + 1j)
    B[:, :20] = (127 / 255) * (1 + 1j)
    C = _dev(ozk_mod, C0)
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S, alpha=-1.0, beta=1.0)
    assert np.array_equal(ozk_mod.to_numpy(C), co.zgemm_lu(C0, A, B, S))


def test_zgemm_64bit_sums_subnormal_and_overflowing_results(ozk_mod, handle):
    """Rows and columns scaled so that products land in the subnormal range, below it, and
    past the largest binary64: the 64-bit epilogue hands those to the general rounding and
    matches the oracle bit for bit (subnormals, zeros, infinities)."""
    S = 5
    A, B = rand_complex(40, 20, 61), rand_complex(20, 24, 62)
    A[0] *= 2.0 ** -1000
    A[1] *= 2.0 ** -1030
    B[:, 0] *= 2.0 ** -60
    A[2] *= 2.0 ** 600
    B[:, 1] *= 2.0 ** 500
    C = _dev(ozk_mod, np.zeros((40, 24), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S)
    ref = co.zgemm(A, B, S)
    got = ozk_mod.to_numpy(C)
    assert np.isinf(ref).any() and (np.abs(ref[ref != 0]) < 2.2250738585072014e-308).any()
    assert np.array_equal(got, ref)


def test_zgemm_full_pairs_bit_exact(ozk_mod, handle):
    m, n, k, S = 70, 33, 20, 4
    A, B = rand_complex(m, k, 41), rand_complex(k, n, 42)
    C = _dev(ozk_mod, np.zeros((m, n), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S, pair_mode=ozk_mod.OZK_PAIRS_FULL)
    assert np.array_equal(ozk_mod.to_numpy(C), co.zgemm(A, B, S, full=True))


def test_zgemm_general_alpha_beta(ozk_mod, handle):
    m, n, k, S = 90, 50, 30, 7
    A, B, C0 = rand_complex(m, k, 5), rand_complex(k, n, 6), rand_complex(m, n, 7)
    al, be = 0.75 - 0.5j, -1.25 + 0.25j
    C = _dev(ozk_mod, C0)
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S, alpha=al, beta=be)
    Z = co.zgemm(A, B, S)
    ref = al * Z + be * C0
    got = ozk_mod.to_numpy(C)
    # binary64 complex arithmetic in a different operation order: a few ulps of |terms|
    scale = np.abs(al) * np.abs(Z) + np.abs(be) * np.abs(C0)
    assert np.all(np.abs(got - ref) <= 8 * np.finfo(float).eps * scale)


def test_config1_full_size_bit_exact_and_error(ozk_mod, handle):
    """512^3 complex, S = 7 (the single-GEMM workload): bitwise equal to the oracle,
    relative Frobenius error vs binary64 <= 1e-13."""
    A, B = synth.zgemm_operands(512, 512, 512)
    C = _dev(ozk_mod, np.zeros((512, 512), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=7)
    got = ozk_mod.to_numpy(C)
    ref = co.zgemm(A, B, 7)
    assert np.array_equal(got, ref)
    X = co.zgemm_fp64(A, B)
    assert np.linalg.norm(got - X) / np.linalg.norm(X) <= 1e-13


def test_split_k_store_lu_and_general(ozk_mod, handle):
    """A product with few tiles and a long K (m = 200, n = 100, k = 800: 8 tiles, 12 exactness
    chunks at S = 7) runs split K: 8 units per tile add their exact partial sums, rounded once by
    the finishing kernel.  Store (transposed operands), LU update and general alpha, beta equal
    the single-unit results (the oracle's) bit for bit, resp. within the binary64 bound of the
    general combination."""
    m, n, k, S = 200, 100, 800, 7
    Aop, Bop, C0 = rand_complex(m, k, 501), rand_complex(k, n, 502), rand_complex(m, n, 503)
    Z = co.zgemm(Aop, Bop, S)
    C = _dev(ozk_mod, np.zeros((m, n), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, stored(Aop, "T")), _dev(ozk_mod, stored(Bop, "C")), C, S=S,
                        transa="T", transb="C")
    assert np.array_equal(ozk_mod.to_numpy(C), Z)
    C = _dev(ozk_mod, C0)
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, Aop), _dev(ozk_mod, Bop), C, S=S, alpha=-1.0, beta=1.0)
    assert np.array_equal(ozk_mod.to_numpy(C), C0 - Z)
    al, be = 0.75 - 0.5j, -1.25 + 2j
    C = _dev(ozk_mod, C0)
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, Aop), _dev(ozk_mod, Bop), C, S=S, alpha=al, beta=be)
    got = ozk_mod.to_numpy(C)
    scale = np.abs(al) * np.abs(Z) + np.abs(be) * np.abs(C0)
    assert np.all(np.abs(got - (al * Z + be * C0)) <= 8 * np.finfo(float).eps * scale)
    assert handle.status() == 0


@pytest.mark.parametrize("S", [3, 5, 7, 10])
def test_large_k_multi_chunk(ozk_mod, handle, S):
    """K' = 5000 spans several exactness chunks: the 128-bit multi-chunk epilogue (at S = 5 in
    the compile-time S = 5 kernel instance)."""
    m, n, k = 64, 16, 2500
    A, B = rand_complex(m, k, 70), rand_complex(k, n, 71)
    C = _dev(ozk_mod, np.zeros((m, n), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S)
    assert np.array_equal(ozk_mod.to_numpy(C), co.zgemm(A, B, S))


@pytest.mark.parametrize("k,lu", [(192, True), (500, False), (1100, True)])
def test_multi_chunk_many_tiles_sampled(ozk_mod, handle, k, lu):
    """S = 7 (the compile-time instance) with 3, 7 and 16 exactness chunks (K' = 2k) over 512
    tiles, several per persistent CTA, so the accumulator hand-offs run across tiles and chunks:
    each output is still the exact sum rounded once.  Row i of op(A) and column j of op(B) fix
    their own exponents, so the oracle's product of sampled rows and columns is the same block
    of the full product, bit for bit (store and LU update)."""
    m, n, S = 2048, 1024, 7
    A, B = rand_complex(m, k, 300 + k), rand_complex(k, n, 301 + k)
    C0 = rand_complex(m, n, 302) if lu else np.zeros((m, n), dtype=np.complex128)
    C = _dev(ozk_mod, C0)
    if lu:
        ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S, alpha=-1.0, beta=1.0)
    else:
        ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=S)
    got = ozk_mod.to_numpy(C)
    assert handle.status() == 0
    rng = np.random.default_rng(k)
    rows = np.sort(rng.choice(m, 48, replace=False))
    cols = np.sort(rng.choice(n, 40, replace=False))
    rows[0], cols[-1] = 0, n - 1                      # the first row tile and the last column tile
    Z = co.zgemm(A[rows], B[:, cols], S)
    want = C0[np.ix_(rows, cols)] - Z if lu else Z
    assert np.array_equal(got[np.ix_(rows, cols)], want)


def test_vbatched_matches_single(ozk_mod, handle):
    shapes = [(40, 30, 20), (129, 64, 16), (7, 3, 20), (200, 100, 5)]
    As, Bs, Cs, refs = [], [], [], []
    for i, (m, n, k) in enumerate(shapes):
        A, B = rand_complex(m, k, 80 + i), rand_complex(k, n, 90 + i)
        As.append(_dev(ozk_mod, A)); Bs.append(_dev(ozk_mod, B))
        Cs.append(_dev(ozk_mod, np.zeros((m, n), dtype=np.complex128)))
        refs.append(co.zgemm(A, B, 6))
    ozk_mod.ozaki_zgemm_vbatched(handle, As, Bs, Cs, S=6)
    for C, r in zip(Cs, refs):
        assert np.array_equal(ozk_mod.to_numpy(C), r)


def test_dmma_within_binary64_bound(ozk_mod, handle):
    m, n, k = 257, 130, 300
    A, B = rand_complex(m, k, 13), rand_complex(k, n, 14)
    C = _dev(ozk_mod, np.zeros((m, n), dtype=np.complex128))
    ozk_mod.ozk_zgemm_dmma(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C)
    got = ozk_mod.to_numpy(C)
    X = co.zgemm_fp64(A, B)
    gamma = 2 * k * np.finfo(float).eps
    assert np.all(np.abs(got - X) <= 2 * gamma * (np.abs(A) @ np.abs(B)))


def test_negative_S_is_the_dmma_gemm(ozk_mod, handle):
    """One slice-count rule across the ABI: S < 0 runs the binary64 DMMA GEMM, in the single
    call (bit for bit ozk_zgemm_dmma) and in the variable-size batch."""
    A, B = rand_complex(70, 33, 21), rand_complex(33, 45, 22)
    C0 = rand_complex(70, 45, 23)
    C1, C2 = _dev(ozk_mod, C0), _dev(ozk_mod, C0)
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C1, S=-1, alpha=-1.0, beta=1.0)
    ozk_mod.ozk_zgemm_dmma(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C2, alpha=-1.0, beta=1.0)
    assert np.array_equal(ozk_mod.to_numpy(C1), ozk_mod.to_numpy(C2))
    shapes = [(17, 9, 30), (40, 21, 5), (3, 64, 64)]
    As = [_dev(ozk_mod, rand_complex(m, k, 30 + i)) for i, (m, n, k) in enumerate(shapes)]
    Bs = [_dev(ozk_mod, rand_complex(k, n, 40 + i)) for i, (m, n, k) in enumerate(shapes)]
    Cs = [_dev(ozk_mod, np.zeros((m, n), dtype=np.complex128)) for m, n, k in shapes]
    ozk_mod.ozaki_zgemm_vbatched(handle, As, Bs, Cs, S=-1)
    for a, b, c in zip(As, Bs, Cs):
        want = _dev(ozk_mod, np.zeros(tuple(c.shape), dtype=np.complex128))
        ozk_mod.ozk_zgemm_dmma(handle, a, b, want)
        assert np.array_equal(ozk_mod.to_numpy(c), ozk_mod.to_numpy(want))
    assert handle.status() == 0


def test_degenerate_calls(ozk_mod, handle):
    import torch
    A = _dev(ozk_mod, rand_complex(5, 4, 1))
    B = _dev(ozk_mod, rand_complex(4, 3, 2))
    C0 = rand_complex(5, 3, 3)
    C = _dev(ozk_mod, C0)
    # alpha = 0: C = beta C
    ozk_mod.ozaki_zgemm(handle, A, B, C, S=4, alpha=0.0, beta=2.0)
    assert np.array_equal(ozk_mod.to_numpy(C), 2.0 * C0)
    # S = 0 is the slice-count selector (tests/test_gpu_selector.py), S < 0 the binary64 DMMA
    # GEMM (test_negative_S_is_the_dmma_gemm); above 16 is invalid
    with pytest.raises(ozk_mod.OzkError):
        ozk_mod.ozaki_zgemm(handle, A, B, C, S=17)


def test_k_parallel_split_matches_row_parallel_split(ozk_mod, handle):
    """Operands with few row blocks and long rows take the K-parallel split (row maxima by a
    pre-pass over K segments, each row block's K tiles shared among CTAs); the same rows inside
    a tall operand take the one-CTA-per-row-block split.  Each output row depends only on its own
    row and B, so both give the same bits, non-finite entries included (flagged, split as zero,
    their row's exponent 0)."""
    m, n, k, S = 40, 12, 700, 7
    A, B = rand_complex(m, k, 611), rand_complex(k, n, 612)
    A[5, 600] = np.nan
    A[30, 10] = np.inf
    small = _dev(ozk_mod, np.zeros((m, n), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), small, S=S)
    assert handle.status() & (1 << 2)
    tall_A = np.vstack([A, rand_complex(6000 - m, k, 613)])
    tall = _dev(ozk_mod, np.zeros((6000, n), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, tall_A), _dev(ozk_mod, B), tall, S=S)
    assert handle.status() & (1 << 2)
    got, want = ozk_mod.to_numpy(small), ozk_mod.to_numpy(tall)[:m]
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(np.nan_to_num(got), np.nan_to_num(want))
    keep = [i for i in range(m) if i not in (5, 30)]
    assert np.array_equal(got[keep], co.zgemm(A[keep], B, S))


@pytest.mark.parametrize("S,ta,tb", [(7, "N", "N"), (7, "C", "T"), (5, "T", "C")])
def test_many_row_blocks_split_bit_exact_on_sampled_rows(ozk_mod, handle, S, ta, tb):
    """Operands of one K tile and thousands of row blocks (the split's one-tile path at full
    occupancy): a 49152 x 64 x 64 product (left operand) and a 64 x 49152 x 64 product (right
    operand), stored transposed or conjugated, bit-exact against the oracle on sampled rows
    (columns), which the oracle computes from those rows (columns) alone."""
    import torch
    k, big = 64, 49152
    rng = np.random.default_rng(7 + S)
    for m, n in ((big, 64), (64, big)):
        Aop = rand_complex(m, k, seed=51 + S)
        Bop = rand_complex(k, n, seed=52 + S)
        Aop[5, :] = 0.9999999999999999 * (1 - 1j)            # top digits 128
        Bop[:, 6] = -0.9999999999999999 + 0.5j
        C = ozk_mod.colmajor_cuda(np.zeros((m, n), dtype=np.complex128))
        ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, stored(Aop, ta)), _dev(ozk_mod, stored(Bop, tb)), C, S=S,
                            transa=ta, transb=tb)
        assert handle.status() == 0
        got = ozk_mod.to_numpy(C)
        if m == big:
            rows = np.concatenate([[0, 5, 31, 32, m - 1], rng.choice(m, 250, replace=False)])
            assert np.array_equal(got[rows], co.zgemm(np.ascontiguousarray(Aop[rows]), Bop, S))
        else:
            cols = np.concatenate([[0, 6, 31, 32, n - 1], rng.choice(n, 250, replace=False)])
            assert np.array_equal(got[:, cols], co.zgemm(Aop, np.ascontiguousarray(Bop[:, cols]), S))
        del C
        torch.cuda.empty_cache()


def test_nonfinite_input_in_a_large_operand_sets_status(ozk_mod, handle):
    """A NaN in one row of a 49152-row operand sets the status."""
    A = rand_complex(49152, 64, 3)
    A[40000, 17] = np.nan
    B = rand_complex(64, 16, 4)
    C = _dev(ozk_mod, np.zeros((49152, 16), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=7)
    assert handle.status() & (1 << 2)
    assert handle.status() == 0


def test_nonfinite_input_sets_status(ozk_mod, handle):
    A = rand_complex(20, 8, 1)
    A[4, 2] = np.nan
    B = rand_complex(8, 6, 2)
    C = _dev(ozk_mod, np.zeros((20, 6), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, _dev(ozk_mod, A), _dev(ozk_mod, B), C, S=5)
    assert handle.status() & (1 << 2)
    assert handle.status() == 0          # cleared after reading
