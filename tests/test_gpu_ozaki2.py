"""GPU parity of the Ozaki-II (CRT) emulated ZGEMM against the oracle (bit-exact: the same
integer images, exact products and one rounding), through the C ABI."""
import numpy as np
import pytest

from gpu_util import op, rand_complex, stored
from oracle import ozaki2 as oz2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [6, 10, 16])
@pytest.mark.parametrize("mnk,ta,tb", [((7, 5, 3), "N", "N"), ((40, 30, 20), "T", "N"), ((129, 65, 33), "N", "C")])
def test_ozaki2_bit_exact(ozk_mod, handle, N, mnk, ta, tb):
    m, n, k = mnk
    A, B = rand_complex(m, k, 3 + N), rand_complex(k, n, 4 + N)
    C = ozk_mod.colmajor_cuda(np.zeros((m, n), dtype=np.complex128))
    ozk_mod.ozaki2_zgemm(handle, ozk_mod.colmajor_cuda(stored(A, ta)), ozk_mod.colmajor_cuda(stored(B, tb)), C,
                         nmod=N, transa=ta, transb=tb)
    assert handle.status() == 0
    assert np.array_equal(ozk_mod.to_numpy(C), oz2.ozaki2_zgemm(A, B, N))


def test_ozaki2_multi_chunk_k(ozk_mod, handle):
    """K' = 2k = 2400 > 1024 terms: several exactness chunks added into the int32 products."""
    m, n, k = 8, 6, 1200
    A, B = rand_complex(m, k, 21, 1.0), rand_complex(k, n, 22, 1.0)
    C = ozk_mod.colmajor_cuda(np.zeros((m, n), dtype=np.complex128))
    ozk_mod.ozaki2_zgemm(handle, ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B), C, nmod=14)
    assert np.array_equal(ozk_mod.to_numpy(C), oz2.ozaki2_zgemm(A, B, 14))


def test_ozaki2_lu_update_and_general(ozk_mod, handle):
    m, n, k = 50, 40, 30
    A, B, C0 = rand_complex(m, k, 31), rand_complex(k, n, 32), rand_complex(m, n, 33)
    Z = oz2.ozaki2_zgemm(A, B, 12)
    C = ozk_mod.colmajor_cuda(C0)
    ozk_mod.ozaki2_zgemm(handle, ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B), C, nmod=12, alpha=-1.0, beta=1.0)
    assert np.array_equal(ozk_mod.to_numpy(C), C0 - Z)                # one binary64 subtraction
    al, be = 0.5 - 1j, 2.0 + 0.25j
    C = ozk_mod.colmajor_cuda(C0)
    ozk_mod.ozaki2_zgemm(handle, ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B), C, nmod=12, alpha=al, beta=be)
    want = al * Z + be * C0
    assert np.abs(ozk_mod.to_numpy(C) - want).max() <= 8 * np.finfo(float).eps * (abs(al) * np.abs(Z) +
                                                                                  abs(be) * np.abs(C0)).max()


def test_ozaki2_error_falls_with_moduli(ozk_mod, handle):
    m = 256
    A, B = rand_complex(m, m, 41, 1.0), rand_complex(m, m, 42, 1.0)
    ref = A @ B
    errs = []
    for N in (8, 10, 12, 14, 16):
        C = ozk_mod.colmajor_cuda(np.zeros((m, m), dtype=np.complex128))
        ozk_mod.ozaki2_zgemm(handle, ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B), C, nmod=N)
        errs.append(np.linalg.norm(ozk_mod.to_numpy(C) - ref) / np.linalg.norm(ref))
    assert all(b < a / 50 or b < 1e-14 for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-14
    with pytest.raises(ozk_mod.OzkError):
        ozk_mod.ozaki2_zgemm(handle, ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B), C, nmod=17)
