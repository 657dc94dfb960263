"""The allocation-free emulated ZGEMM (ozaki_zgemm_noalloc) against the handle-based one.

Callers that cannot allocate device memory when they need a GEMM (for example code running
inside a CUDA graph capture, or inside a framework whose memory pool forbids outside
allocations) use ozaki_zgemm_noalloc, whose scratch is a static array inside the library.
Its results must be the very same numbers as ozaki_zgemm's, call after call, although every
call reuses (and leaves behind) the same scratch contents.  This file is collected last so a
run that stops at the first failure has already run every other test."""
import numpy as np
import pytest

from gpu_util import rand_complex

pytestmark = pytest.mark.gpu


def _call_both(ozk, handle, A, B, C0, S, alpha, beta):
    import torch
    Ad, Bd = ozk.colmajor_cuda(A), ozk.colmajor_cuda(B)
    C1 = ozk.colmajor_cuda(C0)
    C2 = ozk.colmajor_cuda(C0)
    ozk.ozaki_zgemm(handle, Ad, Bd, C1, S=S, alpha=alpha, beta=beta)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ozk.ozaki_zgemm_noalloc(Ad, Bd, C2, S=S, alpha=alpha, beta=beta, device_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return ozk.to_numpy(C1), ozk.to_numpy(C2)


def test_noalloc_matches_handle_path_on_consecutive_calls(ozk_mod, handle):
    # two different problems back to back: the second call runs on scratch the first left behind
    cases = [((300, 170, 90), 7, 1.0, 0.0, 11), ((129, 257, 33), 5, -1.0, 1.0, 12)]
    for (m, n, k), S, alpha, beta, seed in cases:
        A, B, C0 = rand_complex(m, k, seed), rand_complex(k, n, seed + 100), rand_complex(m, n, seed + 200)
        c_handle, c_noalloc = _call_both(ozk_mod, handle, A, B, C0, S, alpha, beta)
        # both paths round the same exact value once: bitwise equal, the tolerance of the
        # store and LU-update epilogue tests
        assert np.array_equal(c_handle, c_noalloc)


def test_noalloc_rejects_problems_beyond_its_scratch(ozk_mod):
    import torch
    big = 4096
    A = torch.zeros((big, big), dtype=torch.complex128, device="cuda").t()   # column major
    C = torch.zeros((big, big), dtype=torch.complex128, device="cuda").t()
    with pytest.raises(ozk_mod.OzkError, match="scratch"):
        ozk_mod.ozaki_zgemm_noalloc(A, A, C, S=7)
