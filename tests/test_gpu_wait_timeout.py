"""Failure path of the bounded device waits: a wait that runs out sets OZK_ERR_TIMEOUT in the
status word, the launch returns without writing its output, and the next call on the same
handle is correct.  The wait is made to run out by the library's test hook (a barrier no thread
arrives at, a budget of 1e5 SM cycles, before any copy or MMA is issued): nothing is left in
flight and the GPU is neither hung nor faulted."""
import numpy as np
import pytest

from gpu_util import rand_complex
from oracle import c_oracle as co

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("S", [5, 7, 9])
def test_timed_out_wait_sets_status_and_the_handle_recovers(ozk_mod, S):
    import torch
    h = ozk_mod.Handle()
    A, B = rand_complex(300, 72, 61), rand_complex(72, 150, 62)
    Ad, Bd = ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B)
    C0 = rand_complex(300, 150, 63)
    C = ozk_mod.colmajor_cuda(C0)
    h.debug_stall_next_gemm(100000)
    ozk_mod.ozaki_zgemm(h, Ad, Bd, C, S=S)
    torch.cuda.synchronize()
    st = h.status()
    assert st & (1 << ozk_mod.OZK_ERR_TIMEOUT)
    assert np.array_equal(ozk_mod.to_numpy(C), C0)          # the timed-out launch wrote nothing
    # the next calls on the same handle run normally, bit for bit the oracle
    for _ in range(2):
        ozk_mod.ozaki_zgemm(h, Ad, Bd, C, S=S)
        assert np.array_equal(ozk_mod.to_numpy(C), co.zgemm(A, B, S))
        assert h.status() == 0
    h.close()


def test_stall_request_applies_to_one_launch_only_and_can_be_cleared(ozk_mod):
    h = ozk_mod.Handle()
    A, B = rand_complex(64, 40, 71), rand_complex(40, 48, 72)
    Ad, Bd = ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B)
    C = ozk_mod.colmajor_cuda(np.zeros((64, 48), dtype=np.complex128))
    h.debug_stall_next_gemm(100000)
    h.debug_stall_next_gemm(0)                              # cleared before any launch
    ozk_mod.ozaki_zgemm(h, Ad, Bd, C, S=6)
    assert h.status() == 0
    assert np.array_equal(ozk_mod.to_numpy(C), co.zgemm(A, B, 6))
    h.close()
