"""Stream capture: the batched KKR step (M = I - tG for every solve, then the lockstep block-LU
tau_00 of all of them) and the emulated ZGEMM replay from one CUDA graph with the very numbers
of the eager calls; sizes first seen during a capture are refused before anything is enqueued."""
import numpy as np
import pytest

import synth
from oracle import kkr

pytestmark = pytest.mark.gpu

B = 16


def _colblocks(t):
    return np.ascontiguousarray(np.transpose(t, (0, 2, 1)))


class _Batch:
    """Device buffers and pointer arrays of a batch of KKR solves with their own t and G."""

    def __init__(self, ozk, sizes, Es):
        import torch
        self.ozk = ozk
        self.sizes = sizes
        self.systems = [synth.kkr_system(L, B, E, atom=i)[:2] for i, (L, E) in enumerate(zip(sizes, Es))]
        dev = torch.device("cuda")
        self.ts = [torch.from_numpy(_colblocks(t)).to(dev) for t, G in self.systems]
        self.Gs = [ozk.colmajor_cuda(G) for t, G in self.systems]
        self.Ms = [torch.empty((L * B, L * B), dtype=torch.complex128, device=dev) for L in sizes]
        # column-major b x b outputs, so that to_numpy reads the logical matrix
        self.taus = [ozk.colmajor_cuda(np.zeros((B, B), dtype=np.complex128)) for _ in sizes]
        p = lambda xs: torch.tensor([x.data_ptr() for x in xs], dtype=torch.int64, device=dev)
        self.pt, self.pg, self.pm, self.ptau = p(self.ts), p(self.Gs), p(self.Ms), p(self.taus)

    def step(self, h, S=7, nb=64):
        self.ozk.kkr_build_m_batched_ptrs(h, self.sizes, B, self.pt, self.pg, self.pm)
        self.ozk.kkr_tau00_batched_ptrs(h, [L * B for L in self.sizes], B, self.pm, self.pt, self.ptau, S=S, nb=nb)

    def results(self):
        return [self.ozk.to_numpy(t) for t in self.taus]


def test_batched_kkr_step_replays_from_one_graph(ozk_mod):
    import torch
    batch = _Batch(ozk_mod, [27, 9, 51, 15], [0.5 + 0.05j, -1.0 + 0.3j, 0.69 + 0.01j, 0.2 + 0.9j])
    h = ozk_mod.Handle()
    batch.step(h)                                  # eager call: sizes the workspace, uploads sizes
    torch.cuda.synchronize()
    assert h.status() == 0
    eager = batch.results()

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        h.set_stream(torch.cuda.current_stream())
        l0 = ozk_mod.launch_count()
        batch.step(h)
        captured = ozk_mod.launch_count() - l0
    h.set_stream(torch.cuda.current_stream())
    assert captured > 10                           # the whole step is in the graph

    for tau in batch.taus:
        tau.fill_(float("nan"))
    for M in batch.Ms:
        M.fill_(float("nan"))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert h.status() == 0
    for got, want in zip(batch.results(), eager):
        assert np.array_equal(got, want)

    # new input values in the same buffers: the replay computes the new solves
    for i, (t, G) in enumerate(batch.systems):
        batch.Gs[i].mul_(0.5)
    g.replay()
    torch.cuda.synchronize()
    for i, (t, G) in enumerate(batch.systems):
        full = kkr.tau00_full(kkr.kkr_build(t, 0.5 * G), t[0])
        assert kkr.rel_err(batch.ozk.to_numpy(batch.taus[i]), full) <= 1e-10
    del g
    h.close()


def test_emulated_zgemm_replays_from_one_graph(ozk_mod):
    import torch
    from gpu_util import rand_complex
    h = ozk_mod.Handle()
    A = ozk_mod.colmajor_cuda(rand_complex(200, 96, 3))
    Bm = ozk_mod.colmajor_cuda(rand_complex(96, 144, 4))
    C = ozk_mod.colmajor_cuda(np.zeros((200, 144), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(h, A, Bm, C, S=6)
    torch.cuda.synchronize()
    eager = ozk_mod.to_numpy(C)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        h.set_stream(torch.cuda.current_stream())
        ozk_mod.ozaki_zgemm(h, A, Bm, C, S=6)
    h.set_stream(torch.cuda.current_stream())
    C.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(ozk_mod.to_numpy(C), eager)
    del g
    h.close()


def test_sizes_first_seen_during_capture_are_refused(ozk_mod):
    import torch
    big = _Batch(ozk_mod, [27, 27], [0.5 + 0.05j, 0.4 + 0.1j])
    small = _Batch(ozk_mod, [15, 9], [0.5 + 0.05j, 0.4 + 0.1j])
    h = ozk_mod.Handle()
    big.step(h)                                    # workspace large enough for `small`
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(ozk_mod.OzkError, match="capture"):
        with torch.cuda.graph(g):
            h.set_stream(torch.cuda.current_stream())
            small.step(h)                          # size lists never seen by this handle
    h.set_stream(torch.cuda.current_stream())
    # a fresh handle has no workspace: growing it during capture is refused as well
    h2 = ozk_mod.Handle()
    g2 = torch.cuda.CUDAGraph()
    ones = np.ones((64, 64), dtype=np.complex128)
    A = ozk_mod.colmajor_cuda(ones)
    C = ozk_mod.colmajor_cuda(np.zeros_like(ones))
    with pytest.raises(ozk_mod.OzkError, match="capture"):
        with torch.cuda.graph(g2):
            h2.set_stream(torch.cuda.current_stream())
            ozk_mod.ozaki_zgemm(h2, A, A, C, S=4)
    h2.set_stream(torch.cuda.current_stream())
    # the handles still work eagerly afterwards
    small.step(h)
    torch.cuda.synchronize()
    assert h.status() == 0
    for i, (t, G) in enumerate(small.systems):
        assert kkr.rel_err(small.results()[i], kkr.tau00_full(kkr.kkr_build(t, G), t[0])) <= 1e-10
    h.close()
    h2.close()
