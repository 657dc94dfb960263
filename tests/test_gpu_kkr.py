"""GPU parity of the KKR tau_00 path (M build, pivot-block inverses, block LU with every GEMM
emulated, batched lockstep solves) against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import c_oracle as co
from oracle import kkr

pytestmark = pytest.mark.gpu


def _system(L, E=0.5 + 0.05j, b=16, atom=0):
    t, G, pos = synth.kkr_system(L, b, E, atom=atom)
    return t, G, kkr.kkr_build(t, G)


def _tblocks(ozk, t):
    import torch
    # L x b x b with column-major blocks: store the transpose of each block row-major
    return torch.from_numpy(np.ascontiguousarray(np.transpose(t, (0, 2, 1)))).to("cuda")


def test_build_m(ozk_mod, handle):
    t, G, M = _system(15)
    Md = ozk_mod.colmajor_cuda(np.zeros_like(M))
    ozk_mod.kkr_build_m(handle, _tblocks(ozk_mod, t), ozk_mod.colmajor_cuda(G), Md)
    got = ozk_mod.to_numpy(Md)
    assert np.abs(got - M).max() <= 32 * np.finfo(float).eps


@pytest.mark.parametrize("S,nb", [(-1, 16), (-1, 32), (5, 16), (5, 64), (7, 48), (7, 64)])
def test_tau00_small_vs_oracles(ozk_mod, handle, S, nb):
    t, G, M = _system(15)
    tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
    ozk_mod.kkr_tau00(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=S, nb=nb)
    assert handle.status() == 0
    got = ozk_mod.to_numpy(tau)
    full = kkr.tau00_full(M, t[0])
    # the oracle's restatement of the same algorithm: one pivot block per panel
    if S < 0:
        assert kkr.rel_err(got, full) < 1e-13
    else:
        # same algorithm and the same emulated GEMMs: only the binary64 pivot inverses differ
        assert kkr.rel_err(got, co.tau00_block(M, t[0], nb, S=S)) < 1e-13
        assert kkr.rel_err(got, full) <= (1e-10 if S >= 7 else 1e-6)


def test_tau00_config2_single_atom(ozk_mod, handle):
    """bcc LIZ 65, b = 16, n = 1040, E = 0.5 + 0.05i, S = 7: within 1e-10 of the binary64
    full-inverse oracle; the error falls with S."""
    t, G, M = _system(65)
    full = co.tau00_full(M, t[0])
    errs = {}
    for S in (3, 5, 7, 9):
        tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
        ozk_mod.kkr_tau00(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=S, nb=64)
        errs[S] = kkr.rel_err(ozk_mod.to_numpy(tau), full)
    assert handle.status() == 0
    assert errs[7] <= 1e-10 and errs[9] <= 1e-12
    assert errs[3] > errs[5] > errs[7]


def test_tau00_wider_panels(ozk_mod, handle):
    t, G, M = _system(27)
    full = kkr.tau00_full(M, t[0])
    for nb in (32, 48, 96, 112):
        tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
        ozk_mod.kkr_tau00(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=7, nb=nb)
        assert kkr.rel_err(ozk_mod.to_numpy(tau), full) <= 1e-10


@pytest.mark.parametrize("S", [7, 9])
def test_batched_equals_single(ozk_mod, handle, S):
    """Batched lockstep solves equal single solves bit for bit; S = 9 takes the 128-bit integer
    images and the 128-bit reconstruction."""
    sizes = [27, 9, 51, 15, 2]
    Es = [0.5 + 0.05j, -1.0 + 0.3j, 0.69 + 0.01j, 0.2 + 0.9j, 0.6 + 0.2j]
    systems = [_system(L, E, atom=i) for i, (L, E) in enumerate(zip(sizes, Es))]
    single = []
    for t, G, M in systems:
        tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
        ozk_mod.kkr_tau00(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=S, nb=64)
        single.append(ozk_mod.to_numpy(tau))
    Ms = [ozk_mod.colmajor_cuda(M) for t, G, M in systems]
    t0s = [ozk_mod.colmajor_cuda(t[0]) for t, G, M in systems]
    taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128)) for _ in systems]
    ozk_mod.kkr_tau00_batched(handle, Ms, t0s, taus, S=S, nb=64)
    assert handle.status() == 0
    for i, (t, G, M) in enumerate(systems):
        got = ozk_mod.to_numpy(taus[i])
        assert np.array_equal(got, single[i])
        assert kkr.rel_err(got, co.tau00_full(M, t[0])) <= 1e-10


@pytest.mark.parametrize("S,W,w", [(7, 128, 48), (7, 96, 32), (5, 192, 64), (9, 64, 32)])
def test_batched_leaf_panels_vs_oracle(ozk_mod, handle, S, W, w):
    """Panels of width W eliminated leaf by leaf (w-wide pivot blocks from the panel's end, a
    ragged front leaf where w does not divide the panel, the frame of each leaf updated by a
    GEMM with a skip box, one deferred K = W update per panel), mixed sizes in one batched call:
    tau_00 against the oracle's leaf-wise block LU of the same M (only the binary64 pivot
    inverses round differently) and within 1e-10 of the binary64 full inverse (S >= 7)."""
    sizes = [27, 9, 15, 2, 20]
    Es = [0.5 + 0.05j, -1.0 + 0.3j, 0.69 + 0.01j, 0.2 + 0.9j, 0.6 + 0.2j]
    systems = [_system(L, E, atom=i) for i, (L, E) in enumerate(zip(sizes, Es))]
    Ms = [ozk_mod.colmajor_cuda(M) for t, G, M in systems]
    t0s = [ozk_mod.colmajor_cuda(t[0]) for t, G, M in systems]
    taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128)) for _ in systems]
    ozk_mod.kkr_tau00_batched(handle, Ms, t0s, taus, S=S, nb=W, leaf=w)
    assert handle.status() == 0
    for i, (t, G, M) in enumerate(systems):
        got = ozk_mod.to_numpy(taus[i])
        assert kkr.rel_err(got, co.tau00_block(M, t[0], W, S=S, leaf=w)) < 1e-13, i
        if S >= 7:
            assert kkr.rel_err(got, co.tau00_full(M, t[0])) <= 1e-10, i


def test_pivot_inverse_forms_agree_across_batch_sizes(ozk_mod, handle):
    """Pivot blocks of order <= 64 are inverted with the block in registers when a launch has
    at most one block per SM and in shared memory otherwise: the same solves in a batch larger
    than the SM count and in a small batch agree to binary64 rounding, and both match the
    oracle's leaf-wise block LU of the same M."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    sizes = [9, 14, 5, 11]
    systems = [_system(L, 0.45 + 0.07j * (i + 1), atom=i) for i, L in enumerate(sizes)]

    def run(reps):
        Ms = [ozk_mod.colmajor_cuda(systems[i % len(systems)][2]) for i in range(reps)]
        t0s = [ozk_mod.colmajor_cuda(systems[i % len(systems)][0][0]) for i in range(reps)]
        taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128)) for _ in range(reps)]
        ozk_mod.kkr_tau00_batched(handle, Ms, t0s, taus, S=7, nb=128, leaf=64)
        assert handle.status() == 0
        return [ozk_mod.to_numpy(x) for x in taus]

    small = run(len(systems))
    large = run(nsm + 8)
    for i, (t, G, M) in enumerate(systems):
        want = co.tau00_block(M, t[0], 128, S=7, leaf=64)
        assert kkr.rel_err(small[i], want) < 1e-13, i
        for r in range(i, nsm + 8, len(systems)):
            assert kkr.rel_err(large[r], small[i]) < 1e-13, (i, r)


def test_one_leaf_panels_equal_the_plain_batched_solve(ozk_mod, handle):
    """w = W is the plain panel-by-panel block LU: bit for bit kkr_tau00_batched with nb = W."""
    sizes = [27, 15, 9]
    systems = [_system(L, 0.4 + 0.1j, atom=i) for i, L in enumerate(sizes)]

    def run(**kw):
        Ms = [ozk_mod.colmajor_cuda(M) for t, G, M in systems]
        t0s = [ozk_mod.colmajor_cuda(t[0]) for t, G, M in systems]
        taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128)) for _ in systems]
        ozk_mod.kkr_tau00_batched(handle, Ms, t0s, taus, S=7, **kw)
        return [ozk_mod.to_numpy(x) for x in taus]

    for a, b_ in zip(run(nb=64), run(nb=64, leaf=64)):
        assert np.array_equal(a, b_)
    assert handle.status() == 0


def test_panel_autotuner_caches_a_pair(ozk_mod):
    """kkr_tau00_autotune_panels times whole-panel and leaf-wise candidates and caches the
    smallest (W, w) within 1 % of the fastest; nb = 0 then runs exactly that pair (bitwise)."""
    import torch
    h = ozk_mod.Handle()
    sizes = [27, 15, 27]
    systems = [_system(L, 0.5 + 0.05j, atom=i) for i, L in enumerate(sizes)]
    (W, w), times = ozk_mod.kkr_tau00_autotune_panels(h, [L * 16 for L in sizes], 16, S=7)
    # the smallest pair (by W, then w) within 1 % of the fastest
    lim = np.float32(1.01) * np.float32(min(times.values()))    # as the library compares
    near = [c for c, v in times.items() if np.float32(v) <= lim]
    assert (W, w) in times and (W, w) == min(near)
    assert (64, 64) in times and (128, 64) in times and (288, 96) in times

    def run(**kw):
        Ms = [ozk_mod.colmajor_cuda(M) for t, G, M in systems]
        t0s = [ozk_mod.colmajor_cuda(t[0]) for t, G, M in systems]
        taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128)) for _ in systems]
        ozk_mod.kkr_tau00_batched(h, Ms, t0s, taus, S=7, **kw)
        torch.cuda.synchronize()
        return [ozk_mod.to_numpy(x) for x in taus]

    for a, f in zip(run(nb=0), run(nb=W, leaf=w)):
        assert np.array_equal(a, f)
    assert h.status() == 0
    h.close()


def test_singular_pivot_sets_status(ozk_mod, handle):
    M = np.eye(32, dtype=np.complex128)
    M[16:, 16:] = 0.0                    # the first eliminated pivot block is exactly singular
    t0 = np.eye(16, dtype=np.complex128)
    tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
    ozk_mod.kkr_tau00(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t0), tau, S=5, nb=64)
    assert handle.status() & (1 << 3)


@pytest.mark.parametrize("S", [-1, 7])
@pytest.mark.parametrize("nb", [48, 64, 80])
def test_pivot_blocks_need_row_interchanges(ozk_mod, handle, S, nb):
    """Pivot blocks whose diagonal is zero (every panel's leading element needs a row
    interchange): the in-place Gauss-Jordan inverse with partial pivoting still gives tau_00
    of the full-inverse oracle.  Pivot blocks of order <= 64 are inverted with the block in
    registers, wider ones in shared memory."""
    rng = np.random.default_rng(20260403)
    b = 16
    n = b + 3 * nb
    M = 0.02 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    # every block of the elimination (centre [0, 16) and three panels of nb) dominated by its
    # reversal permutation, with a zero diagonal
    for lo, hi in ((0, b), (b, b + nb), (b + nb, b + 2 * nb), (b + 2 * nb, n)):
        for r in range(hi - lo):
            M[lo + r, hi - 1 - r] += 1.0
    np.fill_diagonal(M, 0.0)
    t0 = np.eye(b, dtype=np.complex128) * (0.3 + 0.1j)
    tau = ozk_mod.colmajor_cuda(np.zeros((b, b), dtype=np.complex128))
    ozk_mod.kkr_tau00(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t0), tau, S=S, nb=nb)
    assert handle.status() == 0
    got = ozk_mod.to_numpy(tau)
    full = co.tau00_full(M, t0)
    assert kkr.rel_err(got, full) < (1e-12 if S < 0 else 1e-10)
    if S > 0:
        assert kkr.rel_err(got, co.tau00_block(M, t0, nb, S=S)) < 1e-12


@pytest.mark.parametrize("S", [5, 7])
def test_build_m_shared_is_the_emulated_block_row_update(ozk_mod, handle, S):
    """Atoms sharing G: block row i of M_a is (rows ib..ib+b-1 of I) - RN(t_{a,i} G_i) with the
    emulated product, bit for bit, and close to the binary64 M = I - t G."""
    import torch
    L, b, natoms = 9, 16, 5
    n = L * b
    _, G, _ = synth.kkr_system(L, b, 0.3 + 0.2j, atom=0)
    ts = [synth.kkr_t(L, b, atom=a) for a in range(natoms)]
    tdev = [_tblocks(ozk_mod, t) for t in ts]
    Ms = [ozk_mod.colmajor_cuda(np.zeros((n, n), dtype=np.complex128)) for _ in range(natoms)]
    ptr = lambda xs: torch.tensor([x.data_ptr() for x in xs], dtype=torch.int64, device="cuda")
    ozk_mod.kkr_build_m_shared_ptrs(handle, natoms, L, b, ptr(tdev), ozk_mod.colmajor_cuda(G), ptr(Ms), S=S)
    assert handle.status() == 0
    eye = np.eye(n, dtype=np.complex128)
    for a in range(natoms):
        got = ozk_mod.to_numpy(Ms[a])
        for i in range(L):
            rows = slice(i * b, (i + 1) * b)
            want = co.zgemm_lu(eye[rows], ts[a][i], G[rows], S)
            assert np.array_equal(got[rows], want)
        err = np.abs(got - kkr.kkr_build(ts[a], G)).max()
        assert err <= (1e-14 if S == 7 else 1e-9)


@pytest.mark.parametrize("S,nb", [(7, 50), (7, 100), (-1, 50)])
def test_tau00_lmax4_spin_blocks(ozk_mod, handle, S, nb):
    """b = 50 (lmax = 4 with spin): pivot blocks of order 50 and 100 (in-place Gauss-Jordan
    inverses), panel GEMMs with k = 50 or 100 (K' = 100, not a multiple of 16), and the
    256-thread Gauss-Jordan solve of the 50 x 50 centre block."""
    L, b = 9, 50
    t, G, _ = synth.kkr_system(L, b, 0.4 + 0.1j, atom=3)
    M = kkr.kkr_build(t, G)
    tau = ozk_mod.colmajor_cuda(np.zeros((b, b), dtype=np.complex128))
    ozk_mod.kkr_tau00(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=S, nb=nb)
    assert handle.status() == 0
    got = ozk_mod.to_numpy(tau)
    full = co.tau00_full(M, t[0])
    if S > 0:
        assert kkr.rel_err(got, co.tau00_block(M, t[0], nb, S=S)) < 1e-13
        assert kkr.rel_err(got, full) <= 1e-10
    else:
        assert kkr.rel_err(got, full) < 1e-13


def test_autotuned_panel_width_is_cached_and_used(ozk_mod):
    """kkr_tau00_autotune times every nb = b, 2b, ..., 112 and caches the smallest nb within 1 %
    of the fastest; nb = 0 then runs exactly that nb (bitwise equal results)."""
    import torch
    h = ozk_mod.Handle()
    sizes = [27, 15, 27]
    systems = [_system(L, 0.5 + 0.05j, atom=i) for i, L in enumerate(sizes)]
    best, times = ozk_mod.kkr_tau00_autotune(h, [L * 16 for L in sizes], 16, S=7)
    assert sorted(times) == list(range(16, 113, 16)) and best in times
    assert all(v > 0 for v in times.values())
    lim = np.float32(1.01) * np.float32(min(times.values()))    # as the library compares
    assert best == min(c for c, v in times.items() if np.float32(v) <= lim)

    def run(nb):
        Ms = [ozk_mod.colmajor_cuda(M) for t, G, M in systems]
        t0s = [ozk_mod.colmajor_cuda(t[0]) for t, G, M in systems]
        taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128)) for _ in systems]
        ozk_mod.kkr_tau00_batched(h, Ms, t0s, taus, S=7, nb=nb)
        torch.cuda.synchronize()
        return [ozk_mod.to_numpy(x) for x in taus]

    auto, fixed = run(0), run(best)
    assert h.status() == 0
    for a, f, (t, G, M) in zip(auto, fixed, systems):
        assert np.array_equal(a, f)
        assert kkr.rel_err(a, kkr.tau00_full(M, t[0])) <= 1e-10
    h.close()


def test_single_solve_autotuned_panel_width(ozk_mod):
    """kkr_tau00 with nb = 0 (S >= 1) tunes the (panel, leaf) pair for one matrix on its first
    call (cached per handle; eight leaves per panel allowed for one matrix): leaf panels run on
    the batched solver, whole panels on the single-matrix path.  A second call, and the entry
    the cached pair selects, give the same bits; tau_00 matches the oracle's block LU with
    those widths and the full inverse."""
    h = ozk_mod.Handle()
    t, G, M = _system(27)
    n = M.shape[0]
    runs = []
    for _ in range(2):
        tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
        ozk_mod.kkr_tau00(h, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=7, nb=0)
        runs.append(ozk_mod.to_numpy(tau))
    assert h.status() == 0
    assert np.array_equal(runs[0], runs[1])
    (W, w), times = ozk_mod.kkr_tau00_autotune_panels(h, [n], 16, S=7)
    assert (8 * 48, 48) in times and (64, 64) in times
    tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
    ozk_mod.kkr_tau00(h, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=7, nb=0)
    again = ozk_mod.to_numpy(tau)
    taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))]
    if W == w:              # whole panels: the single-matrix path with nb = W
        ozk_mod.kkr_tau00(h, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), taus[0], S=7, nb=W)
    else:                   # leaf panels: the one-matrix case of the batched solver
        ozk_mod.kkr_tau00_batched(h, [ozk_mod.colmajor_cuda(M)], [ozk_mod.colmajor_cuda(t[0])], taus, S=7, nb=W,
                                  leaf=w)
    assert np.array_equal(again, ozk_mod.to_numpy(taus[0]))
    full = kkr.tau00_full(M, t[0])
    assert kkr.rel_err(runs[0], full) <= 1e-10 and kkr.rel_err(again, full) <= 1e-10
    assert kkr.rel_err(again, co.tau00_block(M, t[0], W, S=7, leaf=w)) <= 1e-13
    h.close()


def test_build_m_shared_sizes_uses_leading_blocks_of_G(ozk_mod, handle):
    """Atoms with LIZs of 9, 15 and 27 sites on one lattice: atom a's M is I - t_a G[:n_a, :n_a]
    with the leading block of the 27-site G, block row by block row as the oracle forms it."""
    import torch
    b, S = 16, 7
    Ls = [15, 27, 9, 27]
    _, G, _ = synth.kkr_system(max(Ls), b, 0.2 + 0.3j, atom=0)
    ts = [synth.kkr_t(L, b, atom=a) for a, L in enumerate(Ls)]
    Ms = [ozk_mod.colmajor_cuda(np.full((L * b, L * b), np.nan, dtype=np.complex128)) for L in Ls]
    ptr = lambda xs: torch.tensor([x.data_ptr() for x in xs], dtype=torch.int64, device="cuda")
    tdev = [_tblocks(ozk_mod, t) for t in ts]          # kept alive until the build has run
    Gd = ozk_mod.colmajor_cuda(G)
    ozk_mod.kkr_build_m_shared_sizes_ptrs(handle, Ls, b, ptr(tdev), Gd, ptr(Ms), S=S)
    assert handle.status() == 0
    for a, L in enumerate(Ls):
        n = L * b
        got = ozk_mod.to_numpy(Ms[a])
        eye = np.eye(n, dtype=np.complex128)
        for i in range(L):
            rows = slice(i * b, (i + 1) * b)
            assert np.array_equal(got[rows], co.zgemm_lu(eye[rows], ts[a][i], G[rows, :n], S))
        assert np.abs(got - kkr.kkr_build(ts[a], G[:n, :n])).max() <= 1e-14


def test_build_m_shared_sizes_many_atoms_ragged_chunks(ozk_mod, handle):
    """13 atoms of 2..20 sites with b = 12: the build stacks the atoms by decreasing LIZ and cuts
    every block row into problems of 128 stacked rows, which here split atoms between problems
    (128 is not a multiple of 12); every atom's M is still I - t_a G[:n_a, :n_a] formed block
    row by block row as the oracle forms it, bit for bit, and nothing past n_a is written."""
    import torch
    b, S = 12, 7
    rng = np.random.default_rng(77)
    Ls = [int(v) for v in rng.integers(2, 21, size=13)]
    Lmax = max(Ls)
    _, G, _ = synth.kkr_system(Lmax, b, 0.4 + 0.2j, atom=3)
    ts = [synth.kkr_t(L, b, atom=a) for a, L in enumerate(Ls)]
    nmax = Lmax * b
    # each atom's M sits in the leading block of an nmax x nmax canvas with leading dimension n_a
    canvas = [torch.full((nmax * nmax,), complex("nan+nanj"), dtype=torch.complex128, device="cuda") for _ in Ls]
    ptr = lambda xs: torch.tensor([x.data_ptr() for x in xs], dtype=torch.int64, device="cuda")
    tdev = [_tblocks(ozk_mod, t) for t in ts]
    Gd = ozk_mod.colmajor_cuda(G)
    ozk_mod.kkr_build_m_shared_sizes_ptrs(handle, Ls, b, ptr(tdev), Gd, ptr(canvas), S=S)
    assert handle.status() == 0
    for a, L in enumerate(Ls):
        n = L * b
        flat = canvas[a].cpu().numpy()
        got = flat[:n * n].reshape(n, n).T
        assert np.all(np.isnan(flat[n * n:]))
        eye = np.eye(n, dtype=np.complex128)
        for i in range(L):
            rows = slice(i * b, (i + 1) * b)
            assert np.array_equal(got[rows], co.zgemm_lu(eye[rows], ts[a][i], G[rows, :n], S))


def test_contour_trace_matches_oracle(ozk_mod, handle):
    """tau_00 at 8 contour energies (one batched solve), their traces and the quadrature sum
    against the oracle's full-inverse tau_00."""
    import torch
    E, w = synth.contour(32)
    pick = np.arange(0, 32, 4)
    systems = [_system(9, complex(E[i]), atom=0) for i in pick]
    Ms = [ozk_mod.colmajor_cuda(M) for t, G, M in systems]
    t0s = [ozk_mod.colmajor_cuda(t[0]) for t, G, M in systems]
    taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128)) for _ in systems]
    _, (pm, pt, pu) = ozk_mod.kkr_tau00_batched(handle, Ms, t0s, taus, S=7, nb=64)
    tr, integral = ozk_mod.kkr_contour_trace(handle, pu, 16, w[pick])
    assert handle.status() == 0
    want_tr, want = kkr.contour_trace([kkr.tau00_full(M, t[0]) for t, G, M in systems], w[pick])
    assert np.abs(tr - want_tr).max() <= 1e-10 * np.abs(want_tr).max()
    assert abs(integral - want) <= 1e-10 * abs(want)
    # the traces are those of the returned blocks
    assert np.allclose(tr, [np.trace(ozk_mod.to_numpy(x)) for x in taus], rtol=1e-15, atol=0)


def test_full_size_batch_sampled_atoms(ozk_mod, handle):
    """The timed step at full size: 256 atoms of the bcc LIZ-65 system (n = 1040, b = 16,
    E = 0.5 + 0.05i) sharing G, M built by the shared-G emulated block-row GEMMs, all solves in
    one batched call at S = 5, nb = 64.  Sampled atoms: M bit for bit against the oracle's
    emulated block-row update, tau_00 against the oracle's block LU with the same S and panels
    (only the binary64 pivot inverses round differently) and within 1e-10 of the binary64
    full inverse of the binary64 M."""
    import torch
    L, b, natoms, S, nb = 65, 16, 256, 5, 64
    n = L * b
    E0 = 0.5 + 0.05j
    t_first, G, _ = synth.kkr_system(L, b, E0, atom=0)
    ts = [t_first] + [synth.kkr_t(L, b, atom=a) for a in range(1, natoms)]
    tdev = [_tblocks(ozk_mod, t) for t in ts]
    Ms = [torch.empty((n, n), dtype=torch.complex128, device="cuda") for _ in range(natoms)]
    taus = [torch.zeros((b, b), dtype=torch.complex128, device="cuda") for _ in range(natoms)]
    ptr = lambda xs: torch.tensor([x.data_ptr() for x in xs], dtype=torch.int64, device="cuda")
    pt, pm, ptau = ptr(tdev), ptr(Ms), ptr(taus)
    ozk_mod.kkr_build_m_shared_ptrs(handle, natoms, L, b, pt, ozk_mod.colmajor_cuda(G), pm, S=S)
    torch.cuda.synchronize()
    assert handle.status() == 0
    sample = [0, 131, 255]
    # Ms hold M^T row-major = M column-major: the transpose of the stored array is M
    M_gpu = {a: Ms[a].cpu().numpy().T.copy() for a in sample}
    ozk_mod.kkr_tau00_batched_ptrs(handle, [n] * natoms, b, pm, pt, ptau, S=S, nb=nb)
    torch.cuda.synchronize()
    assert handle.status() == 0
    eye = np.eye(n, dtype=np.complex128)
    for a in sample:
        rows_checked = range(L) if a == 0 else (0, 32, L - 1)
        for i in rows_checked:
            rows = slice(i * b, (i + 1) * b)
            assert np.array_equal(M_gpu[a][rows], co.zgemm_lu(eye[rows], ts[a][i], G[rows], S))
        got = taus[a].cpu().numpy().T
        assert kkr.rel_err(got, co.tau00_block(M_gpu[a], ts[a][0], nb, S=S)) < 1e-13
        assert kkr.rel_err(got, co.tau00_full(kkr.kkr_build(ts[a], G), ts[a][0])) <= 1e-10


def test_batched_dmma_equals_single_dmma(ozk_mod, handle):
    """S < 0: the batched solver with binary64 DMMA GEMMs (L into per-solve scratch) gives every
    solve bit for bit the single-solve DMMA result, within 1e-12 of the binary64 full inverse."""
    sizes = [27, 9, 15, 2]
    Es = [0.5 + 0.05j, -1.0 + 0.3j, 0.69 + 0.01j, 0.2 + 0.9j]
    systems = [_system(L, E, atom=i) for i, (L, E) in enumerate(zip(sizes, Es))]
    single = []
    for t, G, M in systems:
        tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
        ozk_mod.kkr_tau00(handle, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=-1, nb=32)
        single.append(ozk_mod.to_numpy(tau))
    Ms = [ozk_mod.colmajor_cuda(M) for t, G, M in systems]
    t0s = [ozk_mod.colmajor_cuda(t[0]) for t, G, M in systems]
    taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128)) for _ in systems]
    ozk_mod.kkr_tau00_batched(handle, Ms, t0s, taus, S=-1, nb=32)
    assert handle.status() == 0
    for i, (t, G, M) in enumerate(systems):
        got = ozk_mod.to_numpy(taus[i])
        assert np.array_equal(got, single[i])
        assert kkr.rel_err(got, co.tau00_full(M, t[0])) <= 1e-12


def test_config4_full_size_against_binary64_solve(ozk_mod, handle):
    """The largest workload at full size: bcc LIZ 113, b = 50 (lmax = 4 with spin), n = 5650,
    single emulated solves at S = 5 and 7 with 100-wide panels and with the panel and leaf
    widths tuned for this matrix (nb = 0: leaf panels on the batched solver, the configuration
    the benchmark times), within 1e-10 of tau_00 from a binary64 library LU solve of the same M."""
    import torch
    L, b = 113, 50
    t, G, _ = synth.kkr_system(L, b, 0.5 + 0.05j, atom=0)
    M = kkr.kkr_build(t, G)
    ref = kkr.tau00_lapack(M, t[0])
    M0 = ozk_mod.colmajor_cuda(M)
    t0 = ozk_mod.colmajor_cuda(t[0])
    for S in (5, 7):
        for nb in (100, 0):
            Md = M0.clone()
            tau = ozk_mod.colmajor_cuda(np.zeros((b, b), dtype=np.complex128))
            ozk_mod.kkr_tau00(handle, Md, t0, tau, S=S, nb=nb)
            torch.cuda.synchronize()
            assert handle.status() == 0
            assert kkr.rel_err(ozk_mod.to_numpy(tau), ref) <= 1e-10


def test_config3_full_size_sampled_atoms(ozk_mod, handle):
    """The timed workload at full size: 256 atoms with LIZ sizes drawn from 27..169 sites
    (n = 448..2704, b = 16) at three of the 32 contour energies, each energy with its own G.  M
    of every atom is built by the shared-G emulated block-row GEMMs and all 256 tau_00 are solved
    in one batched call at S = 7 with the autotuned panel and leaf widths (the launch
    configuration the benchmark times).  For the smallest and the largest atom at each energy: every block row of
    M bit for bit against the oracle's emulated block-row update, tau_00 against the oracle's
    block LU of the same M (only the binary64 pivot inverses round differently) and within
    1e-10 of a binary64 library solve of the binary64 M."""
    import torch
    b, S, natoms = 16, 7, 256
    Ls = [int(v) for v in synth.liz_sizes(natoms)]
    ns = [L * b for L in Ls]
    E, _ = synth.contour(32)
    zs = [0, 16, 31]
    (W, w), _ = ozk_mod.kkr_tau00_autotune_panels(handle, ns, b, S=S)
    ts = [synth.kkr_t(L, b, atom=a) for a, L in enumerate(Ls)]
    tdev = [_tblocks(ozk_mod, t) for t in ts]
    Ms = [torch.empty((n, n), dtype=torch.complex128, device="cuda") for n in ns]
    taus = [torch.zeros((b, b), dtype=torch.complex128, device="cuda") for _ in ns]
    ptr = lambda xs: torch.tensor([x.data_ptr() for x in xs], dtype=torch.int64, device="cuda")
    pt, pm, ptau = ptr(tdev), ptr(Ms), ptr(taus)
    sample = [int(np.argmin(Ls)), int(np.argmax(Ls))]
    for z, G in zip(zs, synth.kkr_contour_G(169, b, [complex(E[z]) for z in zs], workers=3)):
        Gd = ozk_mod.colmajor_cuda(G)
        ozk_mod.kkr_build_m_shared_sizes_ptrs(handle, Ls, b, pt, Gd, pm, S=S)
        torch.cuda.synchronize()
        M_gpu = {a: Ms[a].cpu().numpy().T.copy() for a in sample}
        ozk_mod.kkr_tau00_batched_ptrs(handle, ns, b, pm, pt, ptau, S=S, nb=W, leaf=w)
        torch.cuda.synchronize()
        assert handle.status() == 0
        for a in sample:
            n = ns[a]
            for i in range(Ls[a]):
                rows = slice(i * b, (i + 1) * b)
                eye = np.zeros((b, n), dtype=np.complex128)
                eye[:, rows] = np.eye(b)
                assert np.array_equal(M_gpu[a][rows], co.zgemm_lu(eye, ts[a][i], G[rows, :n], S)), (z, a, i)
            got = taus[a].cpu().numpy().T
            assert kkr.rel_err(got, co.tau00_block(M_gpu[a], ts[a][0], W, S=S, leaf=w)) < 1e-13, (z, a, W, w)
            ref = kkr.tau00_lapack(kkr.kkr_build(ts[a], G[:n, :n]), ts[a][0])
            assert kkr.rel_err(got, ref) <= 1e-10, (z, a)
