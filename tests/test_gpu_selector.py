"""GPU parity of the slice-count selector (features, perceptron forward / gradient / Adam, probe
residual check, fallback) against the float64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

import synth
from gpu_util import op, rand_complex, stored
from oracle import c_oracle as co
from oracle import selector as sel

pytestmark = pytest.mark.gpu


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


CASES = [
    ((37, 29, 41), "N", "N", 2.0, 0),
    ((64, 130, 17), "T", "N", 6.0, 1),
    ((90, 33, 120), "N", "C", 0.0, 2),
    ((5, 7, 300), "C", "T", 2.0, 3),
]


@pytest.mark.parametrize("mnk,ta,tb,sigma,seed", CASES)
def test_features_match_oracle(ozk_mod, handle, mnk, ta, tb, sigma, seed):
    m, n, k = mnk
    A = rand_complex(m, k, 100 + seed, sigma)
    B = rand_complex(k, n, 200 + seed, sigma)
    A[3 % m, :] = 0                       # a zero row of op(A)
    B[:, 1 % n] = 0                       # a zero column of op(B)
    A[0, :k // 2] = 0
    As, Bs = stored(A, ta), stored(B, tb)
    f = ozk_mod.to_numpy(ozk_mod.selector_features(handle, ozk_mod.colmajor_cuda(As), ozk_mod.colmajor_cuda(Bs),
                                                   ta, tb, seed=77 + seed))
    want, _, _ = sel.features(A, B, sel.probe_vectors(n, 77 + seed), exact=True)
    assert np.abs(f - want).max() <= 2e-6 * max(1.0, np.abs(want).max())


def test_features_of_extreme_scales_and_zero_operand(ozk_mod, handle):
    A = rand_complex(40, 30, 5, 1.0) * 2.0 ** 900
    B = rand_complex(30, 20, 6, 1.0) * 2.0 ** -1000
    f = ozk_mod.to_numpy(ozk_mod.selector_features(handle, ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B), seed=9))
    want, _, _ = sel.features(A, B, sel.probe_vectors(20, 9))
    assert np.all(np.isfinite(f)) and np.abs(f - want).max() <= 2e-6
    Z = np.zeros((30, 20), dtype=np.complex128)
    f0 = ozk_mod.to_numpy(ozk_mod.selector_features(handle, ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(Z), seed=9))
    want0, _, _ = sel.features(A, Z, sel.probe_vectors(20, 9))
    assert np.array_equal(f0, want0.astype(np.float32))


def _random_params(seed):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, math.sqrt(2 / 16), (64, 16))
    W2 = rng.normal(0, math.sqrt(2 / 64), (64, 64))
    W3 = rng.normal(0, math.sqrt(1 / 64), (8, 64))
    return sel.pack(W1, rng.normal(0, 0.1, 64), W2, rng.normal(0, 0.1, 64), W3, rng.normal(-8, 1, 8)).astype(np.float32)


def test_forward_matches_oracle(ozk_mod, handle):
    p = _random_params(1)
    handle.selector_set_params(p)
    X = np.random.default_rng(2).normal(0, 1, (1000, 16)).astype(np.float32)
    Y = ozk_mod.to_numpy(ozk_mod.selector_predict(handle, _cuda(X)))
    want, _, _ = sel.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.abs(Y - want).max() <= 1e-4 * max(1.0, np.abs(want).max())
    assert np.array_equal(handle.selector_get_params(), p)


def test_gradient_and_adam_step_match_oracle(ozk_mod, handle):
    p = _random_params(3)
    handle.selector_set_params(p)
    rng = np.random.default_rng(4)
    X = rng.normal(0, 1, (300, 16)).astype(np.float32)
    T = rng.normal(-8, 3, (300, 8)).astype(np.float32)
    p64, X64, T64 = p.astype(np.float64), X.astype(np.float64), T.astype(np.float64)
    g = ozk_mod.to_numpy(ozk_mod.selector_gradient(handle, _cuda(X), _cuda(T)))
    want = sel.backward(p64, X64, T64)
    assert np.abs(g - want).max() <= 1e-4 * np.abs(want).max()
    lr = 1e-3
    loss = ozk_mod.selector_train_step(handle, _cuda(X), _cuda(T), lr)
    assert loss == pytest.approx(sel.loss(p64, X64, T64), rel=1e-5)
    p1 = handle.selector_get_params().astype(np.float64)
    w1, _, _ = sel.adam_step(p64, want, np.zeros_like(p64), np.zeros_like(p64), 1, lr)
    # first Adam step: lr * g / (|g| + eps); entries whose gradient is far above eps agree
    big = np.abs(want) > 1e-5
    assert np.abs(p1 - w1)[big].max() <= 1e-3 * lr
    assert np.abs(p1 - p64).max() <= lr * (1 + 1e-3)


def test_training_on_the_gpu_tracks_the_oracle(ozk_mod, handle):
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (512, 16)).astype(np.float32)
    A = rng.normal(size=(8, 16))
    T = (X.astype(np.float64) @ A.T - 8.0).astype(np.float32)
    p = _random_params(6)
    handle.selector_set_params(p)
    p64 = p.astype(np.float64)
    m, v = np.zeros_like(p64), np.zeros_like(p64)
    Xd, Td = _cuda(X), _cuda(T)
    for t in range(1, 201):
        ozk_mod.selector_train_step(handle, Xd, Td, 3e-3, want_loss=False)
        p64, m, v = sel.adam_step(p64, sel.backward(p64, X.astype(np.float64), T.astype(np.float64)), m, v, t, 3e-3)
    l_gpu = sel.loss(handle.selector_get_params().astype(np.float64), X, T)
    l_cpu = sel.loss(p64, X, T)
    l0 = sel.loss(p.astype(np.float64), X, T)
    assert l_gpu < l0 / 10 and l_cpu < l0 / 10
    assert l_gpu <= 1.5 * l_cpu + 1e-6                 # float32 and float64 trajectories stay close


def w_rounding_bound(D, X, z, E, chunk=16):
    """Bound on how far the device residual estimate may sit from the exact one: the check's
    W = D X is formed with binary64 multiply-adds over chunks of `chunk` terms (chunk partials
    added in double-double), so each element is off by at most chunk eps sum_l (|Re d|+|Im d|)
    (|Re x|+|Im x|) (two such sums, real and imaginary part); by the triangle inequality the
    estimate ||2^-E W - z|| / ||z|| moves by at most the norm of that bound over ||z||
    (z = 2^-E op(A) op(B) X, here in binary64: only its norm enters)."""
    eps = np.finfo(float).eps
    absD = np.abs(D.real) + np.abs(D.imag)
    absX = np.abs(X.real) + np.abs(X.imag)
    el = chunk * eps * (absD @ absX) * np.sqrt(2.0) * 2.0 ** (-E)
    return float(np.linalg.norm(el) / np.linalg.norm(z)) + 1e-300


def _const_params(pred_log10):
    """Parameters whose every output is the constant pred_log10 (zero weights)."""
    p = np.zeros(sel.NPARAMS, dtype=np.float32)
    p[sel.OFF_B3:] = pred_log10
    return p


def test_selected_S_passes_the_residual_check(ozk_mod, handle):
    import torch
    A, B = rand_complex(200, 150, 11, 1.0), rand_complex(150, 120, 12, 1.0)
    Ad, Bd = ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B)
    p = np.zeros(sel.NPARAMS, dtype=np.float32)
    p[sel.OFF_B3:] = [-3, -5, -8, -11, -14, -16, -16, -16]        # S = 6 meets 1e-10 with margin 0.3
    handle.selector_set_params(p)
    handle.selector_configure(tol=1e-10, margin=0.3)
    C = ozk_mod.colmajor_cuda(np.zeros((200, 120), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, Ad, Bd, C, S=0)
    info = handle.selector_last()
    assert info["S_selected"] == 6 and info["S_used"] == 6 and not info["fallback"] and info["residual_ok"]
    # the returned product is the S = 6 emulated product, bit for bit
    C6 = ozk_mod.colmajor_cuda(np.zeros((200, 120), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, Ad, Bd, C6, S=6)
    got = ozk_mod.to_numpy(C)
    assert np.array_equal(got, ozk_mod.to_numpy(C6))
    # the device residual estimate is the oracle's for that product and those probes, within
    # the rounding of its binary64 chunk sums of W = D X
    X = sel.probe_vectors(120, info["probe_seed"])
    _, zs, E = sel.features(A, B, X, exact=True)
    r = sel.residual_estimate(got, X, zs, E)
    assert abs(info["residual"] - r) <= w_rounding_bound(got, X, (A @ (B @ X)) * 2.0 ** (-E), E)
    assert r <= 1e-10 and np.linalg.norm(got - A @ B) / np.linalg.norm(A @ B) < 1e-10
    torch.cuda.synchronize()


def test_underestimated_error_falls_back_to_S_max(ozk_mod, handle):
    A, B = rand_complex(150, 100, 13, 2.0), rand_complex(100, 90, 14, 2.0)
    Ad, Bd = ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B)
    handle.selector_set_params(_const_params(-30.0))                # claims S = 3 is exact enough
    handle.selector_configure(tol=1e-10, margin=0.0)
    C = ozk_mod.colmajor_cuda(np.zeros((150, 90), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, Ad, Bd, C, S=0)
    info = handle.selector_last()
    assert info["S_selected"] == 3 and info["fallback"] and info["S_used"] == 10 and info["residual_ok"]
    assert info["residual_selected"] > 1e-10
    got = ozk_mod.to_numpy(C)
    assert np.array_equal(got, co.zgemm(A, B, 10))                  # the S = 10 product, bit for bit
    # with the fallback disabled the failed check is an error
    handle.selector_configure(tol=1e-10, margin=0.0, flags=ozk_mod.OZK_SEL_NO_FALLBACK)
    with pytest.raises(ozk_mod.OzkError, match="RESIDUAL"):
        ozk_mod.ozaki_zgemm(handle, Ad, Bd, C, S=0)
    handle.selector_configure()


def test_pessimistic_prediction_selects_S_max_and_general_alpha_beta(ozk_mod, handle):
    A, B = rand_complex(64, 48, 15, 1.0), rand_complex(48, 80, 16, 1.0)
    C0 = rand_complex(64, 80, 17, 1.0)
    handle.selector_set_params(_const_params(0.0))
    handle.selector_configure(tol=1e-10)
    alpha, beta = 0.5 - 2j, 1.5 + 0.25j
    C = ozk_mod.colmajor_cuda(C0)
    ozk_mod.ozaki_zgemm(handle, ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B), C, S=0, alpha=alpha, beta=beta)
    info = handle.selector_last()
    assert info["S_selected"] == 10 and not info["fallback"]
    want = alpha * co.zgemm(A, B, 10) + beta * C0
    got = ozk_mod.to_numpy(C)
    assert np.abs(got - want).max() <= 8 * np.finfo(float).eps * (abs(alpha) * np.abs(co.zgemm(A, B, 10)) +
                                                                  abs(beta) * np.abs(C0)).max()


def test_S0_without_parameters_and_under_capture_is_refused(ozk_mod):
    import torch
    h = ozk_mod.Handle()
    A = ozk_mod.colmajor_cuda(rand_complex(8, 8, 1))
    C = ozk_mod.colmajor_cuda(np.zeros((8, 8), dtype=np.complex128))
    with pytest.raises(ozk_mod.OzkError, match="selector"):
        ozk_mod.ozaki_zgemm(h, A, A, C, S=0)
    h.selector_init(5)
    ozk_mod.ozaki_zgemm(h, A, A, C, S=0)                           # sizes the scratch
    g = torch.cuda.CUDAGraph()
    with pytest.raises(ozk_mod.OzkError, match="capture"):
        with torch.cuda.graph(g):
            h.set_stream(torch.cuda.current_stream())
            ozk_mod.ozaki_zgemm(h, A, A, C, S=0)
    h.set_stream(torch.cuda.current_stream())
    h.close()


def test_parameter_file_round_trip(ozk_mod, handle, tmp_path):
    handle.selector_init(42)
    p = handle.selector_get_params()
    assert np.all(np.isfinite(p)) and np.abs(p).max() > 0
    path = str(tmp_path / "sel.bin")
    handle.selector_save(path)
    h2 = ozk_mod.Handle()
    h2.selector_load(path)
    assert np.array_equal(h2.selector_get_params(), p)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"OZKSEL1\x00" + (7).to_bytes(4, "little"))
    with pytest.raises(ozk_mod.OzkError, match="ARG"):
        h2.selector_load(str(bad))
    with pytest.raises(ozk_mod.OzkError, match="NOFILE"):
        h2.selector_load(str(tmp_path / "missing.bin"))
    h2.close()


def test_rel_diff_matches_numpy(ozk_mod, handle):
    X, Y = rand_complex(70, 33, 21), rand_complex(70, 33, 22)
    r = ozk_mod.rel_diff(handle, ozk_mod.colmajor_cuda(X), ozk_mod.colmajor_cuda(Y))
    assert r == pytest.approx(np.linalg.norm(X - Y) / np.linalg.norm(Y), rel=1e-13)


def test_residual_check_resolves_cancelled_products(ozk_mod, handle):
    """op(A) op(B) cancels to 1e-9 of the operands' scale.  The compensated probe products
    still measure the emulated product's error exactly enough: an S whose true error meets
    the tolerance passes the check (no false fallback), and the estimate matches the exact
    oracle's."""
    rng = np.random.default_rng(31)
    m, k, n = 96, 160, 80
    A = rng.normal(size=(m, k)) + 1j * rng.normal(size=(m, k))
    _, _, vh = np.linalg.svd(A)
    B = vh[m:].conj().T @ (rng.normal(size=(k - m, n)) + 1j * rng.normal(size=(k - m, n)))
    B = B + 1e-9 * (rng.normal(size=(k, n)) + 1j * rng.normal(size=(k, n)))
    Ad, Bd = ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B)
    p = np.zeros(sel.NPARAMS, dtype=np.float32)
    p[sel.OFF_B3:] = [0, 0, 0, 0, 0, 0, 0, -30]                    # always S = 10
    handle.selector_set_params(p)
    handle.selector_configure(tol=1e-6, margin=0.0)
    C = ozk_mod.colmajor_cuda(np.zeros((m, n), dtype=np.complex128))
    ozk_mod.ozaki_zgemm(handle, Ad, Bd, C, S=0)
    info = handle.selector_last()
    got = ozk_mod.to_numpy(C)
    X = sel.probe_vectors(n, info["probe_seed"])
    _, zs, E = sel.features(A, B, X, exact=True)
    r = sel.residual_estimate(got, X, zs, E)
    assert info["S_selected"] == 10 and not info["fallback"] and info["residual_ok"]
    assert r < 1e-6 and info["residual"] == pytest.approx(r, rel=1e-3, abs=1e-20)
    assert abs(info["residual"] - r) <= w_rounding_bound(got, X, (A @ (B @ X)) * 2.0 ** (-E), E)
    handle.selector_configure()


def test_batched_solve_with_selected_S(ozk_mod):
    """S = 0 on the batched KKR solve: the selector's choice over the sampled solves' first
    trailing updates, checked and applied to the whole call (bitwise the explicit-S solve); a
    network that claims S = 3 fails the sampled checks and the call runs at S = 10; S < 0
    solves in binary64."""
    import torch
    from oracle import kkr
    h = ozk_mod.Handle()
    p = np.zeros(sel.NPARAMS, dtype=np.float32)
    p[sel.OFF_B3:] = [-3, -5, -8, -11, -14, -16, -16, -16]        # S = 6 at 1e-10, margin 0.3
    h.selector_set_params(p)
    h.selector_configure(tol=1e-10, margin=0.3)
    systems = [synth.kkr_system(L, 16, 0.5 + 0.05j, atom=i)[:2] for i, L in enumerate([27, 15])]
    Mnp = [kkr.kkr_build(t, G) for t, G in systems]

    def run(S):
        Ms = [ozk_mod.colmajor_cuda(M) for M in Mnp]
        t0s = [ozk_mod.colmajor_cuda(t[0]) for t, G in systems]
        taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128)) for _ in systems]
        ozk_mod.kkr_tau00_batched(h, Ms, t0s, taus, S=S, nb=64)
        torch.cuda.synchronize()
        return [ozk_mod.to_numpy(x) for x in taus]

    auto = run(0)
    info = h.selector_last()
    assert info["S_selected"] == 6 and info["S_used"] == 6 and info["gemms"] == 2 and info["residual_ok"]
    for a, b6 in zip(auto, run(6)):
        assert np.array_equal(a, b6)
    h.selector_set_params(_const_params(-30.0))
    h.selector_configure(tol=1e-10, margin=0.0)
    low = run(0)
    info = h.selector_last()
    assert info["S_selected"] == 3 and info["fallback"] and info["S_used"] == 10 and not info["residual_ok"]
    for a, b10 in zip(low, run(10)):
        assert np.array_equal(a, b10)
    # S < 0 is the binary64 DMMA form of the same batched solve
    for a, d in zip(auto, run(-1)):
        assert kkr.rel_err(a, d) <= 1e-12
    h.close()


def test_single_solve_S_rule(ozk_mod):
    """kkr_tau00 follows the ABI's slice-count rule: S = 0 runs every GEMM of the solve through
    the selector (its choice and residual check per GEMM; here a network that always picks S = 6
    and products that pass the check, so bit for bit the S = 6 solve, with ozk_selector_last
    updated), S < 0 runs every GEMM as a binary64 DMMA GEMM (bit for bit the batched DMMA form)."""
    import torch
    from oracle import kkr
    h = ozk_mod.Handle()
    p = np.zeros(sel.NPARAMS, dtype=np.float32)
    p[sel.OFF_B3:] = [-3, -5, -8, -11, -14, -16, -16, -16]        # S = 6 at 1e-10, margin 0.3
    h.selector_set_params(p)
    h.selector_configure(tol=1e-10, margin=0.3)
    t, G = synth.kkr_system(27, 16, 0.5 + 0.05j, atom=4)[:2]
    M = kkr.kkr_build(t, G)

    def single(S):
        tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
        ozk_mod.kkr_tau00(h, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=S, nb=64)
        torch.cuda.synchronize()
        return ozk_mod.to_numpy(tau)

    auto = single(0)
    seed0 = h.selector_last()["probe_seed"]
    assert np.array_equal(single(0), auto)
    info = h.selector_last()
    assert info["S_selected"] == 6 and info["S_used"] == 6 and not info["fallback"]
    assert info["residual_ok"] and 0 < info["residual"] <= 0.5e-10
    # one selector call per GEMM: two per panel, 7 panels of (432 - 16) columns at nb = 64
    assert info["probe_seed"] - seed0 == 14
    assert info["gemms"] == 14 and info["S_count"] == {6: 14}
    assert np.array_equal(auto, single(6))
    dm = single(-1)
    Ms = [ozk_mod.colmajor_cuda(M)]
    taus = [ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))]
    ozk_mod.kkr_tau00_batched(h, Ms, [ozk_mod.colmajor_cuda(t[0])], taus, S=-1, nb=64)
    assert np.array_equal(dm, ozk_mod.to_numpy(taus[0]))
    full = kkr.tau00_full(M, t[0])
    assert kkr.rel_err(auto, full) <= 1e-10 and kkr.rel_err(dm, full) <= 1e-12
    assert h.status() == 0
    h.close()


def test_single_solve_failed_check_redoes_the_solve_at_S_max(ozk_mod):
    """A network that claims S = 3 is exact enough: the GEMMs of the S = 0 solve run at S = 3,
    their deferred probe checks fail, and the solve is redone from the saved M with every GEMM at
    S = 10 (bit for bit the S = 10 solve); with the fallback disabled the solve reports
    OZK_ERR_RESIDUAL."""
    import torch
    from oracle import kkr
    h = ozk_mod.Handle()
    h.selector_set_params(_const_params(-30.0))
    h.selector_configure(tol=1e-10, margin=0.0)
    t, G = synth.kkr_system(27, 16, 0.5 + 0.05j, atom=5)[:2]
    M = kkr.kkr_build(t, G)

    def single(S):
        tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
        ozk_mod.kkr_tau00(h, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=S, nb=64)
        torch.cuda.synchronize()
        return ozk_mod.to_numpy(tau)

    auto = single(0)
    info = h.selector_last()
    assert info["S_selected"] == 3 and info["fallback"] and info["S_used"] == 10
    assert info["residual_ok"] and info["residual"] <= 0.5e-10 and info["S_count"] == {3: 14}
    assert np.array_equal(auto, single(10))
    assert kkr.rel_err(auto, kkr.tau00_full(M, t[0])) <= 1e-10
    h.selector_configure(tol=1e-10, margin=0.0, flags=ozk_mod.OZK_SEL_NO_FALLBACK)
    with pytest.raises(ozk_mod.OzkError, match="RESIDUAL"):
        single(0)
    assert h.status() == 0
    h.close()


def test_selector_log_records_features_and_targets(ozk_mod):
    """While the selector log is on, every S = 0 GEMM writes its features (those of the probe
    seed it used) and the log10 errors of its products at S = 3..10 against S = 12 (floored at
    -17); GEMMs past the capacity are not recorded and the products are unchanged."""
    import torch
    h = ozk_mod.Handle()
    h.selector_load()
    h.selector_configure(tol=1e-10)
    cap = 2
    F = torch.zeros((cap, 16), dtype=torch.float32, device="cuda")
    T = torch.zeros((cap, 8), dtype=torch.float32, device="cuda")
    inst = [(rand_complex(40, 24, 91 + i), rand_complex(24, 30, 95 + i)) for i in range(3)]
    h.selector_log_begin(F, T)
    seeds, outs = [], []
    for A, B in inst:
        C = ozk_mod.colmajor_cuda(np.zeros((40, 30), dtype=np.complex128))
        ozk_mod.ozaki_zgemm(h, ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B), C, S=0)
        seeds.append(h.selector_last()["probe_seed"])
        outs.append(ozk_mod.to_numpy(C))
    assert h.selector_log_end() == cap
    for i, (A, B) in enumerate(inst[:cap]):
        Ad, Bd = ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B)
        f = ozk_mod.to_numpy(ozk_mod.selector_features(h, Ad, Bd, seed=seeds[i]))
        assert np.array_equal(f, F[i].cpu().numpy())
        ref = ozk_mod.colmajor_cuda(np.zeros((40, 30), dtype=np.complex128))
        ozk_mod.ozaki_zgemm(h, Ad, Bd, ref, S=12)
        for o, S in enumerate(range(3, 11)):
            C = ozk_mod.colmajor_cuda(np.zeros((40, 30), dtype=np.complex128))
            ozk_mod.ozaki_zgemm(h, Ad, Bd, C, S=S)
            e = ozk_mod.rel_diff(h, C, ref)
            want = max(math.log10(e), -17.0) if e > 1e-17 else -17.0
            assert abs(float(T[i, o]) - want) <= 1e-5 * max(1.0, abs(want))
        # the logged call's product is the product at the S the selector used
        assert kkr_rel(outs[i], co.zgemm(A, B, 12)) <= 1e-10
    assert h.status() == 0
    h.close()


def test_selector_log_rows_of_a_solve(ozk_mod):
    """The log hook inside a KKR solve (how the training set is gathered from the contour
    workload): kkr_tau00 with S = 0 writes one row per GEMM of the solve (two per panel), with
    finite features and targets that fall with S (each a log10 relative error at most 0,
    floored at -17); the solve's tau_00 is unchanged in accuracy."""
    import torch
    from oracle import kkr
    h = ozk_mod.Handle()
    h.selector_load()
    h.selector_configure(tol=1e-10)
    t, G = synth.kkr_system(27, 16, 0.5 + 0.05j, atom=9)[:2]
    M = kkr.kkr_build(t, G)
    F = torch.zeros((40, 16), dtype=torch.float32, device="cuda")
    T = torch.zeros((40, 8), dtype=torch.float32, device="cuda")
    tau = ozk_mod.colmajor_cuda(np.zeros((16, 16), dtype=np.complex128))
    h.selector_log_begin(F, T)
    ozk_mod.kkr_tau00(h, ozk_mod.colmajor_cuda(M), ozk_mod.colmajor_cuda(t[0]), tau, S=0, nb=64)
    rows = h.selector_log_end()
    assert rows == 14 == h.selector_last()["gemms"]              # 7 panels of (432 - 16) columns
    Fh, Th = F[:rows].cpu().numpy(), T[:rows].cpu().numpy()
    assert np.all(np.isfinite(Fh)) and np.all(np.isfinite(Th))
    assert np.all(Th <= 0.0) and np.all(Th >= -17.0)
    assert np.all(np.diff(Th, axis=1) <= 0.3)                   # errors fall with S (to the floor)
    assert np.all(Th[:, 0] > Th[:, -1])
    assert not np.any(F[rows:].cpu().numpy())                   # nothing past the solve's rows
    assert kkr.rel_err(ozk_mod.to_numpy(tau), kkr.tau00_full(M, t[0])) <= 1e-10
    assert h.status() == 0
    h.close()


def kkr_rel(X, Y):
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


def test_trained_selector_gains_over_fixed_S(ozk_mod):
    """The committed trained parameters on instances of an unseen seed: every returned product
    meets the tolerance against the S = 12 reference, and the products cost far fewer slice
    pairs than S = 10 (what a caller without the network must use to be safe on this family):
    P_S = S (S + 1) / 2 pairs, plus the S = 10 recomputation of any fallback."""
    import torch
    from paper_2603_29975_gb300 import selector as seltrain
    h = ozk_mod.Handle()
    h.selector_load()                                   # paper_2603_29975_gb300/selector_weights.bin
    h.selector_configure(tol=1e-10)
    inst = seltrain.generate_instances(40, 999, kkr_sizes=(15, 27), energies=1)
    pairs = lambda S: S * (S + 1) // 2
    work, worst = 0, 0.0
    for _, _, A, B in inst:
        Ad, Bd = ozk_mod.colmajor_cuda(A), ozk_mod.colmajor_cuda(B)
        m, n = A.shape[0], B.shape[1]
        C = torch.empty((n, m), dtype=torch.complex128, device="cuda").t()
        ref = torch.empty((n, m), dtype=torch.complex128, device="cuda").t()
        ozk_mod.ozaki_zgemm(h, Ad, Bd, C, S=0)
        ozk_mod.ozaki_zgemm(h, Ad, Bd, ref, S=12)
        info = h.selector_last()
        work += pairs(info["S_selected"]) + (pairs(10) if info["fallback"] else 0)
        worst = max(worst, ozk_mod.rel_diff(h, C, ref))
    assert h.status() == 0
    assert worst <= 1e-10
    assert work <= 0.6 * len(inst) * pairs(10)
    h.close()
