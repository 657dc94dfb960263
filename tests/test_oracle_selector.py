"""Pins of the selector oracle (oracle/selector.py) against finite differences, closed forms,
invariances and the statistics of the probe estimators (CPU only)."""
import math

import numpy as np
import pytest

import synth
from oracle import selector as sel


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, math.sqrt(2 / 16), (64, 16))
    W2 = rng.normal(0, math.sqrt(2 / 64), (64, 64))
    W3 = rng.normal(0, math.sqrt(1 / 64), (8, 64))
    b1, b2, b3 = rng.normal(0, 0.1, 64), rng.normal(0, 0.1, 64), rng.normal(-8, 1, 8)
    return sel.pack(W1 * scale, b1, W2, b2, W3, b3)


def test_layout():
    assert sel.NPARAMS == 5768
    p = np.arange(sel.NPARAMS, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = sel.unpack(p)
    assert W1[1, 0] == 16 and b1[0] == 1024 and W2[0, 1] == 1089 and b2[0] == 5184
    assert W3[1, 0] == 5248 + 64 and b3[-1] == 5767
    assert np.array_equal(sel.pack(W1, b1, W2, b2, W3, b3), p)


def test_backward_matches_central_differences():
    p = _params(1)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (6, 16))
    T = rng.normal(-8, 3, (6, 8))
    _, Z1, Z2 = sel.forward(p, X)
    assert min(np.abs(Z1).min(), np.abs(Z2).min()) > 1e-4      # no ReLU kink within the step
    g = sel.backward(p, X, T)
    h = 1e-6
    fd = np.empty_like(p)
    for q in range(sel.NPARAMS):
        e = np.zeros_like(p)
        e[q] = h
        fd[q] = (sel.loss(p + e, X, T) - sel.loss(p - e, X, T)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-7 * np.abs(g).max() + 1e-10


def test_forward_is_the_composed_affine_map_when_every_unit_is_active():
    rng = np.random.default_rng(3)
    W1, W2, W3 = np.abs(rng.normal(size=(64, 16))), np.abs(rng.normal(size=(64, 64))), rng.normal(size=(8, 64))
    b1, b2, b3 = np.abs(rng.normal(size=64)) + 0.1, np.abs(rng.normal(size=64)) + 0.1, rng.normal(size=8)
    p = sel.pack(W1, b1, W2, b2, W3, b3)
    X = np.abs(rng.normal(size=(5, 16)))
    Y, _, _ = sel.forward(p, X)
    W = W3 @ W2 @ W1
    c = W3 @ (W2 @ b1 + b2) + b3
    assert np.allclose(Y, X @ W.T + c, rtol=1e-12, atol=1e-9)


def test_dead_first_layer_leaves_the_biases():
    rng = np.random.default_rng(4)
    W1, W2, W3 = rng.normal(size=(64, 16)), rng.normal(size=(64, 64)), rng.normal(size=(8, 64))
    b1, b2, b3 = np.full(64, -1e6), rng.normal(size=64), rng.normal(size=8)
    p = sel.pack(W1, b1, W2, b2, W3, b3)
    Y, _, _ = sel.forward(p, rng.normal(size=(3, 16)))
    assert np.allclose(Y, W3 @ np.maximum(b2, 0) + b3, rtol=0, atol=1e-12)
    g = sel.backward(p, rng.normal(size=(3, 16)), np.zeros((3, 8)))
    W1g, b1g, W2g, *_ = sel.unpack(g)
    assert not W1g.any() and not b1g.any() and not W2g.any()


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(5)
    p0, g = rng.normal(size=50), rng.normal(size=50)
    p1, m, v = sel.adam_step(p0, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    # bias-corrected moments are g and g^2 after the first step
    assert np.allclose(p1, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_minimises_a_quadratic():
    c = np.array([3.0, -2.0, 0.5])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 3001):
        p, m, v = sel.adam_step(p, 2 * (p - c), m, v, t, 0.01)
    assert np.abs(p - c).max() < 1e-3


def test_training_loop_fits_an_affine_target():
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, (256, 16))
    A = rng.normal(size=(8, 16))
    T = X @ A.T - 8.0
    p = _params(7)
    m, v = np.zeros_like(p), np.zeros_like(p)
    l0 = sel.loss(p, X, T)
    for t in range(1, 401):
        p, m, v = sel.adam_step(p, sel.backward(p, X, T), m, v, t, 3e-3)
    assert sel.loss(p, X, T) < l0 / 20


def test_choose_rule():
    pred = np.array([-2.0, -4, -6, -8, -10, -12, -14, -16])
    assert sel.choose(pred, 1e-10) == 7
    assert sel.choose(pred, 1e-10, margin=0.5) == 8
    assert sel.choose(pred, 1e-20) == 10
    assert sel.choose(pred, 1.0) == 3
    assert sel.choose(np.full(8, np.nan), 1e-10) == 10


# ----------------------------------------------------------------------------- features

def test_probe_vectors_have_unit_variance_and_are_counter_based():
    X = sel.probe_vectors(200000, 11)
    assert abs(np.mean(np.abs(X) ** 2) - 1.0) < 0.01
    assert abs(np.mean(X)) < 0.01
    assert np.array_equal(sel.probe_vectors(37, 11), X[:37])


def test_crest_and_exponent_spread_of_equal_magnitude_rows():
    k = 24
    p = np.array([0, 3, -5, 7])
    mag = 0.75 * np.exp2(p)                            # frexp exponents are p
    signs = synth.uniform(1, 0, np.arange(4 * k, dtype=np.uint64)).reshape(4, k) < 0.5
    A = (np.where(signs, -1.0, 1.0) * mag[:, None]) * (1 + 1j)
    B = synth.scaled_uniform(2, 0, (k, 9)) + 0j
    f, _, _ = sel.features(A, B, sel.probe_vectors(9, 1))
    assert np.abs(f[3:6]).max() < 1e-14                  # zero up to the rounding of the logs
    assert f[9] == pytest.approx((7 - p.mean()) / 16, abs=1e-15)


def test_crest_of_a_single_nonzero_per_row():
    k = 40
    A = np.zeros((5, k), dtype=np.complex128)
    A[np.arange(5), [0, 7, 9, 31, 39]] = [0.3, -7.0, 1e-3, 2.5, 1e5]
    B = synth.scaled_uniform(3, 0, (k, 6)) + 1j * synth.scaled_uniform(3, 1, (k, 6))
    f, _, _ = sel.features(A, B, sel.probe_vectors(6, 2))
    c = 0.5 * math.log2(2 * k)
    assert f[3] == pytest.approx(c / 8, abs=1e-14) and f[4] == pytest.approx(c / 8, abs=1e-14)
    assert f[5] == pytest.approx(0.0, abs=1e-14)
    assert f[13] == pytest.approx((5 * k - 5) / (5 * k))


def test_features_are_invariant_under_power_of_two_scaling():
    A = synth.scaled_uniform(4, 0, (30, 20), 3.0) + 1j * synth.scaled_uniform(4, 1, (30, 20), 3.0)
    B = synth.scaled_uniform(5, 0, (20, 25), 3.0) + 1j * synth.scaled_uniform(5, 1, (20, 25), 3.0)
    X = sel.probe_vectors(25, 3)
    f, zs, E = sel.features(A, B, X)
    for a, b in ((700, -300), (-900, 5), (1, 1)):
        g, zs2, E2 = sel.features(np.ldexp(A.real, a) + 1j * np.ldexp(A.imag, a),
                                  np.ldexp(B.real, b) + 1j * np.ldexp(B.imag, b), X)
        assert E2 == E + a + b
        assert np.array_equal(zs2, zs)
        assert np.abs(f - g).max() < 1e-12


def test_cancelled_product_has_zero_cancellation_features():
    k = 8
    A = np.zeros((4, k), dtype=np.complex128)
    A[:, :4] = synth.scaled_uniform(6, 0, (4, 4)) + 1j
    B = np.zeros((k, 5), dtype=np.complex128)
    B[4:, :] = synth.scaled_uniform(6, 1, (4, 5)) - 2j        # rows of A orthogonal to columns of B
    f, zs, _ = sel.features(A, B, sel.probe_vectors(5, 4))
    assert not zs.any() and f[11] == 0 and f[12] == 0
    assert f[13] == pytest.approx(0.5) and f[14] == pytest.approx(0.5)


def test_probe_norm_estimate_is_unbiased():
    A = synth.scaled_uniform(7, 0, (40, 30), 1.0) + 1j * synth.scaled_uniform(7, 1, (40, 30), 1.0)
    B = synth.scaled_uniform(8, 0, (30, 50), 1.0) + 1j * synth.scaled_uniform(8, 1, (30, 50), 1.0)
    C2 = float(np.sum(np.abs(A @ B) ** 2))
    est = []
    for seed in range(400):
        X = sel.probe_vectors(50, 1000 + seed)
        f, zs, E = sel.features(A, B, X)
        est.append(50 * np.sum(np.abs(zs) ** 2) / np.sum(np.abs(X) ** 2) * 4.0 ** E)
    assert abs(np.mean(est) / C2 - 1.0) < 0.05
    # f11 is the cancellation log2(|A| |B| / |AB|) / 16 of the estimate
    lc = 0.5 * math.log2(est[-1])
    la, lb = math.log2(np.linalg.norm(A)), math.log2(np.linalg.norm(B))
    assert f[11] == pytest.approx((la + lb - lc) / 16, abs=1e-12)


def test_residual_estimate_measures_the_relative_frobenius_error():
    A = synth.scaled_uniform(9, 0, (40, 30), 1.0) + 1j * synth.scaled_uniform(9, 1, (40, 30), 1.0)
    B = synth.scaled_uniform(10, 0, (30, 35), 1.0) + 1j * synth.scaled_uniform(10, 1, (30, 35), 1.0)
    C = A @ B
    Err = 1e-6 * (synth.scaled_uniform(11, 0, C.shape, 0.0) + 1j * synth.scaled_uniform(11, 1, C.shape, 0.0))
    want = np.linalg.norm(Err) / np.linalg.norm(C)
    r2 = []
    for seed in range(400):
        X = sel.probe_vectors(35, 5000 + seed)
        _, zs, E = sel.features(A, B, X)
        r2.append(sel.residual_estimate(C + Err, X, zs, E) ** 2)
        assert sel.residual_estimate(C, X, zs, E) < 1e-14
    # E||Err x||^2 / E||C x||^2 = ||Err||^2 / ||C||^2; the ratio of sample means converges to it
    assert abs(math.sqrt(np.mean(r2)) / want - 1.0) < 0.1


def test_integer_images_are_exact():
    V = synth.scaled_uniform(12, 0, (7, 5), 8.0) + 1j * synth.scaled_uniform(12, 1, (7, 5), 8.0)
    re, im, e = sel._to_int(V)
    back = np.array([[math.ldexp(int(r), e) + 1j * math.ldexp(int(i), e) for r, i in zip(rr, ii)]
                     for rr, ii in zip(re, im)])
    assert np.array_equal(back, V)
    a = (np.array([[1, -2], [3, 4]], dtype=object), np.array([[0, 1], [1, 0]], dtype=object), -3)
    b = (np.array([[5], [6]], dtype=object), np.array([[-1], [2]], dtype=object), 1)
    pr, pi, pe = sel._int_mul(a, b)
    A = (a[0].astype(float) + 1j * a[1].astype(float)) * 2.0 ** -3
    B = (b[0].astype(float) + 1j * b[1].astype(float)) * 2.0
    assert pe == -2 and np.array_equal(pr.astype(float) * 0.25 + 1j * pi.astype(float) * 0.25, A @ B)


def test_exact_probe_residual_sees_through_cancellation():
    """A product whose result is 1e-9 of the operands' scale: the binary64 probe product has
    errors far above the tolerance, the exact one resolves a planted 1e-12 relative error."""
    rng = np.random.default_rng(13)
    m, k, n = 20, 36, 15
    A = rng.normal(size=(m, k)) + 1j * rng.normal(size=(m, k))
    _, _, vh = np.linalg.svd(A)
    N = vh[m:].conj().T
    B = N @ (rng.normal(size=(k - m, n)) + 1j * rng.normal(size=(k - m, n)))
    B = B + 1e-9 * (rng.normal(size=(k, n)) + 1j * rng.normal(size=(k, n)))
    X = sel.probe_vectors(n, 5)
    _, zx, E = sel.features(A, B, X, exact=True)
    _, zf, _ = sel.features(A, B, X)
    # exact product of the binary64 operands, rounded: relative error ~1e-16
    ar, ai, ea = sel._to_int(A)
    br, bi, eb = sel._to_int(B)
    cr, ci, ec = sel._int_mul((ar, ai, ea), (br, bi, eb))
    C = np.array([[math.ldexp(int(x), ec) for x in row] for row in cr]) + \
        1j * np.array([[math.ldexp(int(x), ec) for x in row] for row in ci])
    assert sel.residual_estimate(C, X, zx, E) < 1e-15
    assert sel.residual_estimate(C, X, zf, E) > 1e-10           # the binary64 check cannot tell
    r = sel.residual_estimate(C * (1 + 1e-12), X, zx, E)
    assert 0.5e-12 < r < 2e-12
