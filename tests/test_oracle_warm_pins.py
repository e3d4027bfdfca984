"""Pins of the warm-start oracle (the MLP and the start-selection arithmetic), CPU only.

Each test ties the oracle to something other than itself: central finite differences of the
loss, a network small enough to evaluate by hand, the closed form of Adam's first step, the
brute-force chi^2 of a residual, the polarized StefCal step of the diagonal oracle, and the
symmetries (global phase) the definitions must respect.
"""
import numpy as np
import pytest

from oracle import blocks, diagonal, mlp, warm
from paper_1502_06974_gb300 import synth


def _tiny_jones(n_ant=5, n_samp=3, seed=11, noise=0.05):
    r = synth.rng_for(seed, 3)
    a1, a2 = synth.baseline_table(n_ant)
    m = synth.complex_noise(r, (n_samp, len(a1), 2, 2), 0.3)
    m[..., 0, 0] += 2.0
    m[..., 1, 1] += 2.0
    g = synth.jones_gains(r, n_ant, 0.2, 0.1)
    d = synth.simulate_jones(g, m, a1, a2) + synth.complex_noise(r, m.shape, noise)
    return d, m, a1, a2, g


# ------------------------------------------------------------------------------------ the network

def test_mlp_gradient_matches_central_differences():
    """Every gradient entry of a small network matches (L(p + h e) - L(p - h e)) / 2h."""
    dims = (5, 7, 6, 3)
    r = np.random.default_rng(1)
    p = mlp.init_params(dims, r) + 0.05 * r.normal(size=mlp.n_params(dims))
    x = r.normal(size=(9, 5))
    t = r.normal(size=(9, 3))
    loss, g = mlp.loss_and_grad(p, dims, x, t)
    h = 1e-6
    num = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        num[k] = (mlp.loss_and_grad(p + e, dims, x, t)[0] - mlp.loss_and_grad(p - e, dims, x, t)[0]) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))
    assert loss == pytest.approx(np.mean((mlp.forward(p, dims, x)[2] - t) ** 2))


def test_mlp_forward_by_hand():
    """A 2-2-2-1 network evaluated by hand: relu cuts the negative unit in each layer."""
    dims = (2, 2, 2, 1)
    W1 = np.array([[1.0, -1.0], [2.0, 0.5]]); b1 = np.array([0.0, -1.0])
    W2 = np.array([[1.0, 0.0], [3.0, -2.0]]); b2 = np.array([0.5, 0.0])
    W3 = np.array([[2.0], [7.0]]); b3 = np.array([-1.0])
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    x = np.array([[1.0, 1.0]])
    # layer 1: [1 + 2, -1 + 0.5 - 1] = [3, -1.5] -> [3, 0]
    # layer 2: [3 + 0.5, 0] = [3.5, 0] -> [3.5, 0];  out: 2 * 3.5 - 1 = 6
    h1, h2, y = mlp.forward(p, dims, x)
    np.testing.assert_allclose(h1, [[3.0, 0.0]])
    np.testing.assert_allclose(h2, [[3.5, 0.0]])
    np.testing.assert_allclose(y, [[6.0]])


def test_adam_first_step_is_signed_learning_rate():
    """With zero moments, bias correction makes the first step lr * g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p1, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_bf16_rounding():
    """Round to nearest, ties to even, at 7 stored mantissa bits (ulp 2^-7 at 1)."""
    u = 2.0 ** -7
    cases = [(1.0, 1.0), (1 + u / 2, 1.0), (1 + u / 2 + 2 ** -20, 1 + u), (1 + 1.5 * u, 1 + 2 * u),
             (1 + u, 1 + u), (-3.0, -3.0), (2.0 ** -130, 2.0 ** -130), (0.0, 0.0)]
    for a, want in cases:
        assert mlp.bf16(np.float32(a)) == np.float64(np.float32(want)), a


def test_bf16_forward_is_close_to_fp64():
    """The bfloat16 forward pass differs from FP64 by rounding only (a few parts in 1e3)."""
    dims = (6, 16, 16, 3)
    r = np.random.default_rng(8)
    p = mlp.init_params(dims, r)
    x = r.normal(size=(20, 6))
    y = mlp.forward(p, dims, x)[2]
    yb = mlp.forward_bf16(p, dims, x)
    assert 0 < np.max(np.abs(yb - y)) <= 2e-2 * np.sqrt(np.mean(y ** 2))


# ------------------------------------------------------------------------------------ features

def test_step_feature_is_the_polarized_stefcal_step():
    """C H^-1 at g1 is exactly the GN gain of the diagonal oracle's polarized step."""
    d, m, a1, a2, g = _tiny_jones()
    g1 = g + 0.1 * synth.complex_noise(synth.rng_for(2, 2), g.shape, 1.0)
    gn, ok = warm.gn_gains(g1, d, m, a1, a2, len(g))
    ref, sing = diagonal.stefcal_jones_step(g1, d, m, a1, a2, len(g))
    assert ok.all() and not sing.any()
    np.testing.assert_allclose(gn, ref, rtol=1e-12, atol=1e-12)


def test_features_are_invariant_under_a_global_phase():
    """Rotating every input gain by one phase (a gauge change) leaves x unchanged and turns rot."""
    r = np.random.default_rng(3)
    n = 6
    hist = synth.jones_gains(synth.rng_for(4, 4), n * 4, 0.1, 0.05).reshape(n, 4, 2, 2)
    gn = hist[:, 0] + 0.01 * synth.complex_noise(synth.rng_for(4, 5), (n, 2, 2), 1.0)
    ok = np.ones(n, bool)
    lead = r.uniform(0, 1, n)
    x0, rot0 = warm.features(hist, gn, ok, lead)
    ph = np.exp(1j * 0.7)
    x1, rot1 = warm.features(hist * ph, gn * ph, ok, lead)
    np.testing.assert_allclose(x1, x0, atol=1e-12)
    np.testing.assert_allclose(rot1, rot0 * ph, atol=1e-12)
    # layout: the first 8 entries are g1 in its own frame, whose xx element is real and >= 0
    assert np.all(np.abs(x0[:, 1]) < 1e-12) and np.all(x0[:, 0] >= 0)
    np.testing.assert_allclose(x0[:, 40], lead)
    assert np.all(x0[:, 41:] == 0)


def test_target_and_proposal_are_inverse():
    """propose(g1, target(g1, g2, rot), rot) returns g2 for any rotation."""
    g1 = synth.jones_gains(synth.rng_for(5, 1), 7, 0.1, 0.05)
    g2 = synth.jones_gains(synth.rng_for(5, 2), 7, 0.1, 0.05)
    rot = np.exp(1j * np.linspace(-3, 3, 7))
    np.testing.assert_allclose(warm.propose(g1, warm.target(g1, g2, rot), rot), g2, atol=1e-13)


def test_singular_h_gives_zero_step():
    """An antenna with no data has H = 0: its step entries are zero, not NaN."""
    d, m, a1, a2, g = _tiny_jones(n_ant=4)
    keep = (a1 != 3) & (a2 != 3)
    gn, ok = warm.gn_gains(g, d[:, keep], m[:, keep], a1[keep], a2[keep], 4)
    assert not ok[3] and ok[:3].all()
    x, _ = warm.features(np.repeat(g[:, None], 4, axis=1), gn, ok, np.zeros(4))
    assert np.all(x[3, 32:40] == 0) and np.all(np.isfinite(x))


# ------------------------------------------------------------------------------------ selection

def test_chi2_difference_from_the_blocks():
    """chi^2(G) - sum |D|^2 = 1/2 sum_p [tr(G_p H_p G_p^H) - 2 Re tr(C_p G_p^H)] (brute force)."""
    d, m, a1, a2, g = _tiny_jones()
    G = g + 0.2 * synth.complex_noise(synth.rng_for(6, 1), g.shape, 1.0)
    b = blocks.jones_blocks(G, d, m, a1, a2, len(g))
    GH = np.conj(np.swapaxes(G, -1, -2))
    e = 0.5 * np.sum(np.real(np.trace(G @ b['H'] @ GH, axis1=1, axis2=2)) -
                     2.0 * np.real(np.trace(b['CD'] @ GH, axis1=1, axis2=2)))
    brute = diagonal.chi2_interval('jones', G, d, m, a1, a2) - np.sum(np.abs(d) ** 2)
    assert e == pytest.approx(brute, rel=1e-12, abs=1e-9)


def test_select_prefers_the_lower_chi2():
    d, m, a1, a2, g = _tiny_jones(noise=0.0)
    iv = dict(vis=d, model=m, ant1=a1, ant2=a2)
    far = g * np.exp(1j * 0.3) + 0.2
    start, used, dc = warm.select(iv, far, g)
    assert used and dc < 0 and np.allclose(start, g)
    start, used, dc = warm.select(iv, g, far)
    assert not used and dc > 0 and np.allclose(start, g)


def test_canonical_gauge():
    """sum tr(G) becomes real >= 0; chi^2 is unchanged; the result does not depend on the input phase."""
    d, m, a1, a2, g = _tiny_jones()
    c = warm.canonical_gauge(g)
    s = np.sum(c[:, 0, 0] + c[:, 1, 1])
    assert abs(s.imag) < 1e-12 and s.real > 0
    assert diagonal.chi2_interval('jones', c, d, m, a1, a2) == pytest.approx(
        diagonal.chi2_interval('jones', g, d, m, a1, a2), rel=1e-12)
    np.testing.assert_allclose(warm.canonical_gauge(g * np.exp(-2.1j)), c, atol=1e-13)
