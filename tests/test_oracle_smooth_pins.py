"""Pins of the smoothing oracle (Sect. 3.4, eqs. stefcal:w, JHJ:diag:smooth) (CPU only).

A zero-width kernel converges to every sample's own StefCal solution (one-sample intervals); a
flat kernel over the whole grid converges to StefCal's solution of the grid as one solution interval
(Sect. 2.3) -- both compared in the canonical phase gauge; the convolution
equals scipy's 2-D convolution with the outer-product kernel; the true gains of a noiseless
observation are a fixed point for any kernel and are recovered from a perturbed start; the taps
are the Gaussian's values.
"""
import numpy as np
import pytest

from oracle import diagonal, smooth
from paper_1502_06974_gb300 import synth


def _grid(kind, nt=5, nf=4, n_ant=5, seed=3, noise=0.05, const=False):
    r = synth.rng_for(seed, 66)
    a1, a2 = synth.baseline_table(n_ant)
    nb = len(a1)
    if kind == 'scalar':
        m = synth.complex_noise(r, (nt, nf, nb), 1.0) + 2.0
        g = synth.scalar_gains(r, (nt, nf, n_ant), 0.2)
        if const:
            g[:] = g[0, 0]
        d = g[:, :, a1] * m * np.conj(g[:, :, a2])
    else:
        m = synth.complex_noise(r, (nt, nf, nb, 2, 2), 0.3)
        m[..., 0, 0] += 2.0; m[..., 1, 1] += 2.0
        g = synth.jones_gains(r, nt * nf * n_ant, 0.2, 0.1).reshape(nt, nf, n_ant, 2, 2)
        if const:
            g[:] = g[0, 0]
        d = g[:, :, a1] @ m @ np.conj(np.swapaxes(g[:, :, a2], -1, -2))
    d = d + synth.complex_noise(r, d.shape, noise)
    return d, m, a1, a2, g


def _unit(kind, nt, nf, n):
    return np.ones((nt, nf, n), complex) if kind == 'scalar' else np.tile(np.eye(2, dtype=complex), (nt, nf, n, 1, 1))


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_canonical_phase_removes_only_a_common_phase(kind):
    d, m, a1, a2, g = _grid(kind)
    c = smooth.canonical_phase(kind, g)
    S = np.sum(c, axis=2) if kind == 'scalar' else np.sum(np.trace(c, axis1=-2, axis2=-1), axis=2)
    assert np.all(np.abs(S.imag) < 1e-12 * np.abs(S)) and np.all(S.real >= 0)
    ratio = (c / g).reshape(5, 4, -1)
    np.testing.assert_allclose(ratio, ratio[:, :, :1] * np.ones_like(ratio), rtol=1e-12)
    np.testing.assert_allclose(np.abs(ratio), 1.0, rtol=1e-12)


def test_gaussian_taps():
    w = smooth.gaussian_taps(1.5)
    x = np.arange(-5, 6)
    np.testing.assert_allclose(w, np.exp(-x ** 2 / 4.5), rtol=1e-15)
    assert list(smooth.gaussian_taps(0.0)) == [1.0]


def test_convolution_equals_library_convolution():
    from scipy.signal import convolve2d
    x = synth.complex_noise(synth.rng_for(1, 1), (7, 6), 1.0)
    wt, wf = smooth.gaussian_taps(1.2), smooth.gaussian_taps(0.7)
    np.testing.assert_allclose(smooth.convolve(x, wt, wf), convolve2d(x, np.outer(wt, wf), mode='same'), atol=1e-12)


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_zero_width_kernel_solves_each_sample_alone(kind):
    d, m, a1, a2, g = _grid(kind)
    it = smooth.iterate_smooth(kind, _unit(kind, 5, 4, 5), d, m, a1, a2, 5, 0.0, 0.0, tol=1e-13, max_iter=20000)
    assert it['converged']
    for t in range(5):
        for f in range(4):
            r = diagonal.iterate(kind, _unit(kind, 5, 4, 5)[t, f], d[t, f][None], m[t, f][None], a1, a2, 5, tol=1e-13,
                                 max_iter=20000)
            ref = smooth.canonical_phase(kind, r['g'][None, None])[0, 0]
            got = smooth.canonical_phase(kind, it['g'][t:t + 1, f:f + 1])[0, 0]
            np.testing.assert_allclose(got, ref, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_flat_kernel_is_one_solution_interval(kind):
    d, m, a1, a2, g = _grid(kind, const=True)       # one set of gains over the grid, noisy data
    taps = (np.ones(2 * 5 - 1), np.ones(2 * 4 - 1))
    it = smooth.iterate_smooth(kind, _unit(kind, 5, 4, 5), d, m, a1, a2, 5, 0.0, 0.0, tol=1e-13, max_iter=20000,
                               taps=taps)
    assert it['converged']
    r = diagonal.iterate(kind, _unit(kind, 5, 4, 5)[0, 0], d.reshape((20,) + d.shape[2:]),
                         m.reshape((20,) + m.shape[2:]), a1, a2, 5, tol=1e-13, max_iter=20000)
    ref = smooth.canonical_phase(kind, r['g'][None, None])[0, 0]
    got = smooth.canonical_phase(kind, it['g'])
    for t in range(5):
        for f in range(4):
            np.testing.assert_allclose(got[t, f], ref, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_noiseless_constant_gains_are_recovered(kind):
    d, m, a1, a2, g = _grid(kind, noise=0.0, const=True)
    wt, wf = smooth.gaussian_taps(1.0), smooth.gaussian_taps(1.0)
    gn = smooth.smooth_step(kind, g, d, m, a1, a2, 5, wt, wf)
    np.testing.assert_allclose(gn, g, rtol=1e-12, atol=1e-12)
    ga = smooth.align_phase(kind, g * np.exp(0.3j), g)   # the alignment undoes a common phase
    np.testing.assert_allclose(ga, g, rtol=1e-12, atol=1e-12)
    start = g + 0.05 * synth.complex_noise(synth.rng_for(2, 2), g.shape, 1.0)
    it = smooth.iterate_smooth(kind, start, d, m, a1, a2, 5, 1.0, 1.0, tol=1e-13, max_iter=3000)
    assert it['converged']
    np.testing.assert_allclose(smooth.canonical_phase(kind, it['g']), smooth.canonical_phase(kind, g), rtol=1e-8,
                               atol=1e-10)
