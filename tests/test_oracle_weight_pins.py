"""Pins of the oracle's per-row weights (Sect. 2.4, eqs. LSmin:w, LM:W, JHJ:DI:tfw, JHR:DI:tfw)
against definitions that do not use them (CPU only).

An integer weight k on every row of a sample is the same as that sample repeated k times (zero:
the sample removed); zero weights on every row of one baseline are the same as the baseline
removed; the weighted closed forms equal J^H W J and J^H W r of the explicit Jacobian; a fixed
point of the weighted iteration is a stationary point of the weighted chi^2 (finite differences).
"""
import numpy as np
import pytest

from oracle import blocks, diagonal, gauge, wirtinger
from paper_1502_06974_gb300 import synth


def _data(kind, n_ant=5, n_samp=4, seed=3, noise=0.1):
    r = synth.rng_for(seed, 55)
    a1, a2 = synth.baseline_table(n_ant)
    nb = len(a1)
    if kind == 'scalar':
        m = synth.complex_noise(r, (n_samp, nb), 1.0) + 2.0
        d = synth.simulate_scalar(synth.scalar_gains(r, n_ant, 0.2), m, a1, a2)
    else:
        m = synth.complex_noise(r, (n_samp, nb, 2, 2), 0.3)
        m[..., 0, 0] += 2.0; m[..., 1, 1] += 2.0
        d = synth.simulate_jones(synth.jones_gains(r, n_ant, 0.2, 0.1), m, a1, a2)
    d = d + synth.complex_noise(r, d.shape, noise)
    return d, m, a1, a2


def _unit(kind, n):
    return np.ones(n, complex) if kind == 'scalar' else np.tile(np.eye(2, dtype=complex), (n, 1, 1))


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_integer_sample_weights_equal_repeated_samples(kind):
    d, m, a1, a2 = _data(kind)
    ws = np.array([2, 0, 1, 3])                              # per sample
    w = np.repeat(ws[:, None], len(a1), axis=1).astype(float)
    rep = np.repeat(np.arange(4), ws)
    g0 = _unit(kind, 5)
    fn = blocks.scalar_blocks if kind == 'scalar' else blocks.jones_blocks
    bw = fn(g0 * 1.1, d, m, a1, a2, 5, w)
    br = fn(g0 * 1.1, d[rep], m[rep], a1, a2, 5)
    for key in bw:
        np.testing.assert_allclose(bw[key], br[key], rtol=1e-12, atol=1e-12)
    itw = diagonal.iterate(kind, g0, d, m, a1, a2, 5, tol=0.0, max_iter=6, weights=w)
    itr = diagonal.iterate(kind, g0, d[rep], m[rep], a1, a2, 5, tol=0.0, max_iter=6)
    np.testing.assert_allclose(itw['g'], itr['g'], rtol=1e-11)
    np.testing.assert_allclose(diagonal.chi2_interval(kind, itw['g'], d, m, a1, a2, w),
                               diagonal.chi2_interval(kind, itw['g'], d[rep], m[rep], a1, a2), rtol=1e-12)


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_zero_weights_on_a_baseline_remove_it(kind):
    d, m, a1, a2 = _data(kind, n_ant=6)
    drop = 4
    w = np.ones((d.shape[0], len(a1)))
    w[:, drop] = 0.0
    keep = np.delete(np.arange(len(a1)), drop)
    g0 = _unit(kind, 6)
    itw = diagonal.iterate(kind, g0, d, m, a1, a2, 6, tol=0.0, max_iter=5, weights=w)
    itr = diagonal.iterate(kind, g0, d[:, keep], m[:, keep], a1[keep], a2[keep], 6, tol=0.0, max_iter=5)
    np.testing.assert_allclose(itw['g'], itr['g'], rtol=1e-11)


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_weighted_closed_forms_equal_explicit_products(kind):
    """Whole J^H W J and J^H W r of the explicit Jacobian (eq. LM:W) against the closed forms."""
    d, m, a1, a2 = _data(kind, n_ant=4, n_samp=3)
    w = synth.rng_for(4, 4).uniform(0.0, 2.0, (3, len(a1)))
    g0 = _unit(kind, 4) * (1.0 + 0.2j)
    ex = wirtinger.Problem(kind, d, m, a1, a2, 4, weights=w)
    cf = wirtinger.ClosedFormProblem(kind, d, m, a1, a2, 4, weights=w)
    He, be = ex.normal_equations(g0)
    Hc, bc = cf.normal_equations(g0)
    np.testing.assert_allclose(Hc, He, atol=1e-11)
    np.testing.assert_allclose(bc, be, atol=1e-11)
    # and it is not the unweighted product
    Hu, _ = wirtinger.Problem(kind, d, m, a1, a2, 4).normal_equations(g0)
    assert np.max(np.abs(Hu - He)) > 1e-3


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_weighted_fixed_point_is_stationary_point_of_weighted_chi2(kind):
    d, m, a1, a2 = _data(kind, n_ant=5, n_samp=4, noise=0.2)
    w = synth.rng_for(5, 5).uniform(0.2, 3.0, (4, len(a1)))
    it = diagonal.iterate(kind, _unit(kind, 5), d, m, a1, a2, 5, tol=1e-13, max_iter=50000, weights=w)
    assert it['converged']
    prob = wirtinger.Problem(kind, d, m, a1, a2, 5, weights=w)
    g = it['g']
    h = 1e-6
    z = prob.to_z(g)
    grad = np.zeros(z.shape, complex)
    for k in range(z.shape[0]):
        e = np.zeros_like(z); e[k] = h
        dx = (prob.chi2(prob.from_z(z + e)) - prob.chi2(prob.from_z(z - e))) / (2 * h)
        dy = (prob.chi2(prob.from_z(z + 1j * e)) - prob.chi2(prob.from_z(z - 1j * e))) / (2 * h)
        grad[k] = 0.5 * (dx + 1j * dy)
    assert np.max(np.abs(grad)) < 1e-6 * prob.chi2(g)
    # the unweighted fixed point is a different point
    itu = diagonal.iterate(kind, _unit(kind, 5), d, m, a1, a2, 5, tol=1e-13, max_iter=50000)
    assert gauge.rel_error(kind, itu['g'], g) > 1e-4


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_weighted_closed_form_lm_reaches_the_weighted_fixed_point(kind):
    d, m, a1, a2 = _data(kind, n_ant=5, n_samp=4, noise=0.2)
    w = synth.rng_for(6, 6).uniform(0.2, 3.0, (4, len(a1)))
    it = diagonal.iterate(kind, _unit(kind, 5), d, m, a1, a2, 5, tol=1e-13, max_iter=50000, weights=w)
    prob = wirtinger.ClosedFormProblem(kind, d, m, a1, a2, 5, weights=w)
    g, _, hist = wirtinger.levenberg_marquardt(prob, _unit(kind, 5), tol=1e-13, max_iter=400, lam0=1e-2, K=10.0,
                                               gauge=True)
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    assert gauge.rel_error(kind, g, it['g']) < 1e-8
