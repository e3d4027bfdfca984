"""Pins of the oracle's direction-dependent methods beyond CohJones (CPU only).

Polarized DD (Sect. 4.4): the explicit Jacobian against Wirtinger finite differences and the
bilinear identity of eq. v_Jg:dd; the closed-form antenna blocks of eqs. JHJ:DD:pol / JHR:DD:pol
against the explicit products.  AllJones (Sect. 3.2.3, scalar and polarized) and polarized
CohJones: the special cases the paper's structure fixes (one direction is StefCal; diagonal
Jones matrices decouple into two scalar problems), noiseless recovery, and fixed points that are
stationary points of chi^2 (J^H r = 0).
"""
import numpy as np
import pytest

from oracle import blocks, diagonal, gauge, wirtinger
from paper_1502_06974_gb300 import synth


def _tiny_dd(kind, n_ant=4, n_samp=3, n_dir=2, seed=5, noise=0.0, pol=0.3):
    """Random DD problem: scalar m [Nd, N_s, N_bl] or 2x2 M [Nd, N_s, N_bl, 2, 2], true gains."""
    r = synth.rng_for(seed, 78)
    a1, a2 = synth.baseline_table(n_ant)
    nb = len(a1)
    if kind == 'dd':
        m = synth.complex_noise(r, (n_dir, n_samp, nb), 1.0)
        g = synth.scalar_gains(r, (n_ant, n_dir), 0.2)
        d = synth.simulate_dd(g, m, a1, a2)
    else:
        m = synth.complex_noise(r, (n_dir, n_samp, nb, 2, 2), pol)
        m += synth.complex_noise(r, (n_dir, n_samp, nb, 1, 1), 1.0) * np.eye(2)
        g = np.stack([synth.jones_gains(r, n_ant, 0.2, 0.1) for _ in range(n_dir)], axis=1)
        d = wirtinger.model_dd_jones(g, m, a1, a2)
    d = d + synth.complex_noise(r, d.shape, noise)
    return d, m, a1, a2, g


def _start(kind, g, eps=0.1, seed=3):
    return g + eps * synth.complex_noise(synth.rng_for(seed, 2), g.shape, 1.0)


def _unit(kind, n_ant, n_dir):
    if kind == 'dd':
        return np.ones((n_ant, n_dir), complex)
    return np.tile(np.eye(2, dtype=complex), (n_ant, n_dir, 1, 1))


# ------------------------------------------------------------------------------------ polarized DD J

def test_dd_jones_jacobian_matches_wirtinger_finite_differences():
    d, m, a1, a2, g = _tiny_dd('dd_jones', n_ant=3, n_samp=2, n_dir=2)
    prob = wirtinger.Problem('dd_jones', d, m, a1, a2, 3, n_dir=2)
    g0 = _start('dd_jones', g, eps=0.3)
    Jk, Jc = prob.partials(g0)
    z = prob.to_z(g0)
    h = 1e-6

    def v(zz):
        return wirtinger.vec2(prob.model_vis(prob.from_z(zz))).reshape(-1)

    for j in range(z.shape[0]):
        e = np.zeros_like(z); e[j] = h
        dx = (v(z + e) - v(z - e)) / (2 * h)
        dy = (v(z + 1j * e) - v(z - 1j * e)) / (2 * h)
        np.testing.assert_allclose(Jk[:, j], 0.5 * (dx - 1j * dy), atol=1e-7)
        np.testing.assert_allclose(Jc[:, j], 0.5 * (dx + 1j * dy), atol=1e-7)


def test_dd_jones_model_is_left_jacobian_times_gains():
    """eq. v_Jg:dd in the polarized form: V = J_L G (bilinearity)."""
    d, m, a1, a2, g = _tiny_dd('dd_jones')
    prob = wirtinger.Problem('dd_jones', d, m, a1, a2, 4, n_dir=2)
    Jk, _ = prob.partials(g)
    np.testing.assert_allclose(Jk @ prob.to_z(g), wirtinger.vec2(prob.model_vis(g)).reshape(-1), atol=1e-12)


def test_dd_jones_closed_forms_equal_explicit_products():
    """eq. JHJ:DD:pol top-left: in CAD order block-diagonal over antennas; the (c, d) 4x4 block of
    antenna p is (H_p[d, c])^T kron I with H_p[d, c] = sum Y^(d) Y^(c)H (the operator R of App. B);
    eq. JHR:DD:pol top: vec(sum R Y^(d)H)."""
    nd, n = 2, 4
    d, m, a1, a2, g = _tiny_dd('dd_jones', n_ant=n, n_samp=2, n_dir=nd, noise=0.1)
    g0 = _start('dd_jones', g, eps=0.2)
    prob = wirtinger.Problem('dd_jones', d, m, a1, a2, n, n_dir=nd)
    H, b = prob.normal_equations(g0)
    cf = blocks.dd_jones_blocks(g0, d, m, a1, a2, n)
    I2 = np.eye(2)
    for p in range(n):
        for q in range(n):
            for c in range(nd):
                for e in range(nd):
                    r0, c0 = 4 * (p * nd + c), 4 * (q * nd + e)
                    blk = H[r0:r0 + 4, c0:c0 + 4]
                    if p != q:
                        assert np.all(blk == 0)
                        continue
                    Hde = cf['H'][p, 2 * e:2 * e + 2, 2 * c:2 * c + 2]
                    np.testing.assert_allclose(blk, np.kron(Hde.T, I2), atol=1e-12)
        for e in range(nd):
            r0 = 4 * (p * nd + e)
            np.testing.assert_allclose(b[r0:r0 + 4], wirtinger.vec2(cf['C'][p][:, 2 * e:2 * e + 2]), atol=1e-12)
    # data form: C = CD - [G^(1) .. G^(Nd)] H (eq. v_Jg:dd summed against Y^H)
    for p in range(n):
        X = np.concatenate(list(g0[p]), axis=1)
        np.testing.assert_allclose(cf['C'][p], cf['CD'][p] - X @ cf['H'][p], atol=1e-12)


# ------------------------------------------------------------------------------------ special cases

def test_alljones_single_direction_is_stefcal():
    """N_d = 1: the diagonal of J^H J is StefCal's, and the residual-form step equals eq. stefcal."""
    r = synth.rng_for(6, 6)
    a1, a2 = synth.baseline_table(6)
    m = synth.complex_noise(r, (3, len(a1)), 1.0) + 2.0
    d = synth.simulate_scalar(synth.scalar_gains(r, 6, 0.2), m, a1, a2) + synth.complex_noise(r, m.shape, 0.1)
    s = diagonal.iterate('scalar', np.ones(6, complex), d, m, a1, a2, 6, tol=0.0, max_iter=10, record=True)
    a = diagonal.iterate('dd', np.ones((6, 1), complex), d, m[None], a1, a2, 6, tol=0.0, max_iter=10,
                         record=True, method='alljones')
    for x, y in zip(s['history'], a['history']):
        np.testing.assert_allclose(y[:, 0], x, rtol=1e-11)


@pytest.mark.parametrize("method", ['cohjones', 'alljones'])
def test_dd_jones_single_direction_is_polarized_stefcal(method):
    d, m, a1, a2, g = _tiny_dd('dd_jones', n_ant=5, n_samp=3, n_dir=1, noise=0.1)
    G0 = np.tile(np.eye(2, dtype=complex), (5, 1, 1))
    s = diagonal.iterate('jones', G0, d, m[0], a1, a2, 5, tol=0.0, max_iter=8, record=True)
    t = diagonal.iterate('dd_jones', G0[:, None], d, m, a1, a2, 5, tol=0.0, max_iter=8, record=True, method=method)
    for x, y in zip(s['history'], t['history']):
        np.testing.assert_allclose(y[:, 0], x, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("method", ['cohjones', 'alljones'])
def test_diagonal_dd_jones_is_two_scalar_dd_problems(method):
    """Diagonal models and a diagonal start: the polarized DD step decouples into the xx and yy
    scalar DD steps of the same method."""
    dx, mx, a1, a2, _ = _tiny_dd('dd', n_ant=5, n_samp=4, n_dir=2, seed=21, noise=0.05)
    dy, my, _, _, _ = _tiny_dd('dd', n_ant=5, n_samp=4, n_dir=2, seed=22, noise=0.05)
    D = np.zeros(dx.shape + (2, 2), complex); M = np.zeros(mx.shape + (2, 2), complex)
    D[..., 0, 0], D[..., 1, 1] = dx, dy
    M[..., 0, 0], M[..., 1, 1] = mx, my
    J = diagonal.iterate('dd_jones', _unit('dd_jones', 5, 2), D, M, a1, a2, 5, tol=0.0, max_iter=6, method=method)
    x = diagonal.iterate('dd', _unit('dd', 5, 2), dx, mx, a1, a2, 5, tol=0.0, max_iter=6, method=method)
    y = diagonal.iterate('dd', _unit('dd', 5, 2), dy, my, a1, a2, 5, tol=0.0, max_iter=6, method=method)
    np.testing.assert_allclose(J['g'][..., 0, 0], x['g'], rtol=1e-11)
    np.testing.assert_allclose(J['g'][..., 1, 1], y['g'], rtol=1e-11)
    assert np.all(J['g'][..., 0, 1] == 0) and np.all(J['g'][..., 1, 0] == 0)


def test_alljones_data_form_shortcut_does_not_hold():
    """Sect. 3.2.3: with the fully diagonal J^H J eq. ghat:precise fails, so g + A^-1 J^H r differs
    from the data form A^-1 J^H d: the residual form is required."""
    d, m, a1, a2, g = _tiny_dd('dd', n_ant=5, n_samp=3, n_dir=2, noise=0.1)
    g0 = _start('dd', g, eps=0.2)
    b = blocks.dd_blocks(g0, d, m, a1, a2, 5)
    a = np.real(np.diagonal(b['A'], axis1=1, axis2=2))
    assert np.max(np.abs((g0 + b['c'] / a) - b['cd'] / a)) > 1e-2


# ------------------------------------------------------------------------------------ solutions

@pytest.mark.parametrize("kind,method", [('dd', 'alljones'), ('dd_jones', 'cohjones'), ('dd_jones', 'alljones')])
def test_noiseless_recovery(kind, method):
    d, m, a1, a2, g = _tiny_dd(kind, n_ant=6, n_samp=12, n_dir=2, seed=8)
    it = diagonal.iterate(kind, _start(kind, g, eps=0.05), d, m, a1, a2, 6, tol=1e-14, max_iter=20000, method=method)
    assert it['converged']
    assert gauge.rel_error(kind, it['g'], g) < 1e-8


@pytest.mark.parametrize("kind,method", [('dd', 'alljones'), ('dd_jones', 'cohjones'), ('dd_jones', 'alljones')])
def test_fixed_point_is_stationary_point_of_chi2(kind, method):
    """A fixed point of the method has J^H r = 0 on the explicit Jacobian (noisy data), the
    stationary point full GN reaches from there."""
    d, m, a1, a2, g = _tiny_dd(kind, n_ant=6, n_samp=12, n_dir=2, seed=9, noise=0.05)
    it = diagonal.iterate(kind, _unit(kind, 6, 2), d, m, a1, a2, 6, tol=1e-13, max_iter=50000, method=method)
    assert it['converged']
    prob = wirtinger.Problem(kind, d, m, a1, a2, 6, n_dir=2)
    _, b = prob.normal_equations(it['g'])
    _, b0 = prob.normal_equations(_unit(kind, 6, 2))
    assert np.linalg.norm(b) < 1e-9 * np.linalg.norm(b0)
    g_gn, _, _ = wirtinger.gauss_newton(prob, it['g'], tol=1e-14)
    assert gauge.rel_error(kind, it['g'], g_gn) < 1e-9
