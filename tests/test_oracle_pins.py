"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties one part of the oracle to something other than itself: Wirtinger finite
differences, the printed structure of the 3-antenna example and of the 4x4 operator forms,
exact identities, closed forms of special cases, brute force on tiny problems.
"""
import os
import re

import numpy as np
import pytest

from oracle import blocks, diagonal, gauge, wirtinger
from paper_1502_06974_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')


def _tiny(kind, n_ant=4, n_samp=3, n_dir=2, seed=5, noise=0.0, pol=0.3):
    """Small random problem: vis, model ([N_s, N_bl] / [Nd, N_s, N_bl] / [N_s, N_bl, 2, 2]), tables, true gains."""
    r = synth.rng_for(seed, 77)
    a1, a2 = synth.baseline_table(n_ant)
    nb = len(a1)
    if kind == 'scalar':
        m = synth.complex_noise(r, (n_samp, nb), 1.0) + 2.0
        g = synth.scalar_gains(r, n_ant, 0.2)
        d = synth.simulate_scalar(g, m, a1, a2)
    elif kind == 'dd':
        m = synth.complex_noise(r, (n_dir, n_samp, nb), 1.0)
        g = synth.scalar_gains(r, (n_ant, n_dir), 0.2)
        d = synth.simulate_dd(g, m, a1, a2)
    else:
        m = synth.complex_noise(r, (n_samp, nb, 2, 2), pol)
        m[..., 0, 0] += 2.0; m[..., 1, 1] += 2.0
        g = synth.jones_gains(r, n_ant, 0.2, 0.1)
        d = synth.simulate_jones(g, m, a1, a2)
    d = d + synth.complex_noise(r, d.shape, noise)
    return d, m, a1, a2, g


def _perturbed_start(kind, g, seed=3, eps=0.3):
    r = synth.rng_for(seed, 1)
    return g + eps * synth.complex_noise(r, g.shape, 1.0)


# ------------------------------------------------------------------------------------ Jacobians

@pytest.mark.parametrize("kind", ['scalar', 'dd', 'jones'])
def test_jacobian_matches_wirtinger_finite_differences(kind):
    """J_k = dv/dz = (dv/dx - i dv/dy)/2 and J_k* = dv/dconj(z) = (dv/dx + i dv/dy)/2 (Sect. 1)."""
    d, m, a1, a2, g = _tiny(kind, n_ant=4, n_samp=2)
    prob = wirtinger.Problem(kind, d, m, a1, a2, 4, n_dir=2)
    g0 = _perturbed_start(kind, g)
    Jk, Jc = prob.partials(g0)
    z = prob.to_z(g0)
    h = 1e-6

    def v(zz):
        x = prob.model_vis(prob.from_z(zz))
        return wirtinger.vec2(x).reshape(-1) if kind == 'jones' else x.reshape(-1)

    for j in range(z.shape[0]):
        e = np.zeros_like(z); e[j] = h
        dx = (v(z + e) - v(z - e)) / (2 * h)
        dy = (v(z + 1j * e) - v(z - 1j * e)) / (2 * h)
        np.testing.assert_allclose(Jk[:, j], 0.5 * (dx - 1j * dy), atol=1e-7)
        np.testing.assert_allclose(Jc[:, j], 0.5 * (dx + 1j * dy), atol=1e-7)


@pytest.mark.parametrize("kind", ['scalar', 'dd', 'jones'])
def test_model_is_half_J_times_augmented_gains(kind):
    """eq. v_Jg / v_Jg:dd: v = J_L g = (1/2) J [g; conj g] (bilinearity)."""
    d, m, a1, a2, g = _tiny(kind)
    prob = wirtinger.Problem(kind, d, m, a1, a2, 4, n_dir=2)
    J = prob.jacobian(g)
    z = prob.to_z(g)
    v_top = (0.5 * J @ np.concatenate([z, np.conj(z)]))[: J.shape[0] // 2]
    vm = prob.model_vis(g)
    vm = wirtinger.vec2(vm).reshape(-1) if kind == 'jones' else vm.reshape(-1)
    np.testing.assert_allclose(v_top, vm, rtol=1e-12, atol=1e-12)
    Jk, _ = prob.partials(g)
    np.testing.assert_allclose(Jk @ z, vm, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind", ['scalar', 'dd', 'jones'])
def test_jhj_hermitian_psd_with_gauge_null_space(kind):
    """J^H J is Hermitian PSD (Sect. 2.1) and annihilates the phase-gauge direction(s)."""
    d, m, a1, a2, g = _tiny(kind, noise=0.05)
    prob = wirtinger.Problem(kind, d, m, a1, a2, 4, n_dir=2)
    g0 = _perturbed_start(kind, g)
    H, _ = prob.normal_equations(g0)
    np.testing.assert_allclose(H, H.conj().T, atol=1e-12)
    w = np.linalg.eigvalsh(H)
    assert w.min() >= -1e-10 * w.max()
    J = prob.jacobian(g0)
    z = prob.to_z(g0)
    if kind == 'dd':
        for dd in range(2):
            zz = np.zeros_like(z).reshape(4, 2); zz[:, dd] = z.reshape(4, 2)[:, dd]
            zz = zz.reshape(-1)
            u = np.concatenate([1j * zz, -1j * np.conj(zz)])
            assert np.linalg.norm(J @ u) < 1e-10 * np.linalg.norm(J) * np.linalg.norm(u)
    else:
        u = np.concatenate([1j * z, -1j * np.conj(z)])
        assert np.linalg.norm(J @ u) < 1e-10 * np.linalg.norm(J) * np.linalg.norm(u)


def _eval_3ant(token, y, r):
    if token == '0':
        return 0.0
    mm = re.fullmatch(r'S\((\d)(\d),(\d)(\d)\)', token)
    if mm:
        i, j, k, l = (int(c) for c in mm.groups())
        return abs(y[i, j]) ** 2 + abs(y[k, l]) ** 2
    mm = re.fullmatch(r'(Bc|B)\((\d),(\d)\)', token)
    if mm:
        i, j = int(mm.group(2)), int(mm.group(3))
        v = y[i, j] * y[j, i]
        return np.conj(v) if mm.group(1) == 'Bc' else v
    mm = re.fullmatch(r'(Cc|C)\((\d)(\d),(\d)(\d)\)', token)
    if mm:
        i, j, k, l = (int(c) for c in mm.groups()[1:])
        v = np.conj(y[i, j]) * r[i, j] + np.conj(y[k, l]) * r[k, l]
        return np.conj(v) if mm.group(1) == 'Cc' else v
    raise ValueError(token)


def _read_pattern(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith('#'):
            rows.append(line.split())
    return rows


def test_three_antenna_example_structure():
    """App. A: every entry of the explicit J^H J and J^H r equals the printed pattern."""
    d, m, a1, a2, g = _tiny('scalar', n_ant=3, n_samp=1, noise=0.1)
    g0 = _perturbed_start('scalar', g)
    prob = wirtinger.Problem('scalar', d, m, a1, a2, 3)
    H, b = prob.normal_equations(g0)
    # y_pq with 1-based indices, both orientations; r likewise
    y = {}; rr = {}
    res = (d - prob.model_vis(g0))[0]
    for bl, (p, q) in enumerate(zip(a1, a2)):
        y[p + 1, q + 1] = m[0, bl] * np.conj(g0[q]); y[q + 1, p + 1] = np.conj(m[0, bl]) * np.conj(g0[p])
        rr[p + 1, q + 1] = res[bl]; rr[q + 1, p + 1] = np.conj(res[bl])
    pat = _read_pattern('jhj_3ant_pattern.txt')
    expect = np.array([[_eval_3ant(t, y, rr) for t in row] for row in pat], dtype=np.complex128)
    np.testing.assert_allclose(H, expect, atol=1e-12)
    assert np.all(H[expect == 0] == 0)          # structural zeros are exact
    pr = _read_pattern('jhr_3ant_pattern.txt')
    np.testing.assert_allclose(b, np.array([_eval_3ant(row[0], y, rr) for row in pr]), atol=1e-12)


def test_operator_4x4_forms_and_identities():
    """App. B eq. RA4x4 / LA4x4 (printed patterns) represent X -> XA and X -> AX on vec X, and
    eq. RAB:LAB, eq. RH:LH hold."""
    pat = _read_pattern('operator_4x4.txt')
    r = synth.rng_for(1, 2)
    A, B, X = (synth.complex_noise(r, (2, 2), 1.0) for _ in range(3))
    el = {'a11': A[0, 0], 'a12': A[0, 1], 'a21': A[1, 0], 'a22': A[1, 1], '0': 0.0}
    i = pat.index(['R']); j = pat.index(['L'])
    WR = np.array([[el[t] for t in row] for row in pat[i + 1:i + 5]])
    WL = np.array([[el[t] for t in row] for row in pat[j + 1:j + 5]])
    vec = wirtinger.vec2
    np.testing.assert_allclose(WR @ vec(X), vec(X @ A), atol=1e-13)
    np.testing.assert_allclose(WL @ vec(X), vec(A @ X), atol=1e-13)
    I2 = np.eye(2)
    np.testing.assert_allclose(WR, np.kron(A.T, I2), atol=1e-14)       # the form partials_jones uses
    np.testing.assert_allclose(WL, np.kron(I2, A), atol=1e-14)
    R = lambda M: np.kron(M.T, I2)
    L = lambda M: np.kron(I2, M)
    np.testing.assert_allclose(R(A) @ R(B), R(B @ A), atol=1e-13)
    np.testing.assert_allclose(L(A) @ L(B), L(A @ B), atol=1e-13)
    np.testing.assert_allclose(R(A).conj().T, R(A.conj().T), atol=1e-14)
    np.testing.assert_allclose(L(A).conj().T, L(A.conj().T), atol=1e-14)
    np.testing.assert_allclose(np.linalg.inv(R(A)), R(np.linalg.inv(A)), atol=1e-12)


# ------------------------------------------------------------------------------------ closed forms

def test_scalar_closed_forms_equal_explicit_products():
    """eqs. JHJ:DI:tf and JHR:DI:tf against J^H J and J^H r built from the explicit J."""
    d, m, a1, a2, g = _tiny('scalar', n_ant=5, n_samp=3, noise=0.1)
    g0 = _perturbed_start('scalar', g)
    prob = wirtinger.Problem('scalar', d, m, a1, a2, 5)
    H, b = prob.normal_equations(g0)
    cf = blocks.scalar_blocks(g0, d, m, a1, a2, 5)
    n = 5
    np.testing.assert_allclose(np.real(np.diag(H[:n, :n])), cf['A'], rtol=1e-12)
    assert np.allclose(H[:n, :n] - np.diag(np.diag(H[:n, :n])), 0, atol=1e-12)   # A is diagonal
    np.testing.assert_allclose(H[:n, n:], cf['B'], atol=1e-12)
    np.testing.assert_allclose(H[n:, :n], np.conj(cf['B']), atol=1e-12)           # C = conj(B)
    np.testing.assert_allclose(H[n:, n:], H[:n, :n], atol=1e-12)                  # D = A
    np.testing.assert_allclose(cf['B'], cf['B'].T, atol=1e-12)
    np.testing.assert_allclose(b[:n], cf['c'], atol=1e-12)
    np.testing.assert_allclose(b[n:], np.conj(cf['c']), atol=1e-12)


def test_dd_closed_forms_and_cad_block_structure():
    """eqs. JHJ:DD:unpol / JHR:DD:unpol; in CAD order the top-left block is N_d x N_d block-diagonal."""
    d, m, a1, a2, g = _tiny('dd', n_ant=4, n_samp=3, n_dir=2, noise=0.1)
    g0 = _perturbed_start('dd', g)
    prob = wirtinger.Problem('dd', d, m, a1, a2, 4, n_dir=2)
    H, b = prob.normal_equations(g0)
    cf = blocks.dd_blocks(g0, d, m, a1, a2, 4)
    nd, n = 2, 4
    UL = H[:n * nd, :n * nd]
    for p in range(n):
        for q in range(n):
            blk = UL[p * nd:(p + 1) * nd, q * nd:(q + 1) * nd]
            if p == q:
                np.testing.assert_allclose(blk, cf['A'][p], atol=1e-12)
            else:
                assert np.all(blk == 0)
    np.testing.assert_allclose(b[:n * nd], cf['c'].reshape(-1), atol=1e-12)


def test_jones_closed_forms_and_product_order():
    """eq. JHJ:pol diagonal = R_{sum Y Y^H} (4x4: H^T kron I) and J^H R top = vec(sum R Y^H).

    The printed order Y^H R (eq. JHR pol and eq. update:DI:diag:pol) does not reproduce the
    explicit product; R Y^H, which follows from R_A X = X A, does.
    """
    d, m, a1, a2, g = _tiny('jones', n_ant=4, n_samp=2, noise=0.1)
    g0 = _perturbed_start('jones', g)
    prob = wirtinger.Problem('jones', d, m, a1, a2, 4)
    H, b = prob.normal_equations(g0)
    cf = blocks.jones_blocks(g0, d, m, a1, a2, 4)
    for p in range(4):
        np.testing.assert_allclose(H[4 * p:4 * p + 4, 4 * p:4 * p + 4], np.kron(cf['H'][p].T, np.eye(2)), atol=1e-12)
        np.testing.assert_allclose(b[4 * p:4 * p + 4], wirtinger.vec2(cf['C'][p]), atol=1e-12)
    # the literal printed order fails
    i, j, D, M = blocks.directed_rows(d, m, a1, a2, 'jones')
    Y = M @ np.conj(np.swapaxes(g0[j], -1, -2))
    R = D - g0[i] @ Y
    lit = np.zeros((4, 2, 2), complex)
    np.add.at(lit, i, np.conj(np.swapaxes(Y, -1, -2)) @ R)
    assert np.max(np.abs(wirtinger.vec2(lit).reshape(-1) - b[:16])) > 1e-3


def test_gradient_of_chi2_is_minus_jhr():
    """d chi^2 / d conj(G_p) = -sum_q R_pq Y_pq^H (finite differences on chi^2)."""
    d, m, a1, a2, g = _tiny('jones', n_ant=4, n_samp=2, noise=0.1)
    g0 = _perturbed_start('jones', g)
    prob = wirtinger.Problem('jones', d, m, a1, a2, 4)
    cf = blocks.jones_blocks(g0, d, m, a1, a2, 4)
    h = 1e-6
    for p in range(4):
        for (u, v) in ((0, 0), (0, 1), (1, 0), (1, 1)):
            e = np.zeros_like(g0); e[p, u, v] = h
            dx = (prob.chi2(g0 + e) - prob.chi2(g0 - e)) / (2 * h)
            dy = (prob.chi2(g0 + 1j * e) - prob.chi2(g0 - 1j * e)) / (2 * h)
            dconj = 0.5 * (dx + 1j * dy)
            assert abs(dconj + cf['C'][p, u, v]) < 1e-6 * max(1.0, abs(cf['C'][p, u, v]))


# ------------------------------------------------------------------------------------ solvers

@pytest.mark.parametrize("kind", ['scalar', 'dd', 'jones'])
def test_noiseless_recovery_all_solvers(kind):
    """With noiseless data the true gains are a zero-residual minimum (Sect. 2.1): GN, LM and the
    diagonal iteration recover them up to the phase gauge."""
    d, m, a1, a2, g = _tiny(kind, n_ant=5, n_samp=3, n_dir=2)
    prob = wirtinger.Problem(kind, d, m, a1, a2, 5, n_dir=2)
    start = _perturbed_start(kind, g, eps=0.1)
    g_gn, _, _ = wirtinger.gauss_newton(prob, start, tol=1e-14)
    g_lm, _, _ = wirtinger.levenberg_marquardt(prob, start, tol=1e-14)
    it = diagonal.iterate(kind, start, d, m, a1, a2, 5, tol=1e-14, max_iter=20000)
    for est in (g_gn, g_lm, it['g']):
        assert gauge.rel_error(kind, est, g) < 1e-8


def test_three_antenna_amplitude_closure():
    """N_ant = 3, noiseless: |g_1|^2 = a_12 conj(a_13) / conj(a_23) with a_pq = d_pq / m_pq."""
    d, m, a1, a2, g = _tiny('scalar', n_ant=3, n_samp=1)
    a = (d / m)[0]                       # baselines 12, 13, 23
    closure = a[0] * np.conj(a[1]) / np.conj(a[2])
    prob = wirtinger.Problem('scalar', d, m, a1, a2, 3)
    g_gn, _, _ = wirtinger.gauss_newton(prob, np.ones(3, complex), tol=1e-14)
    it = diagonal.iterate('scalar', np.ones(3, complex), d, m, a1, a2, 3, tol=1e-14, max_iter=5000)
    assert abs(closure.imag) < 1e-12 * abs(closure)
    for est in (g_gn, it['g'], g):
        np.testing.assert_allclose(abs(est[0]) ** 2, closure.real, rtol=1e-9)


def test_lm_chi2_non_increasing_and_limits():
    """App. C LM: accepted chi^2 never increases; lambda = 0 gives the GN step; lambda -> inf gives
    the steepest-descent direction scaled by D^-1 (eq. LM)."""
    d, m, a1, a2, g = _tiny('jones', n_ant=4, noise=0.2)
    prob = wirtinger.Problem('jones', d, m, a1, a2, 4)
    start = _perturbed_start('jones', g, eps=0.5)
    _, _, hist = wirtinger.levenberg_marquardt(prob, start, tol=1e-13)
    assert all(b <= a for a, b in zip(hist, hist[1:]))
    H, b = prob.normal_equations(start)
    np.testing.assert_allclose(wirtinger.lm_step(H, b, 0.0), wirtinger.min_norm_solve(H, b), atol=1e-12)
    big = wirtinger.lm_step(H, b, 1e12) * 1e12
    sd = b / np.real(np.diag(H))
    assert np.abs(np.vdot(big, sd)) / (np.linalg.norm(big) * np.linalg.norm(sd)) > 1 - 1e-6


@pytest.mark.parametrize("kind", ['scalar', 'dd', 'jones'])
def test_diagonal_fixed_point_is_gn_stationary_point(kind):
    """A fixed point of eq. stefcal (CohJones: the antenna-block step) has J^H r = 0 (eq. JHR:DI1),
    i.e. it is the stationary point full GN reaches."""
    d, m, a1, a2, g = _tiny(kind, n_ant=6, n_samp=3, n_dir=2, noise=0.05)
    start = np.ones_like(g) if kind != 'jones' else np.tile(np.eye(2, dtype=complex), (6, 1, 1))
    it = diagonal.iterate(kind, start, d, m, a1, a2, 6, tol=1e-13, max_iter=50000)
    assert it['converged']
    prob = wirtinger.Problem(kind, d, m, a1, a2, 6, n_dir=2)
    _, b = prob.normal_equations(it['g'])
    _, b0 = prob.normal_equations(start)
    assert np.linalg.norm(b) < 1e-9 * np.linalg.norm(b0)
    g_gn, _, _ = wirtinger.gauss_newton(prob, it['g'], tol=1e-14)
    assert gauge.rel_error(kind, it['g'], g_gn) < 1e-9


def test_brute_force_global_minimum_tiny():
    """Multi-start LM over random starts: no start finds a lower chi^2 than the oracle's solution."""
    d, m, a1, a2, g = _tiny('scalar', n_ant=4, n_samp=2, noise=0.3)
    prob = wirtinger.Problem('scalar', d, m, a1, a2, 4)
    it = diagonal.iterate('scalar', np.ones(4, complex), d, m, a1, a2, 4, tol=1e-13, max_iter=20000)
    best = prob.chi2(it['g'])
    r = synth.rng_for(9, 9)
    for _ in range(25):
        s = synth.complex_noise(r, 4, 1.5)
        gl, _, _ = wirtinger.levenberg_marquardt(prob, s, tol=1e-12)
        assert prob.chi2(gl) >= best * (1 - 1e-9)


def test_cohjones_single_direction_is_stefcal():
    """With N_d = 1 the CohJones block step is the scalar StefCal step (Sect. 3.3 cost table remark)."""
    d, m, a1, a2, g = _tiny('scalar', n_ant=6, n_samp=3, noise=0.1)
    it_s = diagonal.iterate('scalar', np.ones(6, complex), d, m, a1, a2, 6, tol=0.0, max_iter=12, record=True)
    it_d = diagonal.iterate('dd', np.ones((6, 1), complex), d, m[None], a1, a2, 6, tol=0.0, max_iter=12, record=True)
    for a, b in zip(it_s['history'], it_d['history']):
        np.testing.assert_allclose(a, b[:, 0], rtol=1e-12)


def test_diagonal_jones_is_two_scalar_problems():
    """Diagonal model and diagonal start: the 2x2 step decouples into the xx and yy scalar steps."""
    d, m, a1, a2, g = _tiny('scalar', n_ant=5, n_samp=2, noise=0.1, seed=11)
    d2, m2, _, _, _ = _tiny('scalar', n_ant=5, n_samp=2, noise=0.1, seed=12)
    D = np.zeros(d.shape + (2, 2), complex); M = np.zeros_like(D)
    D[..., 0, 0] = d; D[..., 1, 1] = d2; M[..., 0, 0] = m; M[..., 1, 1] = m2
    G0 = np.tile(np.eye(2, dtype=complex), (5, 1, 1))
    J = diagonal.iterate('jones', G0, D, M, a1, a2, 5, tol=0.0, max_iter=8)
    x = diagonal.iterate('scalar', np.ones(5, complex), d, m, a1, a2, 5, tol=0.0, max_iter=8)
    y = diagonal.iterate('scalar', np.ones(5, complex), d2, m2, a1, a2, 5, tol=0.0, max_iter=8)
    np.testing.assert_allclose(J['g'][:, 0, 0], x['g'], rtol=1e-12)
    np.testing.assert_allclose(J['g'][:, 1, 1], y['g'], rtol=1e-12)
    assert np.all(J['g'][:, 0, 1] == 0) and np.all(J['g'][:, 1, 0] == 0)


def test_data_form_equals_residual_form():
    """eq. ghat:precise holds for the diagonal approximation: g + A^-1 J^H r = A^-1 J^H d (eq. stefcal)."""
    for kind in ('scalar', 'jones', 'dd'):
        d, m, a1, a2, g = _tiny(kind, n_ant=5, n_samp=2, n_dir=2, noise=0.1)
        g0 = _perturbed_start(kind, g)
        if kind == 'scalar':
            b = blocks.scalar_blocks(g0, d, m, a1, a2, 5)
            np.testing.assert_allclose(g0 + b['c'] / b['A'], b['cd'] / b['A'], rtol=1e-12)
        elif kind == 'jones':
            b = blocks.jones_blocks(g0, d, m, a1, a2, 5)
            Hi = np.linalg.inv(b['H'])
            np.testing.assert_allclose(g0 + b['C'] @ Hi, b['CD'] @ Hi, rtol=1e-11, atol=1e-12)
        else:
            b = blocks.dd_blocks(g0, d, m, a1, a2, 5)
            for p in range(5):
                np.testing.assert_allclose(g0[p] + np.linalg.solve(b['A'][p], b['c'][p]),
                                           np.linalg.solve(b['A'][p], b['cd'][p]), rtol=1e-11)


def test_schedule_averages_on_even_steps():
    """eq. stefcal-lambda-average with lambda = 1 on even k: g_{k+1} = (g_k + g_GN)/2."""
    d, m, a1, a2, g = _tiny('scalar', n_ant=5, n_samp=2, noise=0.1)
    it = diagonal.iterate('scalar', np.ones(5, complex), d, m, a1, a2, 5, tol=0.0, max_iter=4, record=True)
    h = it['history']
    for k in range(1, 5):
        gn, _ = diagonal.stefcal_scalar_step(h[k - 1], d, m, a1, a2, 5)
        expect = gn if k % 2 == 1 else 0.5 * (h[k - 1] + gn)
        np.testing.assert_allclose(h[k], expect, rtol=1e-13)


# ------------------------------------------------------------------------------------ generator / gauge

def test_gauge_alignment_removes_only_the_phase():
    r = synth.rng_for(4, 4)
    g = synth.jones_gains(r, 7)
    assert gauge.rel_error('jones', g * np.exp(0.7j), g) < 1e-14
    g2 = g.copy(); g2[3, 0, 1] += 1e-3
    assert gauge.rel_error('jones', g2 * np.exp(-1.1j), g) > 1e-4


def test_generator_is_seeded_and_noise_has_stated_sigma():
    b1 = synth.make_config(2, small=True)
    b2 = synth.make_config(2, small=True)
    assert np.array_equal(b1.vis, b2.vis) and np.array_equal(b1.g_true, b2.g_true)
    iv = b1.interval(0)
    v = synth.simulate_jones(iv['g_true'], iv['model'].astype(np.complex128), iv['ant1'], iv['ant2'])
    res = iv['vis'] - v
    s = np.std(np.concatenate([res.real.ravel(), res.imag.ravel()]))
    assert abs(s - 0.01) < 0.001


# ------------------------------------------------------------------------------------ whole J^H J (exact LM)

def test_full_jones_jhj_equals_explicit_product():
    """eq. JHJ:pol in operator form (App. B 4x4 matrices), off-diagonal antenna blocks included,
    equals J^H J and J^H R of the explicit Jacobian after reordering [z; conj z] -> eq. GGvec."""
    d, m, a1, a2, g = _tiny('jones', n_ant=4, n_samp=2, noise=0.1)
    g0 = _perturbed_start('jones', g)
    prob = wirtinger.Problem('jones', d, m, a1, a2, 4)
    H, b = prob.normal_equations(g0)
    Hc, bc = blocks.jones_jhj_full(g0, d, m, a1, a2, 4)
    T = wirtinger.paper_to_wirtinger_order(4)
    np.testing.assert_allclose(Hc, T @ H @ T.T, atol=1e-11)
    np.testing.assert_allclose(bc, T @ b, atol=1e-11)
    # structure of eq. JHJ:pol: top-left block-diagonal, top-right zero on the antenna diagonal
    for p in range(4):
        for q in range(4):
            tl = Hc[4 * p:4 * p + 4, 4 * q:4 * q + 4]
            tr = Hc[4 * p:4 * p + 4, 16 + 4 * q:16 + 4 * q + 4]
            if p != q:
                assert np.all(tl == 0)
            else:
                assert np.all(tr == 0)
    # the top-left diagonal block is the polarized StefCal block R_H, H = sum Y Y^H
    cf = blocks.jones_blocks(g0, d, m, a1, a2, 4)
    for p in range(4):
        np.testing.assert_allclose(Hc[4 * p:4 * p + 4, 4 * p:4 * p + 4], blocks.op_R4(cf['H'][p]), atol=1e-12)


def test_full_scalar_jhj_equals_explicit_product():
    """eq. JHJ:DI (A, B, conj B, A) over the interval's samples equals the explicit J^H J."""
    d, m, a1, a2, g = _tiny('scalar', n_ant=5, n_samp=3, noise=0.1)
    g0 = _perturbed_start('scalar', g)
    H, b = wirtinger.Problem('scalar', d, m, a1, a2, 5).normal_equations(g0)
    Hc, bc = blocks.scalar_jhj_full(g0, d, m, a1, a2, 5)
    np.testing.assert_allclose(Hc, H, atol=1e-11)
    np.testing.assert_allclose(bc, b, atol=1e-11)


def test_gauge_step_is_minimum_norm_gn_at_zero_damping():
    """lm_step with the gauge direction and lambda = 0 is the minimum-norm GN step (eq. GN): the
    added mu u u^H only acts on the null direction of J^H J, which J^H r does not reach."""
    d, m, a1, a2, g = _tiny('jones', n_ant=4, n_samp=3, noise=0.05)
    g0 = _perturbed_start('jones', g, eps=0.05)
    prob = wirtinger.Problem('jones', d, m, a1, a2, 4)
    H, b = prob.normal_equations(g0)
    z = prob.to_z(g0)
    u = wirtinger.gauge_direction(z)
    assert np.linalg.norm(H @ u) < 1e-10 * np.linalg.norm(H)
    np.testing.assert_allclose(wirtinger.lm_step(H, b, 0.0, u), wirtinger.min_norm_solve(H, b), atol=1e-9)
    # with damping the step still lowers chi^2 from a perturbed start
    dz = wirtinger.lm_step(H, b, 1e-2, u)[: z.shape[0]]
    assert prob.chi2(prob.from_z(z + dz)) < prob.chi2(g0)


@pytest.mark.parametrize("kind", ['scalar', 'jones'])
def test_closed_form_lm_recovers_noiseless_gains(kind):
    """App. C LM on the closed-form normal equations, from a perturbed start, recovers the true
    gains up to the phase gauge on noiseless data (zero residual is the global minimum)."""
    from oracle import gauge as gauge_mod
    d, m, a1, a2, g = _tiny(kind, n_ant=5, n_samp=3)
    prob = wirtinger.ClosedFormProblem(kind, d, m, a1, a2, 5)
    for gauge in (False, True):
        gs, it, hist = wirtinger.levenberg_marquardt(prob, _perturbed_start(kind, g, eps=0.2), tol=1e-13,
                                                     lam0=1e-2, K=10.0, gauge=gauge)
        assert gauge_mod.rel_error(kind, gs, g) < 1e-10
        assert all(h1 < h0 for h0, h1 in zip(hist, hist[1:]))


def test_closed_form_lm_stationary_point_and_explicit_agreement():
    """On noisy 2x2 data the closed-form LM stops where the chi^2 gradient vanishes (finite
    differences, Sect. 1: d chi^2 / d conj z = -J^H r) and where the explicit-J LM stops."""
    from oracle import gauge as gauge_mod
    d, m, a1, a2, g = _tiny('jones', n_ant=5, n_samp=2, noise=0.05)
    start = _perturbed_start('jones', g, eps=0.05)
    pc = wirtinger.ClosedFormProblem('jones', d, m, a1, a2, 5)
    pe = wirtinger.Problem('jones', d, m, a1, a2, 5)
    gc_, _, _ = wirtinger.levenberg_marquardt(pc, start, tol=1e-13, lam0=1e-2, gauge=True)
    ge_, _, _ = wirtinger.levenberg_marquardt(pe, start, tol=1e-13, lam0=1e-2)
    assert gauge_mod.rel_error('jones', gc_, ge_) < 1e-9
    h = 1e-6
    c0 = pc.chi2(gc_)
    for p in range(5):
        for (u, v) in ((0, 0), (0, 1), (1, 0), (1, 1)):
            e = np.zeros_like(gc_); e[p, u, v] = h
            dx = (pc.chi2(gc_ + e) - pc.chi2(gc_ - e)) / (2 * h)
            dy = (pc.chi2(gc_ + 1j * e) - pc.chi2(gc_ - 1j * e)) / (2 * h)
            assert abs(dx) + abs(dy) < 1e-6 * c0 + 1e-7


def test_cpu_openmp_lm_matches_oracle_least_squares():
    """The FP64 C++/OpenMP implementation of the same method (the benchmark's all-core CPU comparator)
    converges to the NumPy oracle's least-squares gains on a small 2x2 workload, every interval."""
    from oracle import cpu
    from paper_1502_06974_gb300 import synth as sy
    b = sy.make_config(2, small=True)
    g, iters, status, used = cpu.calibrate_jones_lm(b, tol=1e-10, max_iter=500, K=2.0, threads=2)
    assert used >= 1 and (status == 0).all(), status
    for i in range(b.n_int):
        iv = b.interval(i)
        prob = wirtinger.ClosedFormProblem('jones', iv['vis'], iv['model'], iv['ant1'], iv['ant2'], iv['n_ant'])
        r = diagonal.iterate('jones', b.g0()[iv['gain_slice']], iv['vis'], iv['model'], iv['ant1'], iv['ant2'],
                             iv['n_ant'], tol=0.0, max_iter=20)
        ls, _, _ = wirtinger.levenberg_marquardt(prob, r['g'], tol=1e-12, lam0=1e-2, gauge=True)
        # complex64 storage of the result limits the agreement to FP32 rounding
        assert gauge.rel_error('jones', g[iv['gain_slice']], ls) < 1e-6, i
