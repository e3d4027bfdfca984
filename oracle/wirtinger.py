"""Explicit complex (Wirtinger) Jacobians and the full GN / LM solvers, FP64.

Test infrastructure only (see the package header).

Conventions (Sect. 1): the model v(z, conj z) has m complex entries; the partial Jacobians are
J_k = dv/dz and J_k* = dv/d(conj z) (eq. Jkrk) and the full complex Jacobian is

    J = [[J_k, J_k*], [conj(J_k*), conj(J_k)]]        (eq. JJ, 2m x 2n)

acting on the augmented vector z_aug = [z; conj z].  The GN step is
delta z_aug = (J^H J)^-1 J^H r_aug (eq. GN) and the LM step adds lambda * diag(J^H J)
(eq. LM).  Rows here are the stored baselines (either orientation) times samples; the bottom
half of J holds the conjugate baselines, which is the row reordering Sect. 2.1 allows.

Parameter orderings:
  scalar DI      z = [g_1 .. g_n]
  scalar DD      z = [g_1^(1) .. g_1^(Nd), g_2^(1) ..]   (CAD ordering, Sect. 3.2)
  2x2 DI         z = [vec G_1, vec G_2, ..]  with vec stacking columns (App. B)
  2x2 DD         z = [vec G_1^(1) .. vec G_1^(Nd), vec G_2^(1) ..]  (CAD ordering, Sect. 4.4)
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------- models v(z)

def model_scalar(g, m, a1, a2):
    """v_[pqs] = g_p m_pqs conj(g_q) (eq. cal:DI:tf); m, result [N_s, N_bl]."""
    return g[a1][None, :] * m * np.conj(g[a2])[None, :]


def model_dd(g, m, a1, a2):
    """v = sum_d g_p^(d) m^(d) conj(g_q^(d)) (eq. cal:dd:unpol); g [n_ant, Nd], m [Nd, N_s, N_bl]."""
    return np.einsum('bd,dsb,bd->sb', g[a1], m, np.conj(g[a2]))


def model_jones(G, M, a1, a2):
    """V = G_p M G_q^H (eq. RIME:pol); M [N_s, N_bl, 2, 2]."""
    return G[a1][None] @ M @ np.conj(np.swapaxes(G[a2], -1, -2))[None]


def model_dd_jones(G, M, a1, a2):
    """V = sum_d G_p^(d) M^(d) G_q^(d)H (Sect. 4.4); G [n_ant, Nd, 2, 2], M [Nd, N_s, N_bl, 2, 2]."""
    V = 0
    for d in range(M.shape[0]):
        V = V + G[a1, d][None] @ M[d] @ np.conj(np.swapaxes(G[a2, d], -1, -2))[None]
    return V


def vec2(X):
    """Column-stacking vec of 2x2 matrices (App. B): [x11, x21, x12, x22]."""
    return np.stack([X[..., 0, 0], X[..., 1, 0], X[..., 0, 1], X[..., 1, 1]], axis=-1)


def unvec2(x):
    X = np.empty(x.shape[:-1] + (2, 2), dtype=np.result_type(x, np.complex128))
    X[..., 0, 0] = x[..., 0]
    X[..., 1, 0] = x[..., 1]
    X[..., 0, 1] = x[..., 2]
    X[..., 1, 1] = x[..., 3]
    return X


COMMUTATION_2x2 = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
"""K with vec(X^T) = K vec(X) for 2x2 X."""


# ----------------------------------------------------------------------------- partial Jacobians

def partials_scalar(g, m, a1, a2):
    """J_k, J_k* for scalar DI (eqs. Jk, Jbark with the sample index of Sect. 2.3).

    Row order: sample-major, baseline-minor (as in the data); column j = antenna j.
    dv_pqs/dg_j = m_pqs conj(g_q) delta_jp ; dv_pqs/dconj(g_j) = g_p m_pqs delta_jq.
    """
    ns, nb = m.shape
    n = g.shape[0]
    Jk = np.zeros((ns * nb, n), np.complex128)
    Jc = np.zeros((ns * nb, n), np.complex128)
    for s in range(ns):
        for b in range(nb):
            p, q = int(a1[b]), int(a2[b])
            r = s * nb + b
            Jk[r, p] += m[s, b] * np.conj(g[q])
            Jc[r, q] += g[p] * m[s, b]
    return Jk, Jc


def partials_dd(g, m, a1, a2):
    """J_k, J_k* for scalar DD (Sect. 2.5), columns in CAD order j * Nd + d."""
    nd, ns, nb = m.shape
    n = g.shape[0]
    Jk = np.zeros((ns * nb, n * nd), np.complex128)
    Jc = np.zeros((ns * nb, n * nd), np.complex128)
    for s in range(ns):
        for b in range(nb):
            p, q = int(a1[b]), int(a2[b])
            r = s * nb + b
            for d in range(nd):
                Jk[r, p * nd + d] += m[d, s, b] * np.conj(g[q, d])
                Jc[r, q * nd + d] += g[p, d] * m[d, s, b]
    return Jk, Jc


def partials_jones(G, M, a1, a2):
    """J_k, J_k* for 2x2 DI via vec (App. B): 4 rows per visibility, 4 columns per antenna.

    vec(G_p M G_q^H) = ((M G_q^H)^T kron I) vec(G_p)        -> block at antenna p of J_k
                     = (I kron (G_p M)) K vec(conj G_q)      -> block at antenna q of J_k*
    using vec(ABC) = (C^T kron A) vec(B) and G_q^H = (conj G_q)^T.
    """
    ns, nb = M.shape[:2]
    n = G.shape[0]
    I2 = np.eye(2, dtype=np.complex128)
    Jk = np.zeros((ns * nb * 4, n * 4), np.complex128)
    Jc = np.zeros((ns * nb * 4, n * 4), np.complex128)
    for s in range(ns):
        for b in range(nb):
            p, q = int(a1[b]), int(a2[b])
            r = (s * nb + b) * 4
            Y = M[s, b] @ np.conj(G[q]).T
            Jk[r:r + 4, 4 * p:4 * p + 4] += np.kron(Y.T, I2)
            Jc[r:r + 4, 4 * q:4 * q + 4] += np.kron(I2, G[p] @ M[s, b]) @ COMMUTATION_2x2
    return Jk, Jc


def partials_dd_jones(G, M, a1, a2):
    """J_k, J_k* for 2x2 DD: each direction contributes the 2x2 DI blocks of ``partials_jones``
    with its own model and gains; columns in CAD order ((j * Nd + d) * 4 + vec index)."""
    nd, ns, nb = M.shape[:3]
    n = G.shape[0]
    I2 = np.eye(2, dtype=np.complex128)
    Jk = np.zeros((ns * nb * 4, n * nd * 4), np.complex128)
    Jc = np.zeros((ns * nb * 4, n * nd * 4), np.complex128)
    for s in range(ns):
        for b in range(nb):
            p, q = int(a1[b]), int(a2[b])
            r = (s * nb + b) * 4
            for d in range(nd):
                Y = M[d, s, b] @ np.conj(G[q, d]).T
                cp, cq = 4 * (p * nd + d), 4 * (q * nd + d)
                Jk[r:r + 4, cp:cp + 4] += np.kron(Y.T, I2)
                Jc[r:r + 4, cq:cq + 4] += np.kron(I2, G[p, d] @ M[d, s, b]) @ COMMUTATION_2x2
    return Jk, Jc


def full_jacobian(Jk, Jc):
    """eq. JJ."""
    return np.block([[Jk, Jc], [np.conj(Jc), np.conj(Jk)]])


# ----------------------------------------------------------------------------- problem wrapper

class Problem:
    """One solution interval in a uniform interface for the explicit-Jacobian solvers."""

    def __init__(self, kind, vis, model, a1, a2, n_ant, n_dir=1, weights=None):
        self.kind = kind
        # per-row weights w_pqs [N_s, N_bl] (Sect. 2.4: a diagonal W in eq. LSmin:w); None: unit
        self.weights = None if weights is None else np.asarray(weights, np.float64)
        self.a1 = np.asarray(a1, np.int64)
        self.a2 = np.asarray(a2, np.int64)
        self.n_ant = int(n_ant)
        self.n_dir = int(n_dir)
        self.vis = np.asarray(vis, np.complex128)
        self.model = np.asarray(model, np.complex128)

    # z <-> gains
    def to_z(self, g):
        g = np.asarray(g, np.complex128)
        if self.kind in ('jones', 'dd_jones'):
            return vec2(g).reshape(-1)
        return g.reshape(-1)

    def from_z(self, z):
        if self.kind == 'jones':
            return unvec2(z.reshape(self.n_ant, 4))
        if self.kind == 'dd_jones':
            return unvec2(z.reshape(self.n_ant, self.n_dir, 4))
        if self.kind == 'dd':
            return z.reshape(self.n_ant, self.n_dir)
        return z.copy()

    def model_vis(self, g):
        if self.kind == 'scalar':
            return model_scalar(g, self.model, self.a1, self.a2)
        if self.kind == 'dd':
            return model_dd(g, self.model, self.a1, self.a2)
        if self.kind == 'dd_jones':
            return model_dd_jones(g, self.model, self.a1, self.a2)
        return model_jones(g, self.model, self.a1, self.a2)

    def residual_vec(self, g):
        r = self.vis - self.model_vis(g)
        return vec2(r).reshape(-1) if self.kind in ('jones', 'dd_jones') else r.reshape(-1)

    def partials(self, g):
        if self.kind == 'scalar':
            return partials_scalar(g, self.model, self.a1, self.a2)
        if self.kind == 'dd':
            return partials_dd(g, self.model, self.a1, self.a2)
        if self.kind == 'dd_jones':
            return partials_dd_jones(g, self.model, self.a1, self.a2)
        return partials_jones(g, self.model, self.a1, self.a2)

    def jacobian(self, g):
        return full_jacobian(*self.partials(g))

    def row_weights(self):
        """The diagonal of W over the entries of residual_vec (4 per row for the 2x2 kinds)."""
        if self.weights is None:
            return None
        w = self.weights.reshape(-1)
        return np.repeat(w, 4) if self.kind in ('jones', 'dd_jones') else w

    def chi2(self, g):
        r = self.residual_vec(g)
        w = self.row_weights()
        return float(np.real(np.vdot(r, r if w is None else w * r)))

    def normal_equations(self, g):
        """(J^H W J, J^H W r_aug) at g, eq. GN / eq. LM (eq. LM:W with weights) ingredients."""
        J = self.jacobian(g)
        r = self.residual_vec(g)
        raug = np.concatenate([r, np.conj(r)])
        w = self.row_weights()
        if w is None:
            return J.conj().T @ J, J.conj().T @ raug
        w2 = np.concatenate([w, w])
        return J.conj().T @ (w2[:, None] * J), J.conj().T @ (w2 * raug)


# ----------------------------------------------------------------------------- solvers (App. C)

def min_norm_solve(H, b, rcond=1e-12):
    """Minimum-norm solution of the Hermitian system H x = b (eigendecomposition with cutoff).

    J^H J is singular along the gauge directions (e.g. a global phase, Sect. 2.1), so the GN
    step is taken as the minimum-norm least-squares solution rather than a plain inverse.
    """
    w, V = np.linalg.eigh(H)
    cut = rcond * max(float(np.max(np.abs(w))), 1e-300)
    winv = np.where(w > cut, 1.0 / np.where(w > cut, w, 1.0), 0.0)
    return V @ (winv * (V.conj().T @ b))


def gauss_newton(prob: Problem, g0, tol=1e-12, max_iter=100):
    """Algorithm GN (App. C) with the step of eq. GN; stops when ||dz|| <= tol ||z||.

    Returns (g, iterations, chi2 history).
    """
    z = prob.to_z(g0).copy()
    n = z.shape[0]
    hist = [prob.chi2(prob.from_z(z))]
    for k in range(1, max_iter + 1):
        H, b = prob.normal_equations(prob.from_z(z))
        dz_aug = min_norm_solve(H, b)
        dz = dz_aug[:n]
        z = z + dz
        hist.append(prob.chi2(prob.from_z(z)))
        if np.linalg.norm(dz) <= tol * np.linalg.norm(z):
            return prob.from_z(z), k, hist
    return prob.from_z(z), max_iter, hist


def gauge_direction(z):
    """Unit augmented vector of the phase gauge, u = [i z; -i conj z] / ||.||: the change of
    [z; conj z] under z -> z e^{i phi} (chi^2 does not depend on phi, Sect. 2.1)."""
    u = np.concatenate([1j * z, -1j * np.conj(z)])
    return u / np.linalg.norm(u)


def lm_step(H, b, lam, gauge=None):
    """eq. LM: (J^H J + lambda D)^-1 J^H r_aug with D = diag(J^H J).

    With ``gauge`` (a unit vector u spanning the phase-gauge null direction of J^H J), the step
    is taken in the complement of u: J^H r_aug is projected off u and mu u u^H, mu the mean of
    diag(J^H J), is added to the matrix.  For lambda = 0 this is the minimum-norm GN step; for
    lambda > 0 it keeps the damped matrix well conditioned along u however small lambda gets.
    """
    D = np.diag(np.real(np.diag(H)))
    A = H + lam * D
    if gauge is not None:
        b = b - gauge * np.vdot(gauge, b)
        A = A + np.mean(np.real(np.diag(H))) * np.outer(gauge, np.conj(gauge))
    return min_norm_solve(A, b)


def levenberg_marquardt(prob: Problem, g0, tol=1e-12, max_iter=200, lam0=1.0, K=10.0, gauge=False):
    """Algorithm LM (App. C): accept a step only if chi^2 decreases; lambda /= K on success,
    lambda *= K and retry from the previous point on failure.  chi^2 = ||r||^2.
    ``gauge``: take each step in the complement of the phase-gauge direction (see lm_step).

    Returns (g, accepted-iterations, chi2 history of accepted points).
    """
    z = prob.to_z(g0).copy()
    n = z.shape[0]
    lam = lam0
    chi = prob.chi2(prob.from_z(z))
    hist = [chi]
    it = 0
    for _ in range(max_iter):
        H, b = prob.normal_equations(prob.from_z(z))
        dz = lm_step(H, b, lam, gauge_direction(z) if gauge else None)[:n]
        z_new = z + dz
        chi_new = prob.chi2(prob.from_z(z_new))
        if chi_new < chi:
            z, chi = z_new, chi_new
            lam /= K
            hist.append(chi)
            it += 1
            if np.linalg.norm(dz) <= tol * np.linalg.norm(z):
                break
        else:
            lam *= K
            if lam > 1e16:
                break
    return prob.from_z(z), it, hist


def steepest_descent_direction(prob: Problem, g):
    """Algorithm SD direction (App. C): J^H r_aug (top half)."""
    _, b = prob.normal_equations(g)
    return b[: b.shape[0] // 2]


# ----------------------------------------------------------------------------- closed-form normal equations

class ClosedFormProblem(Problem):
    """A scalar or 2x2 DI interval whose normal equations come from the closed forms of the whole
    J^H J (eq. JHJ:DI for scalar, eq. JHJ:pol for 2x2, blocks.scalar_jhj_full /
    blocks.jones_jhj_full) instead of the explicit J, so that intervals of 64 antennas stay cheap.
    Same interface and ordering ([z; conj z]) as Problem."""

    def __init__(self, kind, vis, model, a1, a2, n_ant, weights=None):
        assert kind in ('scalar', 'jones')
        super().__init__(kind, vis, model, a1, a2, n_ant, weights=weights)

    def normal_equations(self, g):
        from . import blocks
        if self.kind == 'scalar':
            return blocks.scalar_jhj_full(g, self.vis, self.model, self.a1, self.a2, self.n_ant, self.weights)
        H, b = blocks.jones_jhj_full(g, self.vis, self.model, self.a1, self.a2, self.n_ant, self.weights)
        T = paper_to_wirtinger_order(self.n_ant)
        return T.T @ H @ T, T.T @ b


def paper_to_wirtinger_order(n_ant):
    """Permutation T with [vec G; vec G^H] (eq. GGvec) = T [vec G; vec conj G]: vec(G^H) = K vec(conj G)."""
    n4 = 4 * int(n_ant)
    T = np.zeros((2 * n4, 2 * n4))
    T[:n4, :n4] = np.eye(n4)
    T[n4:, n4:] = np.kron(np.eye(int(n_ant)), np.real(COMMUTATION_2x2))
    return T
