"""The paper's approximate-inverse iterations, step by step, FP64.

Test infrastructure only (see the package header).

Methods: StefCal (scalar and 2x2 DI), CohJones (scalar and 2x2 DD: exact inverse of each
antenna's direction block, data form), AllJones (scalar and 2x2 DD: diagonal J^H J, residual form).

Schedule (Sect. 3.1): iterations are numbered k = 1, 2, ...; odd k take the GN step with the
(block-)diagonal J^H J (eq. stefcal-matrix), even k take the LM step with lambda = 1, which for
a (block-)diagonal approximation is the average of the current gains and the GN gains
(eq. stefcal-lambda-average; for CohJones the same average, which Sect. 3.2.2 calls
approximate).  ``schedule='gn'`` takes the GN step every time.

Convergence (App. C, first criterion, made relative): stop after iteration k when
||g_{k+1} - g_k||_F <= tol * ||g_{k+1}||_F over the interval's parameters.
"""
from __future__ import annotations

import numpy as np

from .blocks import dd_blocks, dd_jones_blocks, jones_blocks, scalar_blocks


def _schedule_mix(k, g_old, g_gn, schedule):
    if schedule == 'gn' or (k % 2 == 1):
        return g_gn
    return 0.5 * (g_old + g_gn)


def stefcal_scalar_step(g, vis, model, a1, a2, n_ant, weights=None):
    """One GN step of eq. stefcal: g_p = (sum conj(y) y)^-1 sum conj(y) d.

    Antennas with no data (A_p = 0) keep their gain; returns (g_gn, singular mask).
    """
    b = scalar_blocks(g, vis, model, a1, a2, n_ant, weights)
    sing = ~(b['A'] > 0)
    g_gn = np.where(sing, g, b['cd'] / np.where(sing, 1.0, b['A']))
    return g_gn, sing


def stefcal_jones_step(G, vis, model, a1, a2, n_ant, weights=None):
    """One GN step of the polarized update (eq. update:DI:diag:pol, order [sum D Y^H][sum Y Y^H]^-1)."""
    b = jones_blocks(G, vis, model, a1, a2, n_ant, weights)
    H = b['H']
    det = np.real(H[:, 0, 0] * H[:, 1, 1] - H[:, 0, 1] * H[:, 1, 0])
    sing = ~(det > 0)
    Hs = np.where(sing[:, None, None], np.eye(2), H)
    G_gn = b['CD'] @ np.linalg.inv(Hs)
    G_gn = np.where(sing[:, None, None], G, G_gn)
    return G_gn, sing


def cohjones_step(g, vis, model, a1, a2, n_ant):
    """One GN step of CohJones (Sect. 3.2.2): g_p = A_p^-1 J^H d restricted to antenna p."""
    b = dd_blocks(g, vis, model, a1, a2, n_ant)
    out = g.copy()
    sing = np.zeros(n_ant, bool)
    for p in range(n_ant):
        try:
            np.linalg.cholesky(b['A'][p])
            out[p] = np.linalg.solve(b['A'][p], b['cd'][p])
        except np.linalg.LinAlgError:
            sing[p] = True
    return out, sing


def alljones_step(g, vis, model, a1, a2, n_ant):
    """One GN step of AllJones (Sect. 3.2.3, eq. stefcal:dd:unpol): the whole J^H J taken as its
    diagonal, so the step goes through the residuals, g_p^(d) += c_p^(d) / A_p[d, d] with
    c = sum conj(y^(d)) r.  A direction with no signal at an antenna (A_p[d, d] = 0) keeps its gain."""
    b = dd_blocks(g, vis, model, a1, a2, n_ant)
    a = np.real(np.diagonal(b['A'], axis1=1, axis2=2))           # [n, Nd]
    sing = ~(a > 0)
    out = np.where(sing, g, g + b['c'] / np.where(sing, 1.0, a))
    return out, sing.any(axis=1)


def cohjones_jones_step(G, vis, model, a1, a2, n_ant):
    """One GN step of polarized CohJones (Sect. 4.4): per antenna [G^(1) .. G^(Nd)] = CD H^-1 with
    the 2Nd x 2Nd H of blocks.dd_jones_blocks (the 4Nd x 4Nd operator block is R_H, whose inverse
    is R_{H^-1}, App. B eq. RAB:LAB).  An antenna whose H is not positive definite keeps its gains."""
    b = dd_jones_blocks(G, vis, model, a1, a2, n_ant)
    nd = G.shape[1]
    out = G.copy()
    sing = np.zeros(n_ant, bool)
    for p in range(n_ant):
        try:
            np.linalg.cholesky(b['H'][p])
        except np.linalg.LinAlgError:
            sing[p] = True
            continue
        X = np.linalg.solve(b['H'][p].T, b['CD'][p].T).T              # X H = CD
        out[p] = np.stack([X[:, 2 * d:2 * d + 2] for d in range(nd)])
    return out, sing


def alljones_jones_step(G, vis, model, a1, a2, n_ant):
    """One GN step of polarized AllJones (Sect. 4.4, eq. update:DD:diag:pol, product order as
    [sum R Y^(d)H][sum Y^(d) Y^(d)H]^-1): dG_p^(d) = C^(d) H_p[d, d]^-1, per antenna and direction.
    A (p, d) whose 2x2 block is singular keeps its gain."""
    b = dd_jones_blocks(G, vis, model, a1, a2, n_ant)
    nd = G.shape[1]
    out = G.copy()
    sing = np.zeros(n_ant, bool)
    for p in range(n_ant):
        for d in range(nd):
            Hd = b['H'][p, 2 * d:2 * d + 2, 2 * d:2 * d + 2]
            det = np.real(Hd[0, 0] * Hd[1, 1] - Hd[0, 1] * Hd[1, 0])
            if not (det > 0 and np.real(Hd[0, 0]) > 0):
                sing[p] = True
                continue
            out[p, d] = G[p, d] + b['C'][p][:, 2 * d:2 * d + 2] @ np.linalg.inv(Hd)
    return out, sing


_STEPS = {'scalar': stefcal_scalar_step, 'jones': stefcal_jones_step, 'dd': cohjones_step,
          'dd_jones': cohjones_jones_step}
_ALLJONES = {'dd': alljones_step, 'dd_jones': alljones_jones_step}


def iterate(kind, g0, vis, model, a1, a2, n_ant, tol=1e-12, max_iter=1000, schedule='stefcal',
            record=False, method='cohjones', weights=None):
    """Run the diagonal iteration of ``kind`` on one interval (for the DD kinds, ``method``
    'cohjones' or 'alljones'; per-row ``weights`` [N_s, N_bl] for the DI kinds, Sect. 2.4).

    Returns dict(g, iters, converged, singular, history(optional list of iterates)).
    """
    step = _ALLJONES[kind] if method == 'alljones' else _STEPS[kind]
    g = np.asarray(g0, np.complex128).copy()
    hist = [g.copy()] if record else None
    sing = None
    for k in range(1, max_iter + 1):
        g_gn, sing = (step(g, vis, model, a1, a2, n_ant) if weights is None
                      else step(g, vis, model, a1, a2, n_ant, weights))
        g_new = _schedule_mix(k, g, g_gn, schedule)
        dn = np.linalg.norm((g_new - g).ravel())
        nn = np.linalg.norm(g_new.ravel())
        g = g_new
        if record:
            hist.append(g.copy())
        if dn <= tol * nn:
            return dict(g=g, iters=k, converged=True, singular=sing, history=hist)
    return dict(g=g, iters=max_iter, converged=False, singular=sing, history=hist)


def solve_batch(batch, tol=1e-12, max_iter=1000, schedule='stefcal', intervals=None, g0=None, method='cohjones'):
    """Diagonal iteration on every (or the listed) interval of a synth.Batch.

    Returns (gains like batch.g_true for the listed intervals, iters [k], converged [k]).
    """
    idx = range(batch.n_int) if intervals is None else intervals
    gs, its, conv = [], [], []
    start = batch.g0() if g0 is None else g0
    for i in idx:
        iv = batch.interval(int(i))
        r = iterate(batch.kind, start[iv['gain_slice']], iv['vis'], iv['model'], iv['ant1'], iv['ant2'],
                    iv['n_ant'], tol=tol, max_iter=max_iter, schedule=schedule, method=method,
                    weights=iv.get('weights'))
        gs.append(r['g']); its.append(r['iters']); conv.append(r['converged'])
    return np.concatenate(gs), np.asarray(its), np.asarray(conv)


def chi2_interval(kind, g, vis, model, a1, a2, weights=None):
    """chi^2 = sum |r|^2 over the interval (eq. cal:DI:tf / cal:dd:unpol / cal:DI:pol, squared norm);
    with per-row weights sum w |r|^2 (eq. LSmin:w with a diagonal W)."""
    g = np.asarray(g, np.complex128)
    vis = np.asarray(vis, np.complex128); model = np.asarray(model, np.complex128)
    a1 = np.asarray(a1, np.int64); a2 = np.asarray(a2, np.int64)
    if kind == 'scalar':
        v = g[a1][None] * model * np.conj(g[a2])[None]
    elif kind == 'dd':
        v = np.einsum('bd,dsb,bd->sb', g[a1], model, np.conj(g[a2]))
    elif kind == 'dd_jones':
        v = sum(g[a1, d][None] @ model[d] @ np.conj(np.swapaxes(g[a2, d], -1, -2))[None]
                for d in range(model.shape[0]))
    else:
        v = g[a1][None] @ model @ np.conj(np.swapaxes(g[a2], -1, -2))[None]
    r = np.abs(vis - v) ** 2
    if weights is not None:
        r = r * np.asarray(weights, np.float64).reshape(r.shape[:2] + (1,) * (r.ndim - 2))
    return float(np.sum(r))
