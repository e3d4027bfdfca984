"""Learned warm start for the 2x2 solver: features, proposal, start selection, gauge, FP64.

Test infrastructure only (see the package header).  The warm start is an addition to the paper's
method (motivated by Sect. 3.4: gains vary smoothly in time and frequency); it only
chooses where the paper's iteration starts, and the iteration then runs to the same tolerance.

Per (interval, antenna) row, with g1..g4 the antenna's four previous 2x2 solutions (newest first)
and C = sum D Y^H, H = sum Y Y^H the blocks of the polarized update (eq. update:DI:diag:pol) on
the target interval at gains g1, the network input is, in the frame rotated by e^{-i phi} with
phi = arg(g1[0,0]):

  x = [g1 | g1 - g2 | g2 - g3 | g3 - g4 | C H^-1 - g1 | lead | 0 ... 0]   (48 entries)

each 2x2 complex matrix flattened row-major as (re, im) pairs, lead the scaled lead time.  The
network predicts delta (8 reals, the same flattening) and the proposal is g1 + e^{i phi} delta.
The start is the proposal when chi^2 there is below chi^2 at g1, else g1.

Gauge: chi^2 is unchanged by G_p -> G_p e^{i theta} for all p (Sect. 2.1).  Solutions are put in
a canonical gauge, sum_p tr(G_p) real and non-negative, so consecutive solutions of a smooth
process are themselves smooth and can be differenced.
"""
from __future__ import annotations

import numpy as np

from .blocks import jones_blocks
from .diagonal import chi2_interval

IN_WIDTH = 48


def _flat(G):
    """[n, 2, 2] complex -> [n, 8] reals (re, im) row-major."""
    G = np.asarray(G, np.complex128)
    out = np.empty(G.shape[:-2] + (8,), np.float64)
    f = G.reshape(G.shape[:-2] + (4,))
    out[..., 0::2] = f.real
    out[..., 1::2] = f.imag
    return out


def _unflat(v):
    v = np.asarray(v, np.float64)
    return (v[..., 0::2] + 1j * v[..., 1::2]).reshape(v.shape[:-1] + (2, 2))


def gn_gains(G, vis, model, a1, a2, n_ant):
    """C H^-1 per antenna (the GN step of the polarized update at G); zero where H is singular."""
    b = jones_blocks(G, vis, model, a1, a2, n_ant)
    H = b['H']
    det = np.real(H[:, 0, 0] * H[:, 1, 1] - H[:, 0, 1] * H[:, 1, 0])
    ok = (det > 0) & (np.real(H[:, 0, 0]) > 0)
    Hs = np.where(ok[:, None, None], H, np.eye(2))
    return np.where(ok[:, None, None], b['CD'] @ np.linalg.inv(Hs), 0.0), ok


def features(hist, gn, ok, lead):
    """Network inputs and rotations for rows of one or more intervals.

    hist [n, 4, 2, 2] previous solutions newest first; gn [n, 2, 2] = C H^-1 at hist[:, 0]
    (ok [n] False where H was singular: the step entries are then 0); lead [n].
    Returns x [n, 48] and rot [n] = e^{i phi}.
    """
    hist = np.asarray(hist, np.complex128)
    n = hist.shape[0]
    g1 = hist[:, 0]
    a = g1[:, 0, 0]
    rot = np.where(np.abs(a) > 0, a / np.where(np.abs(a) > 0, np.abs(a), 1.0), 1.0)
    r = np.conj(rot)[:, None, None]
    step = np.where(np.asarray(ok)[:, None, None], np.asarray(gn, np.complex128) - g1, 0.0)
    parts = [g1, hist[:, 0] - hist[:, 1], hist[:, 1] - hist[:, 2], hist[:, 2] - hist[:, 3], step]
    x = np.zeros((n, IN_WIDTH), np.float64)
    for j, P in enumerate(parts):
        x[:, 8 * j:8 * j + 8] = _flat(r * P)
    x[:, 40] = np.asarray(lead, np.float64)
    return x, rot


def propose(g1, delta, rot):
    """g1 + e^{i phi} delta."""
    return np.asarray(g1, np.complex128) + np.asarray(rot)[:, None, None] * _unflat(delta)


def target(g1, g_next, rot):
    """The training target: e^{-i phi} (g_next - g1), flattened."""
    return _flat(np.conj(np.asarray(rot))[:, None, None] * (np.asarray(g_next, np.complex128) -
                                                              np.asarray(g1, np.complex128)))


def canonical_gauge(G):
    """Rotate one interval's gains so that sum_p tr(G_p) is real and non-negative."""
    G = np.asarray(G, np.complex128)
    s = np.sum(G[:, 0, 0] + G[:, 1, 1])
    if abs(s) == 0:
        return G.copy()
    return G * (np.conj(s) / abs(s))


def select(iv, g1, prop):
    """(start, used, chi2(prop) - chi2(g1)) for one interval (dict from Batch.interval)."""
    c1 = chi2_interval('jones', g1, iv['vis'], iv['model'], iv['ant1'], iv['ant2'])
    c2 = chi2_interval('jones', prop, iv['vis'], iv['model'], iv['ant1'], iv['ant2'])
    used = c2 < c1
    return (prop if used else np.asarray(g1, np.complex128)), bool(used), float(c2 - c1)
