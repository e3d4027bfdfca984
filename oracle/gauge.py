"""Gauge alignment and relative gain error, FP64.

Test infrastructure only (see the package header).

chi^2 is unchanged by g_p -> g_p e^{i phi} for all p at once (Sect. 2.1, eq. cal:DI: the phase
cancels in g_p m conj(g_q)); the DD problems (scalar and 2x2) have one such phase per direction and the 2x2 problem
G_p -> G_p e^{i phi}.  Two solutions are compared after rotating the estimate onto the
reference by the least-squares phase.
"""
from __future__ import annotations

import numpy as np


def align(kind, g_est, g_ref):
    """Rotate g_est by the global phase (per direction for 'dd') that best matches g_ref."""
    g_est = np.asarray(g_est, np.complex128); g_ref = np.asarray(g_ref, np.complex128)
    if kind == 'dd':
        ph = np.angle(np.sum(g_ref * np.conj(g_est), axis=0))       # [Nd]
        return g_est * np.exp(1j * ph)[None, :]
    if kind == 'dd_jones':
        ph = np.angle(np.sum(g_ref * np.conj(g_est), axis=(0, 2, 3)))   # [Nd]
        return g_est * np.exp(1j * ph)[None, :, None, None]
    ph = np.angle(np.sum(g_ref * np.conj(g_est)))
    return g_est * np.exp(1j * ph)


def rel_error(kind, g_est, g_ref, n_ant=None, gain_off=None):
    """max over antennas of ||g_est - g_ref|| / ||g_ref|| after alignment.

    If gain_off/n_ant are given the alignment is done per interval.
    """
    g_est = np.asarray(g_est, np.complex128); g_ref = np.asarray(g_ref, np.complex128)
    if gain_off is None:
        parts = [(0, g_ref.shape[0])]
    else:
        parts = [(int(o), int(o) + int(n)) for o, n in zip(gain_off, n_ant)]
    worst = 0.0
    for a, b in parts:
        ge = align(kind, g_est[a:b], g_ref[a:b])
        d = (ge - g_ref[a:b]).reshape(b - a, -1) if kind != 'dd' else (ge - g_ref[a:b])
        r = g_ref[a:b].reshape(b - a, -1) if kind != 'dd' else g_ref[a:b]
        if kind == 'dd':
            e = np.abs(d) / np.abs(r)
        elif kind == 'dd_jones':                 # per antenna and direction
            nd = g_ref.shape[1]
            e = (np.linalg.norm(d.reshape(b - a, nd, 4), axis=2)
                 / np.linalg.norm(r.reshape(b - a, nd, 4), axis=2))
        else:
            e = np.linalg.norm(d, axis=1) / np.linalg.norm(r, axis=1)
        worst = max(worst, float(np.max(e)))
    return worst
