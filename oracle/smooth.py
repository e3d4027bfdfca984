"""Smoothing in time and frequency (Sect. 3.4), FP64: StefCal with the sums convolved by a kernel.

Test infrastructure only (see the package header).

Every time/frequency sample (t0, nu0) has its own gains, solving the weighted problem of
eq. cal:DI:smooth with weights w(t - t0, nu - nu0).  Under the diagonal approximation each update
is eq. stefcal:w, the ratio of two convolutions (eq. JHJ:diag:smooth):
    scalar: g_p(t, nu) = (w o alpha_p)(t, nu) / (w o beta_p)(t, nu),
            alpha_p = sum_q conj(y_pq) d_pq,  beta_p = sum_q |y_pq|^2  (per sample, y = m conj(g_q)),
    2x2:    G_p = (w o C_p) (w o H_p)^-1,  C_p = sum_q D_pq Y_pq^H,  H_p = sum_q Y_pq Y_pq^H
            (the polarized update of eq. update:DI:diag:pol with the same kernel-weighted sums).
The kernel is a separable Gaussian (the paper's example), w = wt(t - t0) wf(nu - nu0) with
wt(x) = exp(-x^2 / 2 sigma_t^2) on the sample grid, cut at |x| <= ceil(3 sigma) (sigma = 0: a
single tap, no smoothing).  The convolutions are the direct sums over the kernel's support,
clipped at the grid edges (the ratio does not depend on the kernel's normalisation).

Schedule as for StefCal (odd iterations the GN gains, even ones their average with the current
gains), with two phase conventions per sample.  Each sample's problem is unchanged by a common
phase of its gains (Sect. 2.1), but the kernel couples neighbouring samples through their phases:
  * the GN gains are first rotated by the common phase that best aligns them with the sample's
    current gains (psi = arg sum_p conj(g_p) gn_p; 2x2: arg sum_p tr(G_p^H Gn_p)): they come back
    rotated by a small per-sample phase even at the solution, and unaligned the iterates drift along
    those phase modes at a constant step (the average of two vectors a phase apart also shrinks
    them), never meeting the stopping rule;
  * every new iterate is put in the canonical gauge (sum_p g_p, 2x2: sum_p tr G_p, real and
    non-negative), so that neighbouring samples share one phase reference: with per-sample phase
    offsets (from the start, say) the convolution averages unaligned gains and biases the solution.
Without smoothing neither changes the solution: at a fixed point sum_p A_p conj(g_p) gn_p is real
(the sum over both orientations of every baseline of conj(v) d), so the alignment is 0 (or pi), and
the canonical rotation only picks the gauge.  One convergence test over the whole grid:
||g_{k+1} - g_k|| <= tol ||g_{k+1}|| summed over every sample and antenna (the samples are coupled).
"""
from __future__ import annotations

import math

import numpy as np

from .blocks import jones_blocks, scalar_blocks


def gaussian_taps(sigma):
    """Taps of the Gaussian kernel at integer offsets -R..R, R = ceil(3 sigma)."""
    if sigma <= 0:
        return np.ones(1)
    R = int(math.ceil(3.0 * sigma))
    x = np.arange(-R, R + 1, dtype=np.float64)
    return np.exp(-0.5 * (x / sigma) ** 2)


def per_sample_sums(kind, g, vis, model, a1, a2, n_ant):
    """alpha, beta (scalar) or C, H (2x2) of every sample: arrays [n_t, n_f, n_ant(, 2, 2)]."""
    nt, nf = vis.shape[:2]
    if kind == 'scalar':
        al = np.zeros((nt, nf, n_ant), np.complex128)
        be = np.zeros((nt, nf, n_ant))
    else:
        al = np.zeros((nt, nf, n_ant, 2, 2), np.complex128)
        be = np.zeros((nt, nf, n_ant, 2, 2), np.complex128)
    for t in range(nt):
        for f in range(nf):
            if kind == 'scalar':
                b = scalar_blocks(g[t, f], vis[t, f][None], model[t, f][None], a1, a2, n_ant)
                al[t, f], be[t, f] = b['cd'], b['A']
            else:
                b = jones_blocks(g[t, f], vis[t, f][None], model[t, f][None], a1, a2, n_ant)
                al[t, f], be[t, f] = b['CD'], b['H']
    return al, be


def convolve(x, wt, wf):
    """(w o x)(t0, f0) = sum_{t, f} wt(t - t0) wf(f - f0) x(t, f) over the grid (axes 0 and 1)."""
    nt, nf = x.shape[:2]
    Rt, Rf = (len(wt) - 1) // 2, (len(wf) - 1) // 2
    out = np.zeros_like(x)
    for t0 in range(nt):
        for f0 in range(nf):
            acc = np.zeros_like(x[0, 0])
            for t in range(max(0, t0 - Rt), min(nt, t0 + Rt + 1)):
                for f in range(max(0, f0 - Rf), min(nf, f0 + Rf + 1)):
                    acc = acc + wt[t - t0 + Rt] * wf[f - f0 + Rf] * x[t, f]
            out[t0, f0] = acc
    return out


def smooth_step(kind, g, vis, model, a1, a2, n_ant, wt, wf):
    """One GN step of eq. JHJ:diag:smooth; antennas whose smoothed sum is singular keep their gains."""
    al, be = per_sample_sums(kind, g, vis, model, a1, a2, n_ant)
    sa, sb = convolve(al, wt, wf), convolve(be, wt, wf)
    if kind == 'scalar':
        sing = ~(sb > 0)
        return np.where(sing, g, sa / np.where(sing, 1.0, sb))
    det = np.real(sb[..., 0, 0] * sb[..., 1, 1] - sb[..., 0, 1] * sb[..., 1, 0])
    sing = ~(det > 0)
    inv = np.linalg.inv(np.where(sing[..., None, None], np.eye(2), sb))
    return np.where(sing[..., None, None], g, sa @ inv)


def canonical_phase(kind, g):
    """Rotate each sample's gains (axes 0, 1 of g) so that sum_p g_p (2x2: sum_p tr G_p) is real, >= 0."""
    S = np.sum(g, axis=2) if kind == 'scalar' else np.sum(np.trace(g, axis1=-2, axis2=-1), axis=2)
    ph = np.where(np.abs(S) > 0, np.exp(-1j * np.angle(S)), 1.0)
    return g * (ph[:, :, None] if kind == 'scalar' else ph[:, :, None, None, None])


def align_phase(kind, gn, g):
    """gn rotated, per sample (axes 0, 1), by the common phase that best aligns it with g."""
    if kind == 'scalar':
        S = np.sum(np.conj(g) * gn, axis=2)
        return gn * np.exp(-1j * np.angle(S))[:, :, None]
    S = np.sum(np.conj(g) * gn, axis=(2, 3, 4))
    return gn * np.exp(-1j * np.angle(S))[:, :, None, None, None]


def iterate_smooth(kind, g0, vis, model, a1, a2, n_ant, sigma_t, sigma_f, tol=1e-10, max_iter=500,
                   schedule='stefcal', taps=None):
    """Returns dict(g [n_t, n_f, n_ant(, 2, 2)], iters, converged).  taps = (wt, wf) replaces the
    Gaussian taps of sigma_t, sigma_f (odd lengths, centred)."""
    wt, wf = (gaussian_taps(sigma_t), gaussian_taps(sigma_f)) if taps is None else taps
    g = np.asarray(g0, np.complex128).copy()
    vis = np.asarray(vis, np.complex128); model = np.asarray(model, np.complex128)
    for k in range(1, max_iter + 1):
        gn = smooth_step(kind, g, vis, model, a1, a2, n_ant, wt, wf)
        gn = align_phase(kind, gn, g)
        new = canonical_phase(kind, gn if (schedule == 'gn' or k % 2 == 1) else 0.5 * (g + gn))
        dn = np.linalg.norm((new - g).ravel())
        nn = np.linalg.norm(new.ravel())
        g = new
        if dn <= tol * nn:
            return dict(g=g, iters=k, converged=True)
    return dict(g=g, iters=max_iter, converged=False)
