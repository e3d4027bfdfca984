"""Seeded synthetic inputs for gain calibration (interferometer, sky, gains, noise).

This module only *simulates observations*: it places antennas, draws a sky of
point sources, evaluates their visibilities, draws true gains and corrupts the
model with them plus Gaussian noise (the measurement equation, Sect. 2.1
eq. RIME:unpol, Sect. 4 eq. RIME:pol, Sect. 2.5 eq. cal:dd:unpol).  It holds no
calibration arithmetic: no Jacobians, no J^H J or J^H r sums, no gain updates.
Both the CUDA path and the CPU oracle are fed from here.

Point-source visibilities follow Sect. 2.5 (the S * k factorisation), with
k = exp(-2 pi i (u l + v m) nu / c) for an array with w = 0 (antennas on the
ground plane, uvw fixed in time).

Data layout produced for every problem (a "batch" of solution intervals):
  rows of interval i are ``row_off[i] .. row_off[i] + n_samp[i] * n_bl[i]``,
  sample-major and baseline-minor; baseline b of interval i is
  ``(ant1[bl_off[i] + b], ant2[bl_off[i] + b])`` with antenna numbers local to
  the interval; its gains start at ``gain_off[i]`` (one slot per antenna, times
  n_dir directions for the direction-dependent case).
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SEED = 150206974
C_LIGHT = 299792458.0
DEG = np.pi / 180.0


def rng_for(seed: int, *keys: int) -> np.random.Generator:
    """PCG64 stream for (seed, keys...): one independent stream per purpose."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed)] + [int(k) for k in keys])))


@dataclass
class Batch:
    """A set of independent solution intervals sharing one data layout."""
    kind: str                      # 'scalar' | 'jones' | 'dd' | 'dd_jones'
    vis: np.ndarray                # scalar/dd: [rows]; jones/dd_jones: [rows, 2, 2]
    model: np.ndarray              # scalar: [rows]; jones: [rows, 2, 2]; dd: [n_dir, rows];
                                   # dd_jones: [n_dir, rows, 2, 2]
    ant1: np.ndarray               # int32 [n_bl_total]
    ant2: np.ndarray               # int32 [n_bl_total]
    row_off: np.ndarray            # int64 [n_int]
    n_samp: np.ndarray             # int32 [n_int]
    n_bl: np.ndarray               # int32 [n_int]
    bl_off: np.ndarray             # int32 [n_int]
    n_ant: np.ndarray              # int32 [n_int]
    gain_off: np.ndarray           # int32 [n_int]
    g_true: np.ndarray             # scalar: [n_gain]; jones: [n_gain,2,2]; dd: [n_gain, n_dir];
                                   # dd_jones: [n_gain, n_dir, 2, 2]
    n_dir: int = 1
    meta: dict = field(default_factory=dict)
    weights: Optional[np.ndarray] = None   # per-row non-negative weights [rows] (None: unit)

    @property
    def n_int(self) -> int:
        return int(self.row_off.shape[0])

    @property
    def n_rows(self) -> int:
        return int(np.sum(self.n_samp.astype(np.int64) * self.n_bl.astype(np.int64)))

    @property
    def n_gain(self) -> int:
        return int(np.sum(self.n_ant))

    def g0(self) -> np.ndarray:
        """Default start: unit gains (identity Jones)."""
        if self.kind == 'jones':
            g = np.zeros((self.n_gain, 2, 2), dtype=self.vis.dtype)
            g[:, 0, 0] = 1.0
            g[:, 1, 1] = 1.0
            return g
        if self.kind == 'dd':
            return np.ones((self.n_gain, self.n_dir), dtype=self.vis.dtype)
        if self.kind == 'dd_jones':
            g = np.zeros((self.n_gain, self.n_dir, 2, 2), dtype=self.vis.dtype)
            g[..., 0, 0] = 1.0
            g[..., 1, 1] = 1.0
            return g
        return np.ones(self.n_gain, dtype=self.vis.dtype)

    def interval(self, i: int) -> dict:
        """Views of interval i (rows reshaped [n_samp, n_bl, ...])."""
        r0 = int(self.row_off[i]); ns = int(self.n_samp[i]); nb = int(self.n_bl[i])
        b0 = int(self.bl_off[i]); na = int(self.n_ant[i]); g0 = int(self.gain_off[i])
        sl = slice(r0, r0 + ns * nb)
        if self.kind == 'dd':
            model = self.model[:, sl].reshape(self.n_dir, ns, nb)
        elif self.kind == 'dd_jones':
            model = self.model[:, sl].reshape(self.n_dir, ns, nb, 2, 2)
        else:
            model = self.model[sl].reshape((ns, nb) + self.model.shape[1:])
        return dict(vis=self.vis[sl].reshape((ns, nb) + self.vis.shape[1:]), model=model,
                    ant1=self.ant1[b0:b0 + nb], ant2=self.ant2[b0:b0 + nb], n_ant=na,
                    g_true=self.g_true[g0:g0 + na], gain_slice=slice(g0, g0 + na),
                    weights=None if self.weights is None else self.weights[sl].reshape(ns, nb))

    def subset(self, idx) -> 'Batch':
        """A new batch holding only intervals ``idx`` (data copied, compacted)."""
        idx = np.asarray(idx, dtype=np.int64)
        rows, grows, bls = [], [], []
        row_off, gain_off, bl_off = [], [], []
        r = g = 0
        bl_map = {}
        nb_tot = 0
        for i in idx:
            iv = int(i)
            r0 = int(self.row_off[iv]); nr = int(self.n_samp[iv]) * int(self.n_bl[iv])
            rows.append(np.arange(r0, r0 + nr)); row_off.append(r); r += nr
            g0 = int(self.gain_off[iv]); na = int(self.n_ant[iv])
            grows.append(np.arange(g0, g0 + na)); gain_off.append(g); g += na
            key = (int(self.bl_off[iv]), int(self.n_bl[iv]))
            if key not in bl_map:
                bl_map[key] = nb_tot
                bls.append(np.arange(key[0], key[0] + key[1])); nb_tot += key[1]
            bl_off.append(bl_map[key])
        rows = np.concatenate(rows); grows = np.concatenate(grows); bls = np.concatenate(bls)
        model = self.model[:, rows] if self.kind in ('dd', 'dd_jones') else self.model[rows]
        return Batch(self.kind, np.ascontiguousarray(self.vis[rows]), np.ascontiguousarray(model),
                     np.ascontiguousarray(self.ant1[bls]), np.ascontiguousarray(self.ant2[bls]),
                     np.asarray(row_off, np.int64), self.n_samp[idx].copy(), self.n_bl[idx].copy(),
                     np.asarray(bl_off, np.int32), self.n_ant[idx].copy(), np.asarray(gain_off, np.int32),
                     np.ascontiguousarray(self.g_true[grows]), self.n_dir, dict(self.meta),
                     None if self.weights is None else np.ascontiguousarray(self.weights[rows]))


# ----------------------------------------------------------------------------- array and sky

def antenna_positions(rng: np.random.Generator, n_ant: int, diameter_m: float = 2000.0) -> np.ndarray:
    """East/north positions uniform in a disk of the given diameter (up = 0)."""
    r = 0.5 * diameter_m * np.sqrt(rng.uniform(0.0, 1.0, n_ant))
    th = rng.uniform(0.0, 2.0 * np.pi, n_ant)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def baseline_table(n_ant: int):
    """All pairs p < q in the order 01, 02, ..., 0(n-1), 12, ... (Sect. 2.1)."""
    p, q = np.triu_indices(n_ant, k=1)
    return p.astype(np.int32), q.astype(np.int32)


def fringe(xy: np.ndarray, ant1: np.ndarray, ant2: np.ndarray, l: np.ndarray, m: np.ndarray,
           freqs: np.ndarray) -> np.ndarray:
    """k[f, b, src] = exp(-2 pi i (u l + v m) nu / c), u = x_q - x_p (Sect. 2.5)."""
    uv = xy[ant2] - xy[ant1]                                          # [b, 2]
    path = uv[:, 0:1] * l[None, :] + uv[:, 1:2] * m[None, :]          # [b, src], metres
    return np.exp(-2j * np.pi * path[None, :, :] * (freqs[:, None, None] / C_LIGHT))


def scalar_sky(rng, n_src, lm_max_deg=2.0):
    flux = 10.0 ** rng.uniform(-1.0, 1.0, n_src)
    l = rng.uniform(-lm_max_deg, lm_max_deg, n_src) * DEG
    m = rng.uniform(-lm_max_deg, lm_max_deg, n_src) * DEG
    return flux, l, m


def polarized_sky(rng, n_src, frac_sigma=0.05, lm_max_deg=2.0):
    I = 10.0 ** rng.uniform(-1.0, 1.0, n_src)
    Q, U, V = (I * rng.normal(0.0, frac_sigma, n_src) for _ in range(3))
    l = rng.uniform(-lm_max_deg, lm_max_deg, n_src) * DEG
    m = rng.uniform(-lm_max_deg, lm_max_deg, n_src) * DEG
    B = np.empty((n_src, 2, 2), dtype=np.complex128)                  # linear-feed coherency
    B[:, 0, 0] = I + Q
    B[:, 0, 1] = U + 1j * V
    B[:, 1, 0] = U - 1j * V
    B[:, 1, 1] = I - Q
    return B, l, m


def polarized_sky_strong(rng, n_src, p_lo=0.3, p_hi=0.7, lm_max_deg=2.0):
    """Strongly polarized point sources: fractional polarization p ~ U(p_lo, p_hi) along a direction
    uniform on the Poincare sphere, (Q, U, V) = I p n; linear-feed coherencies as polarized_sky."""
    I = 10.0 ** rng.uniform(-1.0, 1.0, n_src)
    n = rng.normal(0.0, 1.0, (n_src, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    frac = rng.uniform(p_lo, p_hi, n_src)
    Q, U, V = (I * frac * n[:, k] for k in range(3))
    l = rng.uniform(-lm_max_deg, lm_max_deg, n_src) * DEG
    m = rng.uniform(-lm_max_deg, lm_max_deg, n_src) * DEG
    B = np.empty((n_src, 2, 2), dtype=np.complex128)
    B[:, 0, 0] = I + Q
    B[:, 0, 1] = U + 1j * V
    B[:, 1, 0] = U - 1j * V
    B[:, 1, 1] = I - Q
    return B, l, m


# ----------------------------------------------------------------------------- gains and noise

def scalar_gains(rng, shape, amp_sigma):
    amp = 1.0 + rng.normal(0.0, amp_sigma, shape)
    ph = rng.uniform(-np.pi, np.pi, shape)
    return amp * np.exp(1j * ph)


def jones_gains(rng, n, amp_sigma=0.1, leak_sigma=0.02):
    G = np.zeros((n, 2, 2), dtype=np.complex128)
    G[:, 0, 0] = scalar_gains(rng, n, amp_sigma)
    G[:, 1, 1] = scalar_gains(rng, n, amp_sigma)
    G[:, 0, 1] = rng.normal(0.0, leak_sigma, n) + 1j * rng.normal(0.0, leak_sigma, n)
    G[:, 1, 0] = rng.normal(0.0, leak_sigma, n) + 1j * rng.normal(0.0, leak_sigma, n)
    return G


def complex_noise(rng, shape, sigma):
    """Gaussian with standard deviation sigma in the real and in the imaginary part."""
    return rng.normal(0.0, sigma, shape) + 1j * rng.normal(0.0, sigma, shape)


# ----------------------------------------------------------------------------- forward simulation

def simulate_scalar(g, model, a1, a2):
    return g[a1] * model * np.conj(g[a2])


def simulate_jones(G, model, a1, a2):
    return G[a1] @ model @ np.conj(np.swapaxes(G[a2], -1, -2))


def simulate_dd(g, model, a1, a2):
    # g [n_ant, n_dir]; model [n_dir, ..., n_bl]
    shape = (g.shape[1],) + (1,) * (model.ndim - 2) + (len(a1),)
    gp = np.moveaxis(g[a1], -1, 0).reshape(shape)
    gq = np.moveaxis(g[a2], -1, 0).reshape(shape)
    return np.sum(gp * model * np.conj(gq), axis=0)


def _finish(kind, vis_list, model_list, a1, a2, n_samp, n_bl, bl_off, n_ant, g_list, dtype, n_dir=1, meta=None):
    n_int = len(vis_list)
    sizes = np.array([v.shape[0] * v.shape[1] for v in vis_list], np.int64)
    row_off = np.zeros(n_int, np.int64)
    row_off[1:] = np.cumsum(sizes)[:-1]
    gain_off = np.zeros(n_int, np.int32)
    gain_off[1:] = np.cumsum(np.asarray(n_ant, np.int64))[:-1]
    vis = np.concatenate([v.reshape((-1,) + v.shape[2:]) for v in vis_list]).astype(dtype)
    if kind == 'dd':
        model = np.concatenate([m.reshape(m.shape[0], -1) for m in model_list], axis=1).astype(dtype)
    elif kind == 'dd_jones':
        model = np.concatenate([m.reshape((m.shape[0], -1, 2, 2)) for m in model_list], axis=1).astype(dtype)
    else:
        model = np.concatenate([m.reshape((-1,) + m.shape[2:]) for m in model_list]).astype(dtype)
    g_true = np.concatenate(g_list).astype(np.complex128)
    return Batch(kind, np.ascontiguousarray(vis), np.ascontiguousarray(model), np.asarray(a1, np.int32),
                 np.asarray(a2, np.int32), row_off, np.asarray(n_samp, np.int32), np.asarray(n_bl, np.int32),
                 np.asarray(bl_off, np.int32), np.asarray(n_ant, np.int32), gain_off, g_true, n_dir,
                 meta or {})


# ----------------------------------------------------------------------------- workloads

def make_di_scalar(seed=SEED, n_ant=16, n_t=10, n_chan=4, t_per=None, f_per=None, n_src=5, amp_sigma=0.1,
                   sigma=0.01, dtype=np.complex128, fmin=1.0e9, fmax=1.4e9):
    """Direction-independent scalar gains; intervals of t_per times x f_per channels."""
    t_per = n_t if t_per is None else t_per
    f_per = n_chan if f_per is None else f_per
    rng_sky = rng_for(seed, 1, 0)
    xy = antenna_positions(rng_sky, n_ant)
    a1, a2 = baseline_table(n_ant)
    flux, l, m = scalar_sky(rng_sky, n_src)
    freqs = np.linspace(fmin, fmax, n_chan)
    model_f = np.einsum('fbs,s->fb', fringe(xy, a1, a2, l, m, freqs), flux)      # [f, b]; uvw fixed in time
    vis_l, mod_l, g_l = [], [], []
    n_tb, n_fb = n_t // t_per, n_chan // f_per
    for it in range(n_tb):
        for jf in range(n_fb):
            i = it * n_fb + jf
            r = rng_for(seed, 1, 1 + i)
            g = scalar_gains(r, n_ant, amp_sigma)
            mod = np.repeat(model_f[None, jf * f_per:(jf + 1) * f_per], t_per, axis=0).reshape(t_per * f_per, -1)
            vis = simulate_scalar(g, mod, a1, a2) + complex_noise(r, mod.shape, sigma)
            vis_l.append(vis); mod_l.append(mod); g_l.append(g)
    n = len(vis_l)
    return _finish('scalar', vis_l, mod_l, a1, a2, [t_per * f_per] * n, [len(a1)] * n, [0] * n, [n_ant] * n,
                   g_l, dtype, meta=dict(sigma=sigma, n_src=n_src))


def make_di_jones(seed=SEED, n_ant=64, n_t=60, n_chan=64, t_per=1, f_per=4, n_src=20, amp_sigma=0.1,
                  leak_sigma=0.02, frac_sigma=0.05, sigma=0.01, dtype=np.complex64, fmin=1.0e9, fmax=1.4e9):
    """Direction-independent full-Jones (2x2) gains with polarized point sources."""
    rng_sky = rng_for(seed, 2, 0)
    xy = antenna_positions(rng_sky, n_ant)
    a1, a2 = baseline_table(n_ant)
    B, l, m = polarized_sky(rng_sky, n_src, frac_sigma)
    freqs = np.linspace(fmin, fmax, n_chan)
    model_f = np.einsum('fbs,sij->fbij', fringe(xy, a1, a2, l, m, freqs), B)   # [f, b, 2, 2]
    vis_l, mod_l, g_l = [], [], []
    n_tb, n_fb = n_t // t_per, n_chan // f_per
    for it in range(n_tb):
        for jf in range(n_fb):
            i = it * n_fb + jf
            r = rng_for(seed, 2, 1 + i)
            G = jones_gains(r, n_ant, amp_sigma, leak_sigma)
            mod = np.repeat(model_f[None, jf * f_per:(jf + 1) * f_per], t_per, axis=0).reshape(t_per * f_per, -1, 2, 2)
            vis = simulate_jones(G, mod, a1, a2) + complex_noise(r, mod.shape, sigma)
            vis_l.append(vis); mod_l.append(mod); g_l.append(G)
    n = len(vis_l)
    return _finish('jones', vis_l, mod_l, a1, a2, [t_per * f_per] * n, [len(a1)] * n, [0] * n, [n_ant] * n,
                   g_l, dtype, meta=dict(sigma=sigma, n_src=n_src))


def make_dd(seed=SEED, n_ant=62, n_dir=9, n_t=120, n_chan=16, t_per=10, f_per=16, src_per_dir=3,
            amp_sigma=0.2, sigma=0.02, grid_deg=1.0, cluster_deg=0.1, dtype=np.complex64, fmin=1.0e9, fmax=1.4e9,
            log_flux=(-1.0, 1.0)):
    """Direction-dependent scalar gains: n_dir clusters of point sources on a square grid, source
    fluxes with log10 S uniform in ``log_flux``."""
    rng_sky = rng_for(seed, 3, 0)
    xy = antenna_positions(rng_sky, n_ant)
    a1, a2 = baseline_table(n_ant)
    side = int(np.ceil(np.sqrt(n_dir)))
    cx = (np.arange(n_dir) % side - (side - 1) / 2.0) * grid_deg * DEG
    cy = (np.arange(n_dir) // side - (side - 1) / 2.0) * grid_deg * DEG
    freqs = np.linspace(fmin, fmax, n_chan)
    model_dirs = []
    for d in range(n_dir):
        flux = 10.0 ** rng_sky.uniform(log_flux[0], log_flux[1], src_per_dir)
        l = cx[d] + rng_sky.uniform(-cluster_deg, cluster_deg, src_per_dir) * DEG
        m = cy[d] + rng_sky.uniform(-cluster_deg, cluster_deg, src_per_dir) * DEG
        model_dirs.append(np.einsum('fbs,s->fb', fringe(xy, a1, a2, l, m, freqs), flux))
    model_f = np.stack(model_dirs)                                                  # [d, f, b]
    vis_l, mod_l, g_l = [], [], []
    n_tb, n_fb = n_t // t_per, n_chan // f_per
    for it in range(n_tb):
        for jf in range(n_fb):
            i = it * n_fb + jf
            r = rng_for(seed, 3, 1 + i)
            g = scalar_gains(r, (n_ant, n_dir), amp_sigma)
            mod = np.repeat(model_f[:, None, jf * f_per:(jf + 1) * f_per], t_per, axis=1).reshape(n_dir, t_per * f_per, -1)
            vis = simulate_dd(g, mod, a1, a2) + complex_noise(r, mod.shape[1:], sigma)
            vis_l.append(vis); mod_l.append(mod); g_l.append(g)
    n = len(vis_l)
    return _finish('dd', vis_l, mod_l, a1, a2, [t_per * f_per] * n, [len(a1)] * n, [0] * n, [n_ant] * n,
                   g_l, dtype, n_dir=n_dir, meta=dict(sigma=sigma))


def simulate_dd_jones(G, model, a1, a2):
    """V = sum_d G_p^(d) M^(d) G_q^(d)H; G [n_ant, n_dir, 2, 2], model [n_dir, n_samp, n_bl, 2, 2]."""
    V = 0
    for d in range(model.shape[0]):
        V = V + G[a1, d] @ model[d] @ np.conj(np.swapaxes(G[a2, d], -1, -2))
    return V


def make_dd_jones(seed=SEED, n_ant=62, n_dir=9, n_t=120, n_chan=16, t_per=10, f_per=16, src_per_dir=3,
                  amp_sigma=0.2, leak_sigma=0.02, pol_frac=(0.3, 0.7), sigma=0.02, grid_deg=1.0, cluster_deg=0.1,
                  dtype=np.complex64, fmin=1.0e9, fmax=1.4e9, log_flux=(-0.5, 0.5)):
    """Direction-dependent 2x2 gains: the geometry of make_dd (n_dir clusters on a square grid) with
    strongly polarized sources (polarized_sky_strong, fractional polarization in pol_frac) and a
    2x2 gain per antenna and direction (diagonal 1 + N(0, amp_sigma) amplitudes with uniform
    phases, leakage CN(0, leak_sigma))."""
    rng_sky = rng_for(seed, 6, 0)
    xy = antenna_positions(rng_sky, n_ant)
    a1, a2 = baseline_table(n_ant)
    side = int(np.ceil(np.sqrt(n_dir)))
    cx = (np.arange(n_dir) % side - (side - 1) / 2.0) * grid_deg * DEG
    cy = (np.arange(n_dir) // side - (side - 1) / 2.0) * grid_deg * DEG
    freqs = np.linspace(fmin, fmax, n_chan)
    model_dirs = []
    for d in range(n_dir):
        B, _, _ = polarized_sky_strong(rng_sky, src_per_dir, pol_frac[0], pol_frac[1])
        B *= (10.0 ** rng_sky.uniform(log_flux[0], log_flux[1], src_per_dir))[:, None, None] / np.real(
            B[:, 0, 0] + B[:, 1, 1])[:, None, None] * 2.0
        l = cx[d] + rng_sky.uniform(-cluster_deg, cluster_deg, src_per_dir) * DEG
        m = cy[d] + rng_sky.uniform(-cluster_deg, cluster_deg, src_per_dir) * DEG
        model_dirs.append(np.einsum('fbs,sij->fbij', fringe(xy, a1, a2, l, m, freqs), B))
    model_f = np.stack(model_dirs)                                                  # [d, f, b, 2, 2]
    vis_l, mod_l, g_l = [], [], []
    n_tb, n_fb = n_t // t_per, n_chan // f_per
    for it in range(n_tb):
        for jf in range(n_fb):
            i = it * n_fb + jf
            r = rng_for(seed, 6, 1 + i)
            g = np.stack([jones_gains(r, n_ant, amp_sigma, leak_sigma) for _ in range(n_dir)], axis=1)
            mod = np.repeat(model_f[:, None, jf * f_per:(jf + 1) * f_per], t_per, axis=1).reshape(
                n_dir, t_per * f_per, -1, 2, 2)
            vis = simulate_dd_jones(g, mod, a1, a2) + complex_noise(r, mod.shape[1:], sigma)
            vis_l.append(vis); mod_l.append(mod); g_l.append(g)
    n = len(vis_l)
    return _finish('dd_jones', vis_l, mod_l, a1, a2, [t_per * f_per] * n, [len(a1)] * n, [0] * n, [n_ant] * n,
                   g_l, dtype, n_dir=n_dir, meta=dict(sigma=sigma))


def _uneven_interval(seed, i, kval, na, T, F, n_src, sigma, fmin, fmax):
    """Model, visibilities and true gains of interval i of the uneven workload (its own stream)."""
    r = rng_for(seed, 4, 1 + i)
    a1, a2 = baseline_table(na)
    xy = antenna_positions(r, na)
    freqs = np.linspace(fmin, fmax, F) if F > 1 else np.array([0.5 * (fmin + fmax)])
    if kval == 0:
        flux, l, m = scalar_sky(r, n_src)
        mf = np.einsum('fbs,s->fb', fringe(xy, a1, a2, l, m, freqs), flux)
        mod = np.repeat(mf[None], T, axis=0).reshape(T * F, -1)
        g = scalar_gains(r, na, 0.1)
        v = simulate_scalar(g, mod, a1, a2) + complex_noise(r, mod.shape, sigma)
    else:
        B, l, m = polarized_sky(r, n_src)
        mf = np.einsum('fbs,sij->fbij', fringe(xy, a1, a2, l, m, freqs), B)
        mod = np.repeat(mf[None], T, axis=0).reshape(T * F, -1, 2, 2)
        g = jones_gains(r, na, 0.1, 0.02)
        v = simulate_jones(g, mod, a1, a2) + complex_noise(r, mod.shape, sigma)
    return v, mod, g


def _uneven_worker(job):
    """Fill a share of the uneven workload's intervals into shared-memory arrays (process pool)."""
    from multiprocessing import shared_memory
    names, shapes, dtype, seed, jobs, n_src, sigma, fmin, fmax = job
    shm = [shared_memory.SharedMemory(name=n) for n in names]
    try:
        vis = np.ndarray(shapes[0], dtype=dtype, buffer=shm[0].buf)
        model = np.ndarray(shapes[0], dtype=dtype, buffer=shm[1].buf)
        g_true = np.ndarray(shapes[1], dtype=np.complex128, buffer=shm[2].buf)
        for (i, kval, na, T, F, r0, nr, g0) in jobs:
            v, mod, g = _uneven_interval(seed, i, kval, na, T, F, n_src, sigma, fmin, fmax)
            vis[r0:r0 + nr] = v.reshape((nr,) + tuple(shapes[0][1:]))
            model[r0:r0 + nr] = mod.reshape((nr,) + tuple(shapes[0][1:]))
            g_true[g0:g0 + na] = g
        del vis, model, g_true
    finally:
        for m in shm:
            m.close()
    return len(jobs)


def make_uneven(seed=SEED, n_intervals=4096, ant_choices=(16, 24, 32, 48, 64), t_max=32, f_max=16, n_src=5,
                sigma=0.01, dtype=np.complex64, only: Optional[str] = None, fmin=1.0e9, fmax=1.4e9, workers=1):
    """Independent intervals of uneven size; half scalar, half 2x2 (a Bernoulli draw per interval).

    Returns {'scalar': Batch, 'jones': Batch} (each kind compacted into its own batch) and the
    per-interval draw table under meta['draws'].  Every interval draws from its own stream; with
    workers > 1 they are simulated by a process pool (spawn) into shared memory, with the same result.
    """
    rd = rng_for(seed, 4, 0)
    n_ant = rd.choice(np.asarray(ant_choices), n_intervals)
    T = rd.integers(1, t_max + 1, n_intervals)
    F = rd.integers(1, f_max + 1, n_intervals)
    kind = rd.integers(0, 2, n_intervals)                 # 0 scalar, 1 jones
    tables = {int(n): baseline_table(int(n)) for n in ant_choices}
    out = {}
    for kname, kval in (('scalar', 0), ('jones', 1)):
        if only is not None and only != kname:
            continue
        idx = np.nonzero(kind == kval)[0]
        # shared baseline tables, one per antenna count
        a1_all, a2_all, off = [], [], {}
        o = 0
        for n in ant_choices:
            off[int(n)] = o
            a1_all.append(tables[int(n)][0]); a2_all.append(tables[int(n)][1]); o += len(tables[int(n)][0])
        na_l = n_ant[idx].astype(np.int32)
        nb_l = np.array([len(tables[int(n)][0]) for n in na_l], np.int32)
        ns_l = (T[idx] * F[idx]).astype(np.int32)
        bo_l = np.array([off[int(n)] for n in na_l], np.int32)
        sizes = ns_l.astype(np.int64) * nb_l
        row_off = np.zeros(len(idx), np.int64)
        row_off[1:] = np.cumsum(sizes)[:-1]
        gain_off = np.zeros(len(idx), np.int32)
        gain_off[1:] = np.cumsum(na_l.astype(np.int64))[:-1]
        shape = (int(sizes.sum()),) + (() if kval == 0 else (2, 2))
        gshape = (int(na_l.sum()),) + (() if kval == 0 else (2, 2))
        jobs = [(int(idx[j]), kval, int(na_l[j]), int(T[idx[j]]), int(F[idx[j]]), int(row_off[j]), int(sizes[j]),
                 int(gain_off[j])) for j in range(len(idx))]
        if workers <= 1:
            vis = np.empty(shape, dtype)
            model = np.empty(shape, dtype)
            g_true = np.empty(gshape, np.complex128)
            for (i, kv, na, tt, ff, r0, nr, g0) in jobs:
                v, mod, g = _uneven_interval(seed, i, kv, na, tt, ff, n_src, sigma, fmin, fmax)
                vis[r0:r0 + nr] = v.reshape((nr,) + shape[1:])
                model[r0:r0 + nr] = mod.reshape((nr,) + shape[1:])
                g_true[g0:g0 + na] = g
        else:
            import multiprocessing as mp
            from multiprocessing import shared_memory
            nbytes = [int(np.prod(shape)) * np.dtype(dtype).itemsize] * 2 + [int(np.prod(gshape)) * 16]
            shm = [shared_memory.SharedMemory(create=True, size=max(n, 1)) for n in nbytes]
            try:
                chunks = [jobs[w::workers] for w in range(workers)]
                args = [([m.name for m in shm], (shape, gshape), np.dtype(dtype).str, seed, c, n_src, sigma, fmin,
                         fmax) for c in chunks if c]
                with mp.get_context('spawn').Pool(len(args)) as pool:
                    pool.map(_uneven_worker, args)
                vis = np.ndarray(shape, dtype=dtype, buffer=shm[0].buf).copy()
                model = np.ndarray(shape, dtype=dtype, buffer=shm[1].buf).copy()
                g_true = np.ndarray(gshape, dtype=np.complex128, buffer=shm[2].buf).copy()
            finally:
                for m in shm:
                    m.close()
                    m.unlink()
        out[kname] = Batch(kname, vis, model, np.concatenate(a1_all).astype(np.int32),
                           np.concatenate(a2_all).astype(np.int32), row_off, ns_l, nb_l, bo_l, na_l, gain_off, g_true,
                           1, dict(sigma=sigma, interval_ids=idx))
    out['draws'] = dict(n_ant=n_ant, T=T, F=F, kind=kind)
    return out


def gp_sqrt(x: np.ndarray, length: float) -> np.ndarray:
    """A square root L (L L^T = K) of the squared-exponential covariance K_ij = exp(-(x_i-x_j)^2 / 2 l^2).

    Taken from the eigendecomposition with negative eigenvalues clipped (the kernel matrix of a
    densely sampled smooth process is numerically singular, so Cholesky is not used).
    """
    d = x[:, None] - x[None, :]
    K = np.exp(-0.5 * (d / length) ** 2)
    w, V = np.linalg.eigh(K)
    return V * np.sqrt(np.clip(w, 0.0, None))[None, :]


def make_warm(seed=SEED, n_ant=64, n_t=720, n_chan=64, f_per=8, dt_s=10.0, t_corr_s=1800.0, f_corr_hz=50e6,
              amp_sigma=0.1, phase_sigma=1.0, leak_sigma=0.02, n_src=20, frac_sigma=0.05, sigma=0.01,
              dtype=np.complex64, fmin=1.0e9, fmax=1.4e9, chunk=64):
    """Gains that evolve smoothly: a separable Gaussian process over time and frequency.

    Intervals are 1 time x f_per channels, ordered time-major (interval i = t * n_fb + fb).  The
    gain of an interval is the process at the interval's time and centre frequency, constant over
    the interval's samples.  Per antenna, independent processes (unit variance, squared-exponential
    kernels with the given correlation lengths) drive: the xx and yy amplitudes (1 + amp_sigma z),
    the xx and yy phases (phase_sigma z, radians) and the real and imaginary parts of the two
    leakage terms (leak_sigma z).  Sky, array and noise follow the full-Jones workload.
    """
    n_fb = n_chan // f_per
    rng_sky = rng_for(seed, 5, 0)
    xy = antenna_positions(rng_sky, n_ant)
    a1, a2 = baseline_table(n_ant)
    B, l, m = polarized_sky(rng_sky, n_src, frac_sigma)
    freqs = np.linspace(fmin, fmax, n_chan)
    model_f = np.einsum('fbs,sij->fbij', fringe(xy, a1, a2, l, m, freqs), B)      # [f, b, 2, 2]
    t_c = np.arange(n_t) * dt_s
    f_c = freqs.reshape(n_fb, f_per).mean(axis=1)
    Lt = gp_sqrt(t_c, t_corr_s)
    Lf = gp_sqrt(f_c, f_corr_hz)
    z = rng_for(seed, 5, 1).normal(0.0, 1.0, (8, n_ant, n_t, n_fb))
    z = np.einsum('tu,kauv,fv->katf', Lt, z, Lf)                                      # [8, a, t, fb]
    G = np.zeros((n_t, n_fb, n_ant, 2, 2), np.complex128)
    zt = np.transpose(z, (0, 2, 3, 1))                                                 # [8, t, fb, a]
    G[..., 0, 0] = (1.0 + amp_sigma * zt[0]) * np.exp(1j * phase_sigma * zt[2])
    G[..., 1, 1] = (1.0 + amp_sigma * zt[1]) * np.exp(1j * phase_sigma * zt[3])
    G[..., 0, 1] = leak_sigma * (zt[4] + 1j * zt[5])
    G[..., 1, 0] = leak_sigma * (zt[6] + 1j * zt[7])
    n_int = n_t * n_fb
    G = G.reshape(n_int, n_ant, 2, 2)
    nb = len(a1)
    ns = f_per
    rows = ns * nb
    vis = np.empty((n_int * rows, 2, 2), dtype)
    model = np.empty((n_int * rows, 2, 2), dtype)
    mod_blocks = model_f.reshape(n_fb, f_per * nb, 2, 2)

    def fill(c0):
        # chunks write disjoint rows and draw their noise per interval: the result does not depend
        # on the chunking or the thread count
        c1 = min(n_int, c0 + chunk)
        fb = np.arange(c0, c1) % n_fb
        mod = mod_blocks[fb].reshape(c1 - c0, ns, nb, 2, 2)
        Gp = G[c0:c1][:, a1][:, None]                                                   # [c, 1, b, 2, 2]
        Gq = np.conj(G[c0:c1][:, a2][:, None])
        # V = Gp M Gq^H written out entry by entry (elementwise products run in parallel threads,
        # stacked 2x2 matmuls do not)
        A = [[Gp[..., r, 0] * mod[..., 0, c] + Gp[..., r, 1] * mod[..., 1, c] for c in range(2)] for r in range(2)]
        v = np.empty(mod.shape, np.complex128)
        for r in range(2):
            for c in range(2):
                v[..., r, c] = A[r][0] * Gq[..., c, 0] + A[r][1] * Gq[..., c, 1]
        for j, i in enumerate(range(c0, c1)):
            v[j] += complex_noise(rng_for(seed, 5, 2 + i), (ns, nb, 2, 2), sigma)
        vis[c0 * rows:c1 * rows] = v.reshape(-1, 2, 2)
        model[c0 * rows:c1 * rows] = mod.reshape(-1, 2, 2)

    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(fill, range(0, n_int, chunk)))
    row_off = np.arange(n_int, dtype=np.int64) * rows
    return Batch('jones', vis, model, a1, a2, row_off, np.full(n_int, ns, np.int32), np.full(n_int, nb, np.int32),
                 np.zeros(n_int, np.int32), np.full(n_int, n_ant, np.int32),
                 (np.arange(n_int) * n_ant).astype(np.int32), G.reshape(n_int * n_ant, 2, 2), 1,
                 dict(sigma=sigma, n_t=n_t, n_fb=n_fb, n_src=n_src, dt_s=dt_s))


def make_smooth(kind='jones', seed=SEED, n_ant=64, n_t=240, n_chan=64, dt_s=10.0, t_corr_s=1800.0,
                f_corr_hz=50e6, amp_sigma=0.1, phase_sigma=1.0, n_src=20, sigma=0.2, dtype=np.complex64,
                fmin=1.0e9, df_hz=6.25e6):
    """Per-sample gains for smoothing (Sect. 3.4): every time x channel sample is one "interval" of
    one sample (interval i = t * n_chan + f), with gains drawn from the separable Gaussian process
    of make_warm at that sample.  2x2: make_warm with one channel per interval; scalar: the same
    process for one amplitude and one phase per antenna, an unpolarized sky.  Channels are df_hz
    apart from fmin (the 2x2 warm-start workload's spacing).  meta holds n_t, n_fb."""
    fmax = fmin + df_hz * (n_chan - 1)
    if kind == 'jones':
        return make_warm(seed, n_ant=n_ant, n_t=n_t, n_chan=n_chan, f_per=1, dt_s=dt_s, t_corr_s=t_corr_s,
                         f_corr_hz=f_corr_hz, amp_sigma=amp_sigma, phase_sigma=phase_sigma, n_src=n_src,
                         sigma=sigma, dtype=dtype, fmin=fmin, fmax=fmax)
    rng_sky = rng_for(seed, 7, 0)
    xy = antenna_positions(rng_sky, n_ant)
    a1, a2 = baseline_table(n_ant)
    flux, l, m = scalar_sky(rng_sky, n_src)
    freqs = fmin + df_hz * np.arange(n_chan)
    model_f = np.einsum('fbs,s->fb', fringe(xy, a1, a2, l, m, freqs), flux)           # [f, b]
    Lt = gp_sqrt(np.arange(n_t) * dt_s, t_corr_s)
    Lf = gp_sqrt(freqs, f_corr_hz)
    z = rng_for(seed, 7, 1).normal(0.0, 1.0, (2, n_ant, n_t, n_chan))
    z = np.einsum('tu,kauv,fv->ktfa', Lt, z, Lf)                                      # [2, t, f, a]
    g = (1.0 + amp_sigma * z[0]) * np.exp(1j * phase_sigma * z[1])                      # [t, f, a]
    vis = g[:, :, a1] * model_f[None] * np.conj(g[:, :, a2])
    vis = vis + complex_noise(rng_for(seed, 7, 2), vis.shape, sigma)
    n_int, nb = n_t * n_chan, len(a1)
    model = np.broadcast_to(model_f[None], (n_t, n_chan, nb))
    return Batch('scalar', np.ascontiguousarray(vis.reshape(-1).astype(dtype)),
                 np.ascontiguousarray(model.reshape(-1).astype(dtype)), a1, a2,
                 np.arange(n_int, dtype=np.int64) * nb, np.ones(n_int, np.int32), np.full(n_int, nb, np.int32),
                 np.zeros(n_int, np.int32), np.full(n_int, n_ant, np.int32),
                 (np.arange(n_int) * n_ant).astype(np.int32), g.reshape(-1), 1,
                 dict(sigma=sigma, n_t=n_t, n_fb=n_chan, dt_s=dt_s))


def make_config(k: int, seed: int = SEED, small: bool = False):
    """Synthetic stand-ins for the five workloads (small=True: a reduced copy for CPU tests)."""
    if k == 1:
        return make_di_scalar(seed, n_ant=16, n_t=10, n_chan=4, dtype=np.complex128)
    if k == 2:
        if small:
            return make_di_jones(seed, n_ant=16, n_t=2, n_chan=8, t_per=1, f_per=4)
        return make_di_jones(seed)
    if k == 3:
        if small:
            return make_dd(seed, n_ant=12, n_dir=4, n_t=4, n_chan=8, t_per=2, f_per=8)
        return make_dd(seed)
    if k == 4:
        if small:
            return make_uneven(seed, n_intervals=16, ant_choices=(4, 6, 8), t_max=4, f_max=4)
        return make_uneven(seed)
    if k == 5:
        if small:
            return make_warm(seed, n_ant=16, n_t=48, n_chan=16)
        return make_warm(seed)
    raise ValueError(f"unknown config {k}")
