"""Test helpers: move a synthetic batch to the device and run the oracle on its intervals."""
from __future__ import annotations

import numpy as np
import torch

from paper_1502_06974_gb300 import synth
from paper_1502_06974_gb300.api import Layout


def device_batch(b: synth.Batch, device='cuda'):
    vis = torch.from_numpy(np.ascontiguousarray(b.vis)).to(device)
    model = torch.from_numpy(np.ascontiguousarray(b.model)).to(device)
    g0 = torch.from_numpy(np.ascontiguousarray(b.g0())).to(device)
    return vis, model, g0, Layout.from_batch(b)


def relerr(a, b):
    a = np.asarray(a, np.complex128); b = np.asarray(b, np.complex128)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def per_slot_relerr(a, b, axis_elems=None):
    """max over slots of ||a_p - b_p|| / ||b_p||."""
    a = np.asarray(a, np.complex128).reshape(a.shape[0], -1)
    b = np.asarray(b, np.complex128).reshape(b.shape[0], -1)
    n = np.linalg.norm(b, axis=1)
    n = np.where(n > 0, n, 1.0)
    return float(np.max(np.linalg.norm(a - b, axis=1) / n))


def oracle_ls(kind, vis, model, a1, a2, n_ant, n_stefcal=20, tol=1e-12, K=10.0):
    """FP64 least-squares gains of one interval from the oracle's own unit start: StefCal for
    n_stefcal iterations, then App. C LM on the closed-form whole J^H J (test infrastructure)."""
    from oracle import diagonal, wirtinger
    g0 = (np.tile(np.eye(2, dtype=np.complex128), (n_ant, 1, 1)) if kind == 'jones'
          else np.ones(n_ant, np.complex128))
    r = diagonal.iterate(kind, g0, vis, model, a1, a2, n_ant, tol=0.0, max_iter=n_stefcal)
    prob = wirtinger.ClosedFormProblem(kind, vis, model, a1, a2, n_ant)
    g, _, _ = wirtinger.levenberg_marquardt(prob, r['g'], tol=tol, max_iter=400, lam0=1e-2, K=K, gauge=True)
    return g
