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
