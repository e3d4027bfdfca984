"""Training-set preparation of the learned warm start, in the library's kernels, against FP64 NumPy.

Row gathers are compared bit for bit; column statistics (FP64 on both sides, different summation
order) within 1e-12 relative; standardisation (FP64 then rounded to FP32) within one FP32 rounding
of the FP64 value; the folded network (raw inputs in, raw outputs out) against the oracle's FP64
forward pass of the unfolded network on standardised inputs, scaled back, within 1e-5 of the
largest output (the FP32 forward pass's bar).
"""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_1502_06974_gb300 import api

pytestmark = pytest.mark.gpu


def _data(seed=5, m=3000, w=48):
    r = np.random.default_rng(seed)
    scale = r.uniform(0.1, 5.0, w)
    x = ((r.normal(size=(m, w)) + r.normal(size=w)) * scale).astype(np.float32)
    x[:, 41:] = 0.0                     # constant columns, as the features' padding
    x[:, 40] = 0.25                     # a constant non-zero column
    return x


def test_rows_gather_bit_exact(gpu_lib):
    x = _data()
    idx = np.random.default_rng(1).integers(0, x.shape[0], 5001)
    got = api.rows_gather_f32(torch.from_numpy(x).cuda(), idx).cpu().numpy()
    assert np.array_equal(got, x[idx])


@pytest.mark.parametrize("use_index", [False, True])
def test_col_stats_and_standardize(gpu_lib, use_index):
    x = _data()
    idx = np.sort(np.random.default_rng(2).choice(x.shape[0], 2100, replace=False)) if use_index else None
    xd = torch.from_numpy(x).cuda()
    mu, sd = api.col_stats_f32(xd, idx, zero_const_mean=True)
    sel = x[idx].astype(np.float64) if use_index else x.astype(np.float64)
    rmu, rsd = sel.mean(axis=0), sel.std(axis=0)
    const = rsd < 1e-12
    rsd[const] = 1.0
    rmu[const] = 0.0
    mu, sd = mu.cpu().numpy(), sd.cpu().numpy()
    assert np.all(sd[const] == 1.0) and np.all(mu[const] == 0.0)
    assert np.max(np.abs(mu - rmu) / np.maximum(np.abs(rmu), rsd)) < 1e-12
    assert np.max(np.abs(sd - rsd) / rsd) < 1e-12
    _, sd_keep = api.col_stats_f32(xd, idx, zero_const_mean=False)
    mu_keep, _ = api.col_stats_f32(xd, idx, zero_const_mean=False)
    assert mu_keep.cpu().numpy()[40] == pytest.approx(0.25)           # mean kept when not asked to zero it
    xs = api.standardize_f32(xd, torch.from_numpy(rmu).cuda(), torch.from_numpy(rsd).cuda()).cpu().numpy()
    ref = (x.astype(np.float64) - rmu) / rsd
    assert np.array_equal(xs, ref.astype(np.float32))
    xs2 = api.standardize_f32(xd, None, sd_keep).cpu().numpy()
    assert np.array_equal(xs2, (x.astype(np.float64) / sd_keep.cpu().numpy()).astype(np.float32))


def test_fold_standardization_matches_unfolded_network(gpu_lib):
    dims = api.MLP_DIMS
    x = _data(m=512)
    r = np.random.default_rng(3)
    p = omlp.init_params(dims, r)
    p[dims[0] * dims[1]:dims[0] * dims[1] + dims[1]] = r.normal(0, 0.1, dims[1])   # non-zero b1
    p[-dims[3]:] = r.normal(0, 0.1, dims[3])                                        # non-zero b3
    p = p.astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    mu, sd = api.col_stats_f32(xd, None, zero_const_mean=True)
    tsd = torch.from_numpy(r.uniform(0.01, 2.0, dims[3])).cuda()
    net = api.Mlp(p, 'cuda', dims)
    api.mlp_fold_standardization(net, mu, sd, tsd)
    y = api.mlp_forward_f32(net, xd).cpu().numpy().astype(np.float64)
    xs = (x.astype(np.float64) - mu.cpu().numpy()) / sd.cpu().numpy()
    ref = omlp.forward(p.astype(np.float64), dims, xs)[2] * tsd.cpu().numpy()
    assert np.max(np.abs(y - ref)) < 1e-5 * np.max(np.abs(ref))
