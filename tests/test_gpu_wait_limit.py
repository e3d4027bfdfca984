"""A bounded wait that runs out ends the call with an error status, and the context stays usable.

The 2x2 accumulate kernel of the moment path waits for each tile's bulk copies on an mbarrier with
a bounded number of polls.  With the bound set to zero every such wait gives up at once: the kernel
waits (with the default bound) for the copies it has in flight, records the failure and ends; the
calibrate call must return GC_ERR_CUDA naming the incomplete copy.  Afterwards, with the default
bound restored, the same call on the same context gives bitwise the same result as before.
"""
import pytest
import torch

from helpers import device_batch
from paper_1502_06974_gb300 import _native as N
from paper_1502_06974_gb300 import api, synth

pytestmark = pytest.mark.gpu


def test_bulk_copy_wait_runs_out(gpu_lib, monkeypatch):
    monkeypatch.setenv("GAINCAL_ACC_PREFETCH", "3")   # the bulk-copy accumulate kernel
    b = synth.make_config(2, small=True)
    vis, model, g0, lay = device_batch(b)
    kw = dict(schedule='stefcal', tol=1e-6, max_iter=40, path=N.GC_PATH_MOMENTS)
    g_ref, it_ref, _, st_ref = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), **kw)
    torch.cuda.synchronize()
    api.set_wait_limit(0)
    try:
        with pytest.raises(RuntimeError, match='did not complete'):
            api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), **kw)
    finally:
        api.set_wait_limit(-1)
    torch.cuda.synchronize()                          # no sticky CUDA error
    g, it, _, st = api.calibrate_di_jones2x2(vis, model, lay, g0.clone(), **kw)
    torch.cuda.synchronize()
    assert torch.equal(g, g_ref)
    assert torch.equal(it, it_ref) and torch.equal(st, st_ref)
