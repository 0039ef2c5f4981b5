"""Bounded waits of the tensor-core M2L give up safely (failure detection without a GPU fault).

A wait limit of one try makes the pipeline waits of k_m2l_tc (levels 3-4) and k_m2l_lines
(16 to 64 cells per side and parity) give up on purpose: every CTA stops issuing, drains its own
copies and MMAs, frees its tensor memory and sets the timeout bit, so the evaluation reports
VFMM_ERR_TIMEOUT at vfmm_sync.  The same handle, with the default limit, then evaluates the
same field exactly as before."""
import numpy as np
import pytest

import workload as wl
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,depth", [(32, 3), (64, 4), (128, 5)])
def test_wait_give_up_reports_timeout_and_handle_recovers(n, depth):
    torch = torch_cuda()
    import paper_1110_2921_gb300 as vf
    from paper_1110_2921_gb300 import _native as nv
    f = wl.make_vortex_lattice(n, 4, 1)
    X = torch.tensor(f["x"], dtype=torch.float32, device="cuda")
    G = torch.tensor(f["alpha"], dtype=torch.float32, device="cuda")
    h = vf.VortexFMM(p=10, depth=depth, periodic_levels=2, m2l="bf16x3")
    try:
        h.build_tree(X)
        u0, s0 = h.eval(G, f["sigma"])
        h.sync()
        u0 = u0.double().cpu().numpy()
        s0 = s0.double().cpu().numpy()
        nv.vfmm_set_wait_limit(h.h, 1)
        h.eval(G, f["sigma"])
        with pytest.raises(vf.VfmmError) as e:
            h.sync()
        assert e.value.status == nv.VFMM_ERR_TIMEOUT
        nv.vfmm_set_wait_limit(h.h, 0)
        u1, s1 = h.eval(G, f["sigma"])
        h.sync()
        u1 = u1.double().cpu().numpy()
        s1 = s1.double().cpu().numpy()
    finally:
        h.close()
    assert np.array_equal(u0, u1) and np.array_equal(s0, s1)
