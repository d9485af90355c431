"""crn_residual_host_batch: host-memory states through the pipelined copies
give exactly the device-path residuals, norms and dtmin."""
import numpy as np
import pytest

import coronal_inputs as ci
from _util import problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("count,pinned", [(0, True), (1, True), (5, True), (4, False)])
def test_host_batch_equals_device_residuals(precision, count, pinned):
    import paper_2209_04481_gb300 as pg
    shape = (12, 16, 32)
    g = pg.Grid(*shape, precision=precision, p_b=ci.parker_sound_speed2())
    _, Br = problem(shape)
    g.set_inner_boundary(torch.from_numpy(Br).cuda())
    dt = g.dtype
    Us = [torch.from_numpy(problem(shape, perturb=10 + i)[0]).to(dt) for i in range(count)]
    if pinned:
        Us = [u.pin_memory() for u in Us]
    Rs = [torch.empty_like(u) for u in Us]
    norms = torch.zeros((count, 9), dtype=torch.float64)
    dtmin = torch.zeros(count, dtype=torch.float64)
    g.residual_host_batch(Us, Rs, norms=norms, dtmin=dtmin)
    assert g.last_launch_count == count
    for i, u in enumerate(Us):
        nm = torch.zeros(9, dtype=torch.float64, device="cuda")
        dm = torch.zeros(1, dtype=torch.float64, device="cuda")
        R = g.residual(u.cuda(), norms=nm, dtmin=dm).cpu()
        assert torch.equal(R, Rs[i]), i
        assert torch.equal(nm.cpu(), norms[i]) and dm.item() == dtmin[i].item(), i
    g.sync_status()
