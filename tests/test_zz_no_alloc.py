"""The allocation-free adjoint entry point (ader_adjoint_step_static), for callers that cannot
allocate device memory when they call it: its work memory is a fixed device array inside the
library.  Checked through the C ABI against the allocating entry point on two calls in a row
(the shared array keeps the previous call's contents, which must not leak into the next)."""
import numpy as np
import pytest
import torch

from paper_1905_07987_gb300 import ader, synth
from cases import Case

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(autouse=True, scope="module")
def _build():
    from paper_1905_07987_gb300 import build
    build.build()


def _case(order, ncell, seed):
    mat = synth.elastic_material(ncell, seed=seed)
    hi = tuple(0.5 * n for n in ncell)
    c = Case("elastic", 3, order, ncell, hi=hi, bc="absorbing", material=mat)
    c.point_source(tuple(0.4 * h for h in hi), synth.moment_tensor(seed=seed), 2.0, 0.5)
    return c


def _adjoint(c, u_n, lam0, dJ, static):
    lam = lam0.clone()
    gm = torch.zeros(c.ctx.cells * 3, dtype=torch.float64, device="cuda")
    gM = torch.zeros(6, dtype=torch.float64, device="cuda")
    c.ctx.adjoint_step(0.31, 2e-3, u_n, lam, gm, gM, dJdu=dJ, static=static)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), gm.cpu().numpy(), gM.cpu().numpy()


def _close(a, b):
    return np.abs(a - b).max() <= TOL * max(np.abs(b).max(), 1e-300)


def test_static_adjoint_matches_allocating_adjoint_on_consecutive_calls():
    rng = np.random.default_rng(7)
    for order, ncell in ((3, (3, 2, 3)), (2, (2, 3, 2))):
        c = _case(order, ncell, seed=order)
        for call in range(2):
            u_n = torch.from_numpy(rng.standard_normal(c.ctx.count)).cuda()
            lam0 = torch.from_numpy(rng.standard_normal(c.ctx.count)).cuda()
            dJ = torch.from_numpy(rng.standard_normal(c.ctx.count)).cuda() if call else None
            ref = _adjoint(c, u_n, lam0, dJ, static=False)
            got = _adjoint(c, u_n, lam0, dJ, static=True)
            for a, b in zip(got, ref):
                assert _close(a, b), (order, call)


def test_static_adjoint_rejects_grids_beyond_its_array():
    c = _case(4, (20, 20, 20), seed=1)  # face adjoints alone need about 86 MB
    u = torch.zeros(c.ctx.count, dtype=torch.float64, device="cuda")
    gm = torch.zeros(c.ctx.cells * 3, dtype=torch.float64, device="cuda")
    gM = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(ader.AderError) as e:
        c.ctx.adjoint_step(0.0, 1e-3, u, u.clone(), gm, gM, static=True)
    assert e.value.status == ader.EINVAL
