"""Reflecting spherical boundary (sidm_reflect_boundary) against the oracle
(Sect. 2: outward-moving particles beyond a sphere about the halo are turned
back, the energy unchanged).  Two halos with their own spheres and a third
with none; the same particles are reflected on both sides (the decision is
taken in FP64 on the same FP32 velocities and FP64 positions), and the new
velocities agree to FP32 rounding (1e-6 of the speed) and keep the speed."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_06269_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_06269_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_reflect_boundary_matches_oracle(precision):
    from paper_2506_06269_gb300 import sidm
    halos = [ics.nfw(20000, 61), ics.hernquist(7000, 62), ics.nfw(3000, 63)]
    bounds = [(0.3, -0.1, 0.2, 2.0), (0.0, 0.0, 0.0, 5.0), (0.0, 0.0, 0.0, 0.0)]
    b = ics.batch(halos)
    n = b.n
    ctx = sidm.Context(n_max=n, halo_max=3, ngb_max=32, precision=precision)
    dev = ctx.device
    vdt = np.float32 if precision == "mixed" else np.float64
    vin = b.vel.astype(vdt).astype(np.float64)
    pos = torch.tensor(b.pos, device=dev)
    vel = torch.tensor(vin.astype(vdt), device=dev)
    ids = torch.tensor(b.ids.astype(np.int64), device=dev).to(torch.int32)
    ctx.build_cells(b.offsets, pos, vel, ids)
    perm = ctx.perm(n).cpu().numpy().astype(np.int64)
    bd = torch.tensor(np.array(bounds, dtype=np.float64), device=dev)
    ctx.reflect_boundary(bd, pos, vel)
    assert ctx.status() == 0
    got = np.empty((3, n)); got[:, perm] = vel.cpu().numpy().astype(np.float64)
    ctx.close()
    for h in range(3):
        a, e = int(b.offsets[h]), int(b.offsets[h + 1])
        want = O.reflect(b.pos[:, a:e], vin[:, a:e], bounds[h][:3], bounds[h][3])
        moved_o = np.any(want != vin[:, a:e], axis=0)
        moved_g = np.any(got[:, a:e] != vin[:, a:e], axis=0)
        assert np.array_equal(moved_o, moved_g), h
        speed = np.linalg.norm(want, axis=0)
        tol = 1e-6 if precision == "mixed" else 1e-14
        assert np.all(np.abs(got[:, a:e] - want).max(axis=0) <= tol * speed), h
        if h < 2:
            assert moved_o.sum() > 20
        else:
            assert not moved_o.any()
