"""Local diagnostics (sidm_local_diagnostics) against the FP64 oracle.

Per particle: SPH density over its own kernel, kernel-weighted 1-D velocity
dispersion, effective cross-section (App. C, Eq. effective_cross_section), h/l
(Sect. 3.5, Eq. hDl) and the Knudsen number (Sect. 3.6, Eq. knudsen_number).
Tolerances: the mixed form evaluates W in FP32 from the canonical FP32
distance (relative error ~1e-7 per term) and sums FP64 moments of FP32
velocities; so rho to 1e-5, nu to 1e-5 of the local rms speed, and the
quantities that depend on nu to 1e-4.  The FP64 form differs from the oracle
only by summation order and by the GPU's own quadrature of sigma_eff (below
1e-6): rho to 1e-12, nu to 1e-9 of the rms speed, the rest to 2e-6.
"""
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


TOL = {"mixed": (1e-5, 1e-5, 1e-4), "fp64": (1e-12, 1e-9, 2e-6)}


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_local_diagnostics_match_oracle(precision):
    from paper_2506_06269_gb300 import sidm
    halos = [ics.hernquist(3000, 21), ics.nfw(5017, 22), ics.uniform_box(2000, 23), ics.uniform_box(33, 24)]
    ks = [32, 64, 16, 32]
    xs = [(1, 100.0, 0.5), (0, 10.0, 1.0), (1, 3.0, 0.8), (0, 1.0, 1.0)]
    G = 1.0
    b = ics.batch(halos)
    n = b.n
    ctx = sidm.Context(n_max=n, halo_max=len(halos), ngb_max=128, precision=precision,
                       flags=sidm.SIDM_FLAG_LOCAL_DIAG)
    dev = ctx.device
    vin = b.vel.astype(np.float32).astype(np.float64) if precision == "mixed" else b.vel
    pos = torch.tensor(b.pos, device=dev)
    vel = torch.tensor(vin, dtype=ctx.vdtype, device=dev)
    ids = torch.tensor(b.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(n, dtype=ctx.vdtype, device=dev)
    ctx.build_cells(b.offsets, pos, vel, ids)
    perm = ctx.perm(n).cpu().numpy().astype(np.int64)
    ctx.kernel_sizes(ks, h)
    vel_before = vel.clone()
    g = ctx.local_diagnostics(ctx.xs_tensor(xs), ctx.f64(b.mass), vel, n, G)
    got = {k: np.empty(n) for k in g}
    for k, v in g.items():
        got[k][perm] = v.cpu().numpy().astype(np.float64)
    assert ctx.status() == 0
    assert torch.equal(vel, vel_before)
    ctx.close()
    t_rho, t_nu, t_rest = TOL[precision]
    mode = O.MODE_MIXED if precision == "mixed" else O.MODE_FP64
    for hidx, hh in enumerate(halos):
        a, e = int(b.offsets[hidx]), int(b.offsets[hidx + 1])
        oh, _, _ = O.knn(hh.pos, hh.ids, ks[hidx], mode)
        o = O.local_diag(hh.pos, vin[:, a:e], oh, hh.mass, ks[hidx], xs[hidx], G)
        rms = np.sqrt((vin[:, a:e] ** 2).sum(0).mean())
        np.testing.assert_allclose(got["rho"][a:e], o["rho"], rtol=t_rho, atol=0)
        np.testing.assert_allclose(got["nu"][a:e], o["nu"], rtol=0, atol=t_nu * rms)
        for k in ("sigma_eff", "h_over_l", "kn"):
            np.testing.assert_allclose(got[k][a:e], o[k], rtol=t_rest, atol=0, err_msg=f"{k} halo {hidx}")


def test_local_diagnostics_need_the_flag():
    from paper_2506_06269_gb300 import sidm
    b = ics.batch([ics.uniform_box(200, 3)])
    ctx = sidm.Context(n_max=b.n, halo_max=1, ngb_max=32)
    dev = ctx.device
    pos = torch.tensor(b.pos, device=dev)
    vel = torch.tensor(b.vel.astype(np.float32), device=dev)
    ids = torch.tensor(b.ids.astype(np.int64), device=dev).to(torch.int32)
    ctx.build_cells(b.offsets, pos, vel, ids)
    ctx.kernel_sizes([16], torch.zeros(b.n, device=dev))
    with pytest.raises(sidm.SidmError):
        ctx.local_diagnostics(ctx.xs_tensor([(0, 1.0, 1.0)]), ctx.f64(b.mass), vel, b.n)
    ctx.close()
