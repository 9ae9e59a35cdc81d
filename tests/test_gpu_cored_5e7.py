"""Parity at the largest workload: a cored-isothermal halo matched to NFW,
N = 5e7 particles (King-like core of radius 0.05 r_s, central density 1e3
rho_s; about 2.4 GB of FP32 SoA), run at its full size on the GPU.

The oracle cannot redo a step of 5e7 particles within a test, so it checks the
outputs it can compute one by one, and the step is checked by properties that
hold at any size:
  - kernel sizes (Sect. 2) of 2,304 particles -- random, innermost and
    outermost -- bit-exact at every N_ngb of the sweep {16, 32, 64, 128};
  - the scatter step (N_ngb = 64, sigma(v) of Eq. vel_dep): the change of the
    total kinetic energy equals the FP64 sum of the per-event changes, which
    is at the FP32 rounding level; momentum is conserved to the same level
    (Sect. 2, 5); the number of events is Poisson around half the summed
    pair probabilities (Sect. 3.5).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_06269_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

N, SEED_IC, S0, DT, SEED = 50_000_000, 2, 100.0, 1e-4, 77
SWEEP = (16, 32, 64, 128)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_06269_gb300 import build
    build.build()


def test_cored_nfw_5e7_kernel_size_sweep_and_step_properties():
    from paper_2506_06269_gb300 import sidm
    halo = ics.cored_nfw(N, SEED_IC)
    vmax = ics.nfw_vmax()
    r = np.linalg.norm(halo.pos, axis=0)
    order = np.argsort(r)
    rng = np.random.default_rng(11)
    sample = np.unique(np.concatenate([rng.choice(N, 2048, replace=False), order[:128], order[-128:]]))
    del r, order

    ctx = sidm.Context(n_max=N, halo_max=1, ngb_max=128, event_cap=1 << 21, precision="mixed",
                       flags=sidm.SIDM_FLAG_SUM_P)
    dev = ctx.device
    pos = torch.tensor(halo.pos, device=dev)
    vel = torch.tensor(halo.vel.astype(np.float32), device=dev)
    ids = torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(N, dtype=torch.float32, device=dev)
    ctx.build_cells([0, N], pos, vel, ids)
    perm = ctx.perm(N).to(torch.int64)
    inv = torch.empty_like(perm)
    inv[perm] = torch.arange(N, device=dev)                       # input index -> sorted position
    at = inv[torch.tensor(sample, device=dev)]
    h_gpu = {}
    for k in SWEEP:
        ctx.kernel_sizes([k], h)
        h_gpu[k] = h[at].cpu().numpy()
    assert ctx.status() == 0

    # one scatter step at N_ngb = 64 and its conservation properties
    mass = ctx.f64([halo.mass])
    e0 = torch.zeros((1, 4), dtype=torch.float64, device=dev)
    e1 = torch.zeros((1, 4), dtype=torch.float64, device=dev)
    ctx.energy_momentum(mass, vel, e0)
    ctx.scatter_step(SEED, 0, ctx.xs_tensor([(1, S0, vmax)]), ctx.f64([DT]), mass, vel)
    ctx.energy_momentum(mass, vel, e1)
    st = ctx.stats()
    assert ctx.status() == 0 and st.status == 0
    sum_p = float(ctx.sum_p(N).double().sum().item())
    E0, E1 = e0.cpu().numpy()[0], e1.cpu().numpy()[0]
    ctx.close()

    assert st.n_events > 1000
    lam = 0.5 * sum_p
    assert abs(st.n_events - lam) < 5 * math.sqrt(lam)
    assert abs((E1[0] - E0[0]) - st.d_energy) <= 1e-12 * E0[0]
    assert abs(E1[0] - E0[0]) <= 1e-9 * E0[0]
    p_scale = halo.mass * np.abs(halo.vel).sum() / 3.0
    assert np.all(np.abs(E1[1:] - E0[1:]) <= 1e-9 * p_scale)

    # kernel sizes of the sample for the whole sweep from one oracle search
    hs = O.knn_sample(halo.pos, halo.ids, max(SWEEP), sample, O.MODE_MIXED)
    for k in SWEEP:
        assert np.array_equal(h_gpu[k], hs[:, k - 1].astype(np.float32)), k
