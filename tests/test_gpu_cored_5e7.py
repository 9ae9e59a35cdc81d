"""Parity at the largest workload: a cored-isothermal halo matched to NFW,
N = 5e7 particles (King-like core of radius 0.05 r_s, central density 1e3
rho_s; about 2.4 GB of FP32 SoA), run at its full size on the GPU in the
launch configuration bench.py times (default context, draws with the upper
bound of P, no per-particle sums).

Checked against the FP64 oracle on the same seeded inputs:
  - mixed form, N_ngb = 64: every one of the 5e7 kernel sizes bit-exact
    (Sect. 2; one full oracle search with its k-d tree);
  - the scatter step (sigma(v) of Eq. vel_dep): the oracle's pair pass
    restricted to the pairs with an endpoint in the 1/64 id subset
    (ids divisible by 64) -- every drawn event touching the subset agrees
    except pairs with |P - u| < 1e-6 (Sect. 3.5); subset particles in exactly
    one event (whose partner is in no other event) have the oracle's
    post-scatter velocities to 1e-5 of the pair speed; subset particles in no
    event are bit-unchanged; the total kinetic energy changes by the FP64 sum
    of the per-event changes and momentum is conserved (Sect. 2, 5);
  - kernel sizes of 2,304 particles (random, innermost, outermost) at every
    N_ngb of the sweep {16, 32, 64, 128}, in the mixed and the all-FP64 forms.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_06269_gb300 import ics

from gpu_helpers import compare_events

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

N, SEED_IC, S0, DT, SEED, K = 50_000_000, 2, 100.0, 1e-4, 77, 64
SWEEP = (16, 32, 128, 64)          # 64 last: the scatter step uses its kernel sizes


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_06269_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def halo():
    return ics.cored_nfw(N, SEED_IC)


@pytest.fixture(scope="module")
def sample(halo):
    r = np.linalg.norm(halo.pos, axis=0)
    order = np.argsort(r)
    rng = np.random.default_rng(11)
    return np.unique(np.concatenate([rng.choice(N, 2048, replace=False), order[:128], order[-128:]]))


def _local_event(e):
    """The event e re-indexed onto a two-particle array (i -> 0, j -> 1)."""
    out = np.array([e]).copy()
    out["i"] = 0
    out["j"] = 1
    return out


def test_cored_nfw_5e7_kernel_sizes_events_velocities(halo, sample):
    from paper_2506_06269_gb300 import sidm
    vmax = ics.nfw_vmax()
    vel32 = halo.vel.astype(np.float32)
    ctx = sidm.Context(n_max=N, halo_max=1, ngb_max=128, event_cap=1 << 22, precision="mixed")
    dev = ctx.device
    pos = torch.tensor(halo.pos, device=dev)
    vel = torch.tensor(vel32, device=dev)
    ids = torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(N, dtype=torch.float32, device=dev)
    ctx.build_cells([0, N], pos, vel, ids)
    perm = ctx.perm(N).to(torch.int64)                            # sorted position -> input index
    inv = torch.empty_like(perm)
    inv[perm] = torch.arange(N, device=dev)                       # input index -> sorted position
    at = inv[torch.tensor(sample, device=dev)]
    h_sample = {}
    for k in SWEEP:
        ctx.kernel_sizes([k], h)
        h_sample[k] = h[at].cpu().numpy()
    assert ctx.status() == 0
    h_all = np.empty(N, np.float32)
    h_all[perm.cpu().numpy()] = h.cpu().numpy()                   # N_ngb = 64, input order

    mass = ctx.f64([halo.mass])
    e0 = torch.zeros((1, 4), dtype=torch.float64, device=dev)
    e1 = torch.zeros((1, 4), dtype=torch.float64, device=dev)
    ctx.energy_momentum(mass, vel, e0)
    ctx.scatter_step(SEED, 0, ctx.xs_tensor([(1, S0, vmax)]), ctx.f64([DT]), mass, vel)
    ctx.energy_momentum(mass, vel, e1)
    st = ctx.stats()
    assert ctx.status() == 0 and st.status == 0
    n_ev, ev_g = ctx.events()
    assert n_ev == len(ev_g)
    pm = perm.cpu().numpy()
    v_gpu = np.empty((3, N)); v_gpu[:, pm] = vel.cpu().numpy().astype(np.float64)
    E0, E1 = e0.cpu().numpy()[0], e1.cpu().numpy()[0]
    ctx.close()
    del pos, vel, ids, h, perm, inv
    torch.cuda.empty_cache()

    # conservation of the whole step (FP32 velocities, FP64 sums)
    assert st.n_events > 1000
    assert abs((E1[0] - E0[0]) - st.d_energy) <= 1e-12 * E0[0]
    assert abs(E1[0] - E0[0]) <= 1e-9 * E0[0]
    p_scale = halo.mass * np.abs(halo.vel).sum() / 3.0
    assert np.all(np.abs(E1[1:] - E0[1:]) <= 1e-9 * p_scale)

    # every kernel size, bit-exact
    h_o, _, _ = O.knn(halo.pos, halo.ids, K, O.MODE_MIXED)
    assert np.array_equal(h_all, h_o.astype(np.float32))

    # the oracle's pair pass on the pairs touching the 1/64 id subset
    mask = (halo.ids % 64) == 0
    vin = vel32.astype(np.float64)
    ev_o, st_o, _ = O.pairs(halo.pos, vin, halo.ids, h_o, O.MODE_MIXED, (1, S0, vmax), halo.mass, DT, SEED, 0, 0,
                            mask=mask, ev_cap=1 << 22)
    ev_g = ev_g.copy()
    ev_g["i"] = pm[ev_g["i"]]; ev_g["j"] = pm[ev_g["j"]]
    mine = mask[ev_g["i"]] | mask[ev_g["j"]]
    only_o, only_g = compare_events(ev_g[mine], ev_o)
    assert len(ev_o) > 30

    # velocities: subset particles in exactly one event whose partner has no other
    count = np.bincount(np.concatenate([ev_g["i"], ev_g["j"]]).astype(np.int64), minlength=N)
    differ = set(only_o) | set(only_g)
    checked = 0
    for e in ev_o:
        i, j = int(e["i"]), int(e["j"])
        if int(e["key"]) in differ or count[i] != 1 or count[j] != 1:
            continue
        v1, _ = O.apply_events(_local_event(e), np.full(2, halo.mass), vin[:, [i, j]])
        scale = np.linalg.norm(vin[:, i]) + np.linalg.norm(vin[:, j])
        assert np.abs(v_gpu[:, [i, j]] - v1).max() <= 1e-5 * scale
        checked += 1
    assert checked > 20
    quiet = np.flatnonzero(mask & (count == 0))
    assert quiet.size > 0.9 * mask.sum()
    assert np.array_equal(v_gpu[:, quiet], vin[:, quiet])

    # kernel sizes of the sample at every N_ngb of the sweep, from one oracle search
    hs = O.knn_sample(halo.pos, halo.ids, max(SWEEP), sample, O.MODE_MIXED)
    for k in SWEEP:
        assert np.array_equal(h_sample[k], hs[:, k - 1].astype(np.float32)), k


def test_cored_nfw_5e7_fp64_form_kernel_sizes(halo, sample):
    """The all-FP64 form at full size: sampled kernel sizes over the sweep."""
    from paper_2506_06269_gb300 import sidm
    ctx = sidm.Context(n_max=N, halo_max=1, ngb_max=128, event_cap=1 << 16, precision="fp64")
    dev = ctx.device
    pos = torch.tensor(halo.pos, device=dev)
    vel = torch.tensor(halo.vel, device=dev)
    ids = torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(N, dtype=torch.float64, device=dev)
    ctx.build_cells([0, N], pos, vel, ids)
    perm = ctx.perm(N).to(torch.int64)
    inv = torch.empty_like(perm)
    inv[perm] = torch.arange(N, device=dev)
    at = inv[torch.tensor(sample, device=dev)]
    got = {}
    for k in SWEEP:
        ctx.kernel_sizes([k], h)
        got[k] = h[at].cpu().numpy()
    assert ctx.status() == 0
    ctx.close()
    hs = O.knn_sample(halo.pos, halo.ids, max(SWEEP), sample, O.MODE_FP64)
    for k in SWEEP:
        assert np.array_equal(got[k], hs[:, k - 1]), k
