"""Parity at the full benchmark size, in the launch configuration bench.py times.

Workload: NFW halo truncated at 10 r_s, N = 2^20, N_ngb = 64,
sigma/m = 100 / (1 + (v/v_max)^2)^2, one drift + rebuild + step with the
kernel sizes warm-started from the previous step (default context settings,
as in bench.py).  Checked against the FP64 oracle on host-side inputs:
  - every one of the 2^20 kernel sizes bit-exact (Sect. 2; reading C1/C2');
  - for a sample of particles (random, innermost, outermost), every pair they
    take part in is evaluated by the oracle, and the drawn events involving
    them must agree except pairs with |P - u| < 1e-6 (Sect. 3.5);
  - particles of the sample in exactly one event have the oracle's
    post-scatter velocities to 1e-5 of the pair speed scale (Sect. 2, 5);
    the others of the sample without an event are bit-unchanged.
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

N, K, S0, SEED_IC, DT, SEED = 1 << 20, 64, 100.0, 1, 0.005, 20250617


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_06269_gb300 import build
    build.build()


def test_fullsize_nfw_kernel_sizes_events_velocities():
    from paper_2506_06269_gb300 import sidm
    halo = ics.nfw(N, SEED_IC)
    vmax = ics.nfw_vmax()
    vel32 = halo.vel.astype(np.float32)
    ctx = sidm.Context(n_max=N, halo_max=1, ngb_max=K, event_cap=1 << 17, precision="mixed")
    dev = ctx.device
    pos = torch.tensor(halo.pos, device=dev)
    vel = torch.tensor(vel32, device=dev)
    ids = torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(N, dtype=torch.float32, device=dev)
    # step 0 on the initial state (cold search)
    ctx.build_cells([0, N], pos, vel, ids)
    ctx.kernel_sizes([K], h)
    perm1 = ctx.perm(N).cpu().numpy().astype(np.int64)          # sorted -> input index
    # step 1: a ballistic drift computed on the host (FP64, input order); the GPU
    # receives the same values in the order it left, so the search is warm-started
    pos2 = halo.pos + vel32.astype(np.float64) * DT
    pos.copy_(torch.tensor(pos2[:, perm1], device=dev))
    ctx.diagnostics(reset=True)
    ctx.build_cells([0, N], pos, vel, ids)
    ctx.kernel_sizes([K], h)
    ctx.scatter_step(SEED, 1, ctx.xs_tensor([(1, S0, vmax)]), ctx.f64([DT]), ctx.f64([halo.mass]), vel)
    assert ctx.status() == 0
    diag = ctx.diagnostics(reset=True)
    assert diag[7] < N // 100, "warm start redid too many searches"
    perm2 = ctx.perm(N).cpu().numpy().astype(np.int64)
    to_input = perm1[perm2]                                       # sorted (step 1) -> input index
    h_gpu = np.empty(N, np.float32); h_gpu[to_input] = h.cpu().numpy()
    v_gpu = np.empty((3, N)); v_gpu[:, to_input] = vel.cpu().numpy().astype(np.float64)
    n_ev, ev_g = ctx.events()
    assert n_ev == len(ev_g)
    ctx.close()

    # every kernel size, bit-exact
    h_o, _, _ = O.knn(pos2, halo.ids, K, O.MODE_MIXED)
    assert np.array_equal(h_gpu, h_o.astype(np.float32))

    # sampled pairs and events
    rng = np.random.default_rng(7)
    r = np.linalg.norm(halo.pos, axis=0)
    order = np.argsort(r)
    sample = np.unique(np.concatenate([rng.choice(N, 1024, replace=False), order[:64], order[-64:]]))
    mask = np.zeros(N, bool); mask[sample] = True
    vin = vel32.astype(np.float64)
    ev_o, _, _ = O.pairs(pos2, vin, halo.ids, h_o, O.MODE_MIXED, (1, S0, vmax), halo.mass, DT, SEED, 1, 0,
                         mask=mask)
    ev_g = ev_g.copy()
    ev_g["i"] = to_input[ev_g["i"]]; ev_g["j"] = to_input[ev_g["j"]]
    mine = mask[ev_g["i"]] | mask[ev_g["j"]]
    only_o, only_g = compare_events(ev_g[mine], ev_o)
    assert len(ev_o) > 0

    # velocities of sampled particles in exactly one (GPU) event
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
    assert checked > 0
    quiet = sample[count[sample] == 0]
    assert np.array_equal(v_gpu[:, quiet], vin[:, quiet])


def _local_event(e):
    """The event e re-indexed onto a two-particle array (i -> 0, j -> 1)."""
    out = np.array([e]).copy()
    out["i"] = 0
    out["j"] = 1
    return out


def test_fullsize_energy_drift_1000_steps():
    """1000 steps of the benchmark workload (ballistic drift, cell build,
    kernel sizes, scatter, exact sums every step): the total kinetic energy
    drifts by less than 1e-4 (the scatter conserves it pairwise, Sect. 2), and
    the drift equals the FP64 sum of the per-event changes."""
    from paper_2506_06269_gb300 import sidm
    halo = ics.nfw(N, SEED_IC)
    vmax = ics.nfw_vmax()
    ctx = sidm.Context(n_max=N, halo_max=1, ngb_max=K, event_cap=1 << 17, precision="mixed")
    dev = ctx.device
    pos = torch.tensor(halo.pos, device=dev)
    vel = torch.tensor(halo.vel.astype(np.float32), device=dev)
    ids = torch.tensor(halo.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(N, dtype=torch.float32, device=dev)
    xs, dt, mass = ctx.xs_tensor([(1, S0, vmax)]), ctx.f64([DT]), ctx.f64([halo.mass])
    steps = 1000
    E = torch.zeros((steps + 1, 4), dtype=torch.float64, device=dev)
    stats = torch.zeros((steps, sidm.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    ctx.build_cells([0, N], pos, vel, ids)
    ctx.energy_momentum(mass, vel, E[0])
    for i in range(steps):
        ctx.drift(dt, pos, vel)
        ctx.build_cells([0, N], pos, vel, ids)
        ctx.kernel_sizes([K], h)
        ctx.scatter_step(SEED, i, xs, dt, mass, vel, stats[i])
        ctx.energy_momentum(mass, vel, E[i + 1])
    assert ctx.status() == 0
    e = E[:, 0].cpu().numpy()
    st = np.frombuffer(stats.cpu().numpy().tobytes(), dtype=sidm.STATS_DTYPE)
    ctx.close()
    drift = np.abs(e - e[0]) / e[0]
    print(f"1000 steps: max drift {drift.max():.3g}, events per step {st['n_events'].mean():.0f}")
    assert drift.max() < 1e-4
    assert st["n_events"].sum() > 50 * 1000 and np.all(st["status"] == 0)
    # the drift (ballistic drift leaves the velocities alone) is the sum of
    # the per-step energy changes booked by the scatter
    assert abs((e[-1] - e[0]) - st["d_energy"].sum()) <= 1e-12 * e[0]
