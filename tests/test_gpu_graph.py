"""The batched pass captured in a CUDA graph, as bench.py runs it.

An 8-halo batch (NFW halos of uneven N, N_ngb 16/32/64/128 round-robin,
sigma/m = 10) advances five steps -- drift, cell build, kernel sizes, scatter,
energy/momentum -- once as eager launches and once as one captured CUDA graph
replayed from the same state.  The replay must give the same bits as the eager
steps: positions, velocities, ids, kernel sizes and the energy/momentum sums
after every step, the step statistics, and the events of the last step.
Step 0 of the eager run is checked against the FP64 oracle on the four
smallest halos: kernel sizes bit-exact (Sect. 2), events except pairs with
|P - u| < 1e-6 (Sect. 3.5), velocities within 1e-5 of each scatter's pair
speed (Sect. 2, 5).  The time step is a power of two, so the drift
x + v dt (one FP64 fused multiply-add on the GPU) is exact in the host's
separate product and sum as well.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2506_06269_gb300 import ics

from gpu_helpers import compare_events, tainted_particles, velocity_scale

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

SIZES = (1500, 2600, 4100, 6200, 9000, 14000, 21000, 30000)
KS = (16, 32, 64, 128, 16, 32, 64, 128)
STEPS, SEED, DT = 5, 424242, 2.0 ** -6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_06269_gb300 import build
    build.build()


def _run(b, graph):
    """Prologue (layout, kernel sizes, launch set-up; no state change), then
    STEPS steps, eager or as one replayed graph; per-step copies of the state."""
    from paper_2506_06269_gb300 import sidm
    H, n = b.n_halos, b.n
    ctx = sidm.Context(n_max=n, halo_max=H, ngb_max=128, event_cap=1 << 18)
    dev = ctx.device
    pos = torch.tensor(b.pos, device=dev)
    vel = torch.tensor(b.vel.astype(np.float32), device=dev)
    ids = torch.tensor(b.ids.astype(np.int64), device=dev).to(torch.int32)
    h = torch.zeros(n, dtype=torch.float32, device=dev)
    xs = ctx.xs_tensor([(0, 10.0, 1.0)] * H)
    xs0 = ctx.xs_tensor([(0, 0.0, 1.0)] * H)
    dt = ctx.f64([DT] * H)
    dt0 = ctx.f64([0.0] * H)
    mass = ctx.f64(b.mass)
    rec = {"pos": torch.zeros((STEPS, 3, n), dtype=torch.float64, device=dev),
           "vel": torch.zeros((STEPS, 3, n), dtype=torch.float32, device=dev),
           "ids": torch.zeros((STEPS, n), dtype=torch.int32, device=dev),
           "h": torch.zeros((STEPS, n), dtype=torch.float32, device=dev),
           "E": torch.zeros((STEPS, H, 4), dtype=torch.float64, device=dev),
           "stats": torch.zeros((STEPS, sidm.STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)}
    # prologue: a zero drift and a zero cross-section change nothing, but
    # upload the layout and N_ngb and set up every launch before any capture
    ctx.build_cells(b.offsets, pos, vel, ids)
    perm0 = ctx.perm(n).cpu().numpy().astype(np.int64)
    ctx.kernel_sizes(list(KS), h)
    ctx.drift(dt0, pos, vel)
    ctx.scatter_step(SEED, 99, xs0, dt, mass, vel)
    ctx.energy_momentum(mass, vel, rec["E"][0])
    torch.cuda.synchronize()
    assert ctx.status() == 0
    state0 = (pos.cpu().numpy().copy(), vel.cpu().numpy().copy(), ids.cpu().numpy().copy())

    def step(i):
        ctx.drift(dt, pos, vel)
        ctx.build_cells(b.offsets, pos, vel, ids)
        ctx.kernel_sizes(list(KS), h)
        ctx.scatter_step(SEED, i, xs, dt, mass, vel, rec["stats"][i])
        ctx.energy_momentum(mass, vel, rec["E"][i])
        rec["pos"][i].copy_(pos); rec["vel"][i].copy_(vel); rec["ids"][i].copy_(ids); rec["h"][i].copy_(h)

    out = {"perm0": perm0, "state0": state0}
    if graph:
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            for i in range(STEPS):
                step(i)
        g.replay()
        torch.cuda.synchronize()
        del g
    else:
        for i in range(STEPS):
            step(i)
            if i == 0:
                torch.cuda.synchronize()
                out["perm1"] = ctx.perm(n).cpu().numpy().astype(np.int64)
                out["events0"] = ctx.events()[1].copy()
        torch.cuda.synchronize()
    assert ctx.status() == 0
    out["events_last"] = np.sort(ctx.events()[1], order="key")
    out.update({k: v.cpu().numpy() for k, v in rec.items()})
    out["stats"] = [sidm.parse_stats(rec["stats"][i]) for i in range(STEPS)]
    ctx.close()
    return out


def test_graph_replay_equals_eager_steps_and_step0_matches_oracle():
    halos = [ics.nfw(n, 7000 + t) for t, n in enumerate(SIZES)]
    b = ics.batch(halos)
    eager = _run(b, graph=False)
    replay = _run(b, graph=True)
    for key in ("pos", "vel", "ids", "h", "E"):
        assert np.array_equal(eager[key], replay[key]), key
    for se, sr in zip(eager["stats"], replay["stats"]):
        assert se == sr
    assert sum(s.n_events for s in eager["stats"]) > 100
    assert np.array_equal(eager["events_last"], replay["events_last"])

    # step 0 of the eager run against the oracle, four smallest halos.  Its
    # input is the prologue's state (the arrays in the order of the first cell
    # build) drifted by dt on the host.
    pos0, vel0, ids0 = eager["state0"]
    pos_in = pos0 + vel0.astype(np.float64) * DT
    perm1 = eager["perm1"]                                  # step-0 sorted -> prologue order
    ev = eager["events0"].copy()
    ev["i"] = perm1[ev["i"]]; ev["j"] = perm1[ev["j"]]
    h1 = np.empty(b.n, np.float32); h1[perm1] = eager["h"][0]
    v1 = np.empty((3, b.n)); v1[:, perm1] = eager["vel"][0].astype(np.float64)
    for hidx in np.argsort(SIZES)[:4]:
        a, e = int(b.offsets[hidx]), int(b.offsets[hidx + 1])
        p, v, idh = pos_in[:, a:e], vel0[:, a:e].astype(np.float64), ids0[a:e].view(np.uint32)
        oh, _, _ = O.knn(p, idh, KS[hidx], O.MODE_MIXED)
        assert np.array_equal(h1[a:e], oh.astype(np.float32)), hidx
        oev, _, _ = O.pairs(p, v, idh, oh, O.MODE_MIXED, (0, 10.0, 1.0), b.mass[hidx], DT, SEED, 0, int(hidx))
        vout, _ = O.apply_events(oev, np.full(e - a, b.mass[hidx]), v)
        ge = ev[(ev["i"] >= a) & (ev["i"] < e)].copy()
        ge["i"] -= a; ge["j"] -= a
        only_o, only_g = compare_events(ge, oev)
        bad = tainted_particles(oev, ge, only_o + only_g, e - a)
        scale = velocity_scale(oev, v, np.full(e - a, b.mass[hidx]))
        err = np.abs(v1[:, a:e] - vout).max(axis=0)
        assert np.all(err[~bad] <= 1e-5 * scale[~bad] + 1e-30), hidx
