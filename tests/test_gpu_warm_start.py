"""Warm-started kernel sizes (sidm_warm_start) are bit-identical to cold ones.

The search seeded with the previous step's h only admits candidates inside
knn_slack h_prev (1.07 by default) and redoes, from scratch, every particle that finds fewer than
N_ngb of them; the k-th distance is exact either way (Sect. 2 kernel size).
These tests run a warm and a cold context side by side on identical inputs
through drift + rebuild steps, including steps whose guesses are stale (large
drift), wrong (arrays scrambled between calls) or unusable (N_ngb changed).
"""
import numpy as np
import pytest

from paper_2506_06269_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_06269_gb300 import build
    build.build()


def _pair(batch, precision):
    from paper_2506_06269_gb300 import sidm
    n = batch.n
    ctxs, arrays = [], []
    for warm in (True, False):
        ctx = sidm.Context(n_max=n, halo_max=batch.n_halos, ngb_max=128, precision=precision)
        ctx.warm_start(warm)
        dev = ctx.device
        pos = torch.tensor(batch.pos, dtype=torch.float64, device=dev).contiguous()
        vel = torch.tensor(batch.vel, dtype=ctx.vdtype, device=dev).contiguous()
        ids = torch.tensor(batch.ids.astype(np.int64), device=dev).to(torch.int32).contiguous()
        h = torch.zeros(n, dtype=ctx.vdtype, device=dev)
        ctxs.append(ctx)
        arrays.append([pos, vel, ids, h])
    return ctxs, arrays


def _step(ctxs, arrays, offsets, ks, dt):
    for ctx, (pos, vel, ids, h) in zip(ctxs, arrays):
        if dt:
            ctx.drift(ctx.f64([dt] * (len(offsets) - 1)), pos, vel)
        ctx.build_cells(offsets, pos, vel, ids)
        ctx.kernel_sizes(ks, h)
    torch.cuda.synchronize()
    (pw, vw, iw, hw), (pc, vc, ic, hc) = arrays
    assert torch.equal(iw, ic) and torch.equal(pw, pc)
    assert torch.equal(hw, hc), "warm-started kernel sizes differ from cold ones"
    assert all(c.status() == 0 for c in ctxs)
    return int(ctxs[0].diagnostics(reset=True)[7])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_warm_start_bit_identical_to_cold(precision):
    halo = ics.nfw(1 << 15, 11)
    b = ics.batch([halo])
    ctxs, arrays = _pair(b, precision)
    n = b.n
    redo = [_step(ctxs, arrays, b.offsets, [64], 0.0)]          # cold everywhere (no previous h)
    for _ in range(4):
        redo.append(_step(ctxs, arrays, b.offsets, [64], 2e-3))
    # the guesses were used and mostly held
    assert max(redo[1:]) < n // 4, redo
    # a large drift makes most guesses stale: the fallback path runs and stays exact
    redo.append(_step(ctxs, arrays, b.offsets, [64], 0.5))
    assert redo[-1] > 0, redo
    # scrambled arrays: every guess belongs to another particle
    g = torch.Generator(device="cpu").manual_seed(5)
    perm = torch.randperm(n, generator=g).to(arrays[0][0].device)
    for pos, vel, ids, h in arrays:
        pos.copy_(pos[:, perm])
        vel.copy_(vel[:, perm])
        ids.copy_(ids[perm])
    _step(ctxs, arrays, b.offsets, [64], 0.0)
    # N_ngb changes: the guess is not used, and the result is still exact
    _step(ctxs, arrays, b.offsets, [32], 1e-3)
    _step(ctxs, arrays, b.offsets, [32], 1e-3)
    for c in ctxs:
        c.close()


def test_warm_start_multi_halo_ragged():
    halos = [ics.hernquist(1000, 3), ics.uniform_box(33, 4), ics.nfw(5017, 5), ics.uniform_box(129, 6)]
    b = ics.batch(halos)
    ctxs, arrays = _pair(b, "mixed")
    for dt in (0.0, 1e-3, 1e-3, 0.05):
        _step(ctxs, arrays, b.offsets, [16, 32, 64, 128], dt)
    for c in ctxs:
        c.close()
