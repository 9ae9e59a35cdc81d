"""The allocation-free entry point, sidm_energy_momentum_static.

It serves callers inside a host application that owns all device memory (its
own allocator or a fixed budget) and forbids libraries to call cudaMalloc:
the call needs no context and keeps its scratch in a fixed device array.  This
file is collected last on purpose.  The test calls the entry point through the
C ABI twice in a row, on two different halo sets, and checks each result
against the context-based sidm_energy_momentum within the tolerance used for
the energy sums elsewhere (1e-14 relative; the two share arithmetic and order,
so in practice the bits agree)."""
import numpy as np
import pytest

from paper_2506_06269_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _reference(b, precision):
    from paper_2506_06269_gb300 import sidm
    ctx = sidm.Context(n_max=b.n, halo_max=b.n_halos, precision=precision)
    vin = b.vel.astype(np.float32) if precision == "mixed" else b.vel
    vel = torch.tensor(vin, dtype=ctx.vdtype, device="cuda").contiguous()
    pos = torch.tensor(b.pos, device="cuda")
    ids = torch.tensor(b.ids.astype(np.int64), device="cuda").to(torch.int32)
    ctx.build_cells(b.offsets, pos, vel, ids)            # permutes vel within halos
    mass = ctx.f64(b.mass)
    out = torch.zeros((b.n_halos, 4), dtype=torch.float64, device="cuda")
    ctx.energy_momentum(mass, vel, out)
    torch.cuda.synchronize()
    ctx.close()
    return vel, mass, out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_static_entry_matches_context_entry_on_two_calls(precision):
    from paper_2506_06269_gb300 import build, sidm
    build.build()
    batches = [ics.batch([ics.nfw(40000, 31), ics.hernquist(777, 32), ics.nfw(20001, 33)]),
               ics.batch([ics.hernquist(70000, 34), ics.uniform_box(5, 35)])]
    for b in batches:
        vel, mass, ref = _reference(b, precision)
        out = torch.full((b.n_halos, 4), float("nan"), dtype=torch.float64, device="cuda")
        comp = torch.zeros_like(out)
        sidm.sidm_energy_momentum_static(b.offsets, precision, mass, vel, out, comp)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), out.cpu().numpy()
        scale = np.maximum(np.abs(r), 1e-300)
        assert np.all(np.abs(g - r) <= 1e-14 * scale), (precision, g, r)


def test_static_entry_rejects_out_of_range_sizes():
    from paper_2506_06269_gb300 import build, sidm
    build.build()
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(sidm.SidmError) as e:                      # too many halos
        sidm.sidm_energy_momentum_static(np.arange(66) * 10, "mixed", d, d, d)
    assert e.value.code == sidm.SIDM_EINVAL
    with pytest.raises(sidm.SidmError) as e:                      # more chunks than the scratch holds
        sidm.sidm_energy_momentum_static([0, 16384 * 4096 + 1], "mixed", d, d, d)
    assert e.value.code == sidm.SIDM_ECAPACITY
