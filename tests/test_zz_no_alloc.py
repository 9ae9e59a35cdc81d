"""The allocation-free entry point, sidm_energy_momentum_static.

It serves callers inside a host application that owns all device memory (its
own caching allocator or a fixed budget) and forbids libraries to call
cudaMalloc: the call needs no context and keeps its scratch in a fixed device
array.  This file is collected last on purpose, so that a run stopping at the
first failure has already run every other test.

Each case calls the entry point through the C ABI twice in a row and checks
both results against the context-based sidm_energy_momentum on the same
velocities.  The two share their arithmetic and its order, so the sums and
the compensation terms must agree bit for bit.  Cases: three uneven halos,
an empty halo between two others, 64 halos (some empty, some exactly one
chunk of 16384 particles), and one halo of exactly SIDM_STATIC_MAX_CHUNKS
chunks -- the largest size the scratch holds."""
import numpy as np
import pytest

from paper_2506_06269_gb300 import ics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CHUNK = 16384


def _empty():
    return ics.Halo(pos=np.zeros((3, 0)), vel=np.zeros((3, 0)), ids=np.zeros(0, np.uint32), mass=1.0, name="empty")


def _context_result(offsets, mass, pos, vel, precision):
    """sidm_energy_momentum of the context on the velocities after its cell
    build (which permutes them within each halo); returns them with the result."""
    from paper_2506_06269_gb300 import sidm
    n = int(offsets[-1])
    ctx = sidm.Context(n_max=max(n, 1), halo_max=len(offsets) - 1, precision=precision)
    ids = torch.cat([torch.arange(int(offsets[h + 1] - offsets[h]), dtype=torch.int32, device="cuda")
                     for h in range(len(offsets) - 1)])
    ctx.build_cells(offsets, pos, vel, ids)
    m = ctx.f64(mass)
    out = torch.zeros((len(offsets) - 1, 4), dtype=torch.float64, device="cuda")
    comp = torch.zeros_like(out)
    ctx.energy_momentum(m, vel, out, comp)
    torch.cuda.synchronize()
    ctx.close()
    return m, out.cpu().numpy(), comp.cpu().numpy()


def _two_calls_match(offsets, mass, pos, vel, precision):
    from paper_2506_06269_gb300 import sidm
    m, ref, ref_c = _context_result(offsets, mass, pos, vel, precision)
    for _ in range(2):
        out = torch.full((len(offsets) - 1, 4), float("nan"), dtype=torch.float64, device="cuda")
        comp = torch.full_like(out, float("nan"))
        sidm.sidm_energy_momentum_static(offsets, precision, m, vel, out, comp)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref), precision
        assert np.array_equal(comp.cpu().numpy(), ref_c), precision


def _batch_tensors(b, precision):
    vin = b.vel.astype(np.float32) if precision == "mixed" else b.vel
    vel = torch.tensor(vin, dtype=torch.float32 if precision == "mixed" else torch.float64, device="cuda")
    return torch.tensor(b.pos, device="cuda"), vel.contiguous()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_static_entry_matches_context_entry_on_two_calls(precision):
    from paper_2506_06269_gb300 import build
    build.build()
    rng = np.random.default_rng(5)
    sizes64 = rng.integers(1, 40000, 64)
    sizes64[[3, 17, 40]] = 0                  # empty halos inside the batch
    sizes64[[5, 60]] = CHUNK                  # exactly one chunk
    sizes64[9] = 2 * CHUNK + 1                # a ragged chunk tail
    batches = [
        ics.batch([ics.nfw(40000, 31), ics.hernquist(777, 32), ics.nfw(20001, 33)]),
        ics.batch([ics.hernquist(70000, 34), _empty(), ics.uniform_box(5, 35)]),
        ics.batch([ics.uniform_box(int(s), 100 + h) if s > 0 else _empty() for h, s in enumerate(sizes64)]),
    ]
    for b in batches:
        pos, vel = _batch_tensors(b, precision)
        _two_calls_match(b.offsets, b.mass, pos, vel, precision)


def test_static_entry_at_exact_capacity():
    """One halo of exactly SIDM_STATIC_MAX_CHUNKS chunks (67,108,864 particles)."""
    from paper_2506_06269_gb300 import build, sidm
    build.build()
    n = sidm.SIDM_STATIC_MAX_CHUNKS * CHUNK
    g = torch.Generator(device="cuda")
    g.manual_seed(8)
    pos = torch.rand((3, n), generator=g, dtype=torch.float64, device="cuda")
    vel = torch.randn((3, n), generator=g, dtype=torch.float32, device="cuda")
    _two_calls_match(np.array([0, n], np.int64), [1.0 / n], pos, vel, "mixed")


def test_static_entry_rejects_out_of_range_sizes():
    from paper_2506_06269_gb300 import build, sidm
    build.build()
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(sidm.SidmError) as e:                      # too many halos
        sidm.sidm_energy_momentum_static(np.arange(66) * 10, "mixed", d, d, d)
    assert e.value.code == sidm.SIDM_EINVAL and "n_halos" in str(e.value)
    with pytest.raises(sidm.SidmError) as e:                      # more chunks than the scratch holds
        sidm.sidm_energy_momentum_static([0, CHUNK * sidm.SIDM_STATIC_MAX_CHUNKS + 1], "mixed", d, d, d)
    assert e.value.code == sidm.SIDM_ECAPACITY and "SIDM_STATIC_MAX_CHUNKS" in str(e.value)
