"""The cell build's particle order on the GPU against the oracle's canonical
geometry: within each halo, particles in the stable order of their 51-bit
Morton keys (equal keys keep their input order), which fixes the leaves of 32
and so the per-leaf FP32 frames of the canonical distance (Sect. 2; reading
C2').  Bit-exact.

Cases: ragged halo sizes around the radix sort's 4096-key tiles (1, 31, 4095,
4097, ...), a halo whose particles all coincide (one key: stability decides the
whole order), a halo on a coarse lattice (many runs of equal keys), batches of
40 halos (halo bits above the Morton bits: an eighth digit pass), and a
3.1-million-particle halo (hundreds of tiles in each pass's look-back).  The
caller's positions, velocities and ids come back permuted by the same order.
"""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_06269_gb300 import build
    build.build()


def _halo(kind, n, rng):
    if kind == "uniform":
        return rng.random((3, n)) * 3.0 - 1.0
    if kind == "clump":                         # centrally concentrated, like the NFW cusp
        r = rng.random(n) ** 3
        d = rng.standard_normal((3, n))
        return d / np.linalg.norm(d, axis=0) * r
    if kind == "coincident":
        return np.tile(np.array([[0.25], [-0.5], [0.125]]), (1, n))
    if kind == "lattice":                       # 8^3 sites: runs of equal keys
        return np.floor(rng.random((3, n)) * 8.0) / 8.0
    raise ValueError(kind)


def _check(halos, seed):
    from paper_2506_06269_gb300 import sidm
    rng = np.random.default_rng(seed)
    parts = [_halo(k, n, rng) for k, n in halos]
    sizes = [p.shape[1] for p in parts]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    pos = np.concatenate(parts, axis=1)
    vel = rng.standard_normal((3, n)).astype(np.float32)
    ids = np.concatenate([np.arange(s) for s in sizes]).astype(np.int32)
    ctx = sidm.Context(n_max=n, halo_max=len(halos), ngb_max=8, event_cap=1 << 12)
    dev = ctx.device
    tp = torch.tensor(pos, device=dev)
    tv = torch.tensor(vel, device=dev)
    ti = torch.tensor(ids, device=dev)
    ctx.build_cells(off, tp, tv, ti)
    perm = ctx.perm(n).cpu().numpy().astype(np.int64)
    status = ctx.status()
    out_pos, out_vel, out_id = tp.cpu().numpy(), tv.cpu().numpy(), ti.cpu().numpy()
    ctx.close()
    assert status == 0
    for h in range(len(halos)):
        a, b = int(off[h]), int(off[h + 1])
        order, _, _, _, _ = O.geometry(pos[:, a:b])
        assert np.array_equal(perm[a:b] - a, order.astype(np.int64)), (h, halos[h])
    assert np.array_equal(out_pos, pos[:, perm])
    assert np.array_equal(out_vel, vel[:, perm])
    assert np.array_equal(out_id, ids[perm])


def test_ragged_halos_around_the_tile_size():
    _check([("uniform", 1), ("uniform", 31), ("clump", 4095), ("uniform", 4096), ("clump", 4097),
            ("uniform", 9000), ("clump", 70001)], 1)


def test_equal_keys_keep_their_input_order():
    _check([("coincident", 5000), ("lattice", 20000), ("coincident", 1), ("lattice", 4097)], 2)


def test_forty_halos_sort_eight_digits():
    rng = np.random.default_rng(3)
    kinds = ["uniform", "clump", "lattice", "coincident"]
    _check([(kinds[i % 4], int(rng.integers(1, 6000))) for i in range(40)], 3)


def test_three_million_particles():
    _check([("clump", 3 * (1 << 20) + 12345)], 4)
