"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point declared in include/sidm.h (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sidm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sidm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("sidm_create", "sidm_destroy", "sidm_build_cells", "sidm_kernel_sizes",
                 "sidm_scatter_step", "sidm_energy_momentum", "sidm_status", "sidm_last_error"):
        assert must in names


def test_library_builds_loads_and_exports_every_symbol():
    from paper_2506_06269_gb300 import build, sidm
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(sidm.EXPORTED) == _declared()


def test_binding_refuses_to_run_without_cuda():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2506_06269_gb300 import build, sidm
    build.build()
    with pytest.raises(RuntimeError):
        sidm.Context(n_max=16)
    # the C entry point itself reports the missing device instead of crashing
    cfg = sidm.SidmConfig(n_max=16, halo_max=1, ngb_max=8, event_cap=16)
    with pytest.raises(sidm.SidmError):
        sidm.sidm_create(cfg)


def test_create_rejects_bad_configuration():
    from paper_2506_06269_gb300 import build, sidm
    build.build()
    for kw in (dict(n_max=0), dict(halo_max=0), dict(halo_max=5000), dict(ngb_max=200), dict(event_cap=0),
               dict(precision=7), dict(knn_warps=17), dict(pair_warps=9), dict(pair_warps=-1),
               dict(knn_groups=3), dict(knn_chains=6), dict(knn_flush=33), dict(knn_slack=0.5),
               dict(knn_slack=2.5), dict(pair_per_round=5), dict(knn_batch=4),
               dict(knn_chains=8, knn_groups=2), dict(knn_chains=8)):
        base = dict(n_max=16, halo_max=1, ngb_max=8, event_cap=16, precision=0)
        base.update(kw)
        with pytest.raises(sidm.SidmError) as e:
            sidm.sidm_create(sidm.SidmConfig(**base))
        assert e.value.code == sidm.SIDM_EINVAL
