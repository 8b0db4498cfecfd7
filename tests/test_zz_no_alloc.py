"""dnnmg_residual_noalloc: the residual for callers that may not allocate
device memory (an application that owns every device allocation, or code
that must not call cudaMalloc after set-up).  It must give the context-based
dnnmg_residual's result, call after call, from arrays the caller supplies.

This file is named to be collected last, so that a run that stops at the
first failure has run every other test before it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from parity_util import case_data  # noqa: E402
from paper_2307_14837_gb300 import build, capi  # noqa: E402
from paper_2307_14837_gb300.path import PatchPath  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    capi.load()


def _caller_arrays(p, mesh):
    """What a caller hands over: mesh arrays and the node -> (patch, iota)
    lists in patch order, built here from the context's patch map."""
    pm = p.mesh_data(capi.PATCH_MAP).ravel()
    order = np.argsort(pm, kind="stable").astype(np.int32)       # entries P*27+iota by node, then patch
    counts = np.bincount(pm, minlength=p.n_fine)
    ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    kind = p.mesh_data(capi.FINE_KIND)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dt)
    return dict(cells=dev(mesh["cells"], torch.int32), xyz=dev(mesh["xyz"], torch.float32),
                node_ptr=dev(ptr, torch.int32), node_idx=dev(order, torch.int32),
                fine_dir=dev(((kind == 1) | (kind == 2)).astype(np.uint8), torch.uint8))


def test_noalloc_residual_matches_context_residual_twice():
    d = case_data("cavity8")
    c = d["case"]
    p = PatchPath(d["mesh"], c["nu"], c["dt"], c["theta"], "fp32")
    xc, F = p.to_device(d["xc"]), p.to_device(d["F"])
    ref = p.residual(xc, F)
    a = _caller_arrays(p, d["mesh"])
    scale = float(np.abs(d["F"]).max() + np.abs(d["A"]).max())
    for call in range(2):
        r = torch.full((p.n_fine, 4), float("nan"), device="cuda")
        capi.dnnmg_residual_noalloc(p.n_patches, p.n_fine, a["cells"], a["xyz"], a["node_ptr"], a["node_idx"],
                                    a["fine_dir"], c["nu"], c["dt"], c["theta"], xc, F, r,
                                    torch.cuda.current_stream())
        torch.cuda.synchronize()
        err = (r - ref).abs().max().item() / scale
        assert err <= 1e-5, (call, err)
    p.close()


def test_noalloc_rejects_meshes_beyond_its_scratch():
    dummy = torch.zeros(16, device="cuda")
    with pytest.raises(capi.DnnmgError) as e:
        capi.dnnmg_residual_noalloc(capi.NOALLOC_MAX_PATCHES + 1, 10, dummy, dummy, dummy, dummy, dummy,
                                    0.01, 0.01, 1.0, dummy, dummy, dummy, None)
    assert e.value.status == -1
