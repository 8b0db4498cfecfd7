"""ctypes binding of libdnnmg (include/dnnmg.h): argument marshalling only.

Each ``dnnmg_*`` function here calls the C entry point of the same name and
raises ``DnnmgError`` on a non-zero status.  Device buffers are passed as
torch CUDA tensors (their data pointers are borrowed for the call); every
step of the path runs in the library's CUDA kernels.  There is no fallback:
if the library is not built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FP64, FP32, BF16 = 0, 1, 2
PATCH_MAP, VALENCE, FINE_KIND, FINE_XYZ, EDGE_LENGTHS, GEOMETRY, COARSE_XYZ, COARSE_KIND = 0, 1, 2, 3, 4, 5, 6, 7
BUF_R, BUF_X, BUF_Y, BUF_D = 0, 1, 2, 3
N_IN, N_OUT = 228, 81


class DnnmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libdnnmg status {status}: {msg}")
        self.status = status


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int32), ("xyz", ctypes.POINTER(ctypes.c_double)),
                ("n_cells", ctypes.c_int32), ("cell_vertices", ctypes.POINTER(ctypes.c_int32)),
                ("vertex_bc", ctypes.POINTER(ctypes.c_int32))]


class Params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("dt", ctypes.c_double), ("theta", ctypes.c_double),
                ("precision", ctypes.c_int32), ("features", ctypes.c_int32),
                ("patch_levels", ctypes.c_int32), ("element", ctypes.c_int32)]


class NetDesc(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("widths", ctypes.POINTER(ctypes.c_int32)),
                ("skip", ctypes.c_int32)]


class Sizes(ctypes.Structure):
    _fields_ = [("n_coarse_vertices", ctypes.c_int64), ("n_patches", ctypes.c_int64),
                ("n_fine_nodes", ctypes.c_int64), ("n_coarse_edges", ctypes.c_int64),
                ("n_coarse_faces", ctypes.c_int64), ("n_in", ctypes.c_int32),
                ("n_in_padded", ctypes.c_int32), ("n_out", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("n_coarse_nodes", ctypes.c_int64), ("element", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_VP = ctypes.c_void_p
_SIGS = {
    "dnnmg_create": ([ctypes.POINTER(MeshDesc), ctypes.POINTER(Params), _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "dnnmg_destroy": ([_VP], None),
    "dnnmg_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "dnnmg_last_error": ([_VP], ctypes.c_char_p),
    "dnnmg_get_sizes": ([_VP, ctypes.POINTER(Sizes)], ctypes.c_int),
    "dnnmg_get_mesh_data": ([_VP, ctypes.c_int32, _VP, ctypes.c_size_t], ctypes.c_int),
    "dnnmg_hierarchy_build": ([ctypes.POINTER(MeshDesc), ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_VP)],
                              ctypes.c_int),
    "dnnmg_hierarchy_sizes": ([_VP, ctypes.POINTER(Sizes)], ctypes.c_int),
    "dnnmg_hierarchy_data": ([_VP, ctypes.c_int32, _VP, ctypes.c_size_t], ctypes.c_int),
    "dnnmg_hierarchy_destroy": ([_VP], None),
    "dnnmg_set_stream": ([_VP, _VP], ctypes.c_int),
    "dnnmg_set_network": ([_VP, ctypes.POINTER(NetDesc), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                           ctypes.POINTER(_VP)], ctypes.c_int),
    "dnnmg_prolongate": ([_VP, _VP, _VP], ctypes.c_int),
    "dnnmg_patch_targets": ([_VP, _VP, _VP, _VP, ctypes.c_int64], ctypes.c_int),
    "dnnmg_residual": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "dnnmg_local_restrict": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "dnnmg_network": ([_VP, _VP, _VP, ctypes.c_int64], ctypes.c_int),
    "dnnmg_network_wait_test": ([_VP, _VP, _VP, ctypes.c_int64], ctypes.c_int),
    "dnnmg_arm_wait_test": ([_VP], ctypes.c_int),
    "dnnmg_probe_fma": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)],
                        ctypes.c_int),
    "dnnmg_extend": ([_VP, _VP, _VP], ctypes.c_int),
    "dnnmg_rhs_restrict": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "dnnmg_patch_step": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "dnnmg_patch_step_host": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "dnnmg_get_buffer": ([_VP, ctypes.c_int32, ctypes.POINTER(_VP)], ctypes.c_int),
    "dnnmg_sync": ([_VP, ctypes.c_int64], ctypes.c_int),
    "dnnmg_launch_count": ([_VP], ctypes.c_int64),
    "dnnmg_residual_noalloc": ([ctypes.c_int64, ctypes.c_int64, _VP, _VP, _VP, _VP, _VP, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP], ctypes.c_int),
}

_lib = None


def load(path: str | None = None):
    """Load libdnnmg.so (built by paper_2307_14837_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libdnnmg is not built ({path} missing): run paper_2307_14837_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t):
    """Device (or host) address of a tensor / numpy array / int / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _check(ctx, status):
    if status != 0:
        lib = load()
        msg = lib.dnnmg_strerror(status).decode()
        if ctx:
            extra = lib.dnnmg_last_error(ctx).decode()
            if extra:
                msg += f" ({extra})"
        raise DnnmgError(status, msg)


# -- thin wrappers with the C names ------------------------------------------

def _mesh_desc(mesh):
    """A MeshDesc over contiguous copies of the mesh arrays (returned with
    them, so they outlive the call)."""
    xyz = np.ascontiguousarray(mesh["xyz"], dtype=np.float64)
    cells = np.ascontiguousarray(mesh["cells"], dtype=np.int32)
    bc = np.ascontiguousarray(mesh["vertex_bc"], dtype=np.int32)
    desc = MeshDesc(int(xyz.shape[0]), xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    int(cells.shape[0]), cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return desc, (xyz, cells, bc)


def _mesh_item(sz, item):
    """Shape and dtype of a mesh item for the sizes sz."""
    return {PATCH_MAP: ((sz["n_patches"], sz["n_out"] // 3), np.int32), VALENCE: ((sz["n_fine_nodes"],), np.int32),
            FINE_KIND: ((sz["n_fine_nodes"],), np.int32), FINE_XYZ: ((sz["n_fine_nodes"], 3), np.float64),
            EDGE_LENGTHS: ((sz["n_patches"], 12), np.float64),
            GEOMETRY: ((sz["n_patches"], sz["n_in"] - 8 * (sz["n_out"] // 3)), np.float64),
            COARSE_XYZ: ((sz["n_coarse_nodes"], 3), np.float64), COARSE_KIND: ((sz["n_coarse_nodes"],), np.int32)}[item]


class HostHierarchy:
    """The library's mesh hierarchy built on the host alone (no GPU):
    ``data(item)`` returns the items dnnmg_get_mesh_data gives for a context."""

    def __init__(self, mesh, features=12, patch_levels=1):
        desc, keep = _mesh_desc(mesh)
        handle = _VP()
        _check(None, load().dnnmg_hierarchy_build(ctypes.byref(desc), int(features), int(patch_levels),
                                                  ctypes.byref(handle)))
        del keep
        self.handle = handle.value
        s = Sizes()
        _check(None, load().dnnmg_hierarchy_sizes(self.handle, ctypes.byref(s)))
        self.sizes = {k: getattr(s, k) for k, _ in Sizes._fields_}

    def data(self, item):
        shape, dt = _mesh_item(self.sizes, item)
        out = np.empty(shape, dtype=dt)
        _check(None, load().dnnmg_hierarchy_data(self.handle, item, out.ctypes.data, out.nbytes))
        return out

    def mg_nodes(self, level=0, mg_levels=16, max_levels=32):
        """Nodes of every level of the multigrid hierarchy the solver would
        build on `level` (0 coarse, 1 fine) with at most mg_levels coarser
        levels (solve level first)."""
        n = ctypes.c_int32()
        nodes = np.zeros(max_levels, dtype=np.int64)
        _check(None, load().dnnmg_hierarchy_mg(self.handle, int(level), int(mg_levels), int(max_levels),
                                               ctypes.byref(n), nodes.ctypes.data))
        return [int(v) for v in nodes[:min(n.value, max_levels)]]

    def close(self):
        if self.handle:
            load().dnnmg_hierarchy_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dnnmg_create(mesh, nu, dt, theta, precision, stream=None, features=12, patch_levels=1, element=1):
    """mesh: dict with xyz [nv,3] float64, cells [nc,8] int32, vertex_bc [nv] int32.
    stream: a torch.cuda.Stream, an int handle, or None (default stream).
    features: geometry features per patch, 12 (edge lengths) or 24.
    patch_levels: J of the patches, 1 (27 nodes) or 2 (125 nodes).
    element: 1 (Q1/Q1) or 2 (Q2/Q2, 125-node patches; patch_levels 0 or 2)."""
    lib = load()
    desc, keep = _mesh_desc(mesh)
    prm = Params(float(nu), float(dt), float(theta), int(precision), int(features), int(patch_levels), int(element))
    handle = _VP()
    s = getattr(stream, "cuda_stream", stream)
    _check(None, lib.dnnmg_create(ctypes.byref(desc), ctypes.byref(prm), s, ctypes.byref(handle)))
    del keep
    return handle.value


def dnnmg_destroy(ctx):
    load().dnnmg_destroy(ctx)


def dnnmg_get_sizes(ctx) -> dict:
    s = Sizes()
    _check(ctx, load().dnnmg_get_sizes(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in Sizes._fields_}


def dnnmg_get_mesh_data(ctx, item):
    shape, dt = _mesh_item(dnnmg_get_sizes(ctx), item)
    out = np.empty(shape, dtype=dt)
    _check(ctx, load().dnnmg_get_mesh_data(ctx, item, out.ctypes.data, out.nbytes))
    return out


def dnnmg_set_stream(ctx, stream):
    _check(ctx, load().dnnmg_set_stream(ctx, getattr(stream, "cuda_stream", stream)))


def dnnmg_set_network(ctx, widths, Ws, scales=None, shifts=None, skip=True):
    L = len(Ws)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    keep = [np.ascontiguousarray(W, dtype=np.float64) for W in Ws]
    ks = [np.ascontiguousarray(s, dtype=np.float64) for s in scales] if scales is not None else None
    kt = [np.ascontiguousarray(t, dtype=np.float64) for t in shifts] if shifts is not None else None
    arr = lambda lst: (_VP * L)(*[a.ctypes.data for a in lst]) if lst is not None else None
    desc = NetDesc(L, w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1 if skip else 0)
    _check(ctx, load().dnnmg_set_network(ctx, ctypes.byref(desc), arr(keep), arr(ks), arr(kt)))


def dnnmg_prolongate(ctx, x_coarse, x_fine):
    _check(ctx, load().dnnmg_prolongate(ctx, _ptr(x_coarse), _ptr(x_fine)))


def dnnmg_patch_targets(ctx, x_coarse, v_fine, T, ldt=None):
    """T[P][3 iota + c] = (v_fine - P x_coarse)[node(P, iota)][c] in fp32."""
    _check(ctx, load().dnnmg_patch_targets(ctx, _ptr(x_coarse), _ptr(v_fine), _ptr(T),
                                           int(ldt if ldt is not None else T.shape[1])))


def dnnmg_residual(ctx, x_coarse, F, r):
    _check(ctx, load().dnnmg_residual(ctx, _ptr(x_coarse), _ptr(F), _ptr(r)))


def dnnmg_local_restrict(ctx, x_coarse, r, X):
    _check(ctx, load().dnnmg_local_restrict(ctx, _ptr(x_coarse), _ptr(r), _ptr(X)))


def dnnmg_network(ctx, X, Y, n_rows):
    _check(ctx, load().dnnmg_network(ctx, _ptr(X), _ptr(Y), int(n_rows)))


def dnnmg_network_wait_test(ctx, X, Y, n_rows):
    _check(ctx, load().dnnmg_network_wait_test(ctx, _ptr(X), _ptr(Y), int(n_rows)))


def dnnmg_probe_fma(precision, iters=4096, blocks_per_sm=8) -> float:
    """Measured FMA throughput (TFLOP/s) of the SIMT pipe in FP32 or FP64."""
    t = ctypes.c_double()
    _check(None, load().dnnmg_probe_fma(int(precision), int(iters), int(blocks_per_sm), ctypes.byref(t)))
    return t.value


def dnnmg_arm_wait_test(ctx):
    _check(ctx, load().dnnmg_arm_wait_test(ctx))


def dnnmg_extend(ctx, Y, d):
    _check(ctx, load().dnnmg_extend(ctx, _ptr(Y), _ptr(d)))


def dnnmg_rhs_restrict(ctx, x_coarse, d, b_fine, b_coarse):
    _check(ctx, load().dnnmg_rhs_restrict(ctx, _ptr(x_coarse), _ptr(d), _ptr(b_fine), _ptr(b_coarse)))


def dnnmg_patch_step(ctx, x_coarse, F, b_fine, b_coarse):
    _check(ctx, load().dnnmg_patch_step(ctx, _ptr(x_coarse), _ptr(F), _ptr(b_fine), _ptr(b_coarse)))


def dnnmg_patch_step_host(ctx, x_coarse, F, b_fine, b_coarse):
    _check(ctx, load().dnnmg_patch_step_host(ctx, _ptr(x_coarse), _ptr(F), _ptr(b_fine), _ptr(b_coarse)))


def dnnmg_get_buffer(ctx, which) -> int:
    p = _VP()
    _check(ctx, load().dnnmg_get_buffer(ctx, int(which), ctypes.byref(p)))
    return p.value


def dnnmg_sync(ctx, timeout_us=-1):
    _check(ctx, load().dnnmg_sync(ctx, int(timeout_us)))


def dnnmg_launch_count(ctx) -> int:
    return int(load().dnnmg_launch_count(ctx))


NOALLOC_MAX_PATCHES = 16384


def dnnmg_residual_noalloc(n_patches, n_fine_nodes, cells, xyz, node_ptr, node_idx, fine_dirichlet,
                           nu, dt, theta, x_coarse, F, r, stream=None):
    """The residual without allocation (FP32): every array from the caller."""
    s = getattr(stream, "cuda_stream", stream)
    _check(None, load().dnnmg_residual_noalloc(int(n_patches), int(n_fine_nodes), _ptr(cells), _ptr(xyz),
                                               _ptr(node_ptr), _ptr(node_idx), _ptr(fine_dirichlet), float(nu),
                                               float(dt), float(theta), _ptr(x_coarse), _ptr(F), _ptr(r), s))


# -- Newton solver and time loop -------------------------------------------------

LEVEL_COARSE, LEVEL_FINE = 0, 1


class SolverParams(ctypes.Structure):
    _fields_ = [("alpha0", ctypes.c_double), ("delta0", ctypes.c_double), ("newton_atol", ctypes.c_double),
                ("newton_rtol", ctypes.c_double), ("newton_max", ctypes.c_int32), ("gmres_restart", ctypes.c_int32),
                ("gmres_max", ctypes.c_int32), ("mg_levels", ctypes.c_int32), ("gmres_rtol", ctypes.c_double),
                ("rho_max", ctypes.c_double), ("mg_pre", ctypes.c_int32), ("mg_post", ctypes.c_int32),
                ("mg_omega", ctypes.c_double), ("mg_smoother", ctypes.c_int32), ("mg_bf16", ctypes.c_int32)]


class SolveStats(ctypes.Structure):
    _fields_ = [("newton_iterations", ctypes.c_int32), ("gmres_iterations", ctypes.c_int32),
                ("jacobian_assemblies", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("residual0", ctypes.c_double), ("residual", ctypes.c_double)]


_SIGS.update({
    "dnnmg_solver_defaults": ([ctypes.POINTER(SolverParams)], None),
    "dnnmg_level_info": ([_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)],
                         ctypes.c_int),
    "dnnmg_level_operator": ([_VP, ctypes.c_int32, ctypes.POINTER(SolverParams), _VP, _VP], ctypes.c_int),
    "dnnmg_level_rhs": ([_VP, ctypes.c_int32, _VP, _VP], ctypes.c_int),
    "dnnmg_level_jacobian": ([_VP, ctypes.c_int32, ctypes.POINTER(SolverParams), _VP, _VP, ctypes.c_size_t],
                             ctypes.c_int),
    "dnnmg_solve": ([_VP, ctypes.c_int32, ctypes.POINTER(SolverParams), _VP, _VP, ctypes.POINTER(SolveStats)],
                    ctypes.c_int),
    "dnnmg_time_step": ([_VP, ctypes.c_int32, ctypes.POINTER(SolverParams), _VP, _VP, _VP,
                         ctypes.POINTER(SolveStats)], ctypes.c_int),
    "dnnmg_plain_step": ([_VP, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(SolverParams), _VP,
                          ctypes.POINTER(SolveStats)], ctypes.c_int),
    "dnnmg_level_mg": ([_VP, ctypes.c_int32, ctypes.POINTER(SolverParams), ctypes.c_int32,
                        ctypes.POINTER(ctypes.c_int32), _VP], ctypes.c_int),
    "dnnmg_hierarchy_mg": ([_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                            _VP], ctypes.c_int),
})
ENOCONV = -4


def dnnmg_solver_defaults(**overrides) -> SolverParams:
    p = SolverParams()
    load().dnnmg_solver_defaults(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _stats(s):
    return {k: getattr(s, k) for k, _ in SolveStats._fields_}


def dnnmg_level_mg(ctx, level, prm=None, max_levels=32):
    """Nodes of every level of the level's multigrid hierarchy (solve level first)."""
    n = ctypes.c_int32()
    nodes = np.zeros(max_levels, dtype=np.int64)
    _check(ctx, load().dnnmg_level_mg(ctx, int(level), ctypes.byref(prm) if prm else None, int(max_levels),
                                      ctypes.byref(n), nodes.ctypes.data))
    return [int(v) for v in nodes[:min(n.value, max_levels)]]


def dnnmg_level_info(ctx, level):
    n, g = ctypes.c_int64(), ctypes.c_int32()
    _check(ctx, load().dnnmg_level_info(ctx, int(level), ctypes.byref(n), ctypes.byref(g)))
    return n.value, bool(g.value)


def dnnmg_level_operator(ctx, level, x, Ax, prm=None):
    _check(ctx, load().dnnmg_level_operator(ctx, int(level), ctypes.byref(prm) if prm else None, _ptr(x), _ptr(Ax)))


def dnnmg_level_rhs(ctx, level, x_old, b):
    _check(ctx, load().dnnmg_level_rhs(ctx, int(level), _ptr(x_old), _ptr(b)))


def dnnmg_level_jacobian(ctx, level, x, prm=None):
    n, _ = dnnmg_level_info(ctx, level)
    out = np.empty((4 * n, 4 * n))
    _check(ctx, load().dnnmg_level_jacobian(ctx, int(level), ctypes.byref(prm) if prm else None, _ptr(x),
                                            out.ctypes.data, out.nbytes))
    return out


def _solve_status(ctx, status):
    if status != ENOCONV:
        _check(ctx, status)


def dnnmg_solve(ctx, level, b, x, prm=None):
    st = SolveStats()
    _solve_status(ctx, load().dnnmg_solve(ctx, int(level), ctypes.byref(prm) if prm else None, _ptr(b), _ptr(x),
                                          ctypes.byref(st)))
    return _stats(st)


def dnnmg_time_step(ctx, n_steps, x_coarse, b_coarse, F, prm=None):
    st = SolveStats()
    _check(ctx, load().dnnmg_time_step(ctx, int(n_steps), ctypes.byref(prm) if prm else None, _ptr(x_coarse),
                                       _ptr(b_coarse), _ptr(F), ctypes.byref(st)))
    return _stats(st)


def dnnmg_plain_step(ctx, level, n_steps, x, prm=None):
    st = SolveStats()
    _check(ctx, load().dnnmg_plain_step(ctx, int(level), int(n_steps), ctypes.byref(prm) if prm else None, _ptr(x),
                                        ctypes.byref(st)))
    return _stats(st)


_SIGS.update({
    "dnnmg_restrict": ([_VP, _VP, _VP], ctypes.c_int),
    "dnnmg_trainer_create": ([ctypes.POINTER(NetDesc), ctypes.c_int32, ctypes.c_int64, _VP, ctypes.POINTER(_VP)],
                             ctypes.c_int),
    "dnnmg_trainer_destroy": ([_VP], None),
    "dnnmg_trainer_forward": ([_VP, _VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP, ctypes.c_int64], ctypes.c_int),
    "dnnmg_trainer_backward": ([_VP, _VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP)], ctypes.c_int),
    "dnnmg_mse_loss": ([ctypes.c_int64, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "dnnmg_column_stats": ([_VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP],
                           ctypes.c_int),
    "dnnmg_standardize": ([_VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP, _VP],
                          ctypes.c_int),
    "dnnmg_gather_rows": ([_VP, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_int64, _VP, _VP], ctypes.c_int),
    "dnnmg_add_noise": ([_VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                         ctypes.c_double, ctypes.c_uint64, _VP], ctypes.c_int),
    "dnnmg_adamw": ([ctypes.c_int64, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                     ctypes.c_double, ctypes.c_double, ctypes.c_int32, _VP], ctypes.c_int),
})


_SIGS.update({
    "dnnmg_step_begin": ([_VP, ctypes.POINTER(SolverParams), ctypes.c_int32, _VP, _VP, _VP, _VP,
                          ctypes.POINTER(SolveStats)], ctypes.c_int),
    "dnnmg_step_end": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "dnnmg_net_create": ([ctypes.POINTER(NetDesc), ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                          ctypes.c_int32, ctypes.c_int64, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
})


def dnnmg_step_begin(ctx, x_coarse, b_coarse, F, X, solve=True, prm=None):
    st = SolveStats()
    _solve_status(ctx, load().dnnmg_step_begin(ctx, ctypes.byref(prm) if prm else None, 1 if solve else 0,
                                               _ptr(x_coarse), _ptr(b_coarse), _ptr(F), _ptr(X), ctypes.byref(st)))
    return _stats(st)


def dnnmg_step_end(ctx, Y, F, b_coarse):
    _check(ctx, load().dnnmg_step_end(ctx, _ptr(Y), _ptr(F), _ptr(b_coarse)))


def dnnmg_net_create(widths, Ws, scales, shifts, precision, max_rows, stream=None, skip=True):
    L = len(Ws)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    keep = [np.ascontiguousarray(W, dtype=np.float64) for W in Ws]
    ks = [np.ascontiguousarray(s, dtype=np.float64) for s in scales] if scales is not None else None
    kt = [np.ascontiguousarray(t, dtype=np.float64) for t in shifts] if shifts is not None else None
    arr = lambda lst: (_VP * L)(*[a.ctypes.data for a in lst]) if lst is not None else None
    desc = NetDesc(L, w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1 if skip else 0)
    h = _VP()
    _check(None, load().dnnmg_net_create(ctypes.byref(desc), arr(keep), arr(ks), arr(kt), int(precision),
                                         int(max_rows), getattr(stream, "cuda_stream", stream), ctypes.byref(h)))
    return h.value


def dnnmg_restrict(ctx, b_fine, b_coarse):
    _check(ctx, load().dnnmg_restrict(ctx, _ptr(b_fine), _ptr(b_coarse)))


def _ptr_array(ts):
    return (_VP * len(ts))(*[_ptr(t) for t in ts]) if ts else None


def dnnmg_trainer_create(widths, precision, max_batch, stream=None, skip=True):
    w = np.ascontiguousarray(widths, dtype=np.int32)
    desc = NetDesc(len(widths) - 1, w.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 1 if skip else 0)
    h = _VP()
    s = getattr(stream, "cuda_stream", stream)
    _check(None, load().dnnmg_trainer_create(ctypes.byref(desc), int(precision), int(max_batch), s, ctypes.byref(h)))
    return h.value


def dnnmg_trainer_destroy(tr):
    load().dnnmg_trainer_destroy(tr)


def dnnmg_trainer_forward(tr, X, Ws, bs, Y, batch):
    _check(None, load().dnnmg_trainer_forward(tr, _ptr(X), _ptr_array(Ws), _ptr_array(bs), _ptr(Y), int(batch)))


def dnnmg_trainer_backward(tr, dY, dWs, dbs):
    _check(None, load().dnnmg_trainer_backward(tr, _ptr(dY), _ptr_array(dWs), _ptr_array(dbs)))


def dnnmg_mse_loss(batch, Y, T, loss, dY=None, stream=None):
    _check(None, load().dnnmg_mse_loss(int(batch), _ptr(Y), _ptr(T), _ptr(loss), _ptr(dY),
                                       getattr(stream, "cuda_stream", stream)))


def _dtype_code(t):
    import torch
    return {torch.float64: FP64, torch.float32: FP32, torch.bfloat16: BF16}[t.dtype]


def dnnmg_column_stats(A, mean, sd, cols=None, stream=None):
    """Per-column mean and sample deviation (double device tensors [cols]) of
    the rows of the 2-D tensor A (row stride A.stride(0))."""
    cols = int(cols if cols is not None else A.shape[1])
    _check(None, load().dnnmg_column_stats(_ptr(A), _dtype_code(A), int(A.shape[0]), cols, int(A.stride(0)),
                                           _ptr(mean), _ptr(sd), getattr(stream, "cuda_stream", stream)))


def dnnmg_standardize(A, shift, scale, B, cols=None, stream=None):
    """B[:, :cols] = (A[:, :cols] - shift) / scale (double device tensors)."""
    cols = int(cols if cols is not None else A.shape[1])
    assert B.dtype == A.dtype and B.stride(0) == A.stride(0) and B.shape[0] == A.shape[0]
    _check(None, load().dnnmg_standardize(_ptr(A), _dtype_code(A), int(A.shape[0]), cols, int(A.stride(0)),
                                          _ptr(shift), _ptr(scale), _ptr(B), getattr(stream, "cuda_stream", stream)))


def dnnmg_gather_rows(src, idx, dst, stream=None):
    """dst[i] = src[idx[i]] for contiguous 2-D tensors, idx int64 on the device."""
    assert src.is_contiguous() and dst.is_contiguous() and src.dtype == dst.dtype
    row_bytes = src.stride(0) * src.element_size()
    assert dst.stride(0) * dst.element_size() == row_bytes and dst.shape[0] >= idx.shape[0]
    _check(None, load().dnnmg_gather_rows(_ptr(src), int(src.shape[0]), int(row_bytes), _ptr(idx), int(idx.shape[0]),
                                          _ptr(dst), getattr(stream, "cuda_stream", stream)))


def dnnmg_add_noise(A, c0, c1, sigma, seed, stream=None):
    """A[:, c0:c1] += sigma * (seeded standard normal), in place."""
    _check(None, load().dnnmg_add_noise(_ptr(A), _dtype_code(A), int(A.shape[0]), int(c0), int(c1),
                                        int(A.stride(0)), float(sigma), int(seed) & ((1 << 64) - 1),
                                        getattr(stream, "cuda_stream", stream)))


def dnnmg_adamw(w, g, m, v, lr, beta1, beta2, eps, weight_decay, step, stream=None):
    _check(None, load().dnnmg_adamw(int(w.numel()), _ptr(w), _ptr(g), _ptr(m), _ptr(v), float(lr), float(beta1),
                                    float(beta2), float(eps), float(weight_decay), int(step),
                                    getattr(stream, "cuda_stream", stream)))
