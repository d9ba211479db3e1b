"""ctypes binding of libfvgb (include/fvgb.h): the same entry points under the same
names, argument marshalling only. Device arrays are passed as torch CUDA tensors (or
raw integer addresses); every computation runs in the library's kernels.

Importing this module loads ``libfvgb.so`` from the package directory and raises if
it is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfvgb.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_2203_00925_gb300.build` "
        "(the library has no CPU fallback)")
lib = C.CDLL(LIB_PATH)

FVGB_OK, FVGB_EINVAL, FVGB_EMESH, FVGB_ENOMEM, FVGB_ECUDA = 0, 1, 2, 3, 4
FVGB_ENOCONV, FVGB_ENONFINITE, FVGB_ETIMEOUT, FVGB_EUNSUPPORTED = 5, 6, 7, 8
FVGB_FP64, FVGB_FP32, FVGB_MIXED = 0, 1, 2
FVGB_BC_WALL, FVGB_BC_DIRICHLET, FVGB_BC_NEUMANN = 0, 1, 2
STATUS_NAMES = {0: "FVGB_OK", 1: "FVGB_EINVAL", 2: "FVGB_EMESH", 3: "FVGB_ENOMEM",
                4: "FVGB_ECUDA", 5: "FVGB_ENOCONV", 6: "FVGB_ENONFINITE",
                7: "FVGB_ETIMEOUT", 8: "FVGB_EUNSUPPORTED"}

EXPORTED = [
    "fvgb_mesh_upload", "fvgb_mesh_upload_ensemble", "fvgb_mesh_parts", "fvgb_solve_parts",
    "fvgb_amg_levels",
    "fvgb_mesh_free", "fvgb_mesh_info", "fvgb_mesh_cell_perm",
    "fvgb_mesh_vert_perm",
    "fvgb_permute", "fvgb_gradient", "fvgb_gradient_vertex", "fvgb_vertex_values", "fvgb_fv_residual",
    "fvgb_fv_residual_noalloc",
    "fvgb_fv_step", "fvgb_poisson_apply", "fvgb_poisson_rhs", "fvgb_poisson_solve",
    "fvgb_streamer_step", "fvgb_streamer_reset", "fvgb_streamer_pair", "fvgb_set_graph_mode",
    "fvgb_mpnn_create", "fvgb_mpnn_hierarchy", "fvgb_mpnn_free", "fvgb_mpnn_param_count",
    "fvgb_mpnn_set_params",
    "fvgb_mpnn_get_params", "fvgb_mpnn_set_scales", "fvgb_mpnn_predict", "fvgb_mpnn_loss_grad",
    "fvgb_mpnn_train_step", "fvgb_autotune", "fvgb_set_launch_shape",
    "fvgb_integral", "fvgb_stats_enable", "fvgb_stats_get", "fvgb_sync", "fvgb_test_barrier",
    "fvgb_last_error",
]


class fvgb_bc(C.Structure):
    _fields_ = [("tag", C.c_int32), ("kind", C.c_int32), ("value", C.c_double)]


class fvgb_bcset(C.Structure):
    _fields_ = [("n_bc", C.c_int32), ("bc", C.POINTER(fvgb_bc))]


class fvgb_mesh_part(C.Structure):
    _fields_ = [("n_vert", C.c_int64), ("xyz", C.c_void_p), ("n_cell", C.c_int64),
                ("cell_vert", C.c_void_p), ("n_bface", C.c_int64), ("bface_vert", C.c_void_p),
                ("bface_tag", C.c_void_p), ("bcsets", C.POINTER(fvgb_bcset))]


class fvgb_tcoef(C.Structure):
    _fields_ = [("vel_dev", C.c_void_p), ("vel_const", C.c_double * 3), ("diff", C.c_double),
                ("src_dev", C.c_void_p), ("bcset", C.c_int32), ("recon", C.c_int32)]


class fvgb_solve_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("inner_rtol", C.c_double), ("maxit_inner", C.c_int32),
                ("maxit_outer", C.c_int32), ("prec", C.c_int32), ("inner", C.c_int32)]


class fvgb_solve_info(C.Structure):
    _fields_ = [("outer_its", C.c_int32), ("inner_its_total", C.c_int32),
                ("rel_res", C.c_double), ("bnorm", C.c_double)]

    def as_dict(self):
        return {"outer_its": self.outer_its, "inner_its_total": self.inner_its_total,
                "rel_res": self.rel_res, "bnorm": self.bnorm}


class fvgb_spot(C.Structure):
    _fields_ = [("centre", C.c_double * 3), ("amplitude", C.c_double), ("sigma", C.c_double),
                ("t_on", C.c_double), ("duration", C.c_double)]


class fvgb_streamer_params(C.Structure):
    _fields_ = [("mu", C.c_double), ("A", C.c_double), ("B", C.c_double), ("De", C.c_double),
                ("dt", C.c_double), ("bcset_ne", C.c_int32), ("bcset_phi", C.c_int32),
                ("solve", fvgb_solve_opts), ("warm", C.c_void_p), ("extrapolate", C.c_int32),
                ("recon", C.c_int32), ("stages", C.c_int32), ("t0", C.c_double),
                ("n_spot", C.c_int32), ("spots", C.POINTER(fvgb_spot))]


class fvgb_stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_int64), ("cg_launches", C.c_int64),
                ("cg_iterations", C.c_int64), ("cg_ms", C.c_double), ("solves", C.c_int64),
                ("outer_its", C.c_int64), ("learned_starts", C.c_int64), ("learned_kept", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp, _i32, _i64, _d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_sig = {
    "fvgb_mesh_upload": (C.c_int, [_i32, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _i32,
                                   C.POINTER(fvgb_bcset), _i32, _i32, _vp, C.POINTER(_vp)]),
    "fvgb_mesh_upload_ensemble": (C.c_int, [_i32, _i32, C.POINTER(fvgb_mesh_part), _i32, _i32, _i32,
                                            _vp, C.POINTER(_vp)]),
    "fvgb_mesh_parts": (C.c_int, [_vp, C.POINTER(_i32), _vp]),
    "fvgb_solve_parts": (C.c_int, [_vp, _vp, _vp, _vp]),
    "fvgb_amg_levels": (C.c_int32, [_vp, _i32, _i32, _vp, _i32]),
    "fvgb_mesh_free": (C.c_int, [_vp]),
    "fvgb_mesh_info": (C.c_int, [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64),
                                 C.POINTER(_i64)]),
    "fvgb_mesh_cell_perm": (C.c_int, [_vp, _vp]),
    "fvgb_mesh_vert_perm": (C.c_int, [_vp, _vp]),
    "fvgb_permute": (C.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _vp]),
    "fvgb_gradient": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "fvgb_gradient_vertex": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "fvgb_vertex_values": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "fvgb_fv_residual": (C.c_int, [_vp, C.POINTER(fvgb_tcoef), _vp, _vp, _vp]),
    "fvgb_fv_residual_noalloc": (C.c_int, [_vp, C.POINTER(fvgb_tcoef), _vp, _vp, _vp]),
    "fvgb_fv_step": (C.c_int, [_vp, C.POINTER(fvgb_tcoef), _vp, _d, _i32, _vp, _i32, _vp]),
    "fvgb_poisson_apply": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "fvgb_poisson_rhs": (C.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "fvgb_poisson_solve": (C.c_int, [_vp, _i32, _vp, _vp, C.POINTER(fvgb_solve_opts),
                                     C.POINTER(fvgb_solve_info), _vp]),
    "fvgb_streamer_step": (C.c_int, [_vp, C.POINTER(fvgb_streamer_params), _vp, _vp, _vp, _vp,
                                     _i32, C.POINTER(fvgb_solve_info), _vp]),
    "fvgb_integral": (C.c_int, [_vp, _vp, C.POINTER(_d), _vp]),
    "fvgb_set_graph_mode": (C.c_int, [_vp, _i32]),
    "fvgb_streamer_reset": (C.c_int, [_vp]),
    "fvgb_sync": (C.c_int, [_vp, _vp]),
    "fvgb_test_barrier": (C.c_int, [_vp, _i32, _d]),
    "fvgb_streamer_pair": (C.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "fvgb_mpnn_create": (C.c_int, [_vp, _i32, _i32, C.POINTER(_vp)]),
    "fvgb_mpnn_free": (C.c_int, [_vp]),
    "fvgb_mpnn_hierarchy": (C.c_int, [_i64, _vp, _i32, _vp, C.POINTER(_i32), _vp, _vp, _vp]),
    "fvgb_mpnn_param_count": (C.c_int64, []),
    "fvgb_mpnn_set_params": (C.c_int, [_vp, _vp]),
    "fvgb_mpnn_get_params": (C.c_int, [_vp, _vp]),
    "fvgb_mpnn_set_scales": (C.c_int, [_vp, _d, _d, _d, _d]),
    "fvgb_mpnn_predict": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "fvgb_mpnn_loss_grad": (C.c_int, [_vp, _vp, _vp, _vp, C.POINTER(_d), _vp, _vp]),
    "fvgb_mpnn_train_step": (C.c_int, [_vp, _vp, _vp, _vp, C.c_float, C.POINTER(_d), _vp]),
    "fvgb_autotune": (C.c_int, [_vp, _i32, _vp, _vp]),
    "fvgb_set_launch_shape": (C.c_int, [_vp, _i32, _i32, _i32]),
    "fvgb_stats_enable": (C.c_int, [_vp, _i32]),
    "fvgb_stats_get": (C.c_int, [_vp, C.POINTER(fvgb_stats), _i32]),
    "fvgb_last_error": (C.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class FvgbError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = lib.fvgb_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def _check(status, where):
    if status != FVGB_OK:
        raise FvgbError(status, where)
    return status


def ptr(x):
    """Device (or host) address of a tensor / numpy array / integer / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- entry points under their C names -----------------------------------------------------
def fvgb_mesh_upload(dim, xyz, cell_vert, bface_vert, bface_tag, bcsets, reorder=2,
                     prec=FVGB_FP64, stream=None):
    """Upload a mesh; ``bcsets`` is a list of {tag: (kind, value)} dicts. Host arrays are
    numpy (FP64 coordinates, int32 indices). Returns the opaque handle (an integer)."""
    import numpy as np
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    cell_vert = np.ascontiguousarray(cell_vert, dtype=np.int32)
    bface_vert = np.ascontiguousarray(bface_vert, dtype=np.int32)
    bface_tag = np.ascontiguousarray(bface_tag, dtype=np.int32)
    sets = (fvgb_bcset * len(bcsets))()
    keep = []
    for k, bc in enumerate(bcsets):
        arr = (fvgb_bc * len(bc))()
        for j, (tag, (kind, value)) in enumerate(sorted(bc.items())):
            arr[j] = fvgb_bc(int(tag), int(kind), float(value))
        keep.append(arr)
        sets[k] = fvgb_bcset(len(bc), C.cast(arr, C.POINTER(fvgb_bc)))
    out = _vp()
    _check(lib.fvgb_mesh_upload(dim, xyz.shape[0], ptr(xyz), cell_vert.shape[0], ptr(cell_vert),
                                bface_vert.shape[0], ptr(bface_vert), ptr(bface_tag), len(bcsets),
                                sets, reorder, prec, stream_handle(stream), C.byref(out)),
           "fvgb_mesh_upload")
    return out.value


def _bcset_array(bcsets, keep):
    sets = (fvgb_bcset * len(bcsets))()
    for k, bc in enumerate(bcsets):
        arr = (fvgb_bc * len(bc))()
        for j, (tag, (kind, value)) in enumerate(sorted(bc.items())):
            arr[j] = fvgb_bc(int(tag), int(kind), float(value))
        keep.append(arr)
        sets[k] = fvgb_bcset(len(bc), C.cast(arr, C.POINTER(fvgb_bc)))
    keep.append(sets)
    return sets


def fvgb_mesh_upload_ensemble(dim, meshes, bcsets_per_mesh, reorder=2, prec=FVGB_FP64, stream=None):
    """Upload several independent meshes as one; meshes are objects with xyz, cells,
    bface_vert, bface_tag (numpy), bcsets_per_mesh a list (per mesh) of lists of
    {tag: (kind, value)}. Returns the handle."""
    import numpy as np
    keep = []
    parts = (fvgb_mesh_part * len(meshes))()
    for p, (msh, bcs) in enumerate(zip(meshes, bcsets_per_mesh)):
        xyz = np.ascontiguousarray(msh.xyz, dtype=np.float64)
        cv = np.ascontiguousarray(msh.cells, dtype=np.int32)
        bv = np.ascontiguousarray(msh.bface_vert, dtype=np.int32)
        bt = np.ascontiguousarray(msh.bface_tag, dtype=np.int32)
        keep += [xyz, cv, bv, bt]
        sets = _bcset_array(bcs, keep)
        parts[p] = fvgb_mesh_part(xyz.shape[0], ptr(xyz), cv.shape[0], ptr(cv), bv.shape[0], ptr(bv),
                                  ptr(bt), C.cast(sets, C.POINTER(fvgb_bcset)))
    out = _vp()
    _check(lib.fvgb_mesh_upload_ensemble(dim, len(meshes), parts, len(bcsets_per_mesh[0]), reorder,
                                         prec, stream_handle(stream), C.byref(out)),
           "fvgb_mesh_upload_ensemble")
    return out.value


def fvgb_mesh_parts(m):
    import numpy as np
    n = _i32()
    _check(lib.fvgb_mesh_parts(m, C.byref(n), None), "fvgb_mesh_parts")
    begin = np.empty(n.value + 1, dtype=np.int64)
    _check(lib.fvgb_mesh_parts(m, C.byref(n), ptr(begin)), "fvgb_mesh_parts")
    return n.value, begin


def fvgb_solve_parts(m, n_part):
    import numpy as np
    rel = np.empty(n_part, dtype=np.float64)
    outer = np.empty(n_part, dtype=np.int32)
    inner = np.empty(n_part, dtype=np.int32)
    _check(lib.fvgb_solve_parts(m, ptr(rel), ptr(outer), ptr(inner)), "fvgb_solve_parts")
    return rel, outer, inner


def fvgb_mesh_free(m):
    return _check(lib.fvgb_mesh_free(m), "fvgb_mesh_free")


def fvgb_mesh_info(m):
    n = [_i64() for _ in range(4)]
    _check(lib.fvgb_mesh_info(m, *[C.byref(x) for x in n]), "fvgb_mesh_info")
    return {"n_cell": n[0].value, "n_face": n[1].value, "n_vert": n[2].value, "n_nbr": n[3].value}


def fvgb_mesh_cell_perm(m, n_cell):
    import numpy as np
    perm = np.empty(n_cell, dtype=np.int32)
    _check(lib.fvgb_mesh_cell_perm(m, ptr(perm)), "fvgb_mesh_cell_perm")
    return perm


def fvgb_mesh_vert_perm(m, n_vert):
    import numpy as np
    perm = np.empty(n_vert, dtype=np.int32)
    _check(lib.fvgb_mesh_vert_perm(m, ptr(perm)), "fvgb_mesh_vert_perm")
    return perm


def fvgb_permute(m, src, dst, n_comp, elem_bytes, to_internal, stream=None):
    return _check(lib.fvgb_permute(m, ptr(src), ptr(dst), n_comp, elem_bytes, int(to_internal),
                                   stream_handle(stream)), "fvgb_permute")


def fvgb_gradient(m, bcset, u, grad, stream=None):
    return _check(lib.fvgb_gradient(m, bcset, ptr(u), ptr(grad), stream_handle(stream)), "fvgb_gradient")


def fvgb_gradient_vertex(m, bcset, u, grad, stream=None):
    return _check(lib.fvgb_gradient_vertex(m, bcset, ptr(u), ptr(grad), stream_handle(stream)),
                  "fvgb_gradient_vertex")


def fvgb_vertex_values(m, bcset, u, uv, stream=None):
    return _check(lib.fvgb_vertex_values(m, bcset, ptr(u), ptr(uv), stream_handle(stream)),
                  "fvgb_vertex_values")


def tcoef(vel=None, vel_const=(0.0, 0.0, 0.0), diff=0.0, src=None, bcset=0, recon=0):
    """fvgb_tcoef for device arrays ``vel`` ([dim][n_cell]) and ``src`` ([n_cell]) or None.
    The struct holds raw pointers; it also keeps references to the arrays so that they
    stay allocated for as long as the struct is in use."""
    vc = (C.c_double * 3)(*[float(v) for v in list(vel_const) + [0.0] * (3 - len(vel_const))])
    tc = fvgb_tcoef(ptr(vel), vc, float(diff), ptr(src), int(bcset), int(recon))
    tc._keep = (vel, src)
    return tc


def fvgb_fv_residual(m, tc, u, res, stream=None):
    return _check(lib.fvgb_fv_residual(m, C.byref(tc), ptr(u), ptr(res), stream_handle(stream)),
                  "fvgb_fv_residual")


def fvgb_fv_residual_noalloc(m, tc, u, res, stream=None):
    """fvgb_fv_residual with its scratch in the library's fixed device array (no allocation)."""
    return _check(lib.fvgb_fv_residual_noalloc(m, C.byref(tc), ptr(u), ptr(res),
                                               stream_handle(stream)), "fvgb_fv_residual_noalloc")


def fvgb_fv_step(m, tc, u, dt, nsteps, stage_alpha=None, stream=None):
    arr = None
    n = 0
    if stage_alpha is not None:
        n = len(stage_alpha)
        arr = (C.c_double * n)(*stage_alpha)
    return _check(lib.fvgb_fv_step(m, C.byref(tc), ptr(u), float(dt), int(nsteps),
                                   C.cast(arr, _vp) if arr is not None else None, n,
                                   stream_handle(stream)), "fvgb_fv_step")


def fvgb_poisson_apply(m, bcset, x, y, stream=None):
    return _check(lib.fvgb_poisson_apply(m, bcset, ptr(x), ptr(y), stream_handle(stream)),
                  "fvgb_poisson_apply")


def fvgb_poisson_rhs(m, bcset, f, b, stream=None):
    return _check(lib.fvgb_poisson_rhs(m, bcset, ptr(f), ptr(b), stream_handle(stream)),
                  "fvgb_poisson_rhs")


def solve_opts(rtol=1e-8, inner_rtol=0.1, maxit_inner=20000, maxit_outer=200, prec=FVGB_FP64, inner=0):
    """inner = 0: conjugate gradients on A_T to inner_rtol; k > 0: k multigrid V-cycles."""
    return fvgb_solve_opts(float(rtol), float(inner_rtol), int(maxit_inner), int(maxit_outer), int(prec),
                           int(inner))


def fvgb_amg_levels(m, bcset, prec):
    import numpy as np
    sizes = np.zeros(32, dtype=np.int64)
    n = lib.fvgb_amg_levels(m, int(bcset), int(prec), ptr(sizes), 32)
    return sizes[:n].tolist()


def fvgb_poisson_solve(m, bcset, f, phi, opts, stream=None, check=True):
    info = fvgb_solve_info()
    st = lib.fvgb_poisson_solve(m, bcset, ptr(f), ptr(phi), C.byref(opts), C.byref(info),
                                stream_handle(stream))
    if check:
        _check(st, "fvgb_poisson_solve")
    return st, info


def spot(centre, amplitude=1e25, sigma=0.005, t_on=1.26e-8, duration=0.5e-9):
    c = list(centre) + [0.0] * (3 - len(centre))
    return fvgb_spot((C.c_double * 3)(*[float(v) for v in c]), float(amplitude), float(sigma),
                     float(t_on), float(duration))


def streamer_params(mu=0.0382, A=4332.0, B=2.0e5, De=0.1, dt=1e-9, bcset_ne=0, bcset_phi=1,
                    solve=None, warm=None, extrapolate=False, recon=0, stages=1, t0=0.0, spots=()):
    """fvgb_streamer_params; ``spots`` is a sequence of fvgb_spot (see ``spot``)."""
    arr = (fvgb_spot * max(len(spots), 1))(*spots)
    p = fvgb_streamer_params(mu, A, B, De, dt, bcset_ne, bcset_phi,
                             solve if solve is not None else solve_opts(), warm,
                             int(bool(extrapolate)), int(recon), int(stages), float(t0),
                             len(spots), arr if spots else None)
    p._keep = arr
    return p


def fvgb_streamer_reset(m):
    return _check(lib.fvgb_streamer_reset(m), "fvgb_streamer_reset")


def fvgb_sync(m, stream=None):
    """Synchronise and report the mesh's latched asynchronous status (FvgbError on error)."""
    return _check(lib.fvgb_sync(m, stream_handle(stream)), "fvgb_sync")


def fvgb_test_barrier(m, skip_block=-1, timeout_ms=0.0):
    """Test hook of the CG kernel's bounded grid barrier (see include/fvgb.h)."""
    return _check(lib.fvgb_test_barrier(m, int(skip_block), float(timeout_ms)), "fvgb_test_barrier")


def fvgb_streamer_pair(m, which, phi, dq, phi_prev, dphi, stream=None):
    """Training pair of the last streamer step from the mesh's warm-start history (which 0:
    start from the previous potential, 1: from the extrapolation) into dq, phi_prev, dphi."""
    return _check(lib.fvgb_streamer_pair(m, int(which), ptr(phi), ptr(dq), ptr(phi_prev), ptr(dphi),
                                         stream_handle(stream)), "fvgb_streamer_pair")


def fvgb_mpnn_create(m, bcset, multilevel=True):
    out = _vp()
    _check(lib.fvgb_mpnn_create(m, bcset, int(bool(multilevel)), C.byref(out)), "fvgb_mpnn_create")
    return out.value


def fvgb_mpnn_hierarchy(cen, part_begin=None):
    """Aggregate hierarchy of the network from cell centres cen [n][3] (host): a list of
    (level size, parent of every node below [level-local], neighbours [size][8])."""
    import numpy as np
    cen = np.asarray(cen, dtype=np.float64)
    n = cen.shape[0]
    soa = np.ascontiguousarray(cen.T)
    pb = np.ascontiguousarray([0, n] if part_begin is None else part_begin, dtype=np.int64)
    nl = _i32()
    sizes = np.zeros(16, dtype=np.int64)
    _check(lib.fvgb_mpnn_hierarchy(n, soa.ctypes.data, len(pb) - 1, pb.ctypes.data, C.byref(nl),
                                   sizes.ctypes.data, None, None), "fvgb_mpnn_hierarchy")
    L = nl.value
    below = np.concatenate([[n], sizes[:L - 1]]).astype(np.int64)
    parent = np.zeros(int(below.sum()), dtype=np.int32)
    nbr = np.zeros(int(sizes[:L].sum()) * 8, dtype=np.int32)
    _check(lib.fvgb_mpnn_hierarchy(n, soa.ctypes.data, len(pb) - 1, pb.ctypes.data, C.byref(nl),
                                   sizes.ctypes.data, parent.ctypes.data, nbr.ctypes.data), "fvgb_mpnn_hierarchy")
    out, po, no = [], 0, 0
    for k in range(L):
        nk = int(sizes[k])
        out.append((nk, parent[po:po + below[k]], nbr[8 * no:8 * (no + nk)].reshape(nk, 8)))
        po += int(below[k])
        no += nk
    return out


def fvgb_mpnn_free(net):
    return _check(lib.fvgb_mpnn_free(net), "fvgb_mpnn_free")


def fvgb_mpnn_param_count():
    return int(lib.fvgb_mpnn_param_count())


def fvgb_mpnn_set_params(net, theta):
    import numpy as np
    t = np.ascontiguousarray(theta, dtype=np.float32)
    return _check(lib.fvgb_mpnn_set_params(net, ptr(t)), "fvgb_mpnn_set_params")


def fvgb_mpnn_get_params(net):
    import numpy as np
    t = np.empty(fvgb_mpnn_param_count(), dtype=np.float32)
    _check(lib.fvgb_mpnn_get_params(net, ptr(t)), "fvgb_mpnn_get_params")
    return t


def fvgb_mpnn_set_scales(net, V, s0, s1, s2):
    return _check(lib.fvgb_mpnn_set_scales(net, V, s0, s1, s2), "fvgb_mpnn_set_scales")


def fvgb_mpnn_predict(net, dq, phi_prev, dphi, stream=None):
    return _check(lib.fvgb_mpnn_predict(net, ptr(dq), ptr(phi_prev), ptr(dphi), stream_handle(stream)),
                  "fvgb_mpnn_predict")


def fvgb_mpnn_loss_grad(net, dq, phi_prev, dphi, want_grad=True, stream=None):
    import numpy as np
    loss = _d()
    g = np.empty(fvgb_mpnn_param_count(), dtype=np.float32) if want_grad else None
    _check(lib.fvgb_mpnn_loss_grad(net, ptr(dq), ptr(phi_prev), ptr(dphi), C.byref(loss),
                                   ptr(g) if g is not None else None, stream_handle(stream)),
           "fvgb_mpnn_loss_grad")
    return loss.value, g


def fvgb_mpnn_train_step(net, dq, phi_prev, dphi, lr, want_loss=False, stream=None):
    loss = _d()
    _check(lib.fvgb_mpnn_train_step(net, ptr(dq), ptr(phi_prev), ptr(dphi), float(lr),
                                    C.byref(loss) if want_loss else None, stream_handle(stream)),
           "fvgb_mpnn_train_step")
    return loss.value if want_loss else None


def fvgb_streamer_step(m, params, ne, ni, phi, E, nsteps, stream=None):
    infos = (fvgb_solve_info * max(nsteps, 1))()
    _check(lib.fvgb_streamer_step(m, C.byref(params), ptr(ne), ptr(ni), ptr(phi), ptr(E),
                                  int(nsteps), infos, stream_handle(stream)), "fvgb_streamer_step")
    return [infos[i].as_dict() for i in range(nsteps)]


def fvgb_set_graph_mode(m, on=True):
    return _check(lib.fvgb_set_graph_mode(m, int(bool(on))), "fvgb_set_graph_mode")


def fvgb_autotune(m, force=False, stream=None):
    import numpy as np
    shapes = np.zeros(8, dtype=np.int32)
    _check(lib.fvgb_autotune(m, int(bool(force)), ptr(shapes), stream_handle(stream)), "fvgb_autotune")
    return shapes.reshape(4, 2)


def fvgb_set_launch_shape(m, kernel, threads, ipt=1):
    return _check(lib.fvgb_set_launch_shape(m, kernel, threads, ipt), "fvgb_set_launch_shape")


def fvgb_integral(m, u, stream=None):
    out = _d()
    _check(lib.fvgb_integral(m, ptr(u), C.byref(out), stream_handle(stream)), "fvgb_integral")
    return out.value


def fvgb_stats_enable(m, time_cg=True):
    return _check(lib.fvgb_stats_enable(m, int(bool(time_cg))), "fvgb_stats_enable")


def fvgb_stats_get(m, reset=False):
    st = fvgb_stats()
    _check(lib.fvgb_stats_get(m, C.byref(st), int(bool(reset))), "fvgb_stats_get")
    return st.as_dict()


def fvgb_last_error():
    return lib.fvgb_last_error().decode(errors="replace")
