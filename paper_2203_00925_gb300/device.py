"""Convenience layer over the C ABI for torch CUDA tensors.

``DeviceMesh`` uploads a mesh once and converts fields between the caller's cell order
and the library's internal (Morton) order. All arithmetic runs in libfvgb's kernels;
the host side only moves and reorders data.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi

BC_KIND = {"wall": capi.FVGB_BC_WALL, "dirichlet": capi.FVGB_BC_DIRICHLET,
           "neumann": capi.FVGB_BC_NEUMANN}
PREC = {"fp64": capi.FVGB_FP64, "fp32": capi.FVGB_FP32, "mixed": capi.FVGB_MIXED}


def bcset(spec):
    """{tag: (kind name or code, value)} -> {tag: (code, value)}."""
    return {int(t): (BC_KIND.get(k, k), float(v)) for t, (k, v) in spec.items()}


class DeviceMesh:
    """One mesh, or with ``ensemble=True`` a list of meshes (``bcsets`` then a list per
    mesh) packed into one index space; the caller's order of an ensemble is the meshes'
    cells one after the other."""

    def __init__(self, mesh, bcsets, prec="fp64", reorder=2, device="cuda", stream=None,
                 ensemble=False):
        if not torch.cuda.is_available():
            raise RuntimeError("DeviceMesh needs a CUDA device (no CPU fallback)")
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        torch.cuda.set_device(self.device)
        self.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        self.real = torch.float64 if self.prec == capi.FVGB_FP64 else torch.float32
        if ensemble:
            self.dim = mesh[0].dim
            self.handle = capi.fvgb_mesh_upload_ensemble(
                self.dim, mesh, [[bcset(b) for b in bl] for bl in bcsets], reorder, self.prec, stream)
        else:
            self.dim = mesh.dim
            self.handle = capi.fvgb_mesh_upload(mesh.dim, mesh.xyz, mesh.cells, mesh.bface_vert,
                                                mesh.bface_tag, [bcset(b) for b in bcsets],
                                                reorder, self.prec, stream)
        self.n_part, self.part_begin = capi.fvgb_mesh_parts(self.handle)
        info = capi.fvgb_mesh_info(self.handle)
        self.n_cell, self.n_face, self.n_vert, self.n_nbr = (
            info["n_cell"], info["n_face"], info["n_vert"], info["n_nbr"])
        self.perm = capi.fvgb_mesh_cell_perm(self.handle, self.n_cell)
        self.vperm = capi.fvgb_mesh_vert_perm(self.handle, self.n_vert)

    # ---- order conversion (host marshalling) ------------------------------------------------
    def to_device(self, x_user, dtype=None):
        """Host array in the caller's cell order ([n] or [k, n]) -> internal-order tensor."""
        x = np.asarray(x_user)
        xi = x[..., self.perm]
        return torch.as_tensor(np.ascontiguousarray(xi), dtype=dtype or self.real,
                               device=self.device)

    def to_host(self, t_int):
        """Internal-order tensor ([n] or [k, n]) -> numpy FP64 array in the caller's order."""
        x = t_int.detach().to("cpu", torch.float64).numpy()
        out = np.empty_like(x)
        out[..., self.perm] = x
        return out

    def vert_to_host(self, t_int):
        x = t_int.detach().to("cpu", torch.float64).numpy()
        out = np.empty_like(x)
        out[..., self.vperm] = x
        return out

    def empty(self, *shape, dtype=None):
        return torch.empty(*shape, dtype=dtype or self.real, device=self.device)

    def free(self):
        if getattr(self, "handle", None):
            capi.fvgb_mesh_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
