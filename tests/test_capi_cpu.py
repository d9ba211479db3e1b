"""The C-ABI library loads, exports every entry point its header declares, and rejects
malformed meshes on the host before touching the GPU (CPU only)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from synth.meshgen import jittered_cube, jittered_square

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2203_00925_gb300 import build
    build.build()
    from paper_2203_00925_gb300 import capi as c
    return c


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fvgb_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(capi):
    names = declared_functions()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(capi.lib, n), n
    assert set(capi.EXPORTED) == names


def _bcs3():
    return [{t: (capi_kind("neumann"), 0.0) for t in range(1, 7)}]


def capi_kind(k):
    return {"wall": 0, "dirichlet": 1, "neumann": 2}[k]


def _upload(capi, m, cells=None, bface=None, btag=None, bcs=None, dim=None):
    out = C.c_void_p()
    cells = np.ascontiguousarray(m.cells if cells is None else cells, dtype=np.int32)
    bface = np.ascontiguousarray(m.bface_vert if bface is None else bface, dtype=np.int32)
    btag = np.ascontiguousarray(m.bface_tag if btag is None else btag, dtype=np.int32)
    bcs = _bcs3() if bcs is None else bcs
    sets = (capi.fvgb_bcset * len(bcs))()
    keep = []
    for k, bc in enumerate(bcs):
        arr = (capi.fvgb_bc * len(bc))()
        for j, (t, (kind, v)) in enumerate(sorted(bc.items())):
            arr[j] = capi.fvgb_bc(t, kind, v)
        keep.append(arr)
        sets[k] = capi.fvgb_bcset(len(bc), C.cast(arr, C.POINTER(capi.fvgb_bc)))
    st = capi.lib.fvgb_mesh_upload(m.dim if dim is None else dim, m.xyz.shape[0], m.xyz.ctypes.data,
                                   cells.shape[0], cells.ctypes.data, bface.shape[0],
                                   bface.ctypes.data, btag.ctypes.data, len(bcs), sets, 2, 0, None,
                                   C.byref(out))
    return st, capi.fvgb_last_error()


def test_malformed_meshes_are_rejected_on_the_host(capi):
    m = jittered_cube(2, seed=1)
    st, msg = _upload(capi, m, dim=4)
    assert st == capi.FVGB_EINVAL
    bad = m.cells.copy(); bad[0, [1, 2]] = bad[0, [2, 1]]          # inverted tetrahedron
    st, msg = _upload(capi, m, cells=bad)
    assert st == capi.FVGB_EMESH and "orientation" in msg
    bad = m.cells.copy(); bad[5, 3] = m.xyz.shape[0] + 7             # vertex out of range
    st, msg = _upload(capi, m, cells=bad)
    assert st == capi.FVGB_EMESH and "range" in msg
    st, msg = _upload(capi, m, bface=m.bface_vert[1:], btag=m.bface_tag[1:])   # missing face
    assert st == capi.FVGB_EMESH and "boundary" in msg
    bf = m.bface_vert.copy(); bf[0] = [0, 1, 2]                      # not a boundary face
    st, msg = _upload(capi, m, bface=bf)
    assert st == capi.FVGB_EMESH
    st, msg = _upload(capi, m, bcs=[{t: (2, 0.0) for t in range(1, 6)}])   # tag 6 has no BC
    assert st == capi.FVGB_EMESH and "tag 6" in msg
    dup = np.concatenate([m.cells, m.cells[:1]])                     # face shared by 3 cells
    st, msg = _upload(capi, m, cells=dup)
    assert st == capi.FVGB_EMESH
    m2 = jittered_square(3, 1, 2)
    st, msg = _upload(capi, m2, bcs=[{t: (9, 0.0) for t in range(1, 5)}])   # bad kind
    assert st in (capi.FVGB_EINVAL, capi.FVGB_EMESH)


def _single_tet():
    from synth.meshgen import Mesh
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    cells = np.array([[0, 1, 2, 3]], dtype=np.int32)
    bface = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]], dtype=np.int32)
    return Mesh(3, xyz, cells, bface, np.array([1, 2, 3, 4], dtype=np.int32), 1.0)


def test_singular_gradient_stencil_is_rejected_on_the_host(capi):
    """A lone tetrahedron has no node neighbours: with Neumann faces only, its
    least-squares gradient (Algorithm "grad") has no points and the upload refuses it;
    with Dirichlet faces the ghost points make it well defined (checked on the GPU)."""
    st, msg = _upload(capi, _single_tet(), bcs=[{t: (capi_kind("neumann"), 0.0) for t in range(1, 5)}])
    assert st == capi.FVGB_EMESH and "singular" in msg


def test_null_handle_calls_fail_cleanly(capi):
    assert capi.lib.fvgb_gradient(None, 0, None, None, None) == capi.FVGB_EINVAL
    assert capi.lib.fvgb_poisson_solve(None, 0, None, None, None, None, None) == capi.FVGB_EINVAL
    assert capi.lib.fvgb_mesh_free(None) == capi.FVGB_OK
