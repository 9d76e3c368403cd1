"""CPU checks of the C ABI: the library loads, exports every declared entry point,
and rejects bad descriptors / schemes on the host before touching the GPU.  Also
checks that the oracle and the CUDA library share no code."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2404_08952_gb300 as dg
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(dg.LIB_PATH):
        from paper_2404_08952_gb300 import build
        build.build()
    return dg.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dolinc_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    decl = _declared()
    assert decl, "no declarations found"
    assert decl == set(dg.ABI_SYMBOLS)
    for name in decl:
        assert hasattr(lib, name), name


def _desc_from(m, **over):
    keep = {}
    for key, dt in (("nodes", np.float64), ("face_node_offsets", np.int64), ("face_nodes", np.int64),
                    ("face_owner", np.int64), ("face_neighbour", np.int64), ("face_periodic_shift", np.float64)):
        keep[key] = np.ascontiguousarray(over.get(key, m[key]), dtype=dt)
    d = dg._Desc()
    d.dim = over.get("dim", m["dim"])
    d.n_nodes = keep["nodes"].shape[0]
    d.nodes = dg._ptr(keep["nodes"])
    d.n_cells = over.get("n_cells", m["cell_face_offsets"].shape[0] - 1)
    d.n_faces = keep["face_owner"].shape[0]
    d.face_node_offsets = dg._ptr(keep["face_node_offsets"])
    d.face_nodes = dg._ptr(keep["face_nodes"])
    d.face_owner = dg._ptr(keep["face_owner"])
    d.face_neighbour = dg._ptr(keep["face_neighbour"])
    d.face_periodic_shift = dg._ptr(keep["face_periodic_shift"])
    d.renumber = 0
    return d, keep


def _create(lib, d):
    h = C.c_void_p()
    st = lib.dolinc_mesh_create(C.byref(d), C.byref(h))
    return st, h


def test_host_validation_rejects_bad_meshes(lib):
    m = synth.tri_mesh(4, 4, 0.1, 1)
    st, h = _create(lib, None if False else _desc_from(m, dim=4)[0])
    assert st == 1 or st == 2
    own = m["face_owner"].copy()
    own[3] = 10 ** 6
    d, keep = _desc_from(m, face_owner=own)
    st, h = _create(lib, d)
    assert st == 2 and b"owner" in lib.dolinc_last_error()
    nb = m["face_neighbour"].copy()
    nb[5] = -7
    d, keep = _desc_from(m, face_neighbour=nb)
    st, h = _create(lib, d)
    assert st == 2 and b"neighbour" in lib.dolinc_last_error()
    # reversed face orientation leaves cells unclosed
    fn = m["face_nodes"].reshape(-1, 2)[:, ::-1].ravel()
    d, keep = _desc_from(m, face_nodes=fn)
    st, h = _create(lib, d)
    assert st == 2 and b"closed" in lib.dolinc_last_error() or b"volume" in lib.dolinc_last_error()
    assert lib.dolinc_mesh_create(None, C.byref(h)) == 1
    # empty meshes: no cells, no faces
    for field in ("n_cells", "n_faces"):
        d, keep = _desc_from(m)
        setattr(d, field, 0)
        st, h = _create(lib, d)
        assert st == 2 and b"empty" in lib.dolinc_last_error()


def test_oracle_and_library_share_no_code():
    prod = os.path.join(ROOT, "paper_2404_08952_gb300")
    for dirpath, _, files in os.walk(prod):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".hpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src).lower().replace("the oracle", ""), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".py", ".h")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2404_08952_gb300" not in src and "csrc" not in src, f
