"""Host-side checks of the C ABI that need no GPU: every symbol that
include/*.h declares is exported by the built library, and argument
validation returns error codes instead of crashing."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G.load_library()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(cdg2_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cdg2_mesh_create", "cdg2_mesh_destroy", "cdg2_apply", "cdg2_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_mesh_create_validates(lib):
    import paper_1403_1157_gb300 as G
    with pytest.raises(G.Cdg2Error):
        G.cdg2_mesh_create(4, (2, 2, 2), (1, 1, 1), (1, 1, 1), 1)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_mesh_create(2, (2, 2), (1, 1), (1, 0), 4)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_mesh_create(2, (0, 2), (1, 1), (1, 0), 1)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_mesh_create(2, (2, 2), (1, 1), (1, 0), 2, q1=5)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_mesh_create(2, (2, 2), (1, 1), (1, 0), 2, flux=3)
    m = G.cdg2_mesh_create(3, (4, 3, 2), (1, 0.2, 0.2), (1, 0, 1), 2)
    assert (m.n_elem, m.n_basis, m.n_dof) == (24, 27, 24 * 27 * 6)


def test_apply_rejects_null_and_aliasing(lib):
    import paper_1403_1157_gb300 as G
    m = G.cdg2_mesh_create(2, (4, 2), (1, 0.2), (1, 0), 1)
    p = G.make_params(__import__("cdg2_inputs").default_params())
    rc = lib.cdg2_apply(m.handle, ctypes.byref(p), None, None, 1, 0.0, None)
    assert rc == -1 and "NULL" in G.cdg2_last_error()
    buf = ctypes.c_void_p(16)
    rc = lib.cdg2_apply(m.handle, ctypes.byref(p), buf, buf, 1, 0.0, None)
    assert rc == -1 and "overlap" in G.cdg2_last_error()
    rc = lib.cdg2_apply(m.handle, ctypes.byref(p), buf, ctypes.c_void_p(32), 1 << 10, 0.0, None)
    assert rc == -1 and "flag" in G.cdg2_last_error()
