"""cdg2_vjp_noalloc: the VJP for callers that cannot allocate device memory.

Its scratch is a fixed device array inside the library instead of a cudaMalloc'd
workspace.  Checked through the C ABI against cdg2_vjp on two calls in a row
(the array is reused and must not carry state between calls), within the VJP
tests' tolerance; the second call must leave the device's free memory
unchanged (the first call on a device may load the module that holds the
array); a call without gtheta needs no scratch; and oversize meshes must be
refused with an error.  This
file sorts last so a run that stops at the first failure has run every other
test first; it also passes alone in a fresh process.
"""
import ctypes

import pytest
import torch

import cdg2_inputs as I
from helpers import rel_l2_per_species

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    L = G.load_library()
    vp = ctypes.c_void_p
    L.cdg2_vjp_noalloc.argtypes = [vp, ctypes.POINTER(G.Params), vp, vp, vp, vp, ctypes.c_int, ctypes.c_double, vp]
    L.cdg2_vjp_noalloc.restype = ctypes.c_int
    return L


def _noalloc(lib, G, mesh, p, U, lam, gU, gth, flags):
    pp = G.make_params(p)
    rc = lib.cdg2_vjp_noalloc(mesh.handle, ctypes.byref(pp), ctypes.c_void_p(U.data_ptr()),
                              ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(gU.data_ptr()),
                              ctypes.c_void_p(gth.data_ptr()) if gth is not None else None, flags, 0.0,
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, G.cdg2_last_error()


@pytest.mark.parametrize("dim,cells,k", [(2, (24, 10), 3), (3, (6, 4, 3), 2), (3, (64, 16, 16), 3)])
def test_noalloc_matches_cdg2_vjp_twice(lib, dim, cells, k):
    import paper_1403_1157_gb300 as G
    ext = (1.0, 0.2, 0.2)
    per = (1, 0, 0) if dim == 2 else (1, 0, 1)
    mesh = G.cdg2_mesh_create(dim, cells, ext, per, k)
    p = I.default_params()
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    U = torch.from_numpy(I.random_coefficients(mesh.n_elem, mesh.n_basis, 11)).cuda()
    for call in range(2):
        lam = (torch.from_numpy(I.random_coefficients(mesh.n_elem, mesh.n_basis, 20 + call)) - 1.0).cuda()
        ref_gU = torch.empty_like(U)
        ref_gth = torch.zeros(8, dtype=torch.float64, device="cuda")
        G.cdg2_vjp(mesh, p, U, lam, ref_gU, ref_gth, G.CDG2_MINV)
        gU = torch.full_like(U, float("nan"))
        gth = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        _noalloc(lib, G, mesh, p, U, lam, gU, gth, G.CDG2_MINV)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        assert rel_l2_per_species(gU, ref_gU.cpu().reshape(mesh.shape)) <= TOL
        assert float((gth - ref_gth).abs().max() / ref_gth.abs().max()) <= TOL


def test_noalloc_without_gtheta(lib):
    import paper_1403_1157_gb300 as G
    mesh = G.cdg2_mesh_create(2, (13, 5), (1.0, 0.2), (1, 0), 2)
    p = I.default_params()
    U = torch.from_numpy(I.random_coefficients(mesh.n_elem, mesh.n_basis, 12)).cuda()
    lam = (torch.from_numpy(I.random_coefficients(mesh.n_elem, mesh.n_basis, 13)) - 1.0).cuda()
    ref = torch.empty_like(U)
    G.cdg2_vjp(mesh, p, U, lam, ref, None, G.CDG2_MINV)
    for _ in range(2):
        gU = torch.full_like(U, float("nan"))
        _noalloc(lib, G, mesh, p, U, lam, gU, None, G.CDG2_MINV)
        torch.cuda.synchronize()
        assert rel_l2_per_species(gU, ref.cpu().reshape(mesh.shape)) <= TOL


def test_noalloc_refuses_meshes_beyond_its_scratch(lib):
    import paper_1403_1157_gb300 as G
    # 3D 128x32x32 Q2 needs 65536 VJP thread blocks, more than the 16384 the array holds
    mesh = G.cdg2_mesh_create(3, (128, 32, 32), (1.0, 0.2, 0.2), (1, 0, 1), 2)
    pp = G.make_params(I.default_params())
    dummy = ctypes.c_void_p(256)          # never dereferenced: the size check comes first
    rc = lib.cdg2_vjp_noalloc(mesh.handle, ctypes.byref(pp), dummy, ctypes.c_void_p(512), ctypes.c_void_p(1024),
                              ctypes.c_void_p(2048), G.CDG2_MINV, 0.0, None)
    assert rc == -1
    assert "16384" in G.cdg2_last_error()
