"""CDG2_ERR_DOMAIN: the pole of the tactic sensitivity chi(x, y, a, b) =
a x / (y + b) (Sec. 2) is reported by every operator entry point.

A host-made state puts one cell's c1 (or n1) below -chith, so that
c + chith < 0 at every quadrature point of that cell.  Each call through the
C ABI must return CDG2_ERR_DOMAIN, clear the status, and return CDG2_OK on
the next valid state; with CDG2_ASYNC the status waits for cdg2_mesh_status.
A strictly positive piecewise-constant state with chith = 0 must raise
nothing, also on meshes whose last thread block is ragged (the padding
elements hold U = 0, where chith = 0 is a pole).
"""
import ctypes

import pytest
import torch

import cdg2_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


def _valid(mesh, seed=5):
    return torch.from_numpy(I.random_coefficients(mesh.n_elem, mesh.n_basis, seed, 0.1)).reshape(-1).cuda()


def _poisoned(mesh, species=3, cell=None, seed=5):
    U = torch.from_numpy(I.random_coefficients(mesh.n_elem, mesh.n_basis, seed, 0.1))
    e = mesh.n_elem // 2 if cell is None else cell
    U[e, species, :] = 0.0
    U[e, species, 0] = -1.0              # the cell mean: c1 = -1 / sqrt(det) scale < -chith everywhere
    return U.reshape(-1).cuda()


def _code(fn):
    import paper_1403_1157_gb300 as G
    try:
        fn()
    except G.Cdg2Error as e:
        return e.code
    return 0


@pytest.mark.parametrize("dim,cells,k", [(2, (9, 7), 3), (3, (5, 3, 3), 2)])
@pytest.mark.parametrize("fp32", [False, True])
def test_cartesian_entry_points_report_the_pole(G, dim, cells, k, fp32):
    ext, per = (1.0, 0.2, 0.2), ((1, 0, 0) if dim == 2 else (1, 0, 1))
    mesh = G.cdg2_mesh_create(dim, cells, ext, per, k)
    p = I.default_params()
    dt = torch.float32 if fp32 else torch.float64
    f = G.CDG2_MINV | (G.CDG2_FP32 if fp32 else 0)
    bad, good = _poisoned(mesh).to(dt), _valid(mesh).to(dt)
    lam = _valid(mesh, 9).to(dt)
    out = torch.empty_like(good)
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    calls = {
        "apply": lambda U: G.cdg2_apply(mesh, p, U, out, f),
        "jvp": lambda U: G.cdg2_jvp(mesh, p, U, lam, out, f),
        "vjp": lambda U: G.cdg2_vjp(mesh, p, U, lam, out, gth, f),
    }
    for name, call in calls.items():
        assert _code(lambda: call(bad)) == G.CDG2_ERR_DOMAIN, name
        assert "pole" in G.cdg2_last_error()
        assert _code(lambda: call(good)) == 0, name          # the status was cleared
    # asynchronous: the call returns at once, the status waits for cdg2_mesh_status
    G.cdg2_apply(mesh, p, bad, out, f | G.CDG2_ASYNC)
    assert _code(lambda: G.cdg2_mesh_status(mesh)) == G.CDG2_ERR_DOMAIN
    assert _code(lambda: G.cdg2_mesh_status(mesh)) == 0
    G.cdg2_apply(mesh, p, bad, out, f | G.CDG2_ASYNC)
    assert _code(lambda: G.cdg2_apply(mesh, p, good, out, f)) == G.CDG2_ERR_DOMAIN   # sticky until reported
    assert _code(lambda: G.cdg2_apply(mesh, p, good, out, f)) == 0


def test_n1_pole_of_kappa22(G):
    mesh = G.cdg2_mesh_create(2, (8, 4), (1.0, 0.2), (1, 0), 2)
    p = I.default_params()
    out = torch.empty(mesh.n_dof, dtype=torch.float64, device="cuda")
    assert _code(lambda: G.cdg2_apply(mesh, p, _poisoned(mesh, species=0), out, G.CDG2_MINV)) == G.CDG2_ERR_DOMAIN


def test_noalloc_vjp_reports_the_pole(G):
    L = G.load_library()
    vp = ctypes.c_void_p
    L.cdg2_vjp_noalloc.argtypes = [vp, ctypes.POINTER(G.Params), vp, vp, vp, vp, ctypes.c_int, ctypes.c_double, vp]
    L.cdg2_vjp_noalloc.restype = ctypes.c_int
    mesh = G.cdg2_mesh_create(2, (9, 7), (1.0, 0.2), (1, 0), 3)
    pp = G.make_params(I.default_params())
    lam, gU = _valid(mesh, 9), torch.empty(mesh.n_dof, dtype=torch.float64, device="cuda")
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = vp(torch.cuda.current_stream().cuda_stream)
    for U, want in ((_poisoned(mesh), G.CDG2_ERR_DOMAIN), (_valid(mesh), 0)):
        rc = L.cdg2_vjp_noalloc(mesh.handle, ctypes.byref(pp), vp(U.data_ptr()), vp(lam.data_ptr()),
                                vp(gU.data_ptr()), vp(gth.data_ptr()), G.CDG2_MINV, 0.0, st)
        assert rc == want, G.cdg2_last_error()


@pytest.mark.parametrize("mixed", [False, True])
def test_step_reports_the_pole_and_keeps_u(G, mixed):
    mesh = G.cdg2_mesh_create(2, (8, 4), (1.0, 0.2), (1, 0), 2)
    p = I.default_params()
    U = _poisoned(mesh)
    U0 = U.clone()
    rc, _ = G.cdg2_step(mesh, p, U, 0.0, 1e-3, G.make_opts(scheme=G.CDG2_SDIRK2, mixed=mixed), raise_on_error=False)
    assert rc == G.CDG2_ERR_DOMAIN, G.cdg2_last_error()
    assert torch.equal(U, U0)
    rc, _ = G.cdg2_step(mesh, p, _valid(mesh), 0.0, 1e-3, G.make_opts(scheme=G.CDG2_SDIRK2, mixed=mixed),
                        raise_on_error=False)
    assert rc == 0, G.cdg2_last_error()


def test_simplicial_entry_points_report_the_pole(G):
    w = I.tri_workload(0)
    xy, tri = I.tri_mesh(w.nx, w.ny, w.extent[0], w.extent[1], w.jitter, w.seed)
    tm = G.cdg2_tri_mesh_create(xy, tri, w.k)
    wt = I.tet_workload(0)
    xyz, tet = I.tet_mesh(*wt.cells, *wt.extent, wt.jitter, wt.seed)
    qm = G.cdg2_tet_mesh_create(xyz, tet, wt.k)
    p = I.default_params()
    for mesh, apply, jvp, vjp, status, step in (
            (tm, G.cdg2_tri_apply, G.cdg2_tri_jvp, G.cdg2_tri_vjp, G.cdg2_tri_mesh_status, G.cdg2_tri_step),
            (qm, G.cdg2_tet_apply, G.cdg2_tet_jvp, G.cdg2_tet_vjp, G.cdg2_tet_mesh_status, G.cdg2_tet_step)):
        bad, good, lam = _poisoned(mesh), _valid(mesh), _valid(mesh, 9)
        out = torch.empty_like(good)
        for call in (lambda U: apply(mesh, p, U, out), lambda U: jvp(mesh, p, U, lam, out),
                     lambda U: vjp(mesh, p, U, lam, out)):
            assert _code(lambda: call(bad)) == G.CDG2_ERR_DOMAIN
            assert _code(lambda: call(good)) == 0
        apply(mesh, p, bad, out, G.CDG2_MINV | G.CDG2_ASYNC)
        assert _code(lambda: status(mesh)) == G.CDG2_ERR_DOMAIN
        assert _code(lambda: status(mesh)) == 0
        U = bad.clone()
        rc, _ = step(mesh, p, U, 1e-3, G.make_opts(scheme=G.CDG2_SDIRK2, precond=0), raise_on_error=False)
        assert rc == G.CDG2_ERR_DOMAIN and torch.equal(U, bad)


@pytest.mark.parametrize("dim,cells,k", [(2, (9, 7), 3), (2, (13, 5), 1), (3, (5, 3, 3), 2), (3, (3, 3, 3), 1)])
@pytest.mark.parametrize("fp32", [False, True])
def test_no_false_alarm_on_ragged_blocks(G, dim, cells, k, fp32):
    """chith = 0 puts the pole at zero concentration, which is what the padding of a
    ragged last thread block holds; a positive piecewise-constant state must pass."""
    ext, per = (1.0, 0.2, 0.2), ((1, 0, 0) if dim == 2 else (1, 0, 1))
    mesh = G.cdg2_mesh_create(dim, cells, ext, per, k)
    p = I.default_params()
    p["chith"] = (0.0, 0.0, 0.0, 0.0)
    U = torch.zeros(mesh.shape, dtype=torch.float64)
    U[:, :, 0] = 0.3 + torch.rand(mesh.n_elem, 6, generator=torch.Generator().manual_seed(3), dtype=torch.float64)
    dt = torch.float32 if fp32 else torch.float64
    f = G.CDG2_MINV | (G.CDG2_FP32 if fp32 else 0)
    U = U.reshape(-1).to(dt).cuda()
    lam = _valid(mesh, 9).to(dt)
    out = torch.empty_like(U)
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    G.cdg2_apply(mesh, p, U, out, f)
    G.cdg2_jvp(mesh, p, U, lam, out, f)
    G.cdg2_vjp(mesh, p, U, lam, out, gth, f)
    assert torch.isfinite(out).all() and torch.isfinite(gth).all()
