"""cdg2_tri_step / cdg2_tet_step (SDIRK + Newton + GMRES with the simplicial
JVP, FP64, with no preconditioner or element-block Jacobi) against the
oracle's step on the same meshes.  Bar: 1e-10 relative after the steps when
both solve their Newton systems to ~1e-13 (the oracle with dense Jacobians
and LU); the block preconditioner needs fewer GMRES iterations; invalid
options and a non-finite state return status codes."""
import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from oracle import cdg2_tet_oracle as TT
from oracle import cdg2_tri_oracle as T
from helpers import lift_into_domain, psi_max_tet, psi_max_tri

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


def _params():
    p = I.default_params()
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    return p


def _tight(G, scheme, precond=0):
    return G.make_opts(scheme=scheme, max_newton=30, gmres_restart=40, max_gmres=800, newton_rtol=1e-14,
                       newton_atol=1e-15, gmres_rtol=1e-10, precond=precond)


_ORACLE_RUNS = {}


def _rel(a, b):
    return float((a.cpu() - b).norm() / b.norm())


@pytest.mark.parametrize("nx,ny,k", [(3, 2, 1), (4, 2, 2)])
@pytest.mark.parametrize("scheme,name", [(2, "sdirk2"), (3, "sdirk3")])
@pytest.mark.parametrize("precond", [0, 2])
def test_tri_step_matches_oracle(G, nx, ny, k, scheme, name, precond):
    xy, tri = I.tri_mesh(nx, ny, 1.0, 0.2, 0.2, 700 + k)
    om = T.TriMesh(xy, tri, k)
    p = _params()
    cen, amp = I.gaussian_draws(2, (1.0, 0.2), 4, 70 + k)
    U0 = lift_into_domain(T.project(om, lambda x: O.gaussian_field(om, x, cen, amp, 0.15, 0.05)), psi_max_tri(k))
    dt, nsteps = 1e-3, 2
    key = (nx, ny, k, name)
    if key not in _ORACLE_RUNS:
        ref = U0.clone()
        for _ in range(nsteps):
            ref = T.step(om, ref, p, dt, name)
        _ORACLE_RUNS[key] = ref
    ref = _ORACLE_RUNS[key]
    gm = G.cdg2_tri_mesh_create(xy, tri, k)
    U = U0.reshape(-1).clone().cuda()
    for _ in range(nsteps):
        rc, st = G.cdg2_tri_step(gm, p, U, dt, _tight(G, scheme, precond))
        assert rc == 0 and st["newton_iters"] >= 1 and st["gmres_iters"] >= 1
    assert _rel(U, ref.reshape(-1)) <= 1e-10


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("precond", [0, 2])
def test_tet_step_matches_oracle(G, k, precond):
    xyz, tet = I.tet_mesh(2, 1, 1, 1.0, 0.2, 0.2, 0.15, 710 + k)
    om = TT.TetMesh(xyz, tet, k)
    p = _params()
    cen, amp = I.gaussian_draws(3, (1.0, 0.2, 0.2), 4, 71 + k)
    U0 = lift_into_domain(TT.project(om, lambda x: O.gaussian_field(om, x, cen, amp, 0.15, 0.05)), psi_max_tet(k))
    if ("tet", k) not in _ORACLE_RUNS:
        _ORACLE_RUNS[("tet", k)] = TT.step(om, U0, p, 2e-3, "sdirk2")
    ref = _ORACLE_RUNS[("tet", k)]
    gm = G.cdg2_tet_mesh_create(xyz, tet, k)
    U = U0.reshape(-1).clone().cuda()
    # (a relative 1e-14 of the first Newton residual sits below the rounding floor of the
    # tetrahedral residual at k = 2; 1e-12 of it is still ~1e-13 of the state)
    opts = G.make_opts(scheme=2, max_newton=30, gmres_restart=40, max_gmres=800, newton_rtol=1e-12,
                       newton_atol=1e-13, gmres_rtol=1e-10, precond=precond)
    rc, _ = G.cdg2_tet_step(gm, p, U, 2e-3, opts)
    assert rc == 0 and _rel(U, ref.reshape(-1)) <= 1e-10


def test_simplex_step_status_codes(G):
    xy, tri = I.tri_mesh(3, 2, 1.0, 0.2, 0.2, 720)
    gm = G.cdg2_tri_mesh_create(xy, tri, 1)
    p = _params()
    U = torch.zeros(gm.n_elem, 6, gm.n_basis, dtype=torch.float64, device="cuda")
    U[:, :, 0] = 0.1                    # constant fields, inside the model's domain
    U = U.reshape(-1)
    for bad in (G.make_opts(mixed=True, precond=0), G.make_opts(precond=1), G.make_opts(precond=3),
                G.make_opts(precond=0, flags=G.CDG2_FORCING)):
        rc, _ = G.cdg2_tri_step(gm, p, U, 1e-3, bad, raise_on_error=False)
        assert rc == -1
    V = U.clone()
    V[5] = float("nan")
    W = V.clone()
    rc, _ = G.cdg2_tri_step(gm, p, V, 1e-3, _tight(G, 2), raise_on_error=False)
    assert rc == -4 and "non-finite" in G.cdg2_last_error()
    assert torch.equal(V.isnan(), W.isnan()) and torch.equal(V.nan_to_num(), W.nan_to_num())   # U unchanged
    xyz, tet = I.tet_mesh(2, 1, 1, 1.0, 0.2, 0.2, 0.15, 721)
    tm = G.cdg2_tet_mesh_create(xyz, tet, 1)
    Ut = torch.full((tm.n_dof,), 0.1, dtype=torch.float64, device="cuda")
    rc, _ = G.cdg2_tet_step(tm, p, Ut, 1e-3, G.make_opts(precond=1), raise_on_error=False)
    assert rc == -1


@pytest.mark.parametrize("kind", ["tri", "tet"])
def test_block_jacobi_cuts_gmres_iterations(G, kind):
    """Same step, same tolerances: the element-block Jacobi (whose blocks are
    probed with the diffusion JVP and cached across steps) gives the same state
    and needs fewer Krylov iterations on a stiff step (dt large against h^2)."""
    p = _params()
    if kind == "tri":
        xy, tri = I.tri_mesh(24, 6, 1.0, 0.2, 0.2, 730)
        gm, step = G.cdg2_tri_mesh_create(xy, tri, 2), G.cdg2_tri_step
        cen, psi0 = xy[tri].mean(axis=1), 2.0 ** 0.5
    else:
        xyz, tet = I.tet_mesh(6, 2, 2, 1.0, 0.2, 0.2, 0.15, 731)
        gm, step = G.cdg2_tet_mesh_create(xyz, tet, 2), G.cdg2_tet_step
        cen, psi0 = xyz[tet].mean(axis=1), 6.0 ** 0.5
    # a positive piecewise-constant state (the mean coefficient carries the centroid value)
    U0 = torch.zeros(gm.n_elem, 6, gm.n_basis, dtype=torch.float64)
    for s in range(6):
        U0[:, s, 0] = torch.from_numpy(0.5 + 0.3 * np.sin(2 * np.pi * cen[:, 0] + s) * np.cos(np.pi * cen[:, 1] / 0.2)) / psi0
    U0 = U0.reshape(-1).cuda()
    res, its = {}, {}
    for pc in (0, 2):
        U = U0.clone()
        for _ in range(2):         # the second step reuses the cached blocks
            opts = G.make_opts(scheme=3, max_newton=20, gmres_restart=30, max_gmres=3000, newton_rtol=1e-12,
                               newton_atol=1e-13, gmres_rtol=1e-8, precond=pc)
            rc, st = step(gm, p, U, 1e-2, opts)
            assert rc == 0
            its[pc] = its.get(pc, 0) + st["gmres_iters"]
        res[pc] = U
    assert float((res[2] - res[0]).norm() / res[0].norm()) <= 1e-10
    assert its[2] < its[0], its
