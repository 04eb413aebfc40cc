"""cdg2_tri_step / cdg2_tet_step (SDIRK + Newton + GMRES with the simplicial
JVP, FP64) against the oracle's step on the same meshes.  Bar: 1e-10
relative after the steps when both solve their Newton systems to ~1e-13
(the oracle with dense Jacobians and LU); invalid options and a non-finite
state return status codes."""
import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from oracle import cdg2_tet_oracle as TT
from oracle import cdg2_tri_oracle as T

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


def _tight(G, scheme):
    return G.make_opts(scheme=scheme, max_newton=30, gmres_restart=40, max_gmres=800, newton_rtol=1e-14,
                       newton_atol=1e-15, gmres_rtol=1e-10, precond=0)


def _rel(a, b):
    return float((a.cpu() - b).norm() / b.norm())


@pytest.mark.parametrize("nx,ny,k", [(3, 2, 1), (4, 2, 2)])
@pytest.mark.parametrize("scheme,name", [(2, "sdirk2"), (3, "sdirk3")])
def test_tri_step_matches_oracle(G, nx, ny, k, scheme, name):
    xy, tri = I.tri_mesh(nx, ny, 1.0, 0.2, 0.2, 700 + k)
    om = T.TriMesh(xy, tri, k)
    p = _params()
    cen, amp = I.gaussian_draws(2, (1.0, 0.2), 4, 70 + k)
    U0 = T.project(om, lambda x: O.gaussian_field(om, x, cen, amp, 0.15, 0.05))
    dt, nsteps = 1e-3, 2
    ref = U0.clone()
    for _ in range(nsteps):
        ref = T.step(om, ref, p, dt, name)
    gm = G.cdg2_tri_mesh_create(xy, tri, k)
    U = U0.reshape(-1).clone().cuda()
    for _ in range(nsteps):
        rc, st = G.cdg2_tri_step(gm, p, U, dt, _tight(G, scheme))
        assert rc == 0 and st["newton_iters"] >= 1 and st["gmres_iters"] >= 1
    assert _rel(U, ref.reshape(-1)) <= 1e-10


@pytest.mark.parametrize("k", [1, 2])
def test_tet_step_matches_oracle(G, k):
    xyz, tet = I.tet_mesh(2, 1, 1, 1.0, 0.2, 0.2, 0.15, 710 + k)
    om = TT.TetMesh(xyz, tet, k)
    p = _params()
    cen, amp = I.gaussian_draws(3, (1.0, 0.2, 0.2), 4, 71 + k)
    U0 = TT.project(om, lambda x: O.gaussian_field(om, x, cen, amp, 0.15, 0.05))
    ref = TT.step(om, U0, p, 2e-3, "sdirk2")
    gm = G.cdg2_tet_mesh_create(xyz, tet, k)
    U = U0.reshape(-1).clone().cuda()
    # (a relative 1e-14 of the first Newton residual sits below the rounding floor of the
    # tetrahedral residual at k = 2; 1e-12 of it is still ~1e-13 of the state)
    opts = G.make_opts(scheme=2, max_newton=30, gmres_restart=40, max_gmres=800, newton_rtol=1e-12,
                       newton_atol=1e-13, gmres_rtol=1e-10, precond=0)
    rc, _ = G.cdg2_tet_step(gm, p, U, 2e-3, opts)
    assert rc == 0 and _rel(U, ref.reshape(-1)) <= 1e-10


def test_simplex_step_status_codes(G):
    xy, tri = I.tri_mesh(3, 2, 1.0, 0.2, 0.2, 720)
    gm = G.cdg2_tri_mesh_create(xy, tri, 1)
    p = _params()
    U = torch.full((gm.n_dof,), 0.1, dtype=torch.float64, device="cuda")
    for bad in (G.make_opts(mixed=True, precond=0), G.make_opts(precond=1), G.make_opts(precond=2)):
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
