"""The assembled Jacobian (cdg2_matrix_create / cdg2_assemble_jacobian /
cdg2_spmv) and the step that solves with it (jacobian = 1).

Sec. 3.2 solves matrix-free and sets the fully assembled approach aside; the
assembled J = d(M^{-1} L_h)/dU must be that same derivative.  Checked, on
small meshes, entry by entry against the oracle's dense Jacobian (automatic
differentiation of its FP64 operator) at 1e-12 of the largest entry; at full
size (2D 128x32 Q2) its product with a random vector against the JVP kernel
at 1e-12; and an implicit step solved with it against the matrix-free step
at 1e-10.
"""
import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from helpers import random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


@pytest.mark.parametrize("dim,cells,k,periodic", [(2, (4, 3), 1, (1, 0)), (2, (3, 4), 2, (1, 0)),
                                                  (2, (3, 3), 1, (1, 1)), (3, (3, 2, 3), 1, (1, 0, 1))])
def test_assembled_matches_oracle_dense_jacobian(G, dim, cells, k, periodic):
    ext = (1.0, 0.2, 0.2)[:dim]
    om = O.Mesh(dim, cells, ext, periodic, k)
    gm = G.cdg2_mesh_create(dim, cells, ext, periodic, k)
    p = I.default_params()
    p["chi0"] = (0.2, 0.1, 0.1, 0.1)
    U = random_state(om, seed=17)
    J = torch.func.jacfwd(lambda V: O.apply(om, V, p))(U).reshape(gm.n_dof, gm.n_dof)
    A = G.cdg2_matrix_create(gm)
    Ud = U.reshape(-1).cuda()
    G.cdg2_assemble_jacobian(A, p, Ud)
    cols = torch.zeros(gm.n_dof, gm.n_dof, dtype=torch.float64)
    e = torch.zeros(gm.n_dof, dtype=torch.float64, device="cuda")
    y = torch.empty_like(e)
    for c in range(gm.n_dof):
        e.zero_()
        e[c] = 1.0
        G.cdg2_spmv(A, e, y)
        cols[:, c] = y.cpu()
    err = float((cols - J).abs().max() / J.abs().max())
    assert err <= 1e-12, err


def test_assembled_spmv_matches_jvp_full_size(G):
    w = I.workload(2)
    gm = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    p = I.default_params()
    U = torch.from_numpy(I.random_coefficients(gm.n_elem, gm.n_basis, 5)).reshape(-1).cuda()
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(gm.n_dof)).cuda()
    A = G.cdg2_matrix_create(gm)
    G.cdg2_assemble_jacobian(A, p, U)
    y = torch.empty_like(x)
    G.cdg2_spmv(A, x, y)
    ref = torch.empty_like(x)
    G.cdg2_jvp(gm, p, U, x, ref, G.CDG2_MINV)
    err = float((y - ref).norm() / ref.norm())
    assert err <= 1e-12, err
    # alpha / beta
    z = torch.ones_like(x)
    G.cdg2_spmv(A, x, z, alpha=2.0, beta=-3.0)
    assert float((z - (2.0 * ref - 3.0)).norm() / ref.norm()) <= 1e-12


@pytest.mark.parametrize("precond", [0, 1, 2])
def test_step_with_assembled_jacobian(G, precond):
    w = I.workload(0)
    gm = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    p = I.default_params()
    U0 = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    cen, amp = I.gaussian_draws(w.dim, w.extent, w.n_gauss, w.seed)
    G.cdg2_project_gaussians(gm, cen, amp, w.sigma, w.floor, U0)
    res = {}
    for jac in (0, 1):
        U = U0.clone()
        rc, st = G.cdg2_step(gm, p, U, 0.0, w.dt, G.make_opts(scheme=G.CDG2_SDIRK2, newton_rtol=1e-12,
                                                               gmres_rtol=1e-10, max_gmres=2000, precond=precond,
                                                               jacobian=jac))
        assert rc == 0
        res[jac] = U
    assert float((res[1] - res[0]).norm() / res[0].norm()) <= 1e-10


def test_assembled_rejects_short_periodic_axes_and_mixed(G):
    gm = G.cdg2_mesh_create(2, (2, 3), (1.0, 0.2), (1, 0), 1)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_matrix_create(gm)
    gm2 = G.cdg2_mesh_create(2, (4, 3), (1.0, 0.2), (1, 0), 1)
    U = torch.ones(gm2.n_dof, dtype=torch.float64, device="cuda") * 0.5
    rc, _ = G.cdg2_step(gm2, I.default_params(), U, 0.0, 1e-3, G.make_opts(mixed=True, jacobian=1),
                        raise_on_error=False)
    assert rc == -1
