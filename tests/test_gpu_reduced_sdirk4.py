"""The reduced three-species model of Eq. (2) (model = 1) and the order-4
SDIRK method through the C ABI, against the oracle.  Bars as for the
six-species operator: 1e-12 for apply/JVP/VJP, 1e-10 for steps, 1e-9 for
the step adjoint."""
import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from helpers import gaussian_state, rel_l2_per_species

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


def _reduced_state(om, seed):
    U = gaussian_state(om, n_gauss=8, sigma=0.06, seed=seed)
    U[:, [1, 4, 5], :] = 0.0          # species outside Eq. (2)
    U[:, 3, 0] += 0.02
    return U


@pytest.mark.parametrize("k", [1, 2, 3])
def test_reduced_model_apply_jvp_vjp(G, k):
    cells = (5, 3, 2)
    om = O.Mesh(3, cells, (1.0, 0.2, 0.2), (1, 0, 1), k)
    gm = G.cdg2_mesh_create(3, cells, (1.0, 0.2, 0.2), (1, 0, 1), k)
    p = I.default_params()
    p["model"] = 1
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    U = _reduced_state(om, 30 + k)
    out = torch.empty_like(U.cuda())
    G.cdg2_apply(gm, p, U.cuda(), out, G.CDG2_MINV)
    ref = O.apply(om, U, p)
    assert rel_l2_per_species(out.reshape(ref.shape)[:, [0, 2, 3]], ref[:, [0, 2, 3]]) <= 1e-12
    assert float(out.reshape(ref.shape)[:, [1, 4, 5]].abs().max()) == 0.0
    dU = torch.from_numpy(np.random.default_rng(k).standard_normal(U.shape))
    dU[:, [1, 4, 5], :] = 0.0
    G.cdg2_jvp(gm, p, U.cuda(), dU.cuda(), out, G.CDG2_MINV)
    ref = O.jvp(om, U, dU, p)
    assert rel_l2_per_species(out.reshape(ref.shape)[:, [0, 2, 3]], ref[:, [0, 2, 3]]) <= 1e-12
    lam = torch.from_numpy(np.random.default_rng(10 + k).standard_normal(U.shape))
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    G.cdg2_vjp(gm, p, U.cuda(), lam.cuda(), out, gth, G.CDG2_MINV)
    gU_ref, gth_ref = O.vjp(om, U, lam, p, I.THETA_NAMES)
    assert rel_l2_per_species(out.reshape(gU_ref.shape)[:, [0, 2, 3]], gU_ref[:, [0, 2, 3]]) <= 1e-12
    # coefficients outside Eq. (2) (d2, alpha2, k_ox) have zero gradient on these fields
    for i in (0, 2, 3, 5, 7):
        assert abs(float(gth[i]) - float(gth_ref[i])) <= 1e-12 * float(gth_ref.abs().max())


@pytest.mark.parametrize("model", [0, 1])
def test_sdirk4_step_matches_oracle(G, model):
    om = O.Mesh(2, (8, 2), (1.0, 0.2), (1, 0), 2)
    gm = G.cdg2_mesh_create(2, (8, 2), (1.0, 0.2), (1, 0), 2)
    p = I.default_params()
    p["model"] = model
    U0 = gaussian_state(om, sigma=0.1, seed=1157)
    if model == 1:
        U0[:, [1, 4, 5], :] = 0.0
    dt = 1e-3
    ref = U0.clone()
    for i in range(2):
        ref = O.step(om, ref, p, i * dt, dt, "sdirk4")
    U = U0.clone().cuda()
    o = G.make_opts(scheme=G.CDG2_SDIRK4, max_newton=30, gmres_restart=40, max_gmres=800, newton_rtol=1e-14,
                    newton_atol=1e-15, gmres_rtol=1e-10)
    for i in range(2):
        rc, st = G.cdg2_step(gm, p, U, i * dt, dt, o)
        assert rc == 0 and st["stages"] == 5
    assert float((U.cpu() - ref).norm() / ref.norm()) <= 1e-10


def test_sdirk4_adjoint_matches_oracle(G):
    om = O.Mesh(2, (4, 2), (1.0, 0.2), (1, 0), 1)
    gm = G.cdg2_mesh_create(2, (4, 2), (1.0, 0.2), (1, 0), 1)
    p = I.default_params()
    U = gaussian_state(om, sigma=0.1, seed=12)
    U[:, 3, 0] += 0.05
    dt = 2e-3
    _, stages = O.step_stages(om, U, p, 0.0, dt, "sdirk4")
    lam = torch.from_numpy(np.random.default_rng(3).standard_normal(U.shape))
    lam_ref, gth_ref = O.step_adjoint(om, stages, p, dt, "sdirk4", lam, I.THETA_NAMES)
    o = G.make_opts(scheme=G.CDG2_SDIRK4, max_newton=40, gmres_restart=40, max_gmres=1000, newton_rtol=1e-13,
                    newton_atol=1e-16, gmres_rtol=1e-11)
    st = torch.empty(5 * gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_step_stages(gm, p, U.clone().cuda(), 0.0, dt, st, o)
    lam_d = lam.clone().cuda()
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    G.cdg2_step_adjoint(gm, p, st, 0.0, dt, lam_d, gth, o)
    assert float((lam_d.cpu().reshape(lam.shape) - lam_ref).norm() / lam_ref.norm()) <= 1e-9
    assert float((gth.cpu() - gth_ref).abs().max() / gth_ref.abs().max()) <= 1e-9
