"""Gradients through the implicit steps: cdg2_step_adjoint and the
checkpointed autograd Function against the oracle's dense-Jacobian adjoint
and against central finite differences of the GPU forward solve.

Bars: adjoint vs the oracle's dense adjoint 1e-9 (both limited by their
linear-solve tolerances); the gradient of the final-time integral of n3 with
respect to the 8 reaction coefficients and the initial c2 field against
central differences (step 1e-6): relative error 1e-6; checkpoint spacing and
mixed precision do not change the gradient beyond 1e-10 / 1e-9.
"""
import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from helpers import gaussian_state

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


def _tight(G, scheme, mixed=False):
    return G.make_opts(scheme=scheme, mixed=mixed, max_newton=40, gmres_restart=40, max_gmres=1000,
                       newton_rtol=1e-13, newton_atol=1e-16, gmres_rtol=1e-6 if mixed else 1e-11)


@pytest.mark.parametrize("scheme,name", [(2, "sdirk2"), (3, "sdirk3")])
@pytest.mark.parametrize("precond", [1, 2])
def test_step_adjoint_matches_oracle_dense_adjoint(G, scheme, name, precond):
    om = O.Mesh(2, (4, 2), (1.0, 0.2), (1, 0), 1)
    gm = G.cdg2_mesh_create(2, (4, 2), (1.0, 0.2), (1, 0), 1)
    p = _params()
    U = gaussian_state(om, sigma=0.1, seed=12)
    U[:, 3, 0] += 0.05
    dt = 2e-3
    _, stages = O.step_stages(om, U, p, 0.0, dt, name)
    lam = torch.from_numpy(np.random.default_rng(3).standard_normal(U.shape))
    lam_ref, gth_ref = O.step_adjoint(om, stages, p, dt, name, lam, I.THETA_NAMES)
    o = _tight(G, scheme)
    o.precond = precond
    st = torch.empty(len(stages) * gm.n_dof, dtype=torch.float64, device="cuda")
    Ud = U.clone().cuda()
    G.cdg2_step_stages(gm, p, Ud, 0.0, dt, st, o)
    assert float((st.cpu() - torch.cat([y.reshape(-1) for y in stages])).abs().max()) < 1e-10
    lam_d = lam.clone().cuda()
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    G.cdg2_step_adjoint(gm, p, st, 0.0, dt, lam_d, gth, o)
    assert float((lam_d.cpu().reshape(lam.shape) - lam_ref).norm() / lam_ref.norm()) <= 1e-9
    assert float((gth.cpu() - gth_ref).abs().max() / gth_ref.abs().max()) <= 1e-9


def _plaque_functional_grad(G, gm, p, U0, theta, dt, nsteps, checkpoint, opts):
    """J = int n3(T) = sum_K |K| U_{K,n3,0}; returns J, dJ/dU0, dJ/dtheta."""
    from paper_1403_1157_gb300 import adjoint as Adj
    U0v = U0.clone().requires_grad_(True)
    th = theta.clone().requires_grad_(True)
    UT = Adj.steps(U0v, th, gm, p, 0.0, dt, nsteps, checkpoint, opts)
    vol = float(np.prod([e / c for e, c in zip(gm.desc.extent[: gm.dim], gm.desc.cells[: gm.dim])]))
    Jv = vol * UT.view(gm.n_elem, 6, gm.n_basis)[:, 2, 0].sum()
    Jv.backward()
    return float(Jv.detach()), U0v.grad.detach(), th.grad.detach()


def _forward_J(G, gm, p, U0, theta, dt, nsteps, opts):
    from paper_1403_1157_gb300 import adjoint as Adj
    with torch.no_grad():
        UT = Adj.steps(U0, theta, gm, p, 0.0, dt, nsteps, 1000, opts)
    vol = float(np.prod([e / c for e, c in zip(gm.desc.extent[: gm.dim], gm.desc.cells[: gm.dim])]))
    return vol * float(UT.view(gm.n_elem, 6, gm.n_basis)[:, 2, 0].sum())


def test_gradient_through_steps_matches_central_differences(G):
    """The differentiation workload, scaled down: 2D Q2, seeded Gaussians, several steps with checkpoints."""
    cells, k, nsteps, dt = (16, 4), 2, 6, 1e-3
    om = O.Mesh(2, cells, (1.0, 0.2), (1, 0), k)
    gm = G.cdg2_mesh_create(2, cells, (1.0, 0.2), (1, 0), k)
    p = _params()
    U0 = gaussian_state(om, sigma=0.08, seed=1159).cuda()
    U0.view(gm.n_elem, 6, gm.n_basis)[:, 3, 0] += 0.05
    theta = torch.tensor([p[nm] for nm in I.THETA_NAMES], dtype=torch.float64, device="cuda")
    o = _tight(G, 3)
    J, gU0, gth = _plaque_functional_grad(G, gm, p, U0, theta, dt, nsteps, 2, o)
    for i in range(8):
        h = 1e-6 * max(1.0, abs(float(theta[i])))
        tp, tm = theta.clone(), theta.clone()
        tp[i] += h
        tm[i] -= h
        fd = (_forward_J(G, gm, p, U0, tp, dt, nsteps, o) - _forward_J(G, gm, p, U0, tm, dt, nsteps, o)) / (2 * h)
        assert abs(fd - float(gth[i])) <= 1e-6 * max(abs(fd), 1e-3), (i, fd, float(gth[i]))
    # initial fields: a random direction over all species (n1 drives n3 through d1 n1 - gamma n1)
    rng = np.random.default_rng(5)
    d = torch.from_numpy(rng.standard_normal(U0.shape)).cuda()
    eps = 1e-6
    fd = (_forward_J(G, gm, p, U0 + eps * d, theta, dt, nsteps, o)
          - _forward_J(G, gm, p, U0 - eps * d, theta, dt, nsteps, o)) / (2 * eps)
    ad = float((gU0 * d).sum())
    assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)
    # the initial c2 field reaches n3 only through c3 -> chemotaxis of n1 -> n3; over a few
    # steps that sensitivity is tiny, so compare it on the scale of the full gradient
    dc2 = torch.zeros_like(U0)
    dc2.view(gm.n_elem, 6, gm.n_basis)[:, 4, :] = d.view(gm.n_elem, 6, gm.n_basis)[:, 4, :]
    fd2 = (_forward_J(G, gm, p, U0 + eps * dc2, theta, dt, nsteps, o)
           - _forward_J(G, gm, p, U0 - eps * dc2, theta, dt, nsteps, o)) / (2 * eps)
    ad2 = float((gU0 * dc2).sum())
    assert abs(fd2 - ad2) <= 1e-6 * float(gU0.norm() * dc2.norm())


def test_checkpoint_spacing_and_precision_do_not_change_the_gradient(G):
    cells, k, nsteps, dt = (8, 2), 2, 5, 1e-3
    om = O.Mesh(2, cells, (1.0, 0.2), (1, 0), k)
    gm = G.cdg2_mesh_create(2, cells, (1.0, 0.2), (1, 0), k)
    p = _params()
    U0 = gaussian_state(om, sigma=0.1, seed=7).cuda()
    theta = torch.tensor([p[nm] for nm in I.THETA_NAMES], dtype=torch.float64, device="cuda")
    res = {}
    for cp in (1, 2, 10):
        res[cp] = _plaque_functional_grad(G, gm, p, U0, theta, dt, nsteps, cp, _tight(G, 2))
    for cp in (2, 10):
        assert float((res[cp][1] - res[1][1]).norm() / res[1][1].norm()) <= 1e-10
        assert float((res[cp][2] - res[1][2]).abs().max() / res[1][2].abs().max()) <= 1e-10
    mixed = _plaque_functional_grad(G, gm, p, U0, theta, dt, nsteps, 2, _tight(G, 2, mixed=True))
    assert float((mixed[1] - res[1][1]).norm() / res[1][1].norm()) <= 1e-9
    assert float((mixed[2] - res[1][2]).abs().max() / res[1][2].abs().max()) <= 1e-9
