"""Parity of cdg2_jvp (CUDA, through the C ABI) with the oracle's automatic
differentiation: J(U) dU and the parameter tangent (df/dtheta) dtheta.

Bars: FP64 relative L2 error per species <= 1e-12; FP32 <= 1e-5 on these
meshes.  Also checked against central differences of the GPU apply.
"""
import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from helpers import gaussian_state, random_state, rel_l2_per_species

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5

CASES = [
    (2, (13, 5), 1), (2, (11, 5), 2), (2, (9, 7), 3),
    (3, (5, 3, 3), 1), (3, (5, 3, 2), 2), (3, (3, 3, 2), 3),
]


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


def _pair(G, dim, cells, k, periodic=None):
    ext = (1.0, 0.2, 0.2)
    per = periodic or ((1, 0, 0) if dim == 2 else (1, 0, 1))
    return O.Mesh(dim, cells, ext, per, k), G.cdg2_mesh_create(dim, cells, ext, per, k)


def _chemotactic_params():
    p = I.default_params()
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)     # make the LLF/velocity linearisation matter
    return p


@pytest.mark.parametrize("dim,cells,k", CASES)
def test_jvp_fp64_parity(G, dim, cells, k):
    om, gm = _pair(G, dim, cells, k)
    p = _chemotactic_params()
    U = gaussian_state(om, sigma=0.08, seed=1157 + k)
    dU = random_state(om, seed=40 + k, scale=0.3) - 1.0
    ref = O.jvp(om, U, dU, p)
    out = torch.empty_like(U.cuda())
    G.cdg2_jvp(gm, p, U.cuda(), dU.cuda(), out, G.CDG2_MINV)
    assert rel_l2_per_species(out, ref) <= FP64_TOL


@pytest.mark.parametrize("dim,cells,k", [(2, (9, 7), 2), (3, (4, 3, 2), 2)])
def test_jvp_theta_tangent(G, dim, cells, k):
    om, gm = _pair(G, dim, cells, k)
    p = _chemotactic_params()
    U = gaussian_state(om, sigma=0.08, seed=3)
    U[:, 3, 0] += 0.05      # c1 above both thresholds: the inflow terms are on
    dU = random_state(om, seed=7) - 1.0
    dth = np.random.default_rng(0).standard_normal(8)
    ref = O.jvp_theta(om, U, dU, p, I.THETA_NAMES, dth)
    out = torch.empty_like(U.cuda())
    G.cdg2_jvp(gm, p, U.cuda(), dU.cuda(), out, G.CDG2_MINV, dtheta=dth)
    assert rel_l2_per_species(out, ref) <= FP64_TOL
    # the theta part alone (dU = 0)
    ref0 = O.jvp_theta(om, U, torch.zeros_like(dU), p, I.THETA_NAMES, dth)
    G.cdg2_jvp(gm, p, U.cuda(), torch.zeros_like(dU).cuda(), out, G.CDG2_MINV, dtheta=dth)
    assert rel_l2_per_species(out, ref0) <= FP64_TOL


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1)])
def test_jvp_boundary_variants(G, periodic):
    om, gm = _pair(G, 3, (4, 3, 3), 2, periodic)
    p = _chemotactic_params()
    U = random_state(om, seed=21)
    dU = random_state(om, seed=22) - 1.0
    out = torch.empty_like(U.cuda())
    G.cdg2_jvp(gm, p, U.cuda(), dU.cuda(), out, 0)
    ref = torch.func.jvp(lambda V: O.apply_residual(om, V, O.param_vector(p)), (U,), (dU,))[1]
    assert rel_l2_per_species(out, ref) <= FP64_TOL


@pytest.mark.parametrize("dim,cells,k", [(2, (9, 7), 3), (3, (3, 3, 2), 3)])
def test_jvp_fp32(G, dim, cells, k):
    om, gm = _pair(G, dim, cells, k)
    p = _chemotactic_params()
    U = gaussian_state(om, sigma=0.08, seed=5).float()
    dU = (random_state(om, seed=9) - 1.0).float()
    ref = O.jvp(om, U.double(), dU.double(), p)
    out = torch.empty_like(U.cuda())
    G.cdg2_jvp(gm, p, U.cuda(), dU.cuda(), out, G.CDG2_MINV | G.CDG2_FP32)
    assert rel_l2_per_species(out, ref) <= FP32_TOL


def test_jvp_matches_central_differences_of_apply(G):
    om, gm = _pair(G, 2, (16, 4), 2)
    p = _chemotactic_params()
    U = gaussian_state(om, sigma=0.08, seed=11).cuda()
    dU = (random_state(om, seed=12) - 1.0).cuda()
    jv = torch.empty_like(U)
    G.cdg2_jvp(gm, p, U, dU, jv, G.CDG2_MINV)
    fp, fm = torch.empty_like(U), torch.empty_like(U)
    eps = 1e-6
    G.cdg2_apply(gm, p, U + eps * dU, fp, G.CDG2_MINV)
    G.cdg2_apply(gm, p, U - eps * dU, fm, G.CDG2_MINV)
    fd = (fp - fm) / (2 * eps)
    # The LLF flux has kinks (|v| and max) where a normal derivative of c1 or
    # n1 vanishes; +-eps can straddle one, so the difference quotient is only
    # accurate to about 1e-5 there.  The exact pin is the oracle parity above.
    assert float((fd - jv).norm() / jv.norm()) < 1e-4


@pytest.mark.parametrize("cfg", [1, 3])
def test_jvp_full_size(G, cfg):
    w = I.workload(cfg)
    om = O.Mesh(w.dim, w.cells, w.extent, w.periodic, w.k)
    gm = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    p = I.default_params()
    U = gaussian_state(om, w.n_gauss, w.sigma, w.floor, w.seed)
    dU = torch.from_numpy(I.random_coefficients(om.E, om.nb, 77)) - 1.0
    ref = O.jvp(om, U, dU, p)
    out = torch.empty_like(U.cuda())
    G.cdg2_jvp(gm, p, U.cuda(), dU.cuda(), out, G.CDG2_MINV)
    assert rel_l2_per_species(out, ref) <= FP64_TOL
