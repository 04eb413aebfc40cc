"""Parity of cdg2_vjp (CUDA, through the C ABI) with the oracle's reverse-mode
automatic differentiation: J(U)^T lam and (df/dtheta)^T lam.

Bars: FP64 relative L2 error per species <= 1e-12 (gU) and relative error
<= 1e-12 on the theta gradient; FP32 gU <= 1e-5.  Also: the transpose
identity <lam, J v> = <J^T lam, v> between the GPU's JVP and VJP, and
bitwise reproducibility of repeated calls (no atomics).
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


def _params():
    p = I.default_params()
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    return p


def _theta_rel(got, ref):
    return float((got.cpu() - ref).abs().max() / ref.abs().max())


@pytest.mark.parametrize("dim,cells,k", CASES)
def test_vjp_fp64_parity(G, dim, cells, k):
    om, gm = _pair(G, dim, cells, k)
    p = _params()
    U = gaussian_state(om, sigma=0.08, seed=1157 + k)
    U[:, 3, 0] += 0.02                    # c1 above c1* on part of Gamma_1: beta1 matters
    lam = random_state(om, seed=60 + k) - 1.0
    gU_ref, gth_ref = O.vjp(om, U, lam, p, I.THETA_NAMES)
    gU = torch.empty_like(U.cuda())
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    G.cdg2_vjp(gm, p, U.cuda(), lam.cuda(), gU, gth, G.CDG2_MINV)
    assert rel_l2_per_species(gU, gU_ref) <= FP64_TOL
    assert _theta_rel(gth, gth_ref) <= FP64_TOL


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1)])
def test_vjp_boundary_variants_residual_form(G, periodic):
    om, gm = _pair(G, 3, (4, 3, 3), 2, periodic)
    p = _params()
    U = random_state(om, seed=31)
    lam = random_state(om, seed=32) - 1.0
    theta = torch.tensor([float(p[n]) for n in I.THETA_NAMES], dtype=torch.float64)
    _, fn = torch.func.vjp(lambda V, th: _residual_theta(om, V, p, th), U, theta)
    gU_ref, gth_ref = fn(lam)
    gU = torch.empty_like(U.cuda())
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    G.cdg2_vjp(gm, p, U.cuda(), lam.cuda(), gU, gth, 0)
    assert rel_l2_per_species(gU, gU_ref) <= FP64_TOL
    if float(gth_ref.abs().max()) > 0:
        assert _theta_rel(gth, gth_ref) <= FP64_TOL


def _residual_theta(om, V, p, th):
    pv = O.param_vector(p)
    for i, n in enumerate(I.THETA_NAMES):
        pv[n] = th[i]
    return O.apply_residual(om, V, pv)


@pytest.mark.parametrize("dim,cells,k", [(2, (9, 7), 3), (3, (4, 3, 2), 2)])
def test_vjp_is_transpose_of_gpu_jvp(G, dim, cells, k):
    om, gm = _pair(G, dim, cells, k)
    p = _params()
    U = gaussian_state(om, sigma=0.08, seed=5).cuda()
    v = (random_state(om, seed=6) - 1.0).cuda()
    lam = (random_state(om, seed=7) - 1.0).cuda()
    jv = torch.empty_like(U)
    G.cdg2_jvp(gm, p, U, v, jv, G.CDG2_MINV)
    gU = torch.empty_like(U)
    G.cdg2_vjp(gm, p, U, lam, gU, None, G.CDG2_MINV)
    a, b = float((lam * jv).sum()), float((gU * v).sum())
    assert abs(a - b) <= 1e-12 * float(lam.norm() * jv.norm())
    # theta: <lam, df/dtheta dth> = <gtheta, dth>
    dth = np.random.default_rng(1).standard_normal(8)
    G.cdg2_jvp(gm, p, U, torch.zeros_like(U), jv, G.CDG2_MINV, dtheta=dth)
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    G.cdg2_vjp(gm, p, U, lam, gU, gth, G.CDG2_MINV)
    a, b = float((lam * jv).sum()), float((gth.cpu().numpy() * dth).sum())
    assert abs(a - b) <= 1e-12 * float(lam.norm() * jv.norm())


def test_vjp_bitwise_reproducible(G):
    om, gm = _pair(G, 3, (8, 4, 4), 2)
    p = _params()
    U = gaussian_state(om, sigma=0.06, seed=8).cuda()
    lam = (random_state(om, seed=9) - 1.0).cuda()
    outs = []
    for _ in range(3):
        gU = torch.empty_like(U)
        gth = torch.zeros(8, dtype=torch.float64, device="cuda")
        G.cdg2_vjp(gm, p, U, lam, gU, gth, G.CDG2_MINV)
        outs.append((gU.clone(), gth.clone()))
    for gU, gth in outs[1:]:
        assert torch.equal(gU, outs[0][0]) and torch.equal(gth, outs[0][1])


@pytest.mark.parametrize("dim,cells,k", [(2, (9, 7), 3), (3, (3, 3, 2), 3)])
def test_vjp_fp32(G, dim, cells, k):
    om, gm = _pair(G, dim, cells, k)
    p = _params()
    U = gaussian_state(om, sigma=0.08, seed=5).float()
    lam = (random_state(om, seed=9) - 1.0).float()
    ref, _ = O.vjp(om, U.double(), lam.double(), p)
    gU = torch.empty_like(U.cuda())
    G.cdg2_vjp(gm, p, U.cuda(), lam.cuda(), gU, None, G.CDG2_MINV | G.CDG2_FP32)
    assert rel_l2_per_species(gU, ref) <= FP32_TOL


@pytest.mark.parametrize("cfg", [2, 3])
def test_vjp_full_size(G, cfg):
    w = I.workload(cfg)
    om = O.Mesh(w.dim, w.cells, w.extent, w.periodic, w.k)
    gm = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    p = I.default_params()
    U = gaussian_state(om, w.n_gauss, w.sigma, w.floor, w.seed)
    lam = torch.from_numpy(I.random_coefficients(om.E, om.nb, 78)) - 1.0
    gU_ref, gth_ref = O.vjp(om, U, lam, p, I.THETA_NAMES)
    gU = torch.empty_like(U.cuda())
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    G.cdg2_vjp(gm, p, U.cuda(), lam.cuda(), gU, gth, G.CDG2_MINV)
    assert rel_l2_per_species(gU, gU_ref) <= FP64_TOL
    assert _theta_rel(gth, gth_ref) <= FP64_TOL
