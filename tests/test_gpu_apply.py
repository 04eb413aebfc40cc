"""Parity of cdg2_apply (CUDA, through the C ABI) with the FP64 oracle.

Bars: FP64 relative L2 error per species <= 1e-12; the FP32 path <= 1e-5.
Meshes span several CTAs and leave a ragged last CTA; the full-size
workloads are compared element by element as well.
"""
import itertools

import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from helpers import gaussian_state, random_state, rel_l2_per_species

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


CASES = [
    (2, (13, 5), 1), (2, (11, 5), 2), (2, (9, 7), 3),
    (3, (5, 3, 3), 1), (3, (5, 3, 2), 2), (3, (3, 3, 2), 3),
]


def _pair(G, dim, cells, k, periodic=None):
    ext = (1.0, 0.2, 0.2)
    per = periodic or ((1, 0, 0) if dim == 2 else (1, 0, 1))
    om = O.Mesh(dim, cells, ext, per, k)
    gm = G.cdg2_mesh_create(dim, cells, ext, per, k)
    return om, gm


@pytest.mark.parametrize("dim,cells,k", CASES)
@pytest.mark.parametrize("field", ["gauss", "random"])
def test_apply_fp64_parity(G, dim, cells, k, field):
    om, gm = _pair(G, dim, cells, k)
    p = I.default_params()
    U = gaussian_state(om, sigma=0.08, seed=1157 + k) if field == "gauss" else random_state(om, seed=3 + k)
    ref = O.apply(om, U, p)
    Ud = U.cuda()
    out = torch.empty_like(Ud)
    G.cdg2_apply(gm, p, Ud, out, G.CDG2_MINV)
    torch.cuda.synchronize()
    assert rel_l2_per_species(out, ref) <= FP64_TOL
    # residual form (no M^{-1})
    G.cdg2_apply(gm, p, Ud, out, 0)
    assert rel_l2_per_species(out, O.apply_residual(om, U, O.param_vector(p))) <= FP64_TOL


@pytest.mark.parametrize("periodic", [(0, 0, 0), (1, 1, 1), (0, 0, 1)])
def test_apply_fp64_boundary_variants(G, periodic):
    om, gm = _pair(G, 3, (4, 3, 3), 2, periodic)
    p = I.default_params()
    p["bc_sign"] = -1.0
    U = random_state(om, seed=21)
    ref = O.apply(om, U, p)
    out = torch.empty_like(U.cuda())
    G.cdg2_apply(gm, p, U.cuda(), out, G.CDG2_MINV)
    assert rel_l2_per_species(out, ref) <= FP64_TOL


@pytest.mark.parametrize("dim,cells,k", CASES)
def test_apply_fp32_error_bound(G, dim, cells, k):
    om, gm = _pair(G, dim, cells, k)
    p = I.default_params()
    U = gaussian_state(om, sigma=0.08, seed=1157 + k)
    ref = O.apply(om, U, p)
    Uf = U.to(torch.float32).cuda()
    out = torch.empty_like(Uf)
    G.cdg2_apply(gm, p, Uf, out, G.CDG2_MINV | G.CDG2_FP32)
    # the FP32 input is itself rounded: compare with the oracle on the rounded input
    ref32 = O.apply(om, Uf.double().cpu(), p)
    assert rel_l2_per_species(out, ref32) <= FP32_TOL


@pytest.mark.parametrize("k", [2, 3])
def test_apply_forcing_parity(G, k):
    om, gm = _pair(G, 2, (16, 4), k)
    p = I.default_params()
    ph = I.mms_phases(1158)
    t = 0.37
    U = O.project(om, lambda x: O.mms_solution(x, t, ph, 0.2))
    g = O.mms_forcing(p, ph, 0.2)
    x = om.phys(torch.arange(om.E), om.qpts)
    gx = g(x, t)
    ref = O.apply(om, U, p, forcing=lambda xx, tt: gx, t=t)
    out = torch.empty_like(U.cuda())
    G.cdg2_apply(gm, G.make_params(p, ph), U.cuda(), out, G.CDG2_MINV | G.CDG2_FORCING, t)
    # For the manufactured solution the forcing cancels most of L_h(U) (by up to
    # 16x here), so the bar applies relative to the size of the terms, not of
    # their sum: ||out - ref||_s <= tol * max(||ref||_s, ||M^-1 L_h(U)||_s).
    lh = O.apply(om, U, p)
    d = ((out.cpu().reshape(ref.shape) - ref) ** 2).sum(dim=(0, 2)).sqrt()
    scale = torch.maximum((ref ** 2).sum(dim=(0, 2)).sqrt(), (lh ** 2).sum(dim=(0, 2)).sqrt())
    assert float((d / scale).max()) <= FP64_TOL


@pytest.mark.parametrize("cfg", [0, 1, 3])
def test_apply_full_size_workloads(G, cfg):
    w = I.workload(cfg)
    om = O.Mesh(w.dim, w.cells, w.extent, w.periodic, w.k)
    gm = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    p = I.default_params()
    U = gaussian_state(om, w.n_gauss, w.sigma, w.floor, w.seed)
    ref = O.apply(om, U, p)
    out = torch.empty_like(U.cuda())
    G.cdg2_apply(gm, p, U.cuda(), out, G.CDG2_MINV)
    assert rel_l2_per_species(out, ref) <= FP64_TOL
    # element-by-element: the worst element's relative error stays small too
    d = (out.cpu() - ref).abs().amax(dim=(1, 2)) / ref.abs().amax()
    assert float(d.max()) <= 1e-12


@pytest.mark.parametrize("dim,cells,k", [(2, (13, 5), 1), (2, (9, 7), 3), (3, (5, 3, 2), 2), (3, (3, 3, 2), 3)])
def test_project_gaussians_parity(G, dim, cells, k):
    om, gm = _pair(G, dim, cells, k)
    cen, amp = I.gaussian_draws(dim, om.extent, 4, 99)
    ref = O.project(om, lambda x: O.gaussian_field(om, x, cen, amp, 0.05, 1e-3))
    out = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_project_gaussians(gm, cen, amp, 0.05, 1e-3, out)
    assert rel_l2_per_species(out, ref) <= FP64_TOL
    out32 = torch.empty(gm.n_dof, dtype=torch.float32, device="cuda")
    G.cdg2_project_gaussians(gm, cen, amp, 0.05, 1e-3, out32, G.CDG2_FP32)
    assert rel_l2_per_species(out32, ref) <= 1e-6


@pytest.mark.parametrize("dim,cells,k", [(2, (16, 4), 2), (3, (4, 2, 2), 3)])
def test_project_mms_parity(G, dim, cells, k):
    om, gm = _pair(G, dim, cells, k)
    ph = I.mms_phases(1158)
    ref = O.project(om, lambda x: O.mms_solution(x, 0.25, ph, 0.2))
    out = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_project_mms(gm, G.make_params(I.default_params(), ph), 0.25, out)
    assert rel_l2_per_species(out, ref) <= FP64_TOL


@pytest.mark.parametrize("cfg", [2, 4])
def test_apply_full_size_sampled_rows(G, cfg):
    """2D 128x32 Q2 and the largest workload, 3D 128x32x32 Q2 (21.2M DOF): apply
    and JVP rows of sampled elements against the oracle on the box of the element and its face
    neighbours (which fixes the element's row of M^{-1} L_h): three cells along
    each axis, two at a Gamma_1 / Gamma_2 side, Gamma_{1,in} shifted into the
    box's coordinates.  A periodic wrap keeps its K^- (the last cell) in the
    box's order."""
    w = I.workload(cfg)
    gm = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    p = I.default_params()
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    U = torch.from_numpy(I.random_coefficients(gm.n_elem, gm.n_basis, w.seed, 0.1))
    out = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_apply(gm, p, U.reshape(-1).cuda(), out, G.CDG2_MINV)
    got = out.cpu().reshape(U.shape)
    dU = torch.from_numpy(I.random_coefficients(gm.n_elem, gm.n_basis, w.seed + 1, 0.3))
    G.cdg2_jvp(gm, p, U.reshape(-1).cuda(), dU.reshape(-1).cuda(), out, G.CDG2_MINV)
    got_jvp = out.cpu().reshape(U.shape)
    n = list(w.cells[: w.dim])
    h = [w.extent[a] / n[a] for a in range(w.dim)]
    rng = np.random.default_rng(cfg)
    picks = [tuple(int(rng.integers(0, n[a])) for a in range(w.dim)) for _ in range(24)]
    picks += [tuple([0, 0] + [0] * (w.dim - 2)), tuple([n[0] - 1, n[1] - 1] + [n[a] - 1 for a in range(2, w.dim)]),
              tuple([5, 0] + [3] * (w.dim - 2)), tuple([7, n[1] - 1] + [0] * (w.dim - 2))]
    for idx in picks:
        ranges, local = [], []
        for a in range(w.dim):
            if w.periodic[a] or 0 < idx[a] < n[a] - 1:
                ranges.append([(idx[a] + d) % n[a] for d in (-1, 0, 1)])
                local.append(1)
            elif idx[a] == 0:
                ranges.append([0, 1])
                local.append(0)
            else:
                ranges.append([n[a] - 2, n[a] - 1])
                local.append(1)
        cells = tuple(len(r) for r in ranges)
        ext = tuple(cells[a] * h[a] for a in range(w.dim))
        shift = (idx[0] - local[0]) * h[0]
        om = O.Mesh(w.dim, cells, ext, (0,) * w.dim, w.k,
                    gamma1_in=(0.375 - shift, 0.625 - shift))
        gids = []
        for t in itertools.product(*reversed(ranges)):
            g = list(reversed(t))
            gid, stride = 0, 1
            for a in range(w.dim):
                gid += g[a] * stride
                stride *= n[a]
            gids.append(gid)
        lid, stride = 0, 1
        for a in range(w.dim):
            lid += local[a] * stride
            stride *= cells[a]
        ref = O.apply(om, U[gids], p)[lid]
        e = gids[lid]
        err = float((got[e] - ref).norm() / ref.norm())
        assert err <= 1e-12, (idx, err)
        ref = O.jvp(om, U[gids], dU[gids], p)[lid]
        err = float((got_jvp[e] - ref).norm() / ref.norm())
        assert err <= 1e-12, ("jvp", idx, err)
