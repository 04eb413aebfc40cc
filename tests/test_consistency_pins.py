"""Consistency pins of the oracles (oracle/cdg2_tri_oracle.py,
oracle/cdg2_tet_oracle.py, and oracle/cdg2_oracle.py on hexahedra) against
the strong form of the model (Sec. 2).

For smooth positive fields whose normal derivative vanishes on every wall of
the box (and that are periodic along periodic axes), the chemotactic and
diffusive normal fluxes vanish on the boundary,
so with the inflow data of Eq. (3) switched off the DG operator of Sec. 3.1
must approximate the strong operator L(u) = div(A grad u - F(u, grad u)) +
S(u): ||M^{-1} L_h(P u) - P L(u)|| / ||P L(u)|| = O(h^{k-1}) under
refinement (P the L2 projection; L(u) by automatic differentiation of the
closed-form fields, independent of the DG code).  A sign or orientation
mistake in a face term (the chemotactic flux, the K^+ side, the average in
the consistency term, an inward face normal) makes the error grow like
h^{-1} instead.  The chemotactic sensitivities are raised above the preset
so that the chemotactic terms dominate the check."""
import math

import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from oracle import cdg2_tet_oracle as TT
from oracle import cdg2_tri_oracle as T

AMP = (0.3, 0.25, 0.2, 0.35, 0.3, 0.25)   # per species
MX = (1, 2, 1, 2, 1, 2)                    # cosine modes along x


def params():
    p = I.default_params()
    p.update(chi0=(0.5, 0.3, 0.4, 0.2), beta1=0.0, beta2=0.0, sigma=0.0)
    return p


def walled_fields(ext):
    """u_s = 1 + a_s cos(m_s pi x / L_x) prod_{j>0} cos(pi x_j / L_j): zero normal derivative on every side."""
    def f(x):
        out = []
        for a, m in zip(AMP, MX):
            v = torch.cos(m * math.pi * x[..., 0] / ext[0])
            for j in range(1, len(ext)):
                v = v * torch.cos(math.pi * x[..., j] / ext[j])
            out.append(1.0 + a * v)
        return torch.stack(out)
    return f


def periodic_xz_fields(ext):
    """u_s = 1 + a_s cos(2 m_s pi x / L_x) cos(pi y / L_y) cos(2 pi z / L_z): periodic in x and z, walls in y."""
    def f(x):
        return torch.stack([1.0 + a * torch.cos(2 * m * math.pi * x[..., 0] / ext[0]) * torch.cos(math.pi * x[..., 1] / ext[1])
                            * torch.cos(2 * math.pi * x[..., 2] / ext[2]) for a, m in zip(AMP, MX)])
    return f


def strong_operator(x, fields, p):
    """-div(F - A grad u) + S at points x (..., d), by automatic differentiation."""
    pv = O.param_vector(p)
    d = x.shape[-1]
    x = x.detach().clone().requires_grad_(True)
    u = fields(x)
    g = torch.stack([torch.autograd.grad(u[s].sum(), x, create_graph=True)[0].movedim(-1, 0) for s in range(6)])
    Phi = O.flux_F(u, g, pv) - O.diffusivity(pv)[:, None, None, None] * g
    div = torch.stack([sum(torch.autograd.grad(Phi[s, j].sum(), x, retain_graph=True)[0][..., j] for j in range(d))
                       for s in range(6)])
    return (-div + O.source_S(u, pv)).detach()


def relative_error(mod, mesh, fields, p):
    """||M^{-1} L_h(P u) - P L(u)|| / ||P L(u)|| in the L2 norm of V_h."""
    U = mod.project(mesh, fields)
    PL = mod.project(mesh, lambda x: strong_operator(x, fields, p))
    diff = mod.apply(mesh, U, p) - PL

    def norm(V):
        if isinstance(mesh, O.Mesh):
            return float(mesh.vol * (V ** 2).sum()) ** 0.5      # Cartesian cells: M_K = |K| I
        return float(torch.einsum("esi,eij,esj->", V, mesh.mass, V)) ** 0.5

    return norm(diff) / norm(PL)


@pytest.mark.parametrize("k,min_rate", [(2, 0.8), (3, 1.6)])
def test_triangle_operator_is_consistent_with_the_strong_form(k, min_rate):
    ext = (1.0, 0.2)
    p = params()
    errs = []
    for n in (4, 8):
        xy, tri = I.tri_mesh(4 * n, n, ext[0], ext[1], 0.1, 7)
        errs.append(relative_error(T, T.TriMesh(xy, tri, k), walled_fields(ext), p))
    rate = math.log2(errs[0] / errs[1])
    assert rate >= min_rate, (errs, rate)      # measured: 1.01 (k = 2), 1.94 (k = 3)
    assert errs[1] < 0.2


def test_tetrahedral_operator_is_consistent_with_the_strong_form():
    ext = (0.2, 0.2, 0.2)
    p = params()
    errs = []
    for n in (2, 4):
        xyz, tet = I.tet_mesh(n, n, n, ext[0], ext[1], ext[2], 0.1, 7)
        errs.append(relative_error(TT, TT.TetMesh(xyz, tet, 3), walled_fields(ext), p))
    rate = math.log2(errs[0] / errs[1])
    assert rate >= 1.3, (errs, rate)           # measured: 1.67 at these (pre-asymptotic) sizes, k = 3
    assert errs[1] < 0.3


@pytest.mark.parametrize("k,min_rate", [(2, 0.8), (3, 1.8)])
def test_hexahedral_operator_is_consistent_with_the_strong_form(k, min_rate):
    ext = (0.4, 0.2, 0.2)
    p = params()
    errs = []
    for n in (4, 8):
        mesh = O.Mesh(3, (2 * n, n, n), ext, (True, False, True), k)
        errs.append(relative_error(O, mesh, periodic_xz_fields(ext), p))
    rate = math.log2(errs[0] / errs[1])
    assert rate >= min_rate, (errs, rate)      # measured: 0.95 (k = 2), 2.53 (k = 3)
    assert errs[1] < 0.2
