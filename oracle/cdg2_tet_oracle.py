"""Plain FP64 CPU oracle of the CDG2 operator L_h on tetrahedral meshes.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and does not import it.

What it computes, with the passages it follows (the element and surface
integrals are the triangle oracle's, written for any dimension; this module
supplies the tetrahedral space and geometry):
  * P_k(K) on tetrahedra (Sec. 3.1: the paper's 3D runs use tetrahedra, with
    chi_e = 2): on the reference tetrahedron T = {xi, eta, zeta >= 0,
    xi + eta + zeta <= 1} the orthonormal Dubiner basis (Reading, as for
    triangles: the paper names no basis)
        psi_pqr = c_pqr L_p(xi; s) J_q^{2p+1}(eta; t) P_r^{(2p+2q+2,0)}(2 zeta - 1),
    s = 1 - eta - zeta, t = 1 - zeta, L_p = s^p P_p((2 xi - s) / s) and
    J_q^a = t^q P_q^{(a,0)}((2 eta - t) / t) (polynomials by their scaled
    recurrences), c_pqr = sqrt((2p+1)(2p+2q+2)(2p+2q+2r+3)); modes ordered by
    total degree, then r, then q; mapped affinely, M_K = det J_e I;
  * K^-_e the adjacent tetrahedron with the smaller volume (Sec. 3.1; areas
    within a relative 1e-12 tie, a tie goes to the lower index);
  * boundary faces on y = 0 (Gamma_1) and y = max y (Gamma_2) carry the data of
    Eq. (3); every other boundary face is a no-flow wall; no periodicity.
Readings of the quadrature: volume by the collapsed Gauss rule with (k+2)^3
points (xi = u (1-v)(1-w), eta = v (1-w), zeta = w, weight w_u w_v w_w (1-v)
(1-w)^2, u fastest); each face by the collapsed triangle rule with (k+2)^2
points in K^-'s parametrisation of the face (local face l is the one without
local vertex l, its vertices in increasing local order).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from oracle import cdg2_oracle as O
from oracle import cdg2_tri_oracle as T

F64 = torch.float64

FACE_VERTS = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))   # local face l: the vertices other than l


def modes(k: int):
    """Mode (p, q, r) of basis index i: by total degree, then r, then q."""
    return [(d - q - r, q, r) for d in range(k + 1) for r in range(d + 1) for q in range(d - r + 1)]


def _scaled_jacobi(n: int, alpha: float, y, t):
    """t^n P_n^{(alpha,0)}(y / t) by the recurrence of DLMF 18.9.1 scaled by t^n."""
    j0 = torch.ones_like(y)
    if n == 0:
        return j0
    j1 = (alpha + 1.0) * t + (alpha + 2.0) * (y - t) / 2.0
    for m in range(2, n + 1):
        c = 2 * m + alpha
        a1 = 2.0 * m * (m + alpha) * (c - 2.0)
        a2 = (c - 1.0) * c * (c - 2.0)
        a3 = (c - 1.0) * alpha * alpha
        a4 = 2.0 * (m + alpha - 1.0) * (m - 1.0) * c
        j0, j1 = j1, ((a2 * y + a3 * t) * j1 - a4 * t * t * j0) / a1
    return j1


def dubiner3(k: int, pts):
    """psi_i and its reference gradient (3, P, nb) (autograd) at pts (P, 3)."""
    pts = pts.detach().clone().requires_grad_(True)
    xi, eta, zeta = pts[:, 0], pts[:, 1], pts[:, 2]
    s = 1.0 - eta - zeta
    t = 1.0 - zeta
    L = [torch.ones_like(xi), 2.0 * xi - s]
    for p in range(2, k + 1):
        L.append(((2 * p - 1) * (2.0 * xi - s) * L[p - 1] - (p - 1) * s * s * L[p - 2]) / p)
    cols = []
    for p, q, r in modes(k):
        c = math.sqrt((2 * p + 1) * (2 * p + 2 * q + 2) * (2 * p + 2 * q + 2 * r + 3))
        cols.append(c * L[p] * _scaled_jacobi(q, 2.0 * p + 1.0, 2.0 * eta - t, t)
                    * T.jacobi(r, 2.0 * p + 2.0 * q + 2.0, 2.0 * zeta - 1.0))
    grads = []
    for col in cols:
        if not col.requires_grad:          # the constant mode
            grads.append(torch.zeros_like(pts))
            continue
        (g,) = torch.autograd.grad(col.sum(), pts, retain_graph=True)
        grads.append(g)
    psi = torch.stack([c.detach() for c in cols], dim=1)
    return psi, torch.stack(grads, dim=2).permute(1, 0, 2).contiguous()


def tet_rule(n: int):
    """Collapsed Gauss-Legendre rule on T with n^3 points (u fastest, then v, w)."""
    g, w = O.gauss_legendre01(n)
    pts, wts = [], []
    for c in range(n):
        for b in range(n):
            for a in range(n):
                u, v, ww = float(g[a]), float(g[b]), float(g[c])
                pts.append((u * (1.0 - v) * (1.0 - ww), v * (1.0 - ww), ww))
                wts.append(float(w[a]) * float(w[b]) * float(w[c]) * (1.0 - v) * (1.0 - ww) ** 2)
    return torch.tensor(pts, dtype=F64), torch.tensor(wts, dtype=F64)


class TetMesh:
    """Affine tetrahedra from vertex coordinates xyz (n_v, 3) and positively
    oriented vertex quadruples tet (E, 4); element e maps T by x = x_0 + J_e xi,
    J_e = [x_1 - x_0, x_2 - x_0, x_3 - x_0].  Provides the attributes the
    dimension-generic residuals of cdg2_tri_oracle read."""

    def __init__(self, xyz, tet, k: int, chi_e: float = 2.0, gamma1_in=(0.375, 0.625)):
        self.xy = torch.as_tensor(np.asarray(xyz), dtype=F64)
        self.tri = torch.as_tensor(np.asarray(tet), dtype=torch.long)
        self.k = int(k)
        self.dim = 3
        self.periodic = (False, False, False)
        self.chi_e = float(chi_e)
        self.gamma1_in = tuple(gamma1_in)
        self.E = self.tri.shape[0]
        self.nb = (self.k + 1) * (self.k + 2) * (self.k + 3) // 6
        self.ly = float(self.xy[:, 1].max())
        x = self.xy[self.tri]                                    # (E, 4, 3)
        self.x0 = x[:, 0]
        self.J = torch.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], dim=-1)
        self.det = torch.linalg.det(self.J)
        if not bool((self.det > 0).all()):
            raise ValueError("every tetrahedron must be non-degenerate and positively oriented")
        self.Jinv = torch.linalg.inv(self.J)
        self.area = self.det / 6.0                               # the element volume
        self.qpts, self.qw = tet_rule(self.k + 2)
        self.phi, self.dphi = dubiner3(self.k, self.qpts)
        self.mass = self.det[:, None, None] * torch.einsum("q,qi,qj->ij", self.qw, self.phi, self.phi)[None]
        self.fpts, self.ew = T.triangle_rule(self.k + 2)         # face rule (weights sum to 1/2)
        faces = {}
        for e in range(self.E):
            for l in range(4):
                key = tuple(sorted(int(self.tri[e, v]) for v in FACE_VERTS[l]))
                faces.setdefault(key, []).append((e, l))
        self.interior, self.boundary = [], []
        tol = 1e-12 * max(1.0, self.ly)
        for key, own in sorted(faces.items()):
            if len(own) == 2:
                (e1, l1), (e2, l2) = own
                v1, v2 = float(self.area[e1]), float(self.area[e2])
                tie = abs(v1 - v2) <= 1e-12 * max(v1, v2)
                if (not tie and v1 < v2) or (tie and e1 < e2):
                    self.interior.append((e1, l1, e2, l2))
                else:
                    self.interior.append((e2, l2, e1, l1))
            elif len(own) == 1:
                e, l = own[0]
                ys = [float(self.xy[v, 1]) for v in key]
                tag = 1 if all(abs(y) <= tol for y in ys) else (2 if all(abs(y - self.ly) <= tol for y in ys) else 0)
                self.boundary.append((e, l, tag))
            else:
                raise ValueError("a face is shared by more than two tetrahedra")
        self.iface = []
        for eM, lM, eP, lP in self.interior:
            x, n, E2 = self.face_geometry(eM, lM)
            psiM, dM = dubiner3(self.k, self.ref_coords(eM, x))
            psiP, dP = dubiner3(self.k, self.ref_coords(eP, x))
            self.iface.append((eM, eP, x, n, E2, psiM, self.phys_grad(eM, dM), psiP, self.phys_grad(eP, dP)))
        self.bface = []
        for e, l, tag in self.boundary:
            x, n, E2 = self.face_geometry(e, l)
            self.bface.append((e, tag, x, E2, dubiner3(self.k, self.ref_coords(e, x))[0]))

    def face_geometry(self, e: int, l: int):
        """Points (P, 3) of face l of e in its parametrisation A + s (B - A) + t (C - A),
        the unit normal out of e, and |(B - A) x (C - A)| (the face rule's Jacobian)."""
        A, B, C = (self.xy[self.tri[e, v]] for v in FACE_VERTS[l])
        cr = torch.linalg.cross(B - A, C - A)
        E2 = float(torch.linalg.norm(cr))
        n = cr / E2
        opp = self.xy[self.tri[e, l]]
        if float(n @ (opp - A)) > 0:
            n = -n
        pts = A[None] + self.fpts[:, :1] * (B - A)[None] + self.fpts[:, 1:] * (C - A)[None]
        return pts, n, E2

    def ref_coords(self, e: int, x):
        return (x - self.x0[e][None, :]) @ self.Jinv[e].T

    def phys_grad(self, e: int, dpsi):
        return torch.einsum("mj,mpi->jpi", self.Jinv[e], dpsi)

    def qpoints_phys(self):
        return self.x0[:, None, :] + torch.einsum("ejm,qm->eqj", self.J, self.qpts)


def apply_residual(mesh: TetMesh, U, p):
    return T.apply_residual(mesh, U, p)


def apply(mesh: TetMesh, U, params: dict):
    """f(U) = M^{-1} L_h(U) on the tetrahedral mesh."""
    return T.apply(mesh, U, params)


def jvp(mesh: TetMesh, U, dU, params: dict):
    return T.jvp(mesh, U, dU, params)


def vjp(mesh: TetMesh, U, lam, params: dict):
    return T.vjp(mesh, U, lam, params)


def project(mesh: TetMesh, func):
    return T.project(mesh, func)


def step(mesh: TetMesh, U, params: dict, dt: float, scheme="sdirk2", **kw):
    """One SDIRK step of U' = M^{-1} L_h(U) on the tetrahedral mesh (Sec. 3.2)."""
    return T.step(mesh, U, params, dt, scheme, **kw)
