"""Plain FP64 CPU oracle of the CDG2 operator L_h on triangle meshes.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and does not import it; the mesh comes from
``cdg2_inputs.tri_mesh`` or is given explicitly.

What it computes, with the passages it follows:
  * the DG space of Sec. 3.1 with P_k(K) on triangles (the paper's 2D runs
    use triangles): on the reference triangle T = {xi, eta >= 0, xi + eta <= 1}
    the orthonormal Dubiner basis (Reading: the paper names no basis; any
    orthonormal one gives the diagonal mass matrix Sec. 3.2 mentions),
    mapped affinely to each element;
  * L_h = K_h + I_h (Eq. convDiscr) with the same element and surface
    integrals as on Cartesian meshes (the model functions come from
    ``cdg2_oracle``): the local Lax-Friedrichs flux and the CDG2 flux
    2 chi_e (A r_e([U]))|_{K^-_e}, chi_e = 1.5 for triangles (Sec. 3.1),
    K^-_e the adjacent element with the smaller area (Sec. 3.1; Reading:
    areas within a relative 1e-12 tie, and a tie goes to the lower element
    index), the lifting r_e from its
    variational identity solved with the element's quadrature mass matrix;
  * boundary faces: the influxes of Eq. (3) on y = 0 (Gamma_1) and on
    y = L_1 (Gamma_2); Reading: every other boundary edge (the side walls of
    the rectangle; triangle meshes are not periodic here) is no-flow;
  * f = M^{-1} L_h with the quadrature mass matrix and a dense solve, and
    the derivatives by torch.func automatic differentiation;
  * one SDIRK step of U' = f(U) (Sec. 3.2: a DIRK method, each stage by
    Newton's method): the tableaux of ``cdg2_oracle.sdirk_tableau``, each
    Newton correction by a dense Jacobian and LU on small meshes, by GMRES
    with the JVP otherwise.

Readings of the quadrature (the paper gives none): volume integrals by the
collapsed (Duffy) Gauss-Legendre rule with (k+2)^2 points -- Gauss points
u_i, v_j on [0,1], xi = u (1 - v), eta = v, weight w_i w_j (1 - v), u fastest
-- and k+2 Gauss points per edge.  Everything is dense and unfused.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from oracle import cdg2_oracle as O

F64 = torch.float64
N_SPECIES = 6


# ----------------------------------------------------------------------------
# Basis and quadrature on the reference triangle
# ----------------------------------------------------------------------------
def jacobi(n: int, alpha: float, x):
    """Jacobi polynomial P_n^{(alpha, 0)}(x) by the three-term recurrence
    (DLMF 18.9.1 with beta = 0)."""
    p0 = torch.ones_like(x)
    if n == 0:
        return p0
    p1 = (alpha + 1.0) + (alpha + 2.0) * (x - 1.0) / 2.0
    for m in range(2, n + 1):
        c = 2 * m + alpha
        a1 = 2.0 * m * (m + alpha) * (c - 2.0)
        a2 = (c - 1.0) * c * (c - 2.0)
        a3 = (c - 1.0) * alpha * alpha
        a4 = 2.0 * (m + alpha - 1.0) * (m - 1.0) * c
        p0, p1 = p1, ((a2 * x + a3) * p1 - a4 * p0) / a1
    return p1


def modes(k: int):
    """Mode (p, q) of basis index i: ordered by total degree p + q, then by q."""
    return [(d - q, q) for d in range(k + 1) for q in range(d + 1)]


def dubiner(k: int, pts):
    """psi_i(xi, eta) = c_pq L_p(xi, eta) P_q^{(2p+1,0)}(2 eta - 1) on T, where
    L_p = (1 - eta)^p P_p(2 xi / (1 - eta) - 1) (the Legendre polynomial in the
    collapsed coordinate, a polynomial in xi, eta) and c_pq = sqrt(2 (2p+1)
    (p+q+1)) makes the basis orthonormal on T.  pts: (P, 2).  Returns
    psi (P, nb) and its reference gradient (2, P, nb) (autograd)."""
    pts = pts.detach().clone().requires_grad_(True)
    xi, eta = pts[:, 0], pts[:, 1]
    s = 1.0 - eta
    xt = 2.0 * xi - s
    # L_p by the Legendre recurrence scaled by s^p: L_p = ((2p-1) xt L_{p-1} - (p-1) s^2 L_{p-2}) / p
    L = [torch.ones_like(xi), xt]
    for p in range(2, k + 1):
        L.append(((2 * p - 1) * xt * L[p - 1] - (p - 1) * s * s * L[p - 2]) / p)
    cols = []
    for p, q in modes(k):
        c = math.sqrt(2.0 * (2 * p + 1) * (p + q + 1))
        cols.append(c * L[p] * jacobi(q, 2.0 * p + 1.0, 2.0 * eta - 1.0))
    grads = []
    for col in cols:
        if not col.requires_grad:          # the constant mode
            grads.append(torch.zeros_like(pts))
            continue
        (g,) = torch.autograd.grad(col.sum(), pts, retain_graph=True)
        grads.append(g)
    psi = torch.stack([c.detach() for c in cols], dim=1)
    dpsi = torch.stack(grads, dim=2).permute(1, 0, 2).contiguous()   # (2, P, nb)
    return psi, dpsi


def triangle_rule(n: int):
    """Collapsed Gauss-Legendre rule on T with n^2 points (u fastest)."""
    g, w = O.gauss_legendre01(n)
    pts, wts = [], []
    for j in range(n):
        for i in range(n):
            u, v = float(g[i]), float(g[j])
            pts.append((u * (1.0 - v), v))
            wts.append(float(w[i]) * float(w[j]) * (1.0 - v))
    return torch.tensor(pts, dtype=F64), torch.tensor(wts, dtype=F64)


# ----------------------------------------------------------------------------
# Mesh
# ----------------------------------------------------------------------------
class TriMesh:
    """Affine triangles from vertex coordinates xy (n_v, 2) and counter-
    clockwise vertex triples tri (E, 3).  Element e maps the reference
    triangle by x = x_0 + J_e (xi, eta), J_e = [x_1 - x_0, x_2 - x_0]; its
    basis is phi_i = psi_i o F_e^{-1}.  Local edge l runs from vertex l to
    vertex l + 1 (mod 3).
    """

    def __init__(self, xy, tri, k: int, chi_e: float = 1.5, gamma1_in=(0.375, 0.625)):
        self.xy = torch.as_tensor(np.asarray(xy), dtype=F64)
        self.tri = torch.as_tensor(np.asarray(tri), dtype=torch.long)
        self.k = int(k)
        self.dim = 2
        self.periodic = (False, False)       # Reading: triangle meshes are not periodic here
        self.chi_e = float(chi_e)
        self.gamma1_in = tuple(gamma1_in)
        self.E = self.tri.shape[0]
        self.nb = (self.k + 1) * (self.k + 2) // 2
        self.ly = float(self.xy[:, 1].max())
        x = self.xy[self.tri]                                    # (E, 3, 2)
        self.x0 = x[:, 0]
        self.J = torch.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]], dim=-1)   # columns
        self.det = torch.linalg.det(self.J)
        if not bool((self.det > 0).all()):
            raise ValueError("every triangle must be non-degenerate and counter-clockwise")
        self.Jinv = torch.linalg.inv(self.J)
        self.area = 0.5 * self.det
        # volume rule and tabulation
        self.qpts, self.qw = triangle_rule(self.k + 2)
        self.phi, self.dphi = dubiner(self.k, self.qpts)
        # M_K = int_K phi_i phi_j = det J_e sum_q w_q psi_i psi_j
        self.mass = self.det[:, None, None] * torch.einsum("q,qi,qj->ij", self.qw, self.phi, self.phi)[None]
        g, w = O.gauss_legendre01(self.k + 2)
        self.et = g.to(F64)
        self.ew = w.to(F64)
        # edges: interior (K^-, K^+) and boundary
        edges = {}
        for e in range(self.E):
            for l in range(3):
                a, b = int(self.tri[e, l]), int(self.tri[e, (l + 1) % 3])
                edges.setdefault((min(a, b), max(a, b)), []).append((e, l))
        self.interior, self.boundary = [], []
        tol = 1e-12 * max(1.0, self.ly)
        for key, owners in sorted(edges.items()):
            if len(owners) == 2:
                (e1, l1), (e2, l2) = owners
                a1, a2 = float(self.area[e1]), float(self.area[e2])
                # K^- = the smaller element; Reading: areas within a relative 1e-12
                # are a tie (triangles on one boundary line sharing an apex tie
                # exactly), and a tie goes to the lower index
                tie = abs(a1 - a2) <= 1e-12 * max(a1, a2)
                if (not tie and a1 < a2) or (tie and e1 < e2):
                    self.interior.append((e1, l1, e2, l2))
                else:
                    self.interior.append((e2, l2, e1, l1))
            elif len(owners) == 1:
                e, l = owners[0]
                ya, yb = float(self.xy[key[0], 1]), float(self.xy[key[1], 1])
                if abs(ya) <= tol and abs(yb) <= tol:
                    tag = 1
                elif abs(ya - self.ly) <= tol and abs(yb - self.ly) <= tol:
                    tag = 2
                else:
                    tag = 0
                self.boundary.append((e, l, tag))
            else:
                raise ValueError("an edge is shared by more than two triangles")
        # tabulations at the edge points (geometry only), computed once
        self.iface = []
        for eM, lM, eP, lP in self.interior:
            x, n, length = self.edge_geometry(eM, lM)
            psiM, dM = dubiner(self.k, self.ref_coords(eM, x))
            psiP, dP = dubiner(self.k, self.ref_coords(eP, x))
            self.iface.append((eM, eP, x, n, length, psiM, self.phys_grad(eM, dM), psiP, self.phys_grad(eP, dP)))
        self.bface = []
        for e, l, tag in self.boundary:
            x, n, length = self.edge_geometry(e, l)
            self.bface.append((e, tag, x, length, dubiner(self.k, self.ref_coords(e, x))[0]))

    def edge_geometry(self, e: int, l: int):
        """Points (P, 2), unit outward normal, length of local edge l of e."""
        A = self.xy[self.tri[e, l]]
        B = self.xy[self.tri[e, (l + 1) % 3]]
        d = B - A
        length = float(torch.linalg.norm(d))
        n = torch.tensor([d[1], -d[0]], dtype=F64) / length
        pts = A[None, :] + self.et[:, None] * d[None, :]
        return pts, n, length

    def ref_coords(self, e: int, x):
        """Reference coordinates of physical points x (P, 2) in element e."""
        return (x - self.x0[e][None, :]) @ self.Jinv[e].T

    def phys_grad(self, e: int, dpsi):
        """Physical gradients J_e^{-T} grad_ref of tabulated reference gradients (2, P, nb)."""
        return torch.einsum("mj,mpi->jpi", self.Jinv[e], dpsi)

    def qpoints_phys(self):
        """Physical volume quadrature points (E, Q, 2)."""
        return self.x0[:, None, :] + torch.einsum("ejm,qm->eqj", self.J, self.qpts)


# ----------------------------------------------------------------------------
# The operator L_h (Sec. 3.1) and f = M^{-1} L_h (Sec. 3.2)
# ----------------------------------------------------------------------------
def volume_residual(mesh: TriMesh, U, p):
    """Element integrals of Eq. elementint: int_K (F - A grad U) : grad phi + S . phi."""
    G = torch.einsum("emj,mqi->ejqi", mesh.Jinv, mesh.dphi)        # physical gradients (E, 2, Q, nb)
    uq = torch.einsum("qi,esi->seq", mesh.phi, U)
    gq = torch.einsum("ejqi,esi->sjeq", G, U)
    A = O.diffusivity(p)
    Phi = O.flux_F(uq, gq, p) - A[:, None, None, None] * gq         # (6, 2, E, Q)
    S = O.source_S(uq, p)                                          # (6, E, Q)
    W = mesh.det[:, None] * mesh.qw[None, :]                        # (E, Q)
    R = torch.einsum("eq,sjeq,ejqi->esi", W, Phi, G)
    return R + torch.einsum("eq,seq,qi->esi", W, S, mesh.phi)


def _traces(psi, grad, Ue):
    """Values (6, P) and physical gradients (6, 2, P) of one element's field at
    tabulated points."""
    return (psi @ Ue.T).T, torch.einsum("jpi,si->sjp", grad, Ue)


def lifting_normal(mass, psiM, Delta, n, length, w):
    """r_e([U]) . n^- at the edge points, r_e on K^- only (the lifting identity
    of Sec. 3.1): int_Omega r_e : tau = -int_e [U] : {tau}; on K^- with
    [U] = n^- (x) Delta and {tau} = tau_{K^-} / 2 this is
    M_{K^-} rho_{s,j} = -1/2 int_e n_j Delta_s phi_i.  Delta: (6, P)."""
    rhs = -0.5 * length * torch.einsum("p,j,sp,pi->sji", w, n, Delta, psiM)     # (6, 2, nb)
    rho = torch.linalg.solve(mass, rhs.reshape(-1, rhs.shape[-1]).T).T.reshape(rhs.shape)
    return torch.einsum("j,pi,sji->sp", n, psiM, rho)


def face_residual(mesh: TriMesh, U, p):
    """Surface integrals of Eq. surfaceint on interior edges, as on Cartesian
    meshes (see cdg2_oracle.face_residual) with n^- the outward unit normal of
    K^-, Delta = U^- - U^+, LLF with lambda_s = max(|v^-.n|, |v^+.n|) (a tie
    takes K^-), and A^ = 2 chi_e A r_e([U]) on K^-."""
    R = torch.zeros_like(U)
    A = O.diffusivity(p)
    for eM, eP, x, n, length, psiM, gradM, psiP, gradP in mesh.iface:
        W = length * mesh.ew
        UM, GM = _traces(psiM, gradM, U[eM])
        UP, GP = _traces(psiP, gradP, U[eP])
        Delta = UM - UP                                            # (6, P)
        dnM = torch.einsum("j,jpi->pi", n, gradM)
        dnP = torch.einsum("j,jpi->pi", n, gradP)
        avg_dn = 0.5 * torch.einsum("j,sjp->sp", n, GM + GP)
        FnM = torch.einsum("j,sjp->sp", n, O.flux_F(UM, GM, p))
        FnP = torch.einsum("j,sjp->sp", n, O.flux_F(UP, GP, p))
        v1M, v2M = O.velocity(UM, GM, p)
        v1P, v2P = O.velocity(UP, GP, p)
        lam = []
        for vM, vP in ((v1M, v1P), (v2M, v2P)):
            aM = torch.einsum("j,jp->p", n, vM).abs()
            aP = torch.einsum("j,jp->p", n, vP).abs()
            lam.append(torch.where(aM >= aP, aM, aP))
        lam = torch.stack(lam + [torch.zeros_like(lam[0])] * 4)
        Fhat_n = 0.5 * (FnM + FnP) + 0.5 * lam * Delta
        rn = lifting_normal(mesh.mass[eM], psiM, Delta, n, length, mesh.ew)
        Ahat_n = 2.0 * mesh.chi_e * A[:, None] * rn
        sigma = A[:, None] * avg_dn - Fhat_n + Ahat_n              # multiplies phi^- - phi^+
        tau = 0.5 * A[:, None] * Delta                             # multiplies dn phi^- + dn phi^+
        RM = torch.einsum("p,sp,pi->si", W, sigma, psiM) + torch.einsum("p,sp,pi->si", W, tau, dnM)
        RP = -torch.einsum("p,sp,pi->si", W, sigma, psiP) + torch.einsum("p,sp,pi->si", W, tau, dnP)
        R = R.index_add(0, torch.tensor([eM]), RM[None])
        R = R.index_add(0, torch.tensor([eP]), RP[None])
    return R


def boundary_residual(mesh: TriMesh, U, p):
    """Boundary edges: the influxes of Eq. (3) times bc_sign on Gamma_1 (y = 0;
    n1: mu1 beta1 H(c1 - c1*), c2: nu2 sigma on Gamma_{1,in}) and Gamma_2
    (y = L_1; n2: mu2 beta2 H(c1 - c1**)); no flow elsewhere."""
    R = torch.zeros_like(U)
    for e, tag, x, length, psi in mesh.bface:
        if tag == 0:
            continue
        u = (psi @ U[e].T).T
        z = torch.zeros_like(u[0])
        if tag == 1:
            inside = ((x[:, 0] >= mesh.gamma1_in[0]) & (x[:, 0] <= mesh.gamma1_in[1])).to(F64)
            g0 = p["bc_sign"] * p["mu"][0] * p["beta1"] * O.heaviside(u[3] - p["c1_star"])
            g4 = p["bc_sign"] * p["nu"][1] * p["sigma"] * inside
            if O.reduced(p):
                g4 = torch.zeros_like(g4)
            g = torch.stack([g0, z, z, z, g4, z])
        else:
            g1 = p["bc_sign"] * p["mu"][1] * p["beta2"] * O.heaviside(u[3] - p["c1_star2"])
            if O.reduced(p):
                g1 = torch.zeros_like(g1)
            g = torch.stack([z, g1, z, z, z, z])
        R = R.index_add(0, torch.tensor([e]), torch.einsum("p,sp,pi->si", length * mesh.ew, g, psi)[None])
    return R


def apply_residual(mesh: TriMesh, U, p):
    """<phi, L_h(U)> for every basis function (no M^{-1})."""
    return volume_residual(mesh, U, p) + face_residual(mesh, U, p) + boundary_residual(mesh, U, p)


def minv(mesh: TriMesh, R):
    """M^{-1} with each element's quadrature mass matrix (dense solve)."""
    return torch.linalg.solve(mesh.mass, R.transpose(1, 2)).transpose(1, 2)


def apply(mesh: TriMesh, U, params: dict):
    """f(U) = M^{-1} L_h(U) (Eq. ode): U, result (E, 6, nb) float64."""
    p = O.param_vector(params)
    return minv(mesh, apply_residual(mesh, U, p))


def jvp(mesh: TriMesh, U, dU, params: dict):
    """J(U) dU by torch.func forward mode."""
    return torch.func.jvp(lambda V: apply(mesh, V, params), (U,), (dU,))[1]


def vjp(mesh: TriMesh, U, lam, params: dict):
    """J(U)^T lam by torch.func reverse mode."""
    _, fn = torch.func.vjp(lambda V: apply(mesh, V, params), U)
    return fn(lam)[0]


def project(mesh: TriMesh, func):
    """L2 projection onto V_h (Sec. 3.2) with the volume rule; func(x) -> (6, E, Q)."""
    fx = func(mesh.qpoints_phys())
    R = torch.einsum("eq,seq,qi->esi", mesh.det[:, None] * mesh.qw[None, :], fx, mesh.phi)
    return minv(mesh, R)


def step(mesh: TriMesh, U, params: dict, dt: float, scheme="sdirk2", newton_tol=1e-13, gmres_tol=1e-13,
         max_newton=30):
    """One SDIRK step U_n -> U_{n+1} of U' = f(U) = M^{-1} L_h(U) (Sec. 3.2).

    Stage i solves Y_i - dt a_ii f(Y_i) = U_n + dt sum_{j<i} a_ij K_j by Newton's
    method from the previous stage value (correction: (I - dt a_ii J(Y)) d = -G),
    until ||G||_2 <= newton_tol max(1, ||rhs_i||_2); K_i = f(Y_i) and
    U_{n+1} = U_n + dt sum_i b_i K_i.  Works on any mesh these residuals accept
    (triangles or tetrahedra)."""
    A, b, _ = O.sdirk_tableau(scheme)
    n = U.numel()
    K = []
    Y = U.clone()
    for i in range(len(b)):
        rhs = U.clone()
        for j in range(i):
            rhs = rhs + dt * A[i, j] * K[j]
        gdt = dt * A[i, i]
        scale = max(1.0, float(torch.linalg.norm(rhs)))
        for _it in range(max_newton):
            G = Y - gdt * apply(mesh, Y, params) - rhs
            if float(torch.linalg.norm(G)) <= newton_tol * scale:
                break
            if n <= 3000:
                Jd = torch.func.jacfwd(lambda V: apply(mesh, V, params))(Y).reshape(n, n)
                d = torch.linalg.solve(torch.eye(n, dtype=F64) - gdt * Jd, -G.reshape(-1)).reshape(Y.shape)
            else:
                d = O._gmres(lambda v: v - gdt * jvp(mesh, Y, v, params), -G, gmres_tol)
            Y = Y + d
        else:
            raise RuntimeError("oracle Newton did not converge")
        K.append(apply(mesh, Y, params))
    out = U.clone()
    for i in range(len(b)):
        out = out + dt * b[i] * K[i]
    return out
