"""Plain FP64 CPU oracle of the CDG2 operator L_h for the six-species model.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and does not import it; both sides take their seeded
inputs from ``cdg2_inputs``.

What it computes, with the passages it follows:
  * the model of Sec. 2: Eq. (1) (six species), the tactic sensitivity
    chi(x, y, a, b) = a x / (y + b), the compact form dU/dt = -div(F(U) -
    A grad U) + S(U), and the boundary data of Eq. (3);
  * the DG space of Sec. 3.1 on uniform Cartesian cells with the tensor
    Legendre basis psi_m(xi) = sqrt(2m+1) P_m(2 xi - 1) (orthonormal on the
    unit cell), Gauss-Legendre quadrature with q1 points per direction;
  * L_h = K_h + I_h (Eq. convDiscr): element integrals (Eq. elementint),
    surface integrals with the symmetric average/jump terms, the local
    Lax-Friedrichs convective flux and the CDG2 diffusion flux
    2 chi_e (A r_e([U]))|_{K^-_e} with the lifting r_e defined by its
    variational identity (Eq. surfaceint and the lifting definition);
  * the ODE U' = M^{-1} L_h(U) (Eq. ode) with the element mass matrix built
    by quadrature and inverted by a dense solve (no orthonormality shortcut);
  * the linearisation J(U) dU and its transpose via torch.func automatic
    differentiation of the same code (the definition of the derivative);
  * SDIRK time stepping with Newton and GMRES (Sec. 3.2);
  * the experimental order of convergence of Table 1 (Sec. 4), pinned to
    the paper's printed column.

Everything is evaluated densely: full tensor-product tabulation matrices,
no sum factorisation, no fusion.  Readings where the paper is silent are
marked "Reading:" in the docstrings.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import torch

F64 = torch.float64
N_SPECIES = 6


# ----------------------------------------------------------------------------
# 1D building blocks (Sec. 3.1: P_k per species; orthonormal basis gives the
# diagonal mass matrix mentioned in Sec. 3.2)
# ----------------------------------------------------------------------------
def gauss_legendre01(n: int):
    """n-point Gauss-Legendre rule on [0, 1] (points, weights summing to 1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return torch.tensor((x + 1.0) / 2.0, dtype=F64), torch.tensor(w / 2.0, dtype=F64)


def legendre01(k: int, xi: torch.Tensor):
    """psi_m(xi) = sqrt(2m+1) P_m(2 xi - 1) and d psi_m / d xi for m = 0..k.

    Bonnet recurrence (m+1) P_{m+1} = (2m+1) t P_m - m P_{m-1} and
    P'_{m+1} = P'_{m-1} + (2m+1) P_m.  Returns two (k+1, npts) tensors.
    """
    t = 2.0 * xi - 1.0
    P = [torch.ones_like(t), t]
    dP = [torch.zeros_like(t), torch.ones_like(t)]
    for m in range(1, k):
        P.append(((2 * m + 1) * t * P[m] - m * P[m - 1]) / (m + 1))
        dP.append(dP[m - 1] + (2 * m + 1) * P[m])
    psi = torch.stack([math.sqrt(2 * m + 1) * P[m] for m in range(k + 1)])
    dpsi = torch.stack([2.0 * math.sqrt(2 * m + 1) * dP[m] for m in range(k + 1)])
    return psi, dpsi


def multi_indices(n: int, dim: int):
    """Lexicographic multi-indices (x fastest) of an n^dim tensor grid."""
    return [tuple(reversed(t)) for t in itertools.product(range(n), repeat=dim)]


def tabulate(k: int, pts: torch.Tensor):
    """Tensor basis phi_i and its reference gradient at reference points.

    pts: (P, dim) coordinates in the unit cell.  Returns phi (P, nb) and
    dphi (dim, P, nb) with dphi[j] = d phi / d xi_j.
    """
    P, dim = pts.shape
    psi, dpsi = zip(*[legendre01(k, pts[:, j]) for j in range(dim)])
    idx = multi_indices(k + 1, dim)
    phi = torch.ones(P, len(idx), dtype=F64)
    dphi = torch.ones(dim, P, len(idx), dtype=F64)
    for i, a in enumerate(idx):
        for j in range(dim):
            phi[:, i] = phi[:, i] * psi[j][a[j]]
            for l in range(dim):
                dphi[l, :, i] = dphi[l, :, i] * (dpsi[j][a[j]] if l == j else psi[j][a[j]])
    return phi, dphi


# ----------------------------------------------------------------------------
# Mesh: uniform Cartesian cells (Reading: Q_k on quads/hexes replaces P_k on
# triangles/tets; the structured box replaces the paper's unstructured mesh)
# ----------------------------------------------------------------------------
class Mesh:
    """Uniform Cartesian mesh of the box [0, L_0] x ... with Q_k elements.

    Elements are numbered lexicographically, x fastest.  Axis 1 (y) carries
    the boundaries of Eq. (3) when it is not periodic: y = 0 is Gamma_1 (the
    lumen side), y = L_1 is Gamma_2 (the outer wall); Gamma_{1,in} is the
    part of Gamma_1 with gamma1_in[0] <= x <= gamma1_in[1] (Reading: the
    paper leaves the subset open).  Other non-periodic sides are no-flow.

    chi_e defaults to half the number of faces per element (Sec. 3.1 gives
    N/2 = 1.5 for triangles and 2 for tetrahedra; Reading: 2 for quads, 3
    for hexes by the same rule).  q1 Gauss points per direction default to
    k + 2 (Reading: the paper gives no quadrature for L_h).
    """

    def __init__(self, dim, cells, extent, periodic, k, q1=None, chi_e=None, gamma1_in=(0.375, 0.625),
                 flux="cdg2", penalty=None):
        self.dim = dim
        self.cells = tuple(int(c) for c in cells[:dim])
        self.extent = tuple(float(x) for x in extent[:dim])
        self.periodic = tuple(bool(p) for p in periodic[:dim])
        self.k = int(k)
        self.q1 = int(q1) if q1 else self.k + 2
        self.chi_e = float(chi_e) if chi_e is not None else float(dim)
        self.gamma1_in = tuple(gamma1_in)
        # diffusion flux (Sec. 3.1 uses CDG2; Fig. 2 compares it with BR2 and IP)
        self.flux = flux
        self.penalty = float(penalty) if penalty else 2.0 * dim
        self.h = [self.extent[a] / self.cells[a] for a in range(dim)]
        self.vol = math.prod(self.h)
        self.E = math.prod(self.cells)
        self.nb = (self.k + 1) ** dim
        # element multi-index, x fastest
        self.eidx = torch.tensor([tuple(reversed(t)) for t in itertools.product(*[range(c) for c in reversed(self.cells)])],
                                 dtype=torch.long)
        self.origin = self.eidx.to(F64) * torch.tensor(self.h, dtype=F64)
        # volume quadrature (tensor Gauss rule)
        g, w = gauss_legendre01(self.q1)
        qi = multi_indices(self.q1, dim)
        self.qpts = torch.stack([torch.stack([g[t[j]] for j in range(dim)]) for t in qi])
        self.qw = torch.stack([math.prod(float(w[t[j]]) for j in range(dim)) * torch.ones((), dtype=F64) for t in qi])
        self.phi, self.dphi = tabulate(self.k, self.qpts)
        # element mass matrix by quadrature, M_K = |K| sum_q w_q phi_i phi_j
        self.mass = self.vol * torch.einsum("q,qi,qj->ij", self.qw, self.phi, self.phi)

    def elem_id(self, eidx: torch.Tensor) -> torch.Tensor:
        out = torch.zeros(eidx.shape[0], dtype=torch.long)
        stride = 1
        for a in range(self.dim):
            out = out + eidx[:, a] * stride
            stride *= self.cells[a]
        return out

    def face_points(self, a: int, side: float):
        """Reference points and weights of the face xi_a = side of the unit cell."""
        g, w = gauss_legendre01(self.q1)
        tang = [j for j in range(self.dim) if j != a]
        pts, wts = [], []
        for t in multi_indices(self.q1, self.dim - 1):
            p = [0.0] * self.dim
            p[a] = side
            for m, j in enumerate(tang):
                p[j] = float(g[t[m]])
            pts.append(p)
            wts.append(math.prod(float(w[t[m]]) for m in range(self.dim - 1)))
        return torch.tensor(pts, dtype=F64), torch.tensor(wts, dtype=F64)

    def face_area(self, a: int) -> float:
        return math.prod(self.h[j] for j in range(self.dim) if j != a)

    def interior_faces(self, a: int):
        """(K^-, K^+) element ids of the interior faces normal to axis a.

        Reading of the tie-break (all cells have equal volume, so the paper's
        smaller-volume rule never decides): K^- is the lower-coordinate cell,
        so n^- = +e_a; across a periodic wrap K^- is the last cell.
        """
        n = self.cells[a]
        sel = self.eidx[:, a] < n - 1 if not self.periodic[a] else torch.ones(self.E, dtype=torch.bool)
        minus = self.eidx[sel]
        plus = minus.clone()
        plus[:, a] = (plus[:, a] + 1) % n
        return self.elem_id(minus), self.elem_id(plus)

    def phys(self, elems: torch.Tensor, ref_pts: torch.Tensor) -> torch.Tensor:
        """Physical coordinates (E', P, dim) of reference points in elements."""
        return self.origin[elems][:, None, :] + ref_pts[None, :, :] * torch.tensor(self.h, dtype=F64)


# ----------------------------------------------------------------------------
# Model functions of Sec. 2
# ----------------------------------------------------------------------------
def param_vector(p: dict) -> dict:
    """Coefficient dict with every value as a 0-d float64 tensor."""
    out = {}
    for key, v in p.items():
        out[key] = torch.as_tensor(v, dtype=F64)
    return out


def chi(x, y, a, b):
    """Tactic sensitivity chi(x, y, a, b) = a x / (y + b) (Sec. 2)."""
    return a * x / (y + b)


def reduced(p) -> bool:
    """True for the reduced three-species model of Eq. (2) (Sec. 4.2): p["model"] == 1."""
    return int(p.get("model", 0)) == 1


# species that evolve in the reduced model of Eq. (2): n1, n3, c1
REDUCED_ACTIVE = (1.0, 0.0, 1.0, 1.0, 0.0, 0.0)


def velocity(u, g, p):
    """Chemotactic velocities v_1, v_2 with F_s = U_s v_s (s = n1, n2).

    From the compact form of Sec. 2:
      F_1 = chi(n1, c1; chi11) grad c1 + chi(n1, c3; chi13) grad c3
      F_2 = chi(n2, c1; chi21) grad c1 - chi(n2, n1; chi22) grad n1
    (Reading: the n2-against-n1 sensitivity has its own constants chi22,
    equal to chi21 by default, as the paper reuses chi21 there.)
    u: (6, ...) values, g: (6, d, ...) gradients.  Returns v1, v2 (d, ...).
    """
    n1, c1, c3 = u[0], u[3], u[5]
    a, b = p["chi0"], p["chith"]
    if reduced(p):
        # Eq. (2): n1 follows c1 only; n2 is not part of the model
        return (a[0] / (c1 + b[0])) * g[3], torch.zeros_like(g[0])
    v1 = (a[0] / (c1 + b[0])) * g[3] + (a[1] / (c3 + b[1])) * g[5]
    v2 = (a[2] / (c1 + b[2])) * g[3] - (a[3] / (n1 + b[3])) * g[0]
    return v1, v2


def flux_F(u, g, p):
    """Chemotactic flux F(U) in R^{6 x d} (Sec. 2), zero rows for n3, c1..c3."""
    a, b = p["chi0"], p["chith"]
    n1, n2, c1, c3 = u[0], u[1], u[3], u[5]
    F = torch.zeros_like(g)
    if reduced(p):
        # Eq. (2): F_1 = chi(n1, c1; chi11) grad c1; the other rows are zero
        F0 = chi(n1, c1, a[0], b[0]) * g[3]
        return torch.stack([F0] + [torch.zeros_like(F0)] * 5)
    F0 = chi(n1, c1, a[0], b[0]) * g[3] + chi(n1, c3, a[1], b[1]) * g[5]
    F1 = chi(n2, c1, a[2], b[2]) * g[3] - chi(n2, n1, a[3], b[3]) * g[0]
    F = torch.stack([F0, F1] + [torch.zeros_like(F0)] * 4)
    return F


def diffusivity(p):
    """A = diag(mu1, mu2, mu3, nu1, nu2, nu3) (Sec. 2); inactive species of Eq. (2) get 0."""
    A = torch.stack([p["mu"][0], p["mu"][1], p["mu"][2], p["nu"][0], p["nu"][1], p["nu"][2]])
    if reduced(p):
        A = A * torch.tensor(REDUCED_ACTIVE, dtype=F64)
    return A


def source_S(u, p):
    """Reaction source S(U), written from Eq. (1).

    Reading: the c1 row follows Eq. (1), -alpha1 n1 c1 - alpha2 n2 c1 +
    f1 n3 (the compact S of Sec. 2 prints alpha2 n2 c2); f1(n3) is taken
    constant; F(n3, c3) is the constant gamma < 0 of Sec. 2.
    """
    n1, n2, n3, c1, c2, c3 = u
    if reduced(p):
        # Eq. (2): n1 has no source; n3 gains d1 n1 + d2 n2 - gamma n1 (n2 absent, taken 0);
        # c1 loses alpha1 n1 c1 and gains f1 n3; n2, c2, c3 do not evolve
        z = torch.zeros_like(n1)
        return torch.stack([z, z, p["d1"] * n1 + p["d2"] * n2 - p["gamma"] * n1,
                            -p["alpha1"] * n1 * c1 + p["f1"] * n3, z, z])
    return torch.stack([
        -p["d1"] * n1,
        -p["d2"] * n2,
        p["d1"] * n1 + p["d2"] * n2 - p["gamma"] * n1,
        -p["alpha1"] * n1 * c1 - p["alpha2"] * n2 * c1 + p["f1"] * n3,
        -p["k_ox"] * c2,
        p["k_ox"] * c2,
    ])


def heaviside(x):
    """H(x) = 1 for x > 0, 0 otherwise (Reading: H(0) = 0; H' = 0 a.e.)."""
    return (x > 0).to(F64)


# ----------------------------------------------------------------------------
# The operator L_h (Sec. 3.1) and f = M^{-1} L_h (Sec. 3.2)
# ----------------------------------------------------------------------------
def volume_residual(mesh: Mesh, U, p):
    """Element integrals of Eq. elementint: int_K (F - A grad U) : grad phi + S . phi."""
    h = torch.tensor(mesh.h, dtype=F64)
    uq = torch.einsum("qi,esi->seq", mesh.phi, U)
    gq = torch.einsum("jqi,esi->sjeq", mesh.dphi, U) / h[None, :, None, None]
    A = diffusivity(p)
    Phi = flux_F(uq, gq, p) - A[:, None, None, None] * gq          # (6, d, E, q)
    S = source_S(uq, p)                                            # (6, E, q)
    W = mesh.vol * mesh.qw
    R = torch.einsum("q,sjeq,jqi->esi", W, Phi, mesh.dphi / h[:, None, None])
    R = R + torch.einsum("q,seq,qi->esi", W, S, mesh.phi)
    return R


def lifting_normal(mesh: Mesh, phiM, Delta, nvec, area, wf):
    """r_e([U]) . n^- on the face, r_e restricted to one adjacent cell (lifting identity of Sec. 3.1).

    r_e is the element of [V_h]^d with int_Omega r_e : tau = -int_e [U] : {tau}
    for all tau.  On a cell K adjacent to e (with [U] = n^- (x) Delta, {tau} = tau_K/2 there):
      M_K rho_{s,j} = -1/2 int_e n^-_j Delta_s phi_i^K,
    solved with the quadrature mass matrix, then evaluated at the face points.
    phiM: that cell's basis tabulated at the face points (K^- for CDG2; both cells for BR2).
    Delta: (F, 6, P).  Returns (F, 6, P).
    """
    rhs = -0.5 * area * torch.einsum("p,j,fsp,pi->fsji", wf, nvec, Delta, phiM)
    Fn, S, D, nb = rhs.shape
    rho = torch.linalg.solve(mesh.mass, rhs.reshape(-1, nb).T).T.reshape(Fn, S, D, nb)
    r = torch.einsum("pi,fsji->fsjp", phiM, rho)
    return torch.einsum("j,fsjp->fsp", nvec, r)


def face_residual(mesh: Mesh, U, p):
    """Surface integrals of Eq. surfaceint on interior faces.

    With n^- the unit normal out of K^-, Delta = U^- - U^+, [V] = n^- (x) Delta
    and [phi] = n^- (x) (phi^- - phi^+):
      {A grad phi} : [U]  ->  1/2 A_s (grad phi^- + grad phi^+) . n^- Delta_s
      {A grad U} : [phi]  ->  A_s {grad U_s} . n^- (phi^- - phi^+)
      -(F^ - A^) : [phi]  ->  -(F^_s . n^- - A^_s . n^-) (phi^- - phi^+)
    F^ is local Lax-Friedrichs, F^.n = (F^-.n + F^+.n)/2 + lambda_s Delta_s / 2
    with lambda_s = max(|v_s^- . n|, |v_s^+ . n|) (Reading: F_s = U_s v_s, each
    side with its own broken gradient; on a tie the K^- side is taken);
    A^ = 2 chi_e A r_e([U]) restricted to K^-.
    """
    R = torch.zeros_like(U)
    A = diffusivity(p)
    h = torch.tensor(mesh.h, dtype=F64)
    for a in range(mesh.dim):
        em, ep = mesh.interior_faces(a)
        if em.numel() == 0:
            continue
        nvec = torch.zeros(mesh.dim, dtype=F64)
        nvec[a] = 1.0
        ptsM, wf = mesh.face_points(a, 1.0)
        ptsP, _ = mesh.face_points(a, 0.0)
        phiM, dphiM = tabulate(mesh.k, ptsM)
        phiP, dphiP = tabulate(mesh.k, ptsP)
        gradM = dphiM / h[:, None, None]                      # (d, P, nb) physical
        gradP = dphiP / h[:, None, None]
        dnM = torch.einsum("j,jpi->pi", nvec, gradM)
        dnP = torch.einsum("j,jpi->pi", nvec, gradP)
        area = mesh.face_area(a)
        W = area * wf

        UM = torch.einsum("pi,fsi->sfp", phiM, U[em])
        UP = torch.einsum("pi,fsi->sfp", phiP, U[ep])
        GM = torch.einsum("jpi,fsi->sjfp", gradM, U[em])
        GP = torch.einsum("jpi,fsi->sjfp", gradP, U[ep])
        # The jump Delta = U^- - U^+ at each face point, summed over the basis
        # as sum_i (phi_i^- U_i^- - phi_i^+ U_i^+): each basis function's two
        # contributions are differenced before the sum, so the rounding error
        # scales with the jump instead of with U (both traces are O(1) while
        # the jump of a smooth field is tiny).
        pair = phiM[None, None, :, :] * U[em][:, :, None, :] - phiP[None, None, :, :] * U[ep][:, :, None, :]
        Delta = pair.sum(-1).permute(1, 0, 2)                    # (6, F, P)

        avg_dn = 0.5 * torch.einsum("j,sjfp->sfp", nvec, GM + GP)
        FnM = torch.einsum("j,sjfp->sfp", nvec, flux_F(UM, GM, p))
        FnP = torch.einsum("j,sjfp->sfp", nvec, flux_F(UP, GP, p))
        v1M, v2M = velocity(UM, GM, p)
        v1P, v2P = velocity(UP, GP, p)
        lam = []
        for vM, vP in ((v1M, v1P), (v2M, v2P)):
            aM = torch.einsum("j,jfp->fp", nvec, vM).abs()
            aP = torch.einsum("j,jfp->fp", nvec, vP).abs()
            lam.append(torch.where(aM >= aP, aM, aP))
        zero = torch.zeros_like(lam[0])
        lam = torch.stack(lam + [zero] * 4)
        Fhat_n = 0.5 * (FnM + FnP) + 0.5 * lam * Delta

        if mesh.flux == "cdg2":
            # A^ = 2 chi_e A r_e([U]) restricted to K^-
            rn = lifting_normal(mesh, phiM, Delta.permute(1, 0, 2), nvec, area, wf).permute(1, 0, 2)
            Ahat_n = 2.0 * mesh.chi_e * A[:, None, None] * rn
        elif mesh.flux == "br2":
            # A^ = eta A {r_e([U])}: the lifting on both cells, each evaluated on e from its side
            rM = lifting_normal(mesh, phiM, Delta.permute(1, 0, 2), nvec, area, wf).permute(1, 0, 2)
            rP = lifting_normal(mesh, phiP, Delta.permute(1, 0, 2), nvec, area, wf).permute(1, 0, 2)
            Ahat_n = mesh.penalty * A[:, None, None] * 0.5 * (rM + rP)
        else:
            # interior penalty: A^ . n^- = -C (k+1)^2 A Delta |e| / |K|
            Ahat_n = -mesh.penalty * (mesh.k + 1) ** 2 * (area / mesh.vol) * A[:, None, None] * Delta

        sigma = A[:, None, None] * avg_dn - Fhat_n + Ahat_n       # multiplies phi^- - phi^+
        tau = 0.5 * A[:, None, None] * Delta                       # multiplies dn phi^- + dn phi^+

        RM = torch.einsum("p,sfp,pi->fsi", W, sigma, phiM) + torch.einsum("p,sfp,pi->fsi", W, tau, dnM)
        RP = -torch.einsum("p,sfp,pi->fsi", W, sigma, phiP) + torch.einsum("p,sfp,pi->fsi", W, tau, dnP)
        R = R.index_add(0, em, RM)
        R = R.index_add(0, ep, RP)
    return R


def boundary_residual(mesh: Mesh, U, p):
    """Boundary faces: the prescribed normal fluxes of Eq. (3).

    On a boundary face the term -(F^ - A^) : [phi] carries the normal flux
    (A grad U - F) . n, which the boundary conditions fix (Reading: zero
    chemotactic normal flux, no symmetric terms, and the normal in Eq. (3)
    the inward one, so the data enter as influxes times bc_sign):
      Gamma_1 (y = 0):      n1: mu1 beta1 H(c1 - c1*),  c2: nu2 sigma on Gamma_{1,in}
      Gamma_2 (y = L_y):    n2: mu2 beta2 H(c1 - c1**)
    every other species and side: no flow.
    """
    R = torch.zeros_like(U)
    if mesh.dim < 2 or mesh.periodic[1]:
        return R
    area = mesh.face_area(1)
    for side in (0.0, 1.0):
        pts, wf = mesh.face_points(1, side)
        phi, _ = tabulate(mesh.k, pts)
        target = 0 if side == 0.0 else mesh.cells[1] - 1
        el = mesh.elem_id(mesh.eidx[mesh.eidx[:, 1] == target])
        u = torch.einsum("pi,fsi->sfp", phi, U[el])
        x = mesh.phys(el, pts)                                    # (F, P, d)
        g = torch.zeros_like(u)
        if side == 0.0:
            inside = ((x[..., 0] >= mesh.gamma1_in[0]) & (x[..., 0] <= mesh.gamma1_in[1])).to(F64)
            g0 = p["bc_sign"] * p["mu"][0] * p["beta1"] * heaviside(u[3] - p["c1_star"])
            g4 = p["bc_sign"] * p["nu"][1] * p["sigma"] * inside
            if reduced(p):
                g4 = torch.zeros_like(g4)          # no LDL in Eq. (2)
            g = torch.stack([g0, torch.zeros_like(g0), torch.zeros_like(g0), torch.zeros_like(g0), g4,
                             torch.zeros_like(g0)])
        else:
            g1 = p["bc_sign"] * p["mu"][1] * p["beta2"] * heaviside(u[3] - p["c1_star2"])
            if reduced(p):
                g1 = torch.zeros_like(g1)          # no SMCs in Eq. (2)
            z = torch.zeros_like(g1)
            g = torch.stack([z, g1, z, z, z, z])
        R = R.index_add(0, el, torch.einsum("p,sfp,pi->fsi", area * wf, g, phi))
    return R


def apply_residual(mesh: Mesh, U, p, forcing=None, t=0.0):
    """<phi, L_h(U)> for every basis function: the residual R = M L (no M^{-1}).

    forcing: optional callable g(x, t) -> (6, ...) added as int_K g phi.
    """
    R = volume_residual(mesh, U, p) + face_residual(mesh, U, p) + boundary_residual(mesh, U, p)
    if forcing is not None:
        x = mesh.phys(torch.arange(mesh.E), mesh.qpts)           # (E, q, d)
        gx = forcing(x, t)                                        # (6, E, q)
        R = R + torch.einsum("q,seq,qi->esi", mesh.vol * mesh.qw, gx, mesh.phi)
    return R


def minv(mesh: Mesh, R):
    """Inverse of the block-diagonal mass matrix (Sec. 3.2), dense solve per element."""
    E, S, nb = R.shape
    return torch.linalg.solve(mesh.mass, R.reshape(-1, nb).T).T.reshape(E, S, nb)


def apply(mesh: Mesh, U, params: dict, forcing=None, t=0.0):
    """f(U) = M^{-1} L_h(U) (Eq. ode): U, result (E, 6, nb) float64."""
    p = param_vector(params)
    return minv(mesh, apply_residual(mesh, U, p, forcing, t))


def apply_theta(mesh: Mesh, U, params: dict, theta_names, theta):
    """f(U) with the coefficients named in theta_names taken from the tensor theta."""
    p = param_vector(params)
    for i, name in enumerate(theta_names):
        p[name] = theta[i]
    return minv(mesh, apply_residual(mesh, U, p))


def jvp(mesh: Mesh, U, dU, params: dict):
    """J(U) dU, the derivative of f along dU (torch.func forward mode).

    A forcing term does not depend on U and drops out of the derivative.
    """
    return torch.func.jvp(lambda V: apply(mesh, V, params), (U,), (dU,))[1]


def jvp_theta(mesh: Mesh, U, dU, params: dict, theta_names, dtheta):
    """J(U) dU + (df/dtheta) dtheta (torch.func forward mode over U and theta)."""
    theta = torch.tensor([float(params[n]) for n in theta_names], dtype=F64)
    dth = torch.as_tensor(dtheta, dtype=F64)
    return torch.func.jvp(lambda V, th: apply_theta(mesh, V, params, theta_names, th), (U, theta), (dU, dth))[1]


def vjp(mesh: Mesh, U, lam, params: dict, theta_names=()):
    """(J(U)^T lam, (df/dtheta)^T lam) via torch.func reverse mode."""
    theta = torch.tensor([float(params[n]) for n in theta_names], dtype=F64)
    _, fn = torch.func.vjp(lambda V, th: apply_theta(mesh, V, params, theta_names, th), U, theta)
    gU, gth = fn(lam)
    return gU, gth


# ----------------------------------------------------------------------------
# Initial data, errors
# ----------------------------------------------------------------------------
def gaussian_field(mesh: Mesh, x, centres, amps, sigma, floor):
    """u0_s(x) = floor + sum_g A_g exp(-|x - c_g|^2 / (2 sigma^2)), minimum image in periodic axes."""
    vals = []
    for s in range(N_SPECIES):
        v = torch.full(x.shape[:-1], float(floor), dtype=F64)
        for c, amp in zip(centres[s], amps[s]):
            r2 = torch.zeros(x.shape[:-1], dtype=F64)
            for j in range(mesh.dim):
                d = x[..., j] - c[j]
                if mesh.periodic[j]:
                    L = mesh.extent[j]
                    d = d - L * torch.round(d / L)
                r2 = r2 + d * d
            v = v + amp * torch.exp(-r2 / (2.0 * sigma * sigma))
        vals.append(v)
    return torch.stack(vals)


def project(mesh: Mesh, func):
    """L2 projection onto V_h (Sec. 3.2: U(0) is the projection of U_0), q1-point rule."""
    x = mesh.phys(torch.arange(mesh.E), mesh.qpts)
    fx = func(x)                                                  # (6, E, q)
    R = torch.einsum("q,seq,qi->esi", mesh.vol * mesh.qw, fx, mesh.phi)
    return minv(mesh, R)


def l2_error(mesh: Mesh, U, func, npts=None):
    """Per-species ||U_h - u||_{L2} with a (k+3)-point Gauss rule (order >= 2k+4, Sec. 4)."""
    n = npts or mesh.k + 3
    g, w = gauss_legendre01(n)
    qi = multi_indices(n, mesh.dim)
    pts = torch.stack([torch.stack([g[t[j]] for j in range(mesh.dim)]) for t in qi])
    wts = torch.tensor([math.prod(float(w[t[j]]) for j in range(mesh.dim)) for t in qi], dtype=F64)
    phi, _ = tabulate(mesh.k, pts)
    x = mesh.phys(torch.arange(mesh.E), pts)
    uh = torch.einsum("qi,esi->seq", phi, U)
    err = (uh - func(x)) ** 2
    return torch.sqrt(mesh.vol * torch.einsum("q,seq->s", wts, err))


def eoc(errors):
    """Experimental orders of convergence of a sequence of errors on meshes
    refined by a factor 2 (Sec. 4, Table 1): EOC_l = log2(e_{l-1} / e_l)."""
    return [math.log2(errors[l - 1] / errors[l]) for l in range(1, len(errors))]


# ----------------------------------------------------------------------------
# Manufactured solution (Reading: the paper has no exact solution; this one is
# smooth, positive, and satisfies the no-flow conditions at y = 0 and y = L_y)
# ----------------------------------------------------------------------------
def mms_solution(x, t, phases, Ly):
    """U*_s = 1 + 1/2 cos(2 pi x + phi_s) cos(pi y / L_y) exp(-t)."""
    xx, yy = x[..., 0], x[..., 1]
    tt = torch.as_tensor(t, dtype=F64)
    return torch.stack([1.0 + 0.5 * torch.cos(2 * math.pi * xx + ph) * torch.cos(math.pi * yy / Ly) * torch.exp(-tt)
                        for ph in phases])


def mms_forcing(params: dict, phases, Ly):
    """g = dU*/dt - (-div(F(U*) - A grad U*) + S(U*)), derived by automatic differentiation."""
    p = param_vector(params)
    A = diffusivity(p)

    def g(x, t):
        shape = x.shape[:-1]
        xf = x.reshape(-1, x.shape[-1]).clone().requires_grad_(True)
        tt = torch.full((xf.shape[0],), float(t), dtype=F64, requires_grad=True)
        u = mms_solution(xf, tt, phases, Ly)                       # (6, N)
        d = x.shape[-1]
        gu = torch.stack([torch.autograd.grad(u[s].sum(), xf, create_graph=True)[0].T
                          for s in range(N_SPECIES)])              # (6, d, N)
        ut = torch.stack([torch.autograd.grad(u[s].sum(), tt, retain_graph=True)[0]
                          for s in range(N_SPECIES)])              # (6, N)
        flux = flux_F(u, gu, p) - A[:, None, None] * gu
        div = torch.stack([sum(torch.autograd.grad(flux[s, j].sum(), xf, retain_graph=True)[0][:, j]
                               for j in range(d)) for s in range(N_SPECIES)])
        rhs = -div + source_S(u, p)
        return (ut - rhs).detach().reshape((N_SPECIES,) + shape)

    return g


# ----------------------------------------------------------------------------
# Time stepping (Sec. 3.2): SDIRK + Newton + GMRES, matrix-free
# ----------------------------------------------------------------------------
def sdirk_tableau(name: str):
    """Butcher tableau (A, b, c) of L-stable, stiffly accurate SDIRK methods.

    Reading: the paper names DIRK of order 2, 3 or 4 without tableaux.
    sdirk2, sdirk3: Alexander (1977); sdirk4: Hairer and Wanner's 5-stage method.
    sdirk2: 2 stages, gamma = 1 - 1/sqrt(2), stiffly accurate.
    sdirk3: 3 stages, gamma the root in (1/6, 1/2) of 6 g^3 - 18 g^2 + 9 g - 1,
    c2 = (1 + gamma)/2, b1 = -(6 g^2 - 16 g + 1)/4, b2 = (6 g^2 - 20 g + 5)/4.
    """
    if name == "sdirk2":
        g = 1.0 - 1.0 / math.sqrt(2.0)
        A = np.array([[g, 0.0], [1.0 - g, g]])
    elif name == "sdirk4":
        # Hairer & Wanner, Solving ODEs II, Sec. IV.6: 5 stages, gamma = 1/4, order 4
        A = np.array([[1 / 4, 0, 0, 0, 0],
                      [1 / 2, 1 / 4, 0, 0, 0],
                      [17 / 50, -1 / 25, 1 / 4, 0, 0],
                      [371 / 1360, -137 / 2720, 15 / 544, 1 / 4, 0],
                      [25 / 24, -49 / 48, 125 / 16, -85 / 12, 1 / 4]])
    elif name == "sdirk3":
        roots = np.roots([6.0, -18.0, 9.0, -1.0])
        g = float([r.real for r in roots if abs(r.imag) < 1e-14 and 1 / 6 < r.real < 0.5][0])
        c2 = (1.0 + g) / 2.0
        b1 = -(6 * g * g - 16 * g + 1) / 4.0
        b2 = (6 * g * g - 20 * g + 5) / 4.0
        A = np.array([[g, 0.0, 0.0], [c2 - g, g, 0.0], [b1, b2, g]])
    else:
        raise ValueError(name)
    b = A[-1].copy()
    c = A.sum(axis=1)
    return A, b, c


def _gmres(matvec, rhs, tol, restart=50, maxit=2000):
    """scipy GMRES on flattened float64 vectors."""
    from scipy.sparse.linalg import LinearOperator, gmres
    n = rhs.numel()
    op = LinearOperator((n, n), matvec=lambda v: matvec(torch.from_numpy(np.ascontiguousarray(v)).reshape(rhs.shape))
                        .reshape(-1).numpy(), dtype=np.float64)
    x, info = gmres(op, rhs.reshape(-1).numpy(), rtol=tol, atol=0.0, restart=restart, maxiter=maxit)
    if info != 0:
        raise RuntimeError(f"oracle GMRES did not converge (info={info})")
    return torch.from_numpy(x).reshape(rhs.shape)


def _newton_correction(mesh: Mesh, Y, G, gdt: float, params: dict, gmres_tol: float):
    """Solve (I - gdt J(Y)) d = -G: dense Jacobian and LU for tiny systems, else GMRES."""
    n = Y.numel()
    if n <= 3000:
        J = torch.func.jacfwd(lambda V: apply(mesh, V, params))(Y).reshape(n, n)
        return torch.linalg.solve(torch.eye(n, dtype=F64) - gdt * J, -G.reshape(-1)).reshape(Y.shape)
    return _gmres(lambda v: v - gdt * jvp(mesh, Y, v, params), -G, gmres_tol)


def step(mesh: Mesh, U, params: dict, t: float, dt: float, scheme="sdirk2", forcing=None,
         newton_tol=1e-13, gmres_tol=1e-13, max_newton=30):
    """One SDIRK step U_n -> U_{n+1} for U' = f(U, t) = M^{-1} L_h(U) (+ forcing).

    Stage i solves Y_i - dt a_ii f(Y_i, t + c_i dt) = U_n + dt sum_{j<i} a_ij K_j by
    Newton's method; each Newton correction solves (I - dt a_ii J(Y)) d = -G with
    GMRES using J(Y) v from automatic differentiation (Jacobian-free Newton-Krylov),
    or, for systems of at most 3000 unknowns, with the dense Jacobian and LU.
    Newton stops when ||G||_2 <= newton_tol * max(1, ||rhs_i||_2).
    """
    A, b, c = sdirk_tableau(scheme)
    s = len(b)
    K = []
    for i in range(s):
        ti = t + c[i] * dt
        rhs = U.clone()
        for j in range(i):
            rhs = rhs + dt * A[i, j] * K[j]
        Y = U.clone() if i == 0 else Y
        gdt = dt * A[i, i]
        scale = max(1.0, float(torch.linalg.norm(rhs)))
        for _it in range(max_newton):
            fY = apply(mesh, Y, params, forcing, ti)
            G = Y - gdt * fY - rhs
            if float(torch.linalg.norm(G)) <= newton_tol * scale:
                break
            Y = Y + _newton_correction(mesh, Y, G, gdt, params, gmres_tol)
        else:
            raise RuntimeError("oracle Newton did not converge")
        K.append(apply(mesh, Y, params, forcing, ti))
    out = U.clone()
    for i in range(s):
        out = out + dt * b[i] * K[i]
    return out


def step_stages(mesh: Mesh, U, params: dict, t: float, dt: float, scheme="sdirk2", **kw):
    """step() that also returns the converged stage values Y_1..Y_s."""
    A, b, c = sdirk_tableau(scheme)
    stages = []
    s = len(b)
    K = []
    Y = U.clone()
    for i in range(s):
        ti = t + c[i] * dt
        rhs = U.clone()
        for j in range(i):
            rhs = rhs + dt * A[i, j] * K[j]
        gdt = dt * A[i, i]
        scale = max(1.0, float(torch.linalg.norm(rhs)))
        for _it in range(kw.get("max_newton", 30)):
            fY = apply(mesh, Y, params, kw.get("forcing"), ti)
            G = Y - gdt * fY - rhs
            if float(torch.linalg.norm(G)) <= kw.get("newton_tol", 1e-13) * scale:
                break
            Y = Y + _newton_correction(mesh, Y, G, gdt, params, kw.get("gmres_tol", 1e-13))
        stages.append(Y.clone())
        K.append(apply(mesh, Y, params, kw.get("forcing"), ti))
    out = U.clone()
    for i in range(s):
        out = out + dt * b[i] * K[i]
    return out, stages


def step_adjoint(mesh: Mesh, stages, params: dict, dt: float, scheme, lam, theta_names=()):
    """Discrete adjoint of one SDIRK step with dense Jacobians (tiny meshes only).

    With K_i = f(Y_i), Y_i = U_n + dt sum_j a_ij K_j, U_{n+1} = U_n + dt sum_i b_i K_i,
    the chain rule gives, backwards over the stages:
      r_i = dt b_i lam + dt sum_{j>i} a_ji ybar_j,   (I - dt a_ii J_i)^T g_i = r_i,
      ybar_i = J_i^T g_i,   gtheta += (df/dtheta)(Y_i)^T g_i,   lam_n = lam + sum_i ybar_i,
    with J_i = df/dU at Y_i formed densely by forward-mode differentiation.
    """
    A, b, _c = sdirk_tableau(scheme)
    s = len(b)
    n = lam.numel()
    ybar = [None] * s
    gth = torch.zeros(len(theta_names), dtype=F64)
    for i in reversed(range(s)):
        r = dt * b[i] * lam.reshape(-1)
        for j in range(i + 1, s):
            r = r + dt * A[j, i] * ybar[j]
        J = torch.func.jacfwd(lambda V: apply(mesh, V, params))(stages[i]).reshape(n, n)
        g = torch.linalg.solve((torch.eye(n, dtype=F64) - dt * A[i, i] * J).T, r)
        ybar[i] = J.T @ g
        if theta_names:
            _gU, gt = vjp(mesh, stages[i], g.reshape(lam.shape), params, theta_names)
            gth = gth + gt
    lam_n = lam.reshape(-1) + sum(ybar)
    return lam_n.reshape(lam.shape), gth
