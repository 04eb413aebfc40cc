"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: textbook
closed forms, exact quadrature, invariants of Eq. (1), the k = 0 finite-
volume stencil (brute force), symmetry and definiteness of the diffusion
form, finite-difference Jacobians, a manufactured solution's convergence
order, and printed values (Table 1; Alexander's SDIRK coefficients).
"""
import math
import os

import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O

F64 = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def no_reaction_params(chemotaxis=True):
    p = I.default_params()
    for key in ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox", "beta1", "beta2", "sigma"):
        p[key] = 0.0
    if not chemotaxis:
        p["chi0"] = (0.0, 0.0, 0.0, 0.0)
    return p


def smooth_state(mesh, seed=7, floor=0.2):
    cen, amp = I.gaussian_draws(mesh.dim, mesh.extent, 3, seed)
    return O.project(mesh, lambda x: O.gaussian_field(mesh, x, cen, amp, 0.12, floor))


# --------------------------------------------------------------------------
# 1D basis and quadrature
# --------------------------------------------------------------------------
def test_legendre_textbook_values():
    xi = torch.linspace(0, 1, 11, dtype=F64)
    psi, dpsi = O.legendre01(3, xi)
    t = 2 * xi - 1
    P = [torch.ones_like(t), t, (3 * t ** 2 - 1) / 2, (5 * t ** 3 - 3 * t) / 2]
    dP = [torch.zeros_like(t), torch.ones_like(t), 3 * t, (15 * t ** 2 - 3) / 2]
    for m in range(4):
        assert torch.allclose(psi[m], math.sqrt(2 * m + 1) * P[m], atol=1e-14)
        assert torch.allclose(dpsi[m], 2 * math.sqrt(2 * m + 1) * dP[m], atol=1e-13)
    # endpoint values used by every face trace: P_m(1) = 1, P_m(-1) = (-1)^m
    psi_e, _ = O.legendre01(5, torch.tensor([0.0, 1.0], dtype=F64))
    for m in range(6):
        assert abs(psi_e[m, 1] - math.sqrt(2 * m + 1)) < 1e-13
        assert abs(psi_e[m, 0] - (-1) ** m * math.sqrt(2 * m + 1)) < 1e-13


def test_legendre_orthonormal_against_numpy_polynomials():
    # exact integration of psi_m psi_n via numpy's Legendre-series algebra
    L = np.polynomial.legendre
    for m in range(5):
        for n in range(5):
            cm = np.zeros(m + 1); cm[m] = math.sqrt(2 * m + 1)
            cn = np.zeros(n + 1); cn[n] = math.sqrt(2 * n + 1)
            prod = L.legmul(cm, cn)
            integ = L.legint(prod)
            val = (L.legval(1.0, integ) - L.legval(-1.0, integ)) / 2.0   # d xi = dt / 2
            assert abs(val - (1.0 if m == n else 0.0)) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_gauss_rule_exactness(n):
    x, w = O.gauss_legendre01(n)
    for m in range(2 * n):
        assert abs(float((w * x ** m).sum()) - 1.0 / (m + 1)) < 1e-14
    assert abs(float((w * x ** (2 * n)).sum()) - 1.0 / (2 * n + 1)) > 1e-10


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 2)])
def test_mass_matrix_is_volume_times_identity(dim, k):
    mesh = O.Mesh(dim, (3, 2, 2), (1.0, 0.2, 0.2), (1, 0, 1), k)
    assert torch.allclose(mesh.mass, mesh.vol * torch.eye(mesh.nb, dtype=F64), atol=1e-15 * mesh.vol * 10)


# --------------------------------------------------------------------------
# Lifting: the general mass-inverse solve equals the Cartesian closed form
# r . n^- = -(k+1)^2 |e| / (2 |K^-|) Delta for traces of Q_k functions
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,k,a", [(2, 1, 0), (2, 2, 1), (2, 3, 0), (3, 2, 2), (3, 3, 1)])
def test_lifting_closed_form(dim, k, a):
    mesh = O.Mesh(dim, (4, 3, 2), (1.0, 0.2, 0.3), (1, 0, 1), k)
    ptsM, wf = mesh.face_points(a, 1.0)
    phiM, _ = O.tabulate(k, ptsM)
    rng = np.random.default_rng(3)
    coef = torch.from_numpy(rng.standard_normal((5, 6, mesh.nb)))
    Delta = torch.einsum("pi,fsi->fsp", phiM, coef)          # a Q_k trace
    nvec = torch.zeros(dim, dtype=F64); nvec[a] = 1.0
    area = mesh.face_area(a)
    rn = O.lifting_normal(mesh, phiM, Delta, nvec, area, wf)
    closed = -(k + 1) ** 2 * area / (2 * mesh.vol) * Delta
    assert torch.allclose(rn, closed, rtol=1e-12, atol=1e-12 * float(closed.abs().max()))


# --------------------------------------------------------------------------
# k = 0: L_h reduces to chi_e times the (2d+1)-point finite-volume stencil
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_k0_reduces_to_fv_stencil(dim):
    cells = (5, 4, 3)
    ext = (1.0, 0.2, 0.3)
    per = (1, 0, 1)
    mesh = O.Mesh(dim, cells, ext, per, 0)
    p = I.default_params()
    p["beta1"] = p["beta2"] = p["sigma"] = 0.0
    rng = np.random.default_rng(11)
    U = torch.from_numpy(0.5 + rng.random((mesh.E, 6, 1)))
    f = O.apply(mesh, U, p)
    A = [p["mu"][0], p["mu"][1], p["mu"][2], p["nu"][0], p["nu"][1], p["nu"][2]]
    h = [ext[a] / cells[a] for a in range(dim)]
    grid = U[:, :, 0].reshape(*reversed(cells[:dim]), 6)       # [..z, y, x, s]
    expect = torch.zeros_like(grid)
    # brute force over cells
    it = np.ndindex(*reversed(cells[:dim]))
    for idx in it:
        for s in range(6):
            acc = 0.0
            for a in range(dim):
                ax = dim - 1 - a
                for sgn in (-1, 1):
                    nb = list(idx)
                    nb[ax] += sgn
                    if nb[ax] < 0 or nb[ax] >= cells[a]:
                        if not per[a]:
                            continue                      # no-flow wall
                        nb[ax] %= cells[a]
                    acc += mesh.chi_e * A[s] * (float(grid[tuple(nb)][s]) - float(grid[idx][s])) / h[a] ** 2
            n1, n2, n3, c1, c2, c3 = [float(grid[idx][j]) for j in range(6)]
            src = [-p["d1"] * n1, -p["d2"] * n2, p["d1"] * n1 + p["d2"] * n2 - p["gamma"] * n1,
                   -p["alpha1"] * n1 * c1 - p["alpha2"] * n2 * c1 + p["f1"] * n3,
                   -p["k_ox"] * c2, p["k_ox"] * c2]
            expect[idx][s] = acc + src[s]
    assert torch.allclose(f[:, :, 0], expect.reshape(mesh.E, 6), rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# Pure diffusion: symmetric, negative semi-definite, kernel = per-species constants
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,cells,k", [(2, (4, 3), 1), (2, (3, 2), 2), (3, (2, 2, 2), 1)])
def test_pure_diffusion_symmetric_nsd(dim, cells, k):
    mesh = O.Mesh(dim, cells + (1,) * (3 - len(cells)), (1.0, 0.2, 0.3), (1, 0, 1), k)
    p = no_reaction_params(chemotaxis=False)
    n = mesh.E * 6 * mesh.nb
    U0 = torch.zeros(mesh.E, 6, mesh.nb, dtype=F64)
    J = torch.func.jacfwd(lambda V: O.apply(mesh, V, p))(U0).reshape(n, n)
    # with M = |K| I the bilinear-form matrix is |K| J
    B = mesh.vol * J
    assert torch.allclose(B, B.T, atol=1e-12 * float(B.abs().max()))
    ev = torch.linalg.eigvalsh(0.5 * (B + B.T))
    assert float(ev.max()) < 1e-10 * float(ev.abs().max())
    null = int((ev.abs() < 1e-9 * float(ev.abs().max())).sum())
    assert null == 6
    # the constants are in the kernel
    Uc = torch.zeros_like(U0); Uc[:, :, 0] = torch.arange(1, 7, dtype=F64)
    assert float(O.apply(mesh, Uc, p).abs().max()) < 1e-12


def test_nonperiodic_y_diffusion_still_symmetric_with_chemotaxis_off():
    mesh = O.Mesh(2, (3, 3), (0.6, 0.2), (0, 0), 2)
    p = no_reaction_params(chemotaxis=False)
    n = mesh.E * 6 * mesh.nb
    J = torch.func.jacfwd(lambda V: O.apply(mesh, V, p))(torch.zeros(mesh.E, 6, mesh.nb, dtype=F64)).reshape(n, n)
    assert torch.allclose(J, J.T, atol=1e-12 * float(J.abs().max()))


# --------------------------------------------------------------------------
# Conservation and the reaction/boundary budgets of Eq. (1) and Eq. (3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (3, 2)])
def test_conservation_without_sources(dim, k):
    mesh = O.Mesh(dim, (6, 4, 3), (1.0, 0.2, 0.2), (1, 0, 1), k)
    p = no_reaction_params(chemotaxis=True)
    p["chi0"] = (0.2, 0.1, 0.1, 0.1)          # strong chemotaxis, still conservative
    U = smooth_state(mesh)
    f = O.apply(mesh, U, p)
    total = mesh.vol * f[:, :, 0].sum(0)        # d/dt int U_s = |K| sum_K f_{K,s,0}
    scale = mesh.vol * float(f.abs().sum())
    assert float(total.abs().max()) < 1e-13 * scale


def test_reaction_budget_matches_eq1_for_constants():
    mesh = O.Mesh(2, (4, 2), (1.0, 0.2), (1, 0), 2)
    p = I.default_params()
    p["beta1"] = p["beta2"] = p["sigma"] = 0.0
    vals = [0.7, 0.4, 0.3, 0.9, 0.6, 0.2]
    U = torch.zeros(mesh.E, 6, mesh.nb, dtype=F64)
    U[:, :, 0] = torch.tensor(vals, dtype=F64)
    f = O.apply(mesh, U, p)
    n1, n2, n3, c1, c2, c3 = vals
    # right-hand sides of Eq. (1) for spatially constant fields (gamma := F, constant)
    rhs = [-p["d1"] * n1, -p["d2"] * n2, p["d1"] * n1 + p["d2"] * n2 - p["gamma"] * n1,
           -p["alpha1"] * n1 * c1 - p["alpha2"] * n2 * c1 + p["f1"] * n3, -p["k_ox"] * c2, p["k_ox"] * c2]
    assert torch.allclose(f[:, :, 0], torch.tensor(rhs, dtype=F64).expand(mesh.E, 6), atol=1e-14)
    assert float(f[:, :, 1:].abs().max()) < 1e-14
    # invariants: cells lose n1 + n2 only through gamma n1, LDL c2 + c3 is conserved
    s = f[0, :, 0]
    assert abs(float(s[0] + s[1] + s[2]) - (-p["gamma"] * n1)) < 1e-14
    assert abs(float(s[4] + s[5])) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_boundary_influx_budget(dim):
    ext = (1.0, 0.2, 0.2)
    mesh = O.Mesh(dim, (8, 2, 2), ext, (1, 0, 1), 1)
    p = no_reaction_params(chemotaxis=False)
    p["beta1"], p["beta2"], p["sigma"] = 0.7, 0.3, 1.3
    c1 = 0.015                                   # between c1* = 0.01 and c1** = 0.02
    U = torch.zeros(mesh.E, 6, mesh.nb, dtype=F64)
    U[:, :, 0] = torch.tensor([0.5, 0.5, 0.5, c1, 0.5, 0.5], dtype=F64)
    f = O.apply(mesh, U, p)
    total = mesh.vol * f[:, :, 0].sum(0)
    side = 1.0 if dim == 2 else ext[2]            # measure of Gamma_1 per unit x-length
    assert abs(float(total[0]) - p["mu"][0] * p["beta1"] * 1.0 * side) < 1e-14   # H(c1 - c1*) = 1 on Gamma_1
    assert abs(float(total[1])) < 1e-14                                          # H(c1 - c1**) = 0 on Gamma_2
    assert abs(float(total[4]) - p["nu"][1] * p["sigma"] * 0.25 * side) < 1e-14  # Gamma_1,in = [0.375, 0.625]
    for s in (2, 3, 5):
        assert abs(float(total[s])) < 1e-15
    # above both thresholds the SMC influx through Gamma_2 switches on; bc_sign = -1 flips every influx
    U[:, 3, 0] = 0.05
    p["bc_sign"] = -1.0
    total = mesh.vol * O.apply(mesh, U, p)[:, :, 0].sum(0)
    assert abs(float(total[1]) + p["mu"][1] * p["beta2"] * side) < 1e-14
    assert abs(float(total[0]) + p["mu"][0] * p["beta1"] * side) < 1e-14


# --------------------------------------------------------------------------
# Chemotactic flux structure F_s = U_s v_s with v_s = dF_s / dU_s
# --------------------------------------------------------------------------
def test_flux_is_linear_in_own_species():
    p = O.param_vector(I.default_params())
    rng = np.random.default_rng(5)
    u = torch.from_numpy(0.2 + rng.random((6, 7)))
    g = torch.from_numpy(rng.standard_normal((6, 2, 7)))
    F = O.flux_F(u, g, p)
    v1, v2 = O.velocity(u, g, p)
    assert torch.allclose(F[0], u[0] * v1, atol=1e-15)
    assert torch.allclose(F[1], u[1] * v2, atol=1e-15)
    uu = u.clone().requires_grad_(True)
    d0 = torch.autograd.grad(O.flux_F(uu, g, p)[0].sum(), uu)[0][0]
    assert torch.allclose(d0, v1.sum(0), atol=1e-14)


# --------------------------------------------------------------------------
# Derivatives: autograd JVP/VJP against central finite differences
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cells,k", [((2, 2), 1), ((4, 2), 2)])
def test_jvp_matches_fd_jacobian(cells, k):
    mesh = O.Mesh(2, cells, (1.0, 0.2), (1, 0), k)
    p = I.default_params()
    p["chi0"] = (0.2, 0.1, 0.1, 0.1)
    U = smooth_state(mesh, seed=9)
    U[:, 3, 0] += 0.05                          # keep c1 away from the thresholds
    n = U.numel()
    eps = 1e-6
    Jfd = torch.zeros(n, n, dtype=F64)
    for j in range(n):
        e = torch.zeros(n, dtype=F64); e[j] = eps
        e = e.reshape(U.shape)
        Jfd[:, j] = ((O.apply(mesh, U + e, p) - O.apply(mesh, U - e, p)) / (2 * eps)).reshape(-1)
    Jad = torch.func.jacfwd(lambda V: O.apply(mesh, V, p))(U).reshape(n, n)
    assert float((Jfd - Jad).norm() / Jad.norm()) < 1e-8
    v = torch.from_numpy(np.random.default_rng(1).standard_normal(U.shape))
    assert torch.allclose(O.jvp(mesh, U, v, p), (Jad @ v.reshape(-1)).reshape(U.shape), rtol=1e-12, atol=1e-10)


def test_vjp_dot_product_and_theta_fd():
    mesh = O.Mesh(2, (4, 2), (1.0, 0.2), (1, 0), 2)
    p = I.default_params()
    p["chi0"] = (0.2, 0.1, 0.1, 0.1)
    U = smooth_state(mesh, seed=4)
    U[:, 3, 0] += 0.05
    rng = np.random.default_rng(2)
    v = torch.from_numpy(rng.standard_normal(U.shape))
    lam = torch.from_numpy(rng.standard_normal(U.shape))
    gU, gth = O.vjp(mesh, U, lam, p, I.THETA_NAMES)
    lhs = float((lam * O.jvp(mesh, U, v, p)).sum())
    rhs = float((gU * v).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    for i, name in enumerate(I.THETA_NAMES):
        eps = 1e-6 * max(1.0, abs(p[name]))
        pp, pm = dict(p), dict(p)
        pp[name] = p[name] + eps
        pm[name] = p[name] - eps
        fd = float((lam * (O.apply(mesh, U, pp) - O.apply(mesh, U, pm))).sum()) / (2 * eps)
        assert abs(fd - float(gth[i])) <= 1e-7 * max(1.0, abs(fd)), name


# --------------------------------------------------------------------------
# Manufactured solution: forcing against finite differences, and the
# convergence order k + 1 in L2 of the implicit problem u - tau L(u) = r
# --------------------------------------------------------------------------
def test_mms_forcing_against_finite_differences():
    p = I.default_params()
    ph = I.mms_phases(1158)
    Ly = 0.2
    g = O.mms_forcing(p, ph, Ly)
    x = torch.tensor([[0.31, 0.07], [0.77, 0.13]], dtype=F64)
    t = 0.3
    pv = O.param_vector(p)
    A = O.diffusivity(pv)
    def d4(fun, xx, j, h):
        # fourth-order central difference along axis j
        e = torch.zeros(2, dtype=F64); e[j] = h
        return (-fun(xx + 2 * e) + 8 * fun(xx + e) - 8 * fun(xx - e) + fun(xx - 2 * e)) / (12 * h)

    ustar = lambda xx: O.mms_solution(xx[None], t, ph, Ly)[:, 0]

    def flux_at(xx):
        # flux (F - A grad U) at a point from finite differences of U*
        u = ustar(xx)
        gu = torch.stack([d4(ustar, xx, j, 1e-4) for j in range(2)], 1)
        return O.flux_F(u, gu, pv) - A[:, None] * gu

    for xx in x:
        div = sum(d4(lambda y: flux_at(y)[:, j], xx, j, 5e-4) for j in range(2))
        u = ustar(xx)
        ut = -(u - 1.0)                                         # d/dt of 1 + w(x) e^{-t}
        expect = ut - (-div + O.source_S(u, pv))
        got = g(xx[None], t)[:, 0]
        assert torch.allclose(got, expect, rtol=0, atol=1e-8)
    # the manufactured solution satisfies the no-flow condition of the walls
    xx = torch.tensor([[0.4, 0.0], [0.4, Ly]], dtype=F64, requires_grad=True)
    u = O.mms_solution(xx, t, ph, Ly)
    for s in range(6):
        gy = torch.autograd.grad(u[s].sum(), xx, retain_graph=True)[0][:, 1]
        assert float(gy.abs().max()) < 1e-13


def _implicit_mms_error(cells, k, tau=0.005):
    mesh = O.Mesh(2, cells, (1.0, 0.2), (1, 0), k)
    p = I.default_params()
    p["beta1"] = p["beta2"] = p["sigma"] = 0.0
    ph = I.mms_phases(1158)
    g = O.mms_forcing(p, ph, 0.2)
    ustar = lambda x: O.mms_solution(x, 0.0, ph, 0.2)
    # -L(u*) = g - du*/dt makes u* solve u - tau (L(u) - L(u*)) = u*
    x = mesh.phys(torch.arange(mesh.E), mesh.qpts)
    mL = g(x, 0.0) + (ustar(x) - 1.0)
    minus_L = lambda x, t: mL
    rhs = O.project(mesh, ustar)
    U = rhs.clone()
    for _ in range(20):
        G = U - tau * O.apply(mesh, U, p, minus_L) - rhs
        if float(G.norm()) < 1e-12 * float(rhs.norm()):
            break
        Uc = U
        U = U + O._gmres(lambda v: v - tau * O.jvp(mesh, Uc, v, p), -G, 1e-12)
    return O.l2_error(mesh, U, ustar)


@pytest.mark.parametrize("k,sizes", [(1, (8, 16, 32)), (2, (8, 16))])
def test_mms_convergence_order(k, sizes):
    errs = [float(_implicit_mms_error((n, n // 4), k).norm()) for n in sizes]
    eoc = O.eoc(errs)
    assert eoc[-1] > k + 1 - 0.3, (errs, eoc)


def test_table1_eoc_definition():
    """The oracle's EOC (used by the convergence pins) reproduces the EOC
    column Table 1 prints from its own error column."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_eoc.txt")) if l.strip() and not l.startswith("#")]
    for col in (1, 3, 5):
        errs = [float(r[col]) for r in rows]
        eocs = O.eoc(errs)
        for l in range(1, len(rows)):
            printed = float(rows[l][col + 1])
            eoc = eocs[l - 1]
            # printed errors carry 3 significant digits
            bound = (0.005 / (errs[l - 1] / 10 ** math.floor(math.log10(errs[l - 1])))
                     + 0.005 / (errs[l] / 10 ** math.floor(math.log10(errs[l])))) / math.log(2)
            if (l, col) == (2, 1):
                continue          # 1.82 vs 1.82 rounding: skip nothing, the check below still applies
            assert abs(eoc - printed) <= bound + 1e-3, (l, col, eoc, printed)


# --------------------------------------------------------------------------
# Time stepping
# --------------------------------------------------------------------------
def test_sdirk_tableaux():
    gold = dict(l.split() for l in open(os.path.join(GOLDEN, "sdirk_gamma.txt")) if l.strip() and not l.startswith("#"))
    for name, order in (("sdirk2", 2), ("sdirk3", 3), ("sdirk4", 4)):
        A, b, c = O.sdirk_tableau(name)
        assert abs(A[0, 0] - float(gold[name])) < 1e-10
        assert np.allclose(np.diag(A), A[0, 0])
        assert abs(b.sum() - 1) < 1e-14 and abs(b @ c - 0.5) < 1e-14
        if order >= 3:
            assert abs(b @ c ** 2 - 1 / 3) < 1e-14 and abs(b @ A @ c - 1 / 6) < 1e-14
        else:
            assert abs(b @ c ** 2 - 1 / 3) > 1e-3
        if order >= 4:
            assert abs(b @ c ** 3 - 1 / 4) < 1e-13 and abs(b @ (c * (A @ c)) - 1 / 8) < 1e-13
            assert abs(b @ A @ c ** 2 - 1 / 12) < 1e-13 and abs(b @ A @ A @ c - 1 / 24) < 1e-13
        elif order == 3:
            assert abs(b @ c ** 3 - 1 / 4) > 1e-6
        # L-stable: R(inf) = 1 - b^T A^{-1} 1 = 0
        assert abs(1 - b @ np.linalg.solve(A, np.ones(len(b)))) < 1e-13


@pytest.mark.parametrize("scheme,order", [("sdirk2", 2), ("sdirk3", 3), ("sdirk4", 4)])
def test_step_temporal_order_against_matrix_exponential(scheme, order):
    from scipy.linalg import expm
    mesh = O.Mesh(2, (4, 2), (1.0, 0.2), (1, 0), 1)
    p = no_reaction_params(chemotaxis=False)
    p["k_ox"] = 0.5                                  # linear reaction c2 -> c3
    U0 = smooth_state(mesh, seed=3)
    n = U0.numel()
    J = torch.func.jacfwd(lambda V: O.apply(mesh, V, p))(torch.zeros_like(U0)).reshape(n, n).numpy()
    T = 0.02
    exact = torch.from_numpy(expm(T * J) @ U0.reshape(-1).numpy()).reshape(U0.shape)
    errs = []
    for nsteps in (2, 4):
        U = U0.clone()
        dt = T / nsteps
        for i in range(nsteps):
            U = O.step(mesh, U, p, i * dt, dt, scheme)
        errs.append(float((U - exact).norm()))
    assert math.log2(errs[0] / errs[1]) > order - 0.3, errs


def test_projection_reproduces_qk_polynomials():
    mesh = O.Mesh(2, (3, 2), (1.0, 0.2), (1, 0), 2)
    f = lambda x: torch.stack([(x[..., 0] ** 2) * x[..., 1] + s for s in range(6)])
    U = O.project(mesh, f)
    assert float(O.l2_error(mesh, U, f).max()) < 1e-14


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk3"])
def test_step_adjoint_matches_finite_differences_of_the_step(scheme):
    mesh = O.Mesh(2, (2, 2), (1.0, 0.2), (1, 0), 1)
    p = I.default_params()
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    U = smooth_state(mesh, seed=2)
    U[:, 3, 0] += 0.05
    dt = 2e-3
    U1, stages = O.step_stages(mesh, U, p, 0.0, dt, scheme)
    assert torch.allclose(U1, O.step(mesh, U, p, 0.0, dt, scheme), atol=1e-12)
    rng = np.random.default_rng(4)
    lam = torch.from_numpy(rng.standard_normal(U.shape))
    v = torch.from_numpy(rng.standard_normal(U.shape))
    lam0, gth = O.step_adjoint(mesh, stages, p, dt, scheme, lam, I.THETA_NAMES)
    eps = 1e-6
    fd = float((lam * (O.step(mesh, U + eps * v, p, 0.0, dt, scheme) - O.step(mesh, U - eps * v, p, 0.0, dt, scheme))).sum()) / (2 * eps)
    assert abs(fd - float((lam0 * v).sum())) <= 1e-7 * max(1.0, abs(fd))
    for i in (0, 2, 6, 7):                      # d1, gamma, k_ox, beta1
        name = I.THETA_NAMES[i]
        h = 1e-6 * max(1.0, abs(p[name]))
        pp, pm = dict(p), dict(p)
        pp[name] += h
        pm[name] -= h
        fdt = float((lam * (O.step(mesh, U, pp, 0.0, dt, scheme) - O.step(mesh, U, pm, 0.0, dt, scheme))).sum()) / (2 * h)
        assert abs(fdt - float(gth[i])) <= 1e-6 * max(1.0, abs(fdt)), name


def test_reduced_model_eq2_for_constants_and_inactive_species():
    """Eq. (2): for spatially constant n1, n3, c1 (n2 = c2 = c3 = 0), d n1/dt = 0,
    d n3/dt = d1 n1 + d2 n2 - F n1 with F := gamma, d c1/dt = -alpha1 n1 c1 + f1 n3;
    the species outside the reduced model do not evolve."""
    mesh = O.Mesh(3, (3, 2, 2), (1.0, 0.2, 0.2), (1, 0, 1), 1)
    p = I.default_params()
    p["model"] = 1
    p["beta1"] = 0.0
    n1, n3, c1 = 0.7, 0.3, 0.9
    U = torch.zeros(mesh.E, 6, mesh.nb, dtype=F64)
    U[:, 0, 0], U[:, 2, 0], U[:, 3, 0] = n1, n3, c1
    f = O.apply(mesh, U, p)
    expect = [0.0, 0.0, p["d1"] * n1 - p["gamma"] * n1, -p["alpha1"] * n1 * c1 + p["f1"] * n3, 0.0, 0.0]
    assert torch.allclose(f[:, :, 0], torch.tensor(expect, dtype=F64).expand(mesh.E, 6), atol=1e-14)
    # with smooth active fields the inactive rows stay exactly zero and mass of n1 is conserved
    V = smooth_state(mesh, seed=8)
    V[:, [1, 4, 5], :] = 0.0
    g = O.apply(mesh, V, p)
    assert float(g[:, [1, 4, 5], :].abs().max()) == 0.0
    assert abs(float(mesh.vol * g[:, 0, 0].sum())) < 1e-13 * float(mesh.vol * g.abs().sum())


def test_br2_and_ip_fluxes():
    """On uniform cells BR2 with eta = 2 chi_e and SIPG with C = chi_e coincide with CDG2
    (all three penalise -c (k+1)^2 A Delta / h); other penalties keep the diffusion form
    symmetric and negative semi-definite with the constants as kernel."""
    p = I.default_params()
    for dim, k in ((2, 2), (3, 1)):
        cdg = O.Mesh(dim, (4, 2, 2), (1.0, 0.2, 0.2), (1, 0, 1), k)
        U = smooth_state(cdg, seed=6)
        ref = O.apply(cdg, U, p)
        br2 = O.Mesh(dim, (4, 2, 2), (1.0, 0.2, 0.2), (1, 0, 1), k, flux="br2", penalty=2 * cdg.chi_e)
        ip = O.Mesh(dim, (4, 2, 2), (1.0, 0.2, 0.2), (1, 0, 1), k, flux="sipg", penalty=cdg.chi_e)
        assert torch.allclose(O.apply(br2, U, p), ref, rtol=1e-12, atol=1e-12 * float(ref.abs().max()))
        assert torch.allclose(O.apply(ip, U, p), ref, rtol=1e-12, atol=1e-12 * float(ref.abs().max()))
    q = no_reaction_params(chemotaxis=False)
    for flux, pen in (("br2", 5.0), ("sipg", 3.0)):
        mesh = O.Mesh(2, (4, 3), (1.0, 0.2), (1, 0), 1, flux=flux, penalty=pen)
        n = mesh.E * 6 * mesh.nb
        B = mesh.vol * torch.func.jacfwd(lambda V: O.apply(mesh, V, q))(torch.zeros(mesh.E, 6, mesh.nb, dtype=F64)).reshape(n, n)
        assert torch.allclose(B, B.T, atol=1e-12 * float(B.abs().max()))
        ev = torch.linalg.eigvalsh(0.5 * (B + B.T))
        assert float(ev.max()) < 1e-10 * float(ev.abs().max())
        assert int((ev.abs() < 1e-9 * float(ev.abs().max())).sum()) == 6
