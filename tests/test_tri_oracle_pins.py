"""Pins of the triangle oracle (oracle/cdg2_tri_oracle.py) against what the
mathematics fixes, independent of the oracle's own code paths: Jacobi values
from scipy, exact monomial integrals on the reference triangle, the span and
orthonormality of the basis, finite-difference gradients, the source-only
operator of constant states, the exact weak Laplacian of a polynomial with
zero normal derivative, symmetry / semi-definiteness / null space of pure
CDG2 diffusion, conservation, the smaller-area K^- rule (Sec. 3.1), and
invariance under a cyclic relabelling of every triangle's vertices (which
changes every basis function and edge orientation but not the DG space)."""
import math

import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from oracle import cdg2_tri_oracle as T

F64 = torch.float64


def mesh(nx=4, ny=2, k=2, jitter=0.2, seed=3):
    xy, tri = I.tri_mesh(nx, ny, 1.0, 0.2, jitter, seed)
    return T.TriMesh(xy, tri, k)


def test_jacobi_matches_scipy():
    special = pytest.importorskip("scipy.special")
    x = torch.linspace(-1, 1, 17, dtype=F64)
    for n in range(6):
        for alpha in (0.0, 1.0, 3.0, 5.0, 7.0):
            ref = special.eval_jacobi(n, alpha, 0.0, x.numpy())
            assert np.abs(T.jacobi(n, alpha, x).numpy() - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("k", [1, 2, 3])
def test_triangle_rule_integrates_monomials_exactly(k):
    pts, w = T.triangle_rule(k + 2)
    assert abs(float(w.sum()) - 0.5) < 1e-15
    for a in range(2 * k + 3):
        for b in range(2 * k + 3 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = float((w * pts[:, 0] ** a * pts[:, 1] ** b).sum())
            assert abs(got - exact) <= 1e-14, (a, b)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_dubiner_basis_is_an_orthonormal_basis_of_pk(k):
    pts, w = T.triangle_rule(k + 2)
    psi, _ = T.dubiner(k, pts)
    nb = (k + 1) * (k + 2) // 2
    assert psi.shape[1] == nb
    gram = torch.einsum("q,qi,qj->ij", w, psi, psi)
    assert float((gram - torch.eye(nb, dtype=F64)).abs().max()) <= 1e-13
    # every psi_i is a polynomial of total degree <= k: exact fit by monomials at random points
    rng = np.random.default_rng(k)
    r = rng.random((40, 2))
    r = r[r.sum(1) < 1.0][:30]
    X = torch.tensor(r, dtype=F64)
    mono = torch.stack([X[:, 0] ** a * X[:, 1] ** b for a in range(k + 1) for b in range(k + 1 - a)], dim=1)
    P, _ = T.dubiner(k, X)
    coef = torch.linalg.lstsq(mono, P).solution
    assert float((mono @ coef - P).abs().max()) <= 1e-11
    assert torch.linalg.matrix_rank(P) == nb


def test_dubiner_gradients_match_central_differences():
    k, h = 3, 1e-6
    X = torch.tensor([[0.2, 0.3], [0.6, 0.1], [0.05, 0.8], [1 / 3, 1 / 3]], dtype=F64)
    _, d = T.dubiner(k, X)
    for j in range(2):
        e = torch.zeros(2, dtype=F64)
        e[j] = h
        fd = (T.dubiner(k, X + e)[0] - T.dubiner(k, X - e)[0]) / (2 * h)
        assert float((fd - d[j]).abs().max()) <= 1e-7


def test_constant_state_gives_the_source_only():
    m = mesh(k=2)
    p = I.default_params()
    p["sigma"] = 0.0                                  # no c2 influx on Gamma_{1,in}
    c = torch.tensor([0.3, 0.2, 0.4, 0.005, 0.6, 0.7], dtype=F64)   # c1 below both thresholds
    U = torch.zeros(m.E, 6, m.nb, dtype=F64)
    U[:, :, 0] = c / math.sqrt(2.0)                   # psi_0 = sqrt(2) on T
    f = T.apply(m, U, p)
    S = O.source_S(c[:, None], O.param_vector(p))[:, 0]
    ref = torch.zeros_like(f)
    ref[:, :, 0] = S / math.sqrt(2.0)
    assert float((f - ref).abs().max()) <= 1e-13


def diffusion_only(p):
    q = dict(p)
    q["chi0"] = (0.0, 0.0, 0.0, 0.0)
    for key in ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox", "beta1", "beta2", "sigma"):
        q[key] = 0.0
    return q


def test_weak_laplacian_of_a_neumann_cubic_is_exact():
    """u_s = a_s + b_s x^2 (3 L_x - 2 x) + c_s y^2 (3 L_y - 2 y) has zero normal
    derivative on the rectangle and lies in P_3: all jumps vanish and
    <phi_i, L_h U> = int_K A_s lap(u_s) phi_i exactly."""
    m = mesh(nx=5, ny=3, k=3)
    p = diffusion_only(I.default_params())
    Lx, Ly = 1.0, 0.2
    rng = np.random.default_rng(11)
    a, b, c = (torch.tensor(rng.random(6), dtype=F64) for _ in range(3))

    def u(x):
        X, Y = x[..., 0], x[..., 1]
        return torch.stack([a[s] + b[s] * X ** 2 * (3 * Lx - 2 * X) + c[s] * Y ** 2 * (3 * Ly - 2 * Y)
                            for s in range(6)])

    U = T.project(m, u)
    pv = O.param_vector(p)
    R = T.apply_residual(m, U, pv)
    scale = float(T.volume_residual(m, U, pv).abs().max())   # the terms that cancel into the result
    x = m.qpoints_phys()
    lap = torch.stack([b[s] * (6 * Lx - 12 * x[..., 0]) + c[s] * (6 * Ly - 12 * x[..., 1]) for s in range(6)])
    A = O.diffusivity(O.param_vector(p))
    ref = torch.einsum("eq,seq,qi->esi", m.det[:, None] * m.qw[None], A[:, None, None] * lap, m.phi)
    assert float((R - ref).abs().max()) <= 1e-12 * scale


def test_pure_diffusion_is_symmetric_negative_semidefinite_with_constant_kernel():
    m = mesh(nx=3, ny=2, k=2)
    p = O.param_vector(diffusion_only(I.default_params()))
    U = torch.from_numpy(I.random_coefficients(m.E, m.nb, 4, 0.1))
    n = U.numel()
    J = torch.func.jacrev(lambda V: T.apply_residual(m, V, p))(U).reshape(n, n)
    assert float((J - J.T).abs().max()) <= 1e-12 * float(J.abs().max())
    ev = torch.linalg.eigvalsh(0.5 * (J + J.T))
    scale = float(ev.abs().max())
    assert float(ev.max()) <= 1e-12 * scale
    assert int((ev.abs() <= 1e-10 * scale).sum()) == 6          # one constant per species


def test_diffusion_and_chemotaxis_conserve_every_species():
    m = mesh(nx=4, ny=2, k=2)
    p = dict(I.default_params())
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    for key in ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox", "beta1", "beta2", "sigma"):
        p[key] = 0.0
    U = torch.from_numpy(I.random_coefficients(m.E, m.nb, 5, 0.1))
    R = T.apply_residual(m, U, O.param_vector(p))
    total = R[:, :, 0].sum(0)                        # psi_0 is constant: the integral of L_h
    assert float(total.abs().max()) <= 1e-13 * float(R.abs().max())


def test_k_minus_is_the_smaller_element():
    m = mesh(nx=6, ny=3, k=1, jitter=0.2, seed=9)
    for eM, _, eP, _ in m.interior:
        aM, aP = float(m.area[eM]), float(m.area[eP])
        tie = abs(aM - aP) <= 1e-12 * max(aM, aP)   # boundary triangles sharing an apex tie exactly
        assert (aM < aP and not tie) or (tie and eM < eP)
    u = mesh(nx=3, ny=2, k=1, jitter=0.0)
    assert all(eM < eP for eM, _, eP, _ in u.interior)  # equal areas: the lower index


def test_invariant_under_cyclic_relabelling_of_vertices():
    """The collapsed rule sits differently in a relabelled triangle, so only
    integrands the rule integrates exactly are invariant: chemotaxis off
    (its sensitivities are rational), k = 2 (volume degree <= 6 = 2k + 2),
    no Heaviside data."""
    xy, tri = I.tri_mesh(4, 2, 1.0, 0.2, 0.2, 13)
    rot = np.stack([tri[:, 1], tri[:, 2], tri[:, 0]], axis=1)
    k = 2
    m1, m2 = T.TriMesh(xy, tri, k), T.TriMesh(xy, rot, k)
    p = dict(I.default_params())
    p["chi0"] = (0.0, 0.0, 0.0, 0.0)
    p["beta1"] = p["beta2"] = 0.0

    # a discontinuous DG field on the first labelling, moved exactly (same P_k) to the second basis
    U1 = torch.from_numpy(I.random_coefficients(m1.E, m1.nb, 21, 0.2))
    x = m2.qpoints_phys()
    vals = torch.stack([T.dubiner(k, m1.ref_coords(e, x[e]))[0] @ U1[e].T for e in range(m1.E)])   # (E, Q, 6)
    U2 = T.minv(m2, torch.einsum("eq,eqs,qi->esi", m2.det[:, None] * m2.qw[None], vals, m2.phi))
    f1 = T.apply(m1, U1, p)
    f2 = T.apply(m2, U2, p)
    # compare the resulting functions at the barycentric points of each element
    bary = torch.tensor([[1 / 3, 1 / 3], [0.2, 0.6], [0.6, 0.2], [0.1, 0.1]], dtype=F64)
    for e in range(m1.E):
        x = m1.x0[e] + bary @ m1.J[e].T
        v1 = T.dubiner(k, m1.ref_coords(e, x))[0] @ f1[e].T
        v2 = T.dubiner(k, m2.ref_coords(e, x))[0] @ f2[e].T
        assert float((v1 - v2).abs().max()) <= 1e-11 * float(f1.abs().max())


def test_jvp_matches_central_differences():
    m = mesh(nx=3, ny=2, k=2)
    p = dict(I.default_params())
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    U = torch.from_numpy(I.random_coefficients(m.E, m.nb, 6, 0.05))
    dU = torch.from_numpy(np.random.default_rng(2).standard_normal(U.shape))
    h = 1e-6
    fd = (T.apply(m, U + h * dU, p) - T.apply(m, U - h * dU, p)) / (2 * h)
    jv = T.jvp(m, U, dU, p)
    assert float((fd - jv).norm() / jv.norm()) <= 1e-6
