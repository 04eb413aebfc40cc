"""Pins of the tetrahedral oracle (oracle/cdg2_tet_oracle.py) against what the
mathematics fixes: exact monomial integrals on the reference tetrahedron,
span and orthonormality of the 3D Dubiner basis, finite-difference
gradients, the source-only operator of constant states, the exact weak
Laplacian of a polynomial with zero normal derivative on the box, symmetry /
semi-definiteness / null space of pure diffusion, conservation, the
smaller-volume K^- rule (Sec. 3.1), invariance under an orientation-
preserving relabelling of every tetrahedron's vertices, JVP against central
differences."""
import math

import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from oracle import cdg2_tet_oracle as TT
from oracle import cdg2_tri_oracle as T

F64 = torch.float64


def mesh(nx=2, ny=2, nz=1, k=2, jitter=0.15, seed=3):
    xyz, tet = I.tet_mesh(nx, ny, nz, 1.0, 0.2, 0.2, jitter, seed)
    return TT.TetMesh(xyz, tet, k)


def diffusion_only(p):
    q = dict(p)
    q["chi0"] = (0.0, 0.0, 0.0, 0.0)
    for key in ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox", "beta1", "beta2", "sigma"):
        q[key] = 0.0
    return q


@pytest.mark.parametrize("k", [1, 2, 3])
def test_tet_rule_integrates_monomials_exactly(k):
    pts, w = TT.tet_rule(k + 2)
    assert abs(float(w.sum()) - 1.0 / 6.0) < 1e-15
    for a in range(2 * k + 2):
        for b in range(2 * k + 2 - a):
            for c in range(2 * k + 2 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                got = float((w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c).sum())
                assert abs(got - exact) <= 1e-15, (a, b, c)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_dubiner3_is_an_orthonormal_basis_of_pk(k):
    pts, w = TT.tet_rule(k + 2)
    psi, _ = TT.dubiner3(k, pts)
    nb = (k + 1) * (k + 2) * (k + 3) // 6
    assert psi.shape[1] == nb
    gram = torch.einsum("q,qi,qj->ij", w, psi, psi)
    assert float((gram - torch.eye(nb, dtype=F64)).abs().max()) <= 1e-13
    rng = np.random.default_rng(k)
    r = rng.random((200, 3))
    r = r[r.sum(1) < 1.0][:60]
    X = torch.tensor(r, dtype=F64)
    mono = torch.stack([X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c for a in range(k + 1) for b in range(k + 1 - a)
                        for c in range(k + 1 - a - b)], dim=1)
    P, _ = TT.dubiner3(k, X)
    coef = torch.linalg.lstsq(mono, P).solution
    assert float((mono @ coef - P).abs().max()) <= 1e-10
    assert torch.linalg.matrix_rank(P) == nb


def test_dubiner3_gradients_match_central_differences():
    k, h = 3, 1e-6
    X = torch.tensor([[0.2, 0.3, 0.1], [0.6, 0.1, 0.2], [0.05, 0.1, 0.7], [0.25, 0.25, 0.25]], dtype=F64)
    _, d = TT.dubiner3(k, X)
    for j in range(3):
        e = torch.zeros(3, dtype=F64)
        e[j] = h
        fd = (TT.dubiner3(k, X + e)[0] - TT.dubiner3(k, X - e)[0]) / (2 * h)
        assert float((fd - d[j]).abs().max()) <= 1e-6


def test_constant_state_gives_the_source_only():
    m = mesh(k=1)
    p = I.default_params()
    p["sigma"] = 0.0
    c = torch.tensor([0.3, 0.2, 0.4, 0.005, 0.6, 0.7], dtype=F64)
    U = torch.zeros(m.E, 6, m.nb, dtype=F64)
    U[:, :, 0] = c / math.sqrt(6.0)                  # psi_0 = sqrt(6) on T
    f = TT.apply(m, U, p)
    S = O.source_S(c[:, None], O.param_vector(p))[:, 0]
    ref = torch.zeros_like(f)
    ref[:, :, 0] = S / math.sqrt(6.0)
    assert float((f - ref).abs().max()) <= 1e-13


def test_weak_laplacian_of_a_neumann_cubic_is_exact():
    """u_s = a_s + b_s x^2 (3 Lx - 2x) + c_s y^2 (3 Ly - 2y) + d_s z^2 (3 Lz - 2z):
    zero normal derivative on the box, in P_3: <phi_i, L_h U> = int_K A_s lap(u_s) phi_i."""
    m = mesh(nx=2, ny=1, nz=1, k=3)
    p = diffusion_only(I.default_params())
    L = (1.0, 0.2, 0.2)
    rng = np.random.default_rng(11)
    a, b, c, d = (torch.tensor(rng.random(6), dtype=F64) for _ in range(4))
    co = (b, c, d)

    def u(x):
        return torch.stack([a[s] + sum(co[j][s] * x[..., j] ** 2 * (3 * L[j] - 2 * x[..., j]) for j in range(3))
                            for s in range(6)])

    U = TT.project(m, u)
    pv = O.param_vector(p)
    R = T.apply_residual(m, U, pv)
    scale = max(float(T.volume_residual(m, U, pv).abs().max()), float(T.face_residual(m, U, pv).abs().max()))
    x = m.qpoints_phys()
    lap = torch.stack([sum(co[j][s] * (6 * L[j] - 12 * x[..., j]) for j in range(3)) for s in range(6)])
    A = O.diffusivity(pv)
    ref = torch.einsum("eq,seq,qi->esi", m.det[:, None] * m.qw[None], A[:, None, None] * lap, m.phi)
    # (125-point sums of products much larger than the result: rounding ~1e-12 of the scale;
    # a missing or wrong term would show at O(1))
    assert float((R - ref).abs().max()) <= 1e-11 * scale


def test_pure_diffusion_is_symmetric_negative_semidefinite_with_constant_kernel():
    m = mesh(nx=2, ny=1, nz=1, k=1)
    p = O.param_vector(diffusion_only(I.default_params()))
    U = torch.from_numpy(I.random_coefficients(m.E, m.nb, 4, 0.1))
    n = U.numel()
    J = torch.func.jacrev(lambda V: T.apply_residual(m, V, p))(U).reshape(n, n)
    assert float((J - J.T).abs().max()) <= 1e-12 * float(J.abs().max())
    ev = torch.linalg.eigvalsh(0.5 * (J + J.T))
    scale = float(ev.abs().max())
    assert float(ev.max()) <= 1e-12 * scale
    assert int((ev.abs() <= 1e-10 * scale).sum()) == 6


def test_diffusion_and_chemotaxis_conserve_every_species():
    m = mesh(k=2)
    p = dict(I.default_params())
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    for key in ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox", "beta1", "beta2", "sigma"):
        p[key] = 0.0
    U = torch.from_numpy(I.random_coefficients(m.E, m.nb, 5, 0.1))
    R = T.apply_residual(m, U, O.param_vector(p))
    assert float(R[:, :, 0].sum(0).abs().max()) <= 1e-13 * float(R.abs().max())


def test_k_minus_is_the_smaller_element():
    m = mesh(nx=3, ny=2, nz=2, k=1, jitter=0.15, seed=9)
    for eM, _, eP, _ in m.interior:
        vM, vP = float(m.area[eM]), float(m.area[eP])
        tie = abs(vM - vP) <= 1e-12 * max(vM, vP)
        assert (vM < vP and not tie) or (tie and eM < eP)


def test_invariant_under_even_relabelling_of_vertices():
    """An even permutation keeps each tetrahedron positively oriented; the
    collapsed rules then sit differently, so only exactly integrated
    integrands are compared: chemotaxis off, linear sources, no Heaviside
    data and no Gamma_{1,in} influx (its indicator is discontinuous and a
    boundary face's points follow its own vertex order), k = 1."""
    xyz, tet = I.tet_mesh(2, 2, 1, 1.0, 0.2, 0.2, 0.15, 13)
    rot = tet[:, [1, 2, 0, 3]]
    k = 1
    m1, m2 = TT.TetMesh(xyz, tet, k), TT.TetMesh(xyz, rot, k)
    p = dict(I.default_params())
    p["chi0"] = (0.0, 0.0, 0.0, 0.0)
    p["alpha1"] = p["alpha2"] = 0.0
    p["beta1"] = p["beta2"] = p["sigma"] = 0.0
    U1 = torch.from_numpy(I.random_coefficients(m1.E, m1.nb, 21, 0.2))
    x = m2.qpoints_phys()
    vals = torch.stack([TT.dubiner3(k, m1.ref_coords(e, x[e]))[0] @ U1[e].T for e in range(m1.E)])
    U2 = T.minv(m2, torch.einsum("eq,eqs,qi->esi", m2.det[:, None] * m2.qw[None], vals, m2.phi))
    f1, f2 = TT.apply(m1, U1, p), TT.apply(m2, U2, p)
    bary = torch.tensor([[0.25, 0.25, 0.25], [0.1, 0.2, 0.3], [0.5, 0.1, 0.1]], dtype=F64)
    for e in range(m1.E):
        xe = m1.x0[e] + bary @ m1.J[e].T
        v1 = TT.dubiner3(k, m1.ref_coords(e, xe))[0] @ f1[e].T
        v2 = TT.dubiner3(k, m2.ref_coords(e, xe))[0] @ f2[e].T
        assert float((v1 - v2).abs().max()) <= 1e-11 * float(f1.abs().max())


def test_jvp_matches_central_differences():
    m = mesh(k=1)
    p = dict(I.default_params())
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    U = torch.from_numpy(I.random_coefficients(m.E, m.nb, 6, 0.05))
    dU = torch.from_numpy(np.random.default_rng(2).standard_normal(U.shape))
    h = 1e-6
    fd = (TT.apply(m, U + h * dU, p) - TT.apply(m, U - h * dU, p)) / (2 * h)
    jv = TT.jvp(m, U, dU, p)
    assert float((fd - jv).norm() / jv.norm()) <= 1e-6
