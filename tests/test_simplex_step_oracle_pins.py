"""Pins of the oracle's SDIRK step on simplicial meshes (``step`` of
oracle/cdg2_tri_oracle.py, Sec. 3.2) against what the mathematics fixes:
for a linear operator (pure diffusion) one step is the solution of the whole
stage system as one block linear system, K = (I - dt A (x) J)^{-1} (1 (x) J U),
U_{n+1} = U + dt sum_i b_i K_i (so every tableau entry is checked); for the
full nonlinear model, the step agrees with the Taylor expansion
U + dt f + dt^2/2 J f to third order in dt (halving dt divides the remainder by
8 for every scheme of order >= 2)."""
import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from oracle import cdg2_tet_oracle as TT
from oracle import cdg2_tri_oracle as T

F64 = torch.float64


def diffusion_only(p):
    q = dict(p)
    q["chi0"] = (0.0, 0.0, 0.0, 0.0)
    for key in ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox", "beta1", "beta2", "sigma"):
        q[key] = 0.0
    return q


def block_step(apply, U, dt, scheme):
    A, b, _ = O.sdirk_tableau(scheme)
    s, n = len(b), U.numel()
    J = torch.func.jacrev(apply)(U).reshape(n, n)
    big = torch.eye(s * n, dtype=F64) - dt * torch.kron(torch.from_numpy(A), J)
    K = torch.linalg.solve(big, (J @ U.reshape(-1)).repeat(s)).reshape(s, n)
    return U + dt * (torch.from_numpy(b) @ K).reshape(U.shape)


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk3", "sdirk4"])
def test_linear_triangle_step_is_the_block_solution(scheme):
    xy, tri = I.tri_mesh(3, 2, 1.0, 0.2, 0.2, 5)
    m = T.TriMesh(xy, tri, 1)
    p = diffusion_only(I.default_params())
    U = torch.from_numpy(I.random_coefficients(m.E, m.nb, 8, 0.2))
    dt = 2e-3
    got = T.step(m, U, p, dt, scheme)
    ref = block_step(lambda V: T.apply(m, V, p), U, dt, scheme)
    assert float((got - ref).norm() / (ref - U).norm()) <= 1e-10


def test_linear_tetrahedral_step_is_the_block_solution():
    xyz, tet = I.tet_mesh(2, 1, 1, 1.0, 0.2, 0.2, 0.15, 4)
    m = TT.TetMesh(xyz, tet, 1)
    p = diffusion_only(I.default_params())
    U = torch.from_numpy(I.random_coefficients(m.E, m.nb, 9, 0.2))
    dt = 2e-3
    got = TT.step(m, U, p, dt, "sdirk3")
    ref = block_step(lambda V: TT.apply(m, V, p), U, dt, "sdirk3")
    assert float((got - ref).norm() / (ref - U).norm()) <= 1e-10


@pytest.mark.parametrize("scheme", ["sdirk2", "sdirk3", "sdirk4"])
def test_step_matches_the_taylor_expansion_to_second_order(scheme):
    xy, tri = I.tri_mesh(3, 2, 1.0, 0.2, 0.2, 5)
    m = T.TriMesh(xy, tri, 1)
    p = I.default_params()
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    cen, amp = I.gaussian_draws(2, (1.0, 0.2), 4, 7)
    U0 = T.project(m, lambda x: O.gaussian_field(m, x, cen, amp, 0.2, 0.05))
    f0 = T.apply(m, U0, p)
    Jf = T.jvp(m, U0, f0, p)
    rem = []
    for dt in (4e-4, 2e-4, 1e-4):
        U1 = T.step(m, U0, p, dt, scheme)
        rem.append(float((U1 - U0 - dt * f0 - 0.5 * dt * dt * Jf).norm()))
    # a first-order slip (a wrong b_i or a_ij, a stage at the wrong point) gives ratio 4
    assert 7.0 <= rem[0] / rem[1] <= 9.0 and 7.0 <= rem[1] / rem[2] <= 9.0, rem
