"""Pin of the oracle's local Lax-Friedrichs convective flux (Sec. 3.1).

The paper names the convective flux only as "local Lax-Friedrichs".  The
reading taken by the oracle (and by the kernels) is, per chemotactic species
s in {n1, n2} with F_s = U_s v_s:

    F^_s . n^- = 1/2 (U_s^- v_s^- + U_s^+ v_s^+) . n^- + 1/2 lambda_s Delta_s,
    lambda_s   = max(|v_s^- . n^-|, |v_s^+ . n^-|),   Delta_s = U_s^- - U_s^+,

each side's velocity taken from its own broken gradient, and, for the
derivative, d|x|/dx = sign(x) with the K^- side taken at a tie.

The mesh is two Q1 cells side by side along x (no periodicity), so there is
one interior face, x = h.  Diffusion, reactions and inflows are off, so the
face term reduces to -F^ . n^- (phi^- - phi^+).  The fields are polynomials
of x alone that Q1 holds exactly: their traces and normal derivatives at the
face are known in closed form, the face quadrature integrates the constant
integrand exactly, and

    int_e phi_i^- = |e| psi_a(1) delta_{b0},   int_e phi_i^+ = |e| psi_a(0) delta_{b0}

for the mode i = (a, b) (psi_a(1) = sqrt(2a+1), psi_a(0) = (-1)^a sqrt(2a+1)).
The expected face residual is written from these closed forms, not from the
oracle's code.  Each test case is also checked to separate the reading from
the plausible mistakes (min for max, a dropped 1/2, the upwind sign flipped,
lambda from one side only, the tie derivative taken on K^+): had the oracle
made one of them, its residual would differ from the expected one by far
more than the tolerance.
"""
import math

import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O

F64 = torch.float64
H = 0.5          # cell width along x
LY = 0.2         # face length (the single cell along y)
CHI0 = (0.4, 0.25, 0.3, 0.2)
CHITH = (0.1, 0.2, 0.15, 0.3)
S3 = math.sqrt(3.0)


def _params():
    p = I.default_params()
    for key in ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox", "beta1", "beta2", "sigma"):
        p[key] = 0.0
    p["mu"] = (0.0, 0.0, 0.0)
    p["nu"] = (0.0, 0.0, 0.0)
    p["chi0"] = CHI0
    p["chith"] = CHITH
    return O.param_vector(p)


def _mesh():
    return O.Mesh(2, (2, 1), (2 * H, LY), (False, False), 1)


def _linear_coeffs(trace, slope, minus):
    """Q1 coefficients (modes (0,0), (1,0)) of u = trace + slope (x - H) on K^- (minus) or K^+."""
    # K^-: xi = x / H, u = trace - slope H + slope H xi; K^+: xi = (x - H) / H, u = trace + slope H xi
    mean = trace - slope * H / 2 if minus else trace + slope * H / 2
    return mean, slope * H / (2 * S3)       # psi_1(xi) = sqrt(3) (2 xi - 1)


def _state(n1, n2, c1, c3):
    """U (2 cells, 6 species, 4 modes) from per-side (trace, slope) pairs of n1, n2, c1, c3.

    Each argument is ((trace^-, slope^-), (trace^+, slope^+)); n3 and c2 are zero."""
    U = torch.zeros(2, 6, 4, dtype=F64)
    for s, f in ((0, n1), (1, n2), (3, c1), (5, c3)):
        for cell, minus in ((0, True), (1, False)):
            m0, m1 = _linear_coeffs(*f[cell], minus)
            U[cell, s, 0] = m0
            U[cell, s, 1] = m1
    return U


def _velocities(n1, c1, c3, side):
    """Closed-form normal velocities (v_n1 . n, v_n2 . n) on one side (0: K^-, 1: K^+), n = +e_x."""
    (n1t, n1s), (c1t, c1s), (c3t, c3s) = n1[side], c1[side], c3[side]
    v1 = CHI0[0] / (c1t + CHITH[0]) * c1s + CHI0[1] / (c3t + CHITH[1]) * c3s
    v2 = CHI0[2] / (c1t + CHITH[2]) * c1s - CHI0[3] / (n1t + CHITH[3]) * n1s
    return v1, v2


def _llf(uM, vM, uP, vP, lam_rule="max", half=0.5, upwind=1.0):
    if lam_rule == "max":
        lam = max(abs(vM), abs(vP))
    elif lam_rule == "min":
        lam = min(abs(vM), abs(vP))
    elif lam_rule == "minus":
        lam = abs(vM)
    else:
        lam = abs(vP)
    return 0.5 * (uM * vM + uP * vP) + upwind * half * lam * (uM - uP)


def _face_residual_from_fluxes(Fh):
    """Expected face residual (2, 6, 4) for the face fluxes Fh[s] (s = n1, n2)."""
    R = torch.zeros(2, 6, 4, dtype=F64)
    for s in (0, 1):
        for a in (0, 1):
            psi1 = math.sqrt(2 * a + 1)
            psi0 = (-1) ** a * psi1
            R[0, s, a] = -Fh[s] * LY * psi1           # mode (a, 0) of K^-: -F^ int_e phi^-
            R[1, s, a] = Fh[s] * LY * psi0            # mode (a, 0) of K^+: +F^ int_e phi^+
    return R


# (n1, n2, c1, c3): per side (trace, slope).  c1 and c3 are continuous with a
# kink, n1 and n2 jump.  The cases put the larger |v . n| on K^- for one
# species and on K^+ for the other, with equal and opposite signs of v.
CASES = {
    "minus_faster": (((0.9, 0.3), (0.4, -0.2)), ((0.6, 0.0), (0.25, 0.0)),
                     ((0.7, 2.0), (0.7, 0.5)), ((0.5, 0.3), (0.5, -0.1))),
    "plus_faster": (((0.3, -0.4), (0.8, 0.6)), ((0.2, 0.0), (0.7, 0.0)),
                    ((0.45, -0.4), (0.45, 1.5)), ((0.35, 0.2), (0.35, 0.9))),
    "opposite_signs": (((1.1, 0.0), (0.5, 0.0)), ((0.9, 0.0), (0.3, 0.0)),
                       ((0.6, 1.0), (0.6, -2.0)), ((0.4, -0.5), (0.4, 0.25))),
}

MUTANTS = {
    "min for max": dict(lam_rule="min"),
    "dropped 1/2 on lambda": dict(half=1.0),
    "upwind sign flipped": dict(upwind=-1.0),
    "lambda from K^- only": dict(lam_rule="minus"),
    "lambda from K^+ only": dict(lam_rule="plus"),
}


def _expected(case, **mut):
    n1, n2, c1, c3 = case
    Fh = []
    for s, u in ((0, n1), (1, n2)):
        vM = _velocities(n1, c1, c3, 0)[s]
        vP = _velocities(n1, c1, c3, 1)[s]
        Fh.append(_llf(u[0][0], vM, u[1][0], vP, **mut))
    return _face_residual_from_fluxes(Fh)


@pytest.mark.parametrize("name", sorted(CASES))
def test_llf_face_flux_closed_form(name):
    case = CASES[name]
    R = O.face_residual(_mesh(), _state(*case), _params())
    want = _expected(case)
    scale = float(want.abs().max())
    assert scale > 1e-3
    assert float((R - want).abs().max()) <= 1e-14 * scale, (R, want)


def test_llf_cases_separate_the_plausible_mistakes():
    """Every mutant of the flux formula misses at least one case by > 1e-3 of its size."""
    for mname, mut in MUTANTS.items():
        worst = 0.0
        for case in CASES.values():
            want = _expected(case)
            got = _expected(case, **mut)
            worst = max(worst, float((got - want).abs().max() / want.abs().max()))
        assert worst > 1e-3, mname


def _tie_state():
    """n1 = nT + p |x - H| (a symmetric V: equal traces, opposite slopes), c1 and c3 constant, n2 jumps.

    Then v_n2 . n = -kappa22(nT) d_x n1 is exactly opposite on the two sides
    (the traces agree bit for bit), a tie of the LLF maximum."""
    nT, p = 0.6, 0.8
    return (((nT, -p), (nT, p)), ((0.9, 0.0), (0.2, 0.0)), ((0.5, 0.0), (0.5, 0.0)), ((0.3, 0.0), (0.3, 0.0)))


@pytest.mark.parametrize("cell", [0, 1])
def test_llf_tie_derivative_takes_the_minus_side(cell):
    """At |v^- . n| = |v^+ . n| the derivative of lambda is sign(v^-) dv^- (reading c11),
    checked for a tangent that moves only K^-'s n1 slope and one that moves only K^+'s."""
    case = _tie_state()
    mesh, pv = _mesh(), _params()
    U = _state(*case)
    R = O.face_residual(mesh, U, pv)
    vM = _velocities(case[0], case[2], case[3], 0)[1]
    vP = _velocities(case[0], case[2], case[3], 1)[1]
    assert vM == -vP and vM != 0.0
    assert torch.allclose(R, _expected(case), rtol=0, atol=1e-14)
    dU = torch.zeros_like(U)
    dU[cell, 0, 1] = 1.0                        # d(slope of n1) = 2 sqrt(3) / H on that cell
    _, dR = torch.func.jvp(lambda V: O.face_residual(mesh, V, pv), (U,), (dU,))
    dslope = 2 * S3 / H
    kap = CHI0[3] / (case[0][cell][0] + CHITH[3])
    # a mode-(1,0) tangent also moves n1's trace at the face, by psi_1(1) = sqrt(3) on K^-
    # and psi_1(0) = -sqrt(3) on K^+, and kappa22(n1) moves with it
    dtrace = S3 if cell == 0 else -S3
    slope = case[0][cell][1]
    dv = -kap * dslope + kap / (case[0][cell][0] + CHITH[3]) * dtrace * slope
    (mA, _), (mB, _) = case[1]
    dvM, dvP = (dv, 0.0) if cell == 0 else (0.0, dv)
    dlam_minus_rule = math.copysign(1.0, vM) * dvM
    dlam_plus_rule = math.copysign(1.0, vP) * dvP

    def dF(dlam):
        return 0.5 * (mA * dvM + mB * dvP) + 0.5 * dlam * (mA - mB)    # n2 does not move: dDelta = 0

    want = _face_residual_from_fluxes([0.0, dF(dlam_minus_rule)])
    other = _face_residual_from_fluxes([0.0, dF(dlam_plus_rule)])
    # species n1 has v = 0 on both sides (c1, c3 constant): its flux derivative vanishes
    assert float((dR - want).abs().max()) <= 1e-13 * float(want.abs().max()), (dR, want)
    assert float((other - want).abs().max()) > 1e-3 * float(want.abs().max())
