"""cdg2_step (SDIRK + Newton + GMRES on the GPU) against the oracle's step.

Bars (from the method): FP64 steps and mixed FP32-Krylov steps with FP64
refinement agree with the oracle to 1e-10 relative when both solve their
Newton systems to ~1e-13; the manufactured solution converges at order k+1
in L2 through the GPU stepper; failure paths are exercised by host-side
injections (a NaN in the input state, an iteration cap) and return status
codes.
"""
import math

import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from helpers import gaussian_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


def _pair(G, dim, cells, k):
    ext = (1.0, 0.2, 0.2)
    per = (1, 0, 0) if dim == 2 else (1, 0, 1)
    return O.Mesh(dim, cells, ext, per, k), G.cdg2_mesh_create(dim, cells, ext, per, k)


def _rel(a, b):
    return float((a.cpu() - b).norm() / b.norm())


def _tight(G, scheme, mixed):
    return G.make_opts(scheme=scheme, mixed=mixed, max_newton=30, gmres_restart=40, max_gmres=800,
                       newton_rtol=1e-14, newton_atol=1e-15, gmres_rtol=1e-6 if mixed else 1e-10)


_ORACLE_RUNS = {}


def _oracle_steps(om, U0, p, dt, nsteps, name):
    key = (name, nsteps, dt)
    if key not in _ORACLE_RUNS:
        ref = U0.clone()
        for i in range(nsteps):
            ref = O.step(om, ref, p, i * dt, dt, name)
        _ORACLE_RUNS[key] = ref
    return _ORACLE_RUNS[key]


@pytest.mark.parametrize("scheme,name", [(2, "sdirk2"), (3, "sdirk3")])
@pytest.mark.parametrize("mixed", [False, True])
def test_step_matches_oracle(G, scheme, name, mixed):
    om, gm = _pair(G, 2, (8, 2), 2)
    p = I.default_params()
    U0 = gaussian_state(om, sigma=0.1, seed=1157)
    dt, nsteps = 1e-3, 3
    ref = _oracle_steps(om, U0, p, dt, nsteps, name)
    U = U0.clone().cuda()
    for i in range(nsteps):
        rc, st = G.cdg2_step(gm, p, U, i * dt, dt, _tight(G, scheme, mixed))
        assert rc == 0 and st["newton_iters"] >= 1
    assert _rel(U, ref) <= 1e-10


def test_step_3d_matches_oracle(G):
    om, gm = _pair(G, 3, (4, 2, 2), 1)
    p = I.default_params()
    U0 = gaussian_state(om, sigma=0.1, seed=3)
    ref = O.step(om, U0.clone(), p, 0.0, 2e-3, "sdirk2")
    U = U0.clone().cuda()
    rc, _ = G.cdg2_step(gm, p, U, 0.0, 2e-3, _tight(G, 2, True))
    assert rc == 0 and _rel(U, ref) <= 1e-10


def test_mixed_and_fp64_agree_on_workload0(G):
    w = I.workload(0)
    om, gm = _pair(G, w.dim, w.cells, w.k)
    p = I.default_params()
    U0 = gaussian_state(om, w.n_gauss, w.sigma, w.floor, w.seed).cuda()
    res = {}
    for mixed in (False, True):
        U = U0.clone()
        for i in range(w.steps):
            rc, st = G.cdg2_step(gm, p, U, i * w.dt, w.dt, G.make_opts(scheme=2, mixed=mixed, newton_rtol=1e-12,
                                                                        gmres_rtol=1e-4))
            assert rc == 0
        res[mixed] = U
    assert float((res[True] - res[False]).norm() / res[False].norm()) <= 1e-10


@pytest.mark.parametrize("k", [2])
def test_mms_convergence_through_gpu_steps(G, k):
    """U*(t) is the exact solution with the forcing on; the GPU stepper's L2
    error after a few small SDIRK3 steps converges at order k+1 in h."""
    p = I.default_params()
    p["beta1"] = p["beta2"] = p["sigma"] = 0.0
    ph = I.mms_phases(1158)
    pp = G.make_params(p, ph)
    errs = []
    T, nsteps = 2e-3, 4
    for n in (8, 16, 32):
        om, gm = _pair(G, 2, (n, n // 4), k)
        U = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
        G.cdg2_project_mms(gm, pp, 0.0, U)
        for i in range(nsteps):
            rc, _ = G.cdg2_step(gm, pp, U, i * T / nsteps, T / nsteps,
                                G.make_opts(scheme=3, flags=G.CDG2_FORCING, newton_rtol=1e-10, gmres_rtol=1e-6))
            assert rc == 0
        e = O.l2_error(om, U.cpu().reshape(om.E, 6, om.nb), lambda x: O.mms_solution(x, T, ph, 0.2))
        errs.append(float(e.norm()))
    eoc = math.log2(errs[-2] / errs[-1])
    assert eoc > k + 1 - 0.3, (errs, eoc)


def test_step_nonfinite_input_is_reported(G):
    om, gm = _pair(G, 2, (8, 2), 1)
    p = I.default_params()
    U = gaussian_state(om, sigma=0.1, seed=5).cuda()
    U[3, 2, 1] = float("nan")                         # fault injected on the host side
    rc, st = G.cdg2_step(gm, p, U, 0.0, 1e-3, G.make_opts(), raise_on_error=False)
    assert rc == -4 and "non-finite" in G.cdg2_last_error()


def test_step_iteration_cap_is_reported(G):
    om, gm = _pair(G, 2, (8, 2), 2)
    p = I.default_params()
    U = gaussian_state(om, sigma=0.1, seed=6).cuda()
    U_before = U.clone()
    rc, st = G.cdg2_step(gm, p, U, 0.0, 1e-2, G.make_opts(max_newton=1, newton_rtol=1e-15, newton_atol=0.0,
                                                           gmres_rtol=0.5), raise_on_error=False)
    assert rc == -3 and st["newton_iters"] == 1 and st["residual"][0] > 0
    assert torch.equal(U, U_before)                   # U is left unchanged on failure


def test_step_rejects_bad_options(G):
    om, gm = _pair(G, 2, (4, 2), 1)
    U = torch.zeros(gm.n_dof, dtype=torch.float64, device="cuda")
    for bad in (dict(scheme=5), dict(gmres_restart=0), dict(gmres_restart=65), dict(max_newton=0), dict(precond=3),
                dict(precond=-1)):
        rc, _ = G.cdg2_step(gm, I.default_params(), U, 0.0, 1e-3, G.make_opts(**bad), raise_on_error=False)
        assert rc == -1
    rc, _ = G.cdg2_step(gm, I.default_params(), U, 0.0, 0.0, G.make_opts(), raise_on_error=False)
    assert rc == -1


@pytest.mark.parametrize("mixed", [0, 1, 2])   # 2: the TF32 element kernel (3D Q3), its pre-scaled tangent included
def test_preconditioner_changes_iterations_not_the_solution(G, mixed):
    om, gm = _pair(G, 3, (8, 4, 4), 3)
    p = I.default_params()
    U0 = gaussian_state(om, n_gauss=8, sigma=0.04, seed=1160).cuda()
    out, its = {}, {}
    for pc in (0, 1, 2):
        U = U0.clone()
        rc, st = G.cdg2_step(gm, p, U, 0.0, 1e-3, G.make_opts(scheme=3, mixed=mixed, precond=pc, newton_rtol=1e-11,
                                                               gmres_rtol=1e-4))
        assert rc == 0
        out[pc], its[pc] = U, st["gmres_iters"]
    assert float((out[1] - out[0]).norm() / out[0].norm()) <= 1e-10
    assert float((out[2] - out[0]).norm() / out[0].norm()) <= 1e-10
    assert its[1] < its[0]
    assert its[2] < its[1]   # the element blocks hold the modal diagonal and its couplings


def test_block_preconditioner_fp32_ragged_run(G):
    # 3D Q3 on 5x3x3 cells (45 elements): the FP32 block apply of 64-mode blocks
    # works on runs of 64 elements, so here one ragged run holding every element
    # type (the two wall layers in y and the interior); same solution and about
    # the same GMRES iterations as the FP64 block apply
    om, gm = _pair(G, 3, (5, 3, 3), 3)
    p = I.default_params()
    U0 = gaussian_state(om, n_gauss=8, sigma=0.04, seed=1161).cuda()
    out, its = {}, {}
    for mixed, pc in ((0, 0), (0, 2), (1, 2), (2, 2)):
        U = U0.clone()
        rc, st = G.cdg2_step(gm, p, U, 0.0, 1e-3, G.make_opts(scheme=3, mixed=mixed, precond=pc, newton_rtol=1e-11,
                                                               gmres_rtol=1e-4))
        assert rc == 0
        out[mixed, pc], its[mixed, pc] = U, st["gmres_iters"]
    for key in ((0, 2), (1, 2), (2, 2)):
        assert float((out[key] - out[0, 0]).norm() / out[0, 0].norm()) <= 1e-10
    assert its[0, 2] < its[0, 0]
    for key in ((1, 2), (2, 2)):
        assert its[key] <= 1.25 * its[0, 2] + 2


@pytest.mark.parametrize("mixed", [False, True])
def test_block_preconditioned_step_matches_oracle(G, mixed):
    om, gm = _pair(G, 2, (8, 4), 2)
    p = I.default_params()
    U0 = gaussian_state(om, sigma=0.08, seed=31)
    ref = U0.clone()
    for i in range(2):
        ref = O.step(om, ref, p, i * 1e-3, 1e-3, "sdirk3")
    U = U0.clone().cuda()
    o = _tight(G, 3, mixed)
    o.precond = 2
    for i in range(2):
        rc, st = G.cdg2_step(gm, p, U, i * 1e-3, 1e-3, o)
        assert rc == 0
    assert _rel(U, ref) <= 1e-10
