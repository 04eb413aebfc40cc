"""cdg2_tet_apply (tetrahedral meshes, P_k, chi_e = 2) through the C ABI against
the tetrahedral oracle.  Bar: relative L2 error per species 1e-12 (FP64) on
jittered Kuhn meshes spanning several CTAs, k = 1..3, with and without
M^{-1}, unjittered meshes (volume ties), relabelled vertex orders (every face
frame), the reduced model and bc_sign = -1."""
import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from oracle import cdg2_tet_oracle as TT
from helpers import lift_into_domain, psi_max_tet, rel_l2_per_species

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


def _params():
    p = I.default_params()
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    return p


def _state(om, seed):
    cen, amp = I.gaussian_draws(3, (1.0, 0.2, 0.2), 4, seed)
    U = TT.project(om, lambda x: O.gaussian_field(om, x, cen, amp, 0.08, 1e-3))
    return lift_into_domain(U, psi_max_tet(om.k))


def _discrete_state(om, seed):
    """Random coefficients (cell means O(1), so O(1) jumps).  The derivatives
    are compared on such states: for a smooth projected state the two traces
    nearly agree, so the LLF maximum |v^- . n| vs |v^+ . n| is a near-tie at
    almost every face point and rounding picks its branch; a relative 1e-15
    perturbation of U then moves the oracle's own JVP by ~1e-12."""
    return lift_into_domain(torch.from_numpy(I.random_coefficients(om.E, om.nb, seed)), psi_max_tet(om.k))


def _run(G, xyz, tet, k, p, U, flags):
    gm = G.cdg2_tet_mesh_create(xyz, tet, k)
    out = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_tet_apply(gm, p, U.reshape(-1).contiguous().cuda(), out, flags)
    torch.cuda.synchronize()
    return out.cpu().reshape(U.shape)


@pytest.mark.parametrize("cells,k", [((3, 2, 2), 1), ((3, 2, 1), 2), ((2, 2, 1), 3)])
@pytest.mark.parametrize("minv", [True, False])
def test_tet_apply_matches_oracle(G, cells, k, minv):
    xyz, tet = I.tet_mesh(*cells, 1.0, 0.2, 0.2, 0.15, 400 + k)
    om = TT.TetMesh(xyz, tet, k)
    p = _params()
    U = _state(om, 40 + k)
    U[:, 3, 0] += 0.05
    got = _run(G, xyz, tet, k, p, U, G.CDG2_MINV if minv else 0)
    ref = TT.apply(om, U, p) if minv else TT.apply_residual(om, U, O.param_vector(p))
    assert rel_l2_per_species(got, ref) <= 1e-12


@pytest.mark.parametrize("k", [1, 2])
def test_tet_apply_ties_and_relabelled_vertices(G, k):
    xyz, tet = I.tet_mesh(2, 2, 1, 1.0, 0.2, 0.2, 0.0, 1)        # equal volumes: the lower index is K^-
    rng = np.random.default_rng(k)
    evens = [(0, 1, 2, 3), (1, 2, 0, 3), (2, 0, 1, 3), (0, 2, 3, 1), (0, 3, 1, 2), (1, 0, 3, 2), (2, 3, 0, 1),
             (3, 2, 1, 0), (1, 3, 2, 0), (3, 0, 2, 1), (2, 1, 3, 0), (3, 1, 0, 2)]
    rel = np.stack([tet[i, list(evens[rng.integers(0, 12)])] for i in range(len(tet))])
    for t in (tet, rel):
        om = TT.TetMesh(xyz, t, k)
        p = _params()
        U = lift_into_domain(torch.from_numpy(I.random_coefficients(om.E, om.nb, 3, 0.1)), psi_max_tet(om.k))
        got = _run(G, xyz, t, k, p, U, G.CDG2_MINV)
        assert rel_l2_per_species(got, TT.apply(om, U, p)) <= 1e-12


def test_tet_apply_reduced_model_and_outward_sign(G):
    xyz, tet = I.tet_mesh(3, 2, 1, 1.0, 0.2, 0.2, 0.15, 41)
    k = 2
    om = TT.TetMesh(xyz, tet, k)
    U = _state(om, 5)
    U[:, 3, 0] += 0.05
    for change in ({"model": 1}, {"bc_sign": -1.0}):
        p = _params()
        p.update(change)
        V = U.clone()
        if change.get("model") == 1:
            V[:, [1, 4, 5], :] = 0.0
        got = _run(G, xyz, tet, k, p, V, G.CDG2_MINV)
        assert rel_l2_per_species(got, TT.apply(om, V, p)) <= 1e-12


def test_tet_apply_full_size_sampled_rows(G):
    """32x8x8x6 P3 (1.47M DOF): sampled tetrahedra against the oracle on the patch
    of each tetrahedron and its face neighbours (ascending global index, so the
    tie rule picks the same K^-), which fixes its row of M^{-1} L_h."""
    w = I.tet_workload(1)
    xyz, tet = I.tet_mesh(*w.cells, *w.extent, w.jitter, w.seed)
    gm = G.cdg2_tet_mesh_create(xyz, tet, w.k)
    p = _params()
    U = lift_into_domain(torch.from_numpy(I.random_coefficients(gm.n_elem, gm.n_basis, w.seed, 0.1)), psi_max_tet(w.k))
    out = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_tet_apply(gm, p, U.reshape(-1).cuda(), out, G.CDG2_MINV)
    got = out.cpu().reshape(U.shape)
    owner = {}
    for t in range(len(tet)):
        for l in range(4):
            key = tuple(sorted(int(v) for j, v in enumerate(tet[t]) if j != l))
            owner.setdefault(key, []).append(t)
    nbrs = {t: [] for t in range(len(tet))}
    for ts in owner.values():
        if len(ts) == 2:
            nbrs[ts[0]].append(ts[1])
            nbrs[ts[1]].append(ts[0])
    rng = np.random.default_rng(5)
    sample = list(rng.choice(len(tet), 30, replace=False)) + [0, len(tet) - 1]
    for e in sample:
        cells = sorted({int(e)} | set(nbrs[int(e)]))
        verts = sorted({int(v) for c in cells for v in tet[c]})
        vmap = {v: i for i, v in enumerate(verts)}
        sub = np.array([[vmap[int(v)] for v in tet[c]] for c in cells], dtype=np.int64)
        om = TT.TetMesh(xyz[verts], sub, w.k)
        ref = TT.apply(om, U[cells], p)[cells.index(int(e))]
        err = float((got[int(e)] - ref).norm() / ref.norm())
        assert err <= 1e-12, (int(e), err)


@pytest.mark.parametrize("cells,k", [((3, 2, 2), 1), ((3, 2, 1), 2), ((2, 2, 1), 3)])
def test_tet_jvp_matches_oracle(G, cells, k):
    xyz, tet = I.tet_mesh(*cells, 1.0, 0.2, 0.2, 0.15, 500 + k)
    om = TT.TetMesh(xyz, tet, k)
    p = _params()
    U = _discrete_state(om, 50 + k)
    dU = torch.from_numpy(np.random.default_rng(k).standard_normal(U.shape))
    gm = G.cdg2_tet_mesh_create(xyz, tet, k)
    out = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_tet_jvp(gm, p, U.reshape(-1).cuda(), dU.reshape(-1).contiguous().cuda(), out, G.CDG2_MINV)
    got = out.cpu().reshape(U.shape)
    assert rel_l2_per_species(got, TT.jvp(om, U, dU, p)) <= 1e-12
    # the JVP is the derivative of the GPU apply itself (central differences through the C ABI;
    # the step is small enough that no difference straddles a kink of the LLF max or an upwind
    # sign on these states, where the oracle's own differences agree to 3e-10)
    h = 1e-7
    fd = (_run(G, xyz, tet, k, p, U + h * dU, G.CDG2_MINV) - _run(G, xyz, tet, k, p, U - h * dU, G.CDG2_MINV)) / (2 * h)
    assert float((fd - got).norm() / got.norm()) <= 1e-6


@pytest.mark.parametrize("cells,k", [((3, 2, 2), 1), ((3, 2, 1), 2), ((2, 2, 1), 3)])
@pytest.mark.parametrize("minv", [True, False])
def test_tet_vjp_matches_oracle_and_transposes_the_jvp(G, cells, k, minv):
    xyz, tet = I.tet_mesh(*cells, 1.0, 0.2, 0.2, 0.15, 600 + k)
    om = TT.TetMesh(xyz, tet, k)
    p = _params()
    U = _discrete_state(om, 60 + k)
    rng = np.random.default_rng(20 + k)
    lam = torch.from_numpy(rng.standard_normal(U.shape))
    dU = torch.from_numpy(rng.standard_normal(U.shape))
    gm = G.cdg2_tet_mesh_create(xyz, tet, k)
    flags = G.CDG2_MINV if minv else 0
    gU = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_tet_vjp(gm, p, U.reshape(-1).cuda(), lam.reshape(-1).contiguous().cuda(), gU, flags)
    got = gU.cpu().reshape(U.shape)
    if minv:
        ref = TT.vjp(om, U, lam, p)
    else:
        _, fn = torch.func.vjp(lambda V: TT.apply_residual(om, V, O.param_vector(p)), U)
        ref = fn(lam)[0]
    assert rel_l2_per_species(got, ref) <= 1e-12
    jv = torch.empty_like(gU)
    G.cdg2_tet_jvp(gm, p, U.reshape(-1).cuda(), dU.reshape(-1).contiguous().cuda(), jv, flags)
    lhs = float((lam.reshape(-1) * jv.cpu()).sum())
    rhs = float((got.reshape(-1) * dU.reshape(-1)).sum())
    assert abs(lhs - rhs) <= 1e-10 * max(abs(lhs), 1.0)
    # bitwise reproducible (no atomics)
    gU2 = torch.empty_like(gU)
    G.cdg2_tet_vjp(gm, p, U.reshape(-1).cuda(), lam.reshape(-1).contiguous().cuda(), gU2, flags)
    assert torch.equal(gU, gU2)
