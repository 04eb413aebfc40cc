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
from helpers import rel_l2_per_species

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
    return TT.project(om, lambda x: O.gaussian_field(om, x, cen, amp, 0.08, 1e-3))


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
        U = torch.from_numpy(I.random_coefficients(om.E, om.nb, 3, 0.1))
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
    U = torch.from_numpy(I.random_coefficients(gm.n_elem, gm.n_basis, w.seed, 0.1))
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
