"""cdg2_tri_apply (triangle meshes, P_k, chi_e = 1.5) through the C ABI against
the triangle oracle.  Bar: relative L2 error per species 1e-12 (FP64) on
jittered meshes spanning several CTAs with ragged last CTAs, k = 1..3, with
and without M^{-1}, unjittered meshes (exact area ties), relabelled vertex
orders (every local edge index), the reduced model and bc_sign = -1; at the
full 256x64x2 P3 size, sampled triangles against the oracle on the patch of
each triangle and its edge neighbours (which fixes its row of L_h)."""
import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from oracle import cdg2_tri_oracle as T
from helpers import lift_into_domain, psi_max_tri, rel_l2_per_species

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
    cen, amp = I.gaussian_draws(2, (1.0, 0.2), 4, seed)
    U = T.project(om, lambda x: O.gaussian_field(om, x, cen, amp, 0.08, 1e-3))
    return lift_into_domain(U, psi_max_tri(om.k))


def _run(G, xy, tri, k, p, U, flags):
    gm = G.cdg2_tri_mesh_create(xy, tri, k)
    out = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_tri_apply(gm, p, U.reshape(-1).contiguous().cuda(), out, flags)
    torch.cuda.synchronize()
    return out.cpu().reshape(U.shape)


@pytest.mark.parametrize("nx,ny,k", [(6, 3, 1), (9, 4, 2), (7, 3, 3), (16, 4, 2)])
@pytest.mark.parametrize("minv", [True, False])
def test_tri_apply_matches_oracle(G, nx, ny, k, minv):
    xy, tri = I.tri_mesh(nx, ny, 1.0, 0.2, 0.2, 100 + k)
    om = T.TriMesh(xy, tri, k)
    p = _params()
    U = _state(om, 7 + k)
    got = _run(G, xy, tri, k, p, U, G.CDG2_MINV if minv else 0)
    pv = O.param_vector(p)
    ref = T.apply(om, U, p) if minv else T.apply_residual(om, U, pv)
    assert rel_l2_per_species(got, ref) <= 1e-12


@pytest.mark.parametrize("k", [1, 3])
def test_tri_apply_ties_and_relabelled_vertices(G, k):
    xy, tri = I.tri_mesh(5, 3, 1.0, 0.2, 0.0, 1)          # equal areas: the lower index is K^-
    rng = np.random.default_rng(k)
    shift = rng.integers(0, 3, size=len(tri))
    rel = np.stack([tri[np.arange(len(tri)), (shift + j) % 3] for j in range(3)], axis=1)
    for t in (tri, rel):
        om = T.TriMesh(xy, t, k)
        p = _params()
        U = lift_into_domain(torch.from_numpy(I.random_coefficients(om.E, om.nb, 3, 0.1)), psi_max_tri(om.k))
        got = _run(G, xy, t, k, p, U, G.CDG2_MINV)
        assert rel_l2_per_species(got, T.apply(om, U, p)) <= 1e-12


def test_tri_apply_reduced_model_and_outward_sign(G):
    xy, tri = I.tri_mesh(8, 3, 1.0, 0.2, 0.2, 41)
    k = 2
    om = T.TriMesh(xy, tri, k)
    U = _state(om, 5)
    U[:, 3, 0] += 0.05                                       # c1 above the thresholds on part of Gamma
    for change in ({"model": 1}, {"bc_sign": -1.0}):
        p = _params()
        p.update(change)
        V = U.clone()
        if change.get("model") == 1:
            V[:, [1, 4, 5], :] = 0.0                          # Eq. (2) has no n2, c2, c3
        got = _run(G, xy, tri, k, p, V, G.CDG2_MINV)
        ref = T.apply(om, V, p)
        assert rel_l2_per_species(got, ref) <= 1e-12


def _patch(xy, tri, e, nbrs):
    """The triangles e and its edge neighbours (ascending global index, so the
    tie rule picks the same K^-) with their vertices renumbered."""
    cells = sorted({e} | set(nbrs[e]))
    verts = sorted({int(v) for c in cells for v in tri[c]})
    vmap = {v: i for i, v in enumerate(verts)}
    sub = np.array([[vmap[int(v)] for v in tri[c]] for c in cells], dtype=np.int64)
    return xy[verts], sub, cells.index(e), cells


def test_tri_apply_full_size_sampled_rows(G):
    w = I.tri_workload(1)
    xy, tri = I.tri_mesh(w.nx, w.ny, 1.0, 0.2, w.jitter, w.seed)
    gm = G.cdg2_tri_mesh_create(xy, tri, w.k)
    p = _params()
    U = lift_into_domain(torch.from_numpy(I.random_coefficients(gm.n_elem, gm.n_basis, w.seed, 0.1)), psi_max_tri(w.k))
    out = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_tri_apply(gm, p, U.reshape(-1).cuda(), out, G.CDG2_MINV)
    got = out.cpu().reshape(U.shape)
    # edge neighbours from the vertex pairs
    owner = {}
    for t in range(len(tri)):
        for l in range(3):
            a, b = int(tri[t, l]), int(tri[t, (l + 1) % 3])
            owner.setdefault((min(a, b), max(a, b)), []).append(t)
    nbrs = {t: [] for t in range(len(tri))}
    for ts in owner.values():
        if len(ts) == 2:
            nbrs[ts[0]].append(ts[1])
            nbrs[ts[1]].append(ts[0])
    rng = np.random.default_rng(7)
    sample = list(rng.choice(len(tri), 40, replace=False)) + [0, len(tri) - 1, 2 * w.nx - 1, len(tri) - 2 * w.nx]
    for e in sample:
        pxy, ptri, c, cells = _patch(xy, tri, int(e), nbrs)
        om = T.TriMesh(pxy, ptri, w.k)
        ref = T.apply(om, U[cells], p)[c]
        err = float((got[int(e)] - ref).norm() / ref.norm())
        assert err <= 1e-12, (int(e), err)


@pytest.mark.parametrize("nx,ny,k", [(6, 3, 1), (9, 4, 2), (7, 3, 3)])
def test_tri_jvp_matches_oracle(G, nx, ny, k):
    xy, tri = I.tri_mesh(nx, ny, 1.0, 0.2, 0.2, 200 + k)
    om = T.TriMesh(xy, tri, k)
    p = _params()
    U = _state(om, 17 + k)
    U[:, 3, 0] += 0.05
    dU = torch.from_numpy(np.random.default_rng(k).standard_normal(U.shape))
    gm = G.cdg2_tri_mesh_create(xy, tri, k)
    out = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_tri_jvp(gm, p, U.reshape(-1).cuda(), dU.reshape(-1).contiguous().cuda(), out, G.CDG2_MINV)
    got = out.cpu().reshape(U.shape)
    assert rel_l2_per_species(got, T.jvp(om, U, dU, p)) <= 1e-12
    # the JVP is the derivative of the GPU apply itself (central differences through the C ABI)
    h = 1e-6
    fp = _run(G, xy, tri, k, p, U + h * dU, G.CDG2_MINV)
    fm = _run(G, xy, tri, k, p, U - h * dU, G.CDG2_MINV)
    fd = (fp - fm) / (2 * h)
    # (the LLF max and the signs of the normal velocities have kinks: 1e-4, as for the Cartesian JVP)
    assert float((fd - got).norm() / got.norm()) <= 1e-4


@pytest.mark.parametrize("nx,ny,k", [(6, 3, 1), (9, 4, 2), (7, 3, 3)])
@pytest.mark.parametrize("minv", [True, False])
def test_tri_vjp_matches_oracle_and_transposes_the_jvp(G, nx, ny, k, minv):
    xy, tri = I.tri_mesh(nx, ny, 1.0, 0.2, 0.2, 300 + k)
    om = T.TriMesh(xy, tri, k)
    p = _params()
    U = _state(om, 27 + k)
    U[:, 3, 0] += 0.05
    rng = np.random.default_rng(10 + k)
    lam = torch.from_numpy(rng.standard_normal(U.shape))
    dU = torch.from_numpy(rng.standard_normal(U.shape))
    gm = G.cdg2_tri_mesh_create(xy, tri, k)
    flags = G.CDG2_MINV if minv else 0
    gU = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    G.cdg2_tri_vjp(gm, p, U.reshape(-1).cuda(), lam.reshape(-1).contiguous().cuda(), gU, flags)
    got = gU.cpu().reshape(U.shape)
    if minv:
        ref = T.vjp(om, U, lam, p)
    else:
        _, fn = torch.func.vjp(lambda V: T.apply_residual(om, V, O.param_vector(p)), U)
        ref = fn(lam)[0]
    assert rel_l2_per_species(got, ref) <= 1e-12
    jv = torch.empty_like(gU)
    G.cdg2_tri_jvp(gm, p, U.reshape(-1).cuda(), dU.reshape(-1).contiguous().cuda(), jv, flags)
    lhs = float((lam.reshape(-1) * jv.cpu()).sum())
    rhs = float((got.reshape(-1) * dU.reshape(-1)).sum())
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1.0) * 10
    # bitwise reproducible (no atomics)
    gU2 = torch.empty_like(gU)
    G.cdg2_tri_vjp(gm, p, U.reshape(-1).cuda(), lam.reshape(-1).contiguous().cuda(), gU2, flags)
    assert torch.equal(gU, gU2)
