"""The tensor-core (TF32) element contractions of the FP32 operator (CDG2_TF32).

On 3D Q3 meshes cdg2_apply and cdg2_jvp with CDG2_FP32 | CDG2_TF32 run the
volume terms' contractions as TF32 GEMMs (tcgen05) over blocks of 16
elements.  The result is compared per species with the FP64 path on the same
rounded input (the FP64 path matches the oracle to 1e-12), relative per
species.  TF32 keeps 10 mantissa bits (inputs rounded to 2^-11 relative).
The JVP along a rough tangent (what the Krylov solver applies) stays at
about 5e-5: bar 2e-4.  The apply on random states (cell means O(1)) stays
near 1e-5: bar 1e-4.  On smooth states the volume and face parts of the
weak form cancel for n1 and n2, whose chemotactic and diffusive fluxes go
through the tensor cores, and the error there grows with the mesh
resolution (3e-4 to 1.1e-3 on the test meshes, 3.7e-3 on 3D 64x16x16 Q3;
the other species keep FP32 accuracy, their diffusion being modal): bar
1e-2.  Meshes span several 16-element blocks with a ragged last one,
periodic and wall-bounded axes.  The mixed solver with this operator
(mixed = 2) still converges to the FP64 solution, since its Newton residual
stays in FP64.
"""
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from helpers import gaussian_state, random_state

pytestmark = pytest.mark.gpu

BAR_JVP = 2e-4
BAR_APPLY_ROUGH = 1e-4
BAR_APPLY_SMOOTH = 1e-2


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


def _rel(got, ref, n_elem):
    g = got.double().view(n_elem, 6, -1)
    r = ref.double().view(n_elem, 6, -1)
    return ((g - r).pow(2).sum(dim=(0, 2)).sqrt() / r.pow(2).sum(dim=(0, 2)).sqrt()).tolist()


@pytest.mark.parametrize("cells,periodic", [((5, 3, 3), (1, 0, 1)), ((9, 4, 3), (1, 0, 1)), ((4, 4, 4), (0, 0, 0)),
                                            ((16, 2, 1), (1, 1, 1))])
@pytest.mark.parametrize("field", ["gauss", "random"])
def test_tf32_apply_and_jvp(G, cells, periodic, field):
    ext = (1.0, 0.2, 0.2)
    om = O.Mesh(3, cells, ext, periodic, 3)
    gm = G.cdg2_mesh_create(3, cells, ext, periodic, 3)
    p = I.default_params()
    U = gaussian_state(om, sigma=0.08, seed=5) if field == "gauss" else random_state(om, seed=8)
    U32 = U.reshape(-1).float().cuda()
    Ur = U32.double()
    out = torch.empty_like(U32)
    ref = torch.empty_like(Ur)
    for flags in (G.CDG2_MINV, 0):
        G.cdg2_apply(gm, p, U32, out, flags | G.CDG2_FP32 | G.CDG2_TF32)
        G.cdg2_apply(gm, p, Ur, ref, flags)
        errs = _rel(out, ref, gm.n_elem)
        print("apply", cells, field, flags, max(errs))
        assert max(errs) <= (BAR_APPLY_SMOOTH if field == "gauss" else BAR_APPLY_ROUGH), errs
    dU = (random_state(om, seed=9) - 1.0).reshape(-1).float().cuda()
    G.cdg2_jvp(gm, p, U32, dU, out, G.CDG2_MINV | G.CDG2_FP32 | G.CDG2_TF32)
    G.cdg2_jvp(gm, p, Ur, dU.double(), ref, G.CDG2_MINV)
    errs = _rel(out, ref, gm.n_elem)
    print("jvp", cells, field, max(errs))
    assert max(errs) <= BAR_JVP, errs


def test_tf32_full_size(G):
    w = I.workload(3)
    gm = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    U = torch.empty(gm.n_dof, dtype=torch.float64, device="cuda")
    cen, amp = I.gaussian_draws(w.dim, w.extent, w.n_gauss, w.seed)
    G.cdg2_project_gaussians(gm, cen, amp, w.sigma, w.floor, U)
    p = I.default_params()
    U32 = U.float()
    Ur = U32.double()
    out = torch.empty_like(U32)
    ref = torch.empty_like(U)
    G.cdg2_apply(gm, p, U32, out, G.CDG2_MINV | G.CDG2_FP32 | G.CDG2_TF32)
    G.cdg2_apply(gm, p, Ur, ref, G.CDG2_MINV)
    errs = _rel(out, ref, gm.n_elem)
    print("apply full", errs)
    assert max(errs) <= BAR_APPLY_SMOOTH, errs
    dU = torch.sin(torch.arange(gm.n_dof, device="cuda", dtype=torch.float64) * 0.37).float()
    G.cdg2_jvp(gm, p, U32, dU, out, G.CDG2_MINV | G.CDG2_FP32 | G.CDG2_TF32)
    G.cdg2_jvp(gm, p, Ur, dU.double(), ref, G.CDG2_MINV)
    errs = _rel(out, ref, gm.n_elem)
    print("jvp full", errs)
    assert max(errs) <= BAR_JVP, errs


def test_tf32_rejects_other_meshes_and_dtypes(G):
    gm = G.cdg2_mesh_create(3, (4, 3, 2), (1.0, 0.2, 0.2), (1, 0, 1), 2)
    U = torch.ones(gm.n_dof, dtype=torch.float32, device="cuda")
    out = torch.empty_like(U)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_apply(gm, I.default_params(), U, out, G.CDG2_MINV | G.CDG2_FP32 | G.CDG2_TF32)
    gm3 = G.cdg2_mesh_create(3, (4, 3, 2), (1.0, 0.2, 0.2), (1, 0, 1), 3)
    U64 = torch.ones(gm3.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(G.Cdg2Error):
        G.cdg2_apply(gm3, I.default_params(), U64, torch.empty_like(U64), G.CDG2_MINV | G.CDG2_TF32)


def test_mixed_tf32_step_matches_fp64_step(G):
    """mixed = 2: the same SDIRK3 step to Newton relative residual 1e-12 as the FP64 solver."""
    cells = (8, 4, 4)
    ext = (1.0, 0.2, 0.2)
    om = O.Mesh(3, cells, ext, (1, 0, 1), 3)
    gm = G.cdg2_mesh_create(3, cells, ext, (1, 0, 1), 3)
    p = I.default_params()
    U0 = gaussian_state(om, n_gauss=8, sigma=0.06, seed=1160).reshape(-1).cuda()
    res = {}
    for mixed in (0, 2):
        U = U0.clone()
        rc, st = G.cdg2_step(gm, p, U, 0.0, 1e-3, G.make_opts(scheme=G.CDG2_SDIRK3, mixed=mixed, newton_rtol=1e-12,
                                                               gmres_rtol=1e-4, max_newton=30, precond=2))
        assert rc == 0
        print("mixed", mixed, st["newton_iters"], st["gmres_iters"])
        res[mixed] = U
    assert float((res[2] - res[0]).norm() / res[0].norm()) <= 1e-10
