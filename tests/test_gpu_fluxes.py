"""The BR2 and interior-penalty diffusion fluxes (the schemes Fig. 2 compares
with CDG2) through the C ABI, against the oracle's literal definitions
(BR2: liftings solved on both cells and averaged; SIPG: the penalty term).
Bar: relative L2 error per species 1e-12 for apply, JVP and VJP."""
import numpy as np
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O
from helpers import gaussian_state, rel_l2_per_species

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


@pytest.mark.parametrize("flux,gflux,pen", [("br2", 1, 5.0), ("sipg", 2, 3.0), ("br2", 1, 0.0), ("sipg", 2, 0.0)])
@pytest.mark.parametrize("dim,cells,k", [(2, (11, 5), 2), (3, (4, 3, 2), 3)])
def test_flux_variants(G, flux, gflux, pen, dim, cells, k):
    ext = (1.0, 0.2, 0.2)
    per = (1, 0, 0) if dim == 2 else (1, 0, 1)
    om = O.Mesh(dim, cells, ext, per, k, flux=flux, penalty=pen or None)
    gm = G.cdg2_mesh_create(dim, cells, ext, per, k, flux=gflux, penalty=pen)
    p = I.default_params()
    p["chi0"] = (0.05, 0.02, 0.03, 0.02)
    U = gaussian_state(om, sigma=0.08, seed=70 + k)
    out = torch.empty_like(U.cuda())
    G.cdg2_apply(gm, p, U.cuda(), out, G.CDG2_MINV)
    assert rel_l2_per_species(out, O.apply(om, U, p)) <= 1e-12
    dU = torch.from_numpy(np.random.default_rng(k).standard_normal(U.shape))
    G.cdg2_jvp(gm, p, U.cuda(), dU.cuda(), out, G.CDG2_MINV)
    assert rel_l2_per_species(out, O.jvp(om, U, dU, p)) <= 1e-12
    G.cdg2_vjp(gm, p, U.cuda(), dU.cuda(), out, None, G.CDG2_MINV)
    assert rel_l2_per_species(out, O.vjp(om, U, dU, p)[0]) <= 1e-12
