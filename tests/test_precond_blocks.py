"""The element blocks of the block-Jacobi preconditioner (precond = 2),
computed by the library on the host, against the oracle: the (element,
species) diagonal block of I - gdt J, J the dense Jacobian (autograd) of
the oracle's M^{-1} L_h with chemotaxis and reactions switched off, so that
only the diffusion terms of Sec. 3.1 (volume, consistency, symmetry,
penalty on interior faces) remain.  Elements with both faces, with a
boundary face on Gamma_1, Gamma_2 or a no-flow wall, and a periodic axis
of a single cell (a face shared with itself), for the CDG2, BR2 and SIPG
fluxes.  Host-only: no GPU needed."""
import pytest
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O

F64 = torch.float64


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


def diffusion_only(p):
    q = dict(p)
    q["chi0"] = (0.0, 0.0, 0.0, 0.0)
    for key in ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox"):
        q[key] = 0.0
    return q


CASES = [
    # dim, cells, extent, periodic, k, flux, gflux, penalty
    (2, (4, 3), (1.0, 0.2), (1, 0), 3, "cdg2", 0, 0.0),
    (2, (3, 4), (0.6, 0.2), (0, 0), 2, "cdg2", 0, 0.0),
    (2, (1, 3), (0.3, 0.2), (1, 0), 1, "cdg2", 0, 0.0),
    (2, (4, 3), (1.0, 0.2), (1, 0), 2, "br2", 1, 5.0),
    (2, (4, 3), (1.0, 0.2), (1, 0), 2, "sipg", 2, 3.0),
    (3, (2, 3, 2), (1.0, 0.2, 0.2), (1, 0, 1), 2, "cdg2", 0, 0.0),
    (3, (3, 3, 1), (1.0, 0.2, 0.1), (0, 0, 1), 1, "cdg2", 0, 0.0),
]


@pytest.mark.parametrize("dim,cells,ext,per,k,flux,gflux,pen", CASES)
def test_element_blocks_match_oracle_jacobian(G, dim, cells, ext, per, k, flux, gflux, pen):
    om = O.Mesh(dim, cells, ext, per, k, flux=flux, penalty=pen or None)
    gm = G.cdg2_mesh_create(dim, cells, ext, per, k, flux=gflux, penalty=pen)
    p = diffusion_only(I.default_params())
    # distinct diffusivities per species so that a species mix-up shows
    p["mu"] = (1.1e-2, 4.0e-3, 2.5e-3)
    p["nu"] = (5.0e-2, 3.0e-2, 7.0e-2)
    U = torch.from_numpy(I.random_coefficients(om.E, om.nb, 3, 0.1))
    n = U.numel()
    J = torch.func.jacrev(lambda V: O.apply(om, V, p))(U).reshape(n, n)
    gdt = 0.37
    A = torch.eye(n, dtype=F64) - gdt * J
    nb = om.nb
    scale = float(A.abs().max())
    for e in range(om.E):
        for s in range(6):
            i0 = (e * 6 + s) * nb
            ref = A[i0:i0 + nb, i0:i0 + nb]
            got = G.cdg2_element_block(gm, p, gdt, e, s)
            assert float((got - ref).abs().max()) <= 1e-12 * scale, (e, s)


def test_diffusion_block_is_symmetric_and_its_k_negative_semidefinite(G):
    """K_e is symmetric and negative semi-definite (the pure-diffusion CDG2
    operator is), so I - gdt A_s K_e is symmetric positive definite for gdt > 0."""
    gm = G.cdg2_mesh_create(3, (3, 4, 2), (1.0, 0.2, 0.2), (1, 0, 1), 3)
    p = I.default_params()
    for e in (0, 5, 23):
        for s in (0, 4):
            B = G.cdg2_element_block(gm, p, 1e-3, e, s)
            assert torch.allclose(B, B.T, rtol=0, atol=1e-12 * float(B.abs().max()))
            ev = torch.linalg.eigvalsh(B)
            assert float(ev.min()) >= 1.0 - 1e-12


def test_element_block_validates(G):
    gm = G.cdg2_mesh_create(2, (4, 2), (1.0, 0.2), (1, 0), 1)
    p = I.default_params()
    with pytest.raises(G.Cdg2Error):
        G.cdg2_element_block(gm, p, 0.1, 8, 0)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_element_block(gm, p, 0.1, 0, 6)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_element_block(gm, p, float("nan"), 0, 0)
