"""Host-side checks of the tetrahedral-mesh entry points (no GPU): sizes agree
with the oracle's face classification, and invalid meshes are rejected."""
import numpy as np
import pytest

import cdg2_inputs as I
from oracle import cdg2_tet_oracle as TT


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


@pytest.mark.parametrize("cells,k", [((2, 1, 1), 1), ((3, 2, 2), 3)])
def test_sizes_match_the_oracle(G, cells, k):
    xyz, tet = I.tet_mesh(*cells, 1.0, 0.2, 0.2, 0.15, 5)
    m = G.cdg2_tet_mesh_create(xyz, tet, k)
    om = TT.TetMesh(xyz, tet, k)
    assert (m.n_elem, m.n_basis, m.n_faces) == (om.E, om.nb, len(om.interior))


def test_invalid_meshes_are_rejected(G):
    xyz, tet = I.tet_mesh(2, 1, 1, 1.0, 0.2, 0.2, 0.0, 1)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_tet_mesh_create(xyz, tet, 4)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_tet_mesh_create(xyz, tet[:, [1, 0, 2, 3]].copy(), 1)   # negatively oriented
    bad = tet.copy()
    bad[0, 0] = len(xyz)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_tet_mesh_create(xyz, bad, 1)
