"""Host-side checks of the triangle-mesh entry points (no GPU): sizes agree
with the oracle's edge classification, and invalid meshes are rejected
with an error code."""
import numpy as np
import pytest

import cdg2_inputs as I
from oracle import cdg2_tri_oracle as T


@pytest.fixture(scope="module")
def G():
    import paper_1403_1157_gb300 as G
    from paper_1403_1157_gb300 import build
    build.build()
    return G


@pytest.mark.parametrize("nx,ny,k", [(4, 2, 1), (7, 3, 3), (1, 1, 2)])
def test_sizes_match_the_oracle(G, nx, ny, k):
    xy, tri = I.tri_mesh(nx, ny, 1.0, 0.2, 0.2, 5)
    m = G.cdg2_tri_mesh_create(xy, tri, k)
    om = T.TriMesh(xy, tri, k)
    assert (m.n_elem, m.n_basis, m.n_faces) == (om.E, om.nb, len(om.interior))
    assert m.n_dof == om.E * 6 * om.nb


def test_invalid_meshes_are_rejected(G):
    xy, tri = I.tri_mesh(3, 2, 1.0, 0.2, 0.0, 1)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_tri_mesh_create(xy, tri, 4)                       # k out of range
    with pytest.raises(G.Cdg2Error):
        G.cdg2_tri_mesh_create(xy, tri[:, ::-1].copy(), 1)        # clockwise
    bad = tri.copy()
    bad[0, 0] = len(xy)
    with pytest.raises(G.Cdg2Error):
        G.cdg2_tri_mesh_create(xy, bad, 1)                        # index out of range
    dup = np.concatenate([tri, tri[:1]])
    with pytest.raises(G.Cdg2Error):
        G.cdg2_tri_mesh_create(xy, dup, 1)                        # an edge with three triangles
