"""Pin of the simplicial oracles' spaces against the problem sizes the paper
prints (Sec. 4.1: 81,920 triangles, 7,372,800 degrees of freedom; Sec. 4.2:
113,549 tetrahedra, 13,625,880; six species each, `tests/golden/dof_counts.txt`).
The oracles' Dubiner bases at the printed degrees must have exactly dim P_k
functions per species, be orthonormal on the reference simplex and span P_k;
and only that degree reproduces the printed count."""
import itertools
import os

import torch

from oracle import cdg2_tet_oracle as Tet
from oracle import cdg2_tri_oracle as Tri

F64 = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dof_counts.txt")


def printed_sizes():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                shape, ne, k, ns, dof = line.split()
                rows.append((shape, int(ne), int(k), int(ns), int(dof)))
    return rows


def basis_and_rule(shape, k):
    if shape == "triangle":
        pts, w = Tri.triangle_rule(k + 2)
        psi, _ = Tri.dubiner(k, pts)
        return psi, pts, w, 2, 0.5
    pts, w = Tet.tet_rule(k + 2)
    psi, _ = Tet.dubiner3(k, pts)
    return psi, pts, w, 3, 1.0 / 6.0


def random_simplex_points(dim, n, seed):
    g = torch.Generator().manual_seed(seed)
    x = torch.rand(n, dim + 1, generator=g, dtype=F64)
    x = -torch.log(x)                       # exponential draws: normalised, uniform on the simplex
    return (x / x.sum(dim=1, keepdim=True))[:, :dim]


def test_printed_counts_fix_the_degree():
    sizes = printed_sizes()
    assert {s[0] for s in sizes} == {"triangle", "tetrahedron"}
    for shape, ne, k, ns, dof in sizes:
        modes = Tri.modes if shape == "triangle" else Tet.modes
        matching = [d for d in range(0, 8) if ne * len(modes(d)) * ns == dof]
        assert matching == [k], (shape, matching)


def test_bases_at_the_printed_degrees_are_orthonormal_and_span_pk():
    for shape, ne, k, ns, dof in printed_sizes():
        psi, pts, w, dim, vol = basis_and_rule(shape, k)
        nb = psi.shape[1]
        # dim P_k = binomial(k + dim, dim); the printed size is elements x nb x species
        n_monomials = sum(1 for a in itertools.product(range(k + 1), repeat=dim) if sum(a) <= k)
        assert nb == n_monomials
        assert ne * nb * ns == dof
        assert abs(float(w.sum()) - vol) < 1e-15
        gram = psi.T @ (w[:, None] * psi)
        assert float((gram - torch.eye(nb, dtype=F64)).abs().max()) < 1e-12
        # every monomial of degree <= k is reproduced by its orthogonal projection
        x = random_simplex_points(dim, 40, seed=1403 + dim)
        psi_x = (Tri.dubiner(k, x) if shape == "triangle" else Tet.dubiner3(k, x))[0]
        for a in itertools.product(range(k + 1), repeat=dim):
            if sum(a) > k:
                continue
            mono_q = torch.prod(pts ** torch.tensor(a, dtype=F64), dim=1)
            coef = psi.T @ (w * mono_q)
            mono_x = torch.prod(x ** torch.tensor(a, dtype=F64), dim=1)
            assert float((psi_x @ coef - mono_x).abs().max()) < 1e-11, (shape, a)
