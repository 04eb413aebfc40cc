"""Shared helpers of the test suite: paired meshes and error measures."""
import numpy as np
import torch

import cdg2_inputs as I
from oracle import cdg2_oracle as O

F64 = torch.float64


def oracle_mesh(dim, cells, extent, periodic, k):
    return O.Mesh(dim, cells, extent, periodic, k)


def gpu_mesh(dim, cells, extent, periodic, k):
    import paper_1403_1157_gb300 as G
    return G.cdg2_mesh_create(dim, cells, extent, periodic, k)


def psi_max_cartesian(dim, k):
    """max over the unit cell of |phi_i| for the tensor Legendre basis (at a corner):
    prod_j sqrt(2 a_j + 1), modes in the oracle's order (x fastest)."""
    return torch.tensor([float(np.prod([np.sqrt(2 * a + 1) for a in idx])) for idx in O.multi_indices(k + 1, dim)],
                        dtype=F64)


def _simplex_samples(dim, n=12):
    pts = []
    for i in np.ndindex(*(n + 1,) * dim):
        if sum(i) <= n:
            pts.append([c / n for c in i])
    return torch.tensor(pts, dtype=F64)


def psi_max_tri(k):
    """max of |psi_i| over the reference triangle (a lattice with the vertices and edges)."""
    from oracle import cdg2_tri_oracle as T
    psi, _ = T.dubiner(k, _simplex_samples(2))
    return psi.detach().abs().amax(dim=0)


def psi_max_tet(k):
    """max of |psi_i| over the reference tetrahedron (a lattice with the vertices, edges and faces)."""
    from oracle import cdg2_tet_oracle as TT
    psi, _ = TT.dubiner3(k, _simplex_samples(3))
    return psi.detach().abs().amax(dim=0)


def lift_into_domain(U, psi_max, p=None, margin=0.02):
    """Shift n1, c1 and c3 by constants so that every denominator y + chith of the
    tactic sensitivities chi(x, y, a, b) = a x / (y + b) (Sec. 2) stays >= margin
    anywhere in every element, so the state is inside the model's domain (the
    kernels report CDG2_ERR_DOMAIN otherwise).  Per element the field is at
    least U_0 psi_0 - sum_{i>0} |U_i| max|psi_i| (psi_0 is the constant mode);
    the shift is the same in every element, so smooth fields stay smooth.
    U: (E, 6, nb) float64; returns a new tensor."""
    p = p or I.default_params()
    ch = p["chith"]
    need = {0: ch[3], 3: min(ch[0], ch[2]), 5: ch[1]}
    V = U.clone()
    for s, c in need.items():
        lo = V[:, s, 0] * psi_max[0] - (V[:, s, 1:].abs() * psi_max[1:]).sum(-1)
        lift = margin - c - float(lo.min())
        if lift > 0:
            V[:, s, 0] += lift / float(psi_max[0])
    return V


def gaussian_state(om, n_gauss=4, sigma=0.05, floor=1e-3, seed=1157):
    """Seeded Gaussian initial field projected by the oracle (the input recipe of
    the workloads), shifted into the model's domain where the projection undershoots."""
    cen, amp = I.gaussian_draws(om.dim, om.extent, n_gauss, seed)
    U = O.project(om, lambda x: O.gaussian_field(om, x, cen, amp, sigma, floor))
    return lift_into_domain(U, psi_max_cartesian(om.dim, om.k))


def random_state(om, seed=5, scale=0.1):
    U = torch.from_numpy(I.random_coefficients(om.E, om.nb, seed, scale))
    return lift_into_domain(U, psi_max_cartesian(om.dim, om.k))


def rel_l2_per_species(got, ref):
    """max over species of ||got_s - ref_s||_2 / ||ref_s||_2 (coefficient vectors)."""
    got = got.detach().to("cpu", F64).reshape(ref.shape)
    num = ((got - ref) ** 2).sum(dim=(0, 2)).sqrt()
    den = (ref ** 2).sum(dim=(0, 2)).sqrt().clamp_min(1e-300)
    return float((num / den).max())


def params_tensor_free(p):
    return dict(p)
