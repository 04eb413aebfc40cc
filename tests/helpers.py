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


def gaussian_state(om, n_gauss=4, sigma=0.05, floor=1e-3, seed=1157):
    """Seeded Gaussian initial field projected by the oracle (the input recipe of the workloads)."""
    cen, amp = I.gaussian_draws(om.dim, om.extent, n_gauss, seed)
    return O.project(om, lambda x: O.gaussian_field(om, x, cen, amp, sigma, floor))


def random_state(om, seed=5, scale=0.1):
    return torch.from_numpy(I.random_coefficients(om.E, om.nb, seed, scale))


def rel_l2_per_species(got, ref):
    """max over species of ||got_s - ref_s||_2 / ||ref_s||_2 (coefficient vectors)."""
    got = got.detach().to("cpu", F64).reshape(ref.shape)
    num = ((got - ref) ** 2).sum(dim=(0, 2)).sqrt()
    den = (ref ** 2).sum(dim=(0, 2)).sqrt().clamp_min(1e-300)
    return float((num / den).max())


def params_tensor_free(p):
    return dict(p)
