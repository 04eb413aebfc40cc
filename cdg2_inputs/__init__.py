"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds random-number generation and plain data only (workload
sizes, coefficient presets, Gaussian centres and amplitudes, manufactured-
solution phases).  It contains none of the method's arithmetic: evaluating
and projecting the initial field, the operator and the time stepper live on
each side separately.

Random draws use SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds and a final xor-shift.  A uniform double
on [0,1) takes the top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator; ``uniform()`` returns a double in [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


# Species order of the state vector U = (n1, n2, n3, c1, c2, c3) (Sec. 2).
SPECIES = ("n1", "n2", "n3", "c1", "c2", "c3")
N_SPECIES = 6


def default_params() -> dict:
    """Builder preset of every model coefficient.

    The paper prints no numeric coefficient values; these are documented
    defaults chosen for a smooth, positive, diffusion-dominated regime, not
    the paper's.  Keys follow Eq. (1) and Eq. (3): motilities mu/nu, tactic
    sensitivities chi(x, y, a, b) = a x / (y + b) with (a, b) = (chi0, chith)
    for the pairs 11, 13, 21 (n2 towards c1) and 22 (n2 against n1; the paper
    reuses the 21 constants there, so the defaults are equal), death rates
    d1, d2, debris constant gamma (< 0), neutralisation alpha1, alpha2,
    debris-dependent production f1 (taken constant), oxidation rate k_ox,
    inflow rates beta1, beta2, sigma and thresholds c1_star, c1_star2.
    ``bc_sign`` = +1 reads the normal in Eq. (3) as the inward one (so the
    boundary terms are influxes), -1 as the outward one.
    """
    return dict(
        mu=(1e-2, 5e-3, 1e-3),
        nu=(5e-2, 5e-2, 5e-2),
        chi0=(1e-2, 5e-3, 5e-3, 5e-3),     # chi11, chi13, chi21, chi22
        chith=(0.1, 0.1, 0.1, 0.1),
        d1=0.1, d2=0.05, gamma=-0.1, alpha1=1.0, alpha2=0.5, f1=0.1, k_ox=0.5,
        beta1=1.0, beta2=0.5, sigma=1.0, c1_star=0.01, c1_star2=0.02,
        bc_sign=1.0,
    )


# The 8 reaction coefficients a gradient is taken with respect to.
THETA_NAMES = ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox", "beta1")


@dataclass
class Workload:
    """One named synthetic workload: mesh, degree and stepping sizes."""
    name: str
    dim: int
    cells: tuple
    extent: tuple
    periodic: tuple
    k: int
    n_gauss: int = 4
    sigma: float = 0.05
    floor: float = 1e-3
    seed: int = 1157
    steps: int = 0
    dt: float = 0.0
    mms: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def n_elem(self) -> int:
        return math.prod(self.cells[: self.dim])

    @property
    def n_basis(self) -> int:
        return (self.k + 1) ** self.dim

    @property
    def n_dof(self) -> int:
        return N_SPECIES * self.n_elem * self.n_basis


def workload(cfg: int, k: int | None = None) -> Workload:
    """The five synthetic workloads shaped like the paper's 2D and 3D tests.

    0: 2D 32x8 Q1 (about 6k DOF), 1: 2D 256x64 Q2/Q3 (manufactured
    solution), 2: 2D 128x32 Q2 (differentiation), 3: 3D 64x16x16 Q3 (6.3M
    DOF), 4: 3D 128x32x32 Q2 (21.2M DOF).  Domain [0,1]x[0,0.2](x[0,0.2]),
    y = 0 the lumen side, y = 0.2 the outer wall, periodic in x (and z).
    """
    ext2 = (1.0, 0.2, 1.0)
    ext3 = (1.0, 0.2, 0.2)
    per2 = (1, 0, 0)
    per3 = (1, 0, 1)
    if cfg == 0:
        return Workload("2D 32x8 Q1 seeded Gaussians", 2, (32, 8, 1), ext2, per2, 1 if k is None else k,
                        seed=1157, steps=20, dt=1e-3)
    if cfg == 1:
        kk = 3 if k is None else k
        return Workload(f"2D 256x64 Q{kk} manufactured solution", 2, (256, 64, 1), ext2, per2, kk,
                        seed=1158, steps=20, dt=1e-4, mms=True)
    if cfg == 2:
        return Workload("2D 128x32 Q2 seeded Gaussians", 2, (128, 32, 1), ext2, per2, 2 if k is None else k,
                        seed=1159, steps=50, dt=1e-3, extra=dict(checkpoint=10))
    if cfg == 3:
        return Workload("3D 64x16x16 Q3 seeded Gaussians", 3, (64, 16, 16), ext3, per3, 3 if k is None else k,
                        n_gauss=8, sigma=0.04, seed=1160, steps=10, dt=1e-3)
    if cfg == 4:
        return Workload("3D 128x32x32 Q2 seeded Gaussians", 3, (128, 32, 32), ext3, per3, 2 if k is None else k,
                        n_gauss=8, sigma=0.04, seed=1161, steps=20, dt=1e-3, extra=dict(checkpoint=5))
    raise ValueError(f"unknown workload {cfg}")


def gaussian_draws(dim: int, extent, n_gauss: int, seed: int):
    """Centres and amplitudes of the seeded Gaussian bumps of every species.

    For each species in order, then each bump: the ``dim`` centre
    coordinates (uniform in the box), then the amplitude (uniform in [0,1)).
    Returns (centres[6][n_gauss][dim], amps[6][n_gauss]) as nested lists.
    """
    rng = SplitMix64(seed)
    centres, amps = [], []
    for _s in range(N_SPECIES):
        cs, a_s = [], []
        for _g in range(n_gauss):
            cs.append([rng.uniform() * extent[j] for j in range(dim)])
            a_s.append(rng.uniform())
        centres.append(cs)
        amps.append(a_s)
    return centres, amps


def mms_phases(seed: int):
    """Per-species phases in [0, 2 pi) of the manufactured solution."""
    rng = SplitMix64(seed ^ 0x5EED)
    return [2.0 * math.pi * rng.uniform() for _ in range(N_SPECIES)]


def splitmix64_uniform_array(seed: int, n: int):
    """The first ``n`` SplitMix64 uniforms of ``seed`` as a float64 numpy array.

    Same stream as ``SplitMix64(seed).uniform()`` called ``n`` times: the
    i-th state is seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64).
    """
    import numpy as np
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def random_coefficients(n_elem: int, n_basis: int, seed: int, scale: float = 0.1):
    """A positive random coefficient field [E][6][n_b] as a float64 numpy array.

    Coefficient 0 (the cell mean for the orthonormal basis) is drawn in
    [0.5, 1.5); mode i > 0 in +-scale / (1 + i).  Used for parity cases that
    need arbitrary discrete states rather than smooth ones.
    """
    import numpy as np
    u = splitmix64_uniform_array(seed, n_elem * N_SPECIES * n_basis).reshape(n_elem, N_SPECIES, n_basis)
    i = np.arange(n_basis, dtype=np.float64)
    out = scale * (2.0 * u - 1.0) / (1.0 + i)
    out[:, :, 0] = 0.5 + u[:, :, 0]
    return out


def tri_mesh(nx: int, ny: int, lx: float = 1.0, ly: float = 0.2, jitter: float = 0.0, seed: int = 0):
    """A triangulation of [0, lx] x [0, ly]: an nx x ny grid of vertices moved
    by seeded jitter, each quad cut into two triangles.

    Vertices (i, j), i fastest, sit at (i lx / nx, j ly / ny); interior
    vertices are shifted by jitter * h * (2u - 1) per coordinate (u from
    SplitMix64(seed), x then y per vertex in index order), boundary vertices
    stay.  Quad (i, j) (i fastest) with corners a = (i, j), b = (i+1, j),
    c = (i+1, j+1), d = (i, j+1) gives the triangles (a, b, c), (a, c, d)
    when i + j is even and (a, b, d), (b, c, d) when odd, all counter-
    clockwise.  Returns (xy [n_vert][2] float64, tri [n_tri][3] int64) numpy
    arrays.  jitter < 0.25 keeps every triangle valid.
    """
    import numpy as np
    hx, hy = lx / nx, ly / ny
    nv = (nx + 1) * (ny + 1)
    u = splitmix64_uniform_array(seed, 2 * nv).reshape(nv, 2)
    xy = np.zeros((nv, 2))
    for j in range(ny + 1):
        for i in range(nx + 1):
            v = j * (nx + 1) + i
            xy[v] = (i * hx, j * hy)
            if 0 < i < nx and 0 < j < ny:
                xy[v, 0] += jitter * hx * (2.0 * u[v, 0] - 1.0)
                xy[v, 1] += jitter * hy * (2.0 * u[v, 1] - 1.0)
    tri = []
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            b, c, d = a + 1, a + nx + 2, a + nx + 1
            tri += [(a, b, c), (a, c, d)] if (i + j) % 2 == 0 else [(a, b, d), (b, c, d)]
    return xy, np.array(tri, dtype=np.int64)


@dataclass
class TriWorkload:
    name: str
    nx: int
    ny: int
    k: int
    jitter: float
    seed: int
    extent: tuple = (1.0, 0.2)

    @property
    def n_elem(self) -> int:
        return 2 * self.nx * self.ny

    @property
    def n_basis(self) -> int:
        return (self.k + 1) * (self.k + 2) // 2

    @property
    def n_dof(self) -> int:
        return N_SPECIES * self.n_elem * self.n_basis


def tri_workload(which: int, k: int | None = None) -> TriWorkload:
    """Triangle workloads (the paper's 2D runs use triangles, P_k, chi_e = 1.5):
    0: 16x4 quads (128 triangles) P2, jitter 0.2, seed 1170 (oracle sized);
    1: 256x64 quads (32,768 triangles) P3, jitter 0.2, seed 1171
    (983,040 DOF; the same domain and vertex spacing as the 256x64 Q3 mesh)."""
    if which == 0:
        return TriWorkload("2D triangles 16x4x2 P2 (jittered)", 16, 4, 2 if k is None else k, 0.2, 1170)
    if which == 1:
        return TriWorkload("2D triangles 256x64x2 P3 (jittered)", 256, 64, 3 if k is None else k, 0.2, 1171)
    raise ValueError(f"unknown triangle workload {which}")


def tet_mesh(nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 0.2, lz: float = 0.2, jitter: float = 0.0,
             seed: int = 0):
    """A tetrahedral mesh of [0, lx] x [0, ly] x [0, lz]: an (nx+1)(ny+1)(nz+1)
    vertex grid, interior vertices moved by jitter * h * (2u - 1) per coordinate
    (SplitMix64(seed); x, y, z per vertex in index order, i fastest), each cell
    cut into the six tetrahedra of Kuhn's subdivision: for every ordering
    (a, b, c) of the axes, (v, v + e_a, v + e_a + e_b, v + e_a + e_b + e_c)
    from the cell's lower corner v, axis orderings in lexicographic order; for
    an odd ordering the last two vertices are swapped, so every tetrahedron is
    positively oriented.  The subdivision is conforming across cells.
    Returns (xyz [n_vert][3] float64, tet [n_tet][4] int64) numpy arrays.
    """
    import itertools
    import numpy as np
    h = (lx / nx, ly / ny, lz / nz)
    n = (nx + 1, ny + 1, nz + 1)
    nv = n[0] * n[1] * n[2]
    u = splitmix64_uniform_array(seed, 3 * nv).reshape(nv, 3)
    xyz = np.zeros((nv, 3))
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                v = (k * n[1] + j) * n[0] + i
                xyz[v] = (i * h[0], j * h[1], k * h[2])
                if 0 < i < nx and 0 < j < ny and 0 < k < nz:
                    for a in range(3):
                        xyz[v, a] += jitter * h[a] * (2.0 * u[v, a] - 1.0)

    def vid(i, j, k):
        return (k * n[1] + j) * n[0] + i

    tets = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for perm in itertools.permutations(range(3)):
                    p = [i, j, k]
                    verts = [vid(*p)]
                    for a in perm:
                        p[a] += 1
                        verts.append(vid(*p))
                    inversions = sum(1 for x in range(3) for y in range(x + 1, 3) if perm[x] > perm[y])
                    if inversions % 2:
                        verts[2], verts[3] = verts[3], verts[2]
                    tets.append(verts)
    return xyz, np.array(tets, dtype=np.int64)


@dataclass
class TetWorkload:
    name: str
    cells: tuple
    k: int
    jitter: float
    seed: int
    extent: tuple = (1.0, 0.2, 0.2)

    @property
    def n_elem(self) -> int:
        return 6 * self.cells[0] * self.cells[1] * self.cells[2]

    @property
    def n_basis(self) -> int:
        return (self.k + 1) * (self.k + 2) * (self.k + 3) // 6

    @property
    def n_dof(self) -> int:
        return N_SPECIES * self.n_elem * self.n_basis


def tet_workload(which: int, k: int | None = None) -> TetWorkload:
    """Tetrahedral workloads (the paper's 3D runs use tetrahedra, P_k, chi_e = 2):
    0: 3x2x2 cells (72 tetrahedra) P2, jitter 0.15, seed 1180 (oracle sized);
    1: 32x8x8 cells (12,288 tetrahedra) P3, jitter 0.15, seed 1181 (1,474,560
    DOF on the box of the 3D workloads)."""
    if which == 0:
        return TetWorkload("3D tetrahedra 3x2x2x6 P2 (jittered)", (3, 2, 2), 2 if k is None else k, 0.15, 1180)
    if which == 1:
        return TetWorkload("3D tetrahedra 32x8x8x6 P3 (jittered)", (32, 8, 8), 3 if k is None else k, 0.15, 1181)
    raise ValueError(f"unknown tetrahedral workload {which}")
