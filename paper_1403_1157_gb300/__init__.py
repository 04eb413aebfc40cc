"""Python binding of the CDG2 CUDA library (``include/cdg2.h``).

Argument marshalling only: every step of the operator, its derivatives and
the time stepper runs in the library's CUDA kernels.  PyTorch tensors supply
device memory and streams.  There is no CPU fallback: importing works
without a GPU, but every call needs the built ``libcdg2.so`` and a CUDA
device, and raises otherwise.
"""
from __future__ import annotations

import ctypes
import os

import torch

__all__ = [
    "CDG2_MINV", "CDG2_FORCING", "CDG2_FP32", "Cdg2Error", "Mesh", "load_library", "library_path",
    "make_params", "cdg2_mesh_create", "cdg2_mesh_destroy", "cdg2_mesh_info", "cdg2_apply", "cdg2_last_error",
    "cdg2_project_gaussians", "cdg2_project_mms", "cdg2_jvp", "cdg2_vjp", "cdg2_step",
    "CDG2_SDIRK2", "CDG2_SDIRK3", "CDG2_SDIRK4", "SolverOpts", "Stats", "make_opts", "cdg2_step_stages", "cdg2_step_adjoint",
    "stages_of", "CDG2_ASYNC", "CDG2_ERR_DOMAIN", "cdg2_mesh_status", "cdg2_tri_mesh_status", "cdg2_tet_mesh_status",
    "cdg2_probe_peak", "CDG2_TF32", "Matrix", "cdg2_matrix_create", "cdg2_assemble_jacobian", "cdg2_spmv",
]

CDG2_MINV = 1
CDG2_FORCING = 2
CDG2_FP32 = 4
CDG2_ASYNC = 8
CDG2_TF32 = 16
CDG2_ERR_INVALID_ARG = -1
CDG2_ERR_CUDA = -2
CDG2_ERR_NOT_CONVERGED = -3
CDG2_ERR_NONFINITE = -4
CDG2_ERR_DOMAIN = -5
CDG2_SDIRK2 = 2
CDG2_SDIRK3 = 3
CDG2_SDIRK4 = 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


class Cdg2Error(RuntimeError):
    """A CDG2 call returned a negative status."""

    def __init__(self, code: int, msg: str):
        super().__init__(f"CDG2 error {code}: {msg}")
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("cells", ctypes.c_int * 3),
        ("extent", ctypes.c_double * 3),
        ("periodic", ctypes.c_int * 3),
        ("k", ctypes.c_int),
        ("q1", ctypes.c_int),
        ("chi_e", ctypes.c_double),
        ("gamma1_in", ctypes.c_double * 2),
        ("flux", ctypes.c_int),
        ("penalty", ctypes.c_double),
    ]


class Params(ctypes.Structure):
    _fields_ = [
        ("mu", ctypes.c_double * 3),
        ("nu", ctypes.c_double * 3),
        ("chi0", ctypes.c_double * 4),
        ("chith", ctypes.c_double * 4),
        ("d1", ctypes.c_double), ("d2", ctypes.c_double), ("gamma", ctypes.c_double),
        ("alpha1", ctypes.c_double), ("alpha2", ctypes.c_double), ("f1", ctypes.c_double),
        ("k_ox", ctypes.c_double),
        ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("sigma", ctypes.c_double),
        ("c1_star", ctypes.c_double), ("c1_star2", ctypes.c_double),
        ("bc_sign", ctypes.c_double),
        ("mms_phase", ctypes.c_double * 6),
        ("model", ctypes.c_int),
    ]


class SolverOpts(ctypes.Structure):
    _fields_ = [
        ("scheme", ctypes.c_int), ("mixed", ctypes.c_int), ("flags", ctypes.c_int), ("max_newton", ctypes.c_int),
        ("gmres_restart", ctypes.c_int), ("max_gmres", ctypes.c_int),
        ("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double), ("gmres_rtol", ctypes.c_double),
        ("precond", ctypes.c_int), ("jacobian", ctypes.c_int),
    ]


class TriDesc(ctypes.Structure):
    _fields_ = [
        ("n_vert", ctypes.c_longlong),
        ("xy", ctypes.POINTER(ctypes.c_double)),
        ("n_tri", ctypes.c_longlong),
        ("tri", ctypes.POINTER(ctypes.c_longlong)),
        ("k", ctypes.c_int),
        ("chi_e", ctypes.c_double),
        ("gamma1_in", ctypes.c_double * 2),
    ]


class TetDesc(ctypes.Structure):
    _fields_ = [
        ("n_vert", ctypes.c_longlong),
        ("xyz", ctypes.POINTER(ctypes.c_double)),
        ("n_tet", ctypes.c_longlong),
        ("tet", ctypes.POINTER(ctypes.c_longlong)),
        ("k", ctypes.c_int),
        ("chi_e", ctypes.c_double),
        ("gamma1_in", ctypes.c_double * 2),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("stages", ctypes.c_int), ("newton_iters", ctypes.c_int), ("gmres_iters", ctypes.c_int),
        ("residual0", ctypes.c_double * 5), ("residual", ctypes.c_double * 5), ("seconds", ctypes.c_double),
        ("gmres_reorth", ctypes.c_int),
    ]

    def as_dict(self):
        return {"stages": self.stages, "newton_iters": self.newton_iters, "gmres_iters": self.gmres_iters,
                "residual0": list(self.residual0)[: self.stages], "residual": list(self.residual)[: self.stages],
                "seconds": self.seconds, "gmres_reorth": self.gmres_reorth}


def library_path() -> str:
    return os.path.join(_HERE, "libcdg2.so")


def load_library():
    """Load ``libcdg2.so`` (built in-tree by ``build.py``); raise if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CDG2 CUDA library not built ({path} missing); run paper_1403_1157_gb300.build")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.cdg2_mesh_create.argtypes = [ctypes.POINTER(MeshDesc), ctypes.POINTER(vp)]
    lib.cdg2_mesh_create.restype = i
    lib.cdg2_mesh_destroy.argtypes = [vp]
    lib.cdg2_mesh_destroy.restype = None
    lib.cdg2_mesh_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i),
                                   ctypes.POINTER(ctypes.c_longlong)]
    lib.cdg2_mesh_info.restype = i
    for name in ("cdg2_mesh_status", "cdg2_tri_mesh_status", "cdg2_tet_mesh_status"):
        getattr(lib, name).argtypes = [vp, vp]
        getattr(lib, name).restype = i
    lib.cdg2_apply.argtypes = [vp, ctypes.POINTER(Params), vp, vp, i, d, vp]
    lib.cdg2_apply.restype = i
    dp = ctypes.POINTER(ctypes.c_double)
    lib.cdg2_jvp.argtypes = [vp, ctypes.POINTER(Params), vp, vp, dp, vp, i, d, vp]
    lib.cdg2_jvp.restype = i
    lib.cdg2_vjp.argtypes = [vp, ctypes.POINTER(Params), vp, vp, vp, vp, i, d, vp]
    lib.cdg2_vjp.restype = i
    lib.cdg2_step.argtypes = [vp, ctypes.POINTER(Params), vp, d, d, ctypes.POINTER(SolverOpts), ctypes.POINTER(Stats),
                              vp]
    lib.cdg2_step.restype = i
    lib.cdg2_step_stages.argtypes = [vp, ctypes.POINTER(Params), vp, d, d, ctypes.POINTER(SolverOpts), vp,
                                     ctypes.POINTER(Stats), vp]
    lib.cdg2_step_stages.restype = i
    lib.cdg2_step_adjoint.argtypes = [vp, ctypes.POINTER(Params), vp, d, d, ctypes.POINTER(SolverOpts), vp, vp,
                                      ctypes.POINTER(Stats), vp]
    lib.cdg2_step_adjoint.restype = i
    lib.cdg2_project_gaussians.argtypes = [vp, i, dp, dp, d, d, vp, i, vp]
    lib.cdg2_project_gaussians.restype = i
    lib.cdg2_project_mms.argtypes = [vp, ctypes.POINTER(Params), d, vp, i, vp]
    lib.cdg2_project_mms.restype = i
    lib.cdg2_tri_mesh_create.argtypes = [ctypes.POINTER(TriDesc), ctypes.POINTER(vp)]
    lib.cdg2_tri_mesh_create.restype = i
    lib.cdg2_tri_mesh_destroy.argtypes = [vp]
    lib.cdg2_tri_mesh_destroy.restype = None
    lib.cdg2_tri_mesh_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i),
                                       ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.cdg2_tri_mesh_info.restype = i
    lib.cdg2_tri_apply.argtypes = [vp, ctypes.POINTER(Params), vp, vp, i, vp]
    lib.cdg2_tri_apply.restype = i
    lib.cdg2_tri_jvp.argtypes = [vp, ctypes.POINTER(Params), vp, vp, vp, i, vp]
    lib.cdg2_tri_jvp.restype = i
    lib.cdg2_tri_vjp.argtypes = [vp, ctypes.POINTER(Params), vp, vp, vp, i, vp]
    lib.cdg2_tri_vjp.restype = i
    lib.cdg2_tet_mesh_create.argtypes = [ctypes.POINTER(TetDesc), ctypes.POINTER(vp)]
    lib.cdg2_tet_mesh_create.restype = i
    lib.cdg2_tet_mesh_destroy.argtypes = [vp]
    lib.cdg2_tet_mesh_destroy.restype = None
    lib.cdg2_tet_mesh_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i),
                                       ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.cdg2_tet_mesh_info.restype = i
    lib.cdg2_tet_apply.argtypes = [vp, ctypes.POINTER(Params), vp, vp, i, vp]
    lib.cdg2_tet_apply.restype = i
    for name in ("cdg2_tet_jvp", "cdg2_tet_vjp"):
        getattr(lib, name).argtypes = [vp, ctypes.POINTER(Params), vp, vp, vp, i, vp]
        getattr(lib, name).restype = i
    for name in ("cdg2_tri_step", "cdg2_tet_step"):
        getattr(lib, name).argtypes = [vp, ctypes.POINTER(Params), vp, d, ctypes.POINTER(SolverOpts),
                                       ctypes.POINTER(Stats), vp]
        getattr(lib, name).restype = i
    lib.cdg2_element_block.argtypes = [vp, ctypes.POINTER(Params), d, ctypes.c_longlong, i, dp]
    lib.cdg2_element_block.restype = i
    lib.cdg2_matrix_create.argtypes = [vp, ctypes.POINTER(vp)]
    lib.cdg2_matrix_create.restype = i
    lib.cdg2_matrix_destroy.argtypes = [vp]
    lib.cdg2_matrix_destroy.restype = None
    lib.cdg2_matrix_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                     ctypes.POINTER(ctypes.c_longlong)]
    lib.cdg2_matrix_info.restype = i
    lib.cdg2_assemble_jacobian.argtypes = [vp, ctypes.POINTER(Params), vp, vp]
    lib.cdg2_assemble_jacobian.restype = i
    lib.cdg2_spmv.argtypes = [vp, d, vp, d, vp, vp]
    lib.cdg2_spmv.restype = i
    lib.cdg2_probe_peak.argtypes = [i, i, ctypes.POINTER(ctypes.c_double), vp]
    lib.cdg2_probe_peak.restype = i
    lib.cdg2_last_error.argtypes = []
    lib.cdg2_last_error.restype = ctypes.c_char_p
    _LIB = lib
    return lib


def cdg2_last_error() -> str:
    return load_library().cdg2_last_error().decode()


def _check(code: int):
    if code != 0:
        raise Cdg2Error(code, cdg2_last_error())


def make_params(p: dict, mms_phase=None) -> Params:
    """cdg2_params from a coefficient dict (keys of ``cdg2_inputs.default_params``)."""
    out = Params()
    for j in range(3):
        out.mu[j] = float(p["mu"][j])
        out.nu[j] = float(p["nu"][j])
    for j in range(4):
        out.chi0[j] = float(p["chi0"][j])
        out.chith[j] = float(p["chith"][j])
    for key in ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox", "beta1", "beta2", "sigma",
                "c1_star", "c1_star2", "bc_sign"):
        setattr(out, key, float(p[key]))
    ph = mms_phase if mms_phase is not None else p.get("mms_phase", (0.0,) * 6)
    for j in range(6):
        out.mms_phase[j] = float(ph[j])
    out.model = int(p.get("model", 0))
    return out


class Mesh:
    """Owning handle of a cdg2_mesh."""

    def __init__(self, handle: int, desc: MeshDesc):
        self.handle = handle
        self.desc = desc
        lib = load_library()
        ne, nb, nd = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_longlong()
        _check(lib.cdg2_mesh_info(handle, ctypes.byref(ne), ctypes.byref(nb), ctypes.byref(nd)))
        self.n_elem, self.n_basis, self.n_dof = ne.value, nb.value, nd.value
        self.dim, self.k = desc.dim, desc.k

    @property
    def shape(self):
        return (self.n_elem, 6, self.n_basis)

    def close(self):
        if self.handle:
            load_library().cdg2_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


CDG2_FLUX_CDG2, CDG2_FLUX_BR2, CDG2_FLUX_SIPG = 0, 1, 2


def cdg2_mesh_create(dim, cells, extent, periodic, k, q1=0, chi_e=0.0, gamma1_in=(0.375, 0.625), flux=0,
                     penalty=0.0) -> Mesh:
    desc = MeshDesc()
    desc.dim = int(dim)
    for a in range(3):
        desc.cells[a] = int(cells[a]) if a < len(cells) else 1
        desc.extent[a] = float(extent[a]) if a < len(extent) else 1.0
        desc.periodic[a] = int(periodic[a]) if a < len(periodic) else 1
    desc.k = int(k)
    desc.q1 = int(q1)
    desc.chi_e = float(chi_e)
    desc.gamma1_in[0], desc.gamma1_in[1] = float(gamma1_in[0]), float(gamma1_in[1])
    desc.flux = int(flux)
    desc.penalty = float(penalty)
    h = ctypes.c_void_p()
    _check(load_library().cdg2_mesh_create(ctypes.byref(desc), ctypes.byref(h)))
    return Mesh(h.value, desc)


def cdg2_mesh_destroy(mesh: Mesh):
    mesh.close()


def cdg2_mesh_info(mesh: Mesh):
    return mesh.n_elem, mesh.n_basis, mesh.n_dof


class Matrix:
    """Owning handle of a cdg2_matrix (the assembled Jacobian of a Cartesian mesh)."""

    def __init__(self, mesh: Mesh):
        h = ctypes.c_void_p()
        _check(load_library().cdg2_matrix_create(mesh.handle, ctypes.byref(h)))
        self.handle, self.mesh = h.value, mesh
        b, sl, nc, nb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        _check(load_library().cdg2_matrix_info(self.handle, ctypes.byref(b), ctypes.byref(sl), ctypes.byref(nc),
                                               ctypes.byref(nb)))
        self.block_size, self.slots, self.colours, self.bytes = b.value, sl.value, nc.value, nb.value

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.cdg2_matrix_destroy(self.handle)
            self.handle = None


def cdg2_matrix_create(mesh: Mesh) -> Matrix:
    return Matrix(mesh)


def cdg2_assemble_jacobian(A: Matrix, params, U: torch.Tensor, stream=None):
    """A = J(U) (the Jacobian of M^{-1} L_h at the float64 CUDA state U)."""
    p = _params(params)
    _check(load_library().cdg2_assemble_jacobian(A.handle, ctypes.byref(p), _dev(U, A.mesh, torch.float64, "U"),
                                                 _stream_ptr(stream)))


def cdg2_spmv(A: Matrix, x: torch.Tensor, y: torch.Tensor, alpha: float = 1.0, beta: float = 0.0, stream=None):
    """y = alpha A x + beta y (float64 CUDA vectors of n_dof)."""
    _check(load_library().cdg2_spmv(A.handle, float(alpha), _dev(x, A.mesh, torch.float64, "x"), float(beta),
                                    _dev(y, A.mesh, torch.float64, "y"), _stream_ptr(stream)))
    return y


def cdg2_probe_peak(kind: int, iters: int, stream=None) -> float:
    """Measured FMA throughput in TFLOP/s of the current GPU: kind 0 = FP64, 1 = FP32."""
    out = ctypes.c_double()
    _check(load_library().cdg2_probe_peak(int(kind), int(iters), ctypes.byref(out), _stream_ptr(stream)))
    return out.value


def cdg2_mesh_status(mesh: Mesh, stream=None):
    """Wait for the stream and raise Cdg2Error(CDG2_ERR_DOMAIN) if a kernel queued on
    the mesh (with CDG2_ASYNC) met the pole of chi; clears the status."""
    _check(load_library().cdg2_mesh_status(mesh.handle, _stream_ptr(stream)))


def cdg2_tri_mesh_status(mesh, stream=None):
    """cdg2_mesh_status of a triangle mesh."""
    _check(load_library().cdg2_tri_mesh_status(mesh.handle, _stream_ptr(stream)))


def cdg2_tet_mesh_status(mesh, stream=None):
    """cdg2_mesh_status of a tetrahedral mesh."""
    _check(load_library().cdg2_tet_mesh_status(mesh.handle, _stream_ptr(stream)))


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t: torch.Tensor, mesh: Mesh, dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != mesh.n_dof:
        raise ValueError(f"{name} must be contiguous with {mesh.n_dof} elements")
    return ctypes.c_void_p(t.data_ptr())


def _params(params):
    return params if isinstance(params, Params) else make_params(params)


def cdg2_apply(mesh: Mesh, params, U: torch.Tensor, out: torch.Tensor, flags: int = CDG2_MINV, t: float = 0.0,
               stream=None) -> torch.Tensor:
    """out = M^{-1} L_h(U) (CDG2_MINV) on the given (default: current) stream."""
    dt = torch.float32 if flags & CDG2_FP32 else torch.float64
    p = _params(params)
    _check(load_library().cdg2_apply(mesh.handle, ctypes.byref(p), _dev(U, mesh, dt, "U"),
                                     _dev(out, mesh, dt, "out"), int(flags), float(t), _stream_ptr(stream)))
    return out


def cdg2_project_gaussians(mesh: Mesh, centres, amps, sigma: float, floor_value: float, out: torch.Tensor,
                           flags: int = 0, stream=None) -> torch.Tensor:
    """out = L2 projection of floor + sum of Gaussian bumps (centres[6][n][dim], amps[6][n])."""
    n = len(amps[0])
    flat_c = [float(v) for s in range(6) for b in range(n) for v in centres[s][b][: mesh.dim]]
    flat_a = [float(v) for s in range(6) for v in amps[s]]
    cc = (ctypes.c_double * max(1, len(flat_c)))(*flat_c)
    aa = (ctypes.c_double * max(1, len(flat_a)))(*flat_a)
    dt = torch.float32 if flags & CDG2_FP32 else torch.float64
    _check(load_library().cdg2_project_gaussians(mesh.handle, n, cc, aa, float(sigma), float(floor_value),
                                                 _dev(out, mesh, dt, "out"), int(flags), _stream_ptr(stream)))
    return out


def cdg2_project_mms(mesh: Mesh, params, t: float, out: torch.Tensor, flags: int = 0, stream=None) -> torch.Tensor:
    """out = L2 projection of the manufactured solution at time t (phases from params)."""
    dt = torch.float32 if flags & CDG2_FP32 else torch.float64
    p = _params(params)
    _check(load_library().cdg2_project_mms(mesh.handle, ctypes.byref(p), float(t), _dev(out, mesh, dt, "out"),
                                           int(flags), _stream_ptr(stream)))
    return out


def cdg2_element_block(mesh: Mesh, params, gdt: float, elem: int, species: int) -> torch.Tensor:
    """The block I - gdt A_s K_e that precond = 2 inverts (host call), as an
    (n_basis, n_basis) float64 CPU tensor."""
    nb = mesh.n_basis
    out = (ctypes.c_double * (nb * nb))()
    p = _params(params)
    _check(load_library().cdg2_element_block(mesh.handle, ctypes.byref(p), float(gdt), int(elem), int(species), out))
    return torch.tensor(list(out), dtype=torch.float64).reshape(nb, nb)


class TriMesh:
    """Owning handle of a cdg2_tri_mesh."""

    def __init__(self, handle: int, k: int):
        self.handle = handle
        self.k = k
        ne, nb, nd, nf = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(load_library().cdg2_tri_mesh_info(handle, ctypes.byref(ne), ctypes.byref(nb), ctypes.byref(nd),
                                                 ctypes.byref(nf)))
        self.n_elem, self.n_basis, self.n_dof, self.n_faces = ne.value, nb.value, nd.value, nf.value

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.cdg2_tri_mesh_destroy(self.handle)
            self.handle = None


def cdg2_tri_mesh_create(xy, tri, k: int, chi_e: float = 0.0, gamma1_in=(0.375, 0.625)) -> TriMesh:
    """Triangle mesh from vertex coordinates xy [n_v][2] and counter-clockwise triples tri [n_t][3]."""
    import numpy as np
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int64)
    d = TriDesc()
    d.n_vert = xy.shape[0]
    d.xy = xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_tri = tri.shape[0]
    d.tri = tri.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
    d.k = int(k)
    d.chi_e = float(chi_e)
    d.gamma1_in[0], d.gamma1_in[1] = float(gamma1_in[0]), float(gamma1_in[1])
    h = ctypes.c_void_p()
    _check(load_library().cdg2_tri_mesh_create(ctypes.byref(d), ctypes.byref(h)))
    return TriMesh(h.value, int(k))


def cdg2_tri_apply(mesh: TriMesh, params, U: torch.Tensor, out: torch.Tensor, flags: int = CDG2_MINV,
                   stream=None) -> torch.Tensor:
    """out = M^{-1} L_h(U) on a triangle mesh (float64 CUDA tensors of n_dof values)."""
    for name, t in (("U", U), ("out", out)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == mesh.n_dof):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {mesh.n_dof} values")
    p = _params(params)
    _check(load_library().cdg2_tri_apply(mesh.handle, ctypes.byref(p), ctypes.c_void_p(U.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), int(flags), _stream_ptr(stream)))
    return out


def cdg2_tri_jvp(mesh: TriMesh, params, U: torch.Tensor, dU: torch.Tensor, out: torch.Tensor,
                 flags: int = CDG2_MINV, stream=None) -> torch.Tensor:
    """out = J(U) dU on a triangle mesh (float64 CUDA tensors of n_dof values)."""
    for name, t in (("U", U), ("dU", dU), ("out", out)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == mesh.n_dof):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {mesh.n_dof} values")
    p = _params(params)
    _check(load_library().cdg2_tri_jvp(mesh.handle, ctypes.byref(p), ctypes.c_void_p(U.data_ptr()),
                                       ctypes.c_void_p(dU.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(flags),
                                       _stream_ptr(stream)))
    return out


def cdg2_tri_vjp(mesh: TriMesh, params, U: torch.Tensor, lam: torch.Tensor, gU: torch.Tensor,
                 flags: int = CDG2_MINV, stream=None) -> torch.Tensor:
    """gU = J(U)^T lam on a triangle mesh (float64 CUDA tensors of n_dof values)."""
    for name, t in (("U", U), ("lam", lam), ("gU", gU)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == mesh.n_dof):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {mesh.n_dof} values")
    p = _params(params)
    _check(load_library().cdg2_tri_vjp(mesh.handle, ctypes.byref(p), ctypes.c_void_p(U.data_ptr()),
                                       ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(gU.data_ptr()), int(flags),
                                       _stream_ptr(stream)))
    return gU


class TetMesh:
    """Owning handle of a cdg2_tet_mesh."""

    def __init__(self, handle: int, k: int):
        self.handle = handle
        self.k = k
        ne, nb, nd, nf = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(load_library().cdg2_tet_mesh_info(handle, ctypes.byref(ne), ctypes.byref(nb), ctypes.byref(nd),
                                                 ctypes.byref(nf)))
        self.n_elem, self.n_basis, self.n_dof, self.n_faces = ne.value, nb.value, nd.value, nf.value

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.cdg2_tet_mesh_destroy(self.handle)
            self.handle = None


def cdg2_tet_mesh_create(xyz, tet, k: int, chi_e: float = 0.0, gamma1_in=(0.375, 0.625)) -> TetMesh:
    """Tetrahedral mesh from vertex coordinates xyz [n_v][3] and positively oriented quadruples tet [n_t][4]."""
    import numpy as np
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tet = np.ascontiguousarray(tet, dtype=np.int64)
    d = TetDesc()
    d.n_vert = xyz.shape[0]
    d.xyz = xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    d.n_tet = tet.shape[0]
    d.tet = tet.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))
    d.k = int(k)
    d.chi_e = float(chi_e)
    d.gamma1_in[0], d.gamma1_in[1] = float(gamma1_in[0]), float(gamma1_in[1])
    h = ctypes.c_void_p()
    _check(load_library().cdg2_tet_mesh_create(ctypes.byref(d), ctypes.byref(h)))
    return TetMesh(h.value, int(k))


def cdg2_tet_apply(mesh: TetMesh, params, U: torch.Tensor, out: torch.Tensor, flags: int = CDG2_MINV,
                   stream=None) -> torch.Tensor:
    """out = M^{-1} L_h(U) on a tetrahedral mesh (float64 CUDA tensors of n_dof values)."""
    for name, t in (("U", U), ("out", out)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == mesh.n_dof):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {mesh.n_dof} values")
    p = _params(params)
    _check(load_library().cdg2_tet_apply(mesh.handle, ctypes.byref(p), ctypes.c_void_p(U.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), int(flags), _stream_ptr(stream)))
    return out


def cdg2_tet_jvp(mesh: TetMesh, params, U: torch.Tensor, dU: torch.Tensor, out: torch.Tensor,
                 flags: int = CDG2_MINV, stream=None) -> torch.Tensor:
    """out = J(U) dU on a tetrahedral mesh (float64 CUDA tensors of n_dof values)."""
    for name, t in (("U", U), ("dU", dU), ("out", out)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == mesh.n_dof):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {mesh.n_dof} values")
    p = _params(params)
    _check(load_library().cdg2_tet_jvp(mesh.handle, ctypes.byref(p), ctypes.c_void_p(U.data_ptr()),
                                       ctypes.c_void_p(dU.data_ptr()), ctypes.c_void_p(out.data_ptr()), int(flags),
                                       _stream_ptr(stream)))
    return out


def cdg2_tet_vjp(mesh: TetMesh, params, U: torch.Tensor, lam: torch.Tensor, gU: torch.Tensor,
                 flags: int = CDG2_MINV, stream=None) -> torch.Tensor:
    """gU = J(U)^T lam on a tetrahedral mesh (float64 CUDA tensors of n_dof values)."""
    for name, t in (("U", U), ("lam", lam), ("gU", gU)):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == mesh.n_dof):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {mesh.n_dof} values")
    p = _params(params)
    _check(load_library().cdg2_tet_vjp(mesh.handle, ctypes.byref(p), ctypes.c_void_p(U.data_ptr()),
                                       ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(gU.data_ptr()), int(flags),
                                       _stream_ptr(stream)))
    return gU


def _theta_ptr(dtheta):
    if dtheta is None:
        return None
    vals = [float(v) for v in dtheta]
    if len(vals) != 8:
        raise ValueError("dtheta must hold 8 values (d1, d2, gamma, alpha1, alpha2, f1, k_ox, beta1)")
    return (ctypes.c_double * 8)(*vals)


def cdg2_jvp(mesh: Mesh, params, U: torch.Tensor, dU: torch.Tensor, out: torch.Tensor, flags: int = CDG2_MINV,
             dtheta=None, t: float = 0.0, stream=None) -> torch.Tensor:
    """out = J(U) dU (+ df/dtheta dtheta) on the given (default: current) stream."""
    dt = torch.float32 if flags & CDG2_FP32 else torch.float64
    p = _params(params)
    _check(load_library().cdg2_jvp(mesh.handle, ctypes.byref(p), _dev(U, mesh, dt, "U"), _dev(dU, mesh, dt, "dU"),
                                   _theta_ptr(dtheta), _dev(out, mesh, dt, "out"), int(flags), float(t),
                                   _stream_ptr(stream)))
    return out


def cdg2_vjp(mesh: Mesh, params, U: torch.Tensor, lam: torch.Tensor, gU: torch.Tensor, gtheta: torch.Tensor = None,
             flags: int = CDG2_MINV, t: float = 0.0, stream=None) -> torch.Tensor:
    """gU = J(U)^T lam; gtheta (a CUDA float64 tensor of 8, optional) = (df/dtheta)^T lam."""
    dt = torch.float32 if flags & CDG2_FP32 else torch.float64
    gth = None
    if gtheta is not None:
        if not (gtheta.is_cuda and gtheta.dtype == torch.float64 and gtheta.numel() == 8 and gtheta.is_contiguous()):
            raise ValueError("gtheta must be a contiguous CUDA float64 tensor of 8 values")
        gth = ctypes.c_void_p(gtheta.data_ptr())
    p = _params(params)
    _check(load_library().cdg2_vjp(mesh.handle, ctypes.byref(p), _dev(U, mesh, dt, "U"), _dev(lam, mesh, dt, "lam"),
                                   _dev(gU, mesh, dt, "gU"), gth, int(flags), float(t), _stream_ptr(stream)))
    return gU


def make_opts(scheme=CDG2_SDIRK2, mixed=False, flags=0, max_newton=20, gmres_restart=30, max_gmres=300,
              newton_rtol=1e-10, newton_atol=0.0, gmres_rtol=1e-3, precond=1, jacobian=0) -> SolverOpts:
    o = SolverOpts()
    o.scheme, o.flags, o.max_newton = int(scheme), int(flags), int(max_newton)
    o.mixed = int(mixed) if not isinstance(mixed, bool) else int(mixed)   # 0, 1 (FP32) or 2 (TF32 tensor cores)
    o.gmres_restart, o.max_gmres = int(gmres_restart), int(max_gmres)
    o.newton_rtol, o.newton_atol, o.gmres_rtol = float(newton_rtol), float(newton_atol), float(gmres_rtol)
    o.precond = int(precond)
    o.jacobian = int(jacobian)
    return o


def cdg2_step(mesh: Mesh, params, U: torch.Tensor, t: float, dt: float, opts: SolverOpts = None, stream=None,
              raise_on_error: bool = True):
    """One SDIRK step in place on the float64 CUDA tensor U; returns (status, stats dict)."""
    p = _params(params)
    o = opts if opts is not None else make_opts()
    st = Stats()
    rc = load_library().cdg2_step(mesh.handle, ctypes.byref(p), _dev(U, mesh, torch.float64, "U"), float(t), float(dt),
                                  ctypes.byref(o), ctypes.byref(st), _stream_ptr(stream))
    if rc != 0 and raise_on_error:
        _check(rc)
    return rc, st.as_dict()


def _simplex_step(fn, mesh, params, U: torch.Tensor, dt: float, opts, stream, raise_on_error):
    if not (U.is_cuda and U.dtype == torch.float64 and U.is_contiguous() and U.numel() == mesh.n_dof):
        raise ValueError(f"U must be a contiguous CUDA float64 tensor of {mesh.n_dof} values")
    p = _params(params)
    o = opts if opts is not None else make_opts(precond=0)
    st = Stats()
    rc = fn(mesh.handle, ctypes.byref(p), ctypes.c_void_p(U.data_ptr()), float(dt), ctypes.byref(o), ctypes.byref(st),
            _stream_ptr(stream))
    if rc != 0 and raise_on_error:
        _check(rc)
    return rc, st.as_dict()


def cdg2_tri_step(mesh: "TriMesh", params, U: torch.Tensor, dt: float, opts: SolverOpts = None, stream=None,
                  raise_on_error: bool = True):
    """One SDIRK step (FP64, no preconditioner) in place on U on a triangle mesh; returns (status, stats)."""
    return _simplex_step(load_library().cdg2_tri_step, mesh, params, U, dt, opts, stream, raise_on_error)


def cdg2_tet_step(mesh: "TetMesh", params, U: torch.Tensor, dt: float, opts: SolverOpts = None, stream=None,
                  raise_on_error: bool = True):
    """One SDIRK step (FP64, no preconditioner) in place on U on a tetrahedral mesh; returns (status, stats)."""
    return _simplex_step(load_library().cdg2_tet_step, mesh, params, U, dt, opts, stream, raise_on_error)


def stages_of(opts: SolverOpts) -> int:
    return {CDG2_SDIRK2: 2, CDG2_SDIRK3: 3, CDG2_SDIRK4: 5}[opts.scheme]


def cdg2_step_stages(mesh: Mesh, params, U: torch.Tensor, t: float, dt: float, stages: torch.Tensor,
                     opts: SolverOpts = None, stream=None):
    """cdg2_step that also stores the stage values into stages (float64 CUDA, [s * n_dof])."""
    p = _params(params)
    o = opts if opts is not None else make_opts()
    if not (stages.is_cuda and stages.dtype == torch.float64 and stages.is_contiguous()
            and stages.numel() == stages_of(o) * mesh.n_dof):
        raise ValueError("stages must be a contiguous CUDA float64 tensor of s * n_dof values")
    st = Stats()
    _check(load_library().cdg2_step_stages(mesh.handle, ctypes.byref(p), _dev(U, mesh, torch.float64, "U"), float(t),
                                           float(dt), ctypes.byref(o), ctypes.c_void_p(stages.data_ptr()),
                                           ctypes.byref(st), _stream_ptr(stream)))
    return st.as_dict()


def cdg2_step_adjoint(mesh: Mesh, params, stages: torch.Tensor, t: float, dt: float, lam: torch.Tensor,
                      gtheta: torch.Tensor = None, opts: SolverOpts = None, stream=None):
    """lam <- (dU_{n+1}/dU_n)^T lam; gtheta += (dU_{n+1}/dtheta)^T lam (in place)."""
    p = _params(params)
    o = opts if opts is not None else make_opts()
    gth = None
    if gtheta is not None:
        if not (gtheta.is_cuda and gtheta.dtype == torch.float64 and gtheta.numel() == 8):
            raise ValueError("gtheta must be a CUDA float64 tensor of 8 values")
        gth = ctypes.c_void_p(gtheta.data_ptr())
    st = Stats()
    _check(load_library().cdg2_step_adjoint(mesh.handle, ctypes.byref(p), ctypes.c_void_p(stages.data_ptr()),
                                            float(t), float(dt), ctypes.byref(o), _dev(lam, mesh, torch.float64, "lam"),
                                            gth, ctypes.byref(st), _stream_ptr(stream)))
    return st.as_dict()
