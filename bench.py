"""Benchmark of the CDG2 operator L_h on one GB300 (or N replicas).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference] [--config C] [--k K]

A step is one application of f(U) = M^{-1} L_h(U) (volume terms, face fluxes
with the CDG2 lifting, boundary influxes, inverse mass matrix) over the whole
mesh, in FP64, through the C ABI.  The default workload is the largest one
that the paper's 3D test suggests and one GPU holds: 3D 128x32x32 DG Q2
(21,233,664 DOF, 170 MB of state).  L2 is flushed (a 512 MB write) before
every timed step, outside the step's CUDA events.  The line also carries the
FP32 apply with its error against FP64, the JVP and VJP, the same figures on
3D 64x16x16 Q3 and 2D 256x64 Q3, the implicit solve (FP64 vs mixed), the
gradient through the implicit steps, the simplicial meshes, the end-to-end
rate through the API with host buffers, and the oracle timed on the host.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "L_h apply GDOF/s FP64 vs mixed at stated error; VJP GDOF/s; % HBM roofline"


def apply_flops_per_element(dim: int, k: int) -> int:
    """Floating-point operations per element of one FP64 apply (face-once path).

    Counted from the kernels' loops as they run (an FMA is 2 flops; an add,
    multiply or divide 1).  The 1D passes split even and odd modes (mirror
    symmetry of the Legendre modes at the symmetric Gauss rule): a forward line
    (k+1 modes to k+2 points) costs H (2b + 2) + 2 m flops with H = q // 2 point
    pairs and m the modes of the matrix's parity at the middle point; a
    transposed line 2H + 2Hb + 2m, a two-matrix transposed line 4H + 4Hb + 2b.
    Element kernel: values of all six species at the Gauss points, gradients
    of n1, c1, c3 only; the pointwise flux (43 + 28 d per point: the four
    sensitivities inverted together, Phi formed for n1 and n2 only); the test
    with grad phi for n1, n2 and with phi alone for n3..c3; the diffusion of
    n2..c3 in modal form (the nonzero entries of the 1D stiffness: same parity,
    both modes > 0); per axis the normal expansion of its two faces' tested
    fluxes.  Face kernel, one face per element and axis: normal contraction
    (owning trace, jump, both normal derivatives) of all six species, the
    modal diffusive fluxes of n3..c3 (9 per tangential mode and species),
    tangential interpolation of the four traces of n1, n2, c1, c3, the
    pointwise face flux of n1, n2 (about 90 per point, eight sensitivities
    inverted together), tangential test of sigma and tau of n1, n2.
    """
    b, q, d, s = k + 1, k + 2, dim, 6
    H, mid = q // 2, q % 2
    npar = {1: (b + 1) // 2, -1: b // 2}   # modes of each parity

    def fwd(par):
        return H * (2 * b + 2) + mid * 2 * npar[par]

    def tr(par):
        return 2 * H + 2 * H * b + mid * 2 * npar[par]

    tr2 = 4 * H + 4 * H * b + mid * 2 * b
    if d == 2:
        values = b * fwd(1) + q * fwd(1)
        grads = b * fwd(-1) + q * (fwd(1) + fwd(-1))
        test_grad = q * (tr2 + tr(1)) + b * tr2
        test_val = q * tr(1) + b * tr(1)
        interp, test = fwd(1), tr(1)
    else:
        values = b * b * fwd(1) + q * b * fwd(1) + q * q * fwd(1)
        grads = b * b * fwd(-1) + q * b * (fwd(1) + fwd(-1)) + q * q * (2 * fwd(1) + fwd(-1))
        test_grad = q * q * (tr2 + 2 * tr(1)) + q * b * (tr2 + tr(1)) + b * b * tr2
        test_val = q * q * tr(1) + q * b * tr(1) + b * b * tr(1)
        interp, test = b * fwd(1) + q * fwd(1), q * tr(1) + b * tr(1)
    nz = [0] + [len(range(1 if a % 2 else 2, b, 2)) for a in range(1, b)]   # stiffness entries per row
    modal = sum(2 * nz[a] for a in range(b)) * d * b ** (d - 1) + 2 * b ** d
    normal = b ** (d - 1) * (2 * (5 * b - 2) + 1)
    expand = 8 * b ** d
    volume = 6 * values + 3 * grads + 2 * test_grad + 4 * test_val + 5 * modal
    faces = d * (s * normal + 4 * 9 * b ** (d - 1) + 16 * interp + 4 * test + s * expand)
    pointwise = q ** d * (43 + 28 * d) + d * q ** (d - 1) * 90
    return volume + faces + pointwise


# dram__bytes_read.sum + dram__bytes_write.sum of one FP64 apply (its face and
# element kernels), from one ncu capture (profiles/), keyed by workload and
# valid only for the kernel sources the counters were taken with (first 16 hex
# of their sha256).
NCU_TRAFFIC = {("3D 128x32x32 Q2 seeded Gaussians", "double"): (1425181056, "bac2e07b6856edaa")}
KERNEL_SOURCES = ("paper_1403_1157_gb300/csrc/operator.cu", "paper_1403_1157_gb300/csrc/elem_common.cuh",
                  "paper_1403_1157_gb300/csrc/physics.cuh", "paper_1403_1157_gb300/csrc/tc_elem.cuh",
                  "paper_1403_1157_gb300/csrc/face3.cuh")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, dtype: str):
    entry = NCU_TRAFFIC.get((workload, dtype))
    if entry is None or entry[1] != kernel_source_hash():
        return None
    return entry[0]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_setup(cfg: int, k: int | None):
    import cdg2_inputs as I
    w = I.workload(cfg, k)
    return w, I


def max_over_ranks(value: float, dist, device) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's)."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, n_dof: int, steps: int, total_ms: float) -> float:
    """Whole-job GDOF/s: every rank applies the operator to its own replica of the
    workload (weak scaling), timed by the slowest rank."""
    return world * n_dof * steps / (total_ms * 1e-3) / 1e9


def make_inputs(G, w, I, mesh, dtype_flag=0):
    import torch
    dt = torch.float32 if dtype_flag else torch.float64
    U = torch.empty(mesh.n_dof, dtype=dt, device="cuda")
    p = I.default_params()
    if w.mms:
        ph = I.mms_phases(w.seed)
        G.cdg2_project_mms(mesh, G.make_params(p, ph), 0.0, U, dtype_flag)
    else:
        cen, amp = I.gaussian_draws(w.dim, w.extent, w.n_gauss, w.seed)
        G.cdg2_project_gaussians(mesh, cen, amp, w.sigma, w.floor, U, dtype_flag)
    return U, p


def time_applies(G, torch, mesh, p, U, out, flags, steps, warmup, flush):
    """CUDA-event times (ms) of `steps` applies, L2 flushed before each.  The
    applies are queued with CDG2_ASYNC (no host wait for the domain check) and
    the domain status is read once afterwards."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.fill_(1)
        G.cdg2_apply(mesh, p, U, out, flags | G.CDG2_ASYNC)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.fill_(1)
        a.record(stream)
        G.cdg2_apply(mesh, p, U, out, flags | G.CDG2_ASYNC)
        b.record(stream)
    torch.cuda.synchronize()
    G.cdg2_mesh_status(mesh)
    return [a.elapsed_time(b) for a, b in ev]


def time_op(G, torch, fn, steps, warmup, flush):
    """Mean CUDA-event time (ms) of fn() over `steps` calls, L2 flushed before each."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.fill_(1)
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.fill_(1)
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


# Algorithmic HBM bytes per DOF of one launch sequence: read the inputs and
# write the result once (neighbour traces re-read from L2 are not counted).
BYTES_PER_DOF = {("apply", "f64"): 16, ("apply", "f32"): 8, ("jvp", "f64"): 24, ("jvp", "f32"): 12,
                 ("vjp", "f64"): 24, ("vjp", "f32"): 12, ("apply", "tf32"): 8, ("jvp", "tf32"): 12}

# Tensor-core flops per element of the TF32 element kernel (3D Q3, dense per
# element, padded to 128 points): forward 128 x 64 x (6 values + 3 x 3
# gradients) x 2 per field, test 64 x 128 x (6 + 3 x 2) x 2.
TC_FLOPS_PER_ELEMENT = {"apply": 2 * 128 * 64 * 15 + 2 * 64 * 128 * 12, "jvp": 2 * 2 * 128 * 64 * 15 + 2 * 64 * 128 * 12}

# Floating-point operations per element of one launch sequence (face kernels +
# element kernel), measured: 2 x FMA + ADD + MUL instructions executed
# (smsp__sass_thread_inst_executed_op_{d,f}{fma,add,mul}_pred_on.sum, ncu, one
# launch of each kernel on a small mesh of the same dimension and degree,
# divided by its elements), keyed by (dim, k, op, dtype) and valid only for the
# kernel sources the counters were taken with (first 16 hex of their sha256).
FLOPS_PER_ELEMENT = {
    (3, 2, 'apply', 'f64'): (43229, 'bac2e07b6856edaa'),
    (3, 2, 'apply', 'f32'): (48177, 'bac2e07b6856edaa'),
    (3, 2, 'jvp', 'f64'): (64818, 'bac2e07b6856edaa'),
    (3, 2, 'jvp', 'f32'): (75684, 'bac2e07b6856edaa'),
    (3, 2, 'vjp', 'f64'): (126835, 'bac2e07b6856edaa'),
    (3, 2, 'vjp', 'f32'): (122861, 'bac2e07b6856edaa'),
    (3, 3, 'apply', 'f64'): (94326, 'bac2e07b6856edaa'),
    (3, 3, 'apply', 'f32'): (107442, 'bac2e07b6856edaa'),
    (3, 3, 'jvp', 'f64'): (138598, 'bac2e07b6856edaa'),
    (3, 3, 'jvp', 'f32'): (165252, 'bac2e07b6856edaa'),
    (3, 3, 'vjp', 'f64'): (266801, 'bac2e07b6856edaa'),
    (3, 3, 'vjp', 'f32'): (260276, 'bac2e07b6856edaa'),
    (2, 3, 'apply', 'f64'): (13299, 'bac2e07b6856edaa'),
    (2, 3, 'apply', 'f32'): (14206, 'bac2e07b6856edaa'),
    (2, 3, 'jvp', 'f64'): (19632, 'bac2e07b6856edaa'),
    (2, 3, 'jvp', 'f32'): (22050, 'bac2e07b6856edaa'),
    (2, 3, 'vjp', 'f64'): (32662, 'bac2e07b6856edaa'),
    (2, 3, 'vjp', 'f32'): (31681, 'bac2e07b6856edaa'),
}


def flops_per_element(dim, k, op, dtype):
    """(flops per element, source) for the ALU roofline: the ncu count when it
    matches the current kernel sources, else the loop model for the FP64 apply,
    else None."""
    entry = FLOPS_PER_ELEMENT.get((dim, k, op, dtype))
    if entry is not None and entry[1] == kernel_source_hash():
        return entry[0], "ncu instruction count"
    if op == "apply" and dtype == "f64":
        return apply_flops_per_element(dim, k), "loop model"
    return None, None


def leg(w, ms, op, dtype, peaks):
    """One timed launch sequence: GDOF/s, HBM fraction, ALU fraction (of the measured FMA peak)."""
    n = w.n_dof
    gb_s = BYTES_PER_DOF[(op, dtype)] * n / (ms * 1e-3) / 1e9
    out = {"ms": ms, "value": n / (ms * 1e-3) / 1e9, "unit": "GDOF/s", "hbm_frac": gb_s / peaks["hbm_gbs"]}
    if dtype == "tf32":
        tf = TC_FLOPS_PER_ELEMENT[op] * w.n_elem / (ms * 1e-3) / 1e12
        out.update({"tensor_tflops": tf, "tensor_frac_of_tf32_nominal": tf / 1125.0,
                    "tensor_note": "dense TF32 GEMM flops of the element kernel's contractions (all its launches "
                                   "in the time); nominal dense TF32 rate 1.125 PFLOP/s (half of bf16)"})
        return out
    fl, src = flops_per_element(w.dim, w.k, op, dtype)
    if fl is not None:
        tf = fl * w.n_elem / (ms * 1e-3) / 1e12
        out.update({"tflops": tf, "alu_frac": tf / peaks["fp64_tflops" if dtype == "f64" else "fp32_tflops"],
                    "flops_source": src})
    return out


def rel_err_per_species(torch, got, ref, w):
    e = got.double().view(w.n_elem, 6, -1) - ref.double().view(w.n_elem, 6, -1)
    r = ref.double().view(w.n_elem, 6, -1)
    return float((e.pow(2).sum(dim=(0, 2)).sqrt() / r.pow(2).sum(dim=(0, 2)).sqrt()).max())


def measure_operator(G, torch, w, mesh, p, U, flush, steps, peaks, with_fp64_apply=True):
    """FP64 and FP32 apply, JVP and VJP of one workload (L2 flushed before every
    launch sequence), each with its HBM and ALU fractions, and the FP32 apply's
    error against FP64 on the same (rounded) input."""
    A = G.CDG2_ASYNC
    lam = torch.sin(torch.arange(U.numel(), device="cuda", dtype=torch.float64) * 0.37)
    res = torch.empty_like(U)
    gth = torch.zeros(8, dtype=torch.float64, device="cuda")
    U32, lam32, res32 = U.float(), lam.float(), torch.empty_like(U, dtype=torch.float32)
    cases = {
        ("apply", "f32"): lambda: G.cdg2_apply(mesh, p, U32, res32, G.CDG2_MINV | G.CDG2_FP32 | A),
        ("jvp", "f64"): lambda: G.cdg2_jvp(mesh, p, U, lam, res, G.CDG2_MINV | A),
        ("jvp", "f32"): lambda: G.cdg2_jvp(mesh, p, U32, lam32, res32, G.CDG2_MINV | G.CDG2_FP32 | A),
        ("vjp", "f64"): lambda: G.cdg2_vjp(mesh, p, U, lam, res, gth, G.CDG2_MINV | A),
        ("vjp", "f32"): lambda: G.cdg2_vjp(mesh, p, U32, lam32, res32, gth, G.CDG2_MINV | G.CDG2_FP32 | A),
    }
    if with_fp64_apply:
        cases[("apply", "f64")] = lambda: G.cdg2_apply(mesh, p, U, res, G.CDG2_MINV | A)
    if w.dim == 3 and w.k == 3:
        TF = G.CDG2_MINV | G.CDG2_FP32 | G.CDG2_TF32 | A
        cases[("apply", "tf32")] = lambda: G.cdg2_apply(mesh, p, U32, res32, TF)
        cases[("jvp", "tf32")] = lambda: G.cdg2_jvp(mesh, p, U32, lam32, res32, TF)
    out = {}
    for (op, dt), fn in cases.items():
        ms = time_op(G, torch, fn, steps, 3, flush)
        out[f"{op}_{dt}"] = leg(w, ms, op, dt, peaks)
    G.cdg2_mesh_status(mesh)
    out32 = torch.empty_like(U32)
    G.cdg2_apply(mesh, p, U32, out32, G.CDG2_MINV | G.CDG2_FP32)
    ref64 = torch.empty_like(U)
    G.cdg2_apply(mesh, p, U32.double(), ref64, G.CDG2_MINV)
    out["apply_f32"]["rel_l2_err_vs_fp64_max_species"] = rel_err_per_species(torch, out32, ref64, w)
    if w.dim == 3 and w.k == 3:
        G.cdg2_apply(mesh, p, U32, out32, G.CDG2_MINV | G.CDG2_FP32 | G.CDG2_TF32)
        out["apply_tf32"]["rel_l2_err_vs_fp64_max_species"] = rel_err_per_species(torch, out32, ref64, w)
    return out


def measure_workload(G, torch, I, cfg, flush, steps, peaks):
    """measure_operator on workload cfg, with its name and sizes."""
    w = I.workload(cfg)
    mesh = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    U, p = make_inputs(G, w, I, mesh)
    r = measure_operator(G, torch, w, mesh, p, U, flush, steps, peaks)
    r.update({"workload": w.name, "n_dof": w.n_dof, "n_elem": w.n_elem})
    del mesh
    return r


def smooth_simplex_state(torch, mesh, centroids, psi0):
    """Piecewise-constant positive state: u_s = 0.5 + 0.3 sin(2 pi x + s) cos(pi y / 0.2)
    at each element's centroid in the mean coefficient (psi_0 = psi0), higher modes 0."""
    import numpy as np
    U = np.zeros((mesh.n_elem, 6, mesh.n_basis))
    x, y = centroids[:, 0], centroids[:, 1]
    for s in range(6):
        U[:, s, 0] = (0.5 + 0.3 * np.sin(2 * np.pi * x + s) * np.cos(np.pi * y / 0.2)) / psi0
    return torch.from_numpy(U).reshape(-1).cuda()


def measure_simplex(G, torch, flush, steps, mesh, p, U, apply, jvp, vjp, step, Us, dt):
    """Apply, JVP and VJP timings (L2 flushed) and one timed SDIRK3 step (FP64,
    element-block Jacobi, Newton relative residual 1e-10) from the smooth state Us."""
    out = torch.empty_like(U)
    dU = torch.ones_like(U)
    f = G.CDG2_MINV | G.CDG2_ASYNC
    ms = time_op(G, torch, lambda: apply(mesh, p, U, out, f), steps, 3, flush)
    ms_j = time_op(G, torch, lambda: jvp(mesh, p, U, dU, out, f), steps, 3, flush)
    ms_v = time_op(G, torch, lambda: vjp(mesh, p, U, dU, out, f), steps, 3, flush)
    apply(mesh, p, U, out, G.CDG2_MINV)      # waits, and reports a domain error of the timed calls
    opts = G.make_opts(scheme=G.CDG2_SDIRK3, newton_rtol=1e-10, gmres_rtol=1e-3, precond=2)
    step(mesh, p, Us.clone(), dt, opts, raise_on_error=False)      # allocates the workspace, probes the blocks
    torch.cuda.synchronize()
    V = Us.clone()
    t0 = time.perf_counter()
    rc, st = step(mesh, p, V, dt, opts, raise_on_error=False)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    n = mesh.n_dof
    return {"n_dof": n, "n_elem": mesh.n_elem, "n_faces": mesh.n_faces, "ms": ms,
            "value": n / (ms * 1e-3) / 1e9, "unit": "GDOF/s", "dtype": "f64",
            "jvp": {"ms": ms_j, "value": n / (ms_j * 1e-3) / 1e9, "unit": "GDOF/s"},
            "vjp": {"ms": ms_v, "value": n / (ms_v * 1e-3) / 1e9, "unit": "GDOF/s"},
            "step": {"scheme": "SDIRK3", "dt": dt, "status": rc, "s_per_step": sec,
                     "newton_iters": st["newton_iters"], "gmres_iters": st["gmres_iters"],
                     "newton_rtol": 1e-10, "gmres_rtol": 1e-3, "precond": "element-block Jacobi (blocks cached)",
                     "state": "piecewise-constant 0.5 + 0.3 sin(2 pi x + s) cos(pi y / 0.2)"}}


def measure_tri(G, torch, flush, steps):
    """FP64 cdg2_tri_apply / jvp / vjp on the 256x64x2 P3 triangle mesh (seeded
    jitter, seeded positive coefficients), L2 flushed before every timed launch
    pair, and one SDIRK3 step."""
    import cdg2_inputs as I
    w = I.tri_workload(1)
    xy, tri = I.tri_mesh(w.nx, w.ny, w.extent[0], w.extent[1], w.jitter, w.seed)
    mesh = G.cdg2_tri_mesh_create(xy, tri, w.k)
    p = I.default_params()
    U = torch.from_numpy(I.random_coefficients(mesh.n_elem, mesh.n_basis, w.seed, 0.1)).reshape(-1).cuda()
    Us = smooth_simplex_state(torch, mesh, xy[tri].mean(axis=1), 2.0 ** 0.5)
    r = measure_simplex(G, torch, flush, steps, mesh, p, U, G.cdg2_tri_apply, G.cdg2_tri_jvp, G.cdg2_tri_vjp,
                        G.cdg2_tri_step, Us, 1e-3)
    r.update({"workload": w.name, "kernels": "tri_face_kernel<3> + tri_elem_kernel<3> (one apply)"})
    return r


def measure_tet(G, torch, flush, steps):
    """FP64 cdg2_tet_apply / jvp / vjp on the 32x8x8x6 P3 tetrahedral mesh (seeded
    jitter, seeded positive coefficients), L2 flushed before every timed launch
    pair, and one SDIRK3 step."""
    import cdg2_inputs as I
    w = I.tet_workload(1)
    xyz, tet = I.tet_mesh(*w.cells, *w.extent, w.jitter, w.seed)
    mesh = G.cdg2_tet_mesh_create(xyz, tet, w.k)
    p = I.default_params()
    U = torch.from_numpy(I.random_coefficients(mesh.n_elem, mesh.n_basis, w.seed, 0.1)).reshape(-1).cuda()
    Us = smooth_simplex_state(torch, mesh, xyz[tet].mean(axis=1), 6.0 ** 0.5)
    r = measure_simplex(G, torch, flush, steps, mesh, p, U, G.cdg2_tet_apply, G.cdg2_tet_jvp, G.cdg2_tet_vjp,
                        G.cdg2_tet_step, Us, 1e-3)
    r.update({"workload": w.name, "kernels": "tet_face_kernel<3,2,0> + tet_elem_kernel<3,0> (one apply)"})
    return r


def measure_solve(G, torch, cfg: int, steps: int, precond: int):
    """Implicit SDIRK steps to Newton relative residual 1e-10: FP64 Krylov vs FP32 Krylov + FP64 refinement."""
    import cdg2_inputs as I
    w = I.workload(cfg)
    mesh = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    U0, p = make_inputs(G, w, I, mesh)
    scheme = G.CDG2_SDIRK2 if w.k == 1 else G.CDG2_SDIRK3
    result = {"workload": w.name, "n_dof": w.n_dof, "dt": w.dt, "steps": steps, "scheme": f"SDIRK{scheme}",
              "newton_rtol": 1e-10, "precond": {1: "modal diagonal", 2: "element-block Jacobi"}.get(precond, "none")}
    finals = {}
    # GMRES forcing term eta = 3e-3 for every precision: swept over 1e-4 .. 3e-2 on 3D 64x16x16 Q3
    # (SDIRK3, element blocks), the fastest setting of each of FP64, mixed FP32 and mixed TF32
    modes = [("fp64", 0, 3e-3), ("mixed", 1, 3e-3)]
    if w.dim == 3 and w.k == 3:
        modes.append(("mixed_tf32", 2, 3e-3))
    for mode, mixed, eta in modes:
        U = U0.clone()
        # one untimed step warms up the kernels and allocates the workspace
        G.cdg2_step(mesh, p, U.clone(), 0.0, w.dt, G.make_opts(scheme=scheme, mixed=mixed, newton_rtol=1e-10,
                                                                 gmres_rtol=eta, precond=precond))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        newton = gm = 0
        worst = 0.0
        for i in range(steps):
            rc, st = G.cdg2_step(mesh, p, U, i * w.dt, w.dt, G.make_opts(scheme=scheme, mixed=mixed, newton_rtol=1e-10,
                                                                          gmres_rtol=eta, precond=precond))
            newton += st["newton_iters"]
            gm += st["gmres_iters"]
            worst = max([worst] + [r / r0 for r, r0 in zip(st["residual"], st["residual0"]) if r0 > 0])
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        finals[mode] = U
        result[mode] = {"s_per_step": sec / steps, "newton_iters": newton, "gmres_iters": gm,
                        "gmres_rtol": eta, "max_final_rel_residual": worst,
                        "dof_steps_per_s": w.n_dof * steps / sec}
    d = finals["mixed"] - finals["fp64"]
    result["mixed_vs_fp64_rel_l2"] = float(d.norm() / finals["fp64"].norm())
    result["speedup_mixed_over_fp64"] = result["fp64"]["s_per_step"] / result["mixed"]["s_per_step"]
    if "mixed_tf32" in finals:
        d = finals["mixed_tf32"] - finals["fp64"]
        result["mixed_tf32_vs_fp64_rel_l2"] = float(d.norm() / finals["fp64"].norm())
        result["speedup_mixed_tf32_over_fp64"] = result["fp64"]["s_per_step"] / result["mixed_tf32"]["s_per_step"]
    return result


def measure_assembled(G, torch, cfg: int, flush, steps: int, peaks):
    """The assembled Jacobian (the paper's deferred alternative to the matrix-free
    JVP) on one workload: its assembly by JVP probing, its SpMV against the JVP
    (time, HBM fraction of the SpMV), and one SDIRK step solved with each."""
    import cdg2_inputs as I
    w = I.workload(cfg)
    mesh = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    U, p = make_inputs(G, w, I, mesh)
    A = G.cdg2_matrix_create(mesh)
    G.cdg2_assemble_jacobian(A, p, U)                 # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G.cdg2_assemble_jacobian(A, p, U)
    torch.cuda.synchronize()
    t_asm = time.perf_counter() - t0
    x = torch.sin(torch.arange(U.numel(), device="cuda", dtype=torch.float64) * 0.37)
    y = torch.empty_like(x)
    ms_spmv = time_op(G, torch, lambda: G.cdg2_spmv(A, x, y), steps, 3, flush)
    ms_jvp = time_op(G, torch, lambda: G.cdg2_jvp(mesh, p, U, x, y, G.CDG2_MINV | G.CDG2_ASYNC), steps, 3, flush)
    spmv_bytes = A.bytes + 2 * 8 * w.n_dof
    res = {"workload": w.name, "n_dof": w.n_dof, "block_size": A.block_size, "blocks_per_row": A.slots,
           "colours": A.colours, "matrix_bytes": A.bytes, "assembly_s": t_asm,
           "assembly_jvps": A.colours * A.block_size,
           "spmv": {"ms": ms_spmv, "gb_s": spmv_bytes / (ms_spmv * 1e-3) / 1e9,
                    "hbm_frac": spmv_bytes / (ms_spmv * 1e-3) / 1e9 / peaks["hbm_gbs"]},
           "jvp_fp64_ms": ms_jvp}
    scheme = G.CDG2_SDIRK2 if w.k == 1 else G.CDG2_SDIRK3
    for name, jac in (("matrix_free", 0), ("assembled", 1)):
        opts = G.make_opts(scheme=scheme, newton_rtol=1e-10, gmres_rtol=1e-3, precond=2, jacobian=jac)
        G.cdg2_step(mesh, p, U.clone(), 0.0, w.dt, opts)
        torch.cuda.synchronize()
        V = U.clone()
        t0 = time.perf_counter()
        rc, st = G.cdg2_step(mesh, p, V, 0.0, w.dt, opts)
        torch.cuda.synchronize()
        res["step_" + name] = {"s": time.perf_counter() - t0, "newton_iters": st["newton_iters"],
                               "gmres_iters": st["gmres_iters"], "status": rc}
    del A
    return res


def measure_gradient(G, torch, cfg: int, steps: int | None, mixed: bool, precond: int):
    """Forward + checkpointed discrete-adjoint backward of J = int n3(T) w.r.t. (U0, theta)."""
    import numpy as np

    import cdg2_inputs as I
    from paper_1403_1157_gb300 import adjoint as Adj
    w = I.workload(cfg)
    nsteps = steps or w.steps
    cp = w.extra.get("checkpoint", 10)
    mesh = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    U0, p = make_inputs(G, w, I, mesh)
    theta = torch.tensor([p[n] for n in Adj.THETA_NAMES], dtype=torch.float64, device="cuda")
    scheme = G.CDG2_SDIRK2 if w.k == 1 else G.CDG2_SDIRK3
    opts = G.make_opts(scheme=scheme, mixed=mixed, newton_rtol=1e-10, gmres_rtol=1e-4 if mixed else 1e-3,
                       precond=precond)
    vol = float(np.prod([e / c for e, c in zip(w.extent[: w.dim], w.cells[: w.dim])]))
    U = U0.clone().requires_grad_(True)
    th = theta.clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    UT = Adj.steps(U, th, mesh, p, 0.0, w.dt, nsteps, cp, opts)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    J = vol * UT.view(mesh.n_elem, 6, mesh.n_basis)[:, 2, 0].sum()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return {"workload": w.name, "n_dof": w.n_dof, "steps": nsteps, "checkpoint": cp, "dt": w.dt,
            "precision": "mixed" if mixed else "fp64",
            "precond": {1: "modal diagonal", 2: "element-block Jacobi"}.get(precond, "none"),
            "forward_s": t1 - t0, "backward_s": t2 - t1,
            "functional": "int n3(T)", "dJ_dtheta": [float(v) for v in th.grad],
            "dJ_dU0_norm": float(U.grad.norm())}


def oracle_sample(w):
    """A bounded sample of workload w for the oracle: the full mesh when its
    apply is small, else a slab of the full cross-section (the first axis and
    y in full, the last axis cut to 2 cells, still periodic) with the same
    element size and state recipe."""
    cells = list(w.cells[: w.dim])
    if w.n_dof > 2_000_000:
        cells[-1] = 2
    ext = [w.extent[a] * cells[a] / w.cells[a] for a in range(w.dim)]
    return cells, ext


def cpu_oracle_baseline(w, seconds: float = 12.0, seconds_1_thread: float = 6.0):
    """The oracle (plain FP64 PyTorch CPU) timed on this host on a bounded
    sample of the same workload, on all the threads torch uses and then on one thread."""
    import torch

    import cdg2_inputs as I
    from oracle import cdg2_oracle as O
    cells, ext = oracle_sample(w)
    om = O.Mesh(w.dim, cells, ext, w.periodic, w.k)
    p = I.default_params()
    U = torch.from_numpy(I.random_coefficients(om.E, om.nb, w.seed))
    ndof = 6 * om.E * om.nb

    def timed(limit):
        O.apply(om, U, p)
        reps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < limit:
            O.apply(om, U, p)
            reps += 1
        return reps, time.perf_counter() - t0

    cores = torch.get_num_threads()
    reps, dt = timed(seconds)
    torch.set_num_threads(1)
    try:
        reps1, dt1 = timed(seconds_1_thread)
    finally:
        torch.set_num_threads(cores)
    return {"value": ndof * reps / dt / 1e9, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} oracle applies on {cells} cells ({ndof} DOF each) of {w.name} in {dt:.1f} s",
            "value_1_thread": ndof * reps1 / dt1 / 1e9,
            "sample_1_thread": f"{reps1} applies on one thread in {dt1:.1f} s"}


def run_reference(args):
    """--impl reference: the oracle on the host cores, K timed steps (rank 0 only),
    each step one oracle apply on a bounded sample of the workload."""
    import torch

    import cdg2_inputs as I
    from oracle import cdg2_oracle as O
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = I.workload(args.config, args.k)
    cells, ext = oracle_sample(w)
    p = I.default_params()

    def sample(cells, ext):
        om = O.Mesh(w.dim, cells, ext, w.periodic, w.k)
        return om, torch.from_numpy(I.random_coefficients(om.E, om.nb, w.seed))

    om, U = sample(cells, ext)
    t0 = time.perf_counter()
    O.apply(om, U, p)
    t_one = time.perf_counter() - t0
    # bound the whole run to about two minutes: shrink the sample along y if needed
    budget = 120.0 / max(1, args.steps + args.warmup)
    if t_one > budget:
        cells[1] = max(2, int(cells[1] * budget / t_one))
        ext[1] = w.extent[1] * cells[1] / w.cells[1]
        om, U = sample(cells, ext)
    ndof = 6 * om.E * om.nb
    for _ in range(args.warmup):
        O.apply(om, U, p)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.apply(om, U, p)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = ndof * args.steps / total / 1e9
    sample_txt = f"{args.steps} oracle applies on {cells} cells of {w.name} ({ndof} DOF each)"
    line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w.name, "n_dof": w.n_dof, "sample_cells": cells, "sample_dof": ndof},
            "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": sample_txt},
            "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measured_peaks(G, torch):
    """HBM and bf16 from MEASURED_PEAKS.json; the FP64 and FP32 FMA rates measured
    here with the library's FMA-loop probe (best of 3)."""
    peaks, kind = load_peaks()
    peaks = dict(peaks)
    peaks["fp64_tflops"] = max(G.cdg2_probe_peak(0, 1 << 15) for _ in range(3))
    peaks["fp32_tflops"] = max(G.cdg2_probe_peak(1, 1 << 19) for _ in range(3))
    torch.cuda.synchronize()
    return peaks, kind


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--k", type=int, default=None)
    ap.add_argument("--extra-configs", default="3,1", help="workloads timed beside the headline (comma list; '' none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tri", action="store_true", help="skip the triangle- and tetrahedral-mesh timings")
    ap.add_argument("--solve-config", type=int, default=3, help="workload of the implicit-solve comparison")
    ap.add_argument("--solve-steps", type=int, default=2, help="timed implicit steps per precision (0: skip)")
    ap.add_argument("--grad-config", type=int, default=2, help="workload of the gradient-through-steps timing")
    ap.add_argument("--assembled-config", type=int, default=2,
                    help="workload of the assembled-Jacobian comparison (-1: skip)")
    ap.add_argument("--profile-solve", choices=["mixed", "mixed_tf32", "fp64"], default=None,
                    help="run one implicit step of the solve workload and exit (for ncu launch lists)")
    ap.add_argument("--profile-op", default=None,
                    help="cfg:op:dtype[:reps[:cells]] (several separated by ';'), e.g. 3:jvp:f32:1:16x8x8: only "
                         "those launch sequences, reps times each, on the workload's mesh or a smaller one with "
                         "the given cells, then exit (for ncu captures)")
    ap.add_argument("--precond", type=int, default=2, choices=[0, 1, 2],
                    help="GMRES preconditioner of the solve timing (1: modal diagonal, 2: element blocks)")
    ap.add_argument("--grad-precond", type=int, default=1, choices=[0, 1, 2],
                    help="GMRES preconditioner of the gradient timing (its adjoint solves have smooth right-hand "
                         "sides, where the modal diagonal needs fewer iterations)")
    ap.add_argument("--grad-steps", type=int, default=-1, help="steps of the gradient timing (-1: the workload's; 0: skip)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_solve:
        import torch

        import cdg2_inputs as I
        import paper_1403_1157_gb300 as G
        w = I.workload(args.solve_config)
        mesh = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
        U, p = make_inputs(G, w, I, mesh)
        mixed = {"mixed": 1, "mixed_tf32": 2, "fp64": 0}[args.profile_solve]
        scheme = G.CDG2_SDIRK2 if w.k == 1 else G.CDG2_SDIRK3
        rc, st = G.cdg2_step(mesh, p, U, 0.0, w.dt, G.make_opts(scheme=scheme, mixed=mixed, newton_rtol=1e-10,
                                                                 gmres_rtol=1e-4 if mixed else 1e-3,
                                                                 precond=args.precond))
        print(json.dumps({"profile_solve": args.profile_solve, "precond": args.precond, "workload": w.name,
                          "stats": st}))
        return
    if args.profile_op:
        import torch

        import cdg2_inputs as I
        import paper_1403_1157_gb300 as G
        done = []
        for spec in args.profile_op.split(";"):
            parts = spec.split(":")
            cfg, op, dt = int(parts[0]), parts[1], parts[2]
            reps = int(parts[3]) if len(parts) > 3 else 3
            w = I.workload(cfg)
            cells = tuple(int(c) for c in parts[4].split("x")) if len(parts) > 4 else w.cells[: w.dim]
            ext = tuple(w.extent[a] * cells[a] / w.cells[a] for a in range(w.dim))
            mesh = G.cdg2_mesh_create(w.dim, cells, ext, w.periodic, w.k)
            U, p = make_inputs(G, w, I, mesh)
            fl = G.CDG2_MINV | (G.CDG2_FP32 if dt in ("f32", "tf32") else 0) | (G.CDG2_TF32 if dt == "tf32" else 0)
            if dt in ("f32", "tf32"):
                U = U.float()
            lam = torch.sin(torch.arange(U.numel(), device="cuda", dtype=U.dtype) * 0.37)
            out = torch.empty_like(U)
            gth = torch.zeros(8, dtype=torch.float64, device="cuda")
            for _ in range(reps):
                if op == "apply":
                    G.cdg2_apply(mesh, p, U, out, fl)
                elif op == "jvp":
                    G.cdg2_jvp(mesh, p, U, lam, out, fl)
                else:
                    G.cdg2_vjp(mesh, p, U, lam, out, gth, fl)
            torch.cuda.synchronize()
            done.append({"spec": spec, "workload": w.name, "cells": list(cells), "n_elem": mesh.n_elem})
        print(json.dumps({"profile_op": done}))
        return

    import torch
    import torch.distributed as dist

    import paper_1403_1157_gb300 as G
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w, I = workload_setup(args.config, args.k)
    mesh = G.cdg2_mesh_create(w.dim, w.cells, w.extent, w.periodic, w.k)
    U, p = make_inputs(G, w, I, mesh)
    out = torch.empty_like(U)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    peaks, kind = measured_peaks(G, torch)
    torch.cuda.synchronize()

    # ---- timed region: K FP64 applies, L2 flushed before each ----
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(uuid)
    time.sleep(0.4)
    t_wall = time.perf_counter()
    ms = time_applies(G, torch, mesh, p, U, out, G.CDG2_MINV, args.steps, args.warmup, flush)
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    total_ms = sum(ms)
    if world > 1:
        total_ms = max_over_ranks(total_ms, dist, "cuda")
        dist.barrier()
    ms_step = total_ms / args.steps
    value = job_throughput(world, w.n_dof, args.steps, total_ms)

    # ---- roofline of the timed launch sequence (the face kernels + the element kernel) ----
    head = leg(w, ms_step, "apply", "f64", peaks)
    fl_el, fl_src = flops_per_element(w.dim, w.k, "apply", "f64")
    fl = fl_el * w.n_elem
    achieved_tf = fl / (ms_step * 1e-3) / 1e12

    # ---- FP32 apply, JVP and VJP on the headline workload, then the extra workloads ----
    nsub = max(10, args.steps // 8)
    ops = measure_operator(G, torch, w, mesh, p, U, flush, nsub, peaks, with_fp64_apply=False)
    extras = {}
    for c in [int(x) for x in args.extra_configs.split(",") if x.strip()]:
        if c != args.config:
            r = measure_workload(G, torch, I, c, flush, nsub, peaks)
            extras[r["workload"]] = r

    # ---- end to end through the API: pinned host U -> device, apply, result -> pinned host,
    # then the domain status (the call a user makes to know the result is valid) ----
    hU = U.cpu().pin_memory()
    hout = torch.empty_like(hU).pin_memory()
    dU = torch.empty_like(U)
    stream = torch.cuda.current_stream()
    n_e2e = max(10, args.steps // 4)

    def e2e_step():
        dU.copy_(hU, non_blocking=True)
        G.cdg2_apply(mesh, p, dU, out, G.CDG2_MINV | G.CDG2_ASYNC)
        hout.copy_(out, non_blocking=True)
        G.cdg2_mesh_status(mesh)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n_e2e):
        e2e_step()
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / n_e2e
    nbytes = U.numel() * U.element_size()
    e2e = {"value": world * w.n_dof / (e2e_ms * 1e-3) / 1e9, "unit": "GDOF/s", "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}
    del dU, hU, hout

    tri = measure_tri(G, torch, flush, nsub) if not args.no_tri else None
    tet = measure_tet(G, torch, flush, nsub) if not args.no_tri else None
    solve = measure_solve(G, torch, args.solve_config, args.solve_steps, args.precond) if args.solve_steps > 0 else None
    assembled = measure_assembled(G, torch, args.assembled_config, flush, nsub, peaks) \
        if args.assembled_config >= 0 else None
    grad = None
    if args.grad_steps != 0:
        grad = measure_gradient(G, torch, args.grad_config, None if args.grad_steps < 0 else args.grad_steps, True,
                                args.grad_precond)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_oracle_baseline(w)
    line = {
        "metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_dof": w.n_dof, "n_elem": w.n_elem, "degree": w.k,
                   "l2": "flushed before every timed step (512 MB write outside the step events); "
                         "the state (FP64, in and out) is also larger than L2",
                   "step": "one cdg2_apply (M^-1 L_h, FP64) over the whole mesh"},
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                     "frac": achieved_tf / peaks["fp64_tflops"], "traffic": ncu_traffic(w.name, "double"),
                     "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one apply's launches (bytes), "
                                     "ncu capture of the same workload; null once the kernel sources changed",
                     "algorithmic_bytes": BYTES_PER_DOF[("apply", "f64")] * w.n_dof,
                     "peak_note": "FP64 FMA rate measured in this run by cdg2_probe_peak (FMA loop, 8 chains per "
                                  "thread, 8 x SMs blocks of 256 threads); achieved = flops of one apply / its "
                                  "event time (all its launches)",
                     "flops_per_apply": fl, "flops_source": fl_src,
                     "kernels": (f"3 x face3_kernel<{w.k},0,A,double>" if w.dim == 3 else
                                 f"2 x face_kernel<2,{w.k},0,A,double>") + f" + op_kernel<{w.dim},{w.k},0,double> (one apply)",
                     "hbm_frac": head["hbm_frac"], "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_kind": kind,
                     "fp32_peak_tflops": peaks["fp32_tflops"]},
        "fp32": ops.pop("apply_f32"),
        "derivatives": ops,
        "workloads": extras,
        "triangles": tri,
        "tetrahedra": tet,
        "solve": solve,
        "gradient": grad,
        "assembled": assembled,
        "e2e": e2e,
        "gpu_launches": args.steps * (1 + w.dim),
        "clocks": clk,
        "wall_s_timed_region": t_wall,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
