// Internal types shared by the host layer and the kernels of the CDG2 library.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <string>

#include "cdg2.h"

namespace cdg2 {

constexpr int NS = 6;      // species (n1, n2, n3, c1, c2, c3), Sec. 2
constexpr int MAXK = 3;    // highest supported degree
constexpr int MAXQ = MAXK + 2;

// 1D tables on the reference interval [0,1] for degree k and q1 = k+2 Gauss
// points: psi_a(xi) = sqrt(2a+1) P_a(2 xi - 1) and its derivative.
struct Tab1D {
    double B[MAXQ][MAXK + 1];   // psi_a(xi_q)
    double D[MAXQ][MAXK + 1];   // d psi_a / d xi at xi_q
    double w[MAXQ];             // Gauss weights on [0,1] (sum 1)
    double xi[MAXQ];            // Gauss points on [0,1]
    double e[2][MAXK + 1];      // psi_a(0), psi_a(1)
    double d[2][MAXK + 1];      // psi'_a(0), psi'_a(1)
};

// The 1D tables in a kernel's precision, with the mesh spacing and Gauss
// weights folded in per axis j (derivatives divided by h_j; weighted test
// tables).  Built once per mesh on the host, passed to the operator kernels
// by value, so a kernel's set-up is a plain copy.
template <typename T>
struct TabP {
    T B[MAXQ][MAXK + 1];          // psi_a(xi_q)
    T Bw[MAXQ][MAXK + 1];         // w_q psi_a(xi_q)
    T Dh[3][MAXQ][MAXK + 1];      // psi'_a(xi_q) / h_j
    T Dwh[3][MAXQ][MAXK + 1];     // w_q psi'_a(xi_q) / h_j
    T w[MAXQ];
    T xi[MAXQ];
    T e[2][MAXK + 1];             // psi_a(0), psi_a(1)
    T dh[3][2][MAXK + 1];         // psi'_a(0) / h_j, psi'_a(1) / h_j
    T K1h[3][MAXK + 1][MAXK + 1]; // sum_q w_q psi'_a psi'_b / h_j^2 (exact 1D stiffness)
};

// Uniform Cartesian geometry (Sec. 3.1 tessellation, read as boxes).
struct Geo {
    int dim, k;
    int n[3];          // cells per axis (1 beyond dim)
    int periodic[3];
    double h[3];       // cell sizes (1 beyond dim)
    double L[3];
    double vol;        // |K|
    double chi_e;      // CDG2 lifting factor
    double pen_c;      // face penalty constant c: -c (k+1)^2 A Delta / h (chi_e, eta/2 or C_IP)
    double g1in[2];    // Gamma_{1,in} x-range
    long long E;       // elements
};

// Model coefficients in kernel-argument form (copied from cdg2_params).
struct Coef {
    double A[NS];                  // diag(mu1, mu2, mu3, nu1, nu2, nu3)
    double chi0[4], chith[4];
    double d1, d2, gamma, alpha1, alpha2, f1, k_ox;
    double beta1, beta2, sigma, c1s, c1ss, bc_sign;
    double phase[NS];
    int model;                     // 0: Eq. (1); 1: reduced model of Eq. (2)
};

Coef make_coef(const cdg2_params& p);

// Gauss-Legendre rule with n points on [0,1] (ascending points, weights sum 1).
void gauss01(int n, double* x, double* w);

template <typename T>
TabP<T> make_tabp(const Tab1D& t, const Geo& g) {
    TabP<T> p{};
    for (int q = 0; q < MAXQ; ++q) {
        for (int a = 0; a <= MAXK; ++a) {
            p.B[q][a] = (T)t.B[q][a];
            p.Bw[q][a] = (T)(t.w[q] * t.B[q][a]);
            for (int j = 0; j < 3; ++j) {
                p.Dh[j][q][a] = (T)(t.D[q][a] / g.h[j]);
                p.Dwh[j][q][a] = (T)(t.w[q] * t.D[q][a] / g.h[j]);
            }
        }
        p.w[q] = (T)t.w[q];
        p.xi[q] = (T)t.xi[q];
    }
    for (int f = 0; f < 2; ++f)
        for (int a = 0; a <= MAXK; ++a) {
            p.e[f][a] = (T)t.e[f][a];
            for (int j = 0; j < 3; ++j) p.dh[j][f][a] = (T)(t.d[f][a] / g.h[j]);
        }
    for (int a = 0; a <= MAXK; ++a)
        for (int b = 0; b <= MAXK; ++b) {
            double k1 = 0.0;
            for (int q = 0; q < MAXQ; ++q) k1 += t.w[q] * t.D[q][a] * t.D[q][b];
            for (int j = 0; j < 3; ++j) p.K1h[j][a][b] = (T)(k1 / (g.h[j] * g.h[j]));
        }
    return p;
}

}  // namespace cdg2

struct cdg2_mesh {
    cdg2::Geo geo;
    cdg2::Tab1D tab;
    cdg2::TabP<double> tp64;   // tables of the FP64 and FP32 operator kernels
    cdg2::TabP<float> tp32;
    int nb;            // basis per species per element
    long long ndof;
    // Face buffer of the face-once apply/JVP path (allocated by the first
    // apply or JVP on the mesh, freed by cdg2_mesh_destroy).
    mutable void* fbuf = nullptr;
    mutable size_t fbuf_bytes = 0;
    // Device workspace owned by the mesh, allocated on first use and freed by
    // cdg2_mesh_destroy: per-CTA partial sums of the VJP's theta gradient.
    mutable double* theta_part = nullptr;
    mutable long long theta_part_n = 0;
    // Workspace of cdg2_step: 8 FP64 state vectors, the Krylov basis, reduction scratch.
    mutable void* step_ws = nullptr;
    mutable size_t step_ws_bytes = 0;
    // Domain status word (device int): set by a kernel that meets c + chi^th <= 0.
    mutable int* status = nullptr;
    // Table images of the tensor-core element kernel (3D Q3, CDG2_TF32), built by its first launch.
    mutable void* tc_tables = nullptr;
    // Assembled Jacobian of cdg2_step with jacobian = 1, created by its first use.
    mutable cdg2_matrix* jac = nullptr;
};

namespace cdg2 {

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// One-time set-up that has to be repeated on every device a process uses
// (a kernel's opt-in dynamic shared-memory size is a property of the kernel
// on one device): `setup` runs with the device current, once per device
// ordinal below 64 (every call beyond that).  Two threads may both run it
// the first time; the set-ups used here are idempotent.
struct DeviceOnce {
    std::atomic<unsigned long long> done{0};   // bit d: device d is set up
};

template <typename F>
inline cudaError_t once_per_device(DeviceOnce& o, F&& setup) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return setup();
    const unsigned long long bit = 1ull << dev;
    if (o.done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = setup();
    if (e == cudaSuccess) o.done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// The domain status word of a mesh (one device int, zero until a kernel
// meets a pole of chi): allocated and cleared by the first call.
cudaError_t ensure_status(int** word);
// Wait for `st`, read *word and clear it if set: CDG2_OK, CDG2_ERR_DOMAIN
// (with the message) or CDG2_ERR_CUDA.  word may be null (nothing launched).
int take_domain_status(int* word, cudaStream_t st, const char* who);

// Kernel launchers (operator.cu).  Return the cudaError_t of the launch.
// Every launcher records domain errors in `domain` when it is given, else in
// the mesh's status word (allocating it on the first launch).
cudaError_t launch_apply(const cdg2_mesh& m, const Coef& c, const void* U, void* out, int flags, double t,
                         cudaStream_t stream);
cudaError_t launch_jvp(const cdg2_mesh& m, const Coef& c, const void* U, const void* dU, const double* dtheta,
                       void* out, int flags, cudaStream_t stream);
// out = alpha w + beta J(U) w with w = pscale . dU (pscale: [6][n_basis] per-mode
// scale on the device, or null): the right-preconditioned Krylov operator
// (I - gamma dt J) P^{-1} v in one pass.
cudaError_t launch_jvp_axpby(const cdg2_mesh& m, const Coef& c, const void* U, const void* dU, double alpha,
                             double beta, const double* pscale, void* out, int flags, cudaStream_t stream);
// out = alpha w + beta J(U)^T w with w = pscale . lam (the transposed Krylov operator)
cudaError_t launch_vjp_axpby(const cdg2_mesh& m, const Coef& c, const void* U, const void* lam, double alpha,
                             double beta, const double* pscale, void* out, int flags, cudaStream_t stream);
// VJP: gU = (df/dU)^T lam; when gtheta is non-null also (df/dtheta)^T lam via
// theta_part ([vjp_grid(m)][8] doubles of scratch) and a fixed-order reduction.
cudaError_t launch_vjp(const cdg2_mesh& m, const Coef& c, const void* U, const void* lam, void* gU,
                       double* theta_part, double* gtheta, int flags, cudaStream_t stream, int* domain = nullptr);
long long vjp_grid(const cdg2_mesh& m);
// The assembled Jacobian (assembled.cu): A = J(U) by JVP probing; y = alpha A x + beta y.
int assemble(cdg2_matrix& A, const Coef& c, const double* U, cudaStream_t st, const char* who);
cudaError_t spmv(const cdg2_matrix& A, double alpha, const double* x, double beta, double* y, cudaStream_t st);
size_t face_buffer_bytes(const Geo& g);

}  // namespace cdg2
