// cdg2_step: one diagonally implicit Runge-Kutta step of U' = f(U, t) =
// M^{-1} L_h(U) (+ forcing) (Sec. 3.2, Eq. ode), each stage solved by a
// Jacobian-free Newton-Krylov method with GMRES (Sec. 3.2).
//
// Reading: the paper names DIRK methods of order 2, 3 or 4 without tableaux;
// this uses Alexander's L-stable, stiffly accurate SDIRK2 and SDIRK3 and
// Hairer and Wanner's 5-stage L-stable SDIRK4.
//
// Stage i solves G(Y) = Y - dt a_ii f(Y, t + c_i dt) - rhs_i = 0 with
// rhs_i = U_n + dt sum_{j<i} a_ij K_j.  Newton: the residual G is always
// formed in FP64; the correction solves (I - dt a_ii J(Y)) d = -G by
// restarted GMRES whose Arnoldi step is classical Gram-Schmidt with the
// Daniel-Gragg-Kaufman-Stewart criterion (a second projection pass only when
// the first removed more than half of |w|^2), and whose matrix-vector product
// is one JVP launch (J from the kernel, not a finite difference).  In the mixed mode the Krylov vectors, the JVP and the
// primal state it linearises about are FP32 while G, Y and the convergence
// test stay FP64: iterative refinement, so the converged stage agrees with
// the FP64 solve to the Newton tolerance.
//
// The driver runs on the host; it synchronises the stream to read each
// reduction (Newton residual norms, Gram-Schmidt coefficients).
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cdg2_internal.h"
#include "krylov.h"
#include "precond.h"
#include "simplex_step.h"

namespace cdg2 {

constexpr int MAX_STAGES = 5;

struct Tableau {
    int s;
    double A[MAX_STAGES][MAX_STAGES];
    double b[MAX_STAGES];
    double c[MAX_STAGES];
};

// Alexander (1977): SDIRK2 with gamma = 1 - 1/sqrt(2); SDIRK3 with gamma the
// root in (1/6, 1/2) of 6 g^3 - 18 g^2 + 9 g - 1 (found by Newton's method),
// c2 = (1 + g)/2, b1 = -(6 g^2 - 16 g + 1)/4, b2 = (6 g^2 - 20 g + 5)/4.
static Tableau sdirk_tableau(int scheme) {
    Tableau T;
    std::memset(&T, 0, sizeof(T));
    if (scheme == CDG2_SDIRK2) {
        const double g = 1.0 - 1.0 / std::sqrt(2.0);
        T.s = 2;
        T.A[0][0] = g;
        T.A[1][0] = 1.0 - g;
        T.A[1][1] = g;
    } else if (scheme == CDG2_SDIRK4) {
        // Hairer & Wanner (Solving ODEs II, Sec. IV.6): 5 stages, gamma = 1/4,
        // stiffly accurate, L-stable, order 4.
        static const double a[5][5] = {{1.0 / 4, 0, 0, 0, 0},
                                       {1.0 / 2, 1.0 / 4, 0, 0, 0},
                                       {17.0 / 50, -1.0 / 25, 1.0 / 4, 0, 0},
                                       {371.0 / 1360, -137.0 / 2720, 15.0 / 544, 1.0 / 4, 0},
                                       {25.0 / 24, -49.0 / 48, 125.0 / 16, -85.0 / 12, 1.0 / 4}};
        T.s = 5;
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) T.A[i][j] = a[i][j];
    } else {
        double g = 0.43;
        for (int it = 0; it < 60; ++it) {
            const double p = ((6.0 * g - 18.0) * g + 9.0) * g - 1.0;
            const double dp = (18.0 * g - 36.0) * g + 9.0;
            g -= p / dp;
        }
        const double c2 = 0.5 * (1.0 + g);
        T.s = 3;
        T.A[0][0] = g;
        T.A[1][0] = c2 - g;
        T.A[1][1] = g;
        T.A[2][0] = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0;
        T.A[2][1] = (6.0 * g * g - 20.0 * g + 5.0) / 4.0;
        T.A[2][2] = g;
    }
    for (int i = 0; i < T.s; ++i) {
        T.b[i] = T.A[T.s - 1][i];
        double c = 0.0;
        for (int j = 0; j <= i; ++j) c += T.A[i][j];
        T.c[i] = c;
    }
    return T;
}

// Views into the step workspace.
struct Work {
    long long n;
    int m;
    double* rhs;
    double* Y;
    double* fY;
    double* G;
    double* b64;
    double* K[MAX_STAGES];
    void* basis;      // (m + 2) vectors of the Krylov precision: V_0..V_m, w
    void* dx;         // the Krylov correction
    void* Yk;         // primal state in the Krylov precision (mixed) / unused
    void* bk;         // right-hand side in the Krylov precision (mixed)
    double* red;      // reduction partials
    double* red_out;  // reduction results: Gram-Schmidt dots (2 MAX_KRYLOV + 3), then one norm slot
    double* hdev;     // Gram-Schmidt coefficients of the current Arnoldi step (MAX_KRYLOV + 1)
    double* gram;     // Gram matrix of the Krylov basis, (MAX_KRYLOV + 1)^2
    double* gth;      // 8 doubles: the theta gradient of one adjoint stage
    double* pinv;     // [6][n_basis] right preconditioner P^{-1}
    void* blk;        // element-block table (precond.cu)
    void* ptmp;       // P^{-1} v in the Krylov precision
};

// Right preconditioner of GMRES: the modal diagonal (applied inside the
// JVP/VJP kernel) or the element-block-Jacobi table (its own kernel).
struct Precond {
    const double* pinv = nullptr;
    const BlockTable* bt = nullptr;
};

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Carve the step workspace (grown on demand in *ws, owned by the mesh) for n
// unknowns, nb basis functions per species and blk_bytes of block table.
static int ensure_work(long long n, int nb, size_t blk_bytes, void*& ws, size_t& ws_bytes, int kdim, bool mixed,
                       Work& w) {
    const size_t ks = mixed ? sizeof(float) : sizeof(double);
    const size_t vec64 = align256(sizeof(double) * n);
    const size_t veck = align256(ks * n);
    const size_t red = align256(sizeof(double) * reduction_scratch_doubles(2 * MAX_KRYLOV + 3));
    const size_t out = align256(sizeof(double) * (2 * MAX_KRYLOV + 4));   // dots, then one norm slot
    const size_t hgs = align256(sizeof(double) * (MAX_KRYLOV + 1));
    const size_t gram = align256(sizeof(double) * (MAX_KRYLOV + 1) * (MAX_KRYLOV + 1));
    const size_t gth = align256(sizeof(double) * 8);
    const size_t tab = align256(sizeof(double) * NS * nb);
    const size_t blk = align256(blk_bytes);
    // 5 + MAX_STAGES FP64 vectors; basis (kdim + 2) + dx + Yk + bk + ptmp in the Krylov precision
    const size_t need = (5 + MAX_STAGES) * vec64 + (size_t)(kdim + 6) * veck + red + out + hgs + gram + gth + tab + blk;
    if (ws_bytes < need) {
        if (ws) cudaFree(ws);
        ws = nullptr;
        ws_bytes = 0;
        cudaError_t e = cudaMalloc(&ws, need);
        if (e != cudaSuccess) return cuda_fail(e, "cdg2_step: workspace");
        ws_bytes = need;
    }
    char* p = static_cast<char*>(ws);
    w.n = n;
    w.m = kdim;
    double** v64[5 + MAX_STAGES] = {&w.rhs, &w.Y, &w.fY, &w.G, &w.b64, &w.K[0], &w.K[1], &w.K[2], &w.K[3], &w.K[4]};
    for (auto* q : v64) {
        *q = reinterpret_cast<double*>(p);
        p += vec64;
    }
    w.basis = p;
    p += (size_t)(kdim + 2) * veck;
    w.dx = p;
    p += veck;
    w.Yk = p;
    p += veck;
    w.bk = p;
    p += veck;
    w.red = reinterpret_cast<double*>(p);
    p += red;
    w.red_out = reinterpret_cast<double*>(p);
    p += out;
    w.hdev = reinterpret_cast<double*>(p);
    p += hgs;
    w.gram = reinterpret_cast<double*>(p);
    p += gram;
    w.gth = reinterpret_cast<double*>(p);
    p += gth;
    w.pinv = reinterpret_cast<double*>(p);
    p += tab;
    w.blk = p;
    p += blk;
    w.ptmp = p;
    return CDG2_OK;
}

static int ensure_work(const cdg2_mesh& m, int kdim, bool mixed, Work& w) {
    return ensure_work(m.ndof, m.nb, block_table_bytes(m), m.step_ws, m.step_ws_bytes, kdim, mixed, w);
}

// P^{-1} for every (species, mode): P = 1 - gdt A_s d_i with d_i the modal
// diagonal of the diffusion part of M^{-1} L_h on an interior Cartesian cell:
// sum_j h_j^{-2} (-int psi'^2 + [psi' psi]_0^1 - chi_e (k+1)^2 (psi(0)^2 + psi(1)^2))
// (the first two cancel for Legendre modes; they are kept as computed).
static void modal_pinv(const cdg2_mesh& m, const Coef& c, double gdt, std::vector<double>& out) {
    const Geo& g = m.geo;
    const Tab1D& t = m.tab;
    const int k = g.k, nb1 = k + 1;
    double d1[MAXK + 1];
    for (int a = 0; a <= k; ++a) {
        double vol = 0.0;
        for (int q = 0; q < k + 2; ++q) vol += t.w[q] * t.D[q][a] * t.D[q][a];
        const double face = t.d[1][a] * t.e[1][a] - t.d[0][a] * t.e[0][a];
        const double pen = g.pen_c * (k + 1) * (k + 1) * (t.e[0][a] * t.e[0][a] + t.e[1][a] * t.e[1][a]);
        d1[a] = -vol + face - pen;
    }
    out.assign((size_t)NS * m.nb, 1.0);
    for (int s = 0; s < NS; ++s)
        for (int i = 0; i < m.nb; ++i) {
            int r = i;
            double d = 0.0;
            for (int j = 0; j < g.dim; ++j) {
                const int a = r % nb1;
                r /= nb1;
                d += d1[a] / (g.h[j] * g.h[j]);
            }
            out[(size_t)s * m.nb + i] = 1.0 / (1.0 - gdt * c.A[s] * d);
        }
}

// The preconditioner of one step (SDIRK: one diagonal coefficient a_ii for
// all stages, so one set of blocks per call).
static int setup_precond(const cdg2_mesh& m, const Coef& c, double gdt, int kind, Work& w, Precond& pc,
                         BlockTable& bt) {
    if (kind == 1) {
        std::vector<double> ptab;
        modal_pinv(m, c, gdt, ptab);
        cudaError_t e = cudaMemcpy(w.pinv, ptab.data(), sizeof(double) * ptab.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cdg2_step: preconditioner");
        pc.pinv = w.pinv;
    } else if (kind == 2) {
        if (int rc = build_block_table(m, c, gdt, w.blk, bt)) return rc;
        pc.bt = &bt;
    }
    return CDG2_OK;
}

#define CDG2_TRY(...)                                              \
    do {                                                           \
        cudaError_t e_ = (__VA_ARGS__);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, "cdg2_step"); \
    } while (0)

// ||x||_2 of a vector, read back to the host.
template <typename T>
static int norm2(const Work& w, const T* x, cudaStream_t st, double* out) {
    CDG2_TRY(vec_mdot<T>(w.n, 1, x, w.n, x, w.red, w.red_out, st));
    double v = 0.0;
    CDG2_TRY(cudaMemcpyAsync(&v, w.red_out, sizeof(double), cudaMemcpyDeviceToHost, st));
    CDG2_TRY(cudaStreamSynchronize(st));
    *out = std::sqrt(v);
    return CDG2_OK;
}

// A cycle ends early (done) on convergence, breakdown or the iteration cap;
// otherwise it used all kdim vectors and GMRES restarts from the true residual.
static bool done_cycle_needs_restart(bool done, int jlast, int kdim) { return !done && jlast == kdim - 1; }

// Restarted GMRES(m) for (I - gdt J(Yop)) x = b, x0 = 0, Arnoldi by classical
// Gram-Schmidt applied twice (CGS2; *reorth counts the rare extra passes).
// Stops when ||b - A x||_2 <= rtol ||b||_2 (the Arnoldi estimate) or after
// maxit inner iterations.  T is the Krylov precision.
// The operator's matvec: w = (I - gdt J) P^{-1} v, or with J^T (adjoint).
template <typename T>
static cudaError_t matvec(bool adjoint, const cdg2_mesh& m, const Coef& c, const T* Yop, const T* v, double gdt,
                          const Precond& pc, T* tmp, T* out, int flags, cudaStream_t st) {
    if (pc.bt) {   // v <- P^{-1} v by blocks, then the plain operator
        cudaError_t e = block_apply<T>(m, *pc.bt, v, tmp, st);
        if (e != cudaSuccess) return e;
        v = tmp;
    }
    if (adjoint) return launch_vjp_axpby(m, c, Yop, v, 1.0, -gdt, pc.pinv, out, flags, st);
    return launch_jvp_axpby(m, c, Yop, v, 1.0, -gdt, pc.pinv, out, flags, st);
}

// The Cartesian operator of GMRES: matvec above, and the map of the final
// iterate back from the right-preconditioned space.
template <typename T>
struct CartKrylovOp {
    const cdg2_mesh& m;
    const Coef& c;
    const T* Yop;
    double gdt;
    const Precond& pc;
    int flags;
    bool adjoint;
    int mv(const T* v, T* tmp, T* out, cudaStream_t st) const {
        const int jflags = CDG2_MINV | ((sizeof(T) == 4) ? CDG2_FP32 | (flags & CDG2_TF32) : 0) | (flags & CDG2_FORCING);
        CDG2_TRY(matvec<T>(adjoint, m, c, Yop, v, gdt, pc, tmp, out, jflags, st));
        return CDG2_OK;
    }
    int finish(long long n, T* x, T* tmp, cudaStream_t st) const {
        // right preconditioning: the Krylov iterate lives in P-space, x = P^{-1} y
        if (pc.pinv) CDG2_TRY(vec_scale_modes<T>(n, pc.pinv, NS * m.nb, x, st));
        if (pc.bt) {
            CDG2_TRY(block_apply<T>(m, *pc.bt, x, tmp, st));
            CDG2_TRY(cudaMemcpyAsync(x, tmp, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
        }
        return CDG2_OK;
    }
};

// The GMRES operator with the assembled Jacobian: w = (I - gdt A) P^{-1} v
// (FP64), P the modal diagonal or the element blocks as for the JVP.
struct AssembledKrylovOp {
    const cdg2_mesh& m;
    const cdg2_matrix& A;
    double gdt;
    const Precond& pc;
    int mv(const double* v, double* tmp, double* out, cudaStream_t st) const {
        const long long n = m.ndof;
        if (pc.bt) {
            CDG2_TRY(block_apply<double>(m, *pc.bt, v, tmp, st));
            v = tmp;
        } else if (pc.pinv) {
            CDG2_TRY(cudaMemcpyAsync(tmp, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            CDG2_TRY(vec_scale_modes<double>(n, pc.pinv, NS * m.nb, tmp, st));
            v = tmp;
        }
        CDG2_TRY(spmv(A, -gdt, v, 0.0, out, st));
        CDG2_TRY(vec_axpby<double>(n, 1.0, v, 1.0, out, st));
        return CDG2_OK;
    }
    int finish(long long n, double* x, double* tmp, cudaStream_t st) const {
        if (pc.pinv) CDG2_TRY(vec_scale_modes<double>(n, pc.pinv, NS * m.nb, x, st));
        if (pc.bt) {
            CDG2_TRY(block_apply<double>(m, *pc.bt, x, tmp, st));
            CDG2_TRY(cudaMemcpyAsync(x, tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        }
        return CDG2_OK;
    }
};

template <typename T, typename Op>
static int gmres_op(const Op& op, const T* b, T* x, double rtol, int maxit, const Work& w, cudaStream_t st,
                    int* iters, int* reorth, double* relres) {
    const long long n = w.n;
    const int kdim = w.m;
    T* V = static_cast<T*>(w.basis);
    T* wv = V + (size_t)(kdim + 1) * n;
    T* tmp = static_cast<T*>(w.ptmp);
    const bool packed = vec_packed<T>(n, V, n, wv);
    CDG2_TRY(cudaMemsetAsync(x, 0, sizeof(T) * n, st));
    double beta0 = 0.0;
    if (int rc = norm2<T>(w, b, st, &beta0)) return rc;
    *iters = 0;
    *relres = 0.0;
    if (beta0 == 0.0) return CDG2_OK;
    if (!std::isfinite(beta0)) {
        set_error("cdg2_step: non-finite Newton residual");
        return CDG2_ERR_NONFINITE;
    }
    std::vector<double> H((size_t)(kdim + 1) * kdim), cs(kdim), sn(kdim), g(kdim + 1), y(kdim), hcol(kdim + 1);
    double beta = beta0;
    CDG2_TRY(vec_convert<T, T>(n, b, 1.0 / beta, V, st));   // V_0 = b / ||b||
    int total = 0;
    double resid = beta;
    while (true) {
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jlast = -1;
        bool done = false;
        for (int j = 0; j < kdim; ++j) {
            T* vj = V + (size_t)j * n;
            if (int rc = op.mv(vj, tmp, wv, st)) return rc;   // w = (I - gdt J) P^-1 v_j
            std::fill(hcol.begin(), hcol.end(), 0.0);
            double* nslot = w.red_out + (2 * MAX_KRYLOV + 3);
            double hn = 0.0;
            if (packed) {
                // Classical Gram-Schmidt applied twice (CGS2) in two passes over the
                // basis: one pass forms V^T w and V^T v_j (the new Gram column), a
                // small kernel the coefficients h = (2I - G) V^T w, one pass
                // w -= V h with |w|^2.  A third pass, a plain classical one, only
                // when |w| fell below 1e-2 of its size (severe cancellation, where
                // the rounding of the update itself needs removing).
                CDG2_TRY(vec_gs_dots<T>(n, j + 1, V, n, wv, w.red, w.red_out, w.gram, MAX_KRYLOV + 1, w.hdev, st));
                CDG2_TRY(vec_update_norm16<T>(n, j + 1, V, n, w.hdev, wv, w.red, nslot, st));
                std::vector<double> hp(2 * MAX_KRYLOV + 4), hh(j + 1);
                CDG2_TRY(cudaMemcpyAsync(hp.data(), w.red_out, sizeof(double) * (2 * MAX_KRYLOV + 4),
                                         cudaMemcpyDeviceToHost, st));
                CDG2_TRY(cudaMemcpyAsync(hh.data(), w.hdev, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st));
                CDG2_TRY(cudaStreamSynchronize(st));
                for (int i = 0; i <= j; ++i) hcol[i] = hh[i];
                const double w0 = std::sqrt(std::max(hp[2 * (j + 1)], 0.0));
                hn = std::sqrt(std::max(hp[2 * MAX_KRYLOV + 3], 0.0));
                if (hn < 1e-2 * w0) {
                    CDG2_TRY(vec_mdot<T>(n, j + 1, V, n, wv, w.red, w.red_out, st));
                    CDG2_TRY(vec_update_norm16<T>(n, j + 1, V, n, w.red_out, wv, w.red, nslot, st));
                    CDG2_TRY(cudaMemcpyAsync(hp.data(), w.red_out, sizeof(double) * (2 * MAX_KRYLOV + 4),
                                             cudaMemcpyDeviceToHost, st));
                    CDG2_TRY(cudaStreamSynchronize(st));
                    for (int i = 0; i <= j; ++i) hcol[i] += hp[i];
                    hn = std::sqrt(std::max(hp[2 * MAX_KRYLOV + 3], 0.0));
                    ++*reorth;
                }
            } else {
                // Unaligned layouts: classical Gram-Schmidt with the DGKS criterion:
                // one projection pass (its multi-dot also gives |w| before, the
                // update |w| after); a second pass only when |w'| < |w| / sqrt(2).
                for (int pass = 0; pass < 2; ++pass) {
                    if (pass == 0) CDG2_TRY(vec_mdot_self<T>(n, j + 1, V, n, wv, w.red, w.red_out, st));
                    else CDG2_TRY(vec_mdot<T>(n, j + 1, V, n, wv, w.red, w.red_out, st));
                    CDG2_TRY(vec_update_norm<T>(n, j + 1, V, n, w.red_out, wv, w.red, nslot, st));
                    std::vector<double> hp(2 * MAX_KRYLOV + 4);
                    CDG2_TRY(cudaMemcpyAsync(hp.data(), w.red_out, sizeof(double) * (2 * MAX_KRYLOV + 4),
                                             cudaMemcpyDeviceToHost, st));
                    CDG2_TRY(cudaStreamSynchronize(st));
                    for (int i = 0; i <= j; ++i) hcol[i] += hp[i];
                    hn = std::sqrt(std::max(hp[2 * MAX_KRYLOV + 3], 0.0));
                    if (pass == 1) ++*reorth;
                    if (pass == 1 || !(hn < 0.7071067811865476 * std::sqrt(std::max(hp[j + 1], 0.0)))) break;
                }
            }
            hcol[j + 1] = hn;
            // previous Givens rotations, then a new one zeroing hcol[j + 1]
            for (int i = 0; i < j; ++i) {
                const double a = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
                hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
                hcol[i] = a;
            }
            const double r = std::hypot(hcol[j], hcol[j + 1]);
            cs[j] = r > 0.0 ? hcol[j] / r : 1.0;
            sn[j] = r > 0.0 ? hcol[j + 1] / r : 0.0;
            hcol[j] = r;
            hcol[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; ++i) H[(size_t)i * kdim + j] = hcol[i];
            ++total;
            resid = std::fabs(g[j + 1]);
            jlast = j;
            if (!std::isfinite(resid)) {
                set_error("cdg2_step: non-finite GMRES residual");
                return CDG2_ERR_NONFINITE;
            }
            if (hn == 0.0 || resid <= rtol * beta0 || total >= maxit) {
                done = true;
                break;
            }
            CDG2_TRY(vec_convert<T, T>(n, wv, 1.0 / hn, V + (size_t)(j + 1) * n, st));
        }
        // y = R^{-1} g (upper triangular), x += V y
        for (int i = jlast; i >= 0; --i) {
            double acc = g[i];
            for (int k = i + 1; k <= jlast; ++k) acc -= H[(size_t)i * kdim + k] * y[k];
            y[i] = acc / H[(size_t)i * kdim + i];
        }
        Coeffs yc;
        for (int i = 0; i <= jlast; ++i) yc.v[i] = y[i];
        CDG2_TRY(vec_basis_combine<T>(n, jlast + 1, V, n, yc, x, st));
        if (resid <= rtol * beta0 || total >= maxit || !done_cycle_needs_restart(done, jlast, kdim)) break;
        // restart: r = b - A x into V_0
        if (int rc = op.mv(x, tmp, wv, st)) return rc;
        CDG2_TRY(vec_convert<T, T>(n, b, 1.0, V, st));
        CDG2_TRY(vec_axpby<T>(n, -1.0, wv, 1.0, V, st));
        if (int rc = norm2<T>(w, V, st, &beta)) return rc;
        if (beta <= rtol * beta0) {
            resid = beta;
            break;
        }
        CDG2_TRY(vec_convert<T, T>(n, V, 1.0 / beta, V, st));
    }
    if (int rc = op.finish(n, x, tmp, st)) return rc;
    *iters = total;
    *relres = resid / beta0;
    return CDG2_OK;
}

template <typename T>
static int gmres(const cdg2_mesh& m, const Coef& c, const T* Yop, double gdt, const T* b, T* x, double rtol,
                 int maxit, const Work& w, cudaStream_t st, int flags, const Precond& pc, int* iters,
                 int* reorth, double* relres, bool adjoint = false) {
    const CartKrylovOp<T> op{m, c, Yop, gdt, pc, flags, adjoint};
    return gmres_op<T>(op, b, x, rtol, maxit, w, st, iters, reorth, relres);
}

}  // namespace cdg2

using namespace cdg2;

static int check_opts(const cdg2_solver_opts* o, double dt, const char* who) {
    if ((o->scheme != CDG2_SDIRK2 && o->scheme != CDG2_SDIRK3 && o->scheme != CDG2_SDIRK4) || o->gmres_restart < 1 ||
        o->gmres_restart > MAX_KRYLOV || o->max_newton < 1 || o->max_gmres < 1 || !(dt > 0.0) ||
        (o->flags & ~CDG2_FORCING) || (o->precond < 0 || o->precond > 2) || o->mixed < 0 || o->mixed > 2) {
        set_error(std::string(who) + ": invalid options (scheme 2|3|4, 1 <= gmres_restart <= 64, max_newton, "
                  "max_gmres >= 1, dt > 0, flags in {0, CDG2_FORCING}, precond in {0, 1, 2}, mixed in {0, 1, 2})");
        return CDG2_ERR_INVALID_ARG;
    }
    return CDG2_OK;
}

// The stages of one SDIRK step on any mesh: apply(Y, fY, t_i) evaluates f,
// correct(gdt, &its, &relres) solves the Newton correction for the residual
// in w.G about w.Y and adds it into w.Y (both return a CDG2 status).  U is
// overwritten with U_{n+1}; stages_out (nullable) receives Y_1..Y_s.
// dom: the mesh's domain status word.  It is cleared before every residual
// evaluation and read when Newton has converged: the converged stage value
// must lie in the model's domain, while Newton may pass through iterates
// outside it (the JVPs at such an iterate set the word too; the next
// evaluation clears it).
template <typename Apply, typename Correct>
static int sdirk_run(const Tableau& T, const Work& w, const Apply& apply, const Correct& correct, double* U, double t,
                     double dt, const cdg2_solver_opts* o, cdg2_stats& S, double* stages_out, cudaStream_t st,
                     const char* who, int* dom) {
    const long long n = w.n;
    int status = CDG2_OK;
    CDG2_TRY(cudaMemcpyAsync(w.Y, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    for (int i = 0; i < T.s && status == CDG2_OK; ++i) {
        const double ti = t + T.c[i] * dt;
        const double gdt = dt * T.A[i][i];
        Coeffs a;
        for (int j = 0; j < i; ++j) a.v[j] = dt * T.A[i][j];
        // rhs_i = U_n + dt sum_{j<i} a_ij K_j  (K_j are stored back to back)
        CDG2_TRY(vec_lincomb(n, U, i, w.K[0], w.K[1] - w.K[0], a, w.rhs, st));
        double g0 = 0.0;
        bool converged = false;
        for (int it = 0; it <= o->max_newton; ++it) {
            if (dom) CDG2_TRY(cudaMemsetAsync(dom, 0, sizeof(int), st));
            if (int rc = apply(w.Y, w.fY, ti)) return rc;
            CDG2_TRY(vec_newton_residual(n, w.Y, w.fY, gdt, w.rhs, w.G, st));
            double gn = 0.0;
            if (int rc = norm2<double>(w, w.G, st, &gn)) return rc;
            if (!std::isfinite(gn)) {
                set_error(std::string(who) + ": non-finite Newton residual");
                status = CDG2_ERR_NONFINITE;
                break;
            }
            if (it == 0) g0 = gn;
            S.residual0[i] = g0;
            S.residual[i] = gn;
            if (gn <= std::fmax(o->newton_rtol * g0, o->newton_atol)) {
                if (int rc = take_domain_status(dom, st, who)) {
                    status = rc;
                    break;
                }
                converged = true;
                break;
            }
            if (it == o->max_newton) break;
            ++S.newton_iters;
            int its = 0;
            double rr = 0.0;
            const int rc = correct(gdt, &its, &rr);
            S.gmres_iters += its;
            if (rc != CDG2_OK) {
                status = rc;
                break;
            }
        }
        if (status != CDG2_OK) break;
        if (!converged) {
            set_error(std::string(who) + ": Newton did not reach the tolerance within max_newton iterations");
            status = CDG2_ERR_NOT_CONVERGED;
            break;
        }
        // K_i = f(Y_i): the last residual evaluation was at the converged Y_i
        CDG2_TRY(cudaMemcpyAsync(w.K[i], w.fY, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        if (stages_out)
            CDG2_TRY(cudaMemcpyAsync(stages_out + (size_t)i * n, w.Y, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    }
    if (status == CDG2_OK) {
        Coeffs bb;
        for (int i = 0; i < T.s; ++i) bb.v[i] = dt * T.b[i];
        CDG2_TRY(vec_lincomb(n, U, T.s, w.K[0], w.K[1] - w.K[0], bb, U, st));   // U_{n+1} = U_n + dt sum b_i K_i
    }
    if (dom) CDG2_TRY(cudaMemsetAsync(dom, 0, sizeof(int), st));   // leave nothing for the next call
    CDG2_TRY(cudaStreamSynchronize(st));
    return status;
}

static int run_step(const cdg2_mesh* m, const cdg2_params* p, double* U, double t, double dt,
                    const cdg2_solver_opts* o, cdg2_stats* stats, double* stages_out, void* stream) {
    const auto t_start = std::chrono::steady_clock::now();
    if (!m || !p || !U || !o) {
        set_error("cdg2_step: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (int rc = check_opts(o, dt, "cdg2_step")) return rc;
    if (o->mixed == 2 && (m->geo.dim != 3 || m->geo.k != 3)) {
        set_error("cdg2_step: mixed = 2 (tensor-core TF32 Krylov operator) needs a 3D mesh of degree 3");
        return CDG2_ERR_INVALID_ARG;
    }
    if (o->jacobian != 0 && (o->jacobian != 1 || o->mixed != 0)) {
        set_error("cdg2_step: jacobian must be 0 (matrix-free) or 1 (assembled, with mixed = 0)");
        return CDG2_ERR_INVALID_ARG;
    }
    if (o->jacobian == 1 && !m->jac) {
        if (int rc = cdg2_matrix_create(m, &m->jac)) return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool mixed = o->mixed != 0;
    const int kflags = o->flags | (o->mixed == 2 ? CDG2_TF32 : 0);   // flags of the Krylov operator
    Work w;
    if (int rc = ensure_work(*m, o->gmres_restart, mixed, w)) return rc;
    CDG2_TRY(ensure_status(&m->status));
    const Coef c = make_coef(*p);
    const Tableau T = sdirk_tableau(o->scheme);
    const long long n = w.n;
    Precond pc;
    BlockTable bt;
    if (int rc = setup_precond(*m, c, dt * T.A[0][0], o->precond, w, pc, bt)) return rc;
    cdg2_stats S;
    std::memset(&S, 0, sizeof(S));
    S.stages = T.s;
    auto apply = [&](const double* Y, double* fY, double ti) -> int {
        CDG2_TRY(launch_apply(*m, c, Y, fY, CDG2_MINV | (o->flags & CDG2_FORCING), ti, st));
        return CDG2_OK;
    };
    auto correct = [&](double gdt, int* its, double* rr) -> int {
        int rc;
        if (o->jacobian == 1) {
            // assemble J at the current iterate, then GMRES on the assembled operator
            if (int arc = assemble(*m->jac, c, w.Y, st, "cdg2_step")) return arc;
            CDG2_TRY(vec_convert<double, double>(n, w.G, -1.0, w.b64, st));
            const AssembledKrylovOp op{*m, *m->jac, gdt, pc};
            rc = gmres_op<double>(op, w.b64, static_cast<double*>(w.dx), o->gmres_rtol, o->max_gmres, w, st, its,
                                  &S.gmres_reorth, rr);
            if (rc == CDG2_OK) CDG2_TRY(vec_add_into<double>(n, static_cast<double*>(w.dx), w.Y, st));
        } else if (!mixed) {
            CDG2_TRY(vec_convert<double, double>(n, w.G, -1.0, w.b64, st));
            rc = gmres<double>(*m, c, w.Y, gdt, w.b64, static_cast<double*>(w.dx), o->gmres_rtol, o->max_gmres, w,
                               st, o->flags, pc, its, &S.gmres_reorth, rr);
            if (rc == CDG2_OK) CDG2_TRY(vec_add_into<double>(n, static_cast<double*>(w.dx), w.Y, st));
        } else {
            CDG2_TRY(vec_convert<double, float>(n, w.Y, 1.0, static_cast<float*>(w.Yk), st));
            CDG2_TRY(vec_convert<double, float>(n, w.G, -1.0, static_cast<float*>(w.bk), st));
            rc = gmres<float>(*m, c, static_cast<float*>(w.Yk), gdt, static_cast<float*>(w.bk),
                              static_cast<float*>(w.dx), o->gmres_rtol, o->max_gmres, w, st, kflags, pc, its,
                              &S.gmres_reorth, rr);
            if (rc == CDG2_OK) CDG2_TRY(vec_add_into<float>(n, static_cast<float*>(w.dx), w.Y, st));
        }
        return rc;
    };
    const int status = sdirk_run(T, w, apply, correct, U, t, dt, o, S, stages_out, st, "cdg2_step", m->status);
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = S;
    return status;
}

namespace cdg2 {

// The GMRES operator of a simplicial mesh: w = (I - gdt J(Y)) P^{-1} v (one
// block apply when preconditioned, one JVP launch and one axpby).
struct SimplexKrylovOp {
    const SimplexStepOps& ops;
    const double* Yop;
    double gdt;
    long long n;
    const SimplexPrecond* pc;   // nullptr: no preconditioner
    int mv(const double* v, double* tmp, double* out, cudaStream_t st) const {
        if (pc) {
            CDG2_TRY(simplex_block_apply(*pc, v, tmp, st));
            v = tmp;
        }
        if (int rc = ops.jvp(ops.ctx, Yop, v, out, st)) return rc;
        CDG2_TRY(vec_axpby<double>(n, 1.0, v, -gdt, out, st));
        return CDG2_OK;
    }
    int finish(long long, double* x, double* tmp, cudaStream_t st) const {
        if (pc) {
            CDG2_TRY(simplex_block_apply(*pc, x, tmp, st));
            CDG2_TRY(cudaMemcpyAsync(x, tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        }
        return CDG2_OK;
    }
};

int simplex_step(const SimplexStepOps& ops, double* U, double dt, const cdg2_solver_opts* o, cdg2_stats* stats,
                 void* stream, const char* who) {
    const auto t_start = std::chrono::steady_clock::now();
    if (!U || !o) {
        set_error(std::string(who) + ": NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (int rc = check_opts(o, dt, who)) return rc;
    if (o->mixed || (o->precond != 0 && o->precond != 2) || o->flags != 0) {
        set_error(std::string(who) + ": simplicial meshes step in FP64 without forcing, with no preconditioner "
                  "or element-block Jacobi (mixed = 0, precond 0 or 2, flags = 0)");
        return CDG2_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Work w;
    if (int rc = ensure_work(ops.n, ops.nb, 0, *ops.ws, *ops.ws_bytes, o->gmres_restart, false, w)) return rc;
    const Tableau T = sdirk_tableau(o->scheme);
    const long long n = w.n;
    const SimplexPrecond* pc = nullptr;
    if (o->precond == 2) {
        // SDIRK: one a_ii for every stage, so one set of blocks per step
        if (int rc = simplex_precond_setup(ops, dt * T.A[0][0], w.b64, w.fY, st, who)) return rc;
        pc = ops.pc;
    }
    cdg2_stats S;
    std::memset(&S, 0, sizeof(S));
    S.stages = T.s;
    auto apply = [&](const double* Y, double* fY, double) -> int { return ops.apply(ops.ctx, Y, fY, st); };
    auto correct = [&](double gdt, int* its, double* rr) -> int {
        CDG2_TRY(vec_convert<double, double>(n, w.G, -1.0, w.b64, st));
        const SimplexKrylovOp op{ops, w.Y, gdt, n, pc};
        const int rc = gmres_op<double>(op, w.b64, static_cast<double*>(w.dx), o->gmres_rtol, o->max_gmres, w, st,
                                        its, &S.gmres_reorth, rr);
        if (rc == CDG2_OK) CDG2_TRY(vec_add_into<double>(n, static_cast<double*>(w.dx), w.Y, st));
        return rc;
    };
    const int status = sdirk_run(T, w, apply, correct, U, 0.0, dt, o, S, nullptr, st, who, ops.dom);
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = S;
    return status;
}

}  // namespace cdg2

extern "C" int cdg2_step(const cdg2_mesh* m, const cdg2_params* p, double* U, double t, double dt,
                         const cdg2_solver_opts* o, cdg2_stats* stats, void* stream) {
    return run_step(m, p, U, t, dt, o, stats, nullptr, stream);
}

extern "C" int cdg2_step_stages(const cdg2_mesh* m, const cdg2_params* p, double* U, double t, double dt,
                                const cdg2_solver_opts* o, double* stages, cdg2_stats* stats, void* stream) {
    if (!stages) {
        set_error("cdg2_step_stages: NULL stages");
        return CDG2_ERR_INVALID_ARG;
    }
    return run_step(m, p, U, t, dt, o, stats, stages, stream);
}

// Discrete adjoint of one SDIRK step (the transpose of the linearised step map):
// with K_i = f(Y_i), Y_i = U_n + dt sum_{j<=i} a_ij K_j, U_{n+1} = U_n + dt sum b_i K_i,
// backwards over the stages
//   r_i = dt b_i lam + dt sum_{j>i} a_ji ybar_j,  (I - dt a_ii J_i^T) g_i = r_i,
//   ybar_i = J_i^T g_i,  gtheta += (df/dtheta)(Y_i)^T g_i,
// and lam_n = lam + sum_i ybar_i.  Each stage system is solved by refinement:
// the residual r_i - (I - dt a_ii J_i^T) g in FP64, the correction by GMRES
// (FP64, or FP32 in the mixed mode), until ||residual|| <= newton_rtol ||r_i||.
extern "C" int cdg2_step_adjoint(const cdg2_mesh* m, const cdg2_params* p, const double* stages, double t, double dt,
                                 const cdg2_solver_opts* o, double* lam, double* gtheta, cdg2_stats* stats,
                                 void* stream) {
    (void)t;
    const auto t_start = std::chrono::steady_clock::now();
    if (!m || !p || !stages || !o || !lam) {
        set_error("cdg2_step_adjoint: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (int rc = check_opts(o, dt, "cdg2_step_adjoint")) return rc;
    if (o->flags & CDG2_FORCING) {
        set_error("cdg2_step_adjoint: the forcing's dependence on the coefficients is not differentiated");
        return CDG2_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CDG2_TRY(ensure_status(&m->status));
    CDG2_TRY(cudaMemsetAsync(m->status, 0, sizeof(int), st));   // the call owns the status word
    const bool mixed = o->mixed != 0;
    Work w;
    if (int rc = ensure_work(*m, o->gmres_restart, mixed, w)) return rc;
    const Coef c = make_coef(*p);
    const Tableau T = sdirk_tableau(o->scheme);
    const long long n = w.n;
    const long long ldk = w.K[1] - w.K[0];
    double* gth = w.gth;
    double* part = nullptr;
    if (gtheta) {
        const long long need = vjp_grid(*m) * 8;
        if (m->theta_part_n < need) {
            if (m->theta_part) cudaFree(m->theta_part);
            m->theta_part = nullptr;
            m->theta_part_n = 0;
            CDG2_TRY(cudaMalloc(&m->theta_part, sizeof(double) * need));
            m->theta_part_n = need;
        }
        part = m->theta_part;
    }
    Precond pc;
    BlockTable bt;
    if (int rc = setup_precond(*m, c, dt * T.A[0][0], o->precond, w, pc, bt)) return rc;
    cdg2_stats S;
    std::memset(&S, 0, sizeof(S));
    S.stages = T.s;
    for (int i = T.s - 1; i >= 0; --i) {
        const double* Yi = stages + (size_t)i * n;
        const double gdt = dt * T.A[i][i];
        // r_i = dt b_i lam + dt sum_{j>i} a_ji ybar_j   (ybar_j kept in K[j])
        CDG2_TRY(vec_convert<double, double>(n, lam, dt * T.b[i], w.rhs, st));
        Coeffs a;
        for (int j = i + 1; j < T.s; ++j) a.v[j - i - 1] = dt * T.A[j][i];
        if (i + 1 < T.s) CDG2_TRY(vec_lincomb(n, w.rhs, T.s - 1 - i, w.K[i + 1], ldk, a, w.rhs, st));
        double r0 = 0.0;
        if (int rc = norm2<double>(w, w.rhs, st, &r0)) return rc;
        S.residual0[i] = r0;
        CDG2_TRY(cudaMemsetAsync(w.Y, 0, sizeof(double) * n, st));            // g_i = 0
        bool converged = r0 == 0.0;
        for (int it = 0; it < o->max_newton && !converged; ++it) {
            // residual rr = r_i - (I - gdt J_i^T) g   (FP64)
            CDG2_TRY(launch_vjp_axpby(*m, c, Yi, w.Y, 1.0, -gdt, nullptr, w.G, CDG2_MINV, st));
            CDG2_TRY(vec_axpby<double>(n, 1.0, w.rhs, -1.0, w.G, st));
            double rn = 0.0;
            if (int rc = norm2<double>(w, w.G, st, &rn)) return rc;
            S.residual[i] = rn;
            if (int rc = take_domain_status(m->status, st, "cdg2_step_adjoint")) return rc;
            if (!std::isfinite(rn)) {
                set_error("cdg2_step_adjoint: non-finite residual");
                return CDG2_ERR_NONFINITE;
            }
            if (rn <= std::fmax(o->newton_rtol * r0, o->newton_atol)) {
                converged = true;
                break;
            }
            ++S.newton_iters;
            int its = 0, rc;
            double rr = 0.0;
            if (!mixed) {
                rc = gmres<double>(*m, c, Yi, gdt, w.G, static_cast<double*>(w.dx), o->gmres_rtol, o->max_gmres, w, st,
                                   0, pc, &its, &S.gmres_reorth, &rr, true);
                if (rc == CDG2_OK) CDG2_TRY(vec_add_into<double>(n, static_cast<double*>(w.dx), w.Y, st));
            } else {
                CDG2_TRY(vec_convert<double, float>(n, Yi, 1.0, static_cast<float*>(w.Yk), st));
                CDG2_TRY(vec_convert<double, float>(n, w.G, 1.0, static_cast<float*>(w.bk), st));
                rc = gmres<float>(*m, c, static_cast<float*>(w.Yk), gdt, static_cast<float*>(w.bk),
                                  static_cast<float*>(w.dx), o->gmres_rtol, o->max_gmres, w, st, 0, pc, &its, &S.gmres_reorth, &rr,
                                  true);
                if (rc == CDG2_OK) CDG2_TRY(vec_add_into<float>(n, static_cast<float*>(w.dx), w.Y, st));
            }
            S.gmres_iters += its;
            if (rc != CDG2_OK) return rc;
        }
        if (!converged) {
            // the last correction was not checked: check once more
            CDG2_TRY(launch_vjp_axpby(*m, c, Yi, w.Y, 1.0, -gdt, nullptr, w.G, CDG2_MINV, st));
            CDG2_TRY(vec_axpby<double>(n, 1.0, w.rhs, -1.0, w.G, st));
            double rn = 0.0;
            if (int rc = norm2<double>(w, w.G, st, &rn)) return rc;
            S.residual[i] = rn;
            if (!(rn <= std::fmax(o->newton_rtol * r0, o->newton_atol))) {
                set_error("cdg2_step_adjoint: a stage system did not reach the tolerance within max_newton refinements");
                if (stats) *stats = S;
                return CDG2_ERR_NOT_CONVERGED;
            }
        }
        // ybar_i = J_i^T g_i (into K[i]) and the coefficient gradient of this stage
        CDG2_TRY(launch_vjp(*m, c, Yi, w.Y, w.K[i], part, gtheta ? gth : nullptr, CDG2_MINV, st));
        if (gtheta) CDG2_TRY(vec_axpby<double>(8, 1.0, gth, 1.0, gtheta, st));
    }
    // lam_n = lam + sum_i ybar_i
    Coeffs ones;
    for (int i = 0; i < T.s; ++i) ones.v[i] = 1.0;
    CDG2_TRY(vec_lincomb(n, lam, T.s, w.K[0], ldk, ones, lam, st));
    CDG2_TRY(cudaStreamSynchronize(st));
    if (int rc = take_domain_status(m->status, st, "cdg2_step_adjoint")) return rc;
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (stats) *stats = S;
    return CDG2_OK;
}
