// Vector kernels of the Newton-GMRES solver (Sec. 3.2: the DIRK stages are
// solved by a Jacobian-free Newton-Krylov method with GMRES).  All are
// bandwidth-bound passes over DOF-length vectors with grid-stride loops;
// every reduction is two-stage with a fixed partition and a fixed tree, so
// results are bitwise reproducible (no atomics).  Dot products of FP32
// vectors accumulate in FP32 within a thread and within a warp, and in FP64
// across warps and blocks (FP64 arithmetic per element would bind these
// kernels on GB300, whose FP64 rate is 1/61 of its FP32 rate).
#include <cstdint>
#include <type_traits>

#include "krylov.h"

namespace cdg2 {

constexpr int VT = 256;                       // threads per block of the vector kernels
constexpr int RED_BLOCKS = 4 * 152;           // blocks of every partial reduction (4 per SM)

// y = a x + b y
template <typename T>
__global__ void __launch_bounds__(VT) k_axpby(long long n, double a, const T* __restrict__ x, double b,
                                               T* __restrict__ y) {
    const T aa = T(a), bb = T(b);
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
        y[i] = aa * x[i] + bb * y[i];
}

// out = x + sum_j c_j V_j (j < nv), V_j double vectors with leading dimension ldv
// (x and out may alias: each element is read before it is written by the same thread)
__global__ void __launch_bounds__(VT) k_lincomb(long long n, const double* x, int nv,
                                                 const double* __restrict__ V, long long ldv, Coeffs c,
                                                 double* out) {
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
        double acc = x[i];
        for (int j = 0; j < nv; ++j) acc = fma(c.v[j], V[j * ldv + i], acc);
        out[i] = acc;
    }
}

// G = Y - gdt * fY - rhs
__global__ void __launch_bounds__(VT) k_newton_residual(long long n, const double* __restrict__ Y,
                                                         const double* __restrict__ fY, double gdt,
                                                         const double* __restrict__ rhs, double* __restrict__ G) {
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
        G[i] = Y[i] - gdt * fY[i] - rhs[i];
}

// dst = (T) src   /   Y += (double) x
// (src and dst may alias)
template <typename S, typename D>
__global__ void __launch_bounds__(VT) k_convert(long long n, const S* src, double scale, D* dst) {
    // the narrower of the two types carries the arithmetic
    using C = typename std::conditional<(sizeof(S) < sizeof(D)), S, D>::type;
    const C sc = C(scale);
    if constexpr (std::is_same<S, float>::value && std::is_same<D, float>::value) {
        // 16 bytes per access where both vectors allow it (same element-wise result)
        if (n % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0 && reinterpret_cast<uintptr_t>(dst) % 16 == 0) {
            const long long n4 = n / 4;
            for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n4; i += (long long)gridDim.x * VT) {
                const float4 x = reinterpret_cast<const float4*>(src)[i];
                reinterpret_cast<float4*>(dst)[i] = make_float4(sc * x.x, sc * x.y, sc * x.z, sc * x.w);
            }
            return;
        }
    }
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
        dst[i] = D(sc * C(src[i]));
}

template <typename T>
__global__ void __launch_bounds__(VT) k_add_into(long long n, const T* __restrict__ x, double* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
        y[i] += double(x[i]);
}

constexpr int NWARP = VT / 32;

// Sum of v over the block in a fixed order (warp shuffles in the type of
// the thread's partial, then the warps' partials in FP64, in warp order); the
// result is valid in thread 0.  sh: NWARP doubles.  (FP32 partials stay FP32
// within the warp: FP64 adds run on GB300's narrow FP64 pipe.)
template <typename A>
__device__ __forceinline__ double block_sum(A v, double* sh) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = double(v);
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NWARP; ++i) s += sh[i];
    __syncthreads();
    return s;
}

// NR block sums at once (same order and precision rules as block_sum):
// result r lands in res[r] (shared), valid after the call for every thread.
// sh: NR * NWARP doubles, res: NR doubles.
template <int NR, typename A>
__device__ __forceinline__ void block_sums(A (&v)[NR], double* sh, double* res) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[r] += __shfl_down_sync(0xffffffffu, v[r], off);
    }
    if (lane == 0) {
#pragma unroll
        for (int r = 0; r < NR; ++r) sh[r * NWARP + warp] = double(v[r]);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < NR; r += VT) {
        double s = 0.0;
        for (int i = 0; i < NWARP; ++i) s += sh[r * NWARP + i];
        res[r] = s;
    }
    __syncthreads();
}

// 16 consecutive bytes of T (4 floats or 2 doubles), for 128-bit loads and stores.
template <typename T>
struct Pack {
    static constexpr int W = 16 / sizeof(T);
    T v[W];
};

template <typename T>
__device__ __forceinline__ Pack<T> ld16(const T* p) {
    Pack<T> r;
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        r.v[0] = q.x;
        r.v[1] = q.y;
        r.v[2] = q.z;
        r.v[3] = q.w;
    } else {
        const double2 q = *reinterpret_cast<const double2*>(p);
        r.v[0] = q.x;
        r.v[1] = q.y;
    }
    return r;
}

template <typename T>
__device__ __forceinline__ void st16(T* p, const Pack<T>& r) {
    if constexpr (sizeof(T) == 4)
        *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    else
        *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
}

// part[j][blockIdx.x] = this block's slice of V_j . w for the NVC vectors of
// chunk blockIdx.y (j = NVC * blockIdx.y + jj): w is read once per chunk and
// the NVC independent loads per element keep enough bytes in flight.
constexpr int NVC = 8;
// With self_dot, chunk 0 also forms w . w as row nv (one pass gives the
// projections and the norm before projection).
template <typename T>
__global__ void __launch_bounds__(VT) k_mdot_partial(long long n, int nv, const T* __restrict__ V, long long ldv,
                                                      const T* __restrict__ w, double* __restrict__ part,
                                                      int self_dot) {
    __shared__ double sh[NWARP];
    const int j0 = blockIdx.y * NVC;
    const int nj = nv - j0 < NVC ? nv - j0 : NVC;
    const bool with_self = self_dot && blockIdx.y == 0;
    T acc[NVC];
    T accw = T(0);
#pragma unroll
    for (int jj = 0; jj < NVC; ++jj) acc[jj] = T(0);
    const long long stride = (long long)gridDim.x * VT;
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += stride) {
        const T wi = w[i];
        T v[NVC];
#pragma unroll
        for (int jj = 0; jj < NVC; ++jj) v[jj] = jj < nj ? V[(j0 + jj) * ldv + i] : T(0);
#pragma unroll
        for (int jj = 0; jj < NVC; ++jj) acc[jj] = fma(v[jj], wi, acc[jj]);
        if (with_self) accw = fma(wi, wi, accw);
    }
    for (int jj = 0; jj < nj; ++jj) {
        const double s = block_sum(acc[jj], sh);
        if (threadIdx.x == 0) part[(long long)(j0 + jj) * gridDim.x + blockIdx.x] = s;
    }
    if (with_self) {
        const double s = block_sum(accw, sh);
        if (threadIdx.x == 0) part[(long long)nv * gridDim.x + blockIdx.x] = s;
    }
}

// The Gram-Schmidt dot pass of one Arnoldi step, over 16-byte packs (n, ldv
// multiples of the pack width, V and w 16-byte aligned): for the NVC basis
// vectors of chunk blockIdx.y, part rows j = V_j . w and nv + j = V_j . V_last
// (the newest basis vector, read from its slot in V), and with chunk 0 row
// 2 nv = w . w.  One read of the chunk, w and V_last per block row.
template <typename T>
__global__ void __launch_bounds__(VT, sizeof(T) == 4 ? RED_BLOCKS / 152 : 1) k_mdot2_partial(long long n, int nv, const T* __restrict__ V, long long ldv,
                                                       const T* __restrict__ w, double* __restrict__ part) {
    constexpr int W = Pack<T>::W;
    __shared__ double sh[(2 * NVC + 1) * NWARP];
    __shared__ double res[2 * NVC + 1];
    const int j0 = blockIdx.y * NVC;
    const int nj = nv - j0 < NVC ? nv - j0 : NVC;
    const T* vl = V + (long long)(nv - 1) * ldv;
    T aw[NVC], av[NVC], ww = T(0);
#pragma unroll
    for (int jj = 0; jj < NVC; ++jj) aw[jj] = av[jj] = T(0);
    const long long np = n / W, stride = (long long)gridDim.x * VT;
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < np; i += stride) {
        // all loads of the step issued before the first use (a short last chunk
        // re-reads its last vector; those products are never stored)
        const Pack<T> wi = ld16(w + i * W), li = ld16(vl + i * W);
        Pack<T> v[NVC];
#pragma unroll
        for (int jj = 0; jj < NVC; ++jj) v[jj] = ld16(V + (long long)(j0 + (jj < nj ? jj : nj - 1)) * ldv + i * W);
#pragma unroll
        for (int jj = 0; jj < NVC; ++jj) {
#pragma unroll
            for (int c = 0; c < W; ++c) {
                aw[jj] = fma(v[jj].v[c], wi.v[c], aw[jj]);
                av[jj] = fma(v[jj].v[c], li.v[c], av[jj]);
            }
        }
        if (blockIdx.y == 0) {
#pragma unroll
            for (int c = 0; c < W; ++c) ww = fma(wi.v[c], wi.v[c], ww);
        }
    }
    T acc[2 * NVC + 1];
#pragma unroll
    for (int jj = 0; jj < NVC; ++jj) {
        acc[jj] = aw[jj];
        acc[NVC + jj] = av[jj];
    }
    acc[2 * NVC] = ww;
    block_sums<2 * NVC + 1>(acc, sh, res);
    if ((int)threadIdx.x < nj) {
        part[(long long)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = res[threadIdx.x];
        part[(long long)(nv + j0 + threadIdx.x) * gridDim.x + blockIdx.x] = res[NVC + threadIdx.x];
    }
    if (blockIdx.y == 0 && threadIdx.x == 0) part[(long long)(2 * nv) * gridDim.x + blockIdx.x] = res[2 * NVC];
}

// The CGS2 coefficients of one Arnoldi step from the dot pass (one block):
// G[i][j] = G[j][i] = V_i . V_j (the new column of the Gram matrix of the
// basis), then h = h1 + (I - G) h1 with h1 = V^T w.  In exact arithmetic
// (I - G) h1 is the second Gram-Schmidt pass V^T (w - V h1), so
// w - V h equals w after two classical passes, formed in one update pass.
// dots: [0, nv) V^T w, [nv, 2 nv) V^T V_last, 2 nv: w . w; G: ldg x ldg.
__global__ void __launch_bounds__(64) k_gram_coeffs(int nv, const double* __restrict__ dots, double* __restrict__ G,
                                                     int ldg, double* __restrict__ h) {
    const int j = nv - 1;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        G[(long long)i * ldg + j] = dots[nv + i];
        G[(long long)j * ldg + i] = dots[nv + i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < nv; ++k) acc = fma(G[(long long)i * ldg + k], dots[k], acc);
        h[i] = 2.0 * dots[i] - acc;
    }
}

// w -= sum_j h_j V_j and part[blockIdx.x] = this block's slice of |w|^2
// after the update, over 16-byte packs (the layout conditions of
// k_mdot2_partial; fixed grid of RED_BLOCKS blocks: a deterministic partition)
template <typename T>
__global__ void __launch_bounds__(VT) k_update_norm16(long long n, int nv, const T* __restrict__ V, long long ldv,
                                                      const double* __restrict__ h, T* __restrict__ w,
                                                      double* __restrict__ part) {
    constexpr int W = Pack<T>::W;
    __shared__ T hs[MAX_KRYLOV + 1];
    __shared__ double sh[NWARP];
    for (int j = threadIdx.x; j < nv; j += VT) hs[j] = T(-h[j]);
    __syncthreads();
    T nrm = T(0);
    const long long np = n / W, stride = (long long)gridDim.x * VT;
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < np; i += stride) {
        Pack<T> acc = ld16(w + i * W);
        int j = 0;
        for (; j + NVC <= nv; j += NVC) {
            Pack<T> v[NVC];
#pragma unroll
            for (int jj = 0; jj < NVC; ++jj) v[jj] = ld16(V + (j + jj) * ldv + i * W);
#pragma unroll
            for (int jj = 0; jj < NVC; ++jj)
#pragma unroll
                for (int c = 0; c < W; ++c) acc.v[c] = fma(hs[j + jj], v[jj].v[c], acc.v[c]);
        }
        for (; j < nv; ++j) {
            const Pack<T> v = ld16(V + j * ldv + i * W);
#pragma unroll
            for (int c = 0; c < W; ++c) acc.v[c] = fma(hs[j], v.v[c], acc.v[c]);
        }
        st16(w + i * W, acc);
#pragma unroll
        for (int c = 0; c < W; ++c) nrm = fma(acc.v[c], acc.v[c], nrm);
    }
    const double s = block_sum(nrm, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[j] = sum_b part[j][b] in a fixed order (blockIdx.x = j)
__global__ void __launch_bounds__(VT) k_rows_sum(const double* __restrict__ part, int nparts,
                                                 double* __restrict__ out) {
    __shared__ double sh[NWARP];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nparts; b += VT) acc += part[(long long)blockIdx.x * nparts + b];
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// w -= sum_j h_j V_j and part[blockIdx.x] = this block's slice of |w|^2 after
// the update (fixed grid of RED_BLOCKS blocks: a deterministic partition)
template <typename T>
__global__ void __launch_bounds__(VT) k_update_norm(long long n, int nv, const T* __restrict__ V, long long ldv,
                                                    const double* __restrict__ h, T* __restrict__ w,
                                                    double* __restrict__ part) {
    __shared__ T hs[MAX_KRYLOV + 1];
    __shared__ double sh[NWARP];
    for (int j = threadIdx.x; j < nv; j += VT) hs[j] = T(-h[j]);
    __syncthreads();
    T nrm = T(0);
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
        T acc = w[i];
        int j = 0;
        for (; j + NVC <= nv; j += NVC) {
            T v[NVC];
#pragma unroll
            for (int jj = 0; jj < NVC; ++jj) v[jj] = V[(j + jj) * ldv + i];
#pragma unroll
            for (int jj = 0; jj < NVC; ++jj) acc = fma(hs[j + jj], v[jj], acc);
        }
        for (; j < nv; ++j) acc = fma(hs[j], V[j * ldv + i], acc);
        w[i] = acc;
        nrm = fma(acc, acc, nrm);
    }
    const double s = block_sum(nrm, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// x += sum_j y_j V_j  (y passed by value)
template <typename T>
__global__ void __launch_bounds__(VT) k_basis_combine(long long n, int nv, const T* __restrict__ V, long long ldv,
                                                      Coeffs y, T* __restrict__ x) {
    __shared__ T ys[MAX_KRYLOV + 1];
    for (int j = threadIdx.x; j < nv; j += VT) ys[j] = T(y.v[j]);
    __syncthreads();
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
        T acc = x[i];
        int j = 0;
        for (; j + NVC <= nv; j += NVC) {
            T v[NVC];
#pragma unroll
            for (int jj = 0; jj < NVC; ++jj) v[jj] = V[(j + jj) * ldv + i];
#pragma unroll
            for (int jj = 0; jj < NVC; ++jj) acc = fma(ys[j + jj], v[jj], acc);
        }
        for (; j < nv; ++j) acc = fma(ys[j], V[j * ldv + i], acc);
        x[i] = acc;
    }
}

// x[i] *= table[i % period]  (a per-(species, mode) diagonal on element-major vectors)
template <typename T>
__global__ void __launch_bounds__(VT) k_scale_modes(long long n, const double* __restrict__ table, int period,
                                                    T* __restrict__ x) {
    for (long long i = blockIdx.x * (long long)VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
        x[i] = T(double(x[i]) * table[i % period]);
}

static unsigned grid_for(long long n) {
    long long b = (n + VT - 1) / VT;
    const long long cap = 152LL * 16;   // enough blocks to saturate HBM; loops cover the rest
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t vec_axpby(long long n, double a, const T* x, double b, T* y, cudaStream_t st) {
    k_axpby<T><<<grid_for(n), VT, 0, st>>>(n, a, x, b, y);
    return cudaGetLastError();
}

cudaError_t vec_lincomb(long long n, const double* x, int nv, const double* V, long long ldv, const Coeffs& c,
                        double* out, cudaStream_t st) {
    k_lincomb<<<grid_for(n), VT, 0, st>>>(n, x, nv, V, ldv, c, out);
    return cudaGetLastError();
}

cudaError_t vec_newton_residual(long long n, const double* Y, const double* fY, double gdt, const double* rhs,
                                double* G, cudaStream_t st) {
    k_newton_residual<<<grid_for(n), VT, 0, st>>>(n, Y, fY, gdt, rhs, G);
    return cudaGetLastError();
}

template <typename S, typename D>
cudaError_t vec_convert(long long n, const S* src, double scale, D* dst, cudaStream_t st) {
    k_convert<S, D><<<grid_for(n), VT, 0, st>>>(n, src, scale, dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t vec_add_into(long long n, const T* x, double* y, cudaStream_t st) {
    k_add_into<T><<<grid_for(n), VT, 0, st>>>(n, x, y);
    return cudaGetLastError();
}

template <typename T>
cudaError_t vec_mdot(long long n, int nv, const T* V, long long ldv, const T* w, double* part, double* out,
                     cudaStream_t st) {
    dim3 grid(RED_BLOCKS, (nv + NVC - 1) / NVC);
    k_mdot_partial<T><<<grid, VT, 0, st>>>(n, nv, V, ldv, w, part, 0);
    k_rows_sum<<<nv, VT, 0, st>>>(part, RED_BLOCKS, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t vec_mdot_self(long long n, int nv, const T* V, long long ldv, const T* w, double* part, double* out,
                          cudaStream_t st) {
    dim3 grid(RED_BLOCKS, (nv + NVC - 1) / NVC);
    k_mdot_partial<T><<<grid, VT, 0, st>>>(n, nv, V, ldv, w, part, 1);
    k_rows_sum<<<nv + 1, VT, 0, st>>>(part, RED_BLOCKS, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t vec_update_norm(long long n, int nv, const T* V, long long ldv, const double* h, T* w, double* part,
                            double* norm2_out, cudaStream_t st) {
    k_update_norm<T><<<RED_BLOCKS, VT, 0, st>>>(n, nv, V, ldv, h, w, part);
    k_rows_sum<<<1, VT, 0, st>>>(part, RED_BLOCKS, norm2_out);
    return cudaGetLastError();
}

template <typename T>
bool vec_packed(long long n, const void* V, long long ldv, const void* w) {
    constexpr int W = 16 / sizeof(T);
    return n % W == 0 && ldv % W == 0 && reinterpret_cast<uintptr_t>(V) % 16 == 0 &&
           reinterpret_cast<uintptr_t>(w) % 16 == 0;
}

template <typename T>
cudaError_t vec_gs_dots(long long n, int nv, const T* V, long long ldv, const T* w, double* part, double* dots,
                        double* G, int ldg, double* h, cudaStream_t st) {
    dim3 grid(RED_BLOCKS, (nv + NVC - 1) / NVC);
    k_mdot2_partial<T><<<grid, VT, 0, st>>>(n, nv, V, ldv, w, part);
    k_rows_sum<<<2 * nv + 1, VT, 0, st>>>(part, RED_BLOCKS, dots);
    k_gram_coeffs<<<1, 64, 0, st>>>(nv, dots, G, ldg, h);
    return cudaGetLastError();
}

template <typename T>
cudaError_t vec_update_norm16(long long n, int nv, const T* V, long long ldv, const double* h, T* w, double* part,
                              double* norm2_out, cudaStream_t st) {
    k_update_norm16<T><<<RED_BLOCKS, VT, 0, st>>>(n, nv, V, ldv, h, w, part);
    k_rows_sum<<<1, VT, 0, st>>>(part, RED_BLOCKS, norm2_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t vec_basis_combine(long long n, int nv, const T* V, long long ldv, const Coeffs& y, T* x,
                              cudaStream_t st) {
    k_basis_combine<T><<<grid_for(n), VT, 0, st>>>(n, nv, V, ldv, y, x);
    return cudaGetLastError();
}

template <typename T>
cudaError_t vec_scale_modes(long long n, const double* table, int period, T* x, cudaStream_t st) {
    k_scale_modes<T><<<grid_for(n), VT, 0, st>>>(n, table, period, x);
    return cudaGetLastError();
}

long long reduction_scratch_doubles(int max_vectors) { return (long long)RED_BLOCKS * max_vectors; }

template bool vec_packed<double>(long long, const void*, long long, const void*);
template bool vec_packed<float>(long long, const void*, long long, const void*);
template cudaError_t vec_gs_dots<double>(long long, int, const double*, long long, const double*, double*, double*,
                                         double*, int, double*, cudaStream_t);
template cudaError_t vec_gs_dots<float>(long long, int, const float*, long long, const float*, double*, double*,
                                        double*, int, double*, cudaStream_t);
template cudaError_t vec_update_norm16<double>(long long, int, const double*, long long, const double*, double*,
                                               double*, double*, cudaStream_t);
template cudaError_t vec_update_norm16<float>(long long, int, const float*, long long, const double*, float*,
                                              double*, double*, cudaStream_t);
template cudaError_t vec_scale_modes<double>(long long, const double*, int, double*, cudaStream_t);
template cudaError_t vec_scale_modes<float>(long long, const double*, int, float*, cudaStream_t);
template cudaError_t vec_axpby<double>(long long, double, const double*, double, double*, cudaStream_t);
template cudaError_t vec_axpby<float>(long long, double, const float*, double, float*, cudaStream_t);
template cudaError_t vec_convert<double, float>(long long, const double*, double, float*, cudaStream_t);
template cudaError_t vec_convert<float, double>(long long, const float*, double, double*, cudaStream_t);
template cudaError_t vec_convert<double, double>(long long, const double*, double, double*, cudaStream_t);
template cudaError_t vec_convert<float, float>(long long, const float*, double, float*, cudaStream_t);
template cudaError_t vec_add_into<double>(long long, const double*, double*, cudaStream_t);
template cudaError_t vec_add_into<float>(long long, const float*, double*, cudaStream_t);
template cudaError_t vec_mdot_self<double>(long long, int, const double*, long long, const double*, double*,
                                           double*, cudaStream_t);
template cudaError_t vec_mdot_self<float>(long long, int, const float*, long long, const float*, double*, double*,
                                          cudaStream_t);
template cudaError_t vec_update_norm<double>(long long, int, const double*, long long, const double*, double*,
                                             double*, double*, cudaStream_t);
template cudaError_t vec_update_norm<float>(long long, int, const float*, long long, const double*, float*,
                                            double*, double*, cudaStream_t);
template cudaError_t vec_mdot<double>(long long, int, const double*, long long, const double*, double*, double*,
                                      cudaStream_t);
template cudaError_t vec_mdot<float>(long long, int, const float*, long long, const float*, double*, double*,
                                     cudaStream_t);
template cudaError_t vec_basis_combine<double>(long long, int, const double*, long long, const Coeffs&, double*,
                                               cudaStream_t);
template cudaError_t vec_basis_combine<float>(long long, int, const float*, long long, const Coeffs&, float*,
                                              cudaStream_t);

}  // namespace cdg2
