// Element-block-Jacobi preconditioner of the stage systems (I - gdt J) d = r
// of the DIRK stages (Sec. 3.2 solves them by Newton-GMRES and leaves the
// preconditioner open).  The block of element K and species s is the
// diagonal block of I - gdt J for the diffusion part of M^{-1} L_h:
//     P_Ks = I - gdt A_s K_K,   K_K = sum_j h_j^{-2} S_j^{tau_j} (x) I,
// the Kronecker sum over the axes of a 1D matrix S^tau on [0,1] built from
// the Legendre tables: the volume stiffness and the element's own terms of
// the interior-face diffusion flux of Sec. 3.1 (Eq. convDiscr: consistency,
// symmetry and the CDG2 penalty chi_e (k+1)^2 / h on the jump; BR2 and SIPG
// use their own penalty constant).  Along axis j the element has both faces
// (tau = 0), no low face (1, Gamma_1 or a no-flow wall), no high face (2),
// neither (3), or one face with itself (4, a periodic axis of one cell).
// On the orthonormal basis the tangential mass is the identity, so K_K
// separates by axis.  Boundary faces add nothing: their data do not depend
// on U (Eq. (3), H' = 0).  The chemotaxis and reaction parts are left out:
// with them the blocks change per element and Newton iterate, without them
// there are a few distinct blocks per mesh, and GMRES needs as many
// iterations with either (both measured on small 2D meshes at dt = 1e-3, 1e-2).
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "precond.h"

namespace cdg2 {

namespace {

constexpr int NTAU = 5;

int tau_of(const Geo& g, int j, long long i) {
    if (g.periodic[j]) return g.n[j] == 1 ? 4 : 0;
    if (g.n[j] == 1) return 3;
    if (i == 0) return 1;
    if (i == g.n[j] - 1) return 2;
    return 0;
}

// S^tau[a][b] on the reference interval (multiply by h^-2): row a is the
// test mode, column b the trial mode.
void oned_matrix(const Tab1D& t, int k, double pc, int tau, double* S) {
    const int nb1 = k + 1, nq = k + 2;
    const bool low = tau == 0 || tau == 2, high = tau == 0 || tau == 1, self = tau == 4;
    for (int a = 0; a < nb1; ++a)
        for (int b = 0; b < nb1; ++b) {
            double v = 0.0;
            for (int q = 0; q < nq; ++q) v -= t.w[q] * t.D[q][a] * t.D[q][b];
            const double e0a = t.e[0][a], e1a = t.e[1][a], d0a = t.d[0][a], d1a = t.d[1][a];
            const double e0b = t.e[0][b], e1b = t.e[1][b], d0b = t.d[0][b], d1b = t.d[1][b];
            if (high)   // K is K^-: sigma (phi^-) + tau (d_n phi^-), U^- = U_K
                v += 0.5 * (e1a * d1b + d1a * e1b) - pc * e1a * e1b;
            if (low)    // K is K^+: -sigma (phi^+) + tau (d_n phi^+), U^+ = U_K
                v += -0.5 * (e0a * d0b + d0a * e0b) - pc * e0a * e0b;
            if (self) { // one face with K on both sides: U^- = U^+ = U_K
                const double sig = 0.5 * (d1b + d0b) - pc * (e1b - e0b);
                const double tau_b = 0.5 * (e1b - e0b);
                v += (e1a - e0a) * sig + (d1a + d0a) * tau_b;
            }
            S[a * nb1 + b] = v;
        }
}

// Present tau values per axis and the type numbering.
void type_layout(const Geo& g, BlockTable& bt, std::vector<int> taus[3]) {
    int stride = 1;
    for (int j = 0; j < 3; ++j) {
        taus[j].clear();
        for (int u = 0; u < NTAU; ++u) bt.slot[j][u] = 0;
        if (j >= g.dim) {
            taus[j].push_back(0);
            bt.stride[j] = 0;
            continue;
        }
        bool seen[NTAU] = {false, false, false, false, false};
        for (long long i = 0; i < g.n[j]; ++i) seen[tau_of(g, j, i)] = true;
        for (int u = 0; u < NTAU; ++u)
            if (seen[u]) {
                bt.slot[j][u] = (int)taus[j].size();
                taus[j].push_back(u);
            }
        bt.stride[j] = stride;
        stride *= (int)taus[j].size();
    }
    bt.n_types = stride;
}

// P = I - gdt A_s sum_j h_j^-2 S_j^{tau_j} (x) I on the element basis
// (index a_0 + (k+1) (a_1 + (k+1) a_2)), row-major nb x nb.
void element_block(const cdg2_mesh& m, double As, double gdt, const int tau[3], double* P) {
    const Geo& g = m.geo;
    const int k = g.k, nb1 = k + 1, nb = m.nb;
    const double pc = g.pen_c * (k + 1) * (k + 1);
    std::vector<double> S[3];
    for (int j = 0; j < g.dim; ++j) {
        S[j].resize((size_t)nb1 * nb1);
        oned_matrix(m.tab, k, pc, tau[j], S[j].data());
    }
    for (int r = 0; r < nb; ++r)
        for (int c = 0; c < nb; ++c) {
            int ar[3] = {r % nb1, (r / nb1) % nb1, r / (nb1 * nb1)};
            int ac[3] = {c % nb1, (c / nb1) % nb1, c / (nb1 * nb1)};
            double kv = 0.0;
            for (int j = 0; j < g.dim; ++j) {
                bool other_equal = true;
                for (int l = 0; l < g.dim; ++l)
                    if (l != j && ar[l] != ac[l]) other_equal = false;
                if (other_equal) kv += S[j][(size_t)ar[j] * nb1 + ac[j]] / (g.h[j] * g.h[j]);
            }
            P[(size_t)r * nb + c] = (r == c ? 1.0 : 0.0) - gdt * As * kv;
        }
}

// Gauss-Jordan inverse with partial pivoting; false if singular.
bool invert(int n, std::vector<double>& A, std::vector<double>& X) {
    X.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) X[(size_t)i * n + i] = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * n + col]) > std::fabs(A[(size_t)piv * n + col])) piv = r;
        if (!(std::fabs(A[(size_t)piv * n + col]) > 0.0)) return false;
        if (piv != col)
            for (int c = 0; c < n; ++c) {
                std::swap(A[(size_t)piv * n + c], A[(size_t)col * n + c]);
                std::swap(X[(size_t)piv * n + c], X[(size_t)col * n + c]);
            }
        const double inv = 1.0 / A[(size_t)col * n + col];
        for (int c = 0; c < n; ++c) {
            A[(size_t)col * n + c] *= inv;
            X[(size_t)col * n + c] *= inv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double f = A[(size_t)r * n + col];
            if (f == 0.0) continue;
            for (int c = 0; c < n; ++c) {
                A[(size_t)r * n + c] -= f * A[(size_t)col * n + c];
                X[(size_t)r * n + c] -= f * X[(size_t)col * n + c];
            }
        }
    }
    return true;
}

struct ApplyArgs {
    long long E;
    int nb, dim;
    int n[3], periodic[3];
    int stride[3];
    int slot[3][NTAU];
};

__device__ __forceinline__ int dev_tau(const ApplyArgs& a, int j, long long i) {
    if (a.periodic[j]) return a.n[j] == 1 ? 4 : 0;
    if (a.n[j] == 1) return 3;
    if (i == 0) return 1;
    if (i == a.n[j] - 1) return 2;
    return 0;
}

// Elements per CTA of the block apply: a run long enough that the rows of the
// inverse blocks, loaded into registers once per CTA (and again only where
// the element type changes), are reused over many elements.
template <int NB>
constexpr int block_apply_run() { return 32 * (128 / NB); }

// z = P^{-1} v for one species and a run of CH consecutive elements per CTA.
// Thread (g, i), g < G = 128 / NB, owns output mode i of every G-th element
// of the run and keeps row i of its element type's inverse block in
// registers (reloaded only when the type changes along the run: at boundary
// layers); the run's input slices are staged in shared memory.
template <int NB, typename T>
__global__ void __launch_bounds__(128) k_block_apply(const ApplyArgs a, const T* __restrict__ M,
                                                     const T* __restrict__ v, T* __restrict__ z) {
    constexpr int G = 128 / NB;
    constexpr int CH = block_apply_run<NB>();
    __shared__ __align__(16) T sv[CH][NB];
    __shared__ int stype[CH];
    const int s = blockIdx.y;
    const long long e0 = (long long)blockIdx.x * CH;
    const int ne = (int)min((long long)CH, a.E - e0);
    for (int idx = threadIdx.x; idx < ne * NB; idx += 128) {
        const int e = idx / NB, j = idx % NB;
        sv[e][j] = v[((e0 + e) * NS + s) * NB + j];
    }
    // the element types of the run, once per element (index arithmetic in
    // 64-bit and indexed argument loads are slow per thread)
    for (int e = threadIdx.x; e < ne; e += 128) {
        long long rest = e0 + e;
        int type = 0;
        for (int j = 0; j < a.dim; ++j) {
            const long long ij = rest % a.n[j];
            rest /= a.n[j];
            type += a.slot[j][dev_tau(a, j, ij)] * a.stride[j];
        }
        stype[e] = type;
    }
    __syncthreads();
    const int g = threadIdx.x / NB, i = threadIdx.x % NB;
    if (g >= G) return;
    T m[NB];
    int cur = -1;
    for (int e = g; e < ne; e += G) {
        const int type = stype[e];
        if (type != cur) {
            const T* Mts = M + ((size_t)type * NS + s) * NB * NB;
#pragma unroll
            for (int j = 0; j < NB; ++j) m[j] = Mts[j * NB + i];
            cur = type;
        }
        T acc = T(0);
        if constexpr (sizeof(T) == 4 && NB % 4 == 0) {
            // the row of the input slice read 16 bytes at a time (a broadcast
            // to the warp): a quarter of the shared-memory instructions; four
            // independent partial sums instead of one chain of NB FMAs
            const float4* sv4 = reinterpret_cast<const float4*>(&sv[e][0]);
            float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
            for (int j = 0; j < NB / 4; ++j) {
                const float4 x = sv4[j];
                p0 = fma(m[4 * j], x.x, p0);
                p1 = fma(m[4 * j + 1], x.y, p1);
                p2 = fma(m[4 * j + 2], x.z, p2);
                p3 = fma(m[4 * j + 3], x.w, p3);
            }
            acc = (p0 + p1) + (p2 + p3);
        } else {
#pragma unroll
            for (int j = 0; j < NB; ++j) acc = fma(m[j], sv[e][j], acc);
        }
        z[((e0 + e) * NS + s) * NB + i] = acc;
    }
}

// The component kk (0..3) of a float4; kk is a constant after unrolling.
__device__ __forceinline__ float f4c(const float4& x, int kk) {
    return kk == 0 ? x.x : (kk == 1 ? x.y : (kk == 2 ? x.z : x.w));
}

// The type of element e (as dev_tau and the slots above) in 32-bit index
// arithmetic (E * 6 * nb < 2^31 for every mesh) and with constant argument
// indices: 64-bit divisions and indexed kernel-argument reads (a local copy
// of the arguments) made the type computation a visible part of the apply.
__device__ __forceinline__ int elem_type32(const ApplyArgs& a, long long e) {
    unsigned rest = (unsigned)e;
    int type = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j < a.dim) {
            const unsigned nj = (unsigned)a.n[j];
            const unsigned ij = rest % nj;
            rest /= nj;
            int tau = 0;
            if (a.periodic[j]) tau = nj == 1 ? 4 : 0;
            else if (nj == 1) tau = 3;
            else if (ij == 0) tau = 1;
            else if (ij == nj - 1) tau = 2;
            const int sl = tau == 0 ? a.slot[j][0]
                         : tau == 1 ? a.slot[j][1]
                         : tau == 2 ? a.slot[j][2]
                         : tau == 3 ? a.slot[j][3] : a.slot[j][4];
            type += sl * a.stride[j];
        }
    }
    return type;
}

// z = P^{-1} v for NB = 64 (Q3 hexahedra) in FP32: one CTA of 128 threads
// per (run of 64 elements, species), the run's input slices sx[e][j] and an
// element type's inverse block sm[j][i] = P^{-1}[i][j] staged in shared
// memory.  Register-tiled product: thread (rg, eg) accumulates the rows
// {4rg..4rg+3, 32+4rg..32+4rg+3} of the 4 elements 4eg..4eg+3, so a value
// read from shared memory feeds 4 or 8 FMAs.  (One shared value per FMA, as
// in k_block_apply, caps the product at the shared-memory delivery rate of
// 32 values per cycle per SM: a quarter of the FP32 FMA rate.)  A run that
// crosses a boundary layer holds several element types (fewer than 32: at
// most 3 per axis); it is applied once per type present, each pass storing
// the elements of its type.  The first element's block is staged with the
// input.  vec4: v and z are 16-byte aligned (16-byte global accesses).
__global__ void __launch_bounds__(128, 6) k_block_apply64(const ApplyArgs a, const float* __restrict__ M,
                                                       const float* __restrict__ v, float* __restrict__ z, int vec4) {
    constexpr int NB = 64, RUN = 64, NT = 128;
    __shared__ __align__(16) float sx[RUN][NB];
    __shared__ __align__(16) float sm[NB][NB];
    __shared__ int stype[RUN];
    __shared__ unsigned smask;
    const int s = blockIdx.y, tid = threadIdx.x;
    const long long e0 = (long long)blockIdx.x * RUN;
    const int ne = (int)min((long long)RUN, a.E - e0);
    int cur = elem_type32(a, e0);
    if (tid == 0) smask = 0u;
    if (tid < RUN) stype[tid] = tid < ne ? elem_type32(a, e0 + tid) : -1;   // padding: no type, never stored
    {
        const float4* Mg = reinterpret_cast<const float4*>(M + ((size_t)cur * NS + s) * NB * NB);
        for (int q = tid; q < NB * NB / 4; q += NT) reinterpret_cast<float4*>(&sm[0][0])[q] = Mg[q];
    }
    if (vec4) {
        for (int idx = tid; idx < RUN * NB / 4; idx += NT) {
            const int e = idx / (NB / 4), q = idx % (NB / 4);
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < ne) x = reinterpret_cast<const float4*>(v + ((e0 + e) * NS + s) * NB)[q];
            reinterpret_cast<float4*>(&sx[e][0])[q] = x;
        }
    } else {
        for (int idx = tid; idx < RUN * NB; idx += NT) {
            const int e = idx / NB, j = idx % NB;
            sx[e][j] = e < ne ? v[((e0 + e) * NS + s) * NB + j] : 0.f;
        }
    }
    __syncthreads();
    if (tid < ne) atomicOr(&smask, 1u << stype[tid]);
    __syncthreads();
    unsigned left = smask;   // the types present (the same in every thread)
    const int rg = tid % 8, eg = tid / 8;   // a quarter warp shares eg: its x reads are broadcasts
    for (;;) {
        bool mine = false;
#pragma unroll
        for (int c = 0; c < 4; ++c) mine |= stype[eg * 4 + c] == cur;
        if (mine) {
            float acc[4][8];
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int r = 0; r < 8; ++r) acc[c][r] = 0.f;
#pragma unroll 4
            for (int k = 0; k < NB; k += 4) {
                float4 xr[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) xr[c] = *reinterpret_cast<const float4*>(&sx[eg * 4 + c][k]);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float4 m0 = *reinterpret_cast<const float4*>(&sm[k + kk][4 * rg]);
                    const float4 m1 = *reinterpret_cast<const float4*>(&sm[k + kk][32 + 4 * rg]);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float x = f4c(xr[c], kk);
                        acc[c][0] = fmaf(m0.x, x, acc[c][0]);
                        acc[c][1] = fmaf(m0.y, x, acc[c][1]);
                        acc[c][2] = fmaf(m0.z, x, acc[c][2]);
                        acc[c][3] = fmaf(m0.w, x, acc[c][3]);
                        acc[c][4] = fmaf(m1.x, x, acc[c][4]);
                        acc[c][5] = fmaf(m1.y, x, acc[c][5]);
                        acc[c][6] = fmaf(m1.z, x, acc[c][6]);
                        acc[c][7] = fmaf(m1.w, x, acc[c][7]);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int e = eg * 4 + c;
                if (stype[e] != cur) continue;   // another type's pass, or padding
                float* out = z + ((e0 + e) * NS + s) * NB;
                if (vec4) {
                    reinterpret_cast<float4*>(out + 4 * rg)[0] =
                        make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
                    reinterpret_cast<float4*>(out + 32 + 4 * rg)[0] =
                        make_float4(acc[c][4], acc[c][5], acc[c][6], acc[c][7]);
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        out[4 * rg + r] = acc[c][r];
                        out[32 + 4 * rg + r] = acc[c][4 + r];
                    }
                }
            }
        }
        left &= ~(1u << cur);
        if (left == 0u) break;
        cur = __ffs((int)left) - 1;
        __syncthreads();   // the previous type's block is read by no thread any more
        const float4* Mg = reinterpret_cast<const float4*>(M + ((size_t)cur * NS + s) * NB * NB);
        for (int q = tid; q < NB * NB / 4; q += NT) reinterpret_cast<float4*>(&sm[0][0])[q] = Mg[q];
        __syncthreads();
    }
}

template <int NB, typename T>
static void launch_nb(const ApplyArgs& a, const T* M, const T* v, T* z, cudaStream_t st) {
    if constexpr (NB == 64 && sizeof(T) == 4) {
        auto al16 = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
        const dim3 grid((unsigned)((a.E + 63) / 64), NS);
        k_block_apply64<<<grid, 128, 0, st>>>(a, M, v, z, al16(v) && al16(z) ? 1 : 0);
        return;
    }
    constexpr int CH = block_apply_run<NB>();
    const dim3 grid((unsigned)((a.E + CH - 1) / CH), NS);
    k_block_apply<NB, T><<<grid, 128, 0, st>>>(a, M, v, z);
}

int max_types(const Geo& g) {
    int t = 1;
    for (int j = 0; j < g.dim; ++j) t *= 3;   // at most three tau values on one axis
    return t;
}

}  // namespace

size_t block_table_bytes(const cdg2_mesh& m) {
    const size_t per = (size_t)max_types(m.geo) * NS * m.nb * m.nb;
    return (per * sizeof(double) + 255) / 256 * 256 + (per * sizeof(float) + 255) / 256 * 256;
}

int build_block_table(const cdg2_mesh& m, const Coef& c, double gdt, void* dev, BlockTable& bt) {
    std::vector<int> taus[3];
    type_layout(m.geo, bt, taus);
    const int nb = m.nb;
    const size_t per_block = (size_t)nb * nb;
    std::vector<double> h64((size_t)bt.n_types * NS * per_block);
    std::vector<float> h32(h64.size());
    std::vector<double> P(per_block), X;
    for (int t = 0; t < bt.n_types; ++t) {
        int tau[3] = {0, 0, 0};
        for (int j = 0; j < m.geo.dim; ++j) tau[j] = taus[j][(t / bt.stride[j]) % (int)taus[j].size()];
        for (int s = 0; s < NS; ++s) {
            element_block(m, c.A[s], gdt, tau, P.data());
            if (!invert(nb, P, X)) {
                set_error("cdg2_step: singular preconditioner block (dt * A too large for I - dt a_ii A K)");
                return CDG2_ERR_INVALID_ARG;
            }
            double* dst = h64.data() + ((size_t)t * NS + s) * per_block;
            for (int i = 0; i < nb; ++i)
                for (int j = 0; j < nb; ++j) dst[(size_t)j * nb + i] = X[(size_t)i * nb + j];
        }
    }
    for (size_t i = 0; i < h64.size(); ++i) h32[i] = (float)h64[i];
    const size_t per = (size_t)max_types(m.geo) * NS * per_block;
    char* base = static_cast<char*>(dev);
    double* d64 = reinterpret_cast<double*>(base);
    float* d32 = reinterpret_cast<float*>(base + (per * sizeof(double) + 255) / 256 * 256);
    cudaError_t e = cudaMemcpy(d64, h64.data(), sizeof(double) * h64.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d32, h32.data(), sizeof(float) * h32.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_step: preconditioner blocks");
    bt.m64 = d64;
    bt.m32 = d32;
    return CDG2_OK;
}

template <typename T>
cudaError_t block_apply(const cdg2_mesh& m, const BlockTable& bt, const T* v, T* z, cudaStream_t st) {
    ApplyArgs a;
    a.E = m.geo.E;
    a.nb = m.nb;
    a.dim = m.geo.dim;
    for (int j = 0; j < 3; ++j) {
        a.n[j] = m.geo.n[j];
        a.periodic[j] = m.geo.periodic[j];
        a.stride[j] = bt.stride[j];
        for (int u = 0; u < NTAU; ++u) a.slot[j][u] = bt.slot[j][u];
    }
    const T* M;
    if constexpr (sizeof(T) == 8) M = bt.m64;
    else M = bt.m32;
    switch (a.nb) {
        case 4: launch_nb<4, T>(a, M, v, z, st); break;
        case 8: launch_nb<8, T>(a, M, v, z, st); break;
        case 9: launch_nb<9, T>(a, M, v, z, st); break;
        case 16: launch_nb<16, T>(a, M, v, z, st); break;
        case 27: launch_nb<27, T>(a, M, v, z, st); break;
        case 64: launch_nb<64, T>(a, M, v, z, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t block_apply<double>(const cdg2_mesh&, const BlockTable&, const double*, double*, cudaStream_t);
template cudaError_t block_apply<float>(const cdg2_mesh&, const BlockTable&, const float*, float*, cudaStream_t);

}  // namespace cdg2

using namespace cdg2;

extern "C" int cdg2_element_block(const cdg2_mesh* m, const cdg2_params* p, double gdt, long long elem, int species,
                                  double* out) {
    if (!m || !p || !out) {
        set_error("cdg2_element_block: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (elem < 0 || elem >= m->geo.E || species < 0 || species >= NS || !std::isfinite(gdt)) {
        set_error("cdg2_element_block: element, species or gdt out of range");
        return CDG2_ERR_INVALID_ARG;
    }
    const Coef c = make_coef(*p);
    int tau[3] = {0, 0, 0};
    long long rest = elem;
    for (int j = 0; j < m->geo.dim; ++j) {
        tau[j] = tau_of(m->geo, j, rest % m->geo.n[j]);
        rest /= m->geo.n[j];
    }
    element_block(*m, c.A[species], gdt, tau, out);
    return CDG2_OK;
}
