// Tensor-core element kernel of the FP32 operator on 3D Q3 meshes (apply and
// JVP): the basis-to-quadrature contractions of the volume terms (Sec. 3.1,
// Eq. elementint) as TF32 GEMMs on the fifth-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), batched over 16 elements.
//
// Per CTA (16 consecutive elements, 512 threads, one CTA per SM):
//   1. the forward table image (128 points x 64 modes: psi, dpsi/dx, dpsi/dy,
//      dpsi/dz at the 5^3 Gauss points, rows 125..127 zero) is copied to shared
//      memory, and the coefficients of both fields, rounded to TF32, are
//      staged as the MMAs' B operands (rows species-major: n1, c1, c3, n2, n3,
//      c2, then element);
//   2. one thread issues the forward MMAs: point values of all six species
//      and the gradients of n1, c1, c3 (the fluxes need no others: the
//      diffusion of every species is applied in modal form) into tensor memory,
//      lanes = points, columns = (quantity, species, element);
//   3. the weighted, transposed test table image (64 modes x 128 points, the
//      Gauss weights folded in) replaces the forward one; every thread owns
//      one point and, for its elements, reads the values and gradients of
//      both fields straight from tensor memory, evaluates the pointwise
//      (linearised) flux and source, and writes them as the test MMAs' B
//      operands;
//   4. the test MMAs (M = 64 modes) accumulate the volume residual in tensor
//      memory; it goes to shared memory while bulk copies bring the tile's
//      coefficients and the tested fluxes of its faces (the face kernels'
//      buffer) into the freed table region; the modal diffusion of all species and
//      the two tested face fluxes per axis are added from shared memory, and
//      the epilogue (M^{-1}, alpha w + beta J w) stores.
// Operands use the 128-byte-swizzled K-major layout (TF32 operands must be
// K-major).  Every wait on an mbarrier is bounded: on time-out the kernel sets
// bit 1 of the status word, frees its tensor memory and returns.
#pragma once

#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "elem_common.cuh"
#include "physics.cuh"

namespace cdg2 {
namespace tc {

constexpr int NE = 16;                        // elements per CTA
constexpr int NT = 512;                       // threads per CTA: 4 groups of 4 elements x 4 lane quarters
constexpr int NB = 64, NQ = 125, NP = 128;    // modes, Gauss points, padded points (3D Q3)
constexpr int TAB_BYTES = 4 * NP * NB * 4;    // one table set: 4 tables of 128 x 64 (or 64 x 128) floats
constexpr int TAB1 = NP * NB * 4;             // one table
constexpr int ROWS = NS * NE;                 // B-operand rows of the values (species x element)
constexpr int FWD_FIELD = 2 * ROWS * 128;     // one field's forward operand image: 2 K-blocks x 96 rows x 128 B
constexpr int TST_S = 4 * ROWS * 128;         // test operand of the source: 4 K-blocks x 96 rows x 128 B
constexpr int TST_G = 4 * 32 * 128;           // test operand of one flux direction (n1, n2): 4 K-blocks x 32 rows
constexpr int OPS_BYTES = TST_S + 3 * TST_G;  // 98304: >= both fields' forward operands (49152)
constexpr int TMEM_COLS = 512;
constexpr int FIELD_COLS = 240;               // per field: 96 value columns, 3 x 48 gradient columns
// dynamic shared memory: 1 KB of slack to align the swizzled images to 1024 B,
// the table set, the operand region, then the small arrays
constexpr int SMALL_OFF = TAB_BYTES + OPS_BYTES;
constexpr int SMALL_BYTES = 2048;             // STab<3, float> (1000 B), 5 mbarriers, tmem slot
// epilogue staging in the table region: the tested fluxes of each element's two faces
// per axis ([axis][element][lo, hi] records of 2 x 6 x 16 floats), then the tile's coefficients
constexpr int FACE_REC = 2 * NS * 16 * 4;     // 768 B
constexpr int EPI_COEF = 3 * NE * 2 * FACE_REC;   // 73728: offset of the coefficients (NE x 1536 B)
constexpr int SMEM_BYTES = 1024 + SMALL_OFF + SMALL_BYTES;

// forward species order -> species; the first three have gradients
__host__ __device__ constexpr int fwd_species(int sp) {
    return sp == 0 ? 0 : (sp == 1 ? 3 : (sp == 2 ? 5 : (sp == 3 ? 1 : (sp == 4 ? 2 : 4))));
}
__host__ __device__ constexpr int fwd_slot(int s) {   // inverse of fwd_species
    return s == 0 ? 0 : (s == 3 ? 1 : (s == 5 ? 2 : (s == 1 ? 3 : (s == 2 ? 4 : 5))));
}

// Byte offset of element (row r, k) of a 128-byte-swizzled K-major block
// (k < 32 within the block; 8-row groups of 1024 bytes).
__host__ __device__ constexpr uint32_t sw128(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + (k & 3) * 4);
}

// ---- PTX wrappers ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets,
// descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major): 16 B
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t id, int acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(dt), "l"(ad), "l"(bd), "r"(id), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
}

// Bounded wait for the phase of an mbarrier (2^22 polls, well above any
// legitimate wait of this kernel): false on time-out.
__device__ __forceinline__ bool wait(uint32_t bar, uint32_t phase) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(ok) : "r"(bar), "r"(phase) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void ld_x2(uint32_t a, float& x, float& y) {
    uint32_t r0, r1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(a));
    x = __uint_as_float(r0);
    y = __uint_as_float(r1);
}

__device__ __forceinline__ void ld_x8(uint32_t a, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(a));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Round to the nearest TF32 value (ties away from zero) with two integer
// operations (finite inputs), written as integer instructions so that they
// stay on the integer pipe (the conversion instruction runs on the narrow
// FP64 pipe here).
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t u;
    asm("{\n\t.reg .u32 t;\n\tadd.u32 t, %1, 4096;\n\tand.b32 %0, t, 0xFFFFE000;\n\t}" : "=r"(u) : "r"(__float_as_uint(x)));
    return __uint_as_float(u);
}

// One thread: expect `bytes` on the mbarrier and copy them from global to
// shared memory with bulk asynchronous copies of 16 KB (16-byte aligned,
// sizes multiples of 16), completing on the mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
    for (uint32_t off = 0; off < bytes; off += 16384) {
        const uint32_t n = bytes - off < 16384 ? bytes - off : 16384;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(dst + off), "l"(static_cast<const char*>(src) + off), "r"(n), "r"(bar)
                     : "memory");
    }
}

// Host: round to the nearest TF32 value (10-bit mantissa), ties away from zero.
inline float host_tf32(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// Host: the forward and the test table images of a 3D Q3 mesh, each set
// 4 x 32 KB, forward first.  Forward table t (0: psi, 1..3: dpsi/dx_j / h_j)
// at [point q][mode i]; test table t at [mode i][point q] times the Gauss
// weight w_q.  Points q = q0 + 5 q1 + 25 q2, modes i = a0 + 4 a1 + 16 a2 (x
// fastest, as the coefficients).  Values rounded to TF32, swizzled.
inline void build_tables(const Tab1D& t, const Geo& g, std::vector<float>& img) {
    img.assign(2 * TAB_BYTES / 4, 0.0f);
    auto fwd = [&](int tb, int q, int i) -> float& {
        return img[(tb * TAB1 + (i >> 5) * (NP * 128) + sw128(q, i & 31)) / 4];
    };
    auto tst = [&](int tb, int i, int q) -> float& {
        return img[(TAB_BYTES + tb * TAB1 + (q >> 5) * (NB * 128) + sw128(i, q & 31)) / 4];
    };
    for (int q = 0; q < NQ; ++q) {
        const int q0 = q % 5, q1 = (q / 5) % 5, q2 = q / 25;
        const double w = t.w[q0] * t.w[q1] * t.w[q2];
        for (int i = 0; i < NB; ++i) {
            const int a0 = i % 4, a1 = (i / 4) % 4, a2 = i / 16;
            const double b0 = t.B[q0][a0], b1 = t.B[q1][a1], b2 = t.B[q2][a2];
            const double v[4] = {b0 * b1 * b2, t.D[q0][a0] / g.h[0] * b1 * b2, b0 * t.D[q1][a1] / g.h[1] * b2,
                                 b0 * b1 * t.D[q2][a2] / g.h[2]};
            for (int tb = 0; tb < 4; ++tb) {
                fwd(tb, q, i) = host_tf32((float)v[tb]);
                tst(tb, i, q) = host_tf32((float)(w * v[tb]));
            }
        }
    }
}

}  // namespace tc

// The tensor-core element kernel.  F = 1 (apply) or 2 (JVP: U and the tangent).
template <int MODE>
__global__ void __launch_bounds__(512, 1) tc_elem_kernel(const Geo g, const TabP<float> tab, const OpArgs<float> args,
                                                        const float4* __restrict__ tables) {
    using namespace tc;
    constexpr int F = fields_of(MODE);
    constexpr int D = 3, K = 3;
    extern __shared__ __align__(1024) unsigned char smem_dyn[];
    // the swizzle works on shared-address bits 4..9: align the images to 1024 B ourselves
    unsigned char* smem = smem_dyn + ((1024 - (smem_u32(smem_dyn) & 1023)) & 1023);
    unsigned char* sTab = smem;                          // table set (forward, then test)
    unsigned char* sOps = smem + TAB_BYTES;              // forward operands, then test operands, then sR
    float* sR = reinterpret_cast<float*>(sOps);          // [NE][6][64] volume residual / |K|
    STab<K, float>& tb = *reinterpret_cast<STab<K, float>*>(smem + SMALL_OFF);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + SMALL_OFF + 1024 + 256);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + SMALL_OFF + 1024 + 256 + 48);
    float* sA = reinterpret_cast<float*>(smem + SMALL_OFF + 1024 + 256 + 64);   // A_s (diffusion coefficients)
    static_assert(sizeof(STab<K, float>) <= 1024, "tables of the face expansion exceed their slot");
    const int t = threadIdx.x;
    const long long e0 = (long long)blockIdx.x * NE;
    const uint32_t sbase = smem_u32(smem);
    // bar0: forward MMAs done; bar1: test MMAs done; bar2 / bar3: forward / test tables copied;
    // bar4: the epilogue's face records and coefficients copied
    const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
    const uint32_t bar2 = smem_u32(&bars[2]), bar3 = smem_u32(&bars[3]), bar4 = smem_u32(&bars[4]);
    const CoefT<float>& c = args.c;

    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar2));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar3));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar4));
        asm volatile("fence.mbarrier_init.release.cluster;");
        // forward tables (already swizzled in global memory), copied while the coefficients are staged
        bulk_load(sbase, tables, TAB_BYTES, bar2);
    }
    load_tab<K, float>(tb, tab);
    if (t == 0) {
#pragma unroll
        for (int sp = 0; sp < NS; ++sp) sA[sp] = c.A[sp];
    }
    // coefficients of the 16 elements, TF32, species-major rows (tangent pre-scaled);
    // each thread's loads are issued together
    constexpr int CH = NE * NS * (NB / 4);   // 16-byte chunks per field
    static_assert(CH % NT == 0, "chunks per field must divide among the threads");
#pragma unroll
    for (int fi = 0; fi < F; ++fi) {
        const float* src = fi == 0 ? args.U[0] : args.U[1];
        unsigned char* img = sOps + fi * FWD_FIELD;
        float4 v[CH / NT];
#pragma unroll
        for (int j = 0; j < CH / NT; ++j) {
            const int idx = t + NT * j;
            const int ch = idx % (NB / 4), s = (idx / (NB / 4)) % NS, e = idx / (NS * (NB / 4));
            v[j] = e0 + e < g.E ? __ldg(reinterpret_cast<const float4*>(src + (e0 + e) * (NS * NB) + s * NB) + ch)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < CH / NT; ++j) {
            const int idx = t + NT * j;
            const int ch = idx % (NB / 4), s = (idx / (NB / 4)) % NS, e = idx / (NS * (NB / 4));
            float4 w = v[j];
            if (MODE == MODE_JVP && fi == 1 && args.pscale) {
                const double* ps = args.pscale + s * NB + 4 * ch;
                w.x *= float(ps[0]);
                w.y *= float(ps[1]);
                w.z *= float(ps[2]);
                w.w *= float(ps[3]);
            }
            const int r = fwd_slot(s) * NE + e, k = 4 * ch;
            *reinterpret_cast<float4*>(img + (k >> 5) * (ROWS * 128) + sw128(r, k & 31)) =
                make_float4(to_tf32(w.x), to_tf32(w.y), to_tf32(w.z), to_tf32(w.w));
        }
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tslot)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tm = *reinterpret_cast<volatile uint32_t*>(tslot);

    // ---- forward MMAs: values (N = 96) and gradients of n1, c1, c3 (N = 48) ----
    const bool tabs_in = __syncthreads_and(wait(bar2, 0)) != 0;
    if (t == 0 && tabs_in) {
        for (int fi = 0; fi < F; ++fi) {
            const uint32_t bimg = sbase + TAB_BYTES + fi * FWD_FIELD;
            for (int tt = 0; tt < 4; ++tt) {
                const int n = tt == 0 ? ROWS : 3 * NE;
                const uint32_t col = fi * FIELD_COLS + (tt == 0 ? 0 : ROWS + (tt - 1) * 3 * NE);
                const uint32_t id = idesc(128, n);
                for (int kk = 0; kk < NB / 8; ++kk) {
                    const uint32_t a = sbase + tt * TAB1 + (kk >> 2) * (NP * 128) + (kk & 3) * 32;
                    const uint32_t b = bimg + (kk >> 2) * (ROWS * 128) + (kk & 3) * 32;
                    mma(tm + col, sdesc(a, 1024), sdesc(b, 1024), id, kk > 0);
                }
            }
        }
        commit(bar0);
    }
    // CTA-uniform: the tensor-memory loads below are warp-collective
    bool ok = tabs_in && __syncthreads_and(wait(bar0, 0)) != 0;
    fence_after();

    // ---- the test tables replace the forward ones (the forward MMAs are done), copied during the pointwise phase ----
    if (ok && t == 0) bulk_load(sbase, tables + TAB_BYTES / 16, TAB_BYTES, bar3);

    // ---- pointwise: one point per thread, 4 elements per thread (4 groups of warps) ----
    const int warp = t >> 5, lane = t & 31;
    const int quarter = warp & 3, group = warp >> 2;
    const int q = quarter * 32 + lane;
    const uint32_t tlane = tm + ((uint32_t)(quarter * 32) << 16);
    // (all warps read tensor memory before any thread overwrites the operand region:
    // the forward operands are dead once bar0 has completed, so writes may start at once)
    if (ok) {
        const int q0 = q % 5, q1 = (q / 5) % 5;
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
            const int ea = group * 4 + 2 * pr;
            float u[2][F][NS], gr[2][F][3][3];   // [element][field][...]
#pragma unroll
            for (int fi = 0; fi < F; ++fi) {
                const uint32_t base = tlane + fi * FIELD_COLS;
#pragma unroll
                for (int sp = 0; sp < NS; ++sp) ld_x2(base + sp * NE + ea, u[0][fi][sp], u[1][fi][sp]);
#pragma unroll
                for (int d = 0; d < 3; ++d)
#pragma unroll
                    for (int gg = 0; gg < 3; ++gg)
                        ld_x2(base + ROWS + d * 3 * NE + gg * NE + ea, gr[0][fi][d][gg], gr[1][fi][d][gg]);
            }
            wait_ld();
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int e = ea + h2;
                float Sr[NS], Phi[NS][D];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    Sr[s] = 0.f;
#pragma unroll
                    for (int j = 0; j < D; ++j) Phi[s][j] = 0.f;
                }
                if (q < NQ && e0 + e < g.E) {
                    float uu[NS], gu[NS][D];
#pragma unroll
                    for (int s = 0; s < NS; ++s) {
                        uu[s] = u[h2][0][fwd_slot(s)];
#pragma unroll
                        for (int j = 0; j < D; ++j) gu[s][j] = 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        gu[0][j] = gr[h2][0][j][0];
                        gu[3][j] = gr[h2][0][j][1];
                        gu[5][j] = gr[h2][0][j][2];
                    }
                    if constexpr (MODE == MODE_APPLY) {
                        volume_point<D, float, 2>(c, uu, gu, Phi, Sr);
                        if (args.flags & CDG2_FORCING) {
                            const long long ge = e0 + e;
                            const long long ix = ge % g.n[0], iy = (ge / g.n[0]) % g.n[1];
                            const float x = float(ix * g.h[0]) + float(g.h[0]) * tb.xi[q0];
                            const float y = float(iy * g.h[1]) + float(g.h[1]) * tb.xi[q1];
                            float gf[NS];
                            mms_forcing<float>(x, y, float(args.t), float(g.L[1]), c, gf);
#pragma unroll
                            for (int s = 0; s < NS; ++s) Sr[s] += gf[s];
                        }
                    } else {
                        float du[NS], dg[NS][D];
#pragma unroll
                        for (int s = 0; s < NS; ++s) {
                            du[s] = u[h2][F - 1][fwd_slot(s)];
#pragma unroll
                            for (int j = 0; j < D; ++j) dg[s][j] = 0.f;
                        }
#pragma unroll
                        for (int j = 0; j < D; ++j) {
                            dg[0][j] = gr[h2][F - 1][j][0];
                            dg[3][j] = gr[h2][F - 1][j][1];
                            dg[5][j] = gr[h2][F - 1][j][2];
                        }
                        volume_point_lin<D, float, 2>(c, uu, gu, du, dg, args.has_dtheta != 0, Phi, Sr);
                    }
                }
                // test operands: K = point q; rows species x element
                const int kb = q >> 5, kq = q & 31;
#pragma unroll
                for (int s = 0; s < NS; ++s)
                    *reinterpret_cast<float*>(sOps + kb * (ROWS * 128) + sw128(s * NE + e, kq)) = to_tf32(Sr[s]);
#pragma unroll
                for (int j = 0; j < D; ++j)
#pragma unroll
                    for (int s = 0; s < 2; ++s)
                        *reinterpret_cast<float*>(sOps + TST_S + j * TST_G + kb * (32 * 128) + sw128(s * NE + e, kq)) =
                            to_tf32(Phi[s][j]);
            }
        }
    }
    fence_async();
    fence_before();
    __syncthreads();
    fence_after();

    // ---- test MMAs: R[mode][species x element] (M = 64, weights in the test tables) ----
    if (ok) ok = __syncthreads_and(wait(bar3, 0)) != 0;
    if (t == 0 && ok) {
        for (int tt = 0; tt < 4; ++tt) {
            const int n = tt == 0 ? ROWS : 2 * NE;
            const uint32_t id = idesc(64, n);
            for (int kk = 0; kk < NP / 8; ++kk) {
                const uint32_t a = sbase + tt * TAB1 + (kk >> 2) * (NB * 128) + (kk & 3) * 32;
                const uint32_t b = tt == 0 ? sbase + TAB_BYTES + (kk >> 2) * (ROWS * 128) + (kk & 3) * 32
                                           : sbase + TAB_BYTES + TST_S + (tt - 1) * TST_G + (kk >> 2) * (32 * 128) +
                                                 (kk & 3) * 32;
                mma(tm, sdesc(a, 1024), sdesc(b, 1024), id, (tt > 0 || kk > 0) ? 1 : 0);
            }
        }
        commit(bar1);
    }
    if (ok) ok = __syncthreads_and(wait(bar1, 0)) != 0;
    fence_after();
    // ---- the epilogue's data into the freed table region: face records and coefficients ----
    const int ne_real = (int)(g.E - e0 < NE ? g.E - e0 : NE);
    if (ok) {
        if (t == 0) {
            const uint32_t bytes = (uint32_t)ne_real * (NS * NB * 4 + 6 * FACE_REC);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar4), "r"(bytes) : "memory");
        }
        __syncthreads();
        if (t < 3 * NE * 2) {
            const int a = t / (2 * NE), e = (t / 2) % NE, side = t & 1;
            const long long ge = e0 + e;
            if (ge < g.E) {
                long long f = ge;
                if (side == 0) {
                    const long long nb = neighbour(g, ge, a, 0);
                    f = nb >= 0 ? nb : g.E + low_layer_index(g, ge, a);
                }
                // (the axis' offset by selection: an indexed parameter access would copy the
                // kernel's parameters to local memory)
                const long long off = a == 0 ? args.fb_off[0] : (a == 1 ? args.fb_off[1] : args.fb_off[2]);
                const float* src = args.fbuf + off + f * (2 * NS * 16);
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             :: "r"(sbase + (uint32_t)(((a * NE + e) * 2 + side) * FACE_REC)), "l"(src),
                                "r"((uint32_t)FACE_REC), "r"(bar4)
                             : "memory");
            }
        } else if (t == 3 * NE * 2) {
            const float* src = (F == 1 ? args.U[0] : args.U[1]) + e0 * (NS * NB);
            const uint32_t bytes = (uint32_t)ne_real * (NS * NB * 4);
            for (uint32_t off = 0; off < bytes; off += 16384) {
                const uint32_t n = bytes - off < 16384 ? bytes - off : 16384;
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             :: "r"(sbase + EPI_COEF + off), "l"(reinterpret_cast<const char*>(src) + off), "r"(n),
                                "r"(bar4)
                             : "memory");
            }
        }
    }
    // residual to shared memory: M = 64 puts mode i in lane (i / 16) * 32 + i % 16
    if (ok) {
        const int cbase = group * (ROWS / 4);
        for (int c0 = 0; c0 < ROWS / 4; c0 += 8) {
            float v[8];
            ld_x8(tlane + cbase + c0, v);
            wait_ld();
            if (lane < 16) {
                const int i = quarter * 16 + lane;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int col = cbase + c0 + j, s = col / NE, e = col % NE;
                    sR[(e * NS + s) * NB + i] = v[j];
                }
            }
        }
    } else if (t == 0) {
        atomicOr(c.domain, 2);   // a tensor-core wait timed out
        // give the copies and MMAs in flight one more bounded wait before the block's
        // tensor memory is freed and its shared memory released
        wait(bar2, 0);
        wait(bar0, 0);
        wait(bar3, 0);
        wait(bar1, 0);
    }
    fence_before();
    __syncthreads();
    if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tm), "r"(TMEM_COLS));
    if (!ok) return;
    if (__syncthreads_and(wait(bar4, 0)) == 0) {
        if (t == 0) {
            atomicOr(c.domain, 2);
            wait(bar4, 0);
        }
        __syncthreads();
        return;
    }
    const float* sC = reinterpret_cast<const float*>(sTab + EPI_COEF);   // [e][s][i] of the last field
    const float* sF = reinterpret_cast<const float*>(sTab);              // face records [axis][e][lo, hi][2][6][16]

    // ---- per (element, species, mode), one pass: the modal diffusion of all six species (exact on
    // the orthonormal basis, in FP32: the diffusive fluxes stay off the TF32 contractions), from
    // the field's coefficients; the two tested face fluxes per axis (from the staged records);
    // M^{-1}; store ----
    const float scale = (args.flags & CDG2_MINV) ? 1.f : c.vol;
    const float alphaT = float(args.alpha), betaT = float(args.beta);
    const double* psg = MODE == MODE_JVP ? args.pscale : nullptr;
    // NT is a multiple of NB: all of a thread's items share its mode i, so the mode's table
    // entries are read from shared memory once, into registers
    static_assert(NT % NB == 0, "a thread's items must share one mode");
    const int i = t % NB;
    const int am[3] = {i % 4, (i / 4) % 4, i / 16};
    float k1[3][K], fe0[3], fd0[3], fe1[3], fd1[3];
    int tt[3];
#pragma unroll
    for (int j = 0; j < D; ++j) {
#pragma unroll
        for (int bb = 1; bb <= K; ++bb) k1[j][bb - 1] = tb.K1h[j][am[j]][bb];
        fe0[j] = -tb.e[0][am[j]];
        fd0[j] = tb.dh[j][0][am[j]];
        fe1[j] = tb.e[1][am[j]];
        fd1[j] = tb.dh[j][1][am[j]];
        // tangential index: the other two axes in increasing order
        tt[j] = j == 0 ? am[1] + 4 * am[2] : (j == 1 ? am[0] + 4 * am[2] : am[0] + 4 * am[1]);
    }
    // the loop with and without the tangent's pre-scale (a branch outside it, not per load)
    auto items = [&](auto scaled) {
        constexpr bool SCALED = decltype(scaled)::value;
        for (int idx = t; idx < NE * NS * NB; idx += NT) {
            const int es = idx / NB, e = es / NS, s = es % NS;
            if (e >= ne_real) continue;
            const float* uf = sC + es * NB;
            float md = 0.f;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                // 1D stiffness of axis j: modes b of a_j's parity, both > 0
                const int a = am[j];
                const int stride = j == 0 ? 1 : (j == 1 ? 4 : 16);
                const int base = i - a * stride;
#pragma unroll
                for (int bb = 1; bb <= K; ++bb) {
                    if (a > 0 && ((a ^ bb) & 1) == 0) {
                        const int ci = base + bb * stride;
                        const float uv = SCALED ? uf[ci] * float(psg[s * NB + ci]) : uf[ci];
                        md = fma(k1[j][bb - 1], uv, md);
                    }
                }
            }
            float acc = fma(-sA[s], md, sR[idx]);
#pragma unroll
            for (int a = 0; a < D; ++a) {
                const float* lo = sF + ((a * NE + e) * 2 + 0) * (FACE_REC / 4) + s * 16 + tt[a];
                const float* hi = sF + ((a * NE + e) * 2 + 1) * (FACE_REC / 4) + s * 16 + tt[a];
                acc = fma(fe0[a], lo[0], acc);
                acc = fma(fd0[a], lo[NS * 16], acc);
                acc = fma(fe1[a], hi[0], acc);
                acc = fma(fd1[a], hi[NS * 16], acc);
            }
            if constexpr (MODE == MODE_JVP) {
                float w = sC[idx];
                if (SCALED) w *= float(psg[idx % (NS * NB)]);
                args.out[e0 * (NS * NB) + idx] = alphaT * w + betaT * (acc * scale);
            } else {
                args.out[e0 * (NS * NB) + idx] = acc * scale;
            }
        }
    };
    if (psg)
        items(std::true_type{});
    else
        items(std::false_type{});
}

}  // namespace cdg2
