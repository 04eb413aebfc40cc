// Face kernel of the face-once path on 3D meshes (apply and JVP): the same
// face terms as face_kernel (Sec. 3.1: symmetric diffusive flux with the
// CDG2 penalty, local Lax-Friedrichs chemotactic flux, the boundary
// conditions of Eq. 3), laid out for issue efficiency:
//   - both cells of every face arrive by bulk asynchronous copies (one
//     thread, one mbarrier) where a cell's block is a multiple of 16 bytes
//     and the fields are 16-byte aligned, else by batched loads;
//   - the fluxes of n3, c1, c2, c3 are purely diffusive and linear: with the
//     orthonormal tangential basis and exact face quadrature their tested
//     fluxes follow from the normal contraction in modal form, so only n1,
//     n2, c1, c3 go to the face points and only n1, n2 are tested there;
//     the stage buffers hold just those species;
//   - the boundary data of Eq. 3 at the points of the owning trace (n1, n2
//     through the points; the c2 influx on Gamma_1, which does not depend on
//     U, tested directly);
//   - enough faces per CTA that the pointwise phase has one face point per
//     thread (FPB x n_q^2 <= 128), and the stage buffers alias one another
//     along their lifetimes.
// Output: the same face records as face_kernel, [2][6][n_bt] per face.
#pragma once

namespace cdg2 {

// slot of a species in the face-point stage buffers ({n1, n2, c1, c3}), -1 if none
__host__ __device__ constexpr int set5_slot(int s) { return s < 2 ? s : (s == 3 ? 2 : (s == 5 ? 3 : -1)); }

template <int K, int F, typename T>
struct Face3Plan {
    using S = Shape<3, K>;
    static constexpr int NB = S::NB, NB1 = S::NB1, NQ1 = S::NQ1, NBT = S::NBT, NQT = S::NQT;
    static constexpr int NT = 128;
    // faces per CTA: one thread per face point in the pointwise phase; on Q3
    // the FP64 JVP keeps to 3 faces so that three CTAs fit on an SM, and FP32
    // takes 4 (swept 3 / 4 / 5 on 3D 64x16x16 Q3, TF32 JVP: 0.418 / 0.417 /
    // 0.441 ms)
    static constexpr int FPB = K == 1 ? 14 : (K == 2 ? 8 : (F == 2 && sizeof(T) == 8) ? 3 : (sizeof(T) == 4 ? 4 : 5));
    static_assert(FPB * NQT <= NT, "one face point per thread");
    static constexpr int N5 = SpeciesSet<5>::N;                   // n1, n2, c1, c3
    static constexpr int CELL = NS * NB;                          // one cell, one field
    static constexpr int CELLS = 2 * F * FPB * CELL;              // [side][field][face][6][n_b]
    static constexpr int FC = F * FPB * 4 * N5 * NBT;             // normal contraction [field][face][4][N5][n_bt]
    static constexpr int FT = F * FPB * 4 * N5 * NQ1 * NB1;       // half-interpolated
    static constexpr int FP = F * FPB * 4 * N5 * NQT;             // face-point values
    static constexpr int FS = FPB * 2 * 2 * NQT;                  // weighted sigma, tau of n1, n2 at the points
    static constexpr int TS1 = FPB * 2 * 2 * NB1 * NQ1;           // half-tested
    static constexpr int TS = FPB * 2 * NS * NBT;                 // tested fluxes (the output records)
    static constexpr int XN = cmax(cmax(CELLS, FT), FS + TS1);    // region X: cells, FT, FS + TS1
    static constexpr int YN = cmax(FC, FP);                       // region Y: FC, FP
    static constexpr bool BULK = (CELL * sizeof(T)) % 16 == 0;
    static constexpr int TAB_OFF = 16;                            // after the mbarrier
    static constexpr int X_OFF = (TAB_OFF + (int)sizeof(STab<K, T>) + 15) / 16 * 16;
    static constexpr size_t smem_bytes() { return (size_t)X_OFF + sizeof(T) * (size_t)(XN + YN + TS); }
};

// Bounded wait for phase 0 of the CTA's copy barrier (2^22 polls, far above
// any legitimate copy time): false on time-out.
__device__ __forceinline__ bool face3_wait(uint32_t bar) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(ok) : "r"(bar) : "memory");
        if (ok) return true;
    }
    return false;
}

template <int K, int MODE, int A, typename T>
__global__ void __launch_bounds__(128) face3_kernel(const Geo g, const TabP<T> tab, const OpArgs<T> args,
                                                    const int use_bulk) {
    constexpr int D = 3;
    constexpr int F = fields_of(MODE);
    using P = Face3Plan<K, F, T>;
    constexpr int FPB = P::FPB, NB = P::NB, NB1 = P::NB1, NQ1 = P::NQ1, NBT = P::NBT, NQT = P::NQT;
    constexpr int CELL = P::CELL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    STab<K, T>& tb = *reinterpret_cast<STab<K, T>*>(smem_raw + P::TAB_OFF);
    T* X = reinterpret_cast<T*>(smem_raw + P::X_OFF);
    T* Y = X + P::XN;
    T* Z = Y + P::YN;
    constexpr int N5 = P::N5;
    T* FC = Y;
    T* FT = X;
    T* FPt = Y;
    T* FS = X;
    T* TS1 = X + P::FS;
    T* TS = Z;
    __shared__ long long cm[FPB], cp[FPB];   // minus / plus cell (-1: none)
    __shared__ int kind[FPB];                // -1 unused, 0 interior, 1 high boundary, 2 low boundary
    __shared__ int copies_ok;
    __shared__ T sA[NS];
    __shared__ T psT[MODE == MODE_JVP ? NS * NB : 1];
    const CoefT<T>& c = args.c;
    const long long nf = faces_of_axis(g, A);
    const long long f0 = (long long)blockIdx.x * FPB;
    const int tid = threadIdx.x;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const bool bulk = P::BULK && use_bulk;   // the host checked the fields' 16-byte alignment

    if (tid == 0) {
#pragma unroll
        for (int sp = 0; sp < NS; ++sp) sA[sp] = c.A[sp];
        if (bulk) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    if (tid < FPB) {
        const long long fid = f0 + tid;
        int kd = -1;
        long long em = -1, ep = -1;
        if (fid < g.E) {
            em = fid;
            ep = neighbour(g, fid, A, 1);
            kd = ep >= 0 ? 0 : 1;
        } else if (fid < nf) {
            const long long l = fid - g.E;
            long long ix = 0, iy = 0, iz = 0;
            if (A == 0) { iy = l % g.n[1]; iz = l / g.n[1]; }
            else if (A == 1) { ix = l % g.n[0]; iz = l / g.n[0]; }
            else { ix = l % g.n[0]; iy = l / g.n[0]; }
            ep = ix + (long long)g.n[0] * (iy + (long long)g.n[1] * iz);
            kd = 2;
        }
        cm[tid] = em;
        cp[tid] = ep;
        kind[tid] = kd;
    }
    __syncthreads();
    if (bulk) {
        if (tid == 0) {
            uint32_t bytes = 0;
#pragma unroll 1
            for (int b = 0; b < 2 * F * FPB; ++b) {
                const int j = b % FPB, side = b / (F * FPB);
                if ((side ? cp[j] : cm[j]) >= 0) bytes += CELL * (uint32_t)sizeof(T);
            }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
#pragma unroll 1
            for (int b = 0; b < 2 * F * FPB; ++b) {
                const int j = b % FPB, fi = (b / FPB) % F, side = b / (F * FPB);
                const long long cell = side ? cp[j] : cm[j];
                if (cell < 0) continue;
                const T* src = field(args, fi) + cell * CELL;
                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(X + b * CELL);
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                             :: "r"(dst), "l"(src), "r"((uint32_t)(CELL * sizeof(T))), "r"(bar)
                             : "memory");
            }
        }
    } else {
        // batched loads: a batch of independent loads per thread in flight at once
        constexpr int TOT = P::CELLS, BATCH = 8;
        for (int i0 = tid; i0 < TOT; i0 += BATCH * P::NT) {
            T v[BATCH];
#pragma unroll
            for (int b = 0; b < BATCH; ++b) {
                const int i = i0 + b * P::NT;
                v[b] = T(0);
                if (i < TOT) {
                    const int blk = i / CELL, q = i - blk * CELL;
                    const int j = blk % FPB, fi = (blk / FPB) % F, side = blk / (F * FPB);
                    const long long cell = side ? cp[j] : cm[j];
                    if (cell >= 0) v[b] = field(args, fi)[cell * CELL + q];
                }
            }
#pragma unroll
            for (int b = 0; b < BATCH; ++b) {
                const int i = i0 + b * P::NT;
                if (i < TOT) X[i] = v[b];
            }
        }
    }
    load_tab<K, T>(tb, tab);
    const T* ps = nullptr;
    if constexpr (MODE == MODE_JVP) {
        if (args.pscale) {
            for (int i = tid; i < NS * NB; i += P::NT) psT[i] = T(args.pscale[i]);
            ps = psT;
        }
    }
    if (bulk) {
        if (tid == 0) {
            bool ok = face3_wait(bar);
            if (!ok) {
                if (c.domain) atomicOr(c.domain, 2);
                face3_wait(bar);   // let the copies in flight land before the CTA exits
            }
            copies_ok = ok;
        }
    }
    __syncthreads();
    if (bulk && !copies_ok) return;

    const T invh = c.invh[A];
    const T pen = c.pen_c * T((K + 1) * (K + 1)) * invh;
    // normal contraction: 0 the owning trace (K^- at xi = 1, or K^+ at xi = 0 on a
    // low boundary), 1 the jump (difference-first), 2 d_n U^-, 3 d_n U^+.  The
    // last field (the tangent in the JVP) over all species: n1, n2, c1, c3 to
    // the stage buffer, the modal fluxes of n3, c1, c2, c3 straight to the
    // output records; the JVP's first field (U) over n1, n2, c1, c3 only.
    {
        constexpr int NLAST = FPB * NS * NBT, NFIRST = (F - 1) * FPB * N5 * NBT;
        for (int idx = tid; idx < NLAST + NFIRST; idx += P::NT) {
            int fi, s, j, t;
            if (idx < NLAST) {
                fi = F - 1;
                t = idx % NBT;
                s = (idx / NBT) % NS;
                j = idx / (NBT * NS);
            } else {
                const int r = idx - NLAST;
                fi = 0;
                t = r % NBT;
                s = SpeciesSet<5>::s((r / NBT) % N5);
                j = r / (NBT * N5);
            }
            const int b0 = t % NB1, b1 = t / NB1;
            const T* um = X + (fi * FPB + j) * CELL + s * NB;
            const T* up = X + ((F + fi) * FPB + j) * CELL + s * NB;
            T vm[NB1], vp[NB1];
#pragma unroll
            for (int m = 0; m < NB1; ++m) {
                const int ci = coef_index<D, K, A>(m, b0, b1);
                vm[m] = um[ci];
                vp[m] = up[ci];
                if (MODE == MODE_JVP && fi == 1 && ps) {
                    vm[m] *= ps[s * NB + ci];
                    vp[m] *= ps[s * NB + ci];
                }
            }
            const int kd = kind[j];
            T uo = 0, del = 0, dm = 0, dp = 0;
            if (kd == 2) {
#pragma unroll
                for (int m = 0; m < NB1; ++m) uo = fma(tb.e[0][m], vp[m], uo);
            } else {
#pragma unroll
                for (int m = 0; m < NB1; ++m) uo = fma(tb.e[1][m], vm[m], uo);
            }
            if (kd == 0) {
                del = vm[0] - vp[0];
#pragma unroll
                for (int m = 1; m < NB1; ++m) {
                    del = fma(tb.e[1][m], vm[m], del);
                    del = fma(-tb.e[0][m], vp[m], del);
                }
#pragma unroll
                for (int m = 0; m < NB1; ++m) {
                    dm = fma(tb.dh[A][1][m], vm[m], dm);
                    dp = fma(tb.dh[A][0][m], vp[m], dp);
                }
            }
            const int ss = set5_slot(s);
            if (ss >= 0) {
                T* o = FC + ((fi * FPB + j) * 4) * N5 * NBT + ss * NBT + t;
                o[0 * N5 * NBT] = uo;
                o[1 * N5 * NBT] = del;
                o[2 * N5 * NBT] = dm;
                o[3 * N5 * NBT] = dp;
            }
            if (fi == F - 1 && s >= 2) {
                // sigma_t = A (d_n U^-_t + d_n U^+_t) / 2 - pen A Delta_t, tau_t = A Delta_t / 2,
                // weighted by 1 / h_A; zero on boundary faces (their data are added below)
                const T As = sA[s];
                const bool in = kd == 0;
                T* o = TS + (j * 2) * NS * NBT + s * NBT + t;
                o[0] = in ? invh * As * (T(0.5) * (dm + dp) - pen * del) : T(0);
                o[NS * NBT] = in ? invh * T(0.5) * As * del : T(0);
            }
        }
    }
    __syncthreads();
    sf_sym<0, NB1, NB1, 1, NQ1, false, K + 1, false, 1, 1>(FC, &tb.B[0][0], nullptr, nullptr, NBT, FT, NQ1 * NB1,
                                                       F * FPB * 4 * N5);
    __syncthreads();
    sf_sym<1, NQ1, NB1, 1, NQ1, false, K + 1, false, 1, 1>(FT, &tb.B[0][0], nullptr, nullptr, NQ1 * NB1, FPt, NQT,
                                                       F * FPB * 4 * N5);
    __syncthreads();

    // pointwise fluxes of n1, n2: one face point per thread
    if (tid < FPB * NQT) {
        const int p = tid % NQT, j = tid / NQT;
        const int kd = kind[j];
        const int p0 = p % NQ1, p1 = p / NQ1;
        const T Wp = tb.w[p0] * tb.w[p1] * invh;   // the element kernel accumulates the residual divided by |K|
        T uo[NS], del[NS], dm[NS], dp[NS];
        {
            const T* base = FPt + (j * 4) * N5 * NQT + p;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const int ss = set5_slot(s);
                uo[s] = ss < 0 ? T(0) : base[(0 * N5 + ss) * NQT];
                del[s] = ss < 0 ? T(0) : base[(1 * N5 + ss) * NQT];
                dm[s] = ss < 0 ? T(0) : base[(2 * N5 + ss) * NQT];
                dp[s] = ss < 0 ? T(0) : base[(3 * N5 + ss) * NQT];
            }
        }
        T sig[NS], tau[NS];
        if (kd == 0) {
            T uP[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) uP[s] = uo[s] - del[s];
            if constexpr (MODE == MODE_APPLY) {
                face_point<T>(c, pen, uo, dm, uP, dp, del, sig, tau);
            } else {
                T tuo[NS], tdel[NS], tdm[NS], tdp[NS], tuP[NS];
                const T* base = FPt + ((FPB + j) * 4) * N5 * NQT + p;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const int ss = set5_slot(s);
                    tuo[s] = ss < 0 ? T(0) : base[(0 * N5 + ss) * NQT];
                    tdel[s] = ss < 0 ? T(0) : base[(1 * N5 + ss) * NQT];
                    tdm[s] = ss < 0 ? T(0) : base[(2 * N5 + ss) * NQT];
                    tdp[s] = ss < 0 ? T(0) : base[(3 * N5 + ss) * NQT];
                    tuP[s] = tuo[s] - tdel[s];
                }
                face_point_lin<T>(c, pen, uo, dm, uP, dp, del, tuo, tdm, tuP, tdp, tdel, sig, tau);
            }
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                sig[s] = Wp * sig[s];
                tau[s] = Wp * tau[s];
            }
        } else {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                sig[s] = T(0);
                tau[s] = T(0);
            }
            if (A == 1 && kd > 0) {
                const int f = kd == 2 ? 0 : 1;             // Gamma_1 (y = 0) or Gamma_2 (y = L1)
                const long long cell = kd == 2 ? cp[j] : cm[j];
                const T x = T((cell % g.n[0]) * g.h[0]) + T(g.h[0]) * tb.xi[p0];
                if constexpr (MODE == MODE_APPLY)
                    boundary_point<T>(c, f, x, g, uo, sig, c.beta1, true);
                else
                    boundary_point<T>(c, f, x, g, uo, sig, c.dth[7], false);
                const T sg = kd == 2 ? -Wp : Wp;
#pragma unroll
                for (int s = 0; s < 2; ++s) sig[s] = sg * sig[s];
            }
        }
        T* o = FS + (j * 2) * 2 * NQT + p;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            o[(0 * 2 + s) * NQT] = sig[s];
            o[(1 * 2 + s) * NQT] = tau[s];
        }
    }
    __syncthreads();
    sf_sym<0, NQ1, NQ1, 1, NB1, true, K + 1, false, 1, 1>(FS, &tb.B[0][0], nullptr, nullptr, NQT, TS1, NB1 * NQ1,
                                                      FPB * 2 * 2);
    __syncthreads();
    sf_sym<1, NB1, NQ1, 1, NB1, true, K + 1, false, 1, 1, T, 2, true>(TS1, &tb.B[0][0], nullptr, nullptr, NB1 * NQ1,
                                                                  TS, NBT, FPB * 2 * 2);
    if constexpr (A == 1 && MODE == MODE_APPLY) {
        // the c2 influx on Gamma_1 (Eq. 3), bc_sign A_c2 sigma on Gamma_{1,in}, tested over
        // the points of the low-boundary faces (sigma of the owning cell: -W_p times the data)
        for (int idx = tid; idx < FPB * NBT; idx += P::NT) {
            const int j = idx / NBT, t = idx % NBT;
            if (kind[j] != 2) continue;
            const int t0 = t % NB1, t1 = t / NB1;
            const long long cell = cp[j];
            const T val = T(c.bc_sign) * sA[4] * T(c.sigma);
            T acc = T(0);
            for (int p1 = 0; p1 < NQ1; ++p1)
                for (int p0 = 0; p0 < NQ1; ++p0) {
                    const T x = T((cell % g.n[0]) * g.h[0]) + T(g.h[0]) * tb.xi[p0];
                    const T s4 = (x >= T(g.g1in[0]) && x <= T(g.g1in[1])) ? val : T(0);
                    const T Wp = tb.w[p0] * tb.w[p1] * invh;
                    acc = fma(tb.B[p0][t0] * tb.B[p1][t1], -Wp * s4, acc);
                }
            TS[(j * 2) * NS * NBT + 4 * NBT + t] = acc;
        }
    }
    __syncthreads();
    // coalesced store of the faces' tested fluxes
    T* dst = args.fbuf + args.fb_off[A];
    for (int i = tid; i < P::TS; i += P::NT) {
        const long long fid = f0 + i / (2 * NS * NBT);
        if (fid < nf) dst[f0 * 2 * NS * NBT + i] = TS[i];
    }
}

// Warp-per-face variant (the FP32 kernels on Q3, bound by issue rather than
// by the arithmetic pipe): every warp evaluates one face on its own -- its
// cells by bulk copy on its own mbarrier, then the phases of face3_kernel
// separated by warp barriers only -- so no warp waits for another at a CTA
// barrier; the CTA shares only the tables.
template <int K, int F, typename T>
struct Face3WPlan {
    using S = Shape<3, K>;
    static constexpr int NB = S::NB, NB1 = S::NB1, NQ1 = S::NQ1, NBT = S::NBT, NQT = S::NQT;
    static constexpr int WARPS = 4, NT = 32 * WARPS;
    static_assert(NQT <= 32, "one face point per lane");
    static constexpr int N5 = SpeciesSet<5>::N;
    static constexpr int CELL = NS * NB;
    static constexpr int CELLS = 2 * F * CELL;                    // [side][field][6][n_b]
    static constexpr int FC = F * 4 * N5 * NBT;
    static constexpr int FT = F * 4 * N5 * NQ1 * NB1;
    static constexpr int FP = F * 4 * N5 * NQT;
    static constexpr int FS = 2 * 2 * NQT;
    static constexpr int TS1 = 2 * 2 * NB1 * NQ1;
    static constexpr int TS = 2 * NS * NBT;
    static constexpr int XN = cmax(cmax(CELLS, FT), FS + TS1);
    static constexpr int YN = cmax(FC, FP);
    static constexpr int AL = 16 / (int)sizeof(T);                // one warp's region keeps X 16-byte aligned
    static constexpr int WN = (XN + YN + TS + AL - 1) / AL * AL;
    static constexpr bool BULK = (CELL * sizeof(T)) % 16 == 0;
    static constexpr int TAB_OFF = 64;                            // after the warps' mbarriers
    static constexpr int X_OFF = (TAB_OFF + (int)sizeof(STab<K, T>) + 15) / 16 * 16;
    static constexpr size_t smem_bytes() { return (size_t)X_OFF + sizeof(T) * (size_t)WARPS * WN; }
};

template <int K, int MODE, int A, typename T>
__global__ void __launch_bounds__(128) face3w_kernel(const Geo g, const TabP<T> tab, const OpArgs<T> args,
                                                     const int use_bulk) {
    constexpr int D = 3;
    constexpr int F = fields_of(MODE);
    using P = Face3WPlan<K, F, T>;
    constexpr int NB = P::NB, NB1 = P::NB1, NQ1 = P::NQ1, NBT = P::NBT, NQT = P::NQT, CELL = P::CELL;
    constexpr int N5 = P::N5;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    STab<K, T>& tb = *reinterpret_cast<STab<K, T>*>(smem_raw + P::TAB_OFF);
    __shared__ T sA[NS];
    __shared__ T psT[MODE == MODE_JVP ? NS * NB : 1];
    const CoefT<T>& c = args.c;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T* X = reinterpret_cast<T*>(smem_raw + P::X_OFF) + warp * P::WN;
    T* Y = X + P::XN;
    T* FC = Y;
    T* FT = X;
    T* FPt = Y;
    T* FS = X;
    T* TS1 = X + P::FS;
    T* TS = Y + P::YN;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(smem_raw) + 8 * warp;
    const bool bulk = P::BULK && use_bulk;   // the host checked the fields' 16-byte alignment
    const long long nf = faces_of_axis(g, A);
    const long long fid = (long long)blockIdx.x * P::WARPS + warp;

    // the warp's face (every lane forms the same values)
    int kd = -1;                 // -1 none, 0 interior, 1 high boundary, 2 low boundary
    long long em = -1, ep = -1;  // minus / plus cell (-1: none)
    if (fid < g.E) {
        em = fid;
        ep = neighbour(g, fid, A, 1);
        kd = ep >= 0 ? 0 : 1;
    } else if (fid < nf) {
        const long long l = fid - g.E;
        long long ix = 0, iy = 0, iz = 0;
        if (A == 0) { iy = l % g.n[1]; iz = l / g.n[1]; }
        else if (A == 1) { ix = l % g.n[0]; iz = l / g.n[0]; }
        else { ix = l % g.n[0]; iy = l / g.n[0]; }
        ep = ix + (long long)g.n[0] * (iy + (long long)g.n[1] * iz);
        kd = 2;
    }
    if (kd >= 0) {
        if (bulk) {
            if (lane == 0) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
                const uint32_t bytes = ((em >= 0 ? 1u : 0u) + (ep >= 0 ? 1u : 0u)) * F * CELL * (uint32_t)sizeof(T);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
#pragma unroll
                for (int b = 0; b < 2 * F; ++b) {
                    const int fi = b % F, side = b / F;
                    const long long cell = side ? ep : em;
                    if (cell < 0) continue;
                    const T* src = field(args, fi) + cell * CELL;
                    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(X + b * CELL);
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 :: "r"(dst), "l"(src), "r"((uint32_t)(CELL * sizeof(T))), "r"(bar)
                                 : "memory");
                }
            }
        } else {
            for (int i = lane; i < P::CELLS; i += 32) {
                const int b = i / CELL, q = i - b * CELL;
                const int fi = b % F, side = b / F;
                const long long cell = side ? ep : em;
                X[i] = cell >= 0 ? field(args, fi)[cell * CELL + q] : T(0);
            }
        }
    }
    if (tid == 0) {
#pragma unroll
        for (int sp = 0; sp < NS; ++sp) sA[sp] = c.A[sp];
    }
    load_tab<K, T>(tb, tab);
    const T* ps = nullptr;
    if constexpr (MODE == MODE_JVP) {
        if (args.pscale) {
            for (int i = tid; i < NS * NB; i += P::NT) psT[i] = T(args.pscale[i]);
            ps = psT;
        }
    }
    __syncthreads();   // the tables; from here on the warps are independent
    if (kd < 0) return;
    if (bulk) {
        int ok = 1;
        if (lane == 0) {
            ok = face3_wait(bar) ? 1 : 0;
            if (!ok) {
                if (c.domain) atomicOr(c.domain, 2);
                face3_wait(bar);   // let the copies in flight land before the warp exits
            }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) return;
    }
    __syncwarp();

    const T invh = c.invh[A];
    const T pen = c.pen_c * T((K + 1) * (K + 1)) * invh;
    // normal contraction (as in face3_kernel, one face)
    {
        constexpr int NLAST = NS * NBT, NFIRST = (F - 1) * N5 * NBT;
        // the 1D trace and normal-derivative tables in registers (every item reads all of them)
        T e0r[NB1], e1r[NB1], d0r[NB1], d1r[NB1];
#pragma unroll
        for (int m = 0; m < NB1; ++m) {
            e0r[m] = tb.e[0][m];
            e1r[m] = tb.e[1][m];
            d0r[m] = tb.dh[A][0][m];
            d1r[m] = tb.dh[A][1][m];
        }
        for (int idx = lane; idx < NLAST + NFIRST; idx += 32) {
            int fi, s, t;
            if (idx < NLAST) {
                fi = F - 1;
                t = idx % NBT;
                s = idx / NBT;
            } else {
                const int r = idx - NLAST;
                fi = 0;
                t = r % NBT;
                s = SpeciesSet<5>::s(r / NBT);
            }
            const int b0 = t % NB1, b1 = t / NB1;
            const T* um = X + fi * CELL + s * NB;
            const T* up = X + (F + fi) * CELL + s * NB;
            T vm[NB1], vp[NB1];
            if constexpr (A == 0 && NB1 == 4 && sizeof(T) == 4) {
                // normal axis x: a line's four coefficients are 16 contiguous bytes
                const int c0 = coef_index<D, K, A>(0, b0, b1);
                const float4 qm = *reinterpret_cast<const float4*>(um + c0);
                const float4 qp = *reinterpret_cast<const float4*>(up + c0);
                vm[0] = qm.x; vm[1] = qm.y; vm[2] = qm.z; vm[3] = qm.w;
                vp[0] = qp.x; vp[1] = qp.y; vp[2] = qp.z; vp[3] = qp.w;
                if (MODE == MODE_JVP && fi == 1 && ps) {
#pragma unroll
                    for (int m = 0; m < NB1; ++m) {
                        vm[m] *= ps[s * NB + c0 + m];
                        vp[m] *= ps[s * NB + c0 + m];
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < NB1; ++m) {
                    const int ci = coef_index<D, K, A>(m, b0, b1);
                    vm[m] = um[ci];
                    vp[m] = up[ci];
                    if (MODE == MODE_JVP && fi == 1 && ps) {
                        vm[m] *= ps[s * NB + ci];
                        vp[m] *= ps[s * NB + ci];
                    }
                }
            }
            T uo = 0, del = 0, dm = 0, dp = 0;
            if (kd == 2) {
#pragma unroll
                for (int m = 0; m < NB1; ++m) uo = fma(e0r[m], vp[m], uo);
            } else {
#pragma unroll
                for (int m = 0; m < NB1; ++m) uo = fma(e1r[m], vm[m], uo);
            }
            if (kd == 0) {
                del = vm[0] - vp[0];
#pragma unroll
                for (int m = 1; m < NB1; ++m) {
                    del = fma(e1r[m], vm[m], del);
                    del = fma(-e0r[m], vp[m], del);
                }
#pragma unroll
                for (int m = 0; m < NB1; ++m) {
                    dm = fma(d1r[m], vm[m], dm);
                    dp = fma(d0r[m], vp[m], dp);
                }
            }
            const int ss = set5_slot(s);
            if (ss >= 0) {
                T* o = FC + (fi * 4) * N5 * NBT + ss * NBT + t;
                o[0 * N5 * NBT] = uo;
                o[1 * N5 * NBT] = del;
                o[2 * N5 * NBT] = dm;
                o[3 * N5 * NBT] = dp;
            }
            if (fi == F - 1 && s >= 2) {
                const T As = sA[s];
                const bool in = kd == 0;
                T* o = TS + s * NBT + t;
                o[0] = in ? invh * As * (T(0.5) * (dm + dp) - pen * del) : T(0);
                o[NS * NBT] = in ? invh * T(0.5) * As * del : T(0);
            }
        }
    }
    __syncwarp();
    sf_sym<0, NB1, NB1, 1, NQ1, false, K + 1, false, 1, 1>(FC, &tb.B[0][0], nullptr, nullptr, NBT, FT, NQ1 * NB1,
                                                       F * 4 * N5, lane, 32);
    __syncwarp();
    sf_sym<1, NQ1, NB1, 1, NQ1, false, K + 1, false, 1, 1>(FT, &tb.B[0][0], nullptr, nullptr, NQ1 * NB1, FPt, NQT,
                                                       F * 4 * N5, lane, 32);
    __syncwarp();
    if (lane < NQT) {
        const int p = lane;
        const int p0 = p % NQ1, p1 = p / NQ1;
        const T Wp = tb.w[p0] * tb.w[p1] * invh;
        T uo[NS], del[NS], dm[NS], dp[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const int ss = set5_slot(s);
            uo[s] = ss < 0 ? T(0) : FPt[(0 * N5 + ss) * NQT + p];
            del[s] = ss < 0 ? T(0) : FPt[(1 * N5 + ss) * NQT + p];
            dm[s] = ss < 0 ? T(0) : FPt[(2 * N5 + ss) * NQT + p];
            dp[s] = ss < 0 ? T(0) : FPt[(3 * N5 + ss) * NQT + p];
        }
        T sig[NS], tau[NS];
        if (kd == 0) {
            T uP[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) uP[s] = uo[s] - del[s];
            if constexpr (MODE == MODE_APPLY) {
                face_point<T>(c, pen, uo, dm, uP, dp, del, sig, tau);
            } else {
                T tuo[NS], tdel[NS], tdm[NS], tdp[NS], tuP[NS];
                const T* base = FPt + 4 * N5 * NQT + p;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    const int ss = set5_slot(s);
                    tuo[s] = ss < 0 ? T(0) : base[(0 * N5 + ss) * NQT];
                    tdel[s] = ss < 0 ? T(0) : base[(1 * N5 + ss) * NQT];
                    tdm[s] = ss < 0 ? T(0) : base[(2 * N5 + ss) * NQT];
                    tdp[s] = ss < 0 ? T(0) : base[(3 * N5 + ss) * NQT];
                    tuP[s] = tuo[s] - tdel[s];
                }
                face_point_lin<T>(c, pen, uo, dm, uP, dp, del, tuo, tdm, tuP, tdp, tdel, sig, tau);
            }
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                sig[s] = Wp * sig[s];
                tau[s] = Wp * tau[s];
            }
        } else {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                sig[s] = T(0);
                tau[s] = T(0);
            }
            if (A == 1) {
                const int f = kd == 2 ? 0 : 1;             // Gamma_1 (y = 0) or Gamma_2 (y = L1)
                const long long cell = kd == 2 ? ep : em;
                const T x = T((cell % g.n[0]) * g.h[0]) + T(g.h[0]) * tb.xi[p0];
                if constexpr (MODE == MODE_APPLY)
                    boundary_point<T>(c, f, x, g, uo, sig, c.beta1, true);
                else
                    boundary_point<T>(c, f, x, g, uo, sig, c.dth[7], false);
                const T sg = kd == 2 ? -Wp : Wp;
#pragma unroll
                for (int s = 0; s < 2; ++s) sig[s] = sg * sig[s];
            }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            FS[(0 * 2 + s) * NQT + p] = sig[s];
            FS[(1 * 2 + s) * NQT + p] = tau[s];
        }
    }
    __syncwarp();
    sf_sym<0, NQ1, NQ1, 1, NB1, true, K + 1, false, 1, 1>(FS, &tb.B[0][0], nullptr, nullptr, NQT, TS1, NB1 * NQ1, 2 * 2,
                                                      lane, 32);
    __syncwarp();
    sf_sym<1, NB1, NQ1, 1, NB1, true, K + 1, false, 1, 1, T, 2, true>(TS1, &tb.B[0][0], nullptr, nullptr, NB1 * NQ1,
                                                                  TS, NBT, 2 * 2, lane, 32);
    if constexpr (A == 1 && MODE == MODE_APPLY) {
        // the c2 influx on Gamma_1 (Eq. 3), tested over the points of a low-boundary face
        if (kd == 2) {
            for (int t = lane; t < NBT; t += 32) {
                const int t0 = t % NB1, t1 = t / NB1;
                const T val = T(c.bc_sign) * sA[4] * T(c.sigma);
                T acc = T(0);
                for (int p1 = 0; p1 < NQ1; ++p1)
                    for (int p0 = 0; p0 < NQ1; ++p0) {
                        const T x = T((ep % g.n[0]) * g.h[0]) + T(g.h[0]) * tb.xi[p0];
                        const T s4 = (x >= T(g.g1in[0]) && x <= T(g.g1in[1])) ? val : T(0);
                        const T Wp = tb.w[p0] * tb.w[p1] * invh;
                        acc = fma(tb.B[p0][t0] * tb.B[p1][t1], -Wp * s4, acc);
                    }
                TS[4 * NBT + t] = acc;
            }
        }
    }
    __syncwarp();
    T* dst = args.fbuf + args.fb_off[A] + fid * (2 * NS * NBT);
    for (int i = lane; i < P::TS; i += 32) dst[i] = TS[i];
}

}  // namespace cdg2
