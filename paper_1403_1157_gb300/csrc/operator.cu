// Fused element-centric kernels for f(U) = M^{-1} L_h(U) (Sec. 3.1, Eq.
// convDiscr; Sec. 3.2, Eq. ode) and its directional derivative J(U) dU
// (the Jacobian-vector product of the Jacobian-free Newton-Krylov solver,
// Sec. 3.2).
//
// One CTA owns EPB consecutive elements (a contiguous slab of U), computes
// their volume integrals (Eq. elementint) with sum factorisation, then
// visits their 2*dim faces: it evaluates its own trace and the neighbour's
// trace (read from global memory, mostly L2 hits), forms the face fluxes of
// Eq. surfaceint at every face point, tests them against its own basis and
// accumulates.  Every interior face is thus evaluated by both adjacent
// elements; in exchange there are no atomics, no face buffer in HBM and a
// single pass over U and out.
//
// The kernel has three modes.  MODE 0 applies the operator to U.  MODE 1
// (JVP) carries the primal field U and a tangent dU through the same
// contraction passes and evaluates the linearised pointwise fluxes (the
// contractions are linear, so only the pointwise terms change).  MODE 2
// (VJP) carries U and the cotangent mu: interpolating mu with the forward
// operators gives exactly the transposed test operators' inputs, the
// pointwise maps are replaced by their adjoints, and testing the adjoints
// gives (dR/dU)^T mu.  Each element gathers the adjoint contributions of its
// own faces from both traces, so the transposed face scatter needs no atomics.
//
// The CDG2 lifting r_e on K^- is taken in closed form: on a Cartesian cell
// with the orthonormal tensor basis and a Q_k trace Delta,
//     r_e([U]) . n^- = -(k+1)^2 |e| / (2 |K^-|) Delta   on e,
// because the lifting solve only needs the mass-inverse projection of Delta
// onto the trace space of K^- (exact for a Q_k trace with k+2 Gauss points)
// times sum_m psi_m(1)^2 = (k+1)^2 in the normal direction.
#include <cstdio>

#include <type_traits>

#include "elem_common.cuh"
#include "physics.cuh"

namespace cdg2 {

template <int D, int K, int F>
struct OpPlan {
    using S = Shape<D, K>;
    static constexpr int NT = 128;
    static constexpr int EPB = D == 3 ? (K == 1 ? 4 : (K == 2 ? 2 : 1)) : (F == 1 ? (K == 1 ? 16 : 8) : (K == 1 ? 8 : 4));
    static constexpr int NB1 = S::NB1, NQ1 = S::NQ1;
    // volume phase: per-field sizes for the whole CTA (all F input fields)
    static constexpr int XSZ = F * EPB * NS * NQ1 * ipow(NB1, D - 1);
    static constexpr int YSZ = D == 3 ? F * EPB * NS * NQ1 * NQ1 * NB1 : 0;
    static constexpr int QSZ = F * EPB * NS * S::NQ;
    // 3D: the point values Q overlay X (dead once Y is formed): Y | X / Q
    static constexpr int VOL = D == 3 ? 3 * YSZ + cmax(2 * XSZ, (D + 1) * QSZ) : (D + 1) * QSZ + 2 * XSZ;
    // face phase (the two faces normal to one axis)
    static constexpr int FC = F * EPB * 2 * 4 * NS * S::NBT;
    static constexpr int FT = D == 3 ? F * EPB * 2 * 4 * NS * NQ1 * NB1 : 0;
    static constexpr int FP = F * EPB * 2 * 4 * NS * S::NQT;
    static constexpr int FS = EPB * 2 * 2 * NS * S::NQT;
    static constexpr int TS1 = D == 3 ? EPB * 2 * 2 * NS * NB1 * NQ1 : 0;
    static constexpr int TS = EPB * 2 * 2 * NS * S::NBT;
    static constexpr int FACE = FC + FT + FP + FS + TS1 + TS;
    static constexpr int WORK = cmax(VOL, FACE);
    static constexpr int UR = EPB * NS * S::NB;   // one field's slab
    template <typename T>
    static constexpr size_t tab_bytes() {
        return (sizeof(STab<K, T>) + 15) / 16 * 16;
    }
    template <typename T>
    static constexpr size_t smem_bytes() {
        return tab_bytes<T>() + sizeof(T) * (size_t)((F + 1) * UR + WORK);
    }
};

// Arguments of one launch.
template <typename T>
struct OpArgs {
    const T* U[2];      // U, and the tangent dU when F = 2
    T* out;
    int flags;
    double t;
    int has_dtheta;
    double dtheta[8];   // tangent of (d1, d2, gamma, alpha1, alpha2, f1, k_ox, beta1)
    double* theta_part; // VJP: per-CTA partial sums of (df/dtheta)^T lambda, [gridDim.x][8], or null
    double alpha, beta; // JVP epilogue: out = alpha dU + beta J dU (0, 1 for the plain JVP)
    const double* pscale; // JVP: optional [6][n_basis] scale of the tangent (right preconditioner), or null
    CoefT<T> c;           // coefficients and geometry in the kernel's precision
    T* fbuf;              // face-once path: tested face fluxes, per axis at fb_off[axis], or null
    long long fb_off[3];
    int* domain;          // domain status word of this launch, or null: the mesh's
};

constexpr int MODE_APPLY = 0, MODE_JVP = 1, MODE_VJP = 2;
constexpr int fields_of(int mode) { return mode == MODE_APPLY ? 1 : 2; }

// The input field fi without a run-time index into the kernel arguments (an
// indexed parameter access goes through slow indexed constant loads).
template <typename T>
__device__ __forceinline__ const T* field(const OpArgs<T>& a, int fi) {
    return fi == 0 ? a.U[0] : a.U[1];
}

// ---------------------------------------------------------------------------
// The two faces normal to axis A of every element of the CTA
// ---------------------------------------------------------------------------
template <int D, int K, int MODE, int A, typename T>
__device__ __forceinline__ void op_faces(const Geo& g, const STab<K, T>& tb, const CoefT<T>& c, const OpArgs<T>& args,
                                         const T* sU, T* sR, T* W, long long e0, long long (*nbr)[2],
                                         T th[8], const T* ps) {
    constexpr int F = fields_of(MODE);
    using P = OpPlan<D, K, F>;
    using S = Shape<D, K>;
    constexpr int EPB = P::EPB, NB = S::NB, NB1 = S::NB1, NQ1 = S::NQ1, NBT = S::NBT, NQT = S::NQT;
    T* FC = W;
    T* FT = FC + P::FC;
    T* FP = FT + P::FT;
    T* FS = FP + P::FP;
    T* TS1 = FS + P::FS;
    T* TS = TS1 + P::TS1;
    const T invh = c.invh[A];

    if (threadIdx.x < EPB * 2) {
        const int e = threadIdx.x / 2, f = threadIdx.x % 2;
        const long long ge = e0 + e;
        nbr[e][f] = ge < g.E ? neighbour(g, ge, A, f) : -1;
    }
    __syncthreads();

    // Normal contraction.  Fields per (input field, face, species, tangential mode):
    //   0: own trace at xi_A = f,  1: jump Delta = U^- - U^+,
    //   2: own normal derivative,  3: neighbour normal derivative (at xi_A = 1 - f).
    // The jump is formed difference-first, (U^-_0 - U^+_0) + sum_{m>0} (psi_m(1) U^-_m - psi_m(0) U^+_m),
    // so the rounding error scales with Delta rather than with U (this matters in FP32).
    for (int idx = threadIdx.x; idx < F * EPB * 2 * NS * NBT; idx += blockDim.x) {
        const int t = idx % NBT;
        const int s = (idx / NBT) % NS;
        const int f = (idx / (NBT * NS)) % 2;
        const int e = (idx / (NBT * NS * 2)) % EPB;
        const int fi = idx / (NBT * NS * 2 * EPB);
        const int b0 = t % NB1, b1 = t / NB1;
        const T* own = sU + fi * P::UR + (e * NS + s) * NB;
        T uo = 0, dO = 0, del = 0, dn = 0;
#pragma unroll
        for (int m = 0; m < NB1; ++m) {
            const T v = own[coef_index<D, K, A>(m, b0, b1)];
            uo = fma(tb.e[f][m], v, uo);
            dO = fma(tb.dh[A][f][m], v, dO);
        }
        const long long nb = nbr[e][f];
        if (nb >= 0) {
            const T* nbg = field(args, fi) + (nb * NS + s) * NB;
            T nbv[NB1];   // the neighbour's coefficients along the normal line (tangent: preconditioned)
            const bool scaled = MODE != MODE_APPLY && fi == 1 && ps != nullptr;
#pragma unroll
            for (int m = 0; m < NB1; ++m) {
                const int ci = coef_index<D, K, A>(m, b0, b1);
                nbv[m] = scaled ? nbg[ci] * ps[s * NB + ci] : nbg[ci];
            }
            T ov[NB1];
#pragma unroll
            for (int m = 0; m < NB1; ++m) ov[m] = own[coef_index<D, K, A>(m, b0, b1)];
            const T* um = f ? ov : nbv;     // K^- coefficients
            const T* up = f ? nbv : ov;     // K^+ coefficients
            del = um[0] - up[0];
#pragma unroll
            for (int m = 1; m < NB1; ++m) {
                del = fma(tb.e[1][m], um[m], del);
                del = fma(-tb.e[0][m], up[m], del);
            }
#pragma unroll
            for (int m = 0; m < NB1; ++m) dn = fma(tb.dh[A][1 - f][m], nbv[m], dn);
        }
        T* o = FC + (((fi * EPB + e) * 2 + f) * 4) * NS * NBT + s * NBT + t;
        o[0 * NS * NBT] = uo;
        o[1 * NS * NBT] = del;
        o[2 * NS * NBT] = dO;
        o[3 * NS * NBT] = dn;
    }
    __syncthreads();

    // tangential interpolation to the face points
    if constexpr (D == 2) {
        sf_sym<0, NB1, 1, 1, NQ1, false, K + 1, false, 1, 1>(FC, &tb.B[0][0], nullptr, nullptr, NBT, FP, NQT,
                                                         F * EPB * 2 * 4 * NS);
    } else {
        sf_sym<0, NB1, NB1, 1, NQ1, false, K + 1, false, 1, 1>(FC, &tb.B[0][0], nullptr, nullptr, NBT, FT, NQ1 * NB1,
                                                           F * EPB * 2 * 4 * NS);
        __syncthreads();
        sf_sym<1, NQ1, NB1, 1, NQ1, false, K + 1, false, 1, 1>(FT, &tb.B[0][0], nullptr, nullptr, NQ1 * NB1, FP, NQT,
                                                           F * EPB * 2 * 4 * NS);
    }
    __syncthreads();

    // pointwise fluxes, weighted: W_p = w_p |e|, |e| = |K| / h_A
    const T pen = c.pen_c * T((K + 1) * (K + 1)) * invh;
    for (int idx = threadIdx.x; idx < EPB * 2 * NQT; idx += blockDim.x) {
        const int p = idx % NQT;
        const int f = (idx / NQT) % 2;
        const int e = idx / (NQT * 2);
        T uo[NS], del[NS], dO[NS], dn[NS], sig[NS], tau[NS];
        {
            const T* base = FP + ((e * 2 + f) * 4) * NS * NQT + p;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                uo[s] = base[(0 * NS + s) * NQT];
                del[s] = base[(1 * NS + s) * NQT];
                dO[s] = base[(2 * NS + s) * NQT];
                dn[s] = base[(3 * NS + s) * NQT];
            }
        }
        const int p0 = p % NQ1, p1 = p / NQ1;
        T wp = tb.w[p0];
        if constexpr (D == 3) wp *= tb.w[p1];
        // forward modes: the residual is accumulated divided by |K| (see the kernel's store)
        const T Wp = MODE == MODE_VJP ? wp * c.vol * invh : wp * invh;
        const long long nb = nbr[e][f];
        if (nb >= 0) {
            T uN[NS];   // neighbour trace recovered from the jump
#pragma unroll
            for (int s = 0; s < NS; ++s) uN[s] = f == 1 ? uo[s] - del[s] : uo[s] + del[s];
            if constexpr (MODE == MODE_APPLY) {
                if (f == 1)
                    face_point<T>(c, pen, uo, dO, uN, dn, del, sig, tau);
                else
                    face_point<T>(c, pen, uN, dn, uo, dO, del, sig, tau);
            } else if constexpr (MODE == MODE_VJP) {
                // cotangents of sigma and tau from the traces of mu (second field)
                T sb[NS], tbr[NS];
                const T* base = FP + (((EPB + e) * 2 + f) * 4) * NS * NQT + p;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    sb[s] = Wp * base[(1 * NS + s) * NQT];
                    tbr[s] = Wp * (base[(2 * NS + s) * NQT] + base[(3 * NS + s) * NQT]);
                }
                if (f == 1)
                    face_point_adj<T>(c, pen, true, uo, dO, uN, dn, del, sb, tbr, sig, tau);
                else
                    face_point_adj<T>(c, pen, false, uN, dn, uo, dO, del, sb, tbr, sig, tau);
            } else {
                T tuo[NS], tdel[NS], tdO[NS], tdn[NS], tuN[NS];
                const T* base = FP + (((EPB + e) * 2 + f) * 4) * NS * NQT + p;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    tuo[s] = base[(0 * NS + s) * NQT];
                    tdel[s] = base[(1 * NS + s) * NQT];
                    tdO[s] = base[(2 * NS + s) * NQT];
                    tdn[s] = base[(3 * NS + s) * NQT];
                    tuN[s] = f == 1 ? tuo[s] - tdel[s] : tuo[s] + tdel[s];
                }
                if (f == 1)
                    face_point_lin<T>(c, pen, uo, dO, uN, dn, del, tuo, tdO, tuN, tdn, tdel, sig, tau);
                else
                    face_point_lin<T>(c, pen, uN, dn, uo, dO, del, tuN, tdn, tuo, tdO, tdel, sig, tau);
            }
            if constexpr (MODE != MODE_VJP) {
                const T sgn = f == 1 ? T(1) : T(-1);
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    sig[s] = sgn * Wp * sig[s];
                    tau[s] = Wp * tau[s];
                }
            }
        } else {
            if (A == 1) {
                const long long ge = e0 + e;
                const T x = T((ge % g.n[0]) * g.h[0]) + T(g.h[0]) * tb.xi[p0];
                if constexpr (MODE == MODE_APPLY) {
                    boundary_point<T>(c, f, x, g, uo, sig, c.beta1, true);
                } else if constexpr (MODE == MODE_JVP) {
                    // H' = 0: only a tangent of beta1 moves the boundary data
                    boundary_point<T>(c, f, x, g, uo, sig, c.dth[7], false);
                } else {
                    // H' = 0: the boundary data do not depend on U; their beta1
                    // derivative, tested with mu's own trace, feeds the theta gradient
                    boundary_point<T>(c, f, x, g, uo, sig, T(1), false);
                    const T* base = FP + (((EPB + e) * 2 + f) * 4) * NS * NQT + p;
                    th[7] += Wp * sig[0] * base[0];
#pragma unroll
                    for (int s = 0; s < NS; ++s) sig[s] = T(0);
                }
            } else {
#pragma unroll
                for (int s = 0; s < NS; ++s) sig[s] = T(0);
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                sig[s] = Wp * sig[s];
                tau[s] = T(0);
            }
        }
        T* o = FS + ((e * 2 + f) * 2) * NS * NQT + p;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            o[(0 * NS + s) * NQT] = sig[s];
            o[(1 * NS + s) * NQT] = tau[s];
        }
    }
    __syncthreads();

    // tangential test against the own basis
    if constexpr (D == 2) {
        sf_sym<0, NQ1, 1, 1, NB1, true, K + 1, false, 1, 1>(FS, &tb.B[0][0], nullptr, nullptr, NQT, TS, NBT,
                                                        EPB * 2 * 2 * NS);
    } else {
        sf_sym<0, NQ1, NQ1, 1, NB1, true, K + 1, false, 1, 1>(FS, &tb.B[0][0], nullptr, nullptr, NQT, TS1, NB1 * NQ1,
                                                          EPB * 2 * 2 * NS);
        __syncthreads();
        sf_sym<1, NB1, NQ1, 1, NB1, true, K + 1, false, 1, 1>(TS1, &tb.B[0][0], nullptr, nullptr, NB1 * NQ1, TS, NBT,
                                                          EPB * 2 * 2 * NS);
    }
    __syncthreads();

    // normal expansion: phi_i = psi_{i_A}(f) (tangential part), d_A phi_i = psi'_{i_A}(f) / h_A (...)
    for (int idx = threadIdx.x; idx < EPB * NS * NB; idx += blockDim.x) {
        const int i = idx % NB;
        const int es = idx / NB;          // e * NS + s
        const int e = es / NS, s = es % NS;
        int m, t;
        if constexpr (D == 2) {
            m = A == 0 ? i % NB1 : i / NB1;
            t = A == 0 ? i / NB1 : i % NB1;
        } else {
            if constexpr (A == 0) {
                m = i % NB1;
                t = i / NB1;
            } else if constexpr (A == 1) {
                m = (i / NB1) % NB1;
                t = i % NB1 + NB1 * (i / (NB1 * NB1));
            } else {
                m = i / (NB1 * NB1);
                t = i % (NB1 * NB1);
            }
        }
        T acc = sR[idx];
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const T* ts = TS + ((e * 2 + f) * 2) * NS * NBT + s * NBT + t;
            acc = fma(tb.e[f][m], ts[0], acc);
            acc = fma(tb.dh[A][f][m], ts[NS * NBT], acc);
        }
        sR[idx] = acc;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Face-once path (apply and JVP): every face is evaluated by one CTA of the
// face kernel, which writes its tested fluxes; the element kernel then adds
// them to both adjacent cells with the normal expansion.  This halves the
// face work of the fused path (where both cells evaluate every face); the
// face buffer costs HBM traffic, which the FP64 path has in abundance.
// Faces of axis A: id < E is the high face of cell id (interior, or the
// high boundary); id >= E are the low-boundary faces of the first cell
// layer (non-periodic axes only).  Stored per face: the tangential tests of
// sigma and tau, [2][6][n_bt].  A low-boundary face stores -sigma so that
// the element's low-face expansion (-psi(0) sigma + psi'(0)/h tau) applies.
// ---------------------------------------------------------------------------
template <int D, int K, int F>
struct FacePlan {
    using S = Shape<D, K>;
    static constexpr int NT = 128;
    static constexpr int FPB = D == 3 ? (K == 1 ? 8 : (K == 2 ? 4 : 2)) : (F == 1 ? (K == 1 ? 16 : 8) : (K == 1 ? 8 : 4));
    static constexpr int NB1 = S::NB1, NQ1 = S::NQ1;
    static constexpr int UB = FPB * NS * S::NB;                       // one side, one field
    static constexpr int FC = F * FPB * 4 * NS * S::NBT;
    static constexpr int FT = D == 3 ? F * FPB * 4 * NS * NQ1 * NB1 : 0;
    static constexpr int FP = F * FPB * 4 * NS * S::NQT;
    static constexpr int FS = FPB * 2 * NS * S::NQT;
    static constexpr int TS1 = D == 3 ? FPB * 2 * NS * NB1 * NQ1 : 0;
    static constexpr int TS = FPB * 2 * NS * S::NBT;
    template <typename T>
    static constexpr size_t smem_bytes() {
        return (sizeof(STab<K, T>) + 15) / 16 * 16 + sizeof(T) * (size_t)(2 * F * UB + FC + FT + FP + FS + TS1 + TS);
    }
};

__host__ __device__ inline long long faces_of_axis(const Geo& g, int a) {
    return g.E + (g.periodic[a] ? 0 : g.E / g.n[a]);
}

// Index of the low-boundary face of a cell in the first layer of axis a.
__device__ __forceinline__ long long low_layer_index(const Geo& g, long long e, int a) {
    int c[3];
    cell_coords(g, e, c);
    if (a == 0) return c[1] + (long long)g.n[1] * c[2];
    if (a == 1) return c[0] + (long long)g.n[0] * c[2];
    return c[0] + (long long)g.n[0] * c[1];
}

template <int D, int K, int MODE, int A, typename T>
__global__ void __launch_bounds__(128) face_kernel(const Geo g, const TabP<T> tab, const OpArgs<T> args) {
    constexpr int F = fields_of(MODE);
    using P = FacePlan<D, K, F>;
    using S = Shape<D, K>;
    constexpr int FPB = P::FPB, NB = S::NB, NB1 = S::NB1, NQ1 = S::NQ1, NBT = S::NBT, NQT = S::NQT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    STab<K, T>& tb = *reinterpret_cast<STab<K, T>*>(smem_raw);
    T* sM = reinterpret_cast<T*>(smem_raw + (sizeof(STab<K, T>) + 15) / 16 * 16);   // [F][FPB][NS][NB] minus cells
    T* sP = sM + F * P::UB;                                                       // plus cells
    T* FC = sP + F * P::UB;
    T* FT = FC + P::FC;
    T* FPt = FT + P::FT;
    T* FS = FPt + P::FP;
    T* TS1 = FS + P::FS;
    T* TS = TS1 + P::TS1;
    __shared__ long long cm[FPB], cp[FPB];   // minus / plus cell (-1: none)
    __shared__ int kind[FPB];                // -1 unused, 0 interior, 1 high boundary, 2 low boundary
    __shared__ int any_boundary;             // a boundary face in this CTA: no modal shortcut
    __shared__ T psT[MODE == MODE_JVP ? NS * NB : 1];
    const CoefT<T>& c = args.c;
    const long long nf = faces_of_axis(g, A);
    const long long f0 = (long long)blockIdx.x * FPB;

    load_tab<K, T>(tb, tab);
    const T* ps = nullptr;
    if constexpr (MODE == MODE_JVP) {
        if (args.pscale) {
            for (int i = threadIdx.x; i < NS * NB; i += blockDim.x) psT[i] = T(args.pscale[i]);
            ps = psT;
        }
    }
    if (threadIdx.x < FPB) {
        const long long fid = f0 + threadIdx.x;
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
        cm[threadIdx.x] = em;
        cp[threadIdx.x] = ep;
        kind[threadIdx.x] = kd;
    }
    if (threadIdx.x == 0) any_boundary = 0;
    __syncthreads();
    if (threadIdx.x < FPB && kind[threadIdx.x] > 0) any_boundary = 1;
    // coalesced loads of both cells of every face (the tangent pre-scaled), a
    // batch of independent loads per thread in flight at once
    {
        constexpr int TOT = 2 * F * P::UB, BATCH = 8;
        for (int i0 = threadIdx.x; i0 < TOT; i0 += BATCH * blockDim.x) {
            T v[BATCH];
#pragma unroll
            for (int b = 0; b < BATCH; ++b) {
                const int i = i0 + b * blockDim.x;
                v[b] = T(0);
                if (i < TOT) {
                    const int side = i / (F * P::UB);
                    const int r0 = i % (F * P::UB);
                    const int fi = r0 / P::UB, r = r0 % P::UB;
                    const int j = r / (NS * NB), q = r % (NS * NB);
                    const long long cell = side ? cp[j] : cm[j];
                    if (cell >= 0) v[b] = field(args, fi)[cell * NS * NB + q];
                }
            }
#pragma unroll
            for (int b = 0; b < BATCH; ++b) {
                const int i = i0 + b * blockDim.x;
                if (i < TOT) {
                    const int side = i / (F * P::UB);
                    const int r0 = i % (F * P::UB);
                    const int fi = r0 / P::UB, r = r0 % P::UB;
                    const int q = r % (NS * NB);
                    T w = v[b];
                    if (MODE == MODE_JVP && fi == 1 && ps) w *= ps[q];
                    (side ? sP : sM)[r0] = w;
                }
            }
        }
    }
    __syncthreads();

    const T invh = c.invh[A];
    // normal contraction: 0 the owning trace (K^- at xi = 1, or K^+ at xi = 0 on a
    // low boundary), 1 the jump (difference-first), 2 d_n U^-, 3 d_n U^+
    for (int idx = threadIdx.x; idx < F * FPB * NS * NBT; idx += blockDim.x) {
        const int t = idx % NBT;
        const int s = (idx / NBT) % NS;
        const int j = (idx / (NBT * NS)) % FPB;
        const int fi = idx / (NBT * NS * FPB);
        const int b0 = t % NB1, b1 = t / NB1;
        const T* um = sM + (fi * FPB + j) * NS * NB + s * NB;
        const T* up = sP + (fi * FPB + j) * NS * NB + s * NB;
        T vm[NB1], vp[NB1];
#pragma unroll
        for (int m = 0; m < NB1; ++m) {
            vm[m] = um[coef_index<D, K, A>(m, b0, b1)];
            vp[m] = up[coef_index<D, K, A>(m, b0, b1)];
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
        T* o = FC + ((fi * FPB + j) * 4) * NS * NBT + s * NBT + t;
        o[0 * NS * NBT] = uo;
        o[1 * NS * NBT] = del;
        o[2 * NS * NBT] = dm;
        o[3 * NS * NBT] = dp;
    }
    __syncthreads();
    // Interior faces: the fluxes of n3, c1, c2, c3 are purely diffusive and
    // linear, and with the orthonormal tangential basis and exact face
    // quadrature their tested fluxes follow from the normal contraction in
    // modal form (below); only n1, n2, c1, c3 go to the face points.
    const bool modal = any_boundary == 0;
    if (modal) {
        if constexpr (D == 2) {
            sf_sym<0, NB1, 1, 1, NQ1, false, K + 1, false, 1, 1, T, 5>(FC, &tb.B[0][0], nullptr, nullptr, NBT, FPt,
                                                                     NQT, F * FPB * 4 * SpeciesSet<5>::N);
        } else {
            sf_sym<0, NB1, NB1, 1, NQ1, false, K + 1, false, 1, 1, T, 5>(FC, &tb.B[0][0], nullptr, nullptr, NBT, FT,
                                                                       NQ1 * NB1, F * FPB * 4 * SpeciesSet<5>::N);
            __syncthreads();
            sf_sym<1, NQ1, NB1, 1, NQ1, false, K + 1, false, 1, 1, T, 5>(FT, &tb.B[0][0], nullptr, nullptr, NQ1 * NB1,
                                                                       FPt, NQT, F * FPB * 4 * SpeciesSet<5>::N);
        }
    } else {
        if constexpr (D == 2) {
            sf_sym<0, NB1, 1, 1, NQ1, false, K + 1, false, 1, 1>(FC, &tb.B[0][0], nullptr, nullptr, NBT, FPt, NQT,
                                                             F * FPB * 4 * NS);
        } else {
            sf_sym<0, NB1, NB1, 1, NQ1, false, K + 1, false, 1, 1>(FC, &tb.B[0][0], nullptr, nullptr, NBT, FT,
                                                               NQ1 * NB1, F * FPB * 4 * NS);
            __syncthreads();
            sf_sym<1, NQ1, NB1, 1, NQ1, false, K + 1, false, 1, 1>(FT, &tb.B[0][0], nullptr, nullptr, NQ1 * NB1, FPt,
                                                               NQT, F * FPB * 4 * NS);
        }
    }
    __syncthreads();

    const T pen = c.pen_c * T((K + 1) * (K + 1)) * invh;
    for (int idx = threadIdx.x; idx < FPB * NQT; idx += blockDim.x) {
        const int p = idx % NQT, j = idx / NQT;
        const int kd = kind[j];
        T sig[NS], tau[NS];
        const int p0 = p % NQ1, p1 = p / NQ1;
        T wp = tb.w[p0];
        if constexpr (D == 3) wp *= tb.w[p1];
        const T Wp = wp * invh;   // the element kernel accumulates the residual divided by |K|
        T uo[NS], del[NS], dm[NS], dp[NS];
        {
            const T* base = FPt + (j * 4) * NS * NQT + p;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                uo[s] = base[(0 * NS + s) * NQT];
                del[s] = base[(1 * NS + s) * NQT];
                dm[s] = base[(2 * NS + s) * NQT];
                dp[s] = base[(3 * NS + s) * NQT];
            }
        }
        if (kd == 0) {
            T uP[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) uP[s] = uo[s] - del[s];
            if constexpr (MODE == MODE_APPLY) {
                face_point<T>(c, pen, uo, dm, uP, dp, del, sig, tau);
            } else {
                T tuo[NS], tdel[NS], tdm[NS], tdp[NS], tuP[NS];
                const T* base = FPt + ((FPB + j) * 4) * NS * NQT + p;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    tuo[s] = base[(0 * NS + s) * NQT];
                    tdel[s] = base[(1 * NS + s) * NQT];
                    tdm[s] = base[(2 * NS + s) * NQT];
                    tdp[s] = base[(3 * NS + s) * NQT];
                    tuP[s] = tuo[s] - tdel[s];
                }
                face_point_lin<T>(c, pen, uo, dm, uP, dp, del, tuo, tdm, tuP, tdp, tdel, sig, tau);
            }
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                sig[s] = Wp * sig[s];
                tau[s] = Wp * tau[s];
            }
        } else {
#pragma unroll
            for (int s = 0; s < NS; ++s) {
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
                for (int s = 0; s < NS; ++s) sig[s] = sg * sig[s];
            }
        }
        T* o = FS + (j * 2) * NS * NQT + p;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            o[(0 * NS + s) * NQT] = sig[s];
            o[(1 * NS + s) * NQT] = tau[s];
        }
    }
    __syncthreads();
    if (modal) {
        // n1, n2 through the face points
        if constexpr (D == 2) {
            sf_sym<0, NQ1, 1, 1, NB1, true, K + 1, false, 1, 1, T, 2>(FS, &tb.B[0][0], nullptr, nullptr, NQT, TS, NBT,
                                                                    FPB * 2 * SpeciesSet<2>::N);
        } else {
            sf_sym<0, NQ1, NQ1, 1, NB1, true, K + 1, false, 1, 1, T, 2>(FS, &tb.B[0][0], nullptr, nullptr, NQT, TS1,
                                                                      NB1 * NQ1, FPB * 2 * SpeciesSet<2>::N);
            __syncthreads();
            sf_sym<1, NB1, NQ1, 1, NB1, true, K + 1, false, 1, 1, T, 2>(TS1, &tb.B[0][0], nullptr, nullptr, NB1 * NQ1,
                                                                      TS, NBT, FPB * 2 * SpeciesSet<2>::N);
        }
        // n3, c1, c2, c3 in modal form: sigma_t = A (d_n U^-_t + d_n U^+_t) / 2 - pen A Delta_t,
        // tau_t = A Delta_t / 2 (of the tangent in the JVP), weighted like the point values (1 / h_A)
        constexpr int fl = F - 1;   // the field whose flux is tested
        for (int idx = threadIdx.x; idx < FPB * SpeciesSet<3>::N * NBT; idx += blockDim.x) {
            const int t = idx % NBT, ss = (idx / NBT) % SpeciesSet<3>::N, j = idx / (NBT * SpeciesSet<3>::N);
            const int s = SpeciesSet<3>::s(ss);
            const T* f = FC + ((fl * FPB + j) * 4) * NS * NBT + s * NBT + t;
            const T del = f[1 * NS * NBT], dm = f[2 * NS * NBT], dp = f[3 * NS * NBT];
            const T A_s = c.A[s];
            T* o = TS + (j * 2) * NS * NBT + s * NBT + t;
            o[0] = kind[j] == 0 ? invh * A_s * (T(0.5) * (dm + dp) - pen * del) : T(0);
            o[NS * NBT] = kind[j] == 0 ? invh * T(0.5) * A_s * del : T(0);
        }
    } else {
        if constexpr (D == 2) {
            sf_sym<0, NQ1, 1, 1, NB1, true, K + 1, false, 1, 1>(FS, &tb.B[0][0], nullptr, nullptr, NQT, TS, NBT,
                                                            FPB * 2 * NS);
        } else {
            sf_sym<0, NQ1, NQ1, 1, NB1, true, K + 1, false, 1, 1>(FS, &tb.B[0][0], nullptr, nullptr, NQT, TS1,
                                                              NB1 * NQ1, FPB * 2 * NS);
            __syncthreads();
            sf_sym<1, NB1, NQ1, 1, NB1, true, K + 1, false, 1, 1>(TS1, &tb.B[0][0], nullptr, nullptr, NB1 * NQ1, TS,
                                                              NBT, FPB * 2 * NS);
        }
    }
    __syncthreads();
    // coalesced store of the faces' tested fluxes
    T* dst = args.fbuf + args.fb_off[A];
    for (int i = threadIdx.x; i < P::TS; i += blockDim.x) {
        const long long fid = f0 + i / (2 * NS * NBT);
        if (fid < nf) dst[f0 * 2 * NS * NBT + i] = TS[i];
    }
}

// Element side of the face-once path: add the tested fluxes of the two faces
// normal to axis A to the residual of every cell of the CTA.
template <int D, int K, int A, typename T>
__device__ __forceinline__ void faces_expand(const Geo& g, const STab<K, T>& tb, const CoefT<T>& c,
                                             const T* __restrict__ fb, T* sR, long long e0, int epb,
                                             long long (*fid)[2]) {
    using S = Shape<D, K>;
    constexpr int NB = S::NB, NB1 = S::NB1, NBT = S::NBT;
    if (threadIdx.x < epb) {
        const long long ge = e0 + threadIdx.x;
        long long hi = -1, lo = -1;
        if (ge < g.E) {
            hi = ge;
            const long long nb = neighbour(g, ge, A, 0);
            lo = nb >= 0 ? nb : g.E + low_layer_index(g, ge, A);
        }
        fid[threadIdx.x][0] = lo;
        fid[threadIdx.x][1] = hi;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < epb * NS * NB; idx += blockDim.x) {
        const int i = idx % NB;
        const int es = idx / NB;
        const int e = es / NS, s = es % NS;
        if (fid[e][1] < 0) continue;
        int m, t;
        if constexpr (D == 2) {
            m = A == 0 ? i % NB1 : i / NB1;
            t = A == 0 ? i / NB1 : i % NB1;
        } else {
            if constexpr (A == 0) {
                m = i % NB1;
                t = i / NB1;
            } else if constexpr (A == 1) {
                m = (i / NB1) % NB1;
                t = i % NB1 + NB1 * (i / (NB1 * NB1));
            } else {
                m = i / (NB1 * NB1);
                t = i % (NB1 * NB1);
            }
        }
        const T* lo = fb + fid[e][0] * 2 * NS * NBT + s * NBT + t;
        const T* hi = fb + fid[e][1] * 2 * NS * NBT + s * NBT + t;
        T acc = sR[idx];
        acc = fma(-tb.e[0][m], lo[0], acc);
        acc = fma(tb.dh[A][0][m], lo[NS * NBT], acc);
        acc = fma(tb.e[1][m], hi[0], acc);
        acc = fma(tb.dh[A][1][m], hi[NS * NBT], acc);
        sR[idx] = acc;
    }
    __syncthreads();
}

}  // namespace cdg2

#include "face3.cuh"
#include "tc_elem.cuh"

namespace cdg2 {

template <int D, int K, int MODE, typename T>
__global__ void __launch_bounds__(128) op_kernel(const Geo g, const TabP<T> tab, const OpArgs<T> args) {
    constexpr int F = fields_of(MODE);
    using P = OpPlan<D, K, F>;
    using S = Shape<D, K>;
    constexpr int EPB = P::EPB, NB = S::NB, NQ = S::NQ, NB1 = S::NB1, NQ1 = S::NQ1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    STab<K, T>& tb = *reinterpret_cast<STab<K, T>*>(smem_raw);
    T* sU = reinterpret_cast<T*>(smem_raw + P::template tab_bytes<T>());   // F slabs
    T* sR = sU + F * P::UR;
    T* W = sR + P::UR;
    __shared__ long long nbr[EPB][2];
    __shared__ T psT[MODE != MODE_APPLY ? NS * NB : 1];   // tangent/cotangent pre-scale in the kernel's precision

    const long long e0 = (long long)blockIdx.x * EPB;
    T th[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // VJP: this thread's theta cotangent partials
    load_tab<K, T>(tb, tab);
    const T* ps = nullptr;
    if constexpr (MODE != MODE_APPLY) {
        if (args.pscale) {
            for (int i = threadIdx.x; i < NS * NB; i += blockDim.x) psT[i] = T(args.pscale[i]);
            ps = psT;
        }
    }
    __syncthreads();
    const CoefT<T>& c = args.c;
    {
        constexpr int TOT = F * P::UR, BATCH = 8;
        for (int i0 = threadIdx.x; i0 < TOT; i0 += BATCH * blockDim.x) {
            T v[BATCH];
#pragma unroll
            for (int b = 0; b < BATCH; ++b) {
                const int i = i0 + b * blockDim.x;
                v[b] = T(0);
                if (i < TOT) {
                    const int fi = i / P::UR, r = i % P::UR;
                    if (e0 + r / (NS * NB) < g.E) v[b] = field(args, fi)[e0 * NS * NB + r];
                }
            }
#pragma unroll
            for (int b = 0; b < BATCH; ++b) {
                const int i = i0 + b * blockDim.x;
                if (i < TOT) {
                    const int fi = i / P::UR, r = i % P::UR;
                    T w = v[b];
                    if (MODE != MODE_APPLY && fi == 1 && ps) w *= ps[r % (NS * NB)];
                    sU[i] = w;
                }
            }
        }
    }
    __syncthreads();

    // ---- volume: U, grad U (of every input field) at the Gauss points ----
    // 2D: X0 | X1 | Q.  3D: Y | X0 X1, with Q over X (X is dead once Y is
    // formed, and Q once the test's first pass has read it).
    T* Y = D == 3 ? W : W + 2 * P::XSZ;
    T* X0 = D == 3 ? W + 3 * P::YSZ : W;
    T* X1 = X0 + P::XSZ;
    T* Q = D == 3 ? X0 : W + 2 * P::XSZ;   // D + 1 slots of F*EPB*NS tensors: u, g_0, .., g_{D-1}
    // FP64 forward modes apply the diffusion of n2..c3 in modal form (after the
    // test): gradients are interpolated for n1, c1, c3 only (GS), values for
    // all.  (It saves FP64 pipe work; in FP32 the extra loop costs more than
    // the passes it saves: 3D Q2 JVP 2.16 -> 2.35 ms measured.)
    constexpr bool MODAL = MODE != MODE_VJP && sizeof(T) == 8;
    constexpr int GS = MODAL ? 1 : 0;
    const int nt = F * EPB * NS;
    const int ng = F * EPB * SpeciesSet<GS>::N;
    if constexpr (D == 2) {
        sf_sym<0, NB1, NB1, 1, NQ1, false, K + 1, false, 1, 1>(sU, &tb.B[0][0], nullptr, nullptr, NB, X0, NQ1 * NB1, nt);
        sf_sym<0, NB1, NB1, 1, NQ1, false, K + 1, false, -1, 1, T, GS>(sU, &tb.Dh[0][0][0], nullptr, nullptr, NB, X1,
                                                                      NQ1 * NB1, ng);
        __syncthreads();
        sf_sym<1, NQ1, NB1, 1, NQ1, false, K + 1, false, 1, 1>(X0, &tb.B[0][0], nullptr, nullptr, NQ1 * NB1, Q, NQ, nt);
        sf_sym<1, NQ1, NB1, 1, NQ1, false, K + 1, false, 1, 1, T, GS>(X1, &tb.B[0][0], nullptr, nullptr, NQ1 * NB1,
                                                                     Q + P::QSZ, NQ, ng);
        sf_sym<1, NQ1, NB1, 1, NQ1, false, K + 1, false, -1, 1, T, GS>(X0, &tb.Dh[1][0][0], nullptr, nullptr, NQ1 * NB1,
                                                                      Q + 2 * P::QSZ, NQ, ng);
    } else {
        constexpr int XS = NQ1 * NB1 * NB1, YS = NQ1 * NQ1 * NB1;
        sf_sym<0, NB1, NB1, NB1, NQ1, false, K + 1, false, 1, 1>(sU, &tb.B[0][0], nullptr, nullptr, NB, X0, XS, nt);
        sf_sym<0, NB1, NB1, NB1, NQ1, false, K + 1, false, -1, 1, T, GS>(sU, &tb.Dh[0][0][0], nullptr, nullptr, NB, X1,
                                                                        XS, ng);
        __syncthreads();
        sf_sym<1, NQ1, NB1, NB1, NQ1, false, K + 1, false, 1, 1>(X0, &tb.B[0][0], nullptr, nullptr, XS, Y, YS, nt);
        sf_sym<1, NQ1, NB1, NB1, NQ1, false, K + 1, false, 1, 1, T, GS>(X1, &tb.B[0][0], nullptr, nullptr, XS,
                                                                       Y + P::YSZ, YS, ng);
        sf_sym<1, NQ1, NB1, NB1, NQ1, false, K + 1, false, -1, 1, T, GS>(X0, &tb.Dh[1][0][0], nullptr, nullptr, XS,
                                                                        Y + 2 * P::YSZ, YS, ng);
        __syncthreads();
        sf_sym<2, NQ1, NQ1, NB1, NQ1, false, K + 1, false, 1, 1>(Y, &tb.B[0][0], nullptr, nullptr, YS, Q, NQ, nt);
        sf_sym<2, NQ1, NQ1, NB1, NQ1, false, K + 1, false, 1, 1, T, GS>(Y + P::YSZ, &tb.B[0][0], nullptr, nullptr, YS,
                                                                       Q + P::QSZ, NQ, ng);
        sf_sym<2, NQ1, NQ1, NB1, NQ1, false, K + 1, false, 1, 1, T, GS>(Y + 2 * P::YSZ, &tb.B[0][0], nullptr, nullptr,
                                                                       YS, Q + 2 * P::QSZ, NQ, ng);
        sf_sym<2, NQ1, NQ1, NB1, NQ1, false, K + 1, false, -1, 1, T, GS>(Y, &tb.Dh[2][0][0], nullptr, nullptr, YS,
                                                                        Q + 3 * P::QSZ, NQ, ng);
    }
    __syncthreads();

    // ---- volume: pointwise fluxes (gradients are physical: 1/h_j is in the tables) ----
    // The result goes to the slots of the last input field (the only one tested).
    constexpr int OFF = (F - 1) * EPB * NS * NQ;
    for (int idx = threadIdx.x; idx < EPB * NQ; idx += blockDim.x) {
        const int q = idx % NQ, e = idx / NQ;
        if (e0 + e >= g.E) {
            // padding of a ragged last CTA (U = 0, never stored): no pointwise
            // model there, so its zero state neither trips the domain check
            // nor feeds the theta partials
#pragma unroll
            for (int s = 0; s < NS; ++s)
#pragma unroll
                for (int j = 0; j <= D; ++j) Q[j * P::QSZ + OFF + (e * NS + s) * NQ + q] = T(0);
            continue;
        }
        T u[NS], gr[NS][D], Phi[NS][D], Sr[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            u[s] = Q[(e * NS + s) * NQ + q];
            const bool have = !MODAL || s == 0 || s == 3 || s == 5;   // interpolated gradients
#pragma unroll
            for (int j = 0; j < D; ++j) gr[s][j] = have ? Q[(j + 1) * P::QSZ + (e * NS + s) * NQ + q] : T(0);
        }
        const int q0 = q % NQ1, q1 = (q / NQ1) % NQ1, q2 = q / (NQ1 * NQ1);
        T wq = tb.w[q0] * tb.w[q1];
        if constexpr (D == 3) wq *= tb.w[q2];
        const T Wq = wq * c.vol;
        if constexpr (MODE == MODE_APPLY) {
            volume_point<D, T, MODAL>(c, u, gr, Phi, Sr);
        } else {
            T du[NS], dg[NS][D];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                du[s] = Q[OFF + (e * NS + s) * NQ + q];
                const bool have = !MODAL || s == 0 || s == 3 || s == 5;
#pragma unroll
                for (int j = 0; j < D; ++j) dg[s][j] = have ? Q[(j + 1) * P::QSZ + OFF + (e * NS + s) * NQ + q] : T(0);
            }
            if constexpr (MODE == MODE_JVP) {
                volume_point_lin<D, T, MODAL>(c, u, gr, du, dg, args.has_dtheta != 0, Phi, Sr);
            } else {
                // du, dg are mu and grad mu here; weighted they are the cotangents of S and Phi
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    du[s] *= Wq;
#pragma unroll
                    for (int j = 0; j < D; ++j) dg[s][j] *= Wq;
                }
                // (padding elements of a ragged last CTA hold mu = 0 and add nothing)
                volume_point_adj<D, T>(c, u, gr, du, dg, Sr, Phi, th);
                // the adjoints are already weighted: store them unscaled (gradients / h_j for the test)
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    Q[OFF + (e * NS + s) * NQ + q] = Sr[s];
#pragma unroll
                    for (int j = 0; j < D; ++j) Q[(j + 1) * P::QSZ + OFF + (e * NS + s) * NQ + q] = Phi[s][j];
                }
                continue;
            }
        }
        if constexpr (MODE == MODE_APPLY) {
            if (args.flags & CDG2_FORCING) {
                const long long ge = e0 + e;
                const long long ix = ge % g.n[0], iy = (ge / g.n[0]) % g.n[1];
                const T x = T(ix * g.h[0]) + T(g.h[0]) * tb.xi[q0];
                const T y = T(iy * g.h[1]) + T(g.h[1]) * tb.xi[q1];
                T gf[NS];
                mms_forcing<T>(x, y, T(args.t), T(g.L[1]), c, gf);
#pragma unroll
                for (int s = 0; s < NS; ++s) Sr[s] += gf[s];
            }
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            Q[OFF + (e * NS + s) * NQ + q] = Sr[s];   // weights and 1/h live in the test tables
            if (s < 2 || !MODAL) {                      // (modal: only n1, n2 are tested with grad phi)
#pragma unroll
                for (int j = 0; j < D; ++j) Q[(j + 1) * P::QSZ + OFF + (e * NS + s) * NQ + q] = Phi[s][j];
            }
        }
    }
    __syncthreads();

    // ---- volume: test with phi and grad phi (transposed sum factorisation) ----
    const int nto = EPB * NS;
    T* Qo = Q + OFF;
    // forward modes: Gauss-weighted tables (the residual is accumulated divided by
    // |K|); VJP: its cotangents already carry the weights, plain tables
    const T* TB = MODE == MODE_VJP ? &tb.B[0][0] : &tb.Bw[0][0];
    const T* TD0 = MODE == MODE_VJP ? &tb.Dh[0][0][0] : &tb.Dwh[0][0][0];
    const T* TD1 = MODE == MODE_VJP ? &tb.Dh[1][0][0] : &tb.Dwh[1][0][0];
    const T* TD2 = MODE == MODE_VJP ? &tb.Dh[2][0][0] : &tb.Dwh[2][0][0];
    if constexpr (MODAL) {
        // n1, n2 (set 2): phi and grad phi; n3..c3 (set 3): phi only
        constexpr int N2 = SpeciesSet<2>::N, N3 = SpeciesSet<3>::N;
        if constexpr (D == 2) {
            T* Y0 = X0;
            T* Y1 = X1;
            sf_sym<1, NQ1, NQ1, 1, NB1, true, K + 1, true, 1, -1, T, 2>(Qo, TB, Qo + 2 * P::QSZ, TD1, NQ, Y0,
                                                                       NQ1 * NB1, EPB * N2);
            sf_sym<1, NQ1, NQ1, 1, NB1, true, K + 1, false, 1, 1, T, 2>(Qo + P::QSZ, TB, nullptr, nullptr, NQ, Y1,
                                                                       NQ1 * NB1, EPB * N2);
            sf_sym<1, NQ1, NQ1, 1, NB1, true, K + 1, false, 1, 1, T, 3>(Qo, TB, nullptr, nullptr, NQ, Y0, NQ1 * NB1,
                                                                       EPB * N3);
            __syncthreads();
            sf_sym<0, NQ1, NB1, 1, NB1, true, K + 1, true, 1, -1, T, 2>(Y0, TB, Y1, TD0, NQ1 * NB1, sR, NB, EPB * N2);
            sf_sym<0, NQ1, NB1, 1, NB1, true, K + 1, false, 1, 1, T, 3>(Y0, TB, nullptr, nullptr, NQ1 * NB1, sR, NB,
                                                                       EPB * N3);
        } else {
            constexpr int ZS = NQ1 * NQ1 * NB1, XS = NQ1 * NB1 * NB1;
            T* Z0 = Y;
            T* Z1 = Y + P::YSZ;
            T* Z2 = Y + 2 * P::YSZ;
            sf_sym<2, NQ1, NQ1, NQ1, NB1, true, K + 1, true, 1, -1, T, 2>(Qo, TB, Qo + 3 * P::QSZ, TD2, NQ, Z0, ZS,
                                                                         EPB * N2);
            sf_sym<2, NQ1, NQ1, NQ1, NB1, true, K + 1, false, 1, 1, T, 2>(Qo + 2 * P::QSZ, TB, nullptr, nullptr, NQ, Z1,
                                                                         ZS, EPB * N2);
            sf_sym<2, NQ1, NQ1, NQ1, NB1, true, K + 1, false, 1, 1, T, 2>(Qo + P::QSZ, TB, nullptr, nullptr, NQ, Z2, ZS,
                                                                         EPB * N2);
            sf_sym<2, NQ1, NQ1, NQ1, NB1, true, K + 1, false, 1, 1, T, 3>(Qo, TB, nullptr, nullptr, NQ, Z0, ZS,
                                                                         EPB * N3);
            __syncthreads();
            T* Y0 = X0;
            T* Y1 = X1;
            sf_sym<1, NQ1, NQ1, NB1, NB1, true, K + 1, true, 1, -1, T, 2>(Z0, TB, Z1, TD1, ZS, Y0, XS, EPB * N2);
            sf_sym<1, NQ1, NQ1, NB1, NB1, true, K + 1, false, 1, 1, T, 2>(Z2, TB, nullptr, nullptr, ZS, Y1, XS, EPB * N2);
            sf_sym<1, NQ1, NQ1, NB1, NB1, true, K + 1, false, 1, 1, T, 3>(Z0, TB, nullptr, nullptr, ZS, Y0, XS, EPB * N3);
            __syncthreads();
            sf_sym<0, NQ1, NB1, NB1, NB1, true, K + 1, true, 1, -1, T, 2>(Y0, TB, Y1, TD0, XS, sR, NB, EPB * N2);
            sf_sym<0, NQ1, NB1, NB1, NB1, true, K + 1, false, 1, 1, T, 3>(Y0, TB, nullptr, nullptr, XS, sR, NB,
                                                                         EPB * N3);
        }
        __syncthreads();
        // Diffusion of n2..c3 in modal form: their flux -A_s grad U_s tested with
        // grad phi is, by exact quadrature on the orthonormal tensor basis,
        // -A_s sum_j (K1_j (x) I) U_s with K1_j[a][b] = int psi'_a psi'_b / h_j^2
        // (zero unless a = b mod 2 and a, b > 0).
        const T* Uf = sU + (F - 1) * P::UR;
        for (int idx = threadIdx.x; idx < EPB * SpeciesSet<4>::N * NB; idx += blockDim.x) {
            const int i = idx % NB, es = idx / NB;
            const int e = es / SpeciesSet<4>::N, s = SpeciesSet<4>::s(es % SpeciesSet<4>::N);
            const T* u = Uf + (e * NS + s) * NB;
            T acc = T(0);
            int stride = 1, rest = i;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const int a = rest % NB1;
                rest /= NB1;
                const int base = i - a * stride;
                for (int bb = (a & 1) ? 1 : 2; a > 0 && bb <= K; bb += 2) acc = fma(tb.K1h[j][a][bb], u[base + bb * stride], acc);
                stride *= NB1;
            }
            sR[(e * NS + s) * NB + i] = fma(-T(c.A[s]), acc, sR[(e * NS + s) * NB + i]);
        }
    } else {
        if constexpr (D == 2) {
            // Y0 = B^T_y S' + D^T_y Phi_y',  Y1 = B^T_y Phi_x'
            T* Y0 = X0;
            T* Y1 = X1;
            sf_sym<1, NQ1, NQ1, 1, NB1, true, K + 1, true, 1, -1>(Qo, TB, Qo + 2 * P::QSZ, TD1, NQ, Y0,
                                                             NQ1 * NB1, nto);
            sf_sym<1, NQ1, NQ1, 1, NB1, true, K + 1, false, 1, 1>(Qo + P::QSZ, TB, nullptr, nullptr, NQ, Y1,
                                                              NQ1 * NB1, nto);
            __syncthreads();
            sf_sym<0, NQ1, NB1, 1, NB1, true, K + 1, true, 1, -1>(Y0, TB, Y1, TD0, NQ1 * NB1, sR, NB, nto);
        } else {
            constexpr int ZS = NQ1 * NQ1 * NB1, XS = NQ1 * NB1 * NB1;
            T* Z0 = Y;
            T* Z1 = Y + P::YSZ;
            T* Z2 = Y + 2 * P::YSZ;
            sf_sym<2, NQ1, NQ1, NQ1, NB1, true, K + 1, true, 1, -1>(Qo, TB, Qo + 3 * P::QSZ, TD2, NQ, Z0, ZS,
                                                               nto);
            sf_sym<2, NQ1, NQ1, NQ1, NB1, true, K + 1, false, 1, 1>(Qo + 2 * P::QSZ, TB, nullptr, nullptr, NQ, Z1,
                                                                ZS, nto);
            sf_sym<2, NQ1, NQ1, NQ1, NB1, true, K + 1, false, 1, 1>(Qo + P::QSZ, TB, nullptr, nullptr, NQ, Z2, ZS,
                                                                nto);
            __syncthreads();
            T* Y0 = X0;
            T* Y1 = X1;
            sf_sym<1, NQ1, NQ1, NB1, NB1, true, K + 1, true, 1, -1>(Z0, TB, Z1, TD1, ZS, Y0, XS, nto);
            sf_sym<1, NQ1, NQ1, NB1, NB1, true, K + 1, false, 1, 1>(Z2, TB, nullptr, nullptr, ZS, Y1, XS, nto);
            __syncthreads();
            sf_sym<0, NQ1, NB1, NB1, NB1, true, K + 1, true, 1, -1>(Y0, TB, Y1, TD0, XS, sR, NB, nto);
        }
        __syncthreads();
    }
    __syncthreads();

    // ---- faces ----
    if (MODE != MODE_VJP && args.fbuf != nullptr) {
        faces_expand<D, K, 0, T>(g, tb, c, args.fbuf + args.fb_off[0], sR, e0, EPB, nbr);
        faces_expand<D, K, 1, T>(g, tb, c, args.fbuf + args.fb_off[1], sR, e0, EPB, nbr);
        if constexpr (D == 3) faces_expand<D, K, 2, T>(g, tb, c, args.fbuf + args.fb_off[2], sR, e0, EPB, nbr);
    } else {
        op_faces<D, K, MODE, 0, T>(g, tb, c, args, sU, sR, W, e0, nbr, th, ps);
        op_faces<D, K, MODE, 1, T>(g, tb, c, args, sU, sR, W, e0, nbr, th, ps);
        if constexpr (D == 3) op_faces<D, K, MODE, 2, T>(g, tb, c, args, sU, sR, W, e0, nbr, th, ps);
    }

    // ---- M^{-1} = I / |K| for the orthonormal basis; coalesced store ----
    // forward modes accumulate R / |K|; the VJP accumulates R itself
    const T scale = MODE == MODE_VJP ? ((args.flags & CDG2_MINV) ? c.inv_vol : T(1))
                                     : ((args.flags & CDG2_MINV) ? T(1) : c.vol);
    const T alphaT = T(args.alpha), betaT = T(args.beta);
    for (int i = threadIdx.x; i < P::UR; i += blockDim.x) {
        const long long ge = e0 + i / (NS * NB);
        if (ge < g.E) {
            if constexpr (MODE != MODE_APPLY)
                args.out[e0 * NS * NB + i] = alphaT * sU[P::UR + i] + betaT * (sR[i] * scale);
            else
                args.out[e0 * NS * NB + i] = sR[i] * scale;
        }
    }

    // ---- VJP: deterministic per-CTA reduction of the theta cotangent ----
    if constexpr (MODE == MODE_VJP) {
        if (args.theta_part != nullptr) {
            __syncthreads();   // W is free again: reuse it as a double buffer
            double* red = reinterpret_cast<double*>(W);
            for (int j = 0; j < 8; ++j) red[j * blockDim.x + threadIdx.x] = double(th[j]);
            __syncthreads();
            for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
                if ((int)threadIdx.x < stride)
                    for (int j = 0; j < 8; ++j) red[j * blockDim.x + threadIdx.x] += red[j * blockDim.x + threadIdx.x + stride];
                __syncthreads();
            }
            if (threadIdx.x < 8) args.theta_part[(long long)blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x * blockDim.x] * double(scale);
        }
    }
}

// Fixed-order sum of the per-CTA theta partials: one CTA of 256 threads, each
// thread sums a strided subset in index order, then a tree reduction.
__global__ void __launch_bounds__(256) theta_reduce_kernel(const double* __restrict__ part, long long nblocks,
                                                           double* __restrict__ gtheta) {
    __shared__ double red[8][256];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int j = 0; j < 8; ++j) acc[j] += part[b * 8 + j];
    for (int j = 0; j < 8; ++j) red[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride)
            for (int j = 0; j < 8; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + stride];
        __syncthreads();
    }
    if (threadIdx.x < 8) gtheta[threadIdx.x] = red[threadIdx.x][0];
}

template <typename T>
static const TabP<T>& tab_of(const cdg2_mesh& m) {
    if constexpr (std::is_same<T, double>::value) return m.tp64;
    else return m.tp32;
}

template <int MODE>
static long long grid_of(const cdg2_mesh& m) {
    constexpr int F = fields_of(MODE);
    const int d = m.geo.dim, k = m.geo.k;
    int epb = 1;
    if (d == 2 && k == 1) epb = OpPlan<2, 1, F>::EPB;
    if (d == 2 && k == 2) epb = OpPlan<2, 2, F>::EPB;
    if (d == 2 && k == 3) epb = OpPlan<2, 3, F>::EPB;
    if (d == 3 && k == 1) epb = OpPlan<3, 1, F>::EPB;
    if (d == 3 && k == 2) epb = OpPlan<3, 2, F>::EPB;
    if (d == 3 && k == 3) epb = OpPlan<3, 3, F>::EPB;
    return (m.geo.E + epb - 1) / epb;
}

// The face kernels of the face-once path for axis 0..D-1 (each face once, its
// tested fluxes into the mesh's face buffer), with their one-time attributes.
template <int D, int K, int MODE, typename T>
static cudaError_t launch_faces(const cdg2_mesh& m, OpArgs<T>& a, cudaStream_t st) {
    if (!m.fbuf) {
        const size_t bytes = face_buffer_bytes(m.geo);
        cudaError_t e = cudaMalloc(&m.fbuf, bytes);
        if (e != cudaSuccess) return e;
        m.fbuf_bytes = bytes;
    }
    a.fbuf = static_cast<T*>(m.fbuf);
    constexpr long long per_face = 2LL * NS * Shape<D, K>::NBT;
    long long off = 0;
    for (int ax = 0; ax < 3; ++ax) {
        a.fb_off[ax] = off;
        if (ax < D) off += faces_of_axis(m.geo, ax) * per_face;
    }
    if constexpr (D == 3 && K == 3 && std::is_same<T, float>::value) {
        // FP32 on Q3: one warp per face (issue-bound; no CTA barriers between phases)
        using FPl = Face3WPlan<K, fields_of(MODE), T>;
        constexpr size_t fsmem = FPl::smem_bytes();
        static_assert(fsmem <= 227 * 1024, "face kernel shared memory exceeds 227 KB");
        static DeviceOnce fattr;
        cudaError_t e = once_per_device(fattr, [] {
            cudaError_t r = cudaFuncSetAttribute(face3w_kernel<K, MODE, 0, T>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute(face3w_kernel<K, MODE, 1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fsmem);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute(face3w_kernel<K, MODE, 2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fsmem);
            return r;
        });
        if (e != cudaSuccess) return e;
        auto al16 = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
        const int bulk = FPl::BULK && al16(a.U[0]) && (fields_of(MODE) == 1 || al16(a.U[1]));
        auto fgrid = [&](int ax) { return (unsigned)((faces_of_axis(m.geo, ax) + FPl::WARPS - 1) / FPl::WARPS); };
        face3w_kernel<K, MODE, 0, T><<<fgrid(0), FPl::NT, fsmem, st>>>(m.geo, tab_of<T>(m), a, bulk);
        face3w_kernel<K, MODE, 1, T><<<fgrid(1), FPl::NT, fsmem, st>>>(m.geo, tab_of<T>(m), a, bulk);
        face3w_kernel<K, MODE, 2, T><<<fgrid(2), FPl::NT, fsmem, st>>>(m.geo, tab_of<T>(m), a, bulk);
    } else if constexpr (D == 3) {
        using FPl = Face3Plan<K, fields_of(MODE), T>;
        constexpr size_t fsmem = FPl::smem_bytes();
        static_assert(fsmem <= 227 * 1024, "face kernel shared memory exceeds 227 KB");
        static DeviceOnce fattr;
        cudaError_t e = once_per_device(fattr, [] {
            cudaError_t r = cudaFuncSetAttribute(face3_kernel<K, MODE, 0, T>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute(face3_kernel<K, MODE, 1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fsmem);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute(face3_kernel<K, MODE, 2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fsmem);
            return r;
        });
        if (e != cudaSuccess) return e;
        auto al16 = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
        const int bulk = FPl::BULK && al16(a.U[0]) && (fields_of(MODE) == 1 || al16(a.U[1]));
        auto fgrid = [&](int ax) { return (unsigned)((faces_of_axis(m.geo, ax) + FPl::FPB - 1) / FPl::FPB); };
        face3_kernel<K, MODE, 0, T><<<fgrid(0), FPl::NT, fsmem, st>>>(m.geo, tab_of<T>(m), a, bulk);
        face3_kernel<K, MODE, 1, T><<<fgrid(1), FPl::NT, fsmem, st>>>(m.geo, tab_of<T>(m), a, bulk);
        face3_kernel<K, MODE, 2, T><<<fgrid(2), FPl::NT, fsmem, st>>>(m.geo, tab_of<T>(m), a, bulk);
    } else {
        using FPl = FacePlan<D, K, fields_of(MODE)>;
        constexpr size_t fsmem = FPl::template smem_bytes<T>();
        static_assert(fsmem <= 227 * 1024, "face kernel shared memory exceeds 227 KB");
        static DeviceOnce fattr;
        cudaError_t e = once_per_device(fattr, [] {
            cudaError_t r = cudaFuncSetAttribute(face_kernel<D, K, MODE, 0, T>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute(face_kernel<D, K, MODE, 1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fsmem);
            return r;
        });
        if (e != cudaSuccess) return e;
        auto fgrid = [&](int ax) { return (unsigned)((faces_of_axis(m.geo, ax) + FPl::FPB - 1) / FPl::FPB); };
        face_kernel<D, K, MODE, 0, T><<<fgrid(0), FPl::NT, fsmem, st>>>(m.geo, tab_of<T>(m), a);
        face_kernel<D, K, MODE, 1, T><<<fgrid(1), FPl::NT, fsmem, st>>>(m.geo, tab_of<T>(m), a);
    }
    return cudaSuccess;
}

// CDG2_TF32 on a 3D Q3 mesh: the face kernels (FP32), then the tensor-core
// element kernel (16 elements per CTA).
template <int MODE>
static cudaError_t launch_tc(const cdg2_mesh& m, OpArgs<float> a, cudaStream_t st) {
    if (!m.tc_tables) {
        std::vector<float> img;
        tc::build_tables(m.tab, m.geo, img);
        cudaError_t e = cudaMalloc(&m.tc_tables, img.size() * sizeof(float));
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(m.tc_tables, img.data(), img.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    if (reinterpret_cast<uintptr_t>(a.U[0]) % 16 || reinterpret_cast<uintptr_t>(a.U[1]) % 16) return cudaErrorMisalignedAddress;
    static DeviceOnce attr;
    {
        cudaError_t e = once_per_device(attr, [] {
            return cudaFuncSetAttribute(tc_elem_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        tc::SMEM_BYTES);
        });
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_faces<3, 3, MODE, float>(m, a, st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((m.geo.E + tc::NE - 1) / tc::NE);
    tc_elem_kernel<MODE><<<blocks, tc::NT, tc::SMEM_BYTES, st>>>(m.geo, m.tp32, a,
                                                               static_cast<const float4*>(m.tc_tables));
    return cudaGetLastError();
}

template <int D, int K, int MODE, typename T>
static cudaError_t launch_one(const cdg2_mesh& m, const Coef& c, OpArgs<T> a, cudaStream_t st) {
    using P = OpPlan<D, K, fields_of(MODE)>;
    constexpr size_t smem = P::template smem_bytes<T>();
    static_assert(smem <= 227 * 1024, "operator kernel shared memory exceeds 227 KB");
    static_assert(MODE != MODE_VJP || sizeof(T) * P::WORK >= 8 * 128 * sizeof(double),
                  "theta reduction buffer does not fit the work area");
    static DeviceOnce attr;   // per instantiation and device
    {
        cudaError_t e = once_per_device(attr, [] {
            return cudaFuncSetAttribute(op_kernel<D, K, MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem);
        });
        if (e != cudaSuccess) return e;
    }
    const long long blocks = grid_of<MODE>(m);
    a.c = make_coefT<T>(c, m.geo, a.has_dtheta ? a.dtheta : nullptr);
    if (!a.domain) {
        cudaError_t e = ensure_status(&m.status);
        if (e != cudaSuccess) return e;
        a.domain = m.status;
    }
    a.c.domain = a.domain;
    if constexpr (D == 3 && K == 3 && std::is_same<T, float>::value && MODE != MODE_VJP) {
        if (a.flags & CDG2_TF32) return launch_tc<MODE>(m, a, st);
    }
    a.fbuf = nullptr;
    // Face-once (each face evaluated once, by the face kernels) for the apply
    // and the JVP; the VJP keeps the fused path.
    constexpr bool face_once = MODE != MODE_VJP;
    if constexpr (face_once) {
        cudaError_t e = launch_faces<D, K, MODE, T>(m, a, st);
        if (e != cudaSuccess) return e;
    }
    op_kernel<D, K, MODE, T><<<(unsigned)blocks, P::NT, smem, st>>>(m.geo, tab_of<T>(m), a);
    return cudaGetLastError();
}

template <int MODE, typename T>
static cudaError_t dispatch(const cdg2_mesh& m, const Coef& c, const OpArgs<T>& a, cudaStream_t st) {
    const int d = m.geo.dim, k = m.geo.k;
    if (d == 2 && k == 1) return launch_one<2, 1, MODE, T>(m, c, a, st);
    if (d == 2 && k == 2) return launch_one<2, 2, MODE, T>(m, c, a, st);
    if (d == 2 && k == 3) return launch_one<2, 3, MODE, T>(m, c, a, st);
    if (d == 3 && k == 1) return launch_one<3, 1, MODE, T>(m, c, a, st);
    if (d == 3 && k == 2) return launch_one<3, 2, MODE, T>(m, c, a, st);
    if (d == 3 && k == 3) return launch_one<3, 3, MODE, T>(m, c, a, st);
    return cudaErrorInvalidValue;
}

template <typename T>
static OpArgs<T> make_args(const void* U, const void* dU, void* out, int flags, double t, const double* dtheta,
                           double* theta_part) {
    OpArgs<T> a{};
    a.U[0] = (const T*)U;
    a.U[1] = (const T*)dU;
    a.out = (T*)out;
    a.flags = flags;
    a.t = t;
    a.has_dtheta = dtheta != nullptr;
    for (int i = 0; i < 8; ++i) a.dtheta[i] = dtheta ? dtheta[i] : 0.0;
    a.theta_part = theta_part;
    a.alpha = 0.0;
    a.beta = 1.0;
    a.pscale = nullptr;
    a.fbuf = nullptr;
    for (int i = 0; i < 3; ++i) a.fb_off[i] = 0;
    a.domain = nullptr;
    return a;
}

long long vjp_grid(const cdg2_mesh& m) { return grid_of<MODE_VJP>(m); }

size_t face_buffer_bytes(const Geo& g) {
    long long nbt = 1;
    for (int a = 0; a < g.dim - 1; ++a) nbt *= g.k + 1;
    long long faces = 0;
    for (int a = 0; a < g.dim; ++a) faces += faces_of_axis(g, a);
    return (size_t)faces * 2 * NS * nbt * sizeof(double);
}

cudaError_t launch_apply(const cdg2_mesh& m, const Coef& c, const void* U, void* out, int flags, double t,
                         cudaStream_t st) {
    if (flags & CDG2_FP32)
        return dispatch<MODE_APPLY, float>(m, c, make_args<float>(U, U, out, flags, t, nullptr, nullptr), st);
    return dispatch<MODE_APPLY, double>(m, c, make_args<double>(U, U, out, flags, t, nullptr, nullptr), st);
}

cudaError_t launch_jvp(const cdg2_mesh& m, const Coef& c, const void* U, const void* dU, const double* dtheta,
                       void* out, int flags, cudaStream_t st) {
    if (flags & CDG2_FP32)
        return dispatch<MODE_JVP, float>(m, c, make_args<float>(U, dU, out, flags, 0.0, dtheta, nullptr), st);
    return dispatch<MODE_JVP, double>(m, c, make_args<double>(U, dU, out, flags, 0.0, dtheta, nullptr), st);
}

cudaError_t launch_jvp_axpby(const cdg2_mesh& m, const Coef& c, const void* U, const void* dU, double alpha,
                             double beta, const double* pscale, void* out, int flags, cudaStream_t st) {
    if (flags & CDG2_FP32) {
        OpArgs<float> a = make_args<float>(U, dU, out, flags, 0.0, nullptr, nullptr);
        a.alpha = alpha;
        a.beta = beta;
        a.pscale = pscale;
        return dispatch<MODE_JVP, float>(m, c, a, st);
    }
    OpArgs<double> a = make_args<double>(U, dU, out, flags, 0.0, nullptr, nullptr);
    a.alpha = alpha;
    a.beta = beta;
    a.pscale = pscale;
    return dispatch<MODE_JVP, double>(m, c, a, st);
}

cudaError_t launch_vjp_axpby(const cdg2_mesh& m, const Coef& c, const void* U, const void* lam, double alpha,
                             double beta, const double* pscale, void* out, int flags, cudaStream_t st) {
    if (flags & CDG2_FP32) {
        OpArgs<float> a = make_args<float>(U, lam, out, flags, 0.0, nullptr, nullptr);
        a.alpha = alpha;
        a.beta = beta;
        a.pscale = pscale;
        return dispatch<MODE_VJP, float>(m, c, a, st);
    }
    OpArgs<double> a = make_args<double>(U, lam, out, flags, 0.0, nullptr, nullptr);
    a.alpha = alpha;
    a.beta = beta;
    a.pscale = pscale;
    return dispatch<MODE_VJP, double>(m, c, a, st);
}

cudaError_t launch_vjp(const cdg2_mesh& m, const Coef& c, const void* U, const void* lam, void* gU,
                       double* theta_part, double* gtheta, int flags, cudaStream_t st, int* domain) {
    cudaError_t e;
    if (flags & CDG2_FP32) {
        OpArgs<float> a = make_args<float>(U, lam, gU, flags, 0.0, nullptr, theta_part);
        a.domain = domain;
        e = dispatch<MODE_VJP, float>(m, c, a, st);
    } else {
        OpArgs<double> a = make_args<double>(U, lam, gU, flags, 0.0, nullptr, theta_part);
        a.domain = domain;
        e = dispatch<MODE_VJP, double>(m, c, a, st);
    }
    if (e != cudaSuccess || gtheta == nullptr) return e;
    theta_reduce_kernel<<<1, 256, 0, st>>>(theta_part, grid_of<MODE_VJP>(m), gtheta);
    return cudaGetLastError();
}

}  // namespace cdg2
