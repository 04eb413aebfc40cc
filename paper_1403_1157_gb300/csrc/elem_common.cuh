// Building blocks shared by the element-centric kernels (apply, JVP, VJP):
// compile-time shapes, shared-memory tables, sum-factorised tensor
// contractions and the neighbour lookup of the structured mesh.
#pragma once

#include "cdg2_internal.h"

namespace cdg2 {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Sizes of one element for dimension D and degree K (q1 = K + 2 points).
template <int D, int K>
struct Shape {
    static constexpr int NB1 = K + 1;                 // 1D basis
    static constexpr int NQ1 = K + 2;                 // 1D Gauss points
    static constexpr int NB = ipow(NB1, D);           // basis per species
    static constexpr int NQ = ipow(NQ1, D);           // volume points
    static constexpr int NBT = ipow(NB1, D - 1);      // tangential basis on a face
    static constexpr int NQT = ipow(NQ1, D - 1);      // face points
};

// 1D tables in shared memory in the kernel's precision, at the kernel's
// degree: a copy of the kernel's TabP argument (1/h_j and the Gauss weights
// already folded in, so the pointwise code does no scaling multiplications).
template <int K, typename T>
struct STab {
    T B[K + 2][K + 1];       // psi_a(xi_q)
    T Bw[K + 2][K + 1];      // w_q psi_a(xi_q)
    T Dh[3][K + 2][K + 1];   // psi'_a(xi_q) / h_j
    T Dwh[3][K + 2][K + 1];  // w_q psi'_a(xi_q) / h_j
    T w[K + 2];
    T xi[K + 2];
    T e[2][K + 1];           // psi_a(0), psi_a(1)
    T dh[3][2][K + 1];       // psi'_a(0) / h_j, psi'_a(1) / h_j
    T K1h[3][K + 1][K + 1];  // int_0^1 psi'_a psi'_b / h_j^2 (1D stiffness, exact)
};

template <int K, typename T>
__device__ __forceinline__ void load_tab(STab<K, T>& s, const TabP<T>& t) {
    for (int i = threadIdx.x; i < (K + 2) * (K + 1); i += blockDim.x) {
        const int q = i / (K + 1), a = i % (K + 1);
        s.B[q][a] = t.B[q][a];
        s.Bw[q][a] = t.Bw[q][a];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            s.Dh[j][q][a] = t.Dh[j][q][a];
            s.Dwh[j][q][a] = t.Dwh[j][q][a];
        }
    }
    for (int i = threadIdx.x; i < K + 2; i += blockDim.x) {
        s.w[i] = t.w[i];
        s.xi[i] = t.xi[i];
    }
    for (int i = threadIdx.x; i < 2 * (K + 1); i += blockDim.x) {
        const int f = i / (K + 1), a = i % (K + 1);
        s.e[f][a] = t.e[f][a];
#pragma unroll
        for (int j = 0; j < 3; ++j) s.dh[j][f][a] = t.dh[j][f][a];
    }
    for (int i = threadIdx.x; i < 3 * (K + 1) * (K + 1); i += blockDim.x) {
        const int j = i / ((K + 1) * (K + 1)), a = (i / (K + 1)) % (K + 1), b = i % (K + 1);
        s.K1h[j][a][b] = t.K1h[j][a][b];
    }
}

// a / b: IEEE division in FP64; the fast reciprocal-based divide in FP32
// (2 ulp), which the FP32 path's 1e-5 error budget allows.
template <typename T>
__device__ __forceinline__ T qdiv(T a, T b) {
    return a / b;
}
template <>
__device__ __forceinline__ float qdiv<float>(float a, float b) {
    return __fdividef(a, b);
}

// Reciprocals r_i = 1 / x_i of N values.  FP64: simultaneous inversion
// (Montgomery's trick: prefix products, one division, 3(N-1) multiplications
// instead of N divisions, a few ulp), with the N divisions when the product of
// all values is outside [1e-250, 1e250] or not finite.  FP32: qdiv per value.
template <int N, typename T>
__device__ __forceinline__ void recips(const T* x, T* r) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < N; ++i) r[i] = qdiv<T>(T(1), x[i]);
    } else {
        T p[N];
        p[0] = x[0];
#pragma unroll
        for (int i = 1; i < N; ++i) p[i] = p[i - 1] * x[i];
        const T a = fabs(p[N - 1]);
        if (a > T(1e-250) && a < T(1e250)) {
            T inv = T(1) / p[N - 1];
#pragma unroll
            for (int i = N - 1; i > 0; --i) {
                r[i] = inv * p[i - 1];
                inv = inv * x[i];
            }
            r[0] = inv;
        } else {
#pragma unroll
            for (int i = 0; i < N; ++i) r[i] = T(1) / x[i];
        }
    }
}

template <typename T>
struct Ident {
    using type = T;
};

// One sum-factorisation pass over nt tensors stored back to back.
// Species subsets of the forward volume terms (the diffusion of n2..c3 is
// applied in modal form, see op_kernel): 0 all six; 1 {n1, c1, c3}, whose
// gradients the fluxes need at the points; 2 {n1, n2}, the fluxes tested with
// grad phi; 3 {n3, c1, c2, c3}, tested with phi only; 4 {n2, .., c3};
// 5 {n1, n2, c1, c3}, the face-point traces the chemotactic fluxes need.
template <int SEL>
struct SpeciesSet;
template <>
struct SpeciesSet<0> {
    static constexpr int N = NS;
    __device__ static constexpr int s(int k) { return k; }
};
template <>
struct SpeciesSet<1> {
    static constexpr int N = 3;
    __device__ static constexpr int s(int k) { return k == 0 ? 0 : (k == 1 ? 3 : 5); }
};
template <>
struct SpeciesSet<2> {
    static constexpr int N = 2;
    __device__ static constexpr int s(int k) { return k; }
};
template <>
struct SpeciesSet<3> {
    static constexpr int N = 4;
    __device__ static constexpr int s(int k) { return k + 2; }
};
template <>
struct SpeciesSet<4> {
    static constexpr int N = 5;
    __device__ static constexpr int s(int k) { return k + 1; }
};
template <>
struct SpeciesSet<5> {
    static constexpr int N = 4;
    __device__ static constexpr int s(int k) { return k < 2 ? k : (k == 2 ? 3 : 5); }
};

// One 1D pass of sum factorisation.  Input tensors have extents (I0, I1, I2)
// (x fastest); axis AX (extent NI) is replaced by NO in the output:
//     out[t][..o..] = sum_i M1(o,i) in1[t][..i..]  (+ M2(o,i) in2[t][..i..])
// with M(o,i) = M[o][i] (TR = false: points from modes) or M[i][o] (TR = true:
// modes from points), M stored [point][mode] with row length LD.  One thread
// computes one whole line along AX: its index arithmetic is done once per
// line, the 1D matrices are held in registers, each input is loaded once.
// The matrices have the mirror symmetry of Legendre modes at a symmetric
// Gauss rule, M(NQ-1-q, a) = P (-1)^a M(q, a), P = +1 for values (B, Bw) and
// -1 for derivatives (Dh, Dwh), and only rows q < ceil(NQ/2) are read.
// Forward: out(q) and out(NQ-1-q) are E +- O with E, O the sums over the even
// and odd modes.  Transposed: the inputs are paired as x(q) +- x(NQ-1-q) and
// each mode takes the pair combination of its parity.  For k = 3 this is 14
// operations per line and matrix instead of 20.  SEL restricts the pass to
// the species of SpeciesSet<SEL>: tensor t is then (t / N, species s(t % N))
// of an element-major [..][6] layout, and nt counts only those tensors; with
// IN_COMPACT the input holds only those tensors, back to back.  The lines
// are dealt to the CTA's threads, or, given first >= 0, to `step` threads
// numbered from `first` (a warp working alone).
template <int AX, int I0, int I1, int I2, int NO, bool TR, int LD, bool TWO, int P1, int P2, typename T, int SEL = 0,
          bool IN_COMPACT = false>
__device__ __forceinline__ void sf_sym(const T* __restrict__ in1, const T* __restrict__ M1,
                                       const typename Ident<T>::type* __restrict__ in2,
                                       const typename Ident<T>::type* __restrict__ M2, int in_stride,
                                       T* __restrict__ out, int out_stride, int nt, int first = -1, int step = 0) {
    constexpr int NI = AX == 0 ? I0 : (AX == 1 ? I1 : I2);
    constexpr int NQ = TR ? NI : NO;   // points
    constexpr int NM = TR ? NO : NI;   // modes
    constexpr int H = NQ / 2;          // mirrored pairs (q, NQ-1-q), q < H
    constexpr int MID = NQ % 2;        // a middle point q = H
    static_assert(TR || !TWO, "two-matrix passes are transposed");
    constexpr int NL = I0 * I1 * I2 / NI;
    constexpr int ST = AX == 0 ? 1 : (AX == 1 ? I0 : I0 * I1);
    T m1[H + MID][NM], m2[TWO ? H + MID : 1][TWO ? NM : 1];
#pragma unroll
    for (int q = 0; q < H + MID; ++q)
#pragma unroll
        for (int a = 0; a < NM; ++a) {
            m1[q][a] = M1[q * LD + a];
            if constexpr (TWO) m2[q][a] = M2[q * LD + a];
        }
    const int total = nt * NL;
    const int l0 = first < 0 ? (int)threadIdx.x : first, dl = first < 0 ? (int)blockDim.x : step;
    for (int line = l0; line < total; line += dl) {
        const int tt = line / NL;
        const int r = line - tt * NL;
        int ib, ob;
        if constexpr (AX == 0) {
            ib = r * I0;
            ob = r * NO;
        } else if constexpr (AX == 1) {
            const int a = r % I0, b = r / I0;
            ib = a + b * I0 * I1;
            ob = a + b * I0 * NO;
        } else {
            ib = r;
            ob = r;
        }
        using SS = SpeciesSet<SEL>;
        const int tm = SEL == 0 ? tt : (tt / SS::N) * NS + SS::s(tt % SS::N);
        const int ti = IN_COMPACT ? tt : tm;
        const T* s1 = in1 + ti * in_stride + ib;
        T* d = out + tm * out_stride + ob;
        if constexpr (!TR) {
            T v[NM];
#pragma unroll
            for (int a = 0; a < NM; ++a) v[a] = s1[a * ST];
#pragma unroll
            for (int q = 0; q < H; ++q) {
                T ev = T(0), od = T(0);
#pragma unroll
                for (int a = 0; a < NM; a += 2) ev = fma(m1[q][a], v[a], ev);
#pragma unroll
                for (int a = 1; a < NM; a += 2) od = fma(m1[q][a], v[a], od);
                d[q * ST] = ev + od;
                d[(NQ - 1 - q) * ST] = P1 > 0 ? ev - od : od - ev;
            }
            if constexpr (MID) {
                // the modes of the other parity vanish at the middle point
                T acc = T(0);
#pragma unroll
                for (int a = P1 > 0 ? 0 : 1; a < NM; a += 2) acc = fma(m1[H][a], v[a], acc);
                d[H * ST] = acc;
            }
        } else {
            T sp1[H], sm1[H], mid1 = T(0), sp2[TWO ? H : 1], sm2[TWO ? H : 1], mid2 = T(0);
#pragma unroll
            for (int q = 0; q < H; ++q) {
                const T x = s1[q * ST], y = s1[(NQ - 1 - q) * ST];
                sp1[q] = x + y;
                sm1[q] = x - y;
            }
            if constexpr (MID) mid1 = s1[H * ST];
            if constexpr (TWO) {
                const T* s2 = in2 + ti * in_stride + ib;
#pragma unroll
                for (int q = 0; q < H; ++q) {
                    const T x = s2[q * ST], y = s2[(NQ - 1 - q) * ST];
                    sp2[q] = x + y;
                    sm2[q] = x - y;
                }
                if constexpr (MID) mid2 = s2[H * ST];
            }
#pragma unroll
            for (int a = 0; a < NM; ++a) {
                // mode a pairs with the sums when P (-1)^a = +1, else with the differences
                const bool even1 = (P1 > 0) == (a % 2 == 0);
                T acc = T(0);
#pragma unroll
                for (int q = 0; q < H; ++q) acc = fma(m1[q][a], even1 ? sp1[q] : sm1[q], acc);
                if (MID && even1) acc = fma(m1[MID ? H : 0][a], mid1, acc);
                if constexpr (TWO) {
                    const bool even2 = (P2 > 0) == (a % 2 == 0);
#pragma unroll
                    for (int q = 0; q < H; ++q) acc = fma(m2[q][a], even2 ? sp2[q] : sm2[q], acc);
                    if (MID && even2) acc = fma(m2[MID ? H : 0][a], mid2, acc);
                }
                d[a * ST] = acc;
            }
        }
    }
}

// Index of the element coefficient with normal index m along axis A and
// tangential multi-index (b0, b1) over the remaining axes in increasing order.
template <int D, int K, int A>
__device__ __forceinline__ int coef_index(int m, int b0, int b1) {
    constexpr int N = K + 1;
    if constexpr (D == 2) {
        return A == 0 ? (m + N * b0) : (b0 + N * m);
    } else {
        if constexpr (A == 0) return m + N * (b0 + N * b1);
        if constexpr (A == 1) return b0 + N * (m + N * b1);
        return b0 + N * (b1 + N * m);
    }
}

// Cell coordinates of element e.  Element indices fit in 31 bits
// (cdg2_mesh_create bounds E * 6 * n_b below 2^31), so the divisions are
// 32-bit ones.
__device__ __forceinline__ void cell_coords(const Geo& g, long long e, int c[3]) {
    const unsigned u = (unsigned)e, n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    const unsigned r = u / n0;
    c[0] = (int)(u - r * n0);
    c[1] = (int)(r % n1);
    c[2] = (int)(r / n1);
}

// Neighbour of element e across face f (0: low side, 1: high side) of axis
// a; -1 on a non-periodic boundary.
__device__ __forceinline__ long long neighbour(const Geo& g, long long e, int a, int f) {
    int c[3];
    cell_coords(g, e, c);
    int v = c[a] + (f ? 1 : -1);
    if (v < 0 || v >= g.n[a]) {
        if (!g.periodic[a]) return -1;
        v = v < 0 ? v + g.n[a] : v - g.n[a];
    }
    c[a] = v;
    return c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
}

// The model coefficients converted once, on the host, to the kernel's
// precision, so the pointwise code does no double -> float conversions (on
// GB300 those run on the narrow FP64 pipe).  Same member names as Coef, plus derived
// geometry and the optional parameter tangent.
template <typename T>
struct CoefT {
    T A[NS];
    T chi0[4], chith[4];
    T d1, d2, gamma, alpha1, alpha2, f1, k_ox;
    T beta1, beta2, sigma, c1s, c1ss, bc_sign;
    T phase[NS];
    T dth[8];       // tangent of (d1, d2, gamma, alpha1, alpha2, f1, k_ox, beta1)
    T vol;          // |K|
    T inv_vol;      // 1 / |K| (M^{-1} of the orthonormal basis)
    T invh[3];      // 1 / h_j
    T pen_c;        // face penalty constant (chi_e for CDG2, eta/2 for BR2, C for SIPG)
    T death1;       // 1: Eq. (1); 0: the reduced model of Eq. (2) (no n1 death term)
    int* domain;    // device status word: set to 1 where c + chi^th <= 0 (a pole of chi), or null
};

// Host-side conversion (kernel parameters live in the constant bank, so the
// pointwise code reads these without conversions or shared-memory loads).
template <typename T>
inline CoefT<T> make_coefT(const Coef& c, const Geo& g, const double* dtheta) {
    CoefT<T> d;
    for (int s = 0; s < NS; ++s) {
        d.A[s] = T(c.A[s]);
        d.phase[s] = T(c.phase[s]);
    }
    for (int j = 0; j < 4; ++j) {
        d.chi0[j] = T(c.chi0[j]);
        d.chith[j] = T(c.chith[j]);
    }
    d.d1 = T(c.d1);
    d.d2 = T(c.d2);
    d.gamma = T(c.gamma);
    d.alpha1 = T(c.alpha1);
    d.alpha2 = T(c.alpha2);
    d.f1 = T(c.f1);
    d.k_ox = T(c.k_ox);
    d.beta1 = T(c.beta1);
    d.beta2 = T(c.beta2);
    d.sigma = T(c.sigma);
    d.c1s = T(c.c1s);
    d.c1ss = T(c.c1ss);
    d.bc_sign = T(c.bc_sign);
    for (int j = 0; j < 8; ++j) d.dth[j] = T(dtheta ? dtheta[j] : 0.0);
    d.vol = T(g.vol);
    d.inv_vol = T(1.0 / g.vol);
    for (int j = 0; j < 3; ++j) d.invh[j] = T(1.0 / g.h[j]);
    d.pen_c = T(g.pen_c);
    d.death1 = T(c.model == 1 ? 0.0 : 1.0);
    d.domain = nullptr;
    return d;
}

// Manufactured solution U*_s = 1 + cos(2 pi x + phase_s) cos(pi y / Ly) e^{-t} / 2
// and its forcing g = dU*/dt - (-div(F(U*) - A grad U*) + S(U*)), written out
// by hand: for chi-type fluxes n kappa(c) grad c with kappa(c) = a / (c + b),
// div(n kappa grad c) = kappa grad n . grad c + n kappa' |grad c|^2 + n kappa lap c.
template <typename T, typename C>
__device__ __forceinline__ void mms_forcing(T x, T y, T t, T Ly, const C& c, T g[NS]) {
    const T pi = T(3.14159265358979323846);
    const T et = exp(-t);
    const T ky = pi / Ly;
    const T Cy = cos(ky * y), Sy = sin(ky * y);
    T u[NS], ux[NS], uy[NS], lap[NS];
    for (int s = 0; s < NS; ++s) {
        const T arg = T(2) * pi * x + T(c.phase[s]);
        const T cx = cos(arg), sx = sin(arg);
        u[s] = T(1) + T(0.5) * cx * Cy * et;
        ux[s] = -pi * sx * Cy * et;
        uy[s] = -T(0.5) * cx * ky * Sy * et;
        lap[s] = -T(2) * pi * pi * cx * Cy * et - T(0.5) * cx * ky * ky * Cy * et;
    }
    auto div_chem = [&](int n, int cc, int j) -> T {
        const T a = T(c.chi0[j]), b = T(c.chith[j]);
        const T kap = a / (u[cc] + b);
        const T dkap = -a / ((u[cc] + b) * (u[cc] + b));
        const T gng = ux[n] * ux[cc] + uy[n] * uy[cc];
        const T gg = ux[cc] * ux[cc] + uy[cc] * uy[cc];
        return kap * gng + u[n] * dkap * gg + u[n] * kap * lap[cc];
    };
    T divF[NS] = {div_chem(0, 3, 0) + div_chem(0, 5, 1), div_chem(1, 3, 2) - div_chem(1, 0, 3), 0, 0, 0, 0};
    const T n1 = u[0], n2 = u[1], n3 = u[2], c1 = u[3], c2 = u[4];
    T S[NS];
    S[0] = -T(c.death1) * T(c.d1) * n1;
    S[1] = -T(c.d2) * n2;
    S[2] = T(c.d1) * n1 + T(c.d2) * n2 - T(c.gamma) * n1;
    S[3] = -T(c.alpha1) * n1 * c1 - T(c.alpha2) * n2 * c1 + T(c.f1) * n3;
    S[4] = -T(c.k_ox) * c2;
    S[5] = T(c.k_ox) * c2;
    for (int s = 0; s < NS; ++s) {
        const T ut = -(u[s] - T(1));
        const T rhs = -divF[s] + T(c.A[s]) * lap[s] + S[s];
        g[s] = ut - rhs;
    }
}

}  // namespace cdg2
