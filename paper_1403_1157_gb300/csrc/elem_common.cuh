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

// 1D tables in shared memory in the kernel's precision.
template <int K, typename T>
struct STab {
    T B[K + 2][K + 1];   // psi_a(xi_q)
    T D[K + 2][K + 1];   // psi'_a(xi_q)
    T w[K + 2];
    T xi[K + 2];
    T e[2][K + 1];       // psi_a(0), psi_a(1)
    T d[2][K + 1];       // psi'_a(0), psi'_a(1)
};

template <int K, typename T>
__device__ __forceinline__ void load_tab(STab<K, T>& s, const Tab1D& t) {
    for (int i = threadIdx.x; i < (K + 2) * (K + 1); i += blockDim.x) {
        int q = i / (K + 1), a = i % (K + 1);
        s.B[q][a] = (T)t.B[q][a];
        s.D[q][a] = (T)t.D[q][a];
    }
    for (int i = threadIdx.x; i < K + 2; i += blockDim.x) {
        s.w[i] = (T)t.w[i];
        s.xi[i] = (T)t.xi[i];
    }
    for (int i = threadIdx.x; i < 2 * (K + 1); i += blockDim.x) {
        int f = i / (K + 1), a = i % (K + 1);
        s.e[f][a] = (T)t.e[f][a];
        s.d[f][a] = (T)t.d[f][a];
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

template <typename T>
struct Ident {
    using type = T;
};

// One sum-factorisation pass over nt tensors stored back to back.
// Input tensors have extents (I0, I1, I2) (x fastest); axis AX (extent NI)
// is replaced by NO in the output:
//     out[t][..o..] = sum_i M1(o,i) in1[t][..i..]  (+ M2(o,i) in2[t][..i..])
// M(o,i) = M[o][i] (TR = false) or M[i][o] (TR = true), row length LD.
// One thread computes one whole line along AX: its index arithmetic is done
// once per line, the 1D matrices are held in registers, and each input is
// loaded once for NO outputs (shared-memory traffic, not FMA issue, limits
// these passes).  The sums run over i in increasing order.
template <int AX, int I0, int I1, int I2, int NO, bool TR, int LD, bool TWO, typename T>
__device__ __forceinline__ void sf_pass(const T* __restrict__ in1, const T* __restrict__ M1,
                                        const typename Ident<T>::type* __restrict__ in2,
                                        const typename Ident<T>::type* __restrict__ M2, int in_stride,
                                        T* __restrict__ out, int out_stride, int nt) {
    constexpr int NI = AX == 0 ? I0 : (AX == 1 ? I1 : I2);
    constexpr int NL = I0 * I1 * I2 / NI;                       // lines per tensor
    constexpr int ST = AX == 0 ? 1 : (AX == 1 ? I0 : I0 * I1);  // stride along AX (input and output)
    T m1[NO][NI], m2[TWO ? NO : 1][TWO ? NI : 1];
#pragma unroll
    for (int o = 0; o < NO; ++o)
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            m1[o][i] = TR ? M1[i * LD + o] : M1[o * LD + i];
            if constexpr (TWO) m2[o][i] = TR ? M2[i * LD + o] : M2[o * LD + i];
        }
    const int total = nt * NL;
    for (int line = threadIdx.x; line < total; line += blockDim.x) {
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
        const T* s1 = in1 + tt * in_stride + ib;
        T v1[NI], v2[TWO ? NI : 1];
#pragma unroll
        for (int i = 0; i < NI; ++i) v1[i] = s1[i * ST];
        if constexpr (TWO) {
            const T* s2 = in2 + tt * in_stride + ib;
#pragma unroll
            for (int i = 0; i < NI; ++i) v2[i] = s2[i * ST];
        }
        T* d = out + tt * out_stride + ob;
#pragma unroll
        for (int o = 0; o < NO; ++o) {
            T acc = T(0);
#pragma unroll
            for (int i = 0; i < NI; ++i) acc = fma(m1[o][i], v1[i], acc);
            if constexpr (TWO) {
#pragma unroll
                for (int i = 0; i < NI; ++i) acc = fma(m2[o][i], v2[i], acc);
            }
            d[o * ST] = acc;
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

// Neighbour of element e across face f (0: low side, 1: high side) of axis
// a; -1 on a non-periodic boundary.
__device__ __forceinline__ long long neighbour(const Geo& g, long long e, int a, int f) {
    long long ix = e % g.n[0];
    long long r = e / g.n[0];
    long long iy = r % g.n[1];
    long long iz = r / g.n[1];
    long long c[3] = {ix, iy, iz};
    long long v = c[a] + (f ? 1 : -1);
    if (v < 0 || v >= g.n[a]) {
        if (!g.periodic[a]) return -1;
        v = (v + g.n[a]) % g.n[a];
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
