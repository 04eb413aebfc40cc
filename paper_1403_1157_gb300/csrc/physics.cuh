// Pointwise physics of the model (Sec. 2) at one quadrature point: the
// volume flux and source, the interior-face flux, their linearisations and
// adjoints, and the boundary data of Eq. (3).  Shared by the Cartesian
// operator (operator.cu) and the triangle operator (tri.cu).
#pragma once

#include "elem_common.cuh"

namespace cdg2 {

// ---------------------------------------------------------------------------
// Pointwise physics (Sec. 2)
// ---------------------------------------------------------------------------

// Sign test of a denominator without a floating-point compare (those run on
// the narrow FP64 pipe): the high word of an IEEE value is <= 0 exactly for
// negative values, zeros and the smallest subnormals.
__device__ __forceinline__ int hi_word(double x) { return __double2hiint(x); }
__device__ __forceinline__ int hi_word(float x) { return __float_as_int(x); }

// Denominators of the chemotactic sensitivities (Sec. 2) at one point:
// kappa11(c1), kappa13(c3), kappa21(c1), kappa22(n1) = chi0_i / den_i.
// chi(x, y, a, b) = a x / (y + b) has a pole at y + b = 0: a point with a
// denominator <= 0 lies outside the model's domain, and the kernel records
// it in the status word (the host returns CDG2_ERR_DOMAIN).
template <typename T>
__device__ __forceinline__ void kappa_den(const CoefT<T>& c, const T u[NS], T* den) {
    den[0] = u[3] + T(c.chith[0]);
    den[1] = u[5] + T(c.chith[1]);
    den[2] = u[3] + T(c.chith[2]);
    den[3] = u[0] + T(c.chith[3]);
    const int m = min(min(hi_word(den[0]), hi_word(den[1])), min(hi_word(den[2]), hi_word(den[3])));
    if (m <= 0 && c.domain != nullptr) atomicOr(c.domain, 1);
}

// Volume flux at one quadrature point (Eq. elementint): Phi_s = F_s(U, grad U)
// - A_s grad U_s and S(U) (Reading: the c1 row of S follows Eq. (1),
// -alpha1 n1 c1 - alpha2 n2 c1 + f1 n3).  death1 = 0 drops the n1 death term
// (the reduced model of Eq. (2), which keeps d1 n1 in the n3 equation).
// MODAL = 1: the diffusion of n2..c3 is applied elsewhere in modal form; only
// Phi_0 (with its diffusion) and the chemotactic part of Phi_1 are formed,
// and only the gradients of n1, c1, c3 are read.  MODAL = 2: the diffusion of
// n1 is modal too (Phi_0 is its chemotactic flux alone).
template <int D, typename T, int MODAL = 0>
__device__ __forceinline__ void volume_point(const CoefT<T>& c, const T u[NS], const T g[NS][D], T Phi[NS][D],
                                             T S[NS]) {
    T den[4], r[4];
    kappa_den<T>(c, u, den);
    recips<4, T>(den, r);
    const T k11 = T(c.chi0[0]) * r[0], k13 = T(c.chi0[1]) * r[1];
    const T k21 = T(c.chi0[2]) * r[2], k22 = T(c.chi0[3]) * r[3];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const T v1 = k11 * g[3][j] + k13 * g[5][j];
        const T v2 = k21 * g[3][j] - k22 * g[0][j];
        if constexpr (MODAL == 2)
            Phi[0][j] = u[0] * v1;
        else
            Phi[0][j] = u[0] * v1 - T(c.A[0]) * g[0][j];
        if constexpr (MODAL >= 1) {
            Phi[1][j] = u[1] * v2;
        } else {
            Phi[1][j] = u[1] * v2 - T(c.A[1]) * g[1][j];
#pragma unroll
            for (int s = 2; s < NS; ++s) Phi[s][j] = -T(c.A[s]) * g[s][j];
        }
    }
    const T n1 = u[0], n2 = u[1], n3 = u[2], c1 = u[3], c2 = u[4];
    S[0] = -c.death1 * c.d1 * n1;
    S[1] = -T(c.d2) * n2;
    S[2] = T(c.d1) * n1 + T(c.d2) * n2 - T(c.gamma) * n1;
    S[3] = -T(c.alpha1) * n1 * c1 - T(c.alpha2) * n2 * c1 + T(c.f1) * n3;
    S[4] = -T(c.k_ox) * c2;
    S[5] = T(c.k_ox) * c2;
}

// Linearisation of volume_point along (du, dg), plus the derivative of S
// along a tangent of the reaction coefficients (dth = d(d1, d2, gamma,
// alpha1, alpha2, f1, k_ox, .)), when has_dth.  With kappa = a / (c + b):
// d kappa = -kappa / (c + b) dc.
template <int D, typename T, int MODAL = 0>
__device__ __forceinline__ void volume_point_lin(const CoefT<T>& c, const T u[NS], const T g[NS][D], const T du[NS],
                                                 const T dg[NS][D], bool has_dth, T dPhi[NS][D],
                                                 T dS[NS]) {
    T den[4], r[4];
    kappa_den<T>(c, u, den);
    recips<4, T>(den, r);
    const T r11 = r[0], r13 = r[1], r21 = r[2], r22 = r[3];
    const T k11 = T(c.chi0[0]) * r11, k13 = T(c.chi0[1]) * r13;
    const T k21 = T(c.chi0[2]) * r21, k22 = T(c.chi0[3]) * r22;
    const T dk11 = -k11 * r11 * du[3], dk13 = -k13 * r13 * du[5];
    const T dk21 = -k21 * r21 * du[3], dk22 = -k22 * r22 * du[0];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const T v1 = k11 * g[3][j] + k13 * g[5][j];
        const T v2 = k21 * g[3][j] - k22 * g[0][j];
        const T dv1 = dk11 * g[3][j] + k11 * dg[3][j] + dk13 * g[5][j] + k13 * dg[5][j];
        const T dv2 = dk21 * g[3][j] + k21 * dg[3][j] - dk22 * g[0][j] - k22 * dg[0][j];
        if constexpr (MODAL == 2)
            dPhi[0][j] = du[0] * v1 + u[0] * dv1;
        else
            dPhi[0][j] = du[0] * v1 + u[0] * dv1 - T(c.A[0]) * dg[0][j];
        if constexpr (MODAL >= 1) {
            dPhi[1][j] = du[1] * v2 + u[1] * dv2;
        } else {
            dPhi[1][j] = du[1] * v2 + u[1] * dv2 - T(c.A[1]) * dg[1][j];
#pragma unroll
            for (int s = 2; s < NS; ++s) dPhi[s][j] = -T(c.A[s]) * dg[s][j];
        }
    }
    dS[0] = -c.death1 * c.d1 * du[0];
    dS[1] = -T(c.d2) * du[1];
    dS[2] = T(c.d1) * du[0] + T(c.d2) * du[1] - T(c.gamma) * du[0];
    dS[3] = -T(c.alpha1) * (du[0] * u[3] + u[0] * du[3]) - T(c.alpha2) * (du[1] * u[3] + u[1] * du[3]) +
            T(c.f1) * du[2];
    dS[4] = -T(c.k_ox) * du[4];
    dS[5] = T(c.k_ox) * du[4];
    if (has_dth) {
        const T n1 = u[0], n2 = u[1], n3 = u[2], c1 = u[3], c2 = u[4];
        dS[0] += -c.death1 * c.dth[0] * n1;
        dS[1] += -c.dth[1] * n2;
        dS[2] += c.dth[0] * n1 + c.dth[1] * n2 - c.dth[2] * n1;
        dS[3] += -c.dth[3] * n1 * c1 - c.dth[4] * n2 * c1 + c.dth[5] * n3;
        dS[4] += -c.dth[6] * c2;
        dS[5] += c.dth[6] * c2;
    }
}

// Interior-face flux at one face point (Eq. surfaceint), n^- = +e_a, with the
// jump Delta = U^- - U^+ passed in (formed from coefficient differences):
//   sigma_s = A_s {d_n U_s} - F^_s.n^- + A^_s.n^-   (multiplies phi^- - phi^+)
//   tau_s   = A_s Delta_s / 2                       (multiplies d_n phi^- + d_n phi^+)
// F^ local Lax-Friedrichs with lambda_s = max(|v_s^-.n|, |v_s^+.n|);
// A^ = 2 chi_e A r_e on K^-, r_e.n^- = -(k+1)^2 Delta / (2 h_a).
template <typename T>
__device__ __forceinline__ void face_point(const CoefT<T>& c, T pen, const T uM[NS], const T dM[NS], const T uP[NS],
                                           const T dP[NS], const T del[NS], T sig[NS], T tau[NS]) {
    T Fh[2];
    T den[8], r[8];   // K^- side, then K^+ side
    kappa_den<T>(c, uM, den);
    kappa_den<T>(c, uP, den + 4);
    recips<8, T>(den, r);
    {
        const T vM = T(c.chi0[0]) * r[0] * dM[3] + T(c.chi0[1]) * r[1] * dM[5];
        const T vP = T(c.chi0[0]) * r[4] * dP[3] + T(c.chi0[1]) * r[5] * dP[5];
        const T lam = fmax(fabs(vM), fabs(vP));
        Fh[0] = T(0.5) * (uM[0] * vM + uP[0] * vP) + T(0.5) * lam * del[0];
    }
    {
        const T vM = T(c.chi0[2]) * r[2] * dM[3] - T(c.chi0[3]) * r[3] * dM[0];
        const T vP = T(c.chi0[2]) * r[6] * dP[3] - T(c.chi0[3]) * r[7] * dP[0];
        const T lam = fmax(fabs(vM), fabs(vP));
        Fh[1] = T(0.5) * (uM[1] * vM + uP[1] * vP) + T(0.5) * lam * del[1];
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const T A = T(c.A[s]);
        T sg = A * T(0.5) * (dM[s] + dP[s]) - pen * A * del[s];
        if (s < 2) sg -= Fh[s];
        sig[s] = sg;
        tau[s] = T(0.5) * A * del[s];
    }
}

template <typename T>
__device__ __forceinline__ T sgn0(T x) {
    return x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0));
}

// One side's chemotactic normal velocity of species 0 or 1 and its derivative:
// v_0 = kappa11(c1) d_n c1 + kappa13(c3) d_n c3,  v_1 = kappa21(c1) d_n c1 - kappa22(n1) d_n n1,
// with rk the reciprocals of that side's kappa_den.
template <typename T>
__device__ __forceinline__ void velocity_lin(const CoefT<T>& c, int sp, const T* rk, const T dn[NS], const T du[NS],
                                             const T ddn[NS], T& v, T& dv) {
    if (sp == 0) {
        const T r1 = rk[0], r3 = rk[1];
        const T k1 = T(c.chi0[0]) * r1, k3 = T(c.chi0[1]) * r3;
        v = k1 * dn[3] + k3 * dn[5];
        dv = -k1 * r1 * du[3] * dn[3] + k1 * ddn[3] - k3 * r3 * du[5] * dn[5] + k3 * ddn[5];
    } else {
        const T r1 = rk[2], r0 = rk[3];
        const T k1 = T(c.chi0[2]) * r1, k0 = T(c.chi0[3]) * r0;
        v = k1 * dn[3] - k0 * dn[0];
        dv = -k1 * r1 * du[3] * dn[3] + k1 * ddn[3] + k0 * r0 * du[0] * dn[0] - k0 * ddn[0];
    }
}

// Linearisation of face_point along the tangent traces.  Reading: d|x|/dx =
// sign(x) with sign(0) = 0; at a tie |v^-| = |v^+| the K^- side is taken.
template <typename T>
__device__ __forceinline__ void face_point_lin(const CoefT<T>& c, T pen, const T uM[NS], const T dM[NS], const T uP[NS],
                                               const T dP[NS], const T del[NS], const T duM[NS], const T ddM[NS],
                                               const T duP[NS], const T ddP[NS], const T ddel[NS], T dsig[NS],
                                               T dtau[NS]) {
    T dFh[2];
    T den[8], r[8];   // K^- side, then K^+ side
    kappa_den<T>(c, uM, den);
    kappa_den<T>(c, uP, den + 4);
    recips<8, T>(den, r);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
        T vM, dvM, vP, dvP;
        velocity_lin<T>(c, sp, r, dM, duM, ddM, vM, dvM);
        velocity_lin<T>(c, sp, r + 4, dP, duP, ddP, vP, dvP);
        const T aM = fabs(vM), aP = fabs(vP);
        const bool takeM = aM >= aP;
        const T lam = takeM ? aM : aP;
        const T dlam = takeM ? sgn0(vM) * dvM : sgn0(vP) * dvP;
        dFh[sp] = T(0.5) * (duM[sp] * vM + uM[sp] * dvM + duP[sp] * vP + uP[sp] * dvP) +
                  T(0.5) * (dlam * del[sp] + lam * ddel[sp]);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const T A = T(c.A[s]);
        T sg = A * T(0.5) * (ddM[s] + ddP[s]) - pen * A * ddel[s];
        if (s < 2) sg -= dFh[s];
        dsig[s] = sg;
        dtau[s] = T(0.5) * A * ddel[s];
    }
}

// Adjoint of volume_point: given the weighted cotangents sb = W mu (of S) and
// gb[s][j] = W d_j mu (of Phi_s,j), the cotangents of the inputs,
//   ub_t = sum_s sb_s dS_s/du_t + sum_{s,j} gb_sj dPhi_sj/du_t,
//   Gb_tj = sum_s gb_sj dPhi_sj/dg_tj,
// and th[0..6] += the cotangents of (d1, d2, gamma, alpha1, alpha2, f1, k_ox).
template <int D, typename T>
__device__ __forceinline__ void volume_point_adj(const CoefT<T>& c, const T u[NS], const T g[NS][D], const T sb[NS],
                                                 const T gb[NS][D], T ub[NS], T Gb[NS][D], T th[8]) {
    T den[4], r[4];
    kappa_den<T>(c, u, den);
    recips<4, T>(den, r);
    const T r11 = r[0], r13 = r[1], r21 = r[2], r22 = r[3];
    const T k11 = T(c.chi0[0]) * r11, k13 = T(c.chi0[1]) * r13;
    const T k21 = T(c.chi0[2]) * r21, k22 = T(c.chi0[3]) * r22;
#pragma unroll
    for (int s = 0; s < NS; ++s) ub[s] = T(0);
    T kb11 = 0, kb13 = 0, kb21 = 0, kb22 = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const T v1 = k11 * g[3][j] + k13 * g[5][j];
        const T v2 = k21 * g[3][j] - k22 * g[0][j];
        ub[0] += gb[0][j] * v1;
        ub[1] += gb[1][j] * v2;
        const T vb1 = gb[0][j] * u[0];
        const T vb2 = gb[1][j] * u[1];
#pragma unroll
        for (int s = 0; s < NS; ++s) Gb[s][j] = -T(c.A[s]) * gb[s][j];
        Gb[3][j] += vb1 * k11 + vb2 * k21;
        Gb[5][j] += vb1 * k13;
        Gb[0][j] -= vb2 * k22;
        kb11 += vb1 * g[3][j];
        kb13 += vb1 * g[5][j];
        kb21 += vb2 * g[3][j];
        kb22 -= vb2 * g[0][j];
    }
    ub[3] += -k11 * r11 * kb11 - k21 * r21 * kb21;
    ub[5] += -k13 * r13 * kb13;
    ub[0] += -k22 * r22 * kb22;
    // reaction source
    ub[0] += -c.death1 * c.d1 * sb[0] + (T(c.d1) - T(c.gamma)) * sb[2] - T(c.alpha1) * u[3] * sb[3];
    ub[1] += -T(c.d2) * sb[1] + T(c.d2) * sb[2] - T(c.alpha2) * u[3] * sb[3];
    ub[2] += T(c.f1) * sb[3];
    ub[3] += (-T(c.alpha1) * u[0] - T(c.alpha2) * u[1]) * sb[3];
    ub[4] += -T(c.k_ox) * sb[4] + T(c.k_ox) * sb[5];
    th[0] += u[0] * (sb[2] - c.death1 * sb[0]);
    th[1] += u[1] * (sb[2] - sb[1]);
    th[2] += -u[0] * sb[2];
    th[3] += -u[0] * u[3] * sb[3];
    th[4] += -u[1] * u[3] * sb[3];
    th[5] += u[2] * sb[3];
    th[6] += u[4] * (sb[5] - sb[4]);
}

// Adjoint of face_point with respect to the traces of one side X (the own
// cell: K^- when ownM, else K^+), given the cotangents sb = W (mu^- - mu^+)
// of sigma and tb = W (d_n mu^- + d_n mu^+) of tau.  Returns the cotangents
// of X's value trace (ub) and normal-derivative trace (db).  Delta depends on
// both sides: dDelta/du^X = +1 for K^-, -1 for K^+.  Same derivative
// conventions as face_point_lin.
template <typename T>
__device__ __forceinline__ void face_point_adj(const CoefT<T>& c, T pen, bool ownM, const T uM[NS], const T dM[NS],
                                               const T uP[NS], const T dP[NS], const T del[NS], const T sb[NS],
                                               const T tb[NS], T ub[NS], T db[NS]) {
    const T sX = ownM ? T(1) : T(-1);
    const T* uX = ownM ? uM : uP;
    const T* dX = ownM ? dM : dP;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        ub[s] = sX * T(c.A[s]) * (T(0.5) * tb[s] - pen * sb[s]);
        db[s] = T(0.5) * T(c.A[s]) * sb[s];
    }
    T den[8], r[8];   // K^- side, then K^+ side
    kappa_den<T>(c, uM, den);
    kappa_den<T>(c, uP, den + 4);
    recips<8, T>(den, r);
    const T* rX = ownM ? r : r + 4;
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
        T vM, vP, dummy;
        const T zero[NS] = {0, 0, 0, 0, 0, 0};
        velocity_lin<T>(c, sp, r, dM, zero, zero, vM, dummy);
        velocity_lin<T>(c, sp, r + 4, dP, zero, zero, vP, dummy);
        const bool takeM = fabs(vM) >= fabs(vP);
        const T lam = takeM ? fabs(vM) : fabs(vP);
        const T vX = ownM ? vM : vP;
        const bool fromX = ownM ? takeM : !takeM;
        const T Fb = -sb[sp];                       // sigma_sp contains -F^_sp
        ub[sp] += Fb * (T(0.5) * vX + T(0.5) * lam * sX);
        const T vb = Fb * (T(0.5) * uX[sp] + (fromX ? T(0.5) * del[sp] * sgn0(vX) : T(0)));
        if (sp == 0) {
            const T r1 = rX[0], r3 = rX[1];
            const T k1 = T(c.chi0[0]) * r1, k3 = T(c.chi0[1]) * r3;
            ub[3] += vb * (-k1 * r1 * dX[3]);
            ub[5] += vb * (-k3 * r3 * dX[5]);
            db[3] += vb * k1;
            db[5] += vb * k3;
        } else {
            const T r1 = rX[2], r0 = rX[3];
            const T k1 = T(c.chi0[2]) * r1, k0 = T(c.chi0[3]) * r0;
            ub[3] += vb * (-k1 * r1 * dX[3]);
            ub[0] += vb * (k0 * r0 * dX[0]);
            db[3] += vb * k1;
            db[0] -= vb * k0;
        }
    }
}

// Boundary data of Eq. (3) at one face point of the own cell (Reading: the
// normal is inward, so the data are influxes times bc_sign):
// Gamma_1 (y = 0): n1 mu1 beta1 H(c1 - c1*), c2 nu2 sigma on Gamma_{1,in};
// Gamma_2 (y = L1): n2 mu2 beta2 H(c1 - c1**).  H(0) = 0.  With beta1 scaled
// by `b1` (1 for the data, the tangent d beta1 for their derivative).
template <typename T>
__device__ __forceinline__ void boundary_point(const CoefT<T>& c, int f, T x, const Geo& g, const T uo[NS], T sig[NS],
                                               T b1, bool other_terms) {
#pragma unroll
    for (int s = 0; s < NS; ++s) sig[s] = T(0);
    const T bs = T(c.bc_sign);
    if (f == 0) {
        sig[0] = (uo[3] - T(c.c1s) > T(0)) ? bs * T(c.A[0]) * b1 : T(0);
        if (other_terms)
            sig[4] = (x >= T(g.g1in[0]) && x <= T(g.g1in[1])) ? bs * T(c.A[4]) * T(c.sigma) : T(0);
    } else if (other_terms) {
        sig[1] = (uo[3] - T(c.c1ss) > T(0)) ? bs * T(c.A[1]) * T(c.beta2) : T(0);
    }
}

}  // namespace cdg2
