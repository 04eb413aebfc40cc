// The CDG2 operator on triangle meshes (Sec. 3.1: P_k on triangles, chi_e =
// 1.5): f(U) = M^{-1} L_h(U) in FP64, face-once.
//
// Readings (shared with the oracle; the paper fixes none of them):
//  * basis: on the reference triangle T = {xi, eta >= 0, xi + eta <= 1} the
//    orthonormal Dubiner basis psi_pq = c_pq L_p(xi, eta) P_q^{(2p+1,0)}(2 eta
//    - 1), L_p = (1 - eta)^p P_p(2 xi / (1 - eta) - 1), c_pq = sqrt(2 (2p+1)
//    (p+q+1)), modes ordered by p + q then q; element e uses psi o F_e^{-1}
//    with F_e(xi) = x_0 + J_e xi, so M_K = det J_e I;
//  * quadrature: the collapsed Gauss rule, xi = u (1 - v), eta = v with k+2
//    Gauss points per direction (u fastest), weight w_u w_v (1 - v); k+2
//    Gauss points per edge;
//  * K^-_e: the adjacent element with the smaller area (Sec. 3.1), areas
//    within a relative 1e-12 tie and a tie goes to the lower index;
//  * boundary edges on y = 0 are Gamma_1, on y = max y Gamma_2 (Eq. (3));
//    every other boundary edge is a no-flow wall.
// The CDG2 flux needs r_e([U]) . n^- on K^-: with M_{K^-} = det I the
// lifting identity gives r . n (x_p) = -(|e| / (2 det_-)) sum_p' L[p][p']
// Delta(x_p'), L[p][p'] = sum_i psi_i(x_p) psi_i(x_p') w_p', tabulated per
// local edge of K^-.  Face points are listed in K^-'s orientation of the
// edge; K^+ runs the edge the other way (both counter-clockwise), so its
// point p is its own edge point k+1-p (the Gauss rule is symmetric).
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "physics.cuh"
#include "simplex_elem.cuh"
#include "simplex_host.h"
#include "simplex_step.h"

namespace cdg2 {

constexpr int TMAXB = 10;   // basis functions for k = 3
constexpr int TMAXQ = 25;   // volume points for k = 3
constexpr int TMAXP = 5;    // edge points for k = 3

// Tables in FP64 (device copy staged into shared memory by the kernels).
struct TriTab {
    double VB[TMAXQ][TMAXB];          // psi_i at the volume points
    double VD[2][TMAXQ][TMAXB];       // d psi_i / d xi, d eta
    double VW[TMAXQ];
    double VX[TMAXQ][2];              // reference volume points
    double EB[3][TMAXP][TMAXB];       // psi_i at edge l's points (t ascending from vertex l)
    double ED[2][3][TMAXP][TMAXB];
    double EW[TMAXP];
    double ET[TMAXP];
    double LF[3][TMAXP][TMAXP];       // lifting kernel of K^-'s edge l
    // Warped-product factors on the collapsed volume grid: at xi = u (1-v),
    // eta = v, psi_pq = A_p(u) B_pq(v) with A_p = P_p(2u-1) and
    // B_pq = c_pq (1-v)^p P_q^{(2p+1,0)}(2v-1); mode m = (p+q)(p+q+1)/2 + q.
    double SA[TMAXP][TMAXP], SdA[TMAXP][TMAXP];   // [u point][p]
    double SB[TMAXP][TMAXB], SdB[TMAXP][TMAXB];   // [v point][mode]
    // d_xi = a1 d_u, d_eta = u a1 d_u + d_v with a1 = 1 / (1-v): (a1, u a1) per point
    double SG[TMAXQ][2];
    // reference stiffness matrices, exact under the volume rule: KS[c][i][j] =
    // sum_q w_q d_a psi_i d_b psi_j for c = (a, b) in {00, 11}, and that plus its
    // transpose for c = 01; so that int_K grad psi_i . grad psi_j = det J sum_c
    // G_c KS[c][i][j] with G = J^{-1} J^{-T}
    double KS[3][TMAXB][TMAXB];
};

// Element geometry: x0, y0, J (row-major), J^{-1} (row-major), det J.
constexpr int GEO = 11;

}  // namespace cdg2

struct cdg2_tri_mesh {
    int k = 0, nb = 0, nq = 0, np = 0;
    long long E = 0, NF = 0;
    double chi_e = 1.5, ly = 0.0;
    double g1in[2] = {0.375, 0.625};
    std::vector<double> geo;     // [E][GEO]
    std::vector<int> emap;       // [E][3]: 2 face + side (0: K^-, 1: K^+), or -1 - tag (0 wall, 1 Gamma_1, 2 Gamma_2)
    std::vector<int> face;       // [NF][4]: eM, eP, lM, lP
    std::vector<double> fgeo;    // [NF][4]: n_x, n_y, |e|, det J of K^-
    cdg2::TriTab tab;
    // device copies, uploaded by the first apply (calls on one mesh must be ordered on one stream)
    mutable double* d_geo = nullptr;
    mutable int* d_emap = nullptr;
    mutable int* d_face = nullptr;
    mutable double* d_fgeo = nullptr;
    mutable cdg2::TriTab* d_tab = nullptr;
    mutable double* d_fbuf = nullptr;   // [NF][2][6][nb] tested face fluxes
    mutable void* step_ws = nullptr;    // cdg2_tri_step workspace
    mutable size_t step_ws_bytes = 0;
    mutable cdg2::SimplexPrecond spc;   // element-block Jacobi of the step
    mutable int* status = nullptr;      // domain status word (device int)
};

namespace cdg2 {

namespace {

// psi_i and its reference gradient at (xi, eta).
void dubiner(int k, double xi, double eta, double* psi, double* dxi, double* deta) {
    const double s = 1.0 - eta, xt = 2.0 * xi - s;
    double L[4], Lx[4], Ly[4];
    L[0] = 1.0;
    Lx[0] = 0.0;
    Ly[0] = 0.0;
    if (k >= 1) {
        L[1] = xt;
        Lx[1] = 2.0;
        Ly[1] = 1.0;
    }
    for (int p = 2; p <= k; ++p) {
        L[p] = ((2 * p - 1) * xt * L[p - 1] - (p - 1) * s * s * L[p - 2]) / p;
        Lx[p] = ((2 * p - 1) * (2.0 * L[p - 1] + xt * Lx[p - 1]) - (p - 1) * s * s * Lx[p - 2]) / p;
        Ly[p] = ((2 * p - 1) * (L[p - 1] + xt * Ly[p - 1]) - (p - 1) * (-2.0 * s * L[p - 2] + s * s * Ly[p - 2])) / p;
    }
    int i = 0;
    for (int d = 0; d <= k; ++d)
        for (int q = 0; q <= d; ++q, ++i) {
            const int p = d - q;
            const double c = std::sqrt(2.0 * (2 * p + 1) * (p + q + 1));
            double J, dJ;
            jacobi_d(q, 2.0 * p + 1.0, 2.0 * eta - 1.0, J, dJ);
            psi[i] = c * L[p] * J;
            dxi[i] = c * Lx[p] * J;
            deta[i] = c * (Ly[p] * J + L[p] * 2.0 * dJ);
        }
}

void ref_edge_point(int l, double t, double& xi, double& eta) {
    if (l == 0) {
        xi = t;
        eta = 0.0;
    } else if (l == 1) {
        xi = 1.0 - t;
        eta = t;
    } else {
        xi = 0.0;
        eta = 1.0 - t;
    }
}

void build_tables(int k, TriTab& T) {
    std::memset(&T, 0, sizeof(T));
    const int n = k + 2;
    double g[16], w[16];
    gauss01(n, g, w);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const int q = i + n * j;
            const double xi = g[i] * (1.0 - g[j]), eta = g[j];
            T.VX[q][0] = xi;
            T.VX[q][1] = eta;
            T.VW[q] = w[i] * w[j] * (1.0 - g[j]);
            dubiner(k, xi, eta, T.VB[q], T.VD[0][q], T.VD[1][q]);
        }
    for (int j = 0; j < n; ++j) {
        for (int p = 0; p <= k; ++p) {
            double P, dP;
            jacobi_d(p, 0.0, 2.0 * g[j] - 1.0, P, dP);
            T.SA[j][p] = P;
            T.SdA[j][p] = 2.0 * dP;
        }
        int m = 0;
        for (int d = 0; d <= k; ++d)
            for (int q = 0; q <= d; ++q, ++m) {
                const int p = d - q;
                const double c = std::sqrt(2.0 * (2 * p + 1) * (p + q + 1)), v1 = 1.0 - g[j];
                double Q, dQ;
                jacobi_d(q, 2.0 * p + 1.0, 2.0 * g[j] - 1.0, Q, dQ);
                const double pw = std::pow(v1, p), dpw = p > 0 ? -p * std::pow(v1, p - 1) : 0.0;
                T.SB[j][m] = c * pw * Q;
                T.SdB[j][m] = c * (dpw * Q + pw * 2.0 * dQ);
            }
        for (int i = 0; i < n; ++i) {
            const double a1 = 1.0 / (1.0 - g[j]);
            T.SG[i + n * j][0] = a1;
            T.SG[i + n * j][1] = g[i] * a1;
        }
    }
    for (int p = 0; p < n; ++p) {
        T.EW[p] = w[p];
        T.ET[p] = g[p];
    }
    const int nb = (k + 1) * (k + 2) / 2;
    {
        const int PA[3] = {0, 1, 0}, PB[3] = {0, 1, 1};
        for (int c = 0; c < 3; ++c)
            for (int i = 0; i < nb; ++i)
                for (int j = 0; j < nb; ++j) {
                    double acc = 0.0;
                    for (int q = 0; q < n * n; ++q) {
                        double v = T.VD[PA[c]][q][i] * T.VD[PB[c]][q][j];
                        if (PA[c] != PB[c]) v += T.VD[PB[c]][q][i] * T.VD[PA[c]][q][j];
                        acc += T.VW[q] * v;
                    }
                    T.KS[c][i][j] = acc;
                }
    }
    for (int l = 0; l < 3; ++l) {
        for (int p = 0; p < n; ++p) {
            double xi, eta;
            ref_edge_point(l, g[p], xi, eta);
            dubiner(k, xi, eta, T.EB[l][p], T.ED[0][l][p], T.ED[1][l][p]);
        }
        for (int p = 0; p < n; ++p)
            for (int pp = 0; pp < n; ++pp) {
                double acc = 0.0;
                for (int i = 0; i < nb; ++i) acc += T.EB[l][p][i] * T.EB[l][pp][i];
                T.LF[l][p][pp] = acc * w[pp];
            }
    }
}

}  // namespace

}  // namespace cdg2

namespace cdg2 {

template <int K>
struct TriShape {
    static constexpr int NB = (K + 1) * (K + 2) / 2;
    static constexpr int NQ = (K + 2) * (K + 2);
    static constexpr int NP = K + 2;
};

struct TriArgs {
    const double* U;
    const double* dU;    // JVP: the tangent
    double* out;
    int flags;
    double chi_e;
    long long E, NF;
    const double* geo;
    const int* emap;
    const int* face;
    const double* fgeo;
    const TriTab* tab;
    double* fbuf;
    Geo g;               // only g1in is read (Gamma_{1,in})
    CoefT<double> c;
};

__device__ __forceinline__ void load_tritab(TriTab& s, const TriTab* t) {
    const double* src = reinterpret_cast<const double*>(t);
    double* dst = reinterpret_cast<double*>(&s);
    for (int i = threadIdx.x; i < (int)(sizeof(TriTab) / sizeof(double)); i += blockDim.x) dst[i] = src[i];
}

constexpr int TRI_APPLY = 0, TRI_JVP = 1, TRI_VJP = 2;

// One CTA: FPB interior edges.  Traces of both sides, the K^- lifting, the
// face flux of Eq. surfaceint per point (JVP: its linearisation along the
// tangent; the lifting is linear), and its test against both sides' basis;
// the tested fluxes go to the face buffer ([face][side][6][nb]).  VJP: with
// mu = M^{-1} lambda (or lambda) the cotangents of sigma and tau at point p
// are |e| w_p (mu^- - mu^+) and |e| w_p (d_n mu^- + d_n mu^+); they go back
// through face_point (face_point_adj, per side) and the lifting (its
// transpose), and each side's trace cotangents are tested into the buffer.
template <int K, int FPB, int MODE>
__global__ void __launch_bounds__(128) tri_face_kernel(const TriArgs a) {
    using S = TriShape<K>;
    constexpr int NB = S::NB, NP = S::NP, F = MODE == TRI_APPLY ? 1 : 2;
    __shared__ TriTab tb;
    __shared__ double sU[FPB][2][F][NS][NB];
    __shared__ double sM[FPB][2][2];         // J^{-1} n^- of each side: n^- . J^{-T} g = (J^{-1} n^-) . g
    __shared__ double sF[FPB][4];            // n_x, n_y, |e|, det_-
    __shared__ int sI[FPB][4];               // eM, eP, lM, lP
    __shared__ double sT[FPB][2][F][2][NS][NP];  // [side][field][value, normal derivative][s][p]
    __shared__ double sDN[FPB][2][NP][NB];    // n^- . grad phi_m of each side at the face points
    __shared__ double sD[MODE == TRI_VJP ? 1 : FPB][NS][NP];  // jump of the last field (the lifted one)
    __shared__ double sS[FPB][2][NS][NP];     // w_p sigma, w_p tau (VJP: the cotangents of sigma, tau)
    __shared__ double sA[MODE == TRI_VJP ? FPB : 1][2][2][NS][NP];   // VJP: [side][value, d_n] trace cotangents
    __shared__ double sDet[FPB][2];
    load_tritab(tb, a.tab);
    const long long f0 = (long long)blockIdx.x * FPB;
    const int nf = (int)min((long long)FPB, a.NF - f0);
    for (int i = threadIdx.x; i < nf * 4; i += blockDim.x) {
        const int j = i / 4, c = i % 4;
        sI[j][c] = a.face[(f0 + j) * 4 + c];
        sF[j][c] = a.fgeo[(f0 + j) * 4 + c];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nf * 2; i += blockDim.x) {
        const int j = i / 2, side = i % 2;
        const double* Ji = a.geo + (long long)sI[j][side] * GEO + 6;
        sM[j][side][0] = fma(Ji[0], sF[j][0], Ji[1] * sF[j][1]);
        sM[j][side][1] = fma(Ji[2], sF[j][0], Ji[3] * sF[j][1]);
        sDet[j][side] = Ji[4];
    }
    for (int i = threadIdx.x; i < nf * 2 * F * NS * NB; i += blockDim.x) {
        const int j = i / (2 * F * NS * NB), side = (i / (F * NS * NB)) % 2, fi = (i / (NS * NB)) % F;
        const int r = i % (NS * NB);
        sU[j][side][fi][r / NB][r % NB] = (fi ? a.dU : a.U)[(long long)sI[j][side] * NS * NB + r];
    }
    __syncthreads();   // sM, sDet and sU are read by other threads below
    // normal derivatives of the basis at the face points (K^-'s order; K^+ reads its edge reversed)
    for (int i = threadIdx.x; i < nf * 2 * NP * NB; i += blockDim.x) {
        const int j = i / (2 * NP * NB), side = (i / (NP * NB)) % 2, p = (i / NB) % NP, m = i % NB;
        const int l = sI[j][2 + side];
        const int pp = side ? NP - 1 - p : p;
        sDN[j][side][p][m] = fma(sM[j][side][0], tb.ED[0][l][pp][m], sM[j][side][1] * tb.ED[1][l][pp][m]);
    }
    __syncthreads();
    // traces of both sides at the face points, and the jump of the last field
    for (int i = threadIdx.x; i < nf * F * NS * NP; i += blockDim.x) {
        const int j = i / (F * NS * NP), fi = (i / (NS * NP)) % F;
        const int s = (i / NP) % NS, p = i % NP;
        double val[2];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int l = sI[j][2 + side];
            const int pp = side ? NP - 1 - p : p;
            double v = 0.0, dn = 0.0;
#pragma unroll
            for (int m = 0; m < NB; ++m) {
                const double u = sU[j][side][fi][s][m];
                v = fma(tb.EB[l][pp][m], u, v);
                dn = fma(sDN[j][side][p][m], u, dn);
            }
            // VJP: the cotangent field enters as mu = M^{-1} lambda = lambda / det J (with CDG2_MINV)
            const double sc = (MODE == TRI_VJP && fi == 1 && (a.flags & CDG2_MINV)) ? 1.0 / sDet[j][side] : 1.0;
            val[side] = v * sc;
            sT[j][side][fi][0][s][p] = v * sc;
            sT[j][side][fi][1][s][p] = dn * sc;
        }
        if constexpr (MODE != TRI_VJP) {
            if (fi == F - 1) sD[j][s][p] = val[0] - val[1];
        }
    }
    __syncthreads();
    if constexpr (MODE == TRI_VJP) {
        // cotangents of sigma and tau at every face point
        for (int i = threadIdx.x; i < nf * NS * NP; i += blockDim.x) {
            const int j = i / (NS * NP), s = (i / NP) % NS, p = i % NP;
            const double W = sF[j][2] * tb.EW[p];
            sS[j][0][s][p] = W * (sT[j][0][1][0][s][p] - sT[j][1][1][0][s][p]);
            sS[j][1][s][p] = W * (sT[j][0][1][1][s][p] + sT[j][1][1][1][s][p]);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nf * NP; i += blockDim.x) {
            const int j = i / NP, q = i % NP;
            const int lM = sI[j][2];
            const double lift = -sF[j][2] / (2.0 * sF[j][3]);
            double uM[NS], dM[NS], uP[NS], dP[NS], del[NS], sb[NS], tbb[NS], ub[NS], db[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                uM[s] = sT[j][0][0][0][s][q];
                dM[s] = sT[j][0][0][1][s][q];
                uP[s] = sT[j][1][0][0][s][q];
                dP[s] = sT[j][1][0][1][s][q];
                del[s] = uM[s] - uP[s];
                sb[s] = sS[j][0][s][q];
                tbb[s] = sS[j][1][s][q];
            }
            // the lifting's transpose: Delta(q) feeds sigma(p) through lift LF[p][q]
            double lb[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                double acc = 0.0;
#pragma unroll
                for (int p = 0; p < NP; ++p) acc = fma(sS[j][0][s][p], tb.LF[lM][p][q], acc);
                lb[s] = 2.0 * a.chi_e * a.c.A[s] * lift * acc;
            }
            for (int side = 0; side < 2; ++side) {
                face_point_adj<double>(a.c, 0.0, side == 0, uM, dM, uP, dP, del, sb, tbb, ub, db);
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    sA[j][side][0][s][q] = ub[s] + (side == 0 ? lb[s] : -lb[s]);
                    sA[j][side][1][s][q] = db[s];
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nf * 2 * NS * NB; i += blockDim.x) {
            const int j = i / (2 * NS * NB), side = (i / (NS * NB)) % 2, s = (i / NB) % NS, m = i % NB;
            const int l = sI[j][2 + side];
            double acc = 0.0;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int pp = side ? NP - 1 - p : p;
                acc = fma(sA[j][side][0][s][p], tb.EB[l][pp][m], fma(sA[j][side][1][s][p], sDN[j][side][p][m], acc));
            }
            a.fbuf[((f0 + j) * 2 + side) * NS * NB + s * NB + m] = acc;
        }
        return;
    }
    // pointwise flux with the lifted jump
    for (int i = threadIdx.x; i < nf * NP; i += blockDim.x) {
        const int j = i / NP, p = i % NP;
        const int lM = sI[j][2];
        const double lift = -sF[j][2] / (2.0 * sF[j][3]);
        double uM[NS], dM[NS], uP[NS], dP[NS], del[NS], sig[NS], tau[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            uM[s] = sT[j][0][0][0][s][p];
            dM[s] = sT[j][0][0][1][s][p];
            uP[s] = sT[j][1][0][0][s][p];
            dP[s] = sT[j][1][0][1][s][p];
            del[s] = uM[s] - uP[s];
        }
        if constexpr (MODE == TRI_APPLY) {
            face_point<double>(a.c, 0.0, uM, dM, uP, dP, del, sig, tau);
        } else {
            double duM[NS], ddM[NS], duP[NS], ddP[NS], ddel[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                duM[s] = sT[j][0][F - 1][0][s][p];
                ddM[s] = sT[j][0][F - 1][1][s][p];
                duP[s] = sT[j][1][F - 1][0][s][p];
                ddP[s] = sT[j][1][F - 1][1][s][p];
                ddel[s] = duM[s] - duP[s];
            }
            face_point_lin<double>(a.c, 0.0, uM, dM, uP, dP, del, duM, ddM, duP, ddP, ddel, sig, tau);
        }
        // the lifting of the (tangent) jump of the last field; the Gauss weight goes into sigma and tau
        const double w = tb.EW[p];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            double rn = 0.0;
#pragma unroll
            for (int q = 0; q < NP; ++q) rn = fma(tb.LF[lM][p][q], sD[j][s][q], rn);
            sS[j][0][s][p] = w * fma(2.0 * a.chi_e * a.c.A[s] * lift, rn, sig[s]);
            sS[j][1][s][p] = w * tau[s];
        }
    }
    __syncthreads();
    // test: K^- gets sigma phi^- + tau d_n phi^-, K^+ gets -sigma phi^+ + tau d_n phi^+
    for (int i = threadIdx.x; i < nf * 2 * NS * NB; i += blockDim.x) {
        const int j = i / (2 * NS * NB), side = (i / (NS * NB)) % 2, s = (i / NB) % NS, m = i % NB;
        const int l = sI[j][2 + side];
        double as = 0.0, at = 0.0;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int pp = side ? NP - 1 - p : p;
            as = fma(sS[j][0][s][p], tb.EB[l][pp][m], as);
            at = fma(sS[j][1][s][p], sDN[j][side][p][m], at);
        }
        a.fbuf[((f0 + j) * 2 + side) * NS * NB + s * NB + m] = sF[j][2] * (side ? at - as : at + as);
    }
}

// One CTA: EPB elements.  Volume terms at the collapsed Gauss points by sum
// factorisation over the warped-product basis (coefficients -> B_pq in v ->
// A_p in u, with the derivative factors for the (u, v) gradient, mapped to the
// reference and physical gradient; the pointwise flux, JVP: linearised, VJP:
// its adjoint; the flux mapped back by J^{-1} and the collapsed map, weighted,
// and tested by the transposed passes), the tested fluxes of the element's
// interior edges from the face buffer, the boundary data of Eq. (3) on its
// boundary edges (JVP/VJP: none, H' = 0), M^{-1} = 1 / det J.  Apply and JVP
// take the diffusion of n2..c3 in modal form, -A_s K_e U_s with K_e = det J
// sum_c G_c KS[c] (G = J^{-1} J^{-T}; exact, as the volume rule integrates the
// stiffness exactly): the forward passes carry gradients for n1, c1, c3 only
// and the test passes the flux of n1, n2 only.  The VJP keeps the full passes.
// The point values have an odd stride (6 * 3 + 1) so that threads on
// consecutive points hit distinct banks.
template <int K, int EPB, int MODE>
__global__ void __launch_bounds__(128) tri_elem_kernel(const TriArgs a) {
    using S = TriShape<K>;
    constexpr int NB = S::NB, NQ = S::NQ, NP = S::NP, F = MODE == TRI_APPLY ? 1 : 2;
    constexpr int N = K + 2, K1 = K + 1, QS = NS * 3 + 1;
    constexpr bool MODAL = MODE != TRI_VJP;
    constexpr int NGF = MODAL ? 3 : NS;   // forward slots carrying gradients (species n1, c1, c3 first)
    constexpr int NGT = MODAL ? 2 : NS;   // species tested against a flux
    static_assert(EPB * NB * NB <= EPB * F * NQ * QS, "K_e overlays the point values");
    const TriTab& tb = *a.tab;
    __shared__ double sU[EPB][F][NS][NB];
    __shared__ double sG[EPB][GEO];
    __shared__ double sH[EPB][F][2][NS][K1][N];   // v-pass (h, h_v); then the transposed u-pass
    __shared__ double sQ[EPB][F][NQ][QS];         // [s * 3 + (grad_x, grad_y, value)]; then the weighted flux
    const long long e0 = (long long)blockIdx.x * EPB;
    const int ne = (int)min((long long)EPB, a.E - e0);
    for (int i = threadIdx.x; i < ne * GEO; i += blockDim.x) sG[i / GEO][i % GEO] = a.geo[e0 * GEO + i];
    for (int i = threadIdx.x; i < F * ne * NS * NB; i += blockDim.x) {
        const int fi = i / (ne * NS * NB), r0 = i % (ne * NS * NB);
        const int e = r0 / (NS * NB), r = r0 % (NS * NB);
        sU[e][fi][r / NB][r % NB] = (fi ? a.dU : a.U)[e0 * NS * NB + r0];
    }
    __syncthreads();
    // v-pass: h_p(v_j) = sum_q B_pq(v_j) U_pq, and with B' where gradients are carried
    for (int i = threadIdx.x; i < ne * F * NS * K1 * N; i += blockDim.x) {
        const int e = i / (F * NS * K1 * N), fi = (i / (NS * K1 * N)) % F, sl = (i / (K1 * N)) % NS;
        const int p = (i / N) % K1, j = i % N;
        const int s = MODAL ? modal_fwd_species(sl) : sl;
        double h = 0.0, hv = 0.0;
#pragma unroll
        for (int q = 0; q < K1; ++q) {
            if (q <= K - p) {
                const int m = (p + q) * (p + q + 1) / 2 + q;
                const double u = sU[e][fi][s][m];
                h = fma(tb.SB[j][m], u, h);
                if (sl < NGF) hv = fma(tb.SdB[j][m], u, hv);
            }
        }
        sH[e][fi][0][s][p][j] = h;
        if (sl < NGF) sH[e][fi][1][s][p][j] = hv;
    }
    __syncthreads();
    // u-pass: value and, where carried, the (u, v) gradient, then the reference
    // and physical gradient (consecutive threads on consecutive points)
    for (int i = threadIdx.x; i < ne * F * NS * NQ; i += blockDim.x) {
        const int e = i / (F * NS * NQ), fi = (i / (NS * NQ)) % F, sl = (i / NQ) % NS, q = i % NQ;
        const int s = MODAL ? modal_fwd_species(sl) : sl;
        const int ii = q % N, j = q / N;
        double* Q = &sQ[e][fi][q][s * 3];
        double f = 0.0;
        if (sl < NGF) {
            double fu = 0.0, fv = 0.0;
#pragma unroll
            for (int p = 0; p < K1; ++p) {
                const double h = sH[e][fi][0][s][p][j];
                f = fma(tb.SA[ii][p], h, f);
                fu = fma(tb.SdA[ii][p], h, fu);
                fv = fma(tb.SA[ii][p], sH[e][fi][1][s][p][j], fv);
            }
            const double r0 = tb.SG[q][0] * fu, r1 = fma(tb.SG[q][1], fu, fv);
            const double* Ji = sG[e] + 6;
            Q[0] = Ji[0] * r0 + Ji[2] * r1;
            Q[1] = Ji[1] * r0 + Ji[3] * r1;
        } else {
#pragma unroll
            for (int p = 0; p < K1; ++p) f = fma(tb.SA[ii][p], sH[e][fi][0][s][p][j], f);
        }
        Q[2] = f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ne * NQ; i += blockDim.x) {
        const int e = i / NQ, q = i % NQ;
        double u[F][NS], g[F][NS][2], Phi[NS][2], Sr[NS];
#pragma unroll
        for (int fi = 0; fi < F; ++fi)
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const bool hasg = !MODAL || s == 0 || s == 3 || s == 5;
                u[fi][s] = sQ[e][fi][q][s * 3 + 2];
                g[fi][s][0] = hasg ? sQ[e][fi][q][s * 3] : 0.0;
                g[fi][s][1] = hasg ? sQ[e][fi][q][s * 3 + 1] : 0.0;
            }
        if constexpr (MODE == TRI_APPLY) {
            volume_point<2, double, true>(a.c, u[0], g[0], Phi, Sr);
        } else if constexpr (MODE == TRI_JVP) {
            volume_point_lin<2, double, true>(a.c, u[0], g[0], u[F - 1], g[F - 1], false, Phi, Sr);
        } else {
            // cotangents of S and Phi at the point: det w_q mu and det w_q grad mu,
            // mu = M^{-1} lambda = lambda / det (with CDG2_MINV); back through the
            // flux (w_q is applied below)
            const double det = sG[e][10];
            const double W = (a.flags & CDG2_MINV) ? 1.0 : det;
            double sb[NS], gb[NS][2], th[8];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                sb[s] = W * u[F - 1][s];
                gb[s][0] = W * g[F - 1][s][0];
                gb[s][1] = W * g[F - 1][s][1];
            }
            volume_point_adj<2, double>(a.c, u[0], g[0], sb, gb, Sr, Phi, th);   // Sr <- ub, Phi <- Gb
        }
        // Phi . grad psi = (J_c^{-1} J^{-1} Phi) . grad_(u,v) psi, weighted by w_q
        // (in place: this thread alone owns point q of the last field)
        const double* Ji = sG[e] + 6;
        const double wq = tb.VW[q];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            double* Q = &sQ[e][F - 1][q][s * 3];
            if (s < NGT) {
                const double p0 = Ji[0] * Phi[s][0] + Ji[1] * Phi[s][1];
                const double p1 = Ji[2] * Phi[s][0] + Ji[3] * Phi[s][1];
                Q[0] = wq * fma(tb.SG[q][0], p0, tb.SG[q][1] * p1);
                Q[1] = wq * p1;
            }
            Q[2] = wq * Sr[s];
        }
    }
    __syncthreads();
    // transposed u-pass: X_p(v_j) = sum_i A_p S + A'_p P_u; X^v_p(v_j) = sum_i A_p P_v
    // (species without a flux: A_p S only)
    for (int i = threadIdx.x; i < ne * NS * K1 * N; i += blockDim.x) {
        const int e = i / (NS * K1 * N), s = (i / (K1 * N)) % NS, p = (i / N) % K1, j = i % N;
        double x0 = 0.0, xv = 0.0;
        if (s < NGT) {
#pragma unroll
            for (int ii = 0; ii < N; ++ii) {
                const double* P = &sQ[e][F - 1][ii + N * j][s * 3];
                x0 = fma(tb.SA[ii][p], P[2], fma(tb.SdA[ii][p], P[0], x0));
                xv = fma(tb.SA[ii][p], P[1], xv);
            }
            sH[e][0][1][s][p][j] = xv;
        } else {
#pragma unroll
            for (int ii = 0; ii < N; ++ii) x0 = fma(tb.SA[ii][p], sQ[e][F - 1][ii + N * j][s * 3 + 2], x0);
        }
        sH[e][0][0][s][p][j] = x0;
    }
    __syncthreads();
    // K_e / det J = sum_c G_c KS[c], G_ab = sum_c (J^{-1})_ac (J^{-1})_bc for ab = 00, 11, 01, over the
    // point values (read by the transposed u-pass only)
    double (*sKe)[NB][NB] = reinterpret_cast<double (*)[NB][NB]>(&sQ[0][0][0][0]);
    if constexpr (MODAL) {
        for (int i = threadIdx.x; i < ne * NB * NB; i += blockDim.x) {
            const int e = i / (NB * NB), r = (i / NB) % NB, cc = i % NB;
            const double* Ji = sG[e] + 6;
            const double G0 = fma(Ji[0], Ji[0], Ji[1] * Ji[1]), G1 = fma(Ji[2], Ji[2], Ji[3] * Ji[3]);
            const double G2 = fma(Ji[0], Ji[2], Ji[1] * Ji[3]);
            sKe[e][r][cc] = fma(G0, tb.KS[0][r][cc], fma(G1, tb.KS[1][r][cc], G2 * tb.KS[2][r][cc]));
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < ne * NS * NB; i += blockDim.x) {
        const int e = i / (NS * NB), s = (i / NB) % NS, m = i % NB;
        const double* G = sG[e];
        const double det = G[10];
        int d = 0;
        while ((d + 1) * (d + 2) / 2 <= m) ++d;
        const int p = d - (m - d * (d + 1) / 2);
        double acc = 0.0;
        if (s < NGT) {
#pragma unroll
            for (int j = 0; j < N; ++j)
                acc = fma(tb.SB[j][m], sH[e][0][0][s][p][j], fma(tb.SdB[j][m], sH[e][0][1][s][p][j], acc));
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) acc = fma(tb.SB[j][m], sH[e][0][0][s][p][j], acc);
        }
        if constexpr (MODAL) {
            if (s > 0) {   // the diffusion of n2..c3 (of the tangent in the JVP): -A_s (K_e U_s)_m / det J
                double kd = 0.0;
#pragma unroll
                for (int jj = 0; jj < NB; ++jj) kd = fma(sKe[e][m][jj], sU[e][F - 1][s][jj], kd);
                acc = fma(-a.c.A[s], kd, acc);
            }
        }
        // forward: R = det sum_q w_q (Phi . grad phi + S phi); VJP: the cotangents carry det
        double R = MODE == TRI_VJP ? acc : det * acc;
        const long long ge = e0 + e;
        for (int l = 0; l < 3; ++l) {
            const int code = a.emap[ge * 3 + l];
            if (code >= 0) {
                R += a.fbuf[(long long)code * NS * NB + s * NB + m];
            } else if (MODE == TRI_APPLY && code != -1) {
                // boundary edge l on Gamma_1 (code -2) or Gamma_2 (code -3)
                const int f = -code - 2;
                const double r0x = l == 1 ? 1.0 : 0.0, r0y = l == 2 ? 1.0 : 0.0;   // reference vertex l
                const double r1x = l == 0 ? 1.0 : 0.0, r1y = l == 1 ? 1.0 : 0.0;   // reference vertex l + 1
                const double Ax = G[0] + G[2] * r0x + G[3] * r0y, Ay = G[1] + G[4] * r0x + G[5] * r0y;
                const double Bx = G[0] + G[2] * r1x + G[3] * r1y, By = G[1] + G[4] * r1x + G[5] * r1y;
                const double len = sqrt((Bx - Ax) * (Bx - Ax) + (By - Ay) * (By - Ay));
                double bacc = 0.0;
                for (int p = 0; p < NP; ++p) {
                    double uo[NS] = {0, 0, 0, 0, 0, 0}, sig[NS];
                    double c1 = 0.0;
#pragma unroll
                    for (int mm = 0; mm < NB; ++mm) c1 = fma(tb.EB[l][p][mm], sU[e][0][3][mm], c1);
                    uo[3] = c1;
                    const double x = Ax + tb.ET[p] * (Bx - Ax);
                    boundary_point<double>(a.c, f, x, a.g, uo, sig, a.c.beta1, true);
                    bacc = fma(tb.EW[p], sig[s] * tb.EB[l][p][m], bacc);
                }
                R += len * bacc;
            }
        }
        a.out[ge * NS * NB + s * NB + m] = (MODE != TRI_VJP && (a.flags & CDG2_MINV)) ? R / det : R;
    }
}

}  // namespace cdg2

namespace cdg2 {

constexpr int TRI_EPB = 4;   // elements per CTA

template <int K, int MODE>
static cudaError_t tri_launch(const TriArgs& a, cudaStream_t st) {
    constexpr int FPB = MODE == TRI_APPLY ? 8 : 4;   // faces per CTA (static shared memory <= 48 KB)
    if (a.NF > 0) {
        const unsigned fb = (unsigned)((a.NF + FPB - 1) / FPB);
        tri_face_kernel<K, FPB, MODE><<<fb, 128, 0, st>>>(a);
    }
    constexpr int EPB = MODE == TRI_APPLY ? TRI_EPB : TRI_EPB / 2;   // static shared memory <= 48 KB
    const unsigned eb = (unsigned)((a.E + EPB - 1) / EPB);
    tri_elem_kernel<K, EPB, MODE><<<eb, 128, 0, st>>>(a);
    return cudaGetLastError();
}

static int tri_upload(const cdg2_tri_mesh& m) {
    if (m.d_tab) return CDG2_OK;
    cudaError_t e = cudaSuccess;
    auto up = [&](void** dst, const void* src, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(dst, bytes > 0 ? bytes : 8);
        if (e == cudaSuccess && src && bytes > 0) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up((void**)&m.d_geo, m.geo.data(), sizeof(double) * m.geo.size());
    up((void**)&m.d_emap, m.emap.data(), sizeof(int) * m.emap.size());
    up((void**)&m.d_face, m.face.data(), sizeof(int) * m.face.size());
    up((void**)&m.d_fgeo, m.fgeo.data(), sizeof(double) * m.fgeo.size());
    up((void**)&m.d_fbuf, nullptr, sizeof(double) * (size_t)m.NF * 2 * NS * m.nb);
    up((void**)&m.d_tab, &m.tab, sizeof(TriTab));
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_tri_apply: mesh upload");
    return CDG2_OK;
}

}  // namespace cdg2

using namespace cdg2;

extern "C" int cdg2_tri_mesh_create(const cdg2_tri_desc* d, cdg2_tri_mesh** out) {
    if (!d || !out || !d->xy || !d->tri) {
        set_error("cdg2_tri_mesh_create: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (d->k < 1 || d->k > 3 || d->n_vert < 3 || d->n_tri < 1 || d->n_tri > (1LL << 29)) {
        set_error("cdg2_tri_mesh_create: need 1 <= k <= 3, n_vert >= 3, 1 <= n_tri < 2^29");
        return CDG2_ERR_INVALID_ARG;
    }
    auto* m = new (std::nothrow) cdg2_tri_mesh;
    if (!m) {
        set_error("cdg2_tri_mesh_create: out of host memory");
        return CDG2_ERR_INVALID_ARG;
    }
    m->k = d->k;
    m->nb = (d->k + 1) * (d->k + 2) / 2;
    m->nq = (d->k + 2) * (d->k + 2);
    m->np = d->k + 2;
    m->E = d->n_tri;
    m->chi_e = d->chi_e > 0.0 ? d->chi_e : 1.5;
    m->g1in[0] = d->gamma1_in[0];
    m->g1in[1] = d->gamma1_in[1];
    const double* xy = d->xy;
    double ly = xy[1];
    for (long long v = 0; v < d->n_vert; ++v) ly = std::max(ly, xy[2 * v + 1]);
    m->ly = ly;
    m->geo.assign((size_t)m->E * GEO, 0.0);
    for (long long e = 0; e < m->E; ++e) {
        long long v[3];
        for (int j = 0; j < 3; ++j) {
            v[j] = d->tri[3 * e + j];
            if (v[j] < 0 || v[j] >= d->n_vert) {
                delete m;
                set_error("cdg2_tri_mesh_create: vertex index out of range");
                return CDG2_ERR_INVALID_ARG;
            }
        }
        const double x0 = xy[2 * v[0]], y0 = xy[2 * v[0] + 1];
        const double J00 = xy[2 * v[1]] - x0, J01 = xy[2 * v[2]] - x0;
        const double J10 = xy[2 * v[1] + 1] - y0, J11 = xy[2 * v[2] + 1] - y0;
        const double det = J00 * J11 - J01 * J10;
        if (!(det > 0.0)) {
            delete m;
            set_error("cdg2_tri_mesh_create: triangle " + std::to_string(e) +
                      " is degenerate or clockwise (vertices must be counter-clockwise)");
            return CDG2_ERR_INVALID_ARG;
        }
        double* G = &m->geo[(size_t)e * GEO];
        G[0] = x0;
        G[1] = y0;
        G[2] = J00;
        G[3] = J01;
        G[4] = J10;
        G[5] = J11;
        G[6] = J11 / det;
        G[7] = -J01 / det;
        G[8] = -J10 / det;
        G[9] = J00 / det;
        G[10] = det;
    }
    // edges: sorted vertex pair -> owners (element, local edge)
    std::map<std::pair<long long, long long>, std::vector<std::pair<long long, int>>> edges;
    for (long long e = 0; e < m->E; ++e)
        for (int l = 0; l < 3; ++l) {
            const long long a = d->tri[3 * e + l], b = d->tri[3 * e + (l + 1) % 3];
            edges[{std::min(a, b), std::max(a, b)}].push_back({e, l});
        }
    m->emap.assign((size_t)m->E * 3, -1);
    const double tol = 1e-12 * std::max(1.0, ly);
    for (const auto& kv : edges) {
        const auto& own = kv.second;
        if (own.size() == 2) {
            long long e1 = own[0].first, e2 = own[1].first;
            int l1 = own[0].second, l2 = own[1].second;
            const long long a1 = d->tri[3 * e1 + l1], a2 = d->tri[3 * e2 + l2];
            if (a1 == a2) {
                delete m;
                set_error("cdg2_tri_mesh_create: neighbouring triangles with inconsistent orientation");
                return CDG2_ERR_INVALID_ARG;
            }
            const double ar1 = m->geo[(size_t)e1 * GEO + 10], ar2 = m->geo[(size_t)e2 * GEO + 10];
            const bool tie = std::fabs(ar1 - ar2) <= 1e-12 * std::max(ar1, ar2);
            if (!((!tie && ar1 < ar2) || (tie && e1 < e2))) {
                std::swap(e1, e2);
                std::swap(l1, l2);
            }
            const long long f = (long long)m->face.size() / 4;
            m->face.insert(m->face.end(), {(int)e1, (int)e2, l1, l2});
            const long long va = d->tri[3 * e1 + l1], vb = d->tri[3 * e1 + (l1 + 1) % 3];
            const double dx = xy[2 * vb] - xy[2 * va], dy = xy[2 * vb + 1] - xy[2 * va + 1];
            const double len = std::sqrt(dx * dx + dy * dy);
            m->fgeo.insert(m->fgeo.end(), {dy / len, -dx / len, len, m->geo[(size_t)e1 * GEO + 10]});
            m->emap[(size_t)e1 * 3 + l1] = (int)(2 * f);
            m->emap[(size_t)e2 * 3 + l2] = (int)(2 * f + 1);
        } else if (own.size() == 1) {
            const double ya = xy[2 * kv.first.first + 1], yb = xy[2 * kv.first.second + 1];
            int tag = 0;
            if (std::fabs(ya) <= tol && std::fabs(yb) <= tol) tag = 1;
            else if (std::fabs(ya - ly) <= tol && std::fabs(yb - ly) <= tol) tag = 2;
            m->emap[(size_t)own[0].first * 3 + own[0].second] = -1 - tag;
        } else {
            delete m;
            set_error("cdg2_tri_mesh_create: an edge is shared by more than two triangles");
            return CDG2_ERR_INVALID_ARG;
        }
    }
    m->NF = (long long)m->face.size() / 4;
    build_tables(m->k, m->tab);
    *out = m;
    return CDG2_OK;
}

extern "C" void cdg2_tri_mesh_destroy(cdg2_tri_mesh* m) {
    if (!m) return;
    cudaFree(m->d_geo);
    cudaFree(m->d_emap);
    cudaFree(m->d_face);
    cudaFree(m->d_fgeo);
    cudaFree(m->d_fbuf);
    cudaFree(m->d_tab);
    if (m->step_ws) cudaFree(m->step_ws);
    if (m->status) cudaFree(m->status);
    m->spc.release();
    delete m;
}

extern "C" int cdg2_tri_mesh_info(const cdg2_tri_mesh* m, long long* n_elem, int* n_basis, long long* n_dof,
                                  long long* n_faces) {
    if (!m) {
        set_error("cdg2_tri_mesh_info: NULL mesh");
        return CDG2_ERR_INVALID_ARG;
    }
    if (n_elem) *n_elem = m->E;
    if (n_basis) *n_basis = m->nb;
    if (n_dof) *n_dof = m->E * NS * m->nb;
    if (n_faces) *n_faces = m->NF;
    return CDG2_OK;
}

static int tri_run(const char* who, const cdg2_tri_mesh* m, const cdg2_params* p, const double* U, const double* dU,
                   double* out, int flags, int mode, void* stream) {
    if (!m || !p || !U || !out || (mode != TRI_APPLY && !dU)) {
        set_error(std::string(who) + ": NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (U == out || dU == out) {
        set_error(std::string(who) + ": the inputs and out must not overlap");
        return CDG2_ERR_INVALID_ARG;
    }
    if (flags & ~(CDG2_MINV | CDG2_ASYNC)) {
        set_error(std::string(who) + ": only CDG2_MINV and CDG2_ASYNC are supported on triangle meshes");
        return CDG2_ERR_INVALID_ARG;
    }
    if (int rc = tri_upload(*m)) return rc;
    if (cudaError_t e = ensure_status(&m->status)) return cuda_fail(e, who);
    TriArgs a;
    a.U = U;
    a.dU = dU;
    a.out = out;
    a.flags = flags;
    a.chi_e = m->chi_e;
    a.E = m->E;
    a.NF = m->NF;
    a.geo = m->d_geo;
    a.emap = m->d_emap;
    a.face = m->d_face;
    a.fgeo = m->d_fgeo;
    a.tab = m->d_tab;
    a.fbuf = m->d_fbuf;
    Geo g;
    std::memset(&g, 0, sizeof(g));
    g.dim = 2;
    g.k = m->k;
    g.vol = 1.0;
    for (int j = 0; j < 3; ++j) {
        g.h[j] = 1.0;
        g.n[j] = 1;
    }
    g.g1in[0] = m->g1in[0];
    g.g1in[1] = m->g1in[1];
    a.g = g;
    a.c = make_coefT<double>(make_coef(*p), g, nullptr);
    a.c.domain = m->status;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (mode == TRI_APPLY) {
        switch (m->k) {
            case 1: e = tri_launch<1, TRI_APPLY>(a, st); break;
            case 2: e = tri_launch<2, TRI_APPLY>(a, st); break;
            default: e = tri_launch<3, TRI_APPLY>(a, st); break;
        }
    } else if (mode == TRI_JVP) {
        switch (m->k) {
            case 1: e = tri_launch<1, TRI_JVP>(a, st); break;
            case 2: e = tri_launch<2, TRI_JVP>(a, st); break;
            default: e = tri_launch<3, TRI_JVP>(a, st); break;
        }
    } else {
        switch (m->k) {
            case 1: e = tri_launch<1, TRI_VJP>(a, st); break;
            case 2: e = tri_launch<2, TRI_VJP>(a, st); break;
            default: e = tri_launch<3, TRI_VJP>(a, st); break;
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, who);
    if (flags & CDG2_ASYNC) return CDG2_OK;
    return take_domain_status(m->status, st, who);
}

extern "C" int cdg2_tri_mesh_status(const cdg2_tri_mesh* m, void* stream) {
    if (!m) {
        set_error("cdg2_tri_mesh_status: NULL mesh");
        return CDG2_ERR_INVALID_ARG;
    }
    return take_domain_status(m->status, (cudaStream_t)stream, "cdg2_tri_mesh_status");
}

extern "C" int cdg2_tri_apply(const cdg2_tri_mesh* m, const cdg2_params* p, const double* U, double* out, int flags,
                              void* stream) {
    return tri_run("cdg2_tri_apply", m, p, U, nullptr, out, flags, TRI_APPLY, stream);
}

extern "C" int cdg2_tri_jvp(const cdg2_tri_mesh* m, const cdg2_params* p, const double* U, const double* dU,
                            double* out, int flags, void* stream) {
    return tri_run("cdg2_tri_jvp", m, p, U, dU, out, flags, TRI_JVP, stream);
}

extern "C" int cdg2_tri_vjp(const cdg2_tri_mesh* m, const cdg2_params* p, const double* U, const double* lam,
                            double* gU, int flags, void* stream) {
    return tri_run("cdg2_tri_vjp", m, p, U, lam, gU, flags, TRI_VJP, stream);
}

namespace {
struct TriStepCtx {
    const cdg2_tri_mesh* m;
    const cdg2_params* p;
};
int tri_step_apply(const void* ctx, const double* Y, double* out, cudaStream_t st) {
    const auto* c = static_cast<const TriStepCtx*>(ctx);
    return tri_run("cdg2_tri_step", c->m, c->p, Y, nullptr, out, CDG2_MINV | CDG2_ASYNC, TRI_APPLY, st);
}
int tri_step_jvp(const void* ctx, const double* Y, const double* v, double* out, cudaStream_t st) {
    const auto* c = static_cast<const TriStepCtx*>(ctx);
    return tri_run("cdg2_tri_step", c->m, c->p, Y, v, out, CDG2_MINV | CDG2_ASYNC, TRI_JVP, st);
}
int tri_step_jvp_diffusion(const void* ctx, const double* v, double* out, cudaStream_t st) {
    const auto* c = static_cast<const TriStepCtx*>(ctx);
    const cdg2_params q = cdg2::diffusion_only(*c->p);
    return tri_run("cdg2_tri_step", c->m, &q, v, v, out, CDG2_MINV | CDG2_ASYNC, TRI_JVP, st);
}
}  // namespace

extern "C" int cdg2_tri_step(const cdg2_tri_mesh* m, const cdg2_params* p, double* U, double dt,
                             const cdg2_solver_opts* opts, cdg2_stats* stats, void* stream) {
    if (!m || !p) {
        set_error("cdg2_tri_step: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    const TriStepCtx ctx{m, p};
    cdg2::SimplexStepOps ops;
    ops.n = m->E * NS * m->nb;
    ops.nb = m->nb;
    ops.ws = &m->step_ws;
    ops.ws_bytes = &m->step_ws_bytes;
    ops.ctx = &ctx;
    ops.apply = tri_step_apply;
    ops.jvp = tri_step_jvp;
    ops.jvp_diffusion = tri_step_jvp_diffusion;
    const Coef co = make_coef(*p);
    ops.A = co.A;
    ops.face = m->face.data();
    ops.NF = m->NF;
    ops.pc = &m->spc;
    if (cudaError_t e = ensure_status(&m->status)) return cuda_fail(e, "cdg2_tri_step");
    ops.dom = m->status;
    return cdg2::simplex_step(ops, U, dt, opts, stats, stream, "cdg2_tri_step");
}
