// The CDG2 operator on tetrahedral meshes (Sec. 3.1: P_k on tetrahedra,
// chi_e = 2): f(U) = M^{-1} L_h(U) in FP64, face-once.
//
// Readings (shared with the oracle; the paper fixes none of them):
//  * basis: on the reference tetrahedron T = {xi, eta, zeta >= 0, xi + eta +
//    zeta <= 1} the orthonormal Dubiner basis psi_pqr = c_pqr L_p J_q R_r with
//    L_p = s^p P_p((2 xi - s)/s), s = 1 - eta - zeta; J_q = t^q P_q^{(2p+1,0)}
//    ((2 eta - t)/t), t = 1 - zeta; R_r = P_r^{(2p+2q+2,0)}(2 zeta - 1);
//    c_pqr = sqrt((2p+1)(2p+2q+2)(2p+2q+2r+3)); modes by total degree, then r,
//    then q; mapped affinely by x = x_0 + J_e xi, so M_K = det J_e I;
//  * volume quadrature: the collapsed Gauss rule with (k+2)^3 points (xi =
//    u (1-v)(1-w), eta = v (1-w), zeta = w, weight w_u w_v w_w (1-v)(1-w)^2,
//    u fastest); face quadrature: the collapsed triangle rule with (k+2)^2
//    points (s = u (1-v), t = v, weight w_u w_v (1-v)) in K^-'s parametrisation
//    A + s (B - A) + t (C - A) of the face, local face l being the vertices
//    other than l in increasing local order;
//  * K^-_e: the smaller adjacent tetrahedron (Sec. 3.1); volumes within a
//    relative 1e-12 tie, a tie goes to the lower index;
//  * boundary faces on y = 0 are Gamma_1, on y = max y Gamma_2 (Eq. (3)); other
//    boundary faces are no-flow walls.
// A face point with barycentric coordinates (lambda_a, lambda_b, lambda_c) on
// the face's global vertices sits at sum lambda_i r_{l_i} in an element whose
// local indices of those vertices are (l_a, l_b, l_c): the basis tables are
// kept for each of the 24 ordered triples of local vertices ("frames"); K^-
// reads its own face's frame, K^+ the frame of the same three global
// vertices in its own numbering.  With M_{K^-} = det I, the lifting identity
// gives r . n (x_p) = -(E / (2 det_-)) sum_p' L[p][p'] Delta(x_p'), E =
// |(B - A) x (C - A)|, L[p][p'] = sum_i psi_i(x_p) psi_i(x_p') w_p'.
#include <algorithm>
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

constexpr int TTMAXB = 20;    // basis functions for k = 3
constexpr int TTMAXQ = 125;   // volume points for k = 3
constexpr int TTMAXP = 25;    // face points for k = 3
constexpr int TTMAXN = 5;     // Gauss points per collapsed direction for k = 3
constexpr int TTMAXK1 = 4;    // k + 1
constexpr int TTMAXPQ = 10;   // pairs (p, q) with p + q <= 3
constexpr int NFRAME = 64;    // frame code a * 16 + b * 4 + c (24 of them used)
constexpr int TGEO = 22;      // x0 (3), J (9, row-major), J^{-1} (9, row-major), det J

__host__ __device__ constexpr int frame_code(int a, int b, int c) { return a * 16 + b * 4 + c; }

struct TetTab {
    double VB[TTMAXQ][TTMAXB];            // psi_i at the volume points
    double VD[3][TTMAXQ][TTMAXB];         // reference gradient
    double VW[TTMAXQ];
    double FB[NFRAME][TTMAXP][TTMAXB];    // psi_i at the face points of each frame
    double FD[3][NFRAME][TTMAXP][TTMAXB];
    double LF[NFRAME][TTMAXP][TTMAXP];    // lifting kernel of each frame (read for K^-'s)
    double FW[TTMAXP];                    // face rule weights (sum 1/2)
    double FX[TTMAXP][2];                 // face rule points (s, t)
    // Warped-product factors on the collapsed volume grid: at xi = u (1-v)(1-w),
    // eta = v (1-w), zeta = w, psi_pqr = A_p(u) B_pq(v) C_pqr(w) with
    // A_p = P_p(2u-1), B_pq = (1-v)^p P_q^{(2p+1,0)}(2v-1) and
    // C_pqr = c_pqr (1-w)^{p+q} P_r^{(2p+2q+2,0)}(2w-1); pairs (p, q) ordered
    // by p, then q.
    double SA[TTMAXN][TTMAXK1], SdA[TTMAXN][TTMAXK1];     // [u point][p]
    double SB[TTMAXN][TTMAXPQ], SdB[TTMAXN][TTMAXPQ];     // [v point][pair]
    double SC[TTMAXN][TTMAXB], SdC[TTMAXN][TTMAXB];       // [w point][mode]
    // the reference gradient from the (u, v, w) one at volume point q:
    // d_xi = a1 d_u, d_eta = u a1 d_u + b1 d_v, d_zeta = u a1 d_u + v b1 d_v + d_w,
    // a1 = 1 / ((1-v)(1-w)), b1 = 1 / (1-w); stored (a1, u a1, b1, v b1)
    double SG[TTMAXQ][4];
    // reference stiffness matrices, exact under the volume rule: KS[c][i][j] =
    // sum_q w_q d_a psi_i d_b psi_j for c = (a, b) in {00, 11, 22}, and that plus
    // its transpose for c = (a, b) in {01, 02, 12}; so that int_K grad psi_i .
    // grad psi_j = det J sum_c G_c KS[c][i][j] with G = J^{-1} J^{-T}
    double KS[6][TTMAXB][TTMAXB];
    int PQA[TTMAXK1][TTMAXK1];            // pair index of (p, q), p + q <= k
    int PQM[TTMAXPQ][TTMAXK1];            // mode index of (pair, r), r <= k - p - q
    int MPQ[TTMAXB];                      // pair index of mode m
};

}  // namespace cdg2

struct cdg2_tet_mesh {
    int k = 0, nb = 0;
    long long E = 0, NF = 0;
    double chi_e = 2.0, ly = 0.0;
    double g1in[2] = {0.375, 0.625};
    std::vector<double> geo;     // [E][TGEO]
    std::vector<int> emap;       // [E][4]: 2 face + side, or -1 - tag (0 wall, 1 Gamma_1, 2 Gamma_2)
    std::vector<int> face;       // [NF][4]: eM, eP, frame of K^-, frame of K^+
    std::vector<double> fgeo;    // [NF][5]: n (3), E = |(B - A) x (C - A)|, det J of K^-
    std::vector<cdg2::TetTab> tab;   // one (large) table, host copy
    mutable double* d_geo = nullptr;
    mutable int* d_emap = nullptr;
    mutable int* d_face = nullptr;
    mutable double* d_fgeo = nullptr;
    mutable cdg2::TetTab* d_tab = nullptr;
    mutable double* d_fbuf = nullptr;   // [NF][2][6][nb]
    mutable void* step_ws = nullptr;    // cdg2_tet_step workspace
    mutable size_t step_ws_bytes = 0;
    mutable cdg2::SimplexPrecond spc;   // element-block Jacobi of the step
    mutable int* status = nullptr;      // domain status word (device int)
};

namespace cdg2 {

namespace {

const int FACE_VERTS[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
const double REF_VERT[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

// psi_i and its reference gradient at (xi, eta, zeta).
void dubiner3(int k, double xi, double eta, double zeta, double* psi, double* d0, double* d1, double* d2) {
    const double s = 1.0 - eta - zeta, xt = 2.0 * xi - s;       // d xt = (2, 1, 1), d s = (0, -1, -1)
    const double t = 1.0 - zeta, y = 2.0 * eta - t;             // d y = (0, 2, 1), d t = (0, 0, -1)
    double L[4], dL[3][4];
    L[0] = 1.0;
    for (int j = 0; j < 3; ++j) dL[j][0] = 0.0;
    const double dxt[3] = {2.0, 1.0, 1.0}, ds[3] = {0.0, -1.0, -1.0};
    if (k >= 1) {
        L[1] = xt;
        for (int j = 0; j < 3; ++j) dL[j][1] = dxt[j];
    }
    for (int p = 2; p <= k; ++p) {
        L[p] = ((2 * p - 1) * xt * L[p - 1] - (p - 1) * s * s * L[p - 2]) / p;
        for (int j = 0; j < 3; ++j)
            dL[j][p] = ((2 * p - 1) * (dxt[j] * L[p - 1] + xt * dL[j][p - 1]) -
                        (p - 1) * (2.0 * s * ds[j] * L[p - 2] + s * s * dL[j][p - 2])) / p;
    }
    const double dy[3] = {0.0, 2.0, 1.0}, dt[3] = {0.0, 0.0, -1.0};
    int i = 0;
    for (int d = 0; d <= k; ++d)
        for (int r = 0; r <= d; ++r)
            for (int q = 0; q <= d - r; ++q, ++i) {
                const int p = d - q - r;
                const double al = 2.0 * p + 1.0;
                // J_q = t^q P_q^{(al,0)}(y / t) by the scaled recurrence, with its gradient
                double J0 = 1.0, J1 = 0.0, dJ0[3] = {0, 0, 0}, dJ1[3] = {0, 0, 0};
                double Jq = 1.0, dJq[3] = {0, 0, 0};
                if (q >= 1) {
                    J1 = (al + 1.0) * t + (al + 2.0) * (y - t) / 2.0;
                    for (int j = 0; j < 3; ++j) dJ1[j] = (al + 1.0) * dt[j] + (al + 2.0) * (dy[j] - dt[j]) / 2.0;
                    for (int m = 2; m <= q; ++m) {
                        const double c = 2.0 * m + al;
                        const double a1 = 2.0 * m * (m + al) * (c - 2.0);
                        const double a2 = (c - 1.0) * c * (c - 2.0);
                        const double a3 = (c - 1.0) * al * al;
                        const double a4 = 2.0 * (m + al - 1.0) * (m - 1.0) * c;
                        const double J2 = ((a2 * y + a3 * t) * J1 - a4 * t * t * J0) / a1;
                        double dJ2[3];
                        for (int j = 0; j < 3; ++j)
                            dJ2[j] = ((a2 * dy[j] + a3 * dt[j]) * J1 + (a2 * y + a3 * t) * dJ1[j] -
                                      a4 * (2.0 * t * dt[j] * J0 + t * t * dJ0[j])) / a1;
                        J0 = J1;
                        J1 = J2;
                        for (int j = 0; j < 3; ++j) {
                            dJ0[j] = dJ1[j];
                            dJ1[j] = dJ2[j];
                        }
                    }
                    Jq = J1;
                    for (int j = 0; j < 3; ++j) dJq[j] = dJ1[j];
                }
                double R, dR;
                jacobi_d(r, 2.0 * p + 2.0 * q + 2.0, 2.0 * zeta - 1.0, R, dR);
                const double cst = std::sqrt((2.0 * p + 1) * (2.0 * p + 2 * q + 2) * (2.0 * p + 2 * q + 2 * r + 3));
                psi[i] = cst * L[p] * Jq * R;
                double g[3];
                for (int j = 0; j < 3; ++j) g[j] = cst * (dL[j][p] * Jq * R + L[p] * dJq[j] * R);
                g[2] += cst * L[p] * Jq * 2.0 * dR;
                d0[i] = g[0];
                d1[i] = g[1];
                d2[i] = g[2];
            }
}

void build_tet_tables(int k, TetTab& T) {
    std::memset(&T, 0, sizeof(T));
    const int n = k + 2;
    const int nb = (k + 1) * (k + 2) * (k + 3) / 6;
    double g[16], w[16];
    gauss01(n, g, w);
    for (int c = 0; c < n; ++c)
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                const int q = a + n * (b + n * c);
                const double xi = g[a] * (1.0 - g[b]) * (1.0 - g[c]), eta = g[b] * (1.0 - g[c]), zeta = g[c];
                T.VW[q] = w[a] * w[b] * w[c] * (1.0 - g[b]) * (1.0 - g[c]) * (1.0 - g[c]);
                dubiner3(k, xi, eta, zeta, T.VB[q], T.VD[0][q], T.VD[1][q], T.VD[2][q]);
            }
    {
        const int PA[6] = {0, 1, 2, 0, 0, 1}, PB[6] = {0, 1, 2, 1, 2, 2};
        for (int c = 0; c < 6; ++c)
            for (int i = 0; i < nb; ++i)
                for (int j = 0; j < nb; ++j) {
                    double acc = 0.0;
                    for (int q = 0; q < n * n * n; ++q) {
                        double v = T.VD[PA[c]][q][i] * T.VD[PB[c]][q][j];
                        if (PA[c] != PB[c]) v += T.VD[PB[c]][q][i] * T.VD[PA[c]][q][j];
                        acc += T.VW[q] * v;
                    }
                    T.KS[c][i][j] = acc;
                }
    }
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < n; ++a) {
            const int p = a + n * b;
            T.FX[p][0] = g[a] * (1.0 - g[b]);
            T.FX[p][1] = g[b];
            T.FW[p] = w[a] * w[b] * (1.0 - g[b]);
        }
    // warped-product factors and the (u, v, w) -> reference gradient map
    int na = 0;
    for (int p = 0; p <= k; ++p)
        for (int q = 0; q <= k - p; ++q) T.PQA[p][q] = na++;
    for (int a = 0; a < TTMAXPQ; ++a)
        for (int r = 0; r < TTMAXK1; ++r) T.PQM[a][r] = -1;
    {
        int m = 0;
        for (int d = 0; d <= k; ++d)
            for (int r = 0; r <= d; ++r)
                for (int q = 0; q <= d - r; ++q, ++m) {
                    const int p = d - q - r;
                    T.PQM[T.PQA[p][q]][r] = m;
                    T.MPQ[m] = T.PQA[p][q];
                    const double cst = std::sqrt((2.0 * p + 1) * (2.0 * p + 2 * q + 2) * (2.0 * p + 2 * q + 2 * r + 3));
                    for (int l = 0; l < n; ++l) {
                        const double w1 = 1.0 - g[l];
                        double R, dR;
                        jacobi_d(r, 2.0 * p + 2.0 * q + 2.0, 2.0 * g[l] - 1.0, R, dR);
                        const double pw = std::pow(w1, p + q);
                        const double dpw = (p + q) > 0 ? -(p + q) * std::pow(w1, p + q - 1) : 0.0;
                        T.SC[l][m] = cst * pw * R;
                        T.SdC[l][m] = cst * (dpw * R + pw * 2.0 * dR);
                    }
                }
    }
    for (int j = 0; j < n; ++j) {
        for (int p = 0; p <= k; ++p) {
            double P, dP;
            jacobi_d(p, 0.0, 2.0 * g[j] - 1.0, P, dP);
            T.SA[j][p] = P;
            T.SdA[j][p] = 2.0 * dP;
            for (int q = 0; q <= k - p; ++q) {
                const double v1 = 1.0 - g[j];
                double Q, dQ;
                jacobi_d(q, 2.0 * p + 1.0, 2.0 * g[j] - 1.0, Q, dQ);
                const double pw = std::pow(v1, p), dpw = p > 0 ? -p * std::pow(v1, p - 1) : 0.0;
                T.SB[j][T.PQA[p][q]] = pw * Q;
                T.SdB[j][T.PQA[p][q]] = dpw * Q + pw * 2.0 * dQ;
            }
        }
    }
    for (int c = 0; c < n; ++c)
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a) {
                const int q = a + n * (b + n * c);
                const double a1 = 1.0 / ((1.0 - g[b]) * (1.0 - g[c])), b1 = 1.0 / (1.0 - g[c]);
                T.SG[q][0] = a1;
                T.SG[q][1] = g[a] * a1;
                T.SG[q][2] = b1;
                T.SG[q][3] = g[b] * b1;
            }
    const int np = n * n;
    for (int la = 0; la < 4; ++la)
        for (int lb = 0; lb < 4; ++lb)
            for (int lc = 0; lc < 4; ++lc) {
                if (la == lb || lb == lc || la == lc) continue;
                const int f = frame_code(la, lb, lc);
                for (int p = 0; p < np; ++p) {
                    const double s = T.FX[p][0], t = T.FX[p][1], l0 = 1.0 - s - t;
                    double x[3];
                    for (int j = 0; j < 3; ++j) x[j] = l0 * REF_VERT[la][j] + s * REF_VERT[lb][j] + t * REF_VERT[lc][j];
                    dubiner3(k, x[0], x[1], x[2], T.FB[f][p], T.FD[0][f][p], T.FD[1][f][p], T.FD[2][f][p]);
                }
                for (int p = 0; p < np; ++p)
                    for (int pp = 0; pp < np; ++pp) {
                        double acc = 0.0;
                        for (int i = 0; i < nb; ++i) acc += T.FB[f][p][i] * T.FB[f][pp][i];
                        T.LF[f][p][pp] = acc * T.FW[pp];
                    }
            }
}

}  // namespace

}  // namespace cdg2

namespace cdg2 {

template <int K>
struct TetShape {
    static constexpr int NB = (K + 1) * (K + 2) * (K + 3) / 6;
    static constexpr int NQ = (K + 2) * (K + 2) * (K + 2);
    static constexpr int NP = (K + 2) * (K + 2);
};

struct TetArgs {
    const double* U;
    const double* dU;    // JVP: the tangent; VJP: lambda
    double* out;
    int flags;
    double chi_e;
    long long E, NF;
    const double* geo;
    const int* emap;
    const int* face;
    const double* fgeo;
    const TetTab* tab;
    double* fbuf;
    Geo g;               // only g1in is read (Gamma_{1,in})
    CoefT<double> c;
};

constexpr int TET_APPLY = 0, TET_JVP = 1, TET_VJP = 2;

// One CTA: FPB interior faces.  Traces of both sides at K^-'s face points
// (each side through its frame), the K^- lifting, the face flux (JVP: its
// linearisation; VJP: the cotangents E w_p (mu^- - mu^+) of sigma and
// E w_p (d_n mu^- + d_n mu^+) of tau back through face_point_adj per side and
// the transposed lifting, mu = M^{-1} lambda), and the test against both
// sides' basis into the face buffer ([face][side][6][nb]).
template <int K, int FPB, int MODE>
__global__ void __launch_bounds__(128) tet_face_kernel(const TetArgs a) {
    using S = TetShape<K>;
    constexpr int NB = S::NB, NP = S::NP, F = MODE == TET_APPLY ? 1 : 2;
    const TetTab& tb = *a.tab;
    __shared__ double sU[FPB][2][F][NS][NB];
    __shared__ double sM[FPB][2][3];          // J^{-1} n^- of each side: n^- . J^{-T} g = (J^{-1} n^-) . g
    __shared__ double sDet[FPB][2];
    __shared__ double sF[FPB][5];             // n (3), E, det_-
    __shared__ int sI[FPB][4];                // eM, eP, frame of K^-, frame of K^+
    __shared__ double sDN[FPB][2][NP][NB];    // n^- . grad phi_m of each side at the face points
    __shared__ double sT[FPB][2][F][2][NS][NP];  // [side][field][value, normal derivative][s][p]
    __shared__ double sD[MODE == TET_VJP ? 1 : FPB][NS][NP];  // jump of the last field (the lifted one)
    __shared__ double sS[FPB][2][NS][NP];     // w_p sigma, w_p tau (VJP: the cotangents of sigma, tau)
    __shared__ double sA[MODE == TET_VJP ? FPB : 1][2][2][NS][NP];   // VJP: trace cotangents
    const long long f0 = (long long)blockIdx.x * FPB;
    const int nf = (int)min((long long)FPB, a.NF - f0);
    for (int i = threadIdx.x; i < nf * 5; i += blockDim.x) {
        const int j = i / 5, c = i % 5;
        if (c < 4) sI[j][c] = a.face[(f0 + j) * 4 + c];
        sF[j][c] = a.fgeo[(f0 + j) * 5 + c];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nf * 2; i += blockDim.x) {
        const int j = i / 2, side = i % 2;
        const double* Ji = a.geo + (long long)sI[j][side] * TGEO + 12;
#pragma unroll
        for (int r = 0; r < 3; ++r)
            sM[j][side][r] = fma(Ji[3 * r], sF[j][0], fma(Ji[3 * r + 1], sF[j][1], Ji[3 * r + 2] * sF[j][2]));
        sDet[j][side] = Ji[9];
    }
    for (int i = threadIdx.x; i < nf * 2 * F * NS * NB; i += blockDim.x) {
        const int j = i / (2 * F * NS * NB), side = (i / (F * NS * NB)) % 2, fi = (i / (NS * NB)) % F;
        const int r = i % (NS * NB);
        sU[j][side][fi][r / NB][r % NB] = (fi ? a.dU : a.U)[(long long)sI[j][side] * NS * NB + r];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nf * 2 * NP * NB; i += blockDim.x) {
        const int j = i / (2 * NP * NB), side = (i / (NP * NB)) % 2, p = (i / NB) % NP, m = i % NB;
        const int fr = sI[j][2 + side];
        const double* mv = sM[j][side];
        sDN[j][side][p][m] = fma(mv[0], tb.FD[0][fr][p][m], fma(mv[1], tb.FD[1][fr][p][m], mv[2] * tb.FD[2][fr][p][m]));
    }
    __syncthreads();
    // traces of both sides per (face, field, species, point), and the jump of the last field
    for (int i = threadIdx.x; i < nf * F * NS * NP; i += blockDim.x) {
        const int j = i / (F * NS * NP), fi = (i / (NS * NP)) % F;
        const int s = (i / NP) % NS, p = i % NP;
        double val[2];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int fr = sI[j][2 + side];
            double v = 0.0, dn = 0.0;
#pragma unroll 4
            for (int m = 0; m < NB; ++m) {
                const double u = sU[j][side][fi][s][m];
                v = fma(tb.FB[fr][p][m], u, v);
                dn = fma(sDN[j][side][p][m], u, dn);
            }
            // VJP: the cotangent field enters as mu = M^{-1} lambda = lambda / det J (with CDG2_MINV)
            const double sc = (MODE == TET_VJP && fi == 1 && (a.flags & CDG2_MINV)) ? 1.0 / sDet[j][side] : 1.0;
            val[side] = v * sc;
            sT[j][side][fi][0][s][p] = v * sc;
            sT[j][side][fi][1][s][p] = dn * sc;
        }
        if constexpr (MODE != TET_VJP) {
            if (fi == F - 1) sD[j][s][p] = val[0] - val[1];
        }
    }
    __syncthreads();
    if constexpr (MODE == TET_VJP) {
        for (int i = threadIdx.x; i < nf * NS * NP; i += blockDim.x) {
            const int j = i / (NS * NP), s = (i / NP) % NS, p = i % NP;
            const double W = sF[j][3] * tb.FW[p];
            sS[j][0][s][p] = W * (sT[j][0][1][0][s][p] - sT[j][1][1][0][s][p]);
            sS[j][1][s][p] = W * (sT[j][0][1][1][s][p] + sT[j][1][1][1][s][p]);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nf * NP; i += blockDim.x) {
            const int j = i / NP, q = i % NP;
            const int frM = sI[j][2];
            const double lift = -sF[j][3] / (2.0 * sF[j][4]);
            double uM[NS], dM[NS], uP[NS], dP[NS], del[NS], sb[NS], tbb[NS], ub[NS], db[NS], lb[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                uM[s] = sT[j][0][0][0][s][q];
                dM[s] = sT[j][0][0][1][s][q];
                uP[s] = sT[j][1][0][0][s][q];
                dP[s] = sT[j][1][0][1][s][q];
                del[s] = uM[s] - uP[s];
                sb[s] = sS[j][0][s][q];
                tbb[s] = sS[j][1][s][q];
                double acc = 0.0;
                for (int p = 0; p < NP; ++p) acc = fma(sS[j][0][s][p], tb.LF[frM][p][q], acc);
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
            const int fr = sI[j][2 + side];
            double acc = 0.0;
            for (int p = 0; p < NP; ++p)
                acc = fma(sA[j][side][0][s][p], tb.FB[fr][p][m], fma(sA[j][side][1][s][p], sDN[j][side][p][m], acc));
            a.fbuf[((f0 + j) * 2 + side) * NS * NB + s * NB + m] = acc;
        }
        return;
    }
    for (int i = threadIdx.x; i < nf * NP; i += blockDim.x) {
        const int j = i / NP, p = i % NP;
        const int frM = sI[j][2];
        const double lift = -sF[j][3] / (2.0 * sF[j][4]);
        double uM[NS], dM[NS], uP[NS], dP[NS], del[NS], sig[NS], tau[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            uM[s] = sT[j][0][0][0][s][p];
            dM[s] = sT[j][0][0][1][s][p];
            uP[s] = sT[j][1][0][0][s][p];
            dP[s] = sT[j][1][0][1][s][p];
            del[s] = uM[s] - uP[s];
        }
        if constexpr (MODE == TET_APPLY) {
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
        const double w = tb.FW[p];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            double rn = 0.0;
            for (int q = 0; q < NP; ++q) rn = fma(tb.LF[frM][p][q], sD[j][s][q], rn);
            sS[j][0][s][p] = w * fma(2.0 * a.chi_e * a.c.A[s] * lift, rn, sig[s]);
            sS[j][1][s][p] = w * tau[s];
        }
    }
    __syncthreads();
    // test: K^- gets sigma phi^- + tau d_n phi^-, K^+ gets -sigma phi^+ + tau d_n phi^+
    for (int i = threadIdx.x; i < nf * 2 * NS * NB; i += blockDim.x) {
        const int j = i / (2 * NS * NB), side = (i / (NS * NB)) % 2, s = (i / NB) % NS, m = i % NB;
        const int fr = sI[j][2 + side];
        double as = 0.0, at = 0.0;
        for (int p = 0; p < NP; ++p) {
            as = fma(sS[j][0][s][p], tb.FB[fr][p][m], as);
            at = fma(sS[j][1][s][p], sDN[j][side][p][m], at);
        }
        a.fbuf[((f0 + j) * 2 + side) * NS * NB + s * NB + m] = sF[j][3] * (side ? at - as : at + as);
    }
}

// One CTA: one element.  Values and physical gradients of every field per
// (point, species) by sum factorisation over the warped-product basis on the
// collapsed grid (coefficients -> C_pqr in w -> B_pq in v -> A_p in u, and the
// derivative factors for the (u, v, w) gradient, mapped to the reference and
// then the physical gradient), the pointwise flux (JVP: linearised; VJP: its
// adjoint with the cotangents det w_q mu, det w_q grad mu), the result mapped
// back by J^{-1} and by the collapsed map, weighted, and tested by the
// transposed passes (A_p in u -> B_pq in v -> C_pqr in w), the tested fluxes
// of its interior faces, the boundary data of Eq. (3) on its boundary faces
// (apply only: H' = 0), M^{-1} = 1 / det J (not for the VJP).
// Apply and JVP take the diffusion of n2..c3 in modal form: -A_s K_e U_s with
// the element stiffness K_e = det J sum_c G_c KS[c] (G = J^{-1} J^{-T}; exact,
// as the volume rule integrates the stiffness exactly), so the forward passes
// carry gradients for n1, c1, c3 only (what the fluxes read) and the test
// passes carry the flux for n1, n2 only; the other species are tested against
// the source alone.  The VJP keeps the full passes.  Dynamic shared memory per
// field: U [6][nb], the w-pass [2][6][pairs][n], the v-pass [3][6][k+1][n][n],
// the point values [NQ][6 * 4 + 1] (an odd stride per point: threads on
// consecutive points hit distinct banks).  The w- and v-pass buffers hold the
// values of all six species and the derivatives of the NGF species carrying
// gradients (their slots); the test passes reuse them for the six values and
// the derivative parts of the species with a flux.
template <int K, bool MODAL>
struct TetSF {
    static constexpr int N = K + 2, NPQ = (K + 1) * (K + 2) / 2, K1 = K + 1;
    static constexpr int NB = TetShape<K>::NB, NQ = TetShape<K>::NQ;
    static constexpr int NGF = MODAL ? 3 : NS;   // species carrying gradients in the forward passes
    static constexpr int QS = NS * 4 + 1;
    static constexpr int SU = NS * NB, SG1 = (NS + NGF) * NPQ * N, SH = (NS + 2 * NGF) * K1 * N * N, SQ = NQ * QS;
    static constexpr int FIELD = SU + SG1 + SH + SQ;   // doubles per field
};

template <int K, int MODE>
__global__ void __launch_bounds__(128) tet_elem_kernel(const TetArgs a) {
    using S = TetShape<K>;
    constexpr bool MODAL = MODE != TET_VJP;
    using SF = TetSF<K, MODAL>;
    constexpr int NB = S::NB, NQ = S::NQ, NP = S::NP, F = MODE == TET_APPLY ? 1 : 2;
    constexpr int N = SF::N, NPQ = SF::NPQ, K1 = SF::K1, QS = SF::QS;
    constexpr int NGF = SF::NGF;          // forward slots carrying gradients
    constexpr int NGT = MODAL ? 2 : NS;   // species tested against a flux (<= NGF)
    const TetTab& tb = *a.tab;
    extern __shared__ __align__(16) double tsm[];
    auto sU = [&](int fi) { return reinterpret_cast<double (*)[NB]>(tsm + fi * SF::FIELD); };
    // w-pass (and test v-pass) buffers: the values of species s, the derivative of slot sl
    auto Gv = [&](int fi, int s) { return reinterpret_cast<double (*)[N]>(tsm + fi * SF::FIELD + SF::SU + s * NPQ * N); };
    auto Gg = [&](int fi, int sl) {
        return reinterpret_cast<double (*)[N]>(tsm + fi * SF::FIELD + SF::SU + (NS + sl) * NPQ * N);
    };
    // v-pass (and test u-pass) buffers: c = 0 values of species idx, c = 1, 2 the derivatives of slot idx
    auto Hc = [&](int fi, int c, int idx) {
        return reinterpret_cast<double (*)[N][N]>(tsm + fi * SF::FIELD + SF::SU + SF::SG1 +
                                                  ((c == 0 ? 0 : c == 1 ? NS : NS + NGF) + idx) * K1 * N * N);
    };
    auto sQ = [&](int fi, int q, int s) {   // (d_x, d_y, d_z, value) of species s at point q
        return tsm + fi * SF::FIELD + SF::SU + SF::SG1 + SF::SH + q * QS + s * 4;
    };
    __shared__ double sG[TGEO];
    const long long e = blockIdx.x;
    for (int i = threadIdx.x; i < TGEO; i += blockDim.x) sG[i] = a.geo[e * TGEO + i];
    for (int i = threadIdx.x; i < F * NS * NB; i += blockDim.x) {
        const int fi = i / (NS * NB), r = i % (NS * NB);
        sU(fi)[r / NB][r % NB] = (fi ? a.dU : a.U)[e * NS * NB + r];
    }
    __syncthreads();
    const double* J = sG + 3;
    const double* Ji = sG + 12;
    const double det = sG[21];
    // w-pass: g_pq(w_l) = sum_r C_pqr(w_l) U_pqr, and with C' where gradients are carried
    for (int i = threadIdx.x; i < F * NS * NPQ * N; i += blockDim.x) {
        const int fi = i / (NS * NPQ * N), sl = (i / (NPQ * N)) % NS, pq = (i / N) % NPQ, l = i % N;
        const int s = MODAL ? modal_fwd_species(sl) : sl;
        double g = 0.0, gw = 0.0;
        if (sl < NGF) {
#pragma unroll
            for (int r = 0; r < K1; ++r) {
                const int m = tb.PQM[pq][r];
                if (m >= 0) {
                    const double u = sU(fi)[s][m];
                    g = fma(tb.SC[l][m], u, g);
                    gw = fma(tb.SdC[l][m], u, gw);
                }
            }
            Gg(fi, sl)[pq][l] = gw;
        } else {
#pragma unroll
            for (int r = 0; r < K1; ++r) {
                const int m = tb.PQM[pq][r];
                if (m >= 0) g = fma(tb.SC[l][m], sU(fi)[s][m], g);
            }
        }
        Gv(fi, s)[pq][l] = g;
    }
    __syncthreads();
    // v-pass: h_p(v_j, w_l) = sum_q B_pq(v_j) g_pq(w_l); with B' (d_v) and with g' (d_w)
    for (int i = threadIdx.x; i < F * NS * K1 * N * N; i += blockDim.x) {
        const int fi = i / (NS * K1 * N * N), sl = (i / (K1 * N * N)) % NS, p = (i / (N * N)) % K1;
        const int j = (i / N) % N, l = i % N;
        const int s = MODAL ? modal_fwd_species(sl) : sl;
        double h = 0.0, hv = 0.0, hw = 0.0;
        if (sl < NGF) {
#pragma unroll
            for (int q = 0; q < K1; ++q) {
                if (q <= K - p) {
                    const int pq = tb.PQA[p][q];
                    const double g = Gv(fi, s)[pq][l];
                    h = fma(tb.SB[j][pq], g, h);
                    hv = fma(tb.SdB[j][pq], g, hv);
                    hw = fma(tb.SB[j][pq], Gg(fi, sl)[pq][l], hw);
                }
            }
            Hc(fi, 1, sl)[p][j][l] = hv;
            Hc(fi, 2, sl)[p][j][l] = hw;
        } else {
#pragma unroll
            for (int q = 0; q < K1; ++q) {
                if (q <= K - p) {
                    const int pq = tb.PQA[p][q];
                    h = fma(tb.SB[j][pq], Gv(fi, s)[pq][l], h);
                }
            }
        }
        Hc(fi, 0, s)[p][j][l] = h;
    }
    __syncthreads();
    // u-pass: value, and where carried the (u, v, w) gradient mapped to the
    // reference and physical gradient, at every point (consecutive threads on
    // consecutive points)
    for (int i = threadIdx.x; i < F * NS * NQ; i += blockDim.x) {
        const int fi = i / (NS * NQ), sl = (i / NQ) % NS, q = i % NQ;
        const int s = MODAL ? modal_fwd_species(sl) : sl;
        const int ii = q % N, j = (q / N) % N, l = q / (N * N);
        double* Q = sQ(fi, q, s);
        double f = 0.0;
        if (sl < NGF) {
            double fu = 0.0, fv = 0.0, fw = 0.0;
#pragma unroll
            for (int p = 0; p < K1; ++p) {
                const double h = Hc(fi, 0, s)[p][j][l];
                f = fma(tb.SA[ii][p], h, f);
                fu = fma(tb.SdA[ii][p], h, fu);
                fv = fma(tb.SA[ii][p], Hc(fi, 1, sl)[p][j][l], fv);
                fw = fma(tb.SA[ii][p], Hc(fi, 2, sl)[p][j][l], fw);
            }
            const double r0 = tb.SG[q][0] * fu;
            const double r1 = fma(tb.SG[q][1], fu, tb.SG[q][2] * fv);
            const double r2 = fma(tb.SG[q][1], fu, fma(tb.SG[q][3], fv, fw));
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) Q[jj] = Ji[jj] * r0 + Ji[3 + jj] * r1 + Ji[6 + jj] * r2;   // J^{-T} grad_ref
        } else {
#pragma unroll
            for (int p = 0; p < K1; ++p) f = fma(tb.SA[ii][p], Hc(fi, 0, s)[p][j][l], f);
        }
        Q[3] = f;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
        double u[NS], g[NS][3], Phi[NS][3], Sr[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const double* Q = sQ(0, q, s);
            u[s] = Q[3];
            const bool hasg = !MODAL || s == 0 || s == 3 || s == 5;
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) g[s][jj] = hasg ? Q[jj] : 0.0;
        }
        if constexpr (MODE == TET_APPLY) {
            volume_point<3, double, true>(a.c, u, g, Phi, Sr);
        } else {
            double du[NS], dg[NS][3];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                const double* Q = sQ(F - 1, q, s);
                du[s] = Q[3];
                const bool hasg = !MODAL || s == 0 || s == 3 || s == 5;
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) dg[s][jj] = hasg ? Q[jj] : 0.0;
            }
            if constexpr (MODE == TET_JVP) {
                volume_point_lin<3, double, true>(a.c, u, g, du, dg, false, Phi, Sr);
            } else {
                // mu = M^{-1} lambda = lambda / det (with CDG2_MINV); w_q is applied below
                const double W = (a.flags & CDG2_MINV) ? 1.0 : det;
                double sb[NS], gb[NS][3], th[8];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    sb[s] = W * du[s];
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) gb[s][jj] = W * dg[s][jj];
                }
                volume_point_adj<3, double>(a.c, u, g, sb, gb, Sr, Phi, th);   // Sr <- ub, Phi <- Gb
            }
        }
        // Phi . grad psi = (J_c^{-1} J^{-1} Phi) . grad_(u,v,w) psi; weighted by w_q
        // (in place: this thread alone owns point q of the last field)
        const double wq = tb.VW[q];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            double* Q = sQ(F - 1, q, s);
            if (s < NGT) {
                const double p0 = Ji[0] * Phi[s][0] + Ji[1] * Phi[s][1] + Ji[2] * Phi[s][2];
                const double p1 = Ji[3] * Phi[s][0] + Ji[4] * Phi[s][1] + Ji[5] * Phi[s][2];
                const double p2 = Ji[6] * Phi[s][0] + Ji[7] * Phi[s][1] + Ji[8] * Phi[s][2];
                Q[0] = wq * (tb.SG[q][0] * p0 + tb.SG[q][1] * (p1 + p2));
                Q[1] = wq * (tb.SG[q][2] * p1 + tb.SG[q][3] * p2);
                Q[2] = wq * p2;
            }
            Q[3] = wq * Sr[s];
        }
    }
    __syncthreads();
    // transposed u-pass: X_p(v_j, w_l) = sum_i A_p S + A'_p P_u, A_p P_v, A_p P_w
    // (species without a flux: A_p S only), into the v-pass buffers of field 0
    for (int i = threadIdx.x; i < NS * K1 * N * N; i += blockDim.x) {
        const int s = i / (K1 * N * N), p = (i / (N * N)) % K1, j = (i / N) % N, l = i % N;
        double x0 = 0.0, xv = 0.0, xw = 0.0;
        if (s < NGT) {
#pragma unroll
            for (int ii = 0; ii < N; ++ii) {
                const double* P = sQ(F - 1, ii + N * (j + N * l), s);
                x0 = fma(tb.SA[ii][p], P[3], fma(tb.SdA[ii][p], P[0], x0));
                xv = fma(tb.SA[ii][p], P[1], xv);
                xw = fma(tb.SA[ii][p], P[2], xw);
            }
            Hc(0, 1, s)[p][j][l] = xv;
            Hc(0, 2, s)[p][j][l] = xw;
        } else {
#pragma unroll
            for (int ii = 0; ii < N; ++ii) x0 = fma(tb.SA[ii][p], sQ(F - 1, ii + N * (j + N * l), s)[3], x0);
        }
        Hc(0, 0, s)[p][j][l] = x0;
    }
    __syncthreads();
    // K_e / det J = sum_c G_c KS[c] with G_ab = sum_c (J^{-1})_ac (J^{-1})_bc for ab = 00, 11, 22, 01,
    // 02, 12, over the point values of the last field (dead once the transposed u-pass has read them)
    double (*sKe)[NB] = reinterpret_cast<double (*)[NB]>(sQ(F - 1, 0, 0));
    if constexpr (MODAL) {
        double G[6];
        const int PA[6] = {0, 1, 2, 0, 0, 1}, PB[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int c = 0; c < 6; ++c)
            G[c] = fma(Ji[3 * PA[c]], Ji[3 * PB[c]],
                       fma(Ji[3 * PA[c] + 1], Ji[3 * PB[c] + 1], Ji[3 * PA[c] + 2] * Ji[3 * PB[c] + 2]));
        for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
            const int r = i / NB, cc = i % NB;
            double kk = 0.0;
#pragma unroll
            for (int c = 0; c < 6; ++c) kk = fma(G[c], tb.KS[c][r][cc], kk);
            sKe[r][cc] = kk;
        }
    }
    // transposed v-pass: Y_pq(w_l) = sum_j B_pq X + B'_pq X_v; Y^w_pq = sum_j B_pq X_w
    for (int i = threadIdx.x; i < NS * NPQ * N; i += blockDim.x) {
        const int s = i / (NPQ * N), pq = (i / N) % NPQ, l = i % N;
        int p = 0;
        while (p < K && pq >= tb.PQA[p + 1][0]) ++p;
        double y = 0.0, yw = 0.0;
        if (s < NGT) {
#pragma unroll
            for (int j = 0; j < N; ++j) {
                y = fma(tb.SB[j][pq], Hc(0, 0, s)[p][j][l], fma(tb.SdB[j][pq], Hc(0, 1, s)[p][j][l], y));
                yw = fma(tb.SB[j][pq], Hc(0, 2, s)[p][j][l], yw);
            }
            Gg(0, s)[pq][l] = yw;
        } else {
#pragma unroll
            for (int j = 0; j < N; ++j) y = fma(tb.SB[j][pq], Hc(0, 0, s)[p][j][l], y);
        }
        Gv(0, s)[pq][l] = y;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NS * NB; i += blockDim.x) {
        const int s = i / NB, m = i % NB;
        const int pq = tb.MPQ[m];
        double acc = 0.0;
        if (s < NGT) {
#pragma unroll
            for (int l = 0; l < N; ++l)
                acc = fma(tb.SC[l][m], Gv(0, s)[pq][l], fma(tb.SdC[l][m], Gg(0, s)[pq][l], acc));
        } else {
#pragma unroll
            for (int l = 0; l < N; ++l) acc = fma(tb.SC[l][m], Gv(0, s)[pq][l], acc);
        }
        if constexpr (MODAL) {
            if (s > 0) {   // the diffusion of n2..c3 (of the tangent in the JVP): -A_s (K_e U_s)_m / det J
                double kd = 0.0;
#pragma unroll 4
                for (int jj = 0; jj < NB; ++jj) kd = fma(sKe[m][jj], sU(F - 1)[s][jj], kd);
                acc = fma(-a.c.A[s], kd, acc);
            }
        }
        double R = MODE == TET_VJP ? acc : det * acc;   // (the VJP's cotangents carry det)
        for (int l = 0; l < 4; ++l) {
            const int code = a.emap[e * 4 + l];
            if (code >= 0) {
                R += a.fbuf[(long long)code * NS * NB + s * NB + m];
            } else if (MODE == TET_APPLY && code != -1) {
                // boundary face l on Gamma_1 (code -2) or Gamma_2 (code -3), in e's own frame
                const int f = -code - 2;
                const int va = l == 0 ? 1 : 0, vb = l <= 1 ? 2 : 1, vc = l <= 2 ? 3 : 2;   // the vertices other than l
                const int fr = frame_code(va, vb, vc);
                double X[3][3];   // the face's vertices
                const int vv[3] = {va, vb, vc};
                for (int t = 0; t < 3; ++t) {
                    const double r0 = vv[t] == 1 ? 1.0 : 0.0, r1 = vv[t] == 2 ? 1.0 : 0.0, r2 = vv[t] == 3 ? 1.0 : 0.0;
                    for (int jj = 0; jj < 3; ++jj) X[t][jj] = sG[jj] + J[3 * jj] * r0 + J[3 * jj + 1] * r1 + J[3 * jj + 2] * r2;
                }
                double e1[3], e2[3];
                for (int jj = 0; jj < 3; ++jj) {
                    e1[jj] = X[1][jj] - X[0][jj];
                    e2[jj] = X[2][jj] - X[0][jj];
                }
                const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
                             cz = e1[0] * e2[1] - e1[1] * e2[0];
                const double E2 = sqrt(cx * cx + cy * cy + cz * cz);
                double bacc = 0.0;
                for (int p = 0; p < NP; ++p) {
                    double uo[NS] = {0, 0, 0, 0, 0, 0}, sig[NS];
                    double c1 = 0.0;
                    for (int mm = 0; mm < NB; ++mm) c1 = fma(tb.FB[fr][p][mm], sU(0)[3][mm], c1);
                    uo[3] = c1;
                    const double x = X[0][0] + tb.FX[p][0] * e1[0] + tb.FX[p][1] * e2[0];
                    boundary_point<double>(a.c, f, x, a.g, uo, sig, a.c.beta1, true);
                    bacc = fma(tb.FW[p], sig[s] * tb.FB[fr][p][m], bacc);
                }
                R += E2 * bacc;
            }
        }
        a.out[e * NS * NB + s * NB + m] = (MODE != TET_VJP && (a.flags & CDG2_MINV)) ? R / det : R;
    }
}

}  // namespace cdg2

namespace cdg2 {

template <int K, int MODE>
static cudaError_t tet_launch(const TetArgs& a, cudaStream_t st) {
    constexpr int FPB = MODE == TET_APPLY ? 2 : 1;   // faces per CTA (static shared memory <= 48 KB)
    constexpr int F = MODE == TET_APPLY ? 1 : 2;
    constexpr size_t smem = sizeof(double) * (size_t)F * TetSF<K, MODE != TET_VJP>::FIELD;
    static DeviceOnce attr;   // per instantiation and device
    {
        cudaError_t e = once_per_device(attr, [] {
            return cudaFuncSetAttribute(tet_elem_kernel<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem);
        });
        if (e != cudaSuccess) return e;
    }
    if (a.NF > 0) tet_face_kernel<K, FPB, MODE><<<(unsigned)((a.NF + FPB - 1) / FPB), 128, 0, st>>>(a);
    tet_elem_kernel<K, MODE><<<(unsigned)a.E, 128, smem, st>>>(a);
    return cudaGetLastError();
}

static int tet_upload(const cdg2_tet_mesh& m) {
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
    up((void**)&m.d_tab, m.tab.data(), sizeof(TetTab));
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_tet_apply: mesh upload");
    return CDG2_OK;
}

}  // namespace cdg2

using namespace cdg2;

extern "C" int cdg2_tet_mesh_create(const cdg2_tet_desc* d, cdg2_tet_mesh** out) {
    if (!d || !out || !d->xyz || !d->tet) {
        set_error("cdg2_tet_mesh_create: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (d->k < 1 || d->k > 3 || d->n_vert < 4 || d->n_tet < 1 || d->n_tet > (1LL << 28)) {
        set_error("cdg2_tet_mesh_create: need 1 <= k <= 3, n_vert >= 4, 1 <= n_tet < 2^28");
        return CDG2_ERR_INVALID_ARG;
    }
    auto* m = new (std::nothrow) cdg2_tet_mesh;
    if (!m) {
        set_error("cdg2_tet_mesh_create: out of host memory");
        return CDG2_ERR_INVALID_ARG;
    }
    auto fail = [&](const std::string& msg) {
        delete m;
        set_error("cdg2_tet_mesh_create: " + msg);
        return CDG2_ERR_INVALID_ARG;
    };
    m->k = d->k;
    m->nb = (d->k + 1) * (d->k + 2) * (d->k + 3) / 6;
    m->E = d->n_tet;
    m->chi_e = d->chi_e > 0.0 ? d->chi_e : 2.0;
    m->g1in[0] = d->gamma1_in[0];
    m->g1in[1] = d->gamma1_in[1];
    const double* X = d->xyz;
    double ly = X[1];
    for (long long v = 0; v < d->n_vert; ++v) ly = std::max(ly, X[3 * v + 1]);
    m->ly = ly;
    m->geo.assign((size_t)m->E * TGEO, 0.0);
    for (long long e = 0; e < m->E; ++e) {
        long long v[4];
        for (int j = 0; j < 4; ++j) {
            v[j] = d->tet[4 * e + j];
            if (v[j] < 0 || v[j] >= d->n_vert) return fail("vertex index out of range");
        }
        double J[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) J[r][c] = X[3 * v[c + 1] + r] - X[3 * v[0] + r];
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        if (!(det > 0.0))
            return fail("tetrahedron " + std::to_string(e) + " is degenerate or negatively oriented");
        double* G = &m->geo[(size_t)e * TGEO];
        for (int r = 0; r < 3; ++r) G[r] = X[3 * v[0] + r];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) G[3 + 3 * r + c] = J[r][c];
        // inverse by cofactors
        G[12] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        G[13] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        G[14] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        G[15] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        G[16] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        G[17] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        G[18] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        G[19] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        G[20] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        G[21] = det;
    }
    std::map<std::vector<long long>, std::vector<std::pair<long long, int>>> faces;
    for (long long e = 0; e < m->E; ++e)
        for (int l = 0; l < 4; ++l) {
            std::vector<long long> key;
            for (int t = 0; t < 3; ++t) key.push_back(d->tet[4 * e + FACE_VERTS[l][t]]);
            std::sort(key.begin(), key.end());
            faces[key].push_back({e, l});
        }
    m->emap.assign((size_t)m->E * 4, -1);
    const double tol = 1e-12 * std::max(1.0, ly);
    for (const auto& kv : faces) {
        const auto& own = kv.second;
        if (own.size() == 2) {
            long long e1 = own[0].first, e2 = own[1].first;
            int l1 = own[0].second, l2 = own[1].second;
            const double v1 = m->geo[(size_t)e1 * TGEO + 21], v2 = m->geo[(size_t)e2 * TGEO + 21];
            const bool tie = std::fabs(v1 - v2) <= 1e-12 * std::max(v1, v2);
            if (!((!tie && v1 < v2) || (tie && e1 < e2))) {
                std::swap(e1, e2);
                std::swap(l1, l2);
            }
            // K^-'s face vertices in its order, and their local indices in K^+
            long long gv[3];
            int lp[3];
            for (int t = 0; t < 3; ++t) {
                gv[t] = d->tet[4 * e1 + FACE_VERTS[l1][t]];
                lp[t] = -1;
                for (int c = 0; c < 4; ++c)
                    if (d->tet[4 * e2 + c] == gv[t]) lp[t] = c;
                if (lp[t] < 0 || lp[t] == l2) return fail("inconsistent face between tetrahedra");
            }
            const int frM = frame_code(FACE_VERTS[l1][0], FACE_VERTS[l1][1], FACE_VERTS[l1][2]);
            const int frP = frame_code(lp[0], lp[1], lp[2]);
            const long long f = (long long)m->face.size() / 4;
            m->face.insert(m->face.end(), {(int)e1, (int)e2, frM, frP});
            double A[3], B[3], C[3], opp[3];
            for (int r = 0; r < 3; ++r) {
                A[r] = X[3 * gv[0] + r];
                B[r] = X[3 * gv[1] + r];
                C[r] = X[3 * gv[2] + r];
                opp[r] = X[3 * d->tet[4 * e1 + l1] + r];
            }
            const double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
            const double w[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
            double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
            const double E2 = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            double side = 0.0;
            for (int r = 0; r < 3; ++r) side += cr[r] * (opp[r] - A[r]);
            const double sg = side > 0.0 ? -1.0 : 1.0;   // the normal points away from K^-'s opposite vertex
            m->fgeo.insert(m->fgeo.end(), {sg * cr[0] / E2, sg * cr[1] / E2, sg * cr[2] / E2, E2,
                                           m->geo[(size_t)e1 * TGEO + 21]});
            m->emap[(size_t)e1 * 4 + l1] = (int)(2 * f);
            m->emap[(size_t)e2 * 4 + l2] = (int)(2 * f + 1);
        } else if (own.size() == 1) {
            bool g1 = true, g2 = true;
            for (long long v : kv.first) {
                const double y = X[3 * v + 1];
                g1 = g1 && std::fabs(y) <= tol;
                g2 = g2 && std::fabs(y - ly) <= tol;
            }
            const int tag = g1 ? 1 : (g2 ? 2 : 0);
            m->emap[(size_t)own[0].first * 4 + own[0].second] = -1 - tag;
        } else {
            return fail("a face is shared by more than two tetrahedra");
        }
    }
    m->NF = (long long)m->face.size() / 4;
    m->tab.resize(1);
    build_tet_tables(m->k, m->tab[0]);
    *out = m;
    return CDG2_OK;
}

extern "C" void cdg2_tet_mesh_destroy(cdg2_tet_mesh* m) {
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

extern "C" int cdg2_tet_mesh_info(const cdg2_tet_mesh* m, long long* n_elem, int* n_basis, long long* n_dof,
                                  long long* n_faces) {
    if (!m) {
        set_error("cdg2_tet_mesh_info: NULL mesh");
        return CDG2_ERR_INVALID_ARG;
    }
    if (n_elem) *n_elem = m->E;
    if (n_basis) *n_basis = m->nb;
    if (n_dof) *n_dof = m->E * NS * m->nb;
    if (n_faces) *n_faces = m->NF;
    return CDG2_OK;
}

static int tet_run(const char* who, const cdg2_tet_mesh* m, const cdg2_params* p, const double* U, const double* dU,
                   double* out, int flags, int mode, void* stream) {
    if (!m || !p || !U || !out || (mode != TET_APPLY && !dU)) {
        set_error(std::string(who) + ": NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (U == out || dU == out) {
        set_error(std::string(who) + ": the inputs and out must not overlap");
        return CDG2_ERR_INVALID_ARG;
    }
    if (flags & ~(CDG2_MINV | CDG2_ASYNC)) {
        set_error(std::string(who) + ": only CDG2_MINV and CDG2_ASYNC are supported on tetrahedral meshes");
        return CDG2_ERR_INVALID_ARG;
    }
    if (int rc = tet_upload(*m)) return rc;
    if (cudaError_t e = ensure_status(&m->status)) return cuda_fail(e, who);
    TetArgs a;
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
    g.dim = 3;
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
#define TET_DISPATCH(MODE)                                       \
    switch (m->k) {                                              \
        case 1: e = tet_launch<1, MODE>(a, st); break;           \
        case 2: e = tet_launch<2, MODE>(a, st); break;           \
        default: e = tet_launch<3, MODE>(a, st); break;          \
    }
    if (mode == TET_APPLY) {
        TET_DISPATCH(TET_APPLY)
    } else if (mode == TET_JVP) {
        TET_DISPATCH(TET_JVP)
    } else {
        TET_DISPATCH(TET_VJP)
    }
#undef TET_DISPATCH
    if (e != cudaSuccess) return cuda_fail(e, who);
    if (flags & CDG2_ASYNC) return CDG2_OK;
    return take_domain_status(m->status, st, who);
}

extern "C" int cdg2_tet_mesh_status(const cdg2_tet_mesh* m, void* stream) {
    if (!m) {
        set_error("cdg2_tet_mesh_status: NULL mesh");
        return CDG2_ERR_INVALID_ARG;
    }
    return take_domain_status(m->status, (cudaStream_t)stream, "cdg2_tet_mesh_status");
}

extern "C" int cdg2_tet_apply(const cdg2_tet_mesh* m, const cdg2_params* p, const double* U, double* out, int flags,
                              void* stream) {
    return tet_run("cdg2_tet_apply", m, p, U, nullptr, out, flags, TET_APPLY, stream);
}

extern "C" int cdg2_tet_jvp(const cdg2_tet_mesh* m, const cdg2_params* p, const double* U, const double* dU,
                            double* out, int flags, void* stream) {
    return tet_run("cdg2_tet_jvp", m, p, U, dU, out, flags, TET_JVP, stream);
}

extern "C" int cdg2_tet_vjp(const cdg2_tet_mesh* m, const cdg2_params* p, const double* U, const double* lam,
                            double* gU, int flags, void* stream) {
    return tet_run("cdg2_tet_vjp", m, p, U, lam, gU, flags, TET_VJP, stream);
}

namespace {
struct TetStepCtx {
    const cdg2_tet_mesh* m;
    const cdg2_params* p;
};
int tet_step_apply(const void* ctx, const double* Y, double* out, cudaStream_t st) {
    const auto* c = static_cast<const TetStepCtx*>(ctx);
    return tet_run("cdg2_tet_step", c->m, c->p, Y, nullptr, out, CDG2_MINV | CDG2_ASYNC, TET_APPLY, st);
}
int tet_step_jvp(const void* ctx, const double* Y, const double* v, double* out, cudaStream_t st) {
    const auto* c = static_cast<const TetStepCtx*>(ctx);
    return tet_run("cdg2_tet_step", c->m, c->p, Y, v, out, CDG2_MINV | CDG2_ASYNC, TET_JVP, st);
}
int tet_step_jvp_diffusion(const void* ctx, const double* v, double* out, cudaStream_t st) {
    const auto* c = static_cast<const TetStepCtx*>(ctx);
    const cdg2_params q = cdg2::diffusion_only(*c->p);
    return tet_run("cdg2_tet_step", c->m, &q, v, v, out, CDG2_MINV | CDG2_ASYNC, TET_JVP, st);
}
}  // namespace

extern "C" int cdg2_tet_step(const cdg2_tet_mesh* m, const cdg2_params* p, double* U, double dt,
                             const cdg2_solver_opts* opts, cdg2_stats* stats, void* stream) {
    if (!m || !p) {
        set_error("cdg2_tet_step: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    const TetStepCtx ctx{m, p};
    cdg2::SimplexStepOps ops;
    ops.n = m->E * NS * m->nb;
    ops.nb = m->nb;
    ops.ws = &m->step_ws;
    ops.ws_bytes = &m->step_ws_bytes;
    ops.ctx = &ctx;
    ops.apply = tet_step_apply;
    ops.jvp = tet_step_jvp;
    ops.jvp_diffusion = tet_step_jvp_diffusion;
    const Coef co = make_coef(*p);
    ops.A = co.A;
    ops.face = m->face.data();
    ops.NF = m->NF;
    ops.pc = &m->spc;
    if (cudaError_t e = ensure_status(&m->status)) return cuda_fail(e, "cdg2_tet_step");
    ops.dom = m->status;
    return cdg2::simplex_step(ops, U, dt, opts, stats, stream, "cdg2_tet_step");
}
