// L2 projection of analytic initial data onto V_h (Sec. 3.2: U(0) is the
// projection of U_0): seeded Gaussian bumps and the manufactured solution.
// One CTA per element; the field is evaluated at the q1^d Gauss points into
// shared memory, then every coefficient is w-weighted against phi_i (the
// mass matrix |K| I cancels the |K| of the quadrature weights).
#include <cmath>

#include "elem_common.cuh"

namespace cdg2 {

constexpr int MAXG = 16;   // Gaussian bumps per species

struct GaussArgs {
    int n_gauss;
    double sigma, floor;
    double c[NS][MAXG][3];
    double a[NS][MAXG];
};

template <int D, int K, typename T, int KIND>
__global__ void __launch_bounds__(128) project_kernel(const Geo g, const Tab1D tab, const GaussArgs ga,
                                                      const Coef cf, double t, T* __restrict__ out) {
    using S = Shape<D, K>;
    constexpr int NB = S::NB, NQ = S::NQ, NB1 = S::NB1, NQ1 = S::NQ1;
    __shared__ double fq[NS][NQ];
    __shared__ double B[NQ1][NB1], w[NQ1], xi[NQ1];
    const long long e = blockIdx.x;
    for (int i = threadIdx.x; i < NQ1 * NB1; i += blockDim.x) B[i / NB1][i % NB1] = tab.B[i / NB1][i % NB1];
    for (int i = threadIdx.x; i < NQ1; i += blockDim.x) {
        w[i] = tab.w[i];
        xi[i] = tab.xi[i];
    }
    __syncthreads();
    const long long ix = e % g.n[0], iy = (e / g.n[0]) % g.n[1], iz = e / ((long long)g.n[0] * g.n[1]);
    const long long ic[3] = {ix, iy, iz};
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
        const int qi[3] = {q % NQ1, (q / NQ1) % NQ1, q / (NQ1 * NQ1)};
        double x[3];
        for (int j = 0; j < D; ++j) x[j] = ic[j] * g.h[j] + g.h[j] * xi[qi[j]];
        if constexpr (KIND == 0) {
            for (int s = 0; s < NS; ++s) {
                double v = ga.floor;
                for (int b = 0; b < ga.n_gauss; ++b) {
                    double r2 = 0.0;
                    for (int j = 0; j < D; ++j) {
                        double dx = x[j] - ga.c[s][b][j];
                        if (g.periodic[j]) dx -= g.L[j] * rint(dx / g.L[j]);   // minimum image
                        r2 += dx * dx;
                    }
                    v += ga.a[s][b] * exp(-r2 / (2.0 * ga.sigma * ga.sigma));
                }
                fq[s][q] = v;
            }
        } else {
            const double pi = 3.14159265358979323846;
            for (int s = 0; s < NS; ++s)
                fq[s][q] = 1.0 + 0.5 * cos(2.0 * pi * x[0] + cf.phase[s]) * cos(pi * x[1] / g.L[1]) * exp(-t);
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < NS * NB; idx += blockDim.x) {
        const int s = idx / NB, i = idx % NB;
        const int a0 = i % NB1, a1 = (i / NB1) % NB1, a2 = i / (NB1 * NB1);
        double acc = 0.0;
        for (int q = 0; q < NQ; ++q) {
            const int q0 = q % NQ1, q1 = (q / NQ1) % NQ1, q2 = q / (NQ1 * NQ1);
            double wp = w[q0] * w[q1] * B[q0][a0] * B[q1][a1];
            if constexpr (D == 3) wp *= w[q2] * B[q2][a2];
            acc = fma(wp, fq[s][q], acc);
        }
        out[e * NS * NB + idx] = (T)acc;
    }
}

template <int KIND, typename T>
static cudaError_t launch_t(const cdg2_mesh& m, const GaussArgs& ga, const Coef& cf, double t, void* out,
                            cudaStream_t st) {
    const unsigned blocks = (unsigned)m.geo.E;
    const int d = m.geo.dim, k = m.geo.k;
#define CDG2_PROJ(D, K) \
    if (d == D && k == K) { \
        project_kernel<D, K, T, KIND><<<blocks, 128, 0, st>>>(m.geo, m.tab, ga, cf, t, (T*)out); \
        return cudaGetLastError(); \
    }
    CDG2_PROJ(2, 1)
    CDG2_PROJ(2, 2)
    CDG2_PROJ(2, 3)
    CDG2_PROJ(3, 1)
    CDG2_PROJ(3, 2)
    CDG2_PROJ(3, 3)
#undef CDG2_PROJ
    return cudaErrorInvalidValue;
}

}  // namespace cdg2

using namespace cdg2;

extern "C" {

int cdg2_project_gaussians(const cdg2_mesh* m, int n_gauss, const double* centres, const double* amps, double sigma,
                           double floor_value, void* out, int flags, void* stream) {
    if (!m || !centres || !amps || !out) {
        set_error("cdg2_project_gaussians: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (n_gauss < 0 || n_gauss > MAXG || !(sigma > 0.0) || (flags & ~CDG2_FP32)) {
        set_error("cdg2_project_gaussians: need 0 <= n_gauss <= 16, sigma > 0, flags in {0, CDG2_FP32}");
        return CDG2_ERR_INVALID_ARG;
    }
    GaussArgs ga{};
    ga.n_gauss = n_gauss;
    ga.sigma = sigma;
    ga.floor = floor_value;
    const int d = m->geo.dim;
    for (int s = 0; s < NS; ++s)
        for (int b = 0; b < n_gauss; ++b) {
            for (int j = 0; j < d; ++j) ga.c[s][b][j] = centres[(s * n_gauss + b) * d + j];
            ga.a[s][b] = amps[s * n_gauss + b];
        }
    Coef cf{};
    cudaError_t e = (flags & CDG2_FP32) ? launch_t<0, float>(*m, ga, cf, 0.0, out, (cudaStream_t)stream)
                                        : launch_t<0, double>(*m, ga, cf, 0.0, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_project_gaussians");
    return CDG2_OK;
}

int cdg2_project_mms(const cdg2_mesh* m, const cdg2_params* p, double t, void* out, int flags, void* stream) {
    if (!m || !p || !out) {
        set_error("cdg2_project_mms: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (flags & ~CDG2_FP32) {
        set_error("cdg2_project_mms: flags must be 0 or CDG2_FP32");
        return CDG2_ERR_INVALID_ARG;
    }
    GaussArgs ga{};
    Coef cf = make_coef(*p);
    cudaError_t e = (flags & CDG2_FP32) ? launch_t<1, float>(*m, ga, cf, t, out, (cudaStream_t)stream)
                                        : launch_t<1, double>(*m, ga, cf, t, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_project_mms");
    return CDG2_OK;
}

}  // extern "C"
