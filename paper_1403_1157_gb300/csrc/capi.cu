// C ABI entry points of the CDG2 library: argument checks, mesh set-up and
// kernel dispatch.  All arithmetic of the operator runs in the kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "cdg2_internal.h"

namespace cdg2 {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return CDG2_ERR_CUDA;
}

cudaError_t ensure_status(int** word) {
    if (*word) return cudaSuccess;
    int* p = nullptr;
    cudaError_t e = cudaMalloc(&p, sizeof(int));
    if (e != cudaSuccess) return e;
    e = cudaMemset(p, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(p);
        return e;
    }
    *word = p;
    return cudaSuccess;
}

int take_domain_status(int* word, cudaStream_t st, const char* who) {
    if (!word) return CDG2_OK;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, word, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, who);
    if (h == 0) return CDG2_OK;
    e = cudaMemsetAsync(word, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, who);
    if (h & 2) {
        set_error(std::string(who) + ": a bounded wait for the tensor cores or for bulk asynchronous copies timed "
                  "out in a kernel; its result is undefined");
        return CDG2_ERR_CUDA;
    }
    set_error(std::string(who) + ": a chemotactic sensitivity chi0 x / (y + chith) met y + chith <= 0 at a "
              "quadrature point (the pole of chi, Sec. 2): the state is outside the model's domain");
    return CDG2_ERR_DOMAIN;
}

Coef make_coef(const cdg2_params& p) {
    Coef c;
    c.A[0] = p.mu[0];
    c.A[1] = p.mu[1];
    c.A[2] = p.mu[2];
    c.A[3] = p.nu[0];
    c.A[4] = p.nu[1];
    c.A[5] = p.nu[2];
    for (int j = 0; j < 4; ++j) {
        c.chi0[j] = p.chi0[j];
        c.chith[j] = p.chith[j];
    }
    c.d1 = p.d1;
    c.d2 = p.d2;
    c.gamma = p.gamma;
    c.alpha1 = p.alpha1;
    c.alpha2 = p.alpha2;
    c.f1 = p.f1;
    c.k_ox = p.k_ox;
    c.beta1 = p.beta1;
    c.beta2 = p.beta2;
    c.sigma = p.sigma;
    c.c1s = p.c1_star;
    c.c1ss = p.c1_star2;
    c.bc_sign = p.bc_sign;
    for (int s = 0; s < NS; ++s) c.phase[s] = p.mms_phase[s];
    c.model = p.model;
    if (p.model == 1) {
        // Reduced model of Eq. (2) (Sec. 4.2): only n1, n3, c1 evolve.  Species
        // n2, c2, c3 are inactive (no diffusion, taxis, sources or inflow;
        // their fields are expected to be zero), n1 loses its c3-taxis and its
        // death term, c1 loses the alpha2 term; n3 keeps d1 n1 - gamma n1.
        c.A[1] = c.A[4] = c.A[5] = 0.0;
        c.chi0[1] = c.chi0[2] = c.chi0[3] = 0.0;
        c.d2 = c.alpha2 = c.k_ox = 0.0;
        c.beta2 = c.sigma = 0.0;
    }
    return c;
}

// Legendre P_m(t) and P'_m(t), m = 0..n, by the three-term recurrence.
static void legendre(int n, double t, double* P, double* dP) {
    P[0] = 1.0;
    dP[0] = 0.0;
    if (n == 0) return;
    P[1] = t;
    dP[1] = 1.0;
    for (int m = 1; m < n; ++m) {
        P[m + 1] = ((2 * m + 1) * t * P[m] - m * P[m - 1]) / (m + 1);
        dP[m + 1] = dP[m - 1] + (2 * m + 1) * P[m];
    }
}

// n-point Gauss-Legendre rule on [0,1]: Newton iteration on P_n from the
// Chebyshev-like initial guesses cos(pi (i + 3/4) / (n + 1/2)).
void gauss01(int n, double* x, double* w) {
    double P[16], dP[16];
    for (int i = 0; i < n; ++i) {
        double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            legendre(n, t, P, dP);
            double dt = P[n] / dP[n];
            t -= dt;
            if (std::fabs(dt) < 1e-17) break;
        }
        legendre(n, t, P, dP);
        // roots come out descending in t; store ascending in xi = (1 + t) / 2
        x[n - 1 - i] = 0.5 * (1.0 + t);
        w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dP[n] * dP[n]);   // 2/((1-t^2)P'^2) halved
    }
}

static void tabulate(int k, int q1, Tab1D& T) {
    std::memset(&T, 0, sizeof(T));
    gauss01(q1, T.xi, T.w);
    double P[16], dP[16];
    for (int q = 0; q < q1; ++q) {
        legendre(k, 2.0 * T.xi[q] - 1.0, P, dP);
        for (int a = 0; a <= k; ++a) {
            T.B[q][a] = std::sqrt(2.0 * a + 1.0) * P[a];
            T.D[q][a] = 2.0 * std::sqrt(2.0 * a + 1.0) * dP[a];
        }
    }
    for (int side = 0; side < 2; ++side) {
        legendre(k, side ? 1.0 : -1.0, P, dP);
        for (int a = 0; a <= k; ++a) {
            T.e[side][a] = std::sqrt(2.0 * a + 1.0) * P[a];
            T.d[side][a] = 2.0 * std::sqrt(2.0 * a + 1.0) * dP[a];
        }
    }
}

}  // namespace cdg2

using namespace cdg2;

extern "C" {

const char* cdg2_last_error(void) { return g_err.c_str(); }

int cdg2_mesh_create(const cdg2_mesh_desc* d, cdg2_mesh** out) {
    if (!d || !out) {
        set_error("cdg2_mesh_create: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (d->dim != 2 && d->dim != 3) {
        set_error("cdg2_mesh_create: dim must be 2 or 3");
        return CDG2_ERR_INVALID_ARG;
    }
    if (d->k < 1 || d->k > MAXK) {
        set_error("cdg2_mesh_create: k must be 1, 2 or 3");
        return CDG2_ERR_INVALID_ARG;
    }
    if (d->q1 != 0 && d->q1 != d->k + 2) {
        set_error("cdg2_mesh_create: only q1 = k + 2 Gauss points are supported");
        return CDG2_ERR_INVALID_ARG;
    }
    long long E = 1;
    for (int a = 0; a < d->dim; ++a) {
        if (d->cells[a] < 1 || !(d->extent[a] > 0.0)) {
            set_error("cdg2_mesh_create: cells must be >= 1 and extents > 0");
            return CDG2_ERR_INVALID_ARG;
        }
        E *= d->cells[a];
    }
    int nb = 1;
    for (int a = 0; a < d->dim; ++a) nb *= d->k + 1;
    if (E * NS * (long long)nb > (1LL << 31) - 1) {
        set_error("cdg2_mesh_create: more than 2^31 - 1 degrees of freedom");
        return CDG2_ERR_INVALID_ARG;
    }
    cdg2_mesh* m = new (std::nothrow) cdg2_mesh();
    if (!m) {
        set_error("cdg2_mesh_create: out of host memory");
        return CDG2_ERR_INVALID_ARG;
    }
    Geo& g = m->geo;
    g.dim = d->dim;
    g.k = d->k;
    g.vol = 1.0;
    for (int a = 0; a < 3; ++a) {
        bool in = a < d->dim;
        g.n[a] = in ? d->cells[a] : 1;
        g.periodic[a] = in ? (d->periodic[a] != 0) : 1;
        g.L[a] = in ? d->extent[a] : 1.0;
        g.h[a] = g.L[a] / g.n[a];
        if (in) g.vol *= g.h[a];
    }
    g.chi_e = d->chi_e > 0.0 ? d->chi_e : (double)d->dim;
    if (d->flux < CDG2_FLUX_CDG2 || d->flux > CDG2_FLUX_SIPG) {
        delete m;
        set_error("cdg2_mesh_create: flux must be CDG2_FLUX_CDG2, CDG2_FLUX_BR2 or CDG2_FLUX_SIPG");
        return CDG2_ERR_INVALID_ARG;
    }
    {
        const double pdef = 2.0 * d->dim;
        const double pp = d->penalty > 0.0 ? d->penalty : pdef;
        // CDG2: 2 chi_e A r_e on K^-; BR2: eta A {r_e}; SIPG: the penalty itself.  With
        // r_e . n^- = -(k+1)^2 |e| / (2 |K|) Delta on either cell of these uniform meshes:
        g.pen_c = d->flux == CDG2_FLUX_CDG2 ? g.chi_e : (d->flux == CDG2_FLUX_BR2 ? 0.5 * pp : pp);
    }
    g.g1in[0] = d->gamma1_in[0];
    g.g1in[1] = d->gamma1_in[1];
    g.E = E;
    tabulate(d->k, d->k + 2, m->tab);
    m->tp64 = make_tabp<double>(m->tab, g);
    m->tp32 = make_tabp<float>(m->tab, g);
    m->nb = nb;
    m->ndof = E * NS * nb;
    *out = m;
    return CDG2_OK;
}

void cdg2_mesh_destroy(cdg2_mesh* m) {
    if (!m) return;
    if (m->theta_part) cudaFree(m->theta_part);   // synchronises work queued on it
    if (m->step_ws) cudaFree(m->step_ws);
    if (m->fbuf) cudaFree(m->fbuf);
    if (m->status) cudaFree(m->status);
    if (m->tc_tables) cudaFree(m->tc_tables);
    if (m->jac) cdg2_matrix_destroy(m->jac);
    delete m;
}

int cdg2_mesh_info(const cdg2_mesh* m, long long* n_elem, int* n_basis, long long* n_dof) {
    if (!m) {
        set_error("cdg2_mesh_info: NULL mesh");
        return CDG2_ERR_INVALID_ARG;
    }
    if (n_elem) *n_elem = m->geo.E;
    if (n_basis) *n_basis = m->nb;
    if (n_dof) *n_dof = m->ndof;
    return CDG2_OK;
}

// CDG2_TF32 (tensor-core contractions) is built for FP32 arrays on 3D Q3 meshes.
static int check_tf32(const cdg2_mesh& m, int flags, const char* who) {
    if (!(flags & CDG2_TF32)) return CDG2_OK;
    if (!(flags & CDG2_FP32) || m.geo.dim != 3 || m.geo.k != 3) {
        set_error(std::string(who) + ": CDG2_TF32 needs CDG2_FP32 and a 3D mesh of degree 3");
        return CDG2_ERR_INVALID_ARG;
    }
    return CDG2_OK;
}

int cdg2_mesh_status(const cdg2_mesh* m, void* stream) {
    if (!m) {
        set_error("cdg2_mesh_status: NULL mesh");
        return CDG2_ERR_INVALID_ARG;
    }
    return take_domain_status(m->status, (cudaStream_t)stream, "cdg2_mesh_status");
}

int cdg2_apply(const cdg2_mesh* m, const cdg2_params* p, const void* U, void* out, int flags, double t,
               void* stream) {
    if (!m || !p || !U || !out) {
        set_error("cdg2_apply: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (U == out) {
        set_error("cdg2_apply: U and out must not overlap");
        return CDG2_ERR_INVALID_ARG;
    }
    if (flags & ~(CDG2_MINV | CDG2_FORCING | CDG2_FP32 | CDG2_ASYNC | CDG2_TF32)) {
        set_error("cdg2_apply: unknown flag bits");
        return CDG2_ERR_INVALID_ARG;
    }
    if (int rc = check_tf32(*m, flags, "cdg2_apply")) return rc;
    Coef c = make_coef(*p);
    cudaError_t e = launch_apply(*m, c, U, out, flags, t, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_apply");
    if (flags & CDG2_ASYNC) return CDG2_OK;
    return take_domain_status(m->status, (cudaStream_t)stream, "cdg2_apply");
}

int cdg2_jvp(const cdg2_mesh* m, const cdg2_params* p, const void* U, const void* dU, const double* dtheta,
             void* out, int flags, double t, void* stream) {
    (void)t;   // the forcing does not depend on U or on the coefficients
    if (!m || !p || !U || !dU || !out) {
        set_error("cdg2_jvp: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (out == U || out == dU) {
        set_error("cdg2_jvp: out must not overlap U or dU");
        return CDG2_ERR_INVALID_ARG;
    }
    if (flags & ~(CDG2_MINV | CDG2_FORCING | CDG2_FP32 | CDG2_ASYNC | CDG2_TF32)) {
        set_error("cdg2_jvp: unknown flag bits");
        return CDG2_ERR_INVALID_ARG;
    }
    if (int rc = check_tf32(*m, flags, "cdg2_jvp")) return rc;
    Coef c = make_coef(*p);
    cudaError_t e = launch_jvp(*m, c, U, dU, dtheta, out, flags, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_jvp");
    if (flags & CDG2_ASYNC) return CDG2_OK;
    return take_domain_status(m->status, (cudaStream_t)stream, "cdg2_jvp");
}

int cdg2_vjp(const cdg2_mesh* m, const cdg2_params* p, const void* U, const void* lam, void* gU, double* gtheta,
             int flags, double t, void* stream) {
    (void)t;
    if (!m || !p || !U || !lam || !gU) {
        set_error("cdg2_vjp: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (gU == U || gU == lam) {
        set_error("cdg2_vjp: gU must not overlap U or lam");
        return CDG2_ERR_INVALID_ARG;
    }
    if (flags & ~(CDG2_MINV | CDG2_FORCING | CDG2_FP32 | CDG2_ASYNC)) {
        set_error("cdg2_vjp: unknown flag bits");
        return CDG2_ERR_INVALID_ARG;
    }
    double* part = nullptr;
    if (gtheta) {
        const long long need = vjp_grid(*m) * 8;
        if (m->theta_part_n < need) {
            if (m->theta_part) cudaFree(m->theta_part);
            m->theta_part = nullptr;
            m->theta_part_n = 0;
            cudaError_t e = cudaMalloc(&m->theta_part, sizeof(double) * need);
            if (e != cudaSuccess) return cuda_fail(e, "cdg2_vjp: workspace");
            m->theta_part_n = need;
        }
        part = m->theta_part;
    }
    Coef c = make_coef(*p);
    cudaError_t e = launch_vjp(*m, c, U, lam, gU, part, gtheta, flags, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_vjp");
    if (flags & CDG2_ASYNC) return CDG2_OK;
    return take_domain_status(m->status, (cudaStream_t)stream, "cdg2_vjp");
}

}  // extern "C"
