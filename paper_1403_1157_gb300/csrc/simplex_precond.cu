// Element-block Jacobi for the implicit step on simplicial meshes.
//
// For pure diffusion the operator M^{-1} L_h is linear and species-diagonal,
// and for a fixed element e and species s its diagonal block K_{e,s} (n_b x
// n_b: the response of e's own coefficients to e's own coefficients) is what
// the block preconditioner needs.  The blocks are probed: elements get a
// distance-1 colouring (no two elements sharing a face have one colour), and
// the JVP of the diffusion part applied to "mode i of every element of colour
// c, every species" returns, on each element of colour c, column i of its
// blocks (its neighbours, which could leak into it, are not perturbed).
// colours x n_b probes; the blocks are cached until the diffusivities change.
// For a step with dt a_ii = gdt the preconditioner is (I - gdt K_{e,s})^{-1},
// inverted per block by in-place Gauss-Jordan without pivoting: the diagonal
// blocks of the symmetric negative semi-definite diffusion operator (scaled by
// the element's constant M^{-1}) are symmetric negative semi-definite, so
// I - gdt K is symmetric positive definite with eigenvalues >= 1; a pivot that
// is not positive and finite sets an error flag instead.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cdg2_internal.h"
#include "simplex_step.h"

namespace cdg2 {

void SimplexPrecond::release() {
    cudaFree(K);
    cudaFree(Binv);
    cudaFree(color);
    cudaFree(bad);
    K = Binv = nullptr;
    color = bad = nullptr;
    valid = false;
    gdt = -1.0;
}

cdg2_params diffusion_only(const cdg2_params& p) {
    cdg2_params q = p;
    for (int i = 0; i < 4; ++i) {
        q.chi0[i] = 0.0;
        q.chith[i] = 1.0;   // no sensitivity left: keeps the probe states (0 / 1 entries) off the pole of chi
    }
    q.d1 = q.d2 = q.gamma = q.alpha1 = q.alpha2 = q.f1 = q.k_ox = 0.0;
    q.beta1 = q.beta2 = q.sigma = 0.0;
    return q;
}

// Greedy distance-1 colouring in element order: each element takes the
// smallest colour none of its face neighbours has.
static int colour_elements(long long E, long long NF, const int* face, std::vector<int>& color) {
    std::vector<std::vector<int>> nbr((size_t)E);
    for (long long f = 0; f < NF; ++f) {
        const int a = face[4 * f], b = face[4 * f + 1];
        nbr[(size_t)a].push_back(b);
        nbr[(size_t)b].push_back(a);
    }
    color.assign((size_t)E, -1);
    int nc = 0;
    std::vector<char> used;
    for (long long e = 0; e < E; ++e) {
        used.assign((size_t)nc + 1, 0);
        for (int o : nbr[(size_t)e])
            if (color[(size_t)o] >= 0) used[(size_t)color[(size_t)o]] = 1;
        int c = 0;
        while (used[(size_t)c]) ++c;
        color[(size_t)e] = c;
        nc = std::max(nc, c + 1);
    }
    return nc;
}

// probe[e][s][m] = 1 where colour(e) == c and m == i, else 0.
__global__ void k_probe(long long n, int nb, const int* color, int c, int i, double* probe) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const long long e = t / (NS * nb);
    const int m = (int)(t % nb);
    probe[t] = (color[e] == c && m == i) ? 1.0 : 0.0;
}

// K[e][s][r][i] = resp[e][s][r] on the elements of colour c.
__global__ void k_probe_take(long long n, int nb, const int* color, int c, int i, const double* resp, double* K) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const long long e = t / (NS * nb);
    if (color[e] != c) return;
    const long long blk = t / nb;
    const int r = (int)(t % nb);
    K[(blk * nb + r) * nb + i] = resp[t];
}

// Binv = (I - gdt K)^{-1}, one block per thread, in place in Binv.
__global__ void k_block_invert(long long nblk, int nb, const double* K, double gdt, double* Binv, int* bad) {
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    const double* k = K + b * nb * nb;
    double* a = Binv + b * nb * nb;
    for (int r = 0; r < nb; ++r)
        for (int j = 0; j < nb; ++j) a[r * nb + j] = (r == j ? 1.0 : 0.0) - gdt * k[r * nb + j];
    for (int p = 0; p < nb; ++p) {
        const double piv = a[p * nb + p];
        if (!(piv > 0.0) || !isfinite(piv)) {
            atomicExch(bad, 1);
            return;
        }
        const double inv = 1.0 / piv;
        a[p * nb + p] = 1.0;
        for (int j = 0; j < nb; ++j) a[p * nb + j] *= inv;
        for (int r = 0; r < nb; ++r) {
            if (r == p) continue;
            const double f = a[r * nb + p];
            a[r * nb + p] = 0.0;
            for (int j = 0; j < nb; ++j) a[r * nb + j] = fma(-f, a[p * nb + j], a[r * nb + j]);
        }
    }
}

// out[blk][r] = sum_m Binv[blk][r][m] v[blk][m].
__global__ void k_block_mul(long long n, int nb, const double* Binv, const double* v, double* out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const long long blk = t / nb;
    const double* row = Binv + t * nb;
    const double* x = v + blk * nb;
    double acc = 0.0;
    for (int m = 0; m < nb; ++m) acc = fma(row[m], x[m], acc);
    out[t] = acc;
}

static unsigned grid_of(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t simplex_block_apply(const SimplexPrecond& pc, const double* v, double* out, cudaStream_t st) {
    const long long n = pc.E * NS * pc.nb;
    if (n > 0) k_block_mul<<<grid_of(n), 256, 0, st>>>(n, pc.nb, pc.Binv, v, out);
    return cudaGetLastError();
}

int simplex_precond_setup(const SimplexStepOps& ops, double gdt, double* probe, double* resp, cudaStream_t st,
                          const char* who) {
    SimplexPrecond& pc = *ops.pc;
    const long long E = ops.n / (NS * ops.nb);
    const int nb = ops.nb;
    const long long n = ops.n;
    const std::string tag = std::string(who) + ": block preconditioner";
    bool same = pc.valid && pc.E == E && pc.nb == nb;
    for (int s = 0; s < NS && same; ++s) same = pc.key[s] == ops.A[s];
    if (!same) {
        pc.release();
        std::vector<int> color;
        pc.ncolor = colour_elements(E, ops.NF, ops.face, color);
        pc.E = E;
        pc.nb = nb;
        const size_t blk_bytes = sizeof(double) * (size_t)E * NS * nb * nb;
        cudaError_t e = cudaMalloc(&pc.K, blk_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&pc.Binv, blk_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&pc.color, sizeof(int) * (size_t)E);
        if (e == cudaSuccess) e = cudaMalloc(&pc.bad, sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pc.color, color.data(), sizeof(int) * (size_t)E, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            pc.release();
            return cuda_fail(e, tag.c_str());
        }
        for (int c = 0; c < pc.ncolor; ++c)
            for (int i = 0; i < nb; ++i) {
                k_probe<<<grid_of(n), 256, 0, st>>>(n, nb, pc.color, c, i, probe);
                if (int rc = ops.jvp_diffusion(ops.ctx, probe, resp, st)) {
                    pc.release();
                    return rc;
                }
                k_probe_take<<<grid_of(n), 256, 0, st>>>(n, nb, pc.color, c, i, resp, pc.K);
            }
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            pc.release();
            return cuda_fail(e, tag.c_str());
        }
        for (int s = 0; s < NS; ++s) pc.key[s] = ops.A[s];
        pc.valid = true;
        pc.gdt = -1.0;
    }
    if (pc.gdt != gdt) {
        const long long nblk = E * NS;
        int flag = 0;
        cudaError_t e = cudaMemsetAsync(pc.bad, 0, sizeof(int), st);
        if (e == cudaSuccess && nblk > 0) {
            k_block_invert<<<grid_of(nblk), 256, 0, st>>>(nblk, nb, pc.K, gdt, pc.Binv, pc.bad);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, pc.bad, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, tag.c_str());
        if (flag) {
            set_error(tag + ": a block of I - dt a_ii K is not positive definite");
            pc.gdt = -1.0;
            return CDG2_ERR_NONFINITE;
        }
        pc.gdt = gdt;
    }
    return CDG2_OK;
}

}  // namespace cdg2
