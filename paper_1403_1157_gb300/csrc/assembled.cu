// The assembled Jacobian of f(U) = M^{-1} L_h(U) on a Cartesian mesh (Sec.
// 3.2 contrasts the matrix-free Jacobian-vector products with a "fully
// assembled approach" and leaves the latter aside; this builds it so that
// the two can be compared).
//
// Storage: element-block sparse.  Row block e holds the blocks of e itself
// (slot 0) and of its face neighbours (slot 1 + 2 a + f: axis a, low f = 0 /
// high f = 1), each b x b with b = 6 n_basis, column-major (column c of a
// block is contiguous), so a sparse matrix-vector product reads every block
// coalesced.  Assembly: the JVP of probe vectors that set one (species,
// mode) of every element of one colour of a distance-2 colouring (no two
// elements within two face steps share a colour): for each row element at
// most one element of the colour lies in its closed neighbourhood, so the
// JVP's rows of e are exactly that column of block (e, e').
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "cdg2_internal.h"

struct cdg2_matrix {
    const cdg2_mesh* mesh = nullptr;
    int b = 0;              // block size 6 n_basis
    int slots = 0;          // 1 + 2 dim
    long long E = 0;
    double* blocks = nullptr;   // device [E][slots][b (column)][b (row)]
    int* nbr = nullptr;         // device [E][slots]: column element of each slot, -1 if absent
    int* colour = nullptr;      // device [E]
    int ncolour = 0;
    double* probe = nullptr;    // device ndof: probe vector and JVP result
    double* resp = nullptr;
};

namespace cdg2 {

// Neighbour of element e across face f (0 low, 1 high) of axis a; -1 on a
// wall (host twin of the kernels' lookup).
static long long host_neighbour(const Geo& g, long long e, int a, int f) {
    long long c[3] = {e % g.n[0], (e / g.n[0]) % g.n[1], e / ((long long)g.n[0] * g.n[1])};
    long long v = c[a] + (f ? 1 : -1);
    if (v < 0 || v >= g.n[a]) {
        if (!g.periodic[a]) return -1;
        v = (v + g.n[a]) % g.n[a];
    }
    c[a] = v;
    return c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
}

// probe[e][r] = 1 where colour[e] == col and r == j, else 0
static __global__ void k_jac_probe(long long E, int b, const int* __restrict__ colour, int col, int j, double* __restrict__ v) {
    const long long n = E * b;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long e = i / b;
        const int r = (int)(i - e * b);
        v[i] = (colour[e] == col && r == j) ? 1.0 : 0.0;
    }
}

// column j of every block (e, s) whose column element has colour col := rows of e of the response
static __global__ void k_jac_scatter(long long E, int b, int slots, const int* __restrict__ nbr, const int* __restrict__ colour,
                          int col, int j, const double* __restrict__ y, double* __restrict__ blocks) {
    const long long e = blockIdx.x;
    for (int s = 0; s < slots; ++s) {
        const int ep = nbr[e * slots + s];
        if (ep < 0 || colour[ep] != col) continue;
        double* dst = blocks + ((e * slots + s) * (long long)b + j) * b;
        for (int r = threadIdx.x; r < b; r += blockDim.x) dst[r] = y[e * b + r];
    }
}

// y = alpha A x + beta y: one block per row element, one thread per row
static __global__ void k_spmv(long long E, int b, int slots, const int* __restrict__ nbr, const double* __restrict__ blocks,
                       double alpha, const double* __restrict__ x, double beta, double* __restrict__ y) {
    extern __shared__ double xs[];   // [slots][b]
    const long long e = blockIdx.x;
    for (int i = threadIdx.x; i < slots * b; i += blockDim.x) {
        const int s = i / b, c = i - s * b;
        const int ep = nbr[e * slots + s];
        xs[i] = ep >= 0 ? x[(long long)ep * b + c] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < b; r += blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < slots; ++s) {
            if (nbr[e * slots + s] < 0) continue;
            const double* blk = blocks + (e * slots + s) * (long long)b * b + r;
            const double* xv = xs + s * b;
            for (int c = 0; c < b; ++c) acc = fma(blk[(long long)c * b], xv[c], acc);
        }
        const long long i = e * b + r;
        y[i] = alpha * acc + (beta == 0.0 ? 0.0 : beta * y[i]);
    }
}

static unsigned grid_1d(long long n) {
    long long g = (n + 255) / 256;
    return (unsigned)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
}

int assemble(cdg2_matrix& A, const Coef& c, const double* U, cudaStream_t st, const char* who) {
    const cdg2_mesh& m = *A.mesh;
    for (int col = 0; col < A.ncolour; ++col) {
        for (int j = 0; j < A.b; ++j) {
            k_jac_probe<<<grid_1d(m.ndof), 256, 0, st>>>(A.E, A.b, A.colour, col, j, A.probe);
            cudaError_t e = launch_jvp(m, c, U, A.probe, nullptr, A.resp, CDG2_MINV | CDG2_ASYNC, st);
            if (e != cudaSuccess) return cuda_fail(e, who);
            k_jac_scatter<<<(unsigned)A.E, 128, 0, st>>>(A.E, A.b, A.slots, A.nbr, A.colour, col, j, A.resp, A.blocks);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, who);
    return CDG2_OK;
}

cudaError_t spmv(const cdg2_matrix& A, double alpha, const double* x, double beta, double* y, cudaStream_t st) {
    const int nt = A.b < 128 ? ((A.b + 31) / 32) * 32 : 128;
    const size_t smem = sizeof(double) * (size_t)A.slots * A.b;
    k_spmv<<<(unsigned)A.E, nt, smem, st>>>(A.E, A.b, A.slots, A.nbr, A.blocks, alpha, x, beta, y);
    return cudaGetLastError();
}

// Host part of the set-up: the neighbour table and a greedy distance-2
// colouring in element order.
static void build_structure(const Geo& g, int slots, std::vector<int>& nbr, std::vector<int>& colour, int& ncolour) {
    const long long E = g.E;
    nbr.assign((size_t)E * slots, -1);
    for (long long e = 0; e < E; ++e) {
        nbr[(size_t)e * slots] = (int)e;
        for (int a = 0; a < g.dim; ++a)
            for (int f = 0; f < 2; ++f) nbr[(size_t)e * slots + 1 + 2 * a + f] = (int)host_neighbour(g, e, a, f);
    }
    colour.assign((size_t)E, -1);
    ncolour = 0;
    std::vector<char> used(64);
    for (long long e = 0; e < E; ++e) {
        std::fill(used.begin(), used.end(), 0);
        for (int s = 0; s < slots; ++s) {
            const int n1 = nbr[(size_t)e * slots + s];
            if (n1 < 0) continue;
            for (int t = 0; t < slots; ++t) {
                const int n2 = nbr[(size_t)n1 * slots + t];
                if (n2 >= 0 && colour[(size_t)n2] >= 0 && colour[(size_t)n2] < (int)used.size()) used[colour[(size_t)n2]] = 1;
            }
        }
        int col = 0;
        while (used[col]) ++col;
        colour[(size_t)e] = col;
        if (col + 1 > ncolour) ncolour = col + 1;
    }
}

}  // namespace cdg2

using namespace cdg2;

extern "C" {

int cdg2_matrix_create(const cdg2_mesh* m, cdg2_matrix** out) {
    if (!m || !out) {
        set_error("cdg2_matrix_create: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const Geo& g = m->geo;
    for (int a = 0; a < g.dim; ++a)
        if (g.periodic[a] && g.n[a] < 3) {
            set_error("cdg2_matrix_create: a periodic axis needs at least 3 cells (its two neighbours must differ)");
            return CDG2_ERR_INVALID_ARG;
        }
    cdg2_matrix* A = new (std::nothrow) cdg2_matrix();
    if (!A) {
        set_error("cdg2_matrix_create: out of host memory");
        return CDG2_ERR_INVALID_ARG;
    }
    A->mesh = m;
    A->b = NS * m->nb;
    A->slots = 1 + 2 * g.dim;
    A->E = g.E;
    std::vector<int> nbr, colour;
    build_structure(g, A->slots, nbr, colour, A->ncolour);
    const size_t bytes = sizeof(double) * (size_t)A->E * A->slots * A->b * A->b;
    cudaError_t e = cudaMalloc(&A->blocks, bytes);
    if (e == cudaSuccess) e = cudaMemset(A->blocks, 0, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&A->nbr, sizeof(int) * nbr.size());
    if (e == cudaSuccess) e = cudaMemcpy(A->nbr, nbr.data(), sizeof(int) * nbr.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&A->colour, sizeof(int) * colour.size());
    if (e == cudaSuccess) e = cudaMemcpy(A->colour, colour.data(), sizeof(int) * colour.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&A->probe, sizeof(double) * m->ndof);
    if (e == cudaSuccess) e = cudaMalloc(&A->resp, sizeof(double) * m->ndof);
    if (e != cudaSuccess) {
        cdg2_matrix_destroy(A);
        return cuda_fail(e, "cdg2_matrix_create");
    }
    *out = A;
    return CDG2_OK;
}

void cdg2_matrix_destroy(cdg2_matrix* A) {
    if (!A) return;
    if (A->blocks) cudaFree(A->blocks);
    if (A->nbr) cudaFree(A->nbr);
    if (A->colour) cudaFree(A->colour);
    if (A->probe) cudaFree(A->probe);
    if (A->resp) cudaFree(A->resp);
    delete A;
}

int cdg2_matrix_info(const cdg2_matrix* A, int* block_size, int* slots, int* colours, long long* bytes) {
    if (!A) {
        set_error("cdg2_matrix_info: NULL matrix");
        return CDG2_ERR_INVALID_ARG;
    }
    if (block_size) *block_size = A->b;
    if (slots) *slots = A->slots;
    if (colours) *colours = A->ncolour;
    if (bytes) *bytes = (long long)sizeof(double) * A->E * A->slots * A->b * A->b;
    return CDG2_OK;
}

int cdg2_assemble_jacobian(cdg2_matrix* A, const cdg2_params* p, const double* U, void* stream) {
    if (!A || !p || !U) {
        set_error("cdg2_assemble_jacobian: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    const Coef c = make_coef(*p);
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = assemble(*A, c, U, st, "cdg2_assemble_jacobian")) return rc;
    return take_domain_status(A->mesh->status, st, "cdg2_assemble_jacobian");
}

int cdg2_spmv(const cdg2_matrix* A, double alpha, const double* x, double beta, double* y, void* stream) {
    if (!A || !x || !y) {
        set_error("cdg2_spmv: NULL argument");
        return CDG2_ERR_INVALID_ARG;
    }
    if (x == y) {
        set_error("cdg2_spmv: x and y must not overlap");
        return CDG2_ERR_INVALID_ARG;
    }
    cudaError_t e = spmv(*A, alpha, x, beta, y, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cdg2_spmv");
    return CDG2_OK;
}

}  // extern "C"
