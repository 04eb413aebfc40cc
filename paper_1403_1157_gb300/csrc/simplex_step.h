// The implicit step on simplicial meshes: the SDIRK / Newton / GMRES driver of
// cdg2_step (Sec. 3.2) over an operator given by callbacks, FP64, with no
// preconditioner or element-block Jacobi.  Used by the triangle and
// tetrahedral entry points.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

#include "cdg2.h"

namespace cdg2 {

// Element-block Jacobi of a simplicial mesh (precond = 2): the diagonal blocks
// K_{e,s} of the diffusion part of M^{-1} L_h (probed column by column with the
// JVP under a distance-1 colouring of the elements, cached per diffusivities)
// and the inverses of I - dt a_ii K_{e,s}.  Owned by the mesh.
struct SimplexPrecond {
    double* K = nullptr;       // device [E][6][nb][nb], row-major blocks
    double* Binv = nullptr;    // device [E][6][nb][nb]
    int* color = nullptr;      // device [E]
    int* bad = nullptr;        // device flag: a non-positive pivot
    int ncolor = 0;
    long long E = 0;
    int nb = 0;
    double key[6] = {0, 0, 0, 0, 0, 0};   // the diffusivities K was probed with
    double gdt = -1.0;                    // the dt a_ii Binv was formed with
    bool valid = false;
    void release();
};

// A copy of p with every term but diffusion switched off (chemotaxis, sources
// and boundary influxes zero): its JVP is the diffusion part of the operator.
cdg2_params diffusion_only(const cdg2_params& p);

struct SimplexStepOps {
    long long n;                 // unknowns: n_elem * 6 * n_basis
    int nb;                      // basis functions per species
    void** ws;                   // the mesh's step workspace (grown on demand, freed with the mesh)
    size_t* ws_bytes;
    const void* ctx;             // passed to the callbacks
    // out = M^{-1} L_h(Y); a CDG2 status
    int (*apply)(const void* ctx, const double* Y, double* out, cudaStream_t st);
    // out = J(Y) v for that operator; a CDG2 status
    int (*jvp)(const void* ctx, const double* Y, const double* v, double* out, cudaStream_t st);
    // out = J_diff v, the diffusion part alone (linear; the state is v itself); a CDG2 status
    int (*jvp_diffusion)(const void* ctx, const double* v, double* out, cudaStream_t st);
    const double* A;             // the diffusivities A_s of the step's parameters
    const int* face;             // host [NF][4], the first two entries the elements of an interior face
    long long NF;
    SimplexPrecond* pc;          // the mesh's block-Jacobi state
    int* dom;                    // the mesh's domain status word (device), set by its kernels
};

// Build (or reuse) the blocks K of pc for ops, then form Binv for gdt.
int simplex_precond_setup(const SimplexStepOps& ops, double gdt, double* probe, double* resp, cudaStream_t st,
                          const char* who);
// out = Binv v, blockwise (v and out distinct, n = E 6 nb).
cudaError_t simplex_block_apply(const SimplexPrecond& pc, const double* v, double* out, cudaStream_t st);

// One SDIRK step of U' = M^{-1} L_h(U), U overwritten in place (device FP64).
// Options as cdg2_step, except that mixed and flags must be 0 and precond is
// 0 (none) or 2 (element-block Jacobi).
int simplex_step(const SimplexStepOps& ops, double* U, double dt, const cdg2_solver_opts* o, cdg2_stats* stats,
                 void* stream, const char* who);

}  // namespace cdg2
