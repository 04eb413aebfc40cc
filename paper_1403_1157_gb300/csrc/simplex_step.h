// The implicit step on simplicial meshes: the SDIRK / Newton / GMRES driver of
// cdg2_step (Sec. 3.2) over an operator given by callbacks, FP64, without a
// preconditioner.  Used by the triangle and tetrahedral entry points.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

#include "cdg2.h"

namespace cdg2 {

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
};

// One SDIRK step of U' = M^{-1} L_h(U), U overwritten in place (device FP64).
// Options as cdg2_step, except that mixed, precond and flags must be 0.
int simplex_step(const SimplexStepOps& ops, double* U, double dt, const cdg2_solver_opts* o, cdg2_stats* stats,
                 void* stream, const char* who);

}  // namespace cdg2
