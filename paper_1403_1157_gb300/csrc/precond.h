// Element-block-Jacobi preconditioner of the stage systems (precond.cu).
#pragma once

#include <cuda_runtime.h>

#include "cdg2_internal.h"

namespace cdg2 {

// Inverse diagonal blocks on the device.  An element's type is its boundary
// situation along each axis (tau_j, see precond.cu); the table holds, for
// every type t present in the mesh and species s, (P_ts^{-1})^T as
// M[t][s][j][i] = (P_ts^{-1})_{ij}, in FP64 and in FP32.
struct BlockTable {
    int n_types = 0;
    int stride[3] = {0, 0, 0};   // type = sum_j slot[j][tau_j] * stride[j]
    int slot[3][5] = {};
    const double* m64 = nullptr;
    const float* m32 = nullptr;
};

// Device bytes of a block table for the mesh (both precisions).
size_t block_table_bytes(const cdg2_mesh& m);

// Build P_ts = I - gdt A_s K_t on the host, invert, and copy both precisions
// to dev (block_table_bytes(m) bytes); synchronous.
int build_block_table(const cdg2_mesh& m, const Coef& c, double gdt, void* dev, BlockTable& bt);

// z = P^{-1} v over the whole mesh (v and z must not alias).
template <typename T>
cudaError_t block_apply(const cdg2_mesh& m, const BlockTable& bt, const T* v, T* z, cudaStream_t st);

}  // namespace cdg2
