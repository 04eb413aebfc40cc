// Device helpers shared by the simplicial element kernels (tri.cu, tet.cu).
#pragma once

namespace cdg2 {

// Species of slot sl when an element kernel orders its interpolation passes
// for the MODAL volume flux (volume_point<D, T, true>): the three species whose
// gradients that flux reads (n1, c1, c3) first, then n2, n3, c2 (values only).
__device__ __forceinline__ int modal_fwd_species(int sl) {
    return sl == 0 ? 0 : sl == 1 ? 3 : sl == 2 ? 5 : sl == 3 ? 1 : sl == 4 ? 2 : 4;
}

}  // namespace cdg2
