// The staged pair of one grid bin for the float path: (sc e' + sh, sc Delta)
// with Delta = e1 - e0 and e' = e0 - (1 - 2^-24) Delta, computed in double and
// rounded once.  With unit(l) in [1, 2) holding the position bits, one float
// FMA z = fma(unit, width, coordinate) gives the integrand's staged coordinate
// z = sc (e0 + frac Delta) + sh, frac = (floor(l / 2^9) + 1/2) 2^-23.
//
// The iterate kernels stage a block's grid with it, or load pairs that the
// refinement and staging kernels wrote with it once per grid change (keeping
// the FP64 instructions out of every block of the float path).
#pragma once

#include <cuda_runtime.h>

namespace vegas {

__device__ __forceinline__ float2 stage_pair32(double e0, double e1, double sc, double sh) {
    const double w = e1 - e0;
    const double e = ::fma(-0x1.fffffep-1, w, e0);
    return make_float2((float)::fma(e, sc, sh), (float)(w * sc));
}

// One dimension's row of N staged pairs from its N + 1 edges, by the block's
// threads.
__device__ __forceinline__ void stage_row32(const double* edges, int N, double sc, double sh,
                                            float2* out) {
    for (int j = threadIdx.x; j < N; j += blockDim.x) out[j] = stage_pair32(edges[j], edges[j + 1], sc, sh);
}

}  // namespace vegas
