// Declarations of the per-dimension K3 instantiations (defined in k3_d*.cu).
#pragma once
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include "fjofc_internal.h"

namespace fjofc {
template <int D, typename TD> cudaError_t k3_launch_impl(int grid, const CUtensorMap& tmap, const K3Params& p, cudaStream_t s);
template <int D, typename TD> int k3_bps_impl(int m);
template <int D, typename TD> K3Geom k3_geom_impl(int m);

// The resident out-of-sample form (k_oos_resident.cuh): one CTA per object, -X^T and the
// object's dissimilarities in shared memory ([m][d][nx] + [m][nx] float32).
constexpr int kK3rThreads = 256;
constexpr int kK3rWarps = kK3rThreads / 32;
constexpr int kK3rMaxD = 8;                       // instantiated for d = 1..8
// dynamic shared memory the resident form may use (its few static variables and the
// alignment stay inside the 227 KB per CTA)
constexpr size_t kK3rSmemBudget = size_t(200) * 1024;
// [m][d][nx] -x and [m][nx] delta, then the per-object state: y [m][d], per-warp sums
// [warps][m][d + 3], totals [m][d + 1] (floats), the fidelities [m] and the
// commensurability parts [m] (doubles)
__host__ __device__ inline size_t k3r_state_floats(int m, int d) {
    const size_t f = size_t(m) * d + size_t(kK3rWarps) * m * (d + 3) + size_t(m) * (d + 1);
    return (f + 1) & ~size_t(1);                  // the doubles after it stay 8-byte aligned
}
inline size_t k3r_smem_bytes(int m, int64_t nx, int d) {
    return size_t(m) * size_t(nx) * size_t(d + 1) * sizeof(float) + k3r_state_floats(m, d) * sizeof(float) +
           2 * size_t(m) * sizeof(double);
}
inline bool k3r_fits(int m, int64_t nx, int d) {
    return d >= 1 && d <= kK3rMaxD && k3r_smem_bytes(m, nx, d) <= kK3rSmemBudget;
}
template <int D, typename TD> cudaError_t k3r_launch_impl(int grid, const K3Params& p, cudaStream_t s);
template <int D, typename TD> int k3r_bps_impl(size_t smem);
}  // namespace fjofc
