// Declarations of the per-dimension K1 instantiations (defined in k1_d*.cu).
#pragma once
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include "fjofc_internal.h"

namespace fjofc {
template <int D, typename TD> cudaError_t k1_launch_impl(int grid, const TMaps& tm, const K1Params& p, cudaStream_t s);
template <int D, typename TD> int k1_bps_impl();
template <int D, typename TD> K1Geom k1_geom_impl();
}  // namespace fjofc

namespace fjofc {
template <int D, typename TD> cudaError_t persist_launch_impl(int grid, const TMaps& tm, const PersistParams& P, cudaStream_t s);
template <int D, typename TD> int persist_bps_impl();
template <int D, typename TD> cudaError_t batched_launch_impl(int grid, const BatchLaunch& bl, cudaStream_t s);
template <int D, typename TD> int batched_bps_impl();
}  // namespace fjofc
