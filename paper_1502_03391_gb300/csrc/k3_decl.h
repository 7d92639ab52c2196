// Declarations of the per-dimension K3 instantiations (defined in k3_d*.cu).
#pragma once
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include "fjofc_internal.h"

namespace fjofc {
template <int D, typename TD> cudaError_t k3_launch_impl(int grid, const CUtensorMap& tmap, const K3Params& p, cudaStream_t s);
template <int D, typename TD> int k3_bps_impl();
template <int D, typename TD> K3Geom k3_geom_impl();
}  // namespace fjofc
