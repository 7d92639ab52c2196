// K1 instantiations for embedding dimensions 1..4.
#include "k_guttman_pass.cuh"
namespace fjofc {
FJOFC_INSTANTIATE_K1(1)
FJOFC_INSTANTIATE_K1(2)
FJOFC_INSTANTIATE_K1(3)
FJOFC_INSTANTIATE_K1(4)
}  // namespace fjofc
