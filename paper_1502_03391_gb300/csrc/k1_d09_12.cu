// K1 instantiations for embedding dimensions 9..12.
#include "k_guttman_pass.cuh"
namespace fjofc {
FJOFC_INSTANTIATE_K1(9)
FJOFC_INSTANTIATE_K1(10)
FJOFC_INSTANTIATE_K1(11)
FJOFC_INSTANTIATE_K1(12)
}  // namespace fjofc
