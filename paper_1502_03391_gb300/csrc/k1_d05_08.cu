// K1 instantiations for embedding dimensions 5..8.
#include "k_guttman_pass.cuh"
namespace fjofc {
FJOFC_INSTANTIATE_K1(5)
FJOFC_INSTANTIATE_K1(6)
FJOFC_INSTANTIATE_K1(7)
FJOFC_INSTANTIATE_K1(8)
}  // namespace fjofc
