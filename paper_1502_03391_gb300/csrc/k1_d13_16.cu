// K1 instantiations for embedding dimensions 13..16.
#include "k_guttman_pass.cuh"
namespace fjofc {
FJOFC_INSTANTIATE_K1(13)
FJOFC_INSTANTIATE_K1(14)
FJOFC_INSTANTIATE_K1(15)
FJOFC_INSTANTIATE_K1(16)
}  // namespace fjofc
