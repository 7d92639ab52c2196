// Persistent in-sample kernel instantiations for embedding dimensions 1..4.
#include "k_embed_persistent.cuh"
namespace fjofc {
FJOFC_INSTANTIATE_PERSIST(1)
FJOFC_INSTANTIATE_PERSIST(2)
FJOFC_INSTANTIATE_PERSIST(3)
FJOFC_INSTANTIATE_PERSIST(4)
}  // namespace fjofc
