// Persistent in-sample kernel instantiations for embedding dimensions 5..10.
#include "k_embed_persistent.cuh"
namespace fjofc {
FJOFC_INSTANTIATE_PERSIST(5)
FJOFC_INSTANTIATE_PERSIST(6)
FJOFC_INSTANTIATE_PERSIST(7)
FJOFC_INSTANTIATE_PERSIST(8)
FJOFC_INSTANTIATE_PERSIST(9)
FJOFC_INSTANTIATE_PERSIST(10)
}  // namespace fjofc
