// Persistent in-sample kernel instantiations for embedding dimensions 11..16.
#include "k_embed_persistent.cuh"
namespace fjofc {
FJOFC_INSTANTIATE_PERSIST(11)
FJOFC_INSTANTIATE_PERSIST(12)
FJOFC_INSTANTIATE_PERSIST(13)
FJOFC_INSTANTIATE_PERSIST(14)
FJOFC_INSTANTIATE_PERSIST(15)
FJOFC_INSTANTIATE_PERSIST(16)
}  // namespace fjofc
