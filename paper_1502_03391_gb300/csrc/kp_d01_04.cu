// Persistent in-sample kernel instantiations for embedding dimensions 1..4.
#include "k_embed_persistent.cuh"
namespace fjofc {
FJOFC_INSTANTIATE_PERSIST(1)
FJOFC_INSTANTIATE_PERSIST(2)
FJOFC_INSTANTIATE_PERSIST(3)
FJOFC_INSTANTIATE_PERSIST(4)
}  // namespace fjofc

#ifdef FJOFC_STAMPS
// Instrumented builds: copy the stamps of the last persistent launch (d <= 4) to host.
extern "C" int fjofc_debug_stamps(long long* host, long long count) {
    const long long cap = fjofc::kStampPasses * fjofc::kStampCtas * fjofc::kStampPoints;
    if (count > cap) count = cap;
    return cudaMemcpyFromSymbol(host, fjofc::g_stamps, size_t(count) * sizeof(long long)) == cudaSuccess ? 0 : -1;
}
// Wait cycles of warp 0 per CTA in the ring's waits (rfull, full, xfull, rempty) and the
// number of all-pairs passes, summed over the process (d <= 4 persistent kernels).
extern "C" int fjofc_debug_waits(unsigned long long* host) {
    return cudaMemcpyFromSymbol(host, fjofc::g_waitcyc, sizeof(fjofc::g_waitcyc)) == cudaSuccess ? 0 : -1;
}
#endif
#ifdef FJOFC_SECTIONS
// Cycles thread 0 of every CTA spent per section of the column-strip loop (d <= 4
// persistent kernels), summed over the process: [1024][8].
extern "C" int fjofc_debug_sections(unsigned long long* host) {
    return cudaMemcpyFromSymbol(host, fjofc::g_seccyc, sizeof(fjofc::g_seccyc)) == cudaSuccess ? 0 : -1;
}
#endif
