// k_binned_modes.cu - the batch and routed variants of the binned scatter
// (k_binned.cuh), compiled apart from the single-sketch ones so the two build
// in parallel.
#include "k_binned.cuh"

namespace hs {
namespace binned {

cudaError_t launch_modes_batch_route(int mode, const float *xyz, const SketchDesc &d,
                                     const ScatterArgs &a, bool sampled, size_t smem, uint32_t *C,
                                     cudaStream_t s) {
    switch (mode) {
    case kModeBatch: return launch_mode<kModeBatch>(xyz, d, a, sampled, smem, C, s);
    case kModeRoute: return launch_mode<kModeRoute>(xyz, d, a, sampled, smem, C, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace binned
}  // namespace hs
