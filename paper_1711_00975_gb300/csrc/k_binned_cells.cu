// k_binned_cells.cu - the binned scatter (k_binned.cuh) over cell records of
// kept particles, the output of the compaction pass, for a sketch and for its
// super-item sketch; compiled apart so the variants build in parallel.
#include "k_binned.cuh"

namespace hs {
namespace binned {

cudaError_t launch_modes_cells(int mode, const float *xyz, const SketchDesc &d, const ScatterArgs &a,
                               size_t smem, uint32_t *C, cudaStream_t s) {
    switch (mode) {
    case kModeCells: return launch_mode<kModeCells, false>(xyz, d, a, false, smem, C, s);
    case kModeSuperCells: return launch_mode<kModeSuperCells, false>(xyz, d, a, false, smem, C, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace binned
}  // namespace hs
