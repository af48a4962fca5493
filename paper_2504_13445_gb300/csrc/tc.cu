// Tensor-core (tcgen05) product kernels of the threshold and counting passes.
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "tmap.h"

namespace rkm {

bool rkm_tc_available() { return false; }

rkm_status make_tmaps(const void*, int64_t, const void*, int64_t, int, int, TmapPair*) {
    return RKM_EINVAL;
}

void launch_threshold_tc(const ThresholdArgs&, const void*, const void*, cudaStream_t) {}
void launch_count_tc(const CountArgs&, const void*, const void*, cudaStream_t) {}

}  // namespace rkm
