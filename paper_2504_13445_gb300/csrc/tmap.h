// TMA descriptors of the packed BF16 operands (host side).
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "../../include/rkm.h"

namespace rkm {

struct TmapPair {
    CUtensorMap a;  // users: rows x dp bf16, box 128 rows x 64 elements, 128-byte swizzle
    CUtensorMap b;  // items: rows x dp bf16, box item_tile rows x 64 elements
};

// True when the tensor-core kernels are compiled into this library.
bool rkm_tc_available();

// Encode the two tiled maps (returns RKM_ECUDA if the driver rejects them).
rkm_status make_tmaps(const void* A, int64_t a_rows, const void* B, int64_t b_rows, int dp, int item_tile,
                      TmapPair* out);

}  // namespace rkm
