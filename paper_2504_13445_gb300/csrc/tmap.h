// TMA descriptors of the packed tensor-core operands (host side).
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "../../include/rkm.h"

namespace rkm {

struct TmapPair {
    CUtensorMap a;  // users: rows x dp elements, box 128 rows x 128 bytes, 128-byte swizzle
    CUtensorMap b;  // items: rows x dp elements, box item_tile rows x 128 bytes
};

// True when the tensor-core kernels are compiled into this library.
bool rkm_tc_available();

// Encode the two tiled maps of BF16 (elem_bytes 2) or FP8 (elem_bytes 1) packs (returns
// RKM_ECUDA if the driver rejects them).  A box row is 128 bytes: 64 BF16 or 128 FP8 values.
rkm_status make_tmaps(const void* A, int64_t a_rows, const void* B, int64_t b_rows, int dp, int item_tile,
                      int elem_bytes, TmapPair* out);

}  // namespace rkm
