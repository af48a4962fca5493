// Hooks of the context (api.cu) used by the serving loop (serve.cpp); not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rkm.h"

namespace rkm {

// Score Q (device, q x d, stride ldq) against the resident users of `owner`, using the
// workspace, status word and stream of `work` (which may be `owner`).  Synchronises `s`.
rkm_status query_resident(rkm_ctx* work, const rkm_ctx* owner, const float* Q, int64_t q, int64_t ldq,
                          int32_t* counts, cudaStream_t s);

// A context with the options and device of `parent` and workspace of its own (nullptr when
// its status word cannot be allocated); freed with rkm_destroy.
rkm_ctx* worker_context(const rkm_ctx* parent);

// Shape of the resident set: false when there is none.
bool resident_shape(const rkm_ctx* c, int64_t* n, int* d, int* device);

// Servers attached to a context: rkm_resident_set refuses to run while the count is not zero.
void attach_server(rkm_ctx* c, int delta);

// Kernels launched by the library since it was loaded (all contexts and threads).
unsigned long long launch_count();

// Record `msg` as this host thread's last error and return `s`.
rkm_status fail_with(rkm_status s, const char* msg);

}  // namespace rkm
