// Library context: device scratch owned by the library (never outputs).
#pragma once

#include "common.cuh"

struct orand_ctx_s {
    int device = -1;
    void *scratch = nullptr;     // grown on demand, never shrunk
    size_t scratch_bytes = 0;
    void *ragged = nullptr;      // ragged batcher state (ragged.cu)
};

namespace orand_impl {

// Check ctx belongs to the current device and return at least `bytes` of
// device scratch (256-byte aligned).  Growing frees the old buffer after a
// device synchronisation, so earlier asynchronous users are finished.
orand_status_t ctx_scratch(orand_ctx_t ctx, size_t bytes, void **ptr);

// Device check only (no scratch needed).
orand_status_t ctx_check(orand_ctx_t ctx);

}  // namespace orand_impl
