// ctx_access.hpp -- read-only view of a context for library-internal entry
// points that live outside api.cu.
#pragma once
#include <cstdint>
#include "common.cuh"

struct wally_ctx;

namespace wally {
// Parameter block (host copy, with the device copy in dp.self), device
// ordinal, ring degree and limb count of a context; false for NULL.
bool ctx_view(const wally_ctx *c, const DevParams **dp, int *device, uint32_t *n, uint32_t *L);
// Records a failure message for wally_last_error() and returns code.
int ctx_fail(int code, const char *msg);
}  // namespace wally
