// Functions shared between the library's translation units that are not part
// of the C ABI (hidden: the library exports only what include/dc.h declares).
#pragma once

#include <stddef.h>

#include "../../include/dc.h"

// Scratch bytes one correct_batch call with these items needs on context c.
size_t dc_internal_batch_scratch(dc_ctx* c, const dc_item* items, int n_items);

// correct_batch run with caller-provided device scratch `ws` of ws_bytes
// (at least dc_internal_batch_scratch): the context allocates nothing.
dc_status dc_internal_correct_batch_ws(dc_ctx* c, const dc_c64* in, dc_c64* out,
                                       const dc_item* items, int n_items, const dc_opts* opts,
                                       void* stream, void* ws, size_t ws_bytes);
