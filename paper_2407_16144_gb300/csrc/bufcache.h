// Device buffers of handles: allocated from, and returned to, a process-wide cache of freed
// buffers (reuse of an exact size on the same device; at most kBufferCacheBytes held; the cache
// is dropped and the allocation retried when the device runs out of memory).  A buffer may be released only when
// no work on it is pending (the stream that used it has been synchronised).  Creating and
// freeing handles of the same sizes (a benchmark loop, a serving stream) then costs no device
// allocation and no device-wide synchronisation after the first time.
#pragma once

#include <cstddef>

#include <cuda_runtime.h>

namespace rh {

constexpr size_t kBufferCacheBytes = size_t(4) << 30;
cudaError_t buf_alloc(void **p, size_t bytes);
void buf_release(void *p);
// Frees every cached buffer; returns the bytes freed.
size_t buf_drop_cache();

}  // namespace rh
