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

// A caller's device allocator (rhpdhg_params.dev_alloc, dev_free, alloc_ctx) and the stream its
// buffers are used on.  While an AllocScope is alive on a thread, buf_alloc on that thread takes
// buffers from it; buf_release (on any thread) hands such a buffer back to the allocator's own
// free function and never caches it.
struct DevAllocator {
  void *(*alloc)(size_t bytes, void *stream, void *ctx) = nullptr;
  void (*free)(void *ptr, void *stream, void *ctx) = nullptr;
  void *ctx = nullptr;
  void *stream = nullptr;
};

class AllocScope {
 public:
  explicit AllocScope(const DevAllocator &a);
  ~AllocScope();
  AllocScope(const AllocScope &) = delete;
  AllocScope &operator=(const AllocScope &) = delete;

 private:
  const DevAllocator *prev_;
  DevAllocator mine_;
};

}  // namespace rh
