// gs_notify.cu -- completion notification of a stream through a file
// descriptor, for request loops that sleep instead of polling (serving).
#include <cuda_runtime.h>
#include <unistd.h>

#include <cstdint>

#include "gs.h"

namespace {

// Runs on a CUDA driver thread once the stream reaches it; calls no CUDA API.
void CUDART_CB write_one(void* arg) {
  const uint64_t one = 1;
  const int fd = static_cast<int>(reinterpret_cast<intptr_t>(arg));
  const ssize_t w = write(fd, &one, sizeof(one));
  (void)w;  // a full eventfd counter (2^64 - 2 pending wakeups) cannot occur here
}

}  // namespace

extern "C" int gs_stream_notify(void* stream, int fd) {
  if (fd < 0) return GS_EINVAL;
  if (cudaLaunchHostFunc(static_cast<cudaStream_t>(stream), write_one,
                         reinterpret_cast<void*>(static_cast<intptr_t>(fd))) != cudaSuccess) {
    cudaGetLastError();
    return GS_ECUDA;
  }
  return GS_OK;
}
