// probe.cu -- a read-only streaming kernel: the ceiling a pass that reads each
// byte once and writes almost nothing can reach on this device (the per-bin
// argmin/argmax pass reads y once, Section 2.1, and is compared with it
// beside the copy bandwidth).
#include <stdint.h>

#include "internal.h"

namespace tsds {

constexpr int kReadThreads = 512;
constexpr int kReadCtasPerSm = 2;
constexpr int kReadUnroll = 8;

__device__ __forceinline__ uint64_t fold16(uint4 v) {
  const uint64_t lo = ((uint64_t)v.y << 32) | v.x;
  const uint64_t hi = ((uint64_t)v.w << 32) | v.z;
  return lo ^ hi;
}

// Grid-stride over 16-byte vectors, kReadUnroll independent loads in flight
// per thread; every word enters the XOR so that no load can be dropped.
__global__ void __launch_bounds__(kReadThreads, kReadCtasPerSm)
    k_read_stream(const uint4* __restrict__ v, int64_t nvec, unsigned long long* sink) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t acc = 0;
  for (; i + (kReadUnroll - 1) * stride < nvec; i += kReadUnroll * stride) {
    uint4 r[kReadUnroll];
#pragma unroll
    for (int u = 0; u < kReadUnroll; ++u) r[u] = __ldg(v + i + u * stride);
#pragma unroll
    for (int u = 0; u < kReadUnroll; ++u) acc ^= fold16(r[u]);
  }
  for (; i < nvec; i += stride) acc ^= fold16(__ldg(v + i));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0) atomicXor(sink, (unsigned long long)acc);
}

cudaError_t launch_read_stream(const void* buf, int64_t bytes, uint64_t* sink, cudaStream_t st) {
  const int64_t nvec = bytes / 16;
  if (nvec == 0) return cudaSuccess;
  const int64_t need = (nvec + kReadThreads - 1) / kReadThreads;
  const int64_t full = (int64_t)device_sm_count() * kReadCtasPerSm;
  const int grid = (int)(need < full ? need : full);
  note_launch();
  k_read_stream<<<grid, kReadThreads, 0, st>>>(static_cast<const uint4*>(buf), nvec,
                                                reinterpret_cast<unsigned long long*>(sink));
  return cudaGetLastError();
}

}  // namespace tsds
