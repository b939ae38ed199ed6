// Gather-ceiling probe: random 32-byte record loads from a buffer, with no
// pose arithmetic. It measures the achievable rate of the docking kernel's
// access pattern (one aligned 256-bit load per atom sample) on this device,
// which is the denominator of the docking kernel's roofline. The paper has
// no counterpart; this is a measurement utility.
#include "../../include/ligen.h"
#include "internal.h"

namespace ligen {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeStreams = 8;   // independent loads in flight per thread

__global__ void __launch_bounds__(kProbeThreads) probe_kernel(const float* __restrict__ rec, uint32_t n_rec,
                                                              int iters, uint64_t seed, float* sink) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[kProbeStreams];
#pragma unroll
  for (int s = 0; s < kProbeStreams; ++s) x[s] = (uint32_t)splitmix64(seed ^ (tid * kProbeStreams + s)) | 1u;
  float acc = 0.f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int s = 0; s < kProbeStreams; ++s) {
      x[s] ^= x[s] << 13; x[s] ^= x[s] >> 17; x[s] ^= x[s] << 5;   // xorshift32
      const uint32_t idx = __umulhi(x[s], n_rec);
      float v[8];
      ld_global_v8(rec + (size_t)idx * 8, v);
      acc += (v[0] + v[1]) + (v[2] + v[3]) + (v[4] + v[5]) + (v[6] + v[7]);
    }
  }
  if (acc == 1.2345e-30f) sink[0] = acc;   // keeps the loads alive
}

}  // namespace

int probe_streams() { return kProbeStreams; }

cudaError_t launch_probe(const float* rec, uint32_t n_rec, int iters, uint64_t seed, float* sink, int blocks,
                         cudaStream_t s) {
  probe_kernel<<<blocks, kProbeThreads, 0, s>>>(rec, n_rec, iters, seed, sink);
  return cudaGetLastError();
}

int probe_threads() { return kProbeThreads; }

}  // namespace ligen
