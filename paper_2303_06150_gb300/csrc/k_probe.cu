// Gather-ceiling probe: loads from uniformly random 32-byte records of a
// buffer (4, 8, 16 or all 32 bytes of each), with no pose arithmetic. It
// measures the achievable rate of the docking kernel's access pattern (one
// aligned load of one record per atom sample) on this device,
// which is the denominator of the docking kernel's roofline. The paper has
// no counterpart; this is a measurement utility.
#include "../../include/ligen.h"
#include "internal.h"

namespace ligen {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeStreams = 8;   // independent loads in flight per thread

// Each width loads the way the docking kernel's sampler of that record size
// does: 32 bytes without L1 allocation (FP32 records), 16 bytes through the
// read-only path (FP16 / BF16 records).
template <int BYTES>
__device__ __forceinline__ float probe_load(const float* p) {
  if constexpr (BYTES == 32) {
    float v[8];
    ld_global_v8_na(p, v);
    return (v[0] + v[1]) + (v[2] + v[3]) + (v[4] + v[5]) + (v[6] + v[7]);
  } else if constexpr (BYTES == 16) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return (v.x + v.y) + (v.z + v.w);
  } else if constexpr (BYTES == 8) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return v.x + v.y;
  } else {
    return __ldg(p);
  }
}

// Each load reads BYTES bytes at the start of a uniformly random 32-byte record.
template <int BYTES>
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
      acc += probe_load<BYTES>(rec + (size_t)idx * 8);
    }
  }
  if (acc == 1.2345e-30f) sink[0] = acc;   // keeps the loads alive
}

// Streaming read: thread t of the grid reads 16-byte words t, t + T, ...
// (T threads in all) once per pass, through L2 only (ld.global.cg).
__global__ void __launch_bounds__(kProbeThreads) stream_kernel(const float4* __restrict__ buf, uint64_t n_vec,
                                                               int passes, float* sink) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  float acc = 0.f;
  for (int p = 0; p < passes; ++p) {
    uint64_t i = tid;
    for (; i + 3 * stride < n_vec; i += 4 * stride) {   // four independent loads in flight
      const float4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
      const float4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
      acc += ((a.x + b.y) + (c.z + d.w));
    }
    for (; i < n_vec; i += stride) acc += __ldcg(buf + i).x;
  }
  if (acc == 1.2345e-30f) sink[0] = acc;   // keeps the loads alive
}

}  // namespace

cudaError_t launch_stream_probe(const void* buf, uint64_t n_vec, int passes, float* sink, int blocks,
                                cudaStream_t s) {
  stream_kernel<<<blocks, kProbeThreads, 0, s>>>(reinterpret_cast<const float4*>(buf), n_vec, passes, sink);
  return cudaGetLastError();
}

int probe_streams() { return kProbeStreams; }

cudaError_t launch_probe(const float* rec, uint32_t n_rec, int bytes, int iters, uint64_t seed, float* sink,
                         int blocks, cudaStream_t s) {
  switch (bytes) {
    case 32: probe_kernel<32><<<blocks, kProbeThreads, 0, s>>>(rec, n_rec, iters, seed, sink); break;
    case 16: probe_kernel<16><<<blocks, kProbeThreads, 0, s>>>(rec, n_rec, iters, seed, sink); break;
    case 8: probe_kernel<8><<<blocks, kProbeThreads, 0, s>>>(rec, n_rec, iters, seed, sink); break;
    default: probe_kernel<4><<<blocks, kProbeThreads, 0, s>>>(rec, n_rec, iters, seed, sink); break;
  }
  return cudaGetLastError();
}

int probe_threads() { return kProbeThreads; }

}  // namespace ligen
