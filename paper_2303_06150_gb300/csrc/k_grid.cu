// Grid preparation: node values [z][y][x][c] -> per-(cell, channel) records
// of the 8 coefficients of the cell's trilinear polynomial (or its 8 corner
// values in 16 bits), at rec_index (channel-major, see GridView). One thread
// per (cell, channel); consecutive threads read consecutive channels of the
// same corners (coalesced reads).
#include "internal.h"

namespace ligen {
namespace {

__global__ void grid_prep_kernel(const float* __restrict__ v, int nx, int ny, int nz, int nc,
                                 float* __restrict__ coef) {
  const int cx = nx - 1, cy = ny - 1, cz = nz - 1;
  const size_t total = (size_t)cx * cy * cz * nc;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % nc);
    size_t cell = t / nc;
    const int ix = (int)(cell % cx);
    cell /= cx;
    const int iy = (int)(cell % cy);
    const int iz = (int)(cell / cy);
    auto at = [&](int dx, int dy, int dz) -> float {
      return v[(((size_t)(iz + dz) * ny + (iy + dy)) * nx + (ix + dx)) * nc + c];
    };
    const float c000 = at(0, 0, 0), c100 = at(1, 0, 0), c010 = at(0, 1, 0), c110 = at(1, 1, 0);
    const float c001 = at(0, 0, 1), c101 = at(1, 0, 1), c011 = at(0, 1, 1), c111 = at(1, 1, 1);
    // FP32 differences of differences: each coefficient takes at most three
    // roundings at the grid values' magnitude. (The same sums in FP64 ran on
    // the chip's narrow FP64 pipe: 0.37 ms for a 96^3 x 8 grid against
    // 0.07 ms, measured on GB300.)
    const float dx00 = c100 - c000, dx10 = c110 - c010, dx01 = c101 - c001, dx11 = c111 - c011;
    const float axy = dx10 - dx00, axz = dx01 - dx00;
    float4 lo, hi;
    lo.x = c000;                       // a0
    lo.y = dx00;                       // ax
    lo.z = c010 - c000;                // ay
    lo.w = c001 - c000;                // az
    hi.x = axy;                        // axy
    hi.y = axz;                        // axz
    hi.z = (c011 - c001) - lo.z;       // ayz
    hi.w = (dx11 - dx01) - axy;        // axyz
    float4* rec = reinterpret_cast<float4*>(coef + rec_index(cx, cy, cz, c, ix, iy, iz) * 8);
    rec[0] = lo;
    rec[1] = hi;
  }
}

// 16-bit records: the 8 corner values of each (cell, channel), order
// c000, c100, c010, c110, c001, c101, c011, c111, rounded to nearest. The
// record grid has rec_cells(n) cells per axis: corners past the last node
// repeat it (the padding layers of the clamp-free sampler).
template <int FMT>
__global__ void grid_prep16_kernel(const float* __restrict__ v, int nx, int ny, int nz, int nc,
                                   uint4* __restrict__ out) {
  const int cx = rec_cells(nx, FMT), cy = rec_cells(ny, FMT), cz = rec_cells(nz, FMT);
  const size_t cells = (size_t)cx * cy * cz;
  const size_t total = cells * nc;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % nc);
    size_t cell = t / nc;
    const int ix = (int)(cell % cx);
    const int iy = (int)((cell / cx) % cy);
    const int iz = (int)(cell / ((size_t)cx * cy));
    auto at = [&](int dx, int dy, int dz) -> float {
      const int x = min(ix + dx, nx - 1), y = min(iy + dy, ny - 1), z = min(iz + dz, nz - 1);
      return v[(((size_t)z * ny + y) * nx + x) * nc + c];
    };
    unsigned int w[4];
    const float pairs[4][2] = {{at(0, 0, 0), at(1, 0, 0)}, {at(0, 1, 0), at(1, 1, 0)},
                               {at(0, 0, 1), at(1, 0, 1)}, {at(0, 1, 1), at(1, 1, 1)}};
    for (int k = 0; k < 4; ++k) {
      if constexpr (FMT == kRecF16) {
        __half2 h = __floats2half2_rn(pairs[k][0], pairs[k][1]);
        w[k] = *reinterpret_cast<unsigned int*>(&h);
      } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(pairs[k][0], pairs[k][1]);
        w[k] = *reinterpret_cast<unsigned int*>(&h);
      }
    }
    out[rec_index(cx, cy, cz, c, ix, iy, iz)] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

}  // namespace

cudaError_t launch_grid_prep_fmt(const float* values, int nx, int ny, int nz, int nc, int fmt, void* rec,
                                 cudaStream_t s) {
  if (fmt == kRecF32) return launch_grid_prep(values, nx, ny, nz, nc, (float*)rec, s);
  const size_t total = rec_count(rec_cells(nx, fmt), rec_cells(ny, fmt), rec_cells(nz, fmt), nc);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (total + 255) / 256;
  const int blocks = (int)(want < (size_t)sms * 16 ? want : (size_t)sms * 16);
  if (fmt == kRecF16)
    grid_prep16_kernel<kRecF16><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(values, nx, ny, nz, nc, (uint4*)rec);
  else
    grid_prep16_kernel<kRecBF16><<<blocks > 0 ? blocks : 1, 256, 0, s>>>(values, nx, ny, nz, nc, (uint4*)rec);
  return cudaGetLastError();
}

cudaError_t launch_grid_prep(const float* values, int nx, int ny, int nz, int nc, float* coef,
                             cudaStream_t s) {
  const size_t total = (size_t)(nx - 1) * (ny - 1) * (nz - 1) * nc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (total + 255) / 256;
  const int blocks = (int)(want < (size_t)sms * 16 ? want : (size_t)sms * 16);
  grid_prep_kernel<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(values, nx, ny, nz, nc, coef);
  return cudaGetLastError();
}

}  // namespace ligen
