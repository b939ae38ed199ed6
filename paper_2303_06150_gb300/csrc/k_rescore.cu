// FP64 re-score of kept poses and re-ranking: FP64 arithmetic on the GPU is
// spent only on the K kept poses of each ligand, where near-ties between
// FP32 scores decide the ranking.
//
// Everything is recomputed in FP64 from the caller's FP32 inputs: the input
// centroid, the torsions (bond by bond, about the current axes), the
// rotation q/|q|, the translation, and the trilinear value from the eight
// FP32 node values of the caller's [z][y][x][c] grid. One warp per pose.
// Re-ranking: one warp per ligand orders its K poses by FP64 score
// (descending; ties by the restart that produced them) and rewrites poses,
// scores and restart ids in that order.
#include <cmath>

#include "../../include/ligen.h"
#include "internal.h"

namespace ligen {
namespace {

constexpr int kResWarps = 4;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ double trilinear64(const RescoreArgs& a, double x, double y, double z, int c) {
  const double u[3] = {(x - a.origin[0]) / a.h, (y - a.origin[1]) / a.h, (z - a.origin[2]) / a.h};
  const int n[3] = {a.nx, a.ny, a.nz};
  int i[3];
  double f[3];
  for (int k = 0; k < 3; ++k) {
    if (!(u[k] >= 0.0 && u[k] <= n[k] - 1)) return a.penalty;
    i[k] = min((int)floor(u[k]), n[k] - 2);
    f[k] = u[k] - i[k];
  }
  double e = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        const size_t node = (((size_t)(i[2] + dz) * a.ny + (i[1] + dy)) * a.nx + (i[0] + dx));
        if (!lg_check(a.check, c >= 0 && c < a.nc && node < (size_t)a.nx * a.ny * a.nz, kChkRescoreNode))
          continue;
        e += w * (double)a.values[node * a.nc + c];
      }
  return e;
}

__global__ void __launch_bounds__(32 * kResWarps) rescore_kernel(const RescoreArgs a) {
  __shared__ double ys[kResWarps][LIGEN_MAX_ATOMS * 3];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t gp = (size_t)blockIdx.x * kResWarps + w;
  if (gp >= (size_t)a.lig.L * a.K) return;
  const int l = (int)(gp / a.K), p = (int)(gp % a.K);
  if (a.status[l] != 0 ||
      !lg_check(a.check, a.lig.atom_off[l + 1] - a.lig.atom_off[l] <= LIGEN_MAX_ATOMS, kChkItemShape)) {
    if (lane == 0) a.s64[gp] = -INFINITY;
    return;
  }
  const int a0 = a.lig.atom_off[l];
  const int N = a.lig.atom_off[l + 1] - a0;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  const float* pose = a.poses + (size_t)a.K * (7 * (size_t)l + r0) + (size_t)p * (7 + n);
  double* y = ys[w];
  double c0[3] = {0.0, 0.0, 0.0};
  for (int i = lane; i < N; i += 32)
    for (int k = 0; k < 3; ++k) c0[k] += (double)a.lig.xyz[3 * (a0 + i) + k];
  for (int k = 0; k < 3; ++k) c0[k] = warp_sum_d(c0[k]) / N;
  for (int i = lane; i < N; i += 32)
    for (int k = 0; k < 3; ++k) y[3 * i + k] = (double)a.lig.xyz[3 * (a0 + i) + k] - c0[k];
  __syncwarp();
  for (int b = 0; b < n; ++b) {
    const uchar4 bi = a.pk.binfo[r0 + b];
    if (!lg_check(a.check, bi.x < N && bi.y < N && bi.z < N, kChkAtomIndex)) continue;
    const double pv[3] = {y[3 * bi.y], y[3 * bi.y + 1], y[3 * bi.y + 2]};
    double kx = pv[0] - y[3 * bi.x], ky = pv[1] - y[3 * bi.x + 1], kz = pv[2] - y[3 * bi.x + 2];
    const double kn = sqrt(kx * kx + ky * ky + kz * kz);
    kx /= kn; ky /= kn; kz /= kn;
    double s, c;
    sincos((double)pose[7 + b], &s, &c);
    const uint8_t* fr = a.pk.frag + (size_t)(r0 + b) * kFragStride;
    for (int t = lane; t < bi.z; t += 32) {
      const int i = fr[t];
      if (!lg_check(a.check, i < N, kChkAtomIndex)) continue;
      const double dx = y[3 * i] - pv[0], dy = y[3 * i + 1] - pv[1], dz = y[3 * i + 2] - pv[2];
      const double kd = kx * dx + ky * dy + kz * dz;
      y[3 * i] = pv[0] + kx * kd + (dx - kx * kd) * c + (ky * dz - kz * dy) * s;
      y[3 * i + 1] = pv[1] + ky * kd + (dy - ky * kd) * c + (kz * dx - kx * dz) * s;
      y[3 * i + 2] = pv[2] + kz * kd + (dz - kz * kd) * c + (kx * dy - ky * dx) * s;
    }
    __syncwarp();
  }
  const double qn = sqrt((double)pose[3] * pose[3] + (double)pose[4] * pose[4] + (double)pose[5] * pose[5] +
                         (double)pose[6] * pose[6]);
  const double qw = pose[3] / qn, qx = pose[4] / qn, qy = pose[5] / qn, qz = pose[6] / qn;
  const double R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                       2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                       2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
  double S = 0.0;
  for (int i = lane; i < N; i += 32) {
    double x[3];
    for (int r = 0; r < 3; ++r)
      x[r] = R[3 * r] * y[3 * i] + R[3 * r + 1] * y[3 * i + 1] + R[3 * r + 2] * y[3 * i + 2] + (double)pose[r];
    S -= trilinear64(a, x[0], x[1], x[2], a.lig.type[a0 + i]);
  }
  S = warp_sum_d(S);
  if (lane == 0) a.s64[gp] = S;
}

// Re-rank the K poses of each ligand by FP64 score; ties go to the lower
// restart (or the lower current rank when restart ids are not kept).
__global__ void __launch_bounds__(32 * kResWarps) rerank_kernel(const RescoreArgs a) {
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.x * kResWarps + (threadIdx.x >> 5);
  if (l >= a.lig.L) return;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  const int plen = 7 + n;
  const size_t base = (size_t)a.K * (7 * (size_t)l + r0);
  const double* s = a.s64 + (size_t)l * a.K;
  double last_s = INFINITY;
  int last_key = -1;
  for (int rank = 0; rank < a.K; ++rank) {
    double bs = -INFINITY;
    int bkey = 0x7fffffff, bp = 0;
    for (int p = lane; p < a.K; p += 32) {
      const double v = isnan(s[p]) ? -INFINITY : s[p];
      const int key = a.tmp_top ? a.tmp_top[(size_t)l * a.K + p] : p;
      const bool after = (v < last_s) || (v == last_s && key > last_key);
      if (after && (v > bs || (v == bs && key < bkey))) { bs = v; bkey = key; bp = p; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double os = __shfl_xor_sync(kFull, bs, o);
      const int ok = __shfl_xor_sync(kFull, bkey, o);
      const int op = __shfl_xor_sync(kFull, bp, o);
      if (os > bs || (os == bs && ok < bkey)) { bs = os; bkey = ok; bp = op; }
    }
    last_s = bs;
    last_key = bkey;
    for (int e = lane; e < plen; e += 32)
      a.poses[base + (size_t)rank * plen + e] = a.tmp_poses[base + (size_t)bp * plen + e];
    if (lane == 0) {
      a.scores[(size_t)l * a.K + rank] = (float)bs;
      if (a.out_s64) a.out_s64[(size_t)l * a.K + rank] = bs;
      if (a.top_restart) a.top_restart[(size_t)l * a.K + rank] = a.tmp_top[(size_t)l * a.K + bp];
    }
  }
}

}  // namespace

cudaError_t launch_rescore(const RescoreArgs& a, cudaStream_t s) {
  const size_t total = (size_t)a.lig.L * a.K;
  if (total == 0) return cudaSuccess;
  rescore_kernel<<<(unsigned)((total + kResWarps - 1) / kResWarps), 32 * kResWarps, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rerank_kernel<<<(unsigned)((a.lig.L + kResWarps - 1) / kResWarps), 32 * kResWarps, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ligen
