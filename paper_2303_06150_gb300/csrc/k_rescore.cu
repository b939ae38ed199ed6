// FP64 re-score of kept poses and re-ranking: FP64 arithmetic on the GPU is
// spent only on the K kept poses of each ligand, where near-ties between
// FP32 scores decide the ranking.
//
// Everything is recomputed in FP64 from the caller's FP32 inputs: the input
// centroid, the torsions (bond by bond, about the current axes), the
// rotation q/|q|, the translation, and the trilinear value from the eight
// FP32 node values of the caller's [z][y][x][c] grid.
//
// Mapping. GB300 issues FP64 at a small fraction of its FP32 rate, so the
// FP64 instruction count decides the time. A group of kRsLanes lanes scores
// one pose and a warp holds kRsPoses poses of the same ligand: the per-bond
// work (axis length, its reciprocal) is one FP64 instruction stream for all
// of the warp's poses, each group's lanes split the moving atoms and the
// atoms, and the torsions' sines and cosines are computed once per bond by
// one lane of the group and passed by shuffle (measured on GB300, re-scoring
// the 600,000 kept poses of the screening library: 28 ms with a warp per
// pose and every lane repeating the per-bond work). Positions are scaled by
// 1/h (one FP64 product) instead of divided by h; the two differ by FP64
// rounding only.
// Re-ranking: one warp per ligand orders its K poses by FP64 score
// (descending; ties by the restart that produced them) and rewrites poses,
// scores and restart ids in that order.
#include <cmath>

#include "../../include/ligen.h"
#include "internal.h"

namespace ligen {
namespace {

constexpr int kResWarps = 4;
constexpr int kRsLanes = 8;
constexpr int kRsPoses = 32 / kRsLanes;            // poses per warp (one ligand)
constexpr int kRsK = LIGEN_MAX_ROT / kRsLanes;     // bonds per lane of a group
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ double group_sum_d(double v) {
#pragma unroll
  for (int o = kRsLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ double trilinear64(const RescoreArgs& a, double inv_h, double x, double y, double z, int c) {
  const double u[3] = {(x - a.origin[0]) * inv_h, (y - a.origin[1]) * inv_h, (z - a.origin[2]) * inv_h};
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
  extern __shared__ double ys[];   // [kResWarps * kRsPoses][max_atoms * 3]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int grp = lane / kRsLanes, sub = lane % kRsLanes;
  const int wpl = (a.K + kRsPoses - 1) / kRsPoses;   // warps per ligand
  const size_t gw = (size_t)blockIdx.x * kResWarps + w;
  if (gw >= (size_t)a.lig.L * wpl) return;   // uniform over the warp
  const int l = (int)(gw / wpl);
  const int p0 = (int)(gw % wpl) * kRsPoses + grp;
  const bool own = p0 < a.K;
  const int p = own ? p0 : a.K - 1;          // spare groups shadow the last pose
  const size_t gp = (size_t)l * a.K + p;
  if (a.status[l] != 0 ||
      !lg_check(a.check, a.lig.atom_off[l + 1] - a.lig.atom_off[l] <= a.max_atoms, kChkItemShape)) {
    if (own && sub == 0) a.s64[gp] = -INFINITY;
    return;
  }
  const int a0 = a.lig.atom_off[l];
  const int N = a.lig.atom_off[l + 1] - a0;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  const float* pose = a.poses + (size_t)a.K * (7 * (size_t)l + r0) + (size_t)p * (7 + n);
  double* y = ys + (size_t)(w * kRsPoses + grp) * a.max_atoms * 3;
  double c0[3] = {0.0, 0.0, 0.0};
  for (int i = lane; i < N; i += 32)
    for (int k = 0; k < 3; ++k) c0[k] += (double)a.lig.xyz[3 * (a0 + i) + k];
  for (int k = 0; k < 3; ++k) c0[k] = warp_sum_d(c0[k]) / N;
  for (int i = sub; i < N; i += kRsLanes)
    for (int k = 0; k < 3; ++k) y[3 * i + k] = (double)a.lig.xyz[3 * (a0 + i) + k] - c0[k];
  // sine and cosine of bond b held by lane b % kRsLanes of the group
  double bs[kRsK], bc[kRsK];
#pragma unroll
  for (int k = 0; k < kRsK; ++k) {
    bs[k] = 0.0;
    bc[k] = 1.0;
    if (sub + k * kRsLanes < n) sincos((double)pose[7 + sub + k * kRsLanes], &bs[k], &bc[k]);
  }
  __syncwarp();
  for (int b = 0; b < n; ++b) {   // uniform over the warp (one ligand)
    const uchar4 bi = a.pk.binfo[r0 + b];
    if (!lg_check(a.check, bi.x < N && bi.y < N && bi.z < N, kChkAtomIndex)) continue;
    double sb = bs[0], cb = bc[0];
#pragma unroll
    for (int k = 1; k < kRsK; ++k)
      if (b / kRsLanes == k) { sb = bs[k]; cb = bc[k]; }
    const double s = __shfl_sync(kFull, sb, b % kRsLanes, kRsLanes);
    const double c = __shfl_sync(kFull, cb, b % kRsLanes, kRsLanes);
    const double pv[3] = {y[3 * bi.y], y[3 * bi.y + 1], y[3 * bi.y + 2]};
    double kx = pv[0] - y[3 * bi.x], ky = pv[1] - y[3 * bi.x + 1], kz = pv[2] - y[3 * bi.x + 2];
    const double inv = 1.0 / sqrt(kx * kx + ky * ky + kz * kz);
    kx *= inv; ky *= inv; kz *= inv;
    const uint8_t* fr = a.pk.frag + (size_t)(r0 + b) * kFragStride;
    for (int t = sub; t < bi.z; t += kRsLanes) {
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
  const double qi = 1.0 / qn;
  const double qw = pose[3] * qi, qx = pose[4] * qi, qy = pose[5] * qi, qz = pose[6] * qi;
  const double R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                       2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                       2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
  const double inv_h = 1.0 / a.h;
  double S = 0.0;
  for (int i = sub; i < N; i += kRsLanes) {
    double x[3];
    for (int r = 0; r < 3; ++r)
      x[r] = R[3 * r] * y[3 * i] + R[3 * r + 1] * y[3 * i + 1] + R[3 * r + 2] * y[3 * i + 2] + (double)pose[r];
    S -= trilinear64(a, inv_h, x[0], x[1], x[2], a.lig.type[a0 + i]);
  }
  S = group_sum_d(S);
  if (own && sub == 0) a.s64[gp] = S;
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
  const size_t smem = (size_t)kResWarps * kRsPoses * a.max_atoms * 3 * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const size_t warps = (size_t)a.lig.L * ((a.K + kRsPoses - 1) / kRsPoses);
  rescore_kernel<<<(unsigned)((warps + kResWarps - 1) / kResWarps), 32 * kResWarps, smem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rerank_kernel<<<(unsigned)((a.lig.L + kResWarps - 1) / kResWarps), 32 * kResWarps, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ligen
