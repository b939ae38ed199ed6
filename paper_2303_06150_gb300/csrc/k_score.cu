// Pose scoring: a group of kScoreLanes lanes per pose, two poses of one
// ligand per warp (the warp's per-bond work, the torsion rebuild, serves
// both; measured on GB300, scoring the 600,000 kept poses of the screening
// library took 1.17 ms per call against 1.24 ms with a warp per pose, grid
// preparation and packing included; 0.86 ms since the FP32 grid records are
// prepared in FP32).
//
// The pose (t, q, theta) is turned into atom positions exactly as the docking
// output defines them: torsions bond by bond in index order on the centred
// input coordinates (each about the current axis from its fixed endpoint to
// its moving endpoint), then the rotation R(q / |q|) and the translation t.
// Each lane then samples its atoms and the group sums S = -sum_i E_i. A warp
// whose ligand has one pose left shadows it in the spare group, which
// writes nothing.
#include <cmath>

#include "../../include/ligen.h"
#include "internal.h"

namespace ligen {
namespace {

constexpr int kScoreWarps = 4;
constexpr int kScoreLanes = 16;
constexpr int kScorePoses = 32 / kScoreLanes;   // poses per warp
static_assert(LIGEN_MAX_ROT <= 2 * kScoreLanes, "two torsions per lane");

// The record of bond b, held by lane b % kScoreLanes of this lane's group.
__device__ __forceinline__ uchar4 bond_of(uchar4 mine, int b) {
  const unsigned w = __shfl_sync(0xffffffffu, *reinterpret_cast<const unsigned*>(&mine), b % kScoreLanes, kScoreLanes);
  return *reinterpret_cast<const uchar4*>(&w);
}

__global__ void __launch_bounds__(32 * kScoreWarps) score_kernel(const ScoreArgs a) {
  __shared__ float4 ys[kScoreWarps * kScorePoses][LIGEN_MAX_ATOMS];
  const int w = threadIdx.x >> 5, grp = (threadIdx.x & 31) / kScoreLanes, sub = threadIdx.x % kScoreLanes;
  const int wpl = (a.P + kScorePoses - 1) / kScorePoses;   // warps per ligand
  const size_t gw = (size_t)blockIdx.x * kScoreWarps + w;
  if (gw >= (size_t)a.lig.L * wpl) return;   // uniform over the warp
  const int l = (int)(gw / wpl);
  const int p0 = (int)(gw % wpl) * kScorePoses + grp;
  const bool own = p0 < a.P;
  const int p = own ? p0 : a.P - 1;
  const size_t gp = (size_t)l * a.P + p;
  const unsigned full = 0xffffffffu;
  if (a.pk.status[l] != 0) {   // uniform over the warp (one ligand)
    if (own && sub == 0) a.out_scores[gp] = -INFINITY;
    return;
  }
  const int a0 = a.lig.atom_off[l];
  const int N = a.lig.atom_off[l + 1] - a0;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  const float* pose = a.poses + (size_t)a.P * (7 * (size_t)l + r0) + (size_t)p * (7 + n);
  if (!lg_check(a.grid.check, N <= a.max_atoms, kChkItemShape)) {
    if (own && sub == 0) a.out_scores[gp] = -INFINITY;
    return;
  }
  float4* y = ys[w * kScorePoses + grp];
  for (int i = sub; i < N; i += kScoreLanes) y[i] = a.pk.xc[a0 + i];
  // sin and cos of torsions sub and sub + kScoreLanes and their bond records,
  // handed to the rebuild by shuffles (one sincosf per lane instead of n)
  float s_lo = 0.f, c_lo = 1.f, s_hi = 0.f, c_hi = 1.f;
  uchar4 bi_lo = make_uchar4(0, 0, 0, 0), bi_hi = bi_lo;
  if (sub < n) {
    sincosf(pose[7 + sub], &s_lo, &c_lo);
    bi_lo = a.pk.binfo[r0 + sub];
  }
  if (sub + kScoreLanes < n) {
    sincosf(pose[7 + kScoreLanes + sub], &s_hi, &c_hi);
    bi_hi = a.pk.binfo[r0 + kScoreLanes + sub];
  }
  __syncwarp();
  for (int b = 0; b < n; ++b) {   // b is uniform over the warp (one ligand)
    const bool lo = b < kScoreLanes;
    const float s = __shfl_sync(full, lo ? s_lo : s_hi, b % kScoreLanes, kScoreLanes);
    const float c = __shfl_sync(full, lo ? c_lo : c_hi, b % kScoreLanes, kScoreLanes);
    const uchar4 bi = bond_of(lo ? bi_lo : bi_hi, b);
    if (!lg_check(a.grid.check, bi.x < N && bi.y < N && bi.z < N, kChkAtomIndex)) continue;
    const float4 pv = y[bi.y], pu = y[bi.x];
    float kx = pv.x - pu.x, ky = pv.y - pu.y, kz = pv.z - pu.z;
    const float kn = rsqrtf(kx * kx + ky * ky + kz * kz);
    kx *= kn; ky *= kn; kz *= kn;
    const uint8_t* fr = a.pk.frag + (size_t)(r0 + b) * kFragStride;
    for (int t = sub; t < bi.z; t += kScoreLanes) {
      const int i = fr[t];
      if (!lg_check(a.grid.check, i < N, kChkAtomIndex)) continue;
      float4 v = y[i];
      const float dx = v.x - pv.x, dy = v.y - pv.y, dz = v.z - pv.z;
      const float kd = kx * dx + ky * dy + kz * dz;
      const float ex = dx - kx * kd, ey = dy - ky * kd, ez = dz - kz * kd;
      const float qx = ky * dz - kz * dy, qy = kz * dx - kx * dz, qz = kx * dy - ky * dx;
      v.x = pv.x + kx * kd + ex * c + qx * s;
      v.y = pv.y + ky * kd + ey * c + qy * s;
      v.z = pv.z + kz * kd + ez * c + qz * s;
      y[i] = v;
    }
    __syncwarp();
  }
  const Quat q = qnormalize({pose[3], pose[4], pose[5], pose[6]});
  float R[9];
  qmat(q, R);
  float acc = 0.f;
  for (int i = sub; i < N; i += kScoreLanes) {
    const float4 v = y[i];
    float u[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float x = fmaf(R[3 * r], v.x, fmaf(R[3 * r + 1], v.y, fmaf(R[3 * r + 2], v.z, pose[r])));
      u[r] = (x - a.origin[r]) * a.inv_h;
    }
    acc -= grid_sample(a.grid, u[0], u[1], u[2], __float_as_int(v.w));
  }
#pragma unroll
  for (int o = kScoreLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(full, acc, o);
  if (own && sub == 0) a.out_scores[gp] = acc;
}

}  // namespace

cudaError_t launch_score(const ScoreArgs& a, cudaStream_t s) {
  if ((size_t)a.lig.L * a.P == 0) return cudaSuccess;
  const size_t warps = (size_t)a.lig.L * ((a.P + kScorePoses - 1) / kScorePoses);
  const size_t blocks = (warps + kScoreWarps - 1) / kScoreWarps;
  score_kernel<<<(unsigned)blocks, 32 * kScoreWarps, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ligen
