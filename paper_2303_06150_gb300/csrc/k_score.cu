// Pose scoring: a group of kScoreLanes lanes per pose, two poses of one
// ligand per warp (the warp's per-bond work, the torsion rebuild, serves
// both; measured on GB300, scoring the 600,000 kept poses of the screening
// library took 1.17 ms per call against 1.24 ms with a warp per pose, grid
// preparation and packing included; 0.86 ms since the FP32 grid records are
// prepared in FP32, 0.68 ms with the occupancy below).
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
#include "pose_build.cuh"

namespace ligen {
namespace {

constexpr int kScoreWarps = 4;
constexpr int kScoreLanes = 16;
constexpr int kScorePoses = 32 / kScoreLanes;   // poses per warp

// Eight resident CTAs (64 registers) and shared memory sized by the call's
// largest ligand rather than the 256-atom limit: the kernel is latency-bound
// (ncu: 44% issue slots busy, long-scoreboard stalls first), and more warps
// hide more of it. Measured on GB300, scoring the 600,000 kept screening
// poses: 0.80 -> 0.68 ms per call against six CTAs with 32 KB of static
// shared memory each.
__global__ void __launch_bounds__(32 * kScoreWarps, 8) score_kernel(const ScoreArgs a) {
  extern __shared__ float4 ys[];   // [kScoreWarps * kScorePoses][max_atoms]
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
  float4* y = ys + (size_t)(w * kScorePoses + grp) * a.max_atoms;
  for (int i = sub; i < N; i += kScoreLanes) y[i] = a.pk.xc[a0 + i];
  GroupBonds<kScoreLanes> bonds;
  bonds.load(a.pk, r0, n, pose + 7, sub);
  __syncwarp();
  group_torsions<kScoreLanes>(a.pk, r0, n, N, bonds, y, a.grid.check, sub);
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
  const size_t smem = (size_t)kScoreWarps * kScorePoses * a.max_atoms * sizeof(float4);   // <= 32 KB
  score_kernel<<<(unsigned)blocks, 32 * kScoreWarps, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ligen
