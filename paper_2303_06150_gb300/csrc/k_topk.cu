// Top-K selection and pose compaction: one warp per ligand.
//
// The ligand's R restart scores are held in registers (lane j owns restarts
// j, j + 32, ...; up to kRegSlots per lane) with a per-lane mask of taken
// restarts. Round k takes the best untaken restart in the order (score
// descending, restart index ascending): each lane proposes its best untaken
// slot (slots ascend in restart index), a shuffle argmax picks the warp's,
// and the owning lane marks it taken. Ligands with more restarts than the
// registers hold rank from memory instead: round k takes the best restart
// ranked after the one taken in round k-1, so no marks are needed. The
// winners are taken 32 at a time and the j-th lane rebuilds the j-th
// winner's pose from its restart index (random stream), its cube rotation
// and its torsion counts, all 32 at once, written as t[3], q[4] (w >= 0),
// theta[n] in [-pi, pi). A NaN score (only possible from a NaN grid) ranks as
// -infinity, so the order stays total and K <= R rounds always find a
// restart.
#include <cmath>

#include "../../include/ligen.h"
#include "internal.h"

namespace ligen {
namespace {

constexpr int kTopkWarps = 4;
constexpr int kRegSlots = 8;   // restarts per lane held in registers (R <= 256)

// Warp argmax over (score descending, restart ascending).
__device__ __forceinline__ void warp_best(float& bs, int& br) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, bs, o);
    const int orr = __shfl_xor_sync(0xffffffffu, br, o);
    if (os > bs || (os == bs && orr < br)) { bs = os; br = orr; }
  }
}

__global__ void __launch_bounds__(32 * kTopkWarps) topk_kernel(const TopkArgs a) {
  const int lane = threadIdx.x & 31;
  const int l = blockIdx.x * kTopkWarps + (threadIdx.x >> 5);
  if (l >= a.L) return;
  const int r0 = a.rot_off[l];
  const int n = a.rot_off[l + 1] - r0;
  const int plen = 7 + n;
  float* poses = a.out_poses + (size_t)a.K * (7 * (size_t)l + r0);
  float* scores = a.out_scores + (size_t)l * a.K;
  if (a.status[l] != 0) {
    for (int k = 0; k < a.K; ++k) {
      if (lane == 0) scores[k] = -INFINITY;
      if (a.top_restart && lane == 0) a.top_restart[(size_t)l * a.K + k] = -1;
      for (int e = lane; e < plen; e += 32) poses[(size_t)k * plen + e] = (e == 3) ? 1.f : 0.f;
    }
    return;
  }
  const float* rs = a.res_score + (size_t)l * a.R;
  const bool in_regs = a.R <= 32 * kRegSlots;
  float v[kRegSlots];
  unsigned taken = 0;
#pragma unroll
  for (int i = 0; i < kRegSlots; ++i) {
    const int r = lane + 32 * i;
    v[i] = -INFINITY;
    if (in_regs && r < a.R) v[i] = isnan(rs[r]) ? -INFINITY : rs[r];   // total order
    else taken |= 1u << i;                                             // no such restart
  }
  float last_s = INFINITY;
  int last_r = -1;
  // K winners in chunks of 32: select the chunk's winners (lane j keeps
  // the j-th), then every lane rebuilds its winner's pose at once
  for (int k0 = 0; k0 < a.K; k0 += 32) {
    const int kn = a.K - k0 < 32 ? a.K - k0 : 32;
    float my_s = -INFINITY;
    int my_r = 0;
    for (int j = 0; j < kn; ++j) {
      float bs = -INFINITY;
      int br = 0x7fffffff;
      if (in_regs) {
#pragma unroll
        for (int i = 0; i < kRegSlots; ++i) {
          const int r = lane + 32 * i;
          if (!(taken >> i & 1u) && (v[i] > bs || (v[i] == bs && r < br))) { bs = v[i]; br = r; }
        }
        warp_best(bs, br);
        if ((br & 31) == lane && br < a.R) taken |= 1u << (br >> 5);
      } else {
        for (int r = lane; r < a.R; r += 32) {
          const float s = isnan(rs[r]) ? -INFINITY : rs[r];
          const bool after = (s < last_s) || (s == last_s && r > last_r);
          if (after && (s > bs || (s == bs && r < br))) { bs = s; br = r; }
        }
        warp_best(bs, br);
      }
      if (br >= a.R) br = a.R - 1;   // unreachable while K <= R; keeps every index in range
      last_s = bs;
      last_r = br;
      if (lane == j) {
        my_s = bs;
        my_r = br;
      }
    }
    if (lane >= kn) continue;
    // rebuild the winner's pose
    const int k = k0 + lane, br = my_r;
    float u[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) u[q] = restart_uniform(a.seed, (uint32_t)l, (uint32_t)br, (uint32_t)q);
    const Quat qr = qnormalize(shoemake(u[0], u[1], u[2]));
    Quat q = qnormalize(qmul(qr, cube_quat(a.res_k[(size_t)l * a.R + br])));
    if (q.w < 0.f) q = {-q.w, -q.x, -q.y, -q.z};
    float* out = poses + (size_t)k * plen;
    const uint8_t* cnt = a.res_cnt + (size_t)r0 * a.R + (size_t)br * n;
#pragma unroll
    for (int e = 0; e < 3; ++e) out[e] = a.center[e] + (2.0f * u[3 + e] - 1.0f) * a.jitter;
    out[3] = q.w;
    out[4] = q.x;
    out[5] = q.y;
    out[6] = q.z;
    for (int b = 0; b < n; ++b) {
      int deg = ((int)cnt[b] * a.step_deg) % 360;
      if (deg >= 180) deg -= 360;
      out[7 + b] = (float)deg * 0.017453292519943295f;
    }
    scores[k] = my_s;
    if (a.top_restart) a.top_restart[(size_t)l * a.K + k] = br;
  }
}

}  // namespace

cudaError_t launch_topk(const TopkArgs& a, cudaStream_t s) {
  if (a.L == 0) return cudaSuccess;
  const int blocks = (a.L + kTopkWarps - 1) / kTopkWarps;
  topk_kernel<<<blocks, 32 * kTopkWarps, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ligen
