// Pose scoring: S = -sum_i E_i of given poses (t, q, theta), the atom
// positions as the docking output defines them (torsions bond by bond in
// index order on the centred input coordinates, each about the current axis
// from its fixed endpoint to its moving endpoint; then R(q / |q|) and t).
// Three kernels:
//   score_lane_kernel  16 or more poses per ligand: one pose per lane, the
//                      torsions as forward kinematics (fk_pose.cuh), launched
//                      by rotatable-bond class (see its comment);
//   fk_table_kernel    the ligand-only part of the forward kinematics, once
//                      per library or call (owners, parents, orders, axes,
//                      the atoms listed by owner);
//   score_kernel       fewer poses: a group of kScoreLanes lanes per pose,
//                      two poses of one ligand per warp, the torsions
//                      applied atom by atom (pose_build.cuh). Measured on
//                      GB300 on the 600,000 kept screening poses, before
//                      the pose-per-lane kernel: 1.17 ms per call against
//                      1.24 ms with a warp per pose, grid preparation and
//                      packing included; 0.86 ms with the FP32 grid records
//                      prepared in FP32, 0.68 ms with the occupancy below.
//                      A warp whose ligand has one pose left shadows it in
//                      the spare group, which writes nothing.
#include <cmath>
#include <map>
#include <mutex>

#include "../../include/ligen.h"
#include "internal.h"
#include "fk_pose.cuh"
#include "pose_build.cuh"

namespace ligen {
namespace {

// grid_sample without a branch around the load: the position is clamped
// into the box first, so the record address is always valid and the load
// is unconditional (the compiler can issue the loads of several atoms
// before using any), and the penalty is selected afterwards for a point
// outside the box. Inside the box the clamp changes nothing and the value
// is grid_sample's, bit for bit; a NaN coordinate clamps to 0 and takes the
// penalty, as in grid_sample.
__device__ __forceinline__ float grid_sample_nb(const GridView& g, float ux, float uy, float uz, int c) {
  const bool inb = (ux >= 0.f) & (ux <= g.mx) & (uy >= 0.f) & (uy <= g.my) & (uz >= 0.f) & (uz <= g.mz);
  const float vx = fminf(fmaxf(ux, 0.f), g.mx), vy = fminf(fmaxf(uy, 0.f), g.my), vz = fminf(fmaxf(uz, 0.f), g.mz);
  const float fx = fminf(floorf(vx), g.mx - 1.f);
  const float fy = fminf(floorf(vy), g.my - 1.f);
  const float fz = fminf(floorf(vz), g.mz - 1.f);
  const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
  const float dx = vx - fx, dy = vy - fy, dz = vz - fz;
  const size_t ri = rec_index(g.cx, g.cy, g.cz, c, ix, iy, iz);
  if (!lg_check(g.check, c >= 0 && c < g.nc && ri < g.n_rec, kChkGridRecord)) return g.penalty;
  float a[8];
  ld_global_v8_na(g.coef + ri * 8, a);
  const float t1 = fmaf(dz, a[7], a[4]);
  float t2 = fmaf(dy, t1, a[1]);
  t2 = fmaf(dz, a[5], t2);
  const float t3 = fmaf(dz, a[6], a[2]);
  float e = fmaf(dz, a[3], a[0]);
  e = fmaf(dy, t3, e);
  e = fmaf(dx, t2, e);
  return inb ? e : g.penalty;
}


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

// Pose-group scoring, for calls with many poses per ligand: one warp per
// (ligand, 32/G poses), a group of G lanes per pose (G = 1 in use: lane p
// scores pose p on its own), with the torsions applied as forward
// kinematics (fk_pose.cuh) instead of atom by atom: the group's first lane
// builds the n + 1 transforms of its pose, 48 bytes each, in shared memory
// [slot][pose][12] (a 48-byte stride keeps 128-bit accesses free of bank
// conflicts); per atom one 3x4 transform of its owner (9 FMA) and one
// branch-free record load, 8 in flight per lane. Shared memory grows with
// the bonds, so the caller launches ligands by rotatable-bond class. Groups
// past the ligand's last pose shadow it and write nothing.
template <int G>
__host__ __device__ inline size_t lane_carve(int acap, int ncap, unsigned char* base, FkLigand* S, float** T) {
  const size_t tbytes = (size_t)(ncap + 1) * (32 / G) * 12 * sizeof(float);
  if (T) *T = (float*)base;
  return tbytes + fk_ligand_carve(acap, ncap, base ? base + tbytes : nullptr, S);
}

// Work item gw = (ligand entry, 32/G poses) of the warp.
template <int G>
__device__ __forceinline__ void score_lane_item(const ScoreArgs& a, size_t gw, const FkLigand& S, float* T) {
  constexpr int PW = 32 / G;   // poses per warp
  const int acap = a.max_atoms, ncap = a.max_rot;
  const int lane = threadIdx.x & 31, grp = lane / G, sub = lane % G;
  const int wpl = (a.P + PW - 1) / PW;    // warps per ligand
  const int li = (int)(gw / wpl);
  const int l = a.list ? a.list[li] : li;
  const int p0 = (int)(gw % wpl) * PW + grp;
  const bool own = p0 < a.P;
  const int p = own ? p0 : a.P - 1;
  const size_t gp = (size_t)l * a.P + p;
  // the ligand's status and ranges read together (one round trip)
  const int status = a.pk.status[l];
  const int a0 = a.lig.atom_off[l], a1 = a.lig.atom_off[l + 1];
  const int r0 = a.lig.rot_off[l], r1 = a.lig.rot_off[l + 1];
  const int N = a1 - a0, n = r1 - r0;
  if (status != 0 || !lg_check(a.grid.check, N <= acap && n <= ncap, kChkItemShape)) {   // uniform
    if (own && sub == 0) a.out_scores[gp] = -INFINITY;
    return;
  }
  // The pose read before the ligand is staged, so that its loads overlap the
  // staging: t and q into registers, theta_b into element 0 of the pose's
  // transform slot b (read there by fk_transforms before it writes the slot),
  // instead of one dependent load per bond inside the forward kinematics.
  const float* pose = a.poses + (size_t)a.P * (7 * (size_t)l + r0) + (size_t)p * (7 + n);
  const size_t stride = (size_t)PW * 12;   // between a pose's transform slots
  float* Tg = T + 12 * grp;
  float pt[3], pq[4];
  if (sub == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) pt[k] = pose[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) pq[k] = pose[3 + k];
#pragma unroll 4
    for (int b = 0; b < n; ++b) Tg[(size_t)b * stride] = pose[7 + b];
  }
  if (!lg_check(a.grid.check, fk_load(a.pk, l, a0, N, r0, n, S, lane), kChkAtomIndex)) {
    if (own && sub == 0) a.out_scores[gp] = -INFINITY;
    return;
  }
  if (sub == 0) {
    const Quat q = qnormalize({pq[0], pq[1], pq[2], pq[3]});
    fk_transforms(S, n, pt, q, Tg, stride, a.origin, a.inv_h, Tg, stride);
  }
  if (G > 1) __syncwarp();
  // samples: unconditional loads, 8 gathers in flight per lane. The atoms
  // are listed by owner, so the owner's transform stays in registers across
  // its atoms and is read again only where the owner changes (a uniform
  // branch: every lane is at the same atom).
  float acc = 0.f;
  int cur = -1;
  float4 m0, m1, m2;
#pragma unroll 8
  for (int i = sub; i < N; i += G) {
    const float4 X = S.sx[i];
    const int o = S.own[i];
    if (o != cur) {
      fk_get(T + ((size_t)o * PW + grp) * 12, m0, m1, m2);
      cur = o;
    }
    const float ux = fmaf(m0.x, X.x, fmaf(m0.y, X.y, fmaf(m0.z, X.z, m0.w)));
    const float uy = fmaf(m1.x, X.x, fmaf(m1.y, X.y, fmaf(m1.z, X.z, m1.w)));
    const float uz = fmaf(m2.x, X.x, fmaf(m2.y, X.y, fmaf(m2.z, X.z, m2.w)));
    acc -= grid_sample_nb(a.grid, ux, uy, uz, __float_as_int(X.w));
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (own && sub == 0) a.out_scores[gp] = acc;
}

// Persistent: a one-warp CTA per resident slot, taking work items
// blockIdx.x, blockIdx.x + gridDim.x, ... (one CTA per item left the
// block scheduler starting 20,000 one-warp CTAs per call).
template <int G>
__global__ void __launch_bounds__(32, 16) score_lane_kernel(const ScoreArgs a) {
  extern __shared__ __align__(16) unsigned char lane_smem[];
  FkLigand S;
  float* T;
  lane_carve<G>(a.max_atoms, a.max_rot, lane_smem, &S, &T);
  const size_t items = (size_t)a.n_list * ((a.P + 32 / G - 1) / (32 / G));
  for (size_t gw = blockIdx.x; gw < items; gw += gridDim.x) {
    score_lane_item<G>(a, gw, S, T);
    __syncwarp();   // every lane done with this item's staged ligand and transforms
  }
}

// Resident CTAs of score_lane_kernel<G> for `smem` bytes, per device and
// carve-up size, queried once (the first query also sets the kernel's
// shared-memory limit to the largest carve-up any call can ask for, the
// same value every time).
template <int G>
cudaError_t slots_sl(size_t smem, size_t* slots) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, size_t> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find({dev, smem});
  if (it != cache.end()) {
    *slots = it->second;
    return cudaSuccess;
  }
  const size_t cap = lane_carve<G>(LIGEN_MAX_ATOMS, LIGEN_MAX_ROT, nullptr, nullptr, nullptr);
  int nsm = 0, per_sm = 0;
  e = cudaFuncSetAttribute(score_lane_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, score_lane_kernel<G>, 32, smem);
  if (e != cudaSuccess) return e;
  *slots = cache[{dev, smem}] = (size_t)nsm * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

template <int G>
cudaError_t config_sl(const ScoreArgs& a, LaunchCfg* c) {
  c->smem = lane_carve<G>(a.max_atoms, a.max_rot, nullptr, nullptr, nullptr);
  size_t slots = 0;
  const cudaError_t e = slots_sl<G>(c->smem, &slots);
  if (e != cudaSuccess) return e;
  const size_t items = (size_t)a.n_list * ((a.P + 32 / G - 1) / (32 / G));
  c->blocks = (unsigned)(items < slots ? items : slots);
  return cudaSuccess;
}

// One warp per ligand: the ligand staged as fk_stage<true> stages it, then
// the parts the scoring and gradient kernels read (owners, parents, orders,
// depth offsets, axes) written to the table, with the malformed flag.
constexpr int kTabWarps = 4;

__global__ void __launch_bounds__(32 * kTabWarps) fk_table_kernel(const LigandsDev lig, const Packed pk, int acap,
                                                                  int ncap) {
  extern __shared__ __align__(16) unsigned char tab_smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.x * kTabWarps + w;
  if (l >= lig.L) return;   // uniform over the warp
  const size_t lig_bytes = fk_ligand_carve(acap, ncap, nullptr, nullptr);
  const size_t per = lig_bytes + LIGEN_MAX_ATOMS;   // + each atom's position in the owner-ordered list
  FkLigand S;
  fk_ligand_carve(acap, ncap, tab_smem + (size_t)w * per, &S);
  uint8_t* pos = tab_smem + (size_t)w * per + lig_bytes;
  uint8_t* row = pk.fk_loff + (size_t)l * kFkLoffBytes;
  const int a0 = lig.atom_off[l], N = lig.atom_off[l + 1] - a0;
  const int r0 = lig.rot_off[l], n = lig.rot_off[l + 1] - r0;
  bool ok = pk.status[l] == 0 && N >= 1 && N <= acap && n >= 0 && n <= ncap;
  if (ok) ok = fk_stage<true>(pk, a0, N, r0, n, S, lane);
  if (!ok) {   // nothing of the ligand is read: only the flag
    if (lane < kFkLoffBytes) row[lane] = lane == kFkBad ? 1 : 0;
    if (lane + 32 < kFkLoffBytes) row[lane + 32] = lane + 32 == kFkBad ? 1 : 0;
    return;
  }
  // the atoms listed by owner (bond 0's, ..., bond n-1's, the root's; a
  // stable counting sort), so that a pose's consecutive atoms mostly share
  // one transform
  if (lane == 0) {
    int start[LIGEN_MAX_ROT + 2];
    for (int o = 0; o <= n + 1; ++o) start[o] = 0;
    for (int i = 0; i < N; ++i) ++start[S.own[i] + 1];
    for (int o = 0; o < n + 1; ++o) start[o + 1] += start[o];
    for (int i = 0; i < N; ++i) pos[i] = (uint8_t)start[S.own[i]]++;
  }
  __syncwarp();
  for (int i = lane; i < N; i += 32) {
    pk.fk_xs[a0 + pos[i]] = S.sx[i];
    pk.fk_own[a0 + pos[i]] = S.own[i];
  }
  for (int b = lane; b < n; b += 32) {
    pk.fk_ax[r0 + b] = S.ax[b];
    pk.fk_bond[r0 + b] = make_uchar4(S.par[b], S.ord[b], S.lord[b], pos[S.sb[b].y]);
  }
  const int depths = S.loff[LIGEN_MAX_ROT];
  for (int k = lane; k < kFkLoffBytes; k += 32)
    row[k] = k <= depths || k == LIGEN_MAX_ROT ? S.loff[k] : 0;   // k == kFkBad: 0
}

}  // namespace

cudaError_t launch_fk_table(const LigandsDev& lig, const Packed& pk, int max_atoms, int max_rot, cudaStream_t s) {
  if (lig.L == 0) return cudaSuccess;
  const size_t smem = (size_t)kTabWarps * (fk_ligand_carve(max_atoms, max_rot, nullptr, nullptr) + LIGEN_MAX_ATOMS);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fk_table_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned blocks = (unsigned)((lig.L + kTabWarps - 1) / kTabWarps);
  fk_table_kernel<<<blocks, 32 * kTabWarps, smem, s>>>(lig, pk, max_atoms, max_rot);
  return cudaGetLastError();
}

// One lane per pose. Measured on GB300, scoring the 600,000 kept screening
// poses: 0.255 ms with 1 lane per pose, 0.275 ms with 2 (one transform set
// per pose, half the shared memory per warp, half of each lane's samples)
// and 0.38 ms with 4 (class launches one after another); 0.169 against
// 0.207 ms for 1 and 2 lanes with the class launches side by side; 2 lanes
// for the classes of 12 or more bonds only (half the transform slots per
// warp, more warps per SM): 0.156 against 0.151 ms, from 16 bonds the same.
cudaError_t score_lanes_config(const ScoreArgs& a, LaunchCfg* c) { return config_sl<1>(a, c); }

cudaError_t launch_score_lanes(const ScoreArgs& a, const LaunchCfg& c, cudaStream_t s) {
  if ((size_t)a.n_list * a.P == 0 || c.blocks == 0) return cudaSuccess;
  score_lane_kernel<1><<<c.blocks, 32, c.smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_score(const ScoreArgs& a, cudaStream_t s) {
  if ((size_t)a.lig.L * a.P == 0) return cudaSuccess;
  const size_t warps = (size_t)a.lig.L * ((a.P + kScorePoses - 1) / kScorePoses);
  const size_t blocks = (warps + kScoreWarps - 1) / kScoreWarps;
  const size_t smem = (size_t)kScoreWarps * kScorePoses * a.max_atoms * sizeof(float4);   // <= 32 KB
  score_kernel<<<(unsigned)blocks, 32 * kScoreWarps, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ligen
