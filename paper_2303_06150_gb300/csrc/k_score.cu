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

// Pose-per-lane scoring, for calls with many poses per ligand: one warp per
// (ligand, 32 poses), lane p scoring pose p on its own. All lanes of the
// warp walk the same atoms and bonds (one ligand). The warp first stages the
// ligand in shared memory with coalesced loads (centred coordinates and
// types, bond records, moving-atom lists), so the per-lane loops read
// broadcast shared memory instead of dependent global loads; then every
// per-pose step is one lane's register work: no shuffles, no per-bond
// synchronisation. A lane keeps its pose's body coordinates in three
// shared-memory planes [atom][32] (lane-consecutive words: no bank
// conflicts) sized for the launch's largest ligand, which is why the caller
// launches ligands by size class. The torsions run in index order about
// each bond's current axis, then the rigid motion and the trilinear
// samples. Lanes past the ligand's last pose shadow it and write nothing.
struct LaneSmem {
  float* px;      // [cap][32] per-lane body coordinates
  float* py;
  float* pz;
  float4* sx;     // [cap] the ligand's centred input coordinates (w = type)
  uchar4* sb;     // [max_rot] bond records
  uint8_t* sf;    // [max_rot][fstride] moving-atom lists
  int fstride;
};

// A moving side has at most N/2 atoms (the smaller side of the cut), so a
// list of a ligand of at most `cap` atoms fits the first cap/2 bytes of its
// kFragStride-byte slot, rounded to a whole 16-byte vector.
__host__ __device__ inline int lane_fstride(int cap) {
  const int s = ((cap / 2 + 15) / 16) * 16;
  return s < 16 ? 16 : (s > kFragStride ? kFragStride : s);
}

__host__ __device__ inline size_t lane_carve(int cap, int max_rot, unsigned char* base, LaneSmem* S) {
  const int fs = lane_fstride(cap);
  const size_t planes = (size_t)3 * 32 * cap * sizeof(float);
  const size_t o_sx = planes;
  const size_t o_sb = o_sx + (size_t)cap * sizeof(float4);
  const size_t o_sf = o_sb + (size_t)((max_rot + 3) / 4 * 4) * sizeof(uchar4);
  const size_t end = o_sf + (size_t)max_rot * fs;
  if (S) {
    S->fstride = fs;
    S->px = (float*)base;
    S->py = S->px + 32 * cap;
    S->pz = S->py + 32 * cap;
    S->sx = (float4*)(base + o_sx);
    S->sb = (uchar4*)(base + o_sb);
    S->sf = base + o_sf;
  }
  return end;
}

__global__ void __launch_bounds__(32, 16) score_lane_kernel(const ScoreArgs a) {
  extern __shared__ __align__(16) unsigned char lane_smem[];
  const int cap = a.max_atoms;
  LaneSmem S;
  lane_carve(cap, a.max_rot, lane_smem, &S);
  const int lane = threadIdx.x & 31;
  const int wpl = (a.P + 31) / 32;    // warps per ligand
  const size_t gw = blockIdx.x;
  if (gw >= (size_t)a.n_list * wpl) return;
  const int li = (int)(gw / wpl);
  const int l = a.list ? a.list[li] : li;
  const int p0 = (int)(gw % wpl) * 32 + lane;
  const bool own = p0 < a.P;
  const int p = own ? p0 : a.P - 1;
  const size_t gp = (size_t)l * a.P + p;
  if (a.pk.status[l] != 0) {   // uniform over the warp (one ligand)
    if (own) a.out_scores[gp] = -INFINITY;
    return;
  }
  const int a0 = a.lig.atom_off[l];
  const int N = a.lig.atom_off[l + 1] - a0;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  if (!lg_check(a.grid.check, N <= cap && n <= a.max_rot, kChkItemShape)) {
    if (own) a.out_scores[gp] = -INFINITY;
    return;
  }
  // stage the ligand: coalesced, all lanes
  for (int i = lane; i < N; i += 32) S.sx[i] = a.pk.xc[a0 + i];
  for (int b = lane; b < n; b += 32) S.sb[b] = a.pk.binfo[r0 + b];
  {   // the first fstride bytes of every list (16-byte vectors)
    const int per = S.fstride / 16;
    const uint4* src = reinterpret_cast<const uint4*>(a.pk.frag + (size_t)r0 * kFragStride);
    uint4* dst = reinterpret_cast<uint4*>(S.sf);
    for (int v = lane; v < n * per; v += 32) dst[v] = src[(v / per) * (kFragStride / 16) + v % per];
  }
  const float* pose = a.poses + (size_t)a.P * (7 * (size_t)l + r0) + (size_t)p * (7 + n);
  float t[3], q4[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = pose[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) q4[k] = pose[3 + k];
  __syncwarp();
  float* px = S.px + lane;
  float* py = S.py + lane;
  float* pz = S.pz + lane;
#pragma unroll 4
  for (int i = 0; i < N; ++i) {
    const float4 X = S.sx[i];
    px[32 * i] = X.x;
    py[32 * i] = X.y;
    pz[32 * i] = X.z;
  }
  for (int b = 0; b < n; ++b) {   // index order, each about its current axis
    const uchar4 bi = S.sb[b];
    if (!lg_check(a.grid.check, bi.x < N && bi.y < N && bi.z <= S.fstride, kChkAtomIndex)) continue;
    float sn, cs;
    sincosf(pose[7 + b], &sn, &cs);
    const float vx = px[32 * bi.y], vy = py[32 * bi.y], vz = pz[32 * bi.y];
    float kx = vx - px[32 * bi.x], ky = vy - py[32 * bi.x], kz = vz - pz[32 * bi.x];
    const float kn = rsqrtf(kx * kx + ky * ky + kz * kz);
    kx *= kn; ky *= kn; kz *= kn;
    const uint8_t* fr = S.sf + b * S.fstride;
#pragma unroll 4
    for (int k = 0; k < bi.z; ++k) {
      const int i = fr[k];
      if (!lg_check(a.grid.check, i < N, kChkAtomIndex)) continue;
      const float dx = px[32 * i] - vx, dy = py[32 * i] - vy, dz = pz[32 * i] - vz;
      const float kd = kx * dx + ky * dy + kz * dz;
      const float ex = dx - kx * kd, ey = dy - ky * kd, ez = dz - kz * kd;
      const float qx = ky * dz - kz * dy, qy = kz * dx - kx * dz, qz = kx * dy - ky * dx;
      px[32 * i] = vx + kx * kd + ex * cs + qx * sn;
      py[32 * i] = vy + ky * kd + ey * cs + qy * sn;
      pz[32 * i] = vz + kz * kd + ez * cs + qz * sn;
    }
  }
  const Quat q = qnormalize({q4[0], q4[1], q4[2], q4[3]});
  float R[9];
  qmat(q, R);
  float acc = 0.f;
#pragma unroll 8
  for (int i = 0; i < N; ++i) {   // unconditional loads: 8 gathers in flight per lane
    const float x = px[32 * i], y = py[32 * i], z = pz[32 * i];
    float u[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float w = fmaf(R[3 * r], x, fmaf(R[3 * r + 1], y, fmaf(R[3 * r + 2], z, t[r])));
      u[r] = (w - a.origin[r]) * a.inv_h;
    }
    acc -= grid_sample_nb(a.grid, u[0], u[1], u[2], __float_as_int(S.sx[i].w));
  }
  if (own) a.out_scores[gp] = acc;
}

}  // namespace

size_t score_lane_smem_bytes(int cap, int max_rot) { return lane_carve(cap, max_rot, nullptr, nullptr); }

cudaError_t launch_score_lanes(const ScoreArgs& a, cudaStream_t s) {
  if ((size_t)a.n_list * a.P == 0) return cudaSuccess;
  const size_t smem = score_lane_smem_bytes(a.max_atoms, a.max_rot);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(score_lane_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const size_t blocks = (size_t)a.n_list * ((a.P + 31) / 32);
  score_lane_kernel<<<(unsigned)blocks, 32, smem, s>>>(a);
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
