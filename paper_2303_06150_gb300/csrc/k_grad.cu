// Pose gradients and gradient refinement: a group of kGradLanes lanes per
// pose, 32 / kGradLanes poses (of one ligand) per warp.
//
// S(t, q, theta) = -sum_i E(x_i), x_i = R(q/|q|) y_i + t, y_i the centred
// input coordinates after the torsions. Per atom g_i = dS/dx_i = -grad E(x_i)
// (one-sided at cell faces, zero outside the box); then
//   dS/dt       = sum_i g_i
//   dS/dq       = (I - q^ q^T) (sum_i g_i . (dR/dq^_k) y_i)_k / |q|
//   dS/dtheta_b = sum_{i moving for b} g_i . (w_b x (x_i - x_v)),
// with w_b the unit axis of bond b in the final pose (torsions commute, so
// theta_b may be taken as the last rotation). Atom coordinates are rebuilt
// from the pose at every evaluation; nothing is kept between calls.
//
// Refinement: per pose, `steps` iterations of normalised-step projected
// ascent (t clamped to the box, q renormalised, theta wrapped); a step is
// kept when it raises S, otherwise the step sizes are halved.
//
// Mapping. The poses of a warp belong to one ligand, so every group runs the
// same atom and bond loops in lockstep and the per-bond work (the torsion
// rebuild with its sincos, the group sums) is shared by 32 / kGradLanes
// poses instead of occupying a whole warp for one pose, whose 32 lanes
// mostly idle on ligands of a few dozen atoms. A warp whose ligand has fewer
// poses left than groups shadows the last pose in the spare groups and
// writes nothing for them.
#include <cmath>

#include "../../include/ligen.h"
#include "internal.h"

namespace ligen {
namespace {

constexpr int kGradWarps = 4;
// Lanes per pose: measured on GB300 (refining 8,000 screening ligands' top
// 16 poses), 16 lanes are 1-2% faster than 8 and 40% faster than 4.
constexpr int kGradLanes = 16;
constexpr int kPosesPerWarp = 32 / kGradLanes;
constexpr int kGroups = kGradWarps * kPosesPerWarp;  // poses per CTA
constexpr unsigned kFull = 0xffffffffu;
constexpr float kPiF = 3.14159265358979323846f;

// Sum over the kGradLanes lanes of a group (every group of the warp at once).
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = kGradLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

struct PoseMem {
  float4* y;   // [max_atoms] body coordinates after torsions (w = type)
  float* x;    // [max_atoms][3] world coordinates
  float* g;    // [max_atoms][3] dS/dx
};

// S of `pose` for ligand l; with `grad` (shared, 7 + n floats) also dS/dpose.
// Every lane of the group returns S. Called by all lanes of the warp.
__device__ float group_score_grad(const GradArgs& a, int l, const float* pose, const PoseMem& W, float* grad) {
  const int sub = threadIdx.x % kGradLanes;
  const int a0 = a.lig.atom_off[l];
  const int N = a.lig.atom_off[l + 1] - a0;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  for (int i = sub; i < N; i += kGradLanes) W.y[i] = a.pk.xc[a0 + i];
  __syncwarp();
  for (int b = 0; b < n; ++b) {
    const uchar4 bi = a.pk.binfo[r0 + b];
    if (!lg_check(a.grid.check, bi.x < N && bi.y < N && bi.z < N, kChkAtomIndex)) continue;
    const float4 pv = W.y[bi.y], pu = W.y[bi.x];
    float kx = pv.x - pu.x, ky = pv.y - pu.y, kz = pv.z - pu.z;
    const float kn = rsqrtf(kx * kx + ky * ky + kz * kz);
    kx *= kn; ky *= kn; kz *= kn;
    float s, c;
    sincosf(pose[7 + b], &s, &c);
    const uint8_t* fr = a.pk.frag + (size_t)(r0 + b) * kFragStride;
    for (int t = sub; t < bi.z; t += kGradLanes) {
      const int i = fr[t];
      if (!lg_check(a.grid.check, i < N, kChkAtomIndex)) continue;
      float4 v = W.y[i];
      const float dx = v.x - pv.x, dy = v.y - pv.y, dz = v.z - pv.z;
      const float kd = kx * dx + ky * dy + kz * dz;
      const float ex = dx - kx * kd, ey = dy - ky * kd, ez = dz - kz * kd;
      const float qx = ky * dz - kz * dy, qy = kz * dx - kx * dz, qz = kx * dy - ky * dx;
      v.x = pv.x + kx * kd + ex * c + qx * s;
      v.y = pv.y + ky * kd + ey * c + qy * s;
      v.z = pv.z + kz * kd + ez * c + qz * s;
      W.y[i] = v;
    }
    __syncwarp();
  }
  const float qn = sqrtf(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
  const Quat q = {pose[3] / qn, pose[4] / qn, pose[5] / qn, pose[6] / qn};
  float R[9];
  qmat(q, R);
  // dR/dq^ of the polynomial rotation matrix
  const float dR[4][9] = {
      {0.f, -2.f * q.z, 2.f * q.y, 2.f * q.z, 0.f, -2.f * q.x, -2.f * q.y, 2.f * q.x, 0.f},
      {0.f, 2.f * q.y, 2.f * q.z, 2.f * q.y, -4.f * q.x, -2.f * q.w, 2.f * q.z, 2.f * q.w, -4.f * q.x},
      {-4.f * q.y, 2.f * q.x, 2.f * q.w, 2.f * q.x, 0.f, 2.f * q.z, -2.f * q.w, 2.f * q.z, -4.f * q.y},
      {-4.f * q.z, -2.f * q.w, 2.f * q.x, 2.f * q.w, -4.f * q.z, 2.f * q.y, 2.f * q.x, 2.f * q.y, 0.f}};
  float S = 0.f, gt[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
  for (int i = sub; i < N; i += kGradLanes) {
    const float4 v = W.y[i];
    float x[3], u[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      x[r] = fmaf(R[3 * r], v.x, fmaf(R[3 * r + 1], v.y, fmaf(R[3 * r + 2], v.z, pose[r])));
      u[r] = (x[r] - a.origin[r]) * a.inv_h;
    }
    if (!grad) {
      S -= grid_sample(a.grid, u[0], u[1], u[2], __float_as_int(v.w));
      continue;
    }
    float gx, gy, gz;
    S -= grid_sample_grad(a.grid, u[0], u[1], u[2], __float_as_int(v.w), &gx, &gy, &gz);
    const float gi[3] = {-gx * a.inv_h, -gy * a.inv_h, -gz * a.inv_h};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      gt[r] += gi[r];
      W.x[3 * i + r] = x[r];
      W.g[3 * i + r] = gi[r];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int r = 0; r < 3; ++r)
        dq[k] += gi[r] * fmaf(dR[k][3 * r], v.x, fmaf(dR[k][3 * r + 1], v.y, dR[k][3 * r + 2] * v.z));
  }
  S = group_sum(S);
  if (!grad) return S;
#pragma unroll
  for (int r = 0; r < 3; ++r) gt[r] = group_sum(gt[r]);
#pragma unroll
  for (int k = 0; k < 4; ++k) dq[k] = group_sum(dq[k]);
  __syncwarp();
  if (sub == 0) {
    const float proj = q.w * dq[0] + q.x * dq[1] + q.y * dq[2] + q.z * dq[3];
    const float qh[4] = {q.w, q.x, q.y, q.z};
    for (int r = 0; r < 3; ++r) grad[r] = gt[r];
    for (int k = 0; k < 4; ++k) grad[3 + k] = (dq[k] - qh[k] * proj) / qn;
  }
  for (int b = 0; b < n; ++b) {
    const uchar4 bi = a.pk.binfo[r0 + b];
    if (!lg_check(a.grid.check, bi.x < N && bi.y < N && bi.z < N, kChkAtomIndex)) continue;
    const float* xv = W.x + 3 * bi.y;
    const float* xu = W.x + 3 * bi.x;
    float ox = xv[0] - xu[0], oy = xv[1] - xu[1], oz = xv[2] - xu[2];
    const float on = rsqrtf(ox * ox + oy * oy + oz * oz);
    ox *= on; oy *= on; oz *= on;
    const uint8_t* fr = a.pk.frag + (size_t)(r0 + b) * kFragStride;
    float acc = 0.f;
    for (int t = sub; t < bi.z; t += kGradLanes) {
      const int i = fr[t];
      if (!lg_check(a.grid.check, i < N, kChkAtomIndex)) continue;
      const float dx = W.x[3 * i] - xv[0], dy = W.x[3 * i + 1] - xv[1], dz = W.x[3 * i + 2] - xv[2];
      acc += W.g[3 * i] * (oy * dz - oz * dy) + W.g[3 * i + 1] * (oz * dx - ox * dz) +
             W.g[3 * i + 2] * (ox * dy - oy * dx);
    }
    acc = group_sum(acc);
    if (sub == 0) grad[7 + b] = acc;
  }
  __syncwarp();
  return S;
}

// Bytes of one pose's region: body coordinates (16 per atom) then world
// coordinates and gradients (12 + 12 per atom), rounded up to 16 so that the
// next region's float4 array stays 16-byte aligned.
__host__ __device__ __forceinline__ size_t pose_region(int max_atoms) {
  return ((size_t)max_atoms * 40 + 15) & ~(size_t)15;
}

__device__ __forceinline__ PoseMem pose_mem(unsigned char* smem, int max_atoms, int slot) {
  const size_t per = pose_region(max_atoms);
  unsigned char* base = smem + per * slot;
  PoseMem W;
  W.y = (float4*)base;
  W.x = (float*)(base + (size_t)max_atoms * 16);
  W.g = W.x + 3 * max_atoms;
  return W;
}

// The pose of this lane's group: warp gw of the grid covers ligand
// gw / warps_per_ligand, poses (gw % warps_per_ligand) * kPosesPerWarp + group.
struct Slot {
  int l, p;        // ligand and pose (the shadowed last pose for a spare group)
  bool own;        // false for a spare group: computes, writes nothing
  int slot;        // this group's index in the CTA
  bool in_grid;    // false when the whole warp is past the last ligand
};

__device__ __forceinline__ Slot slot_of(const GradArgs& a) {
  const int w = threadIdx.x >> 5, grp = (threadIdx.x & 31) / kGradLanes;
  const int wpl = (a.P + kPosesPerWarp - 1) / kPosesPerWarp;
  const size_t gw = (size_t)blockIdx.x * kGradWarps + w;
  Slot s;
  s.in_grid = gw < (size_t)a.lig.L * wpl;
  s.l = s.in_grid ? (int)(gw / wpl) : 0;
  const int p = (int)(gw % wpl) * kPosesPerWarp + grp;
  s.own = s.in_grid && p < a.P;
  s.p = p < a.P ? p : a.P - 1;
  s.slot = w * kPosesPerWarp + grp;
  return s;
}

__global__ void __launch_bounds__(32 * kGradWarps) grad_kernel(const GradArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float gbuf[kGroups][7 + LIGEN_MAX_ROT];
  const Slot sl = slot_of(a);
  if (!sl.in_grid) return;   // uniform over the warp
  const int sub = threadIdx.x % kGradLanes;
  const int l = sl.l;
  const size_t gp = (size_t)l * a.P + sl.p;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  const size_t off = (size_t)a.P * (7 * (size_t)l + r0) + (size_t)sl.p * (7 + n);
  if (a.pk.status[l] != 0 ||
      !lg_check(a.grid.check, a.lig.atom_off[l + 1] - a.lig.atom_off[l] <= a.max_atoms, kChkItemShape)) {
    if (sl.own) {   // the early return is uniform over the warp (one ligand)
      if (sub == 0) a.out_scores[gp] = -INFINITY;
      for (int e = sub; e < 7 + n; e += kGradLanes) a.out_grads[off + e] = 0.f;
    }
    return;
  }
  const PoseMem W = pose_mem(smem, a.max_atoms, sl.slot);
  const float S = group_score_grad(a, l, a.poses + off, W, gbuf[sl.slot]);
  if (sl.own) {
    if (sub == 0) a.out_scores[gp] = S;
    for (int e = sub; e < 7 + n; e += kGradLanes) a.out_grads[off + e] = gbuf[sl.slot][e];
  }
}

__global__ void __launch_bounds__(32 * kGradWarps) refine_kernel(const GradArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float gbuf[kGroups][7 + LIGEN_MAX_ROT];
  __shared__ float pbuf[kGroups][7 + LIGEN_MAX_ROT];
  __shared__ float cbuf[kGroups][7 + LIGEN_MAX_ROT];
  const Slot sl = slot_of(a);
  if (!sl.in_grid) return;   // uniform over the warp
  const int sub = threadIdx.x % kGradLanes;
  const int l = sl.l;
  const size_t gp = (size_t)l * a.P + sl.p;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  const int plen = 7 + n;
  float* pose_g = a.inout_poses + (size_t)a.P * (7 * (size_t)l + r0) + (size_t)sl.p * plen;
  if (a.pk.status[l] != 0 ||
      !lg_check(a.grid.check, a.lig.atom_off[l + 1] - a.lig.atom_off[l] <= a.max_atoms, kChkItemShape)) {
    if (sl.own && sub == 0) a.out_scores[gp] = -INFINITY;
    return;   // uniform over the warp (one ligand)
  }
  const PoseMem W = pose_mem(smem, a.max_atoms, sl.slot);
  float* pose = pbuf[sl.slot];
  float* cand = cbuf[sl.slot];
  float* grad = gbuf[sl.slot];
  for (int e = sub; e < plen; e += kGradLanes) pose[e] = pose_g[e];
  __syncwarp();
  float S = group_score_grad(a, l, pose, W, grad);
  float st = a.step_t, sq = a.step_q, sth = a.step_theta;
  for (int s = 0; s < a.steps; ++s) {
    float nt = 0.f, nq = 0.f, nth = 0.f;
    for (int e = sub; e < plen; e += kGradLanes) {
      const float v = grad[e] * grad[e];
      if (e < 3) nt += v; else if (e < 7) nq += v; else nth += v;
    }
    nt = sqrtf(group_sum(nt));
    nq = sqrtf(group_sum(nq));
    nth = sqrtf(group_sum(nth));
    const float qn = sqrtf(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
    float qq[4], qm = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      qq[k] = pose[3 + k] / qn + (nq > 0.f ? sq * grad[3 + k] / nq : 0.f);
      qm += qq[k] * qq[k];
    }
    qm = sqrtf(qm);
    for (int e = sub; e < plen; e += kGradLanes) {
      float v;
      if (e < 3) {
        v = pose[e] + (nt > 0.f ? st * grad[e] / nt : 0.f);
        v = fminf(fmaxf(v, a.box_lo[e]), a.box_hi[e]);
      } else if (e < 7) {
        v = qq[e - 3] / qm;
      } else {
        v = pose[e] + (nth > 0.f ? sth * grad[e] / nth : 0.f);
        v = fmodf(v + kPiF, 2.f * kPiF);
        if (v < 0.f) v += 2.f * kPiF;
        v -= kPiF;
      }
      cand[e] = v;
    }
    __syncwarp();
    const float S2 = group_score_grad(a, l, cand, W, nullptr);
    const bool take = S2 > S;   // identical in every lane of the group (group sums)
    if (sl.own && a.out_accept && sub == 0) a.out_accept[gp * a.steps + s] = take ? 1 : 0;
    if (take) {
      for (int e = sub; e < plen; e += kGradLanes) pose[e] = cand[e];
    } else {
      st *= 0.5f; sq *= 0.5f; sth *= 0.5f;
    }
    __syncwarp();
    // A group that moved needs the gradient at its new pose. The evaluation
    // is warp-wide, so when any group moved every group re-evaluates at its
    // current pose: for the others that is the pose they already had, and
    // the same arithmetic gives the same S and gradient.
    if (__any_sync(kFull, take)) S = group_score_grad(a, l, pose, W, grad);
  }
  if (sl.own) {
    const float sgn = pose[3] < 0.f ? -1.f : 1.f;
    for (int e = sub; e < plen; e += kGradLanes) pose_g[e] = (e >= 3 && e < 7) ? sgn * pose[e] : pose[e];
    if (sub == 0) a.out_scores[gp] = S;
  }
}

}  // namespace

size_t grad_smem_bytes(int max_atoms) { return (size_t)kGroups * pose_region(max_atoms); }

cudaError_t launch_grad(const GradArgs& a, bool refine, cudaStream_t s) {
  if ((size_t)a.lig.L * a.P == 0) return cudaSuccess;
  const size_t smem = grad_smem_bytes(a.max_atoms);
  auto* k = refine ? refine_kernel : grad_kernel;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const size_t warps = (size_t)a.lig.L * ((a.P + kPosesPerWarp - 1) / kPosesPerWarp);
  const size_t blocks = (warps + kGradWarps - 1) / kGradWarps;
  k<<<(unsigned)blocks, 32 * kGradWarps, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ligen
