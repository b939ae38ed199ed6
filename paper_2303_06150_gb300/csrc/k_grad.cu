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
// kept when it raises S, otherwise the step sizes are halved. Each iteration
// evaluates the candidate once, score and gradient together, so a kept step
// already has the gradient for the next one (measured on GB300, refining
// 8,000 screening ligands' top 16 poses for 50 steps: 10.1 ms, against 14.1
// ms with a score-only candidate evaluation followed by a gradient
// re-evaluation after every kept step).
//
// Mapping. The poses of a warp belong to one ligand, so every group runs the
// same atom and bond loops in lockstep and the per-bond work (the torsion
// rebuild, the group sums) is shared by 32 / kGradLanes poses instead of
// occupying a whole warp for one pose, whose 32 lanes mostly idle on ligands
// of a few dozen atoms. A warp whose ligand has fewer
// poses left than groups shadows the last pose in the spare groups and
// writes nothing for them.
#include <cmath>

#include "../../include/ligen.h"
#include "internal.h"
#include "pose_build.cuh"

namespace ligen {
namespace {

constexpr int kGradWarps = 4;
// Lanes per pose: measured on GB300 (refining 8,000 screening ligands' top
// 16 poses), 16 lanes are 1-2% faster than 8 and 40% faster than 4; with the
// one-evaluation step and the shared bond values, 8 lanes (four poses per
// warp, three CTAs per SM) come within 1% either way.
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

// S of `pose` for ligand l and dS/dpose into `grad` (shared, 7 + n floats).
// Every lane of the group returns S. Called by all lanes of the warp.
__device__ float group_score_grad(const GradArgs& a, int l, const float* pose, const PoseMem& W, float* grad) {
  const int sub = threadIdx.x % kGradLanes;
  const int a0 = a.lig.atom_off[l];
  const int N = a.lig.atom_off[l + 1] - a0;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  for (int i = sub; i < N; i += kGradLanes) W.y[i] = a.pk.xc[a0 + i];
  GroupBonds<kGradLanes> bonds;   // also read by the torsion-gradient loop below
  bonds.load(a.pk, r0, n, pose + 7, sub);
  __syncwarp();
  group_torsions<kGradLanes>(a.pk, r0, n, N, bonds, W.y, a.grid.check, sub);
  const float qn = sqrtf(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
  const float rqn = 1.f / qn;
  const Quat q = {pose[3] * rqn, pose[4] * rqn, pose[5] * rqn, pose[6] * rqn};
  float R[9];
  qmat(q, R);
  // dR/dq^ of the polynomial rotation matrix
  const float dR[4][9] = {
      {0.f, -2.f * q.z, 2.f * q.y, 2.f * q.z, 0.f, -2.f * q.x, -2.f * q.y, 2.f * q.x, 0.f},
      {0.f, 2.f * q.y, 2.f * q.z, 2.f * q.y, -4.f * q.x, -2.f * q.w, 2.f * q.z, 2.f * q.w, -4.f * q.x},
      {-4.f * q.y, 2.f * q.x, 2.f * q.w, 2.f * q.x, 0.f, 2.f * q.z, -2.f * q.w, 2.f * q.z, -4.f * q.y},
      {-4.f * q.z, -2.f * q.w, 2.f * q.x, 2.f * q.w, -4.f * q.z, 2.f * q.y, 2.f * q.x, 2.f * q.y, 0.f}};
  // dS/dq^_k = sum_i g_i . (dR/dq^_k) y_i = sum_rc (dR/dq^_k)_rc Gy_rc with
  // Gy = sum_i g_i y_i^T: 9 FMAs per atom, the contraction once per pose
  float S = 0.f, gt[3] = {0.f, 0.f, 0.f}, Gy[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) Gy[e] = 0.f;
  for (int i = sub; i < N; i += kGradLanes) {
    const float4 v = W.y[i];
    float x[3], u[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      x[r] = fmaf(R[3 * r], v.x, fmaf(R[3 * r + 1], v.y, fmaf(R[3 * r + 2], v.z, pose[r])));
      u[r] = (x[r] - a.origin[r]) * a.inv_h;
    }
    float gx, gy, gz;
    S -= grid_sample_grad(a.grid, u[0], u[1], u[2], __float_as_int(v.w), &gx, &gy, &gz);
    const float gi[3] = {-gx * a.inv_h, -gy * a.inv_h, -gz * a.inv_h};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      gt[r] += gi[r];
      W.x[3 * i + r] = x[r];
      W.g[3 * i + r] = gi[r];
      Gy[3 * r] = fmaf(gi[r], v.x, Gy[3 * r]);
      Gy[3 * r + 1] = fmaf(gi[r], v.y, Gy[3 * r + 1]);
      Gy[3 * r + 2] = fmaf(gi[r], v.z, Gy[3 * r + 2]);
    }
  }
  S = group_sum(S);
#pragma unroll
  for (int r = 0; r < 3; ++r) gt[r] = group_sum(gt[r]);
#pragma unroll
  for (int e = 0; e < 9; ++e) Gy[e] = group_sum(Gy[e]);
  float dq[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float acc = 0.f;
#pragma unroll
    for (int e = 0; e < 9; ++e) acc = fmaf(dR[k][e], Gy[e], acc);
    dq[k] = acc;
  }
  __syncwarp();
  if (sub == 0) {
    const float proj = q.w * dq[0] + q.x * dq[1] + q.y * dq[2] + q.z * dq[3];
    const float qh[4] = {q.w, q.x, q.y, q.z};
    for (int r = 0; r < 3; ++r) grad[r] = gt[r];
    for (int k = 0; k < 4; ++k) grad[3 + k] = (dq[k] - qh[k] * proj) * rqn;
  }
  for (int b = 0; b < n; ++b) {
    const uchar4 bi = bonds.bond(b);
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

// Six resident CTAs (at most 80 registers; a few bytes spill): measured on
// GB300, 4% faster than the unconstrained 96 registers (five CTAs) and 7%
// faster than eight CTAs at 64 registers.
__global__ void __launch_bounds__(32 * kGradWarps, 6) refine_kernel(const GradArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float gbuf[2][kGroups][7 + LIGEN_MAX_ROT];
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
  float* grad = gbuf[0][sl.slot];     // gradient at `pose`
  float* grad_c = gbuf[1][sl.slot];   // gradient at the candidate
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
    // step sizes over gradient norms: one division each, then products
    const float kt = nt > 0.f ? st / nt : 0.f;
    const float kq = nq > 0.f ? sq / nq : 0.f;
    const float kth = nth > 0.f ? sth / nth : 0.f;
    const float rqn = 1.f / sqrtf(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
    float qq[4], qm = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      qq[k] = fmaf(kq, grad[3 + k], pose[3 + k] * rqn);
      qm += qq[k] * qq[k];
    }
    const float rqm = 1.f / sqrtf(qm);
    for (int e = sub; e < plen; e += kGradLanes) {
      float v;
      if (e < 3) {
        v = fmaf(kt, grad[e], pose[e]);
        v = fminf(fmaxf(v, a.box_lo[e]), a.box_hi[e]);
      } else if (e < 7) {
        v = qq[e - 3] * rqm;
      } else {
        // wrap to [-pi, pi): a step from a wrapped angle needs at most one
        // turn (w - 2 pi is exact there, as fmodf would give); other
        // inputs take the general reduction
        const float w0 = fmaf(kth, grad[e], pose[e]) + kPiF;
        float w = w0;
        if (w >= 2.f * kPiF) w -= 2.f * kPiF;
        else if (w < 0.f) w += 2.f * kPiF;
        if (!(w >= 0.f && w < 2.f * kPiF)) {
          w = fmodf(w0, 2.f * kPiF);
          if (w < 0.f) w += 2.f * kPiF;
        }
        v = w - kPiF;
      }
      cand[e] = v;
    }
    __syncwarp();
    // The candidate is evaluated with its gradient: a kept step then needs
    // no second evaluation (the buffers swap), a rejected one drops it.
    const float S2 = group_score_grad(a, l, cand, W, grad_c);
    const bool take = S2 > S;   // identical in every lane of the group (group sums)
    if (sl.own && a.out_accept && sub == 0) a.out_accept[gp * a.steps + s] = take ? 1 : 0;
    if (take) {
      for (int e = sub; e < plen; e += kGradLanes) pose[e] = cand[e];
      S = S2;
      float* t = grad;
      grad = grad_c;
      grad_c = t;
    } else {
      st *= 0.5f; sq *= 0.5f; sth *= 0.5f;
    }
    __syncwarp();
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
