// Pose gradients and gradient refinement. Two kernels: grad_lane_kernel
// (4 or more poses per ligand; the main path) puts a group of G = 1, 2 or 4
// lanes on each pose and builds the torsions as forward kinematics
// (fk_pose.cuh, the table of fk_table_kernel), the torsion gradients from
// subtree sums, launched by rotatable-bond class; grad_kernel / refine_kernel
// (fewer poses) put a group of kGradLanes lanes on each pose, 32 / kGradLanes
// poses (of one ligand) per warp, and apply the torsions atom by atom. What
// follows holds for both.
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
// rebuild, the group sums) is shared by the warp's poses instead of
// occupying a whole warp for one pose, whose 32 lanes mostly idle on ligands
// of a few dozen atoms. A warp whose ligand has fewer
// poses left than groups shadows the last pose in the spare groups and
// writes nothing for them.
#include <cmath>

#include "../../include/ligen.h"
#include "fk_pose.cuh"
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

// --------------------------------------------------------------------------
// Pose-group gradients and refinement on forward kinematics (fk_pose.cuh).
//
// One warp per (ligand, PW poses), a group of G = 32 / PW lanes per pose. A
// pose's n + 1 transforms are built once into shared memory
// [slot][pose][12], the group's lanes sharing the bonds of each depth of
// the bond tree (fk_transforms_group); each lane of the group then takes atoms
// sub, sub + G, ... : position u = T_owner x (grid units), value and
// gradient of the cell polynomial, du = dS/du. Per lane it accumulates
//   dS/dt contribution  sum du,
//   the rotation term   Gp = sum du (x - t)^T   (x the position in A),
//   per owner bond b    F_b = sum du,  tau_b = sum u x du.
// The bond sums become subtree sums (children added into parents, in
// reverse bond order), so F_b and tau_b cover b's whole moving side, and
//   dS/dtheta_b = w_b . (tau_b - u_v x F_b)
// with w_b the unit axis and u_v the axis point of bond b in the pose, from
// the parent's transform (torsions commute, so theta_b may be taken as the
// last rotation), the group's lanes sharing the bonds; dS/dq through q/|q|
// from Gy = Gp R (y = R^T (x - t) the body coordinates), as in the group
// kernel above. Nothing is stored between
// evaluations but the pose, its gradient and the transforms.
//
// Refinement runs the group kernel's steps (normalised-step projected
// ascent, keep if S rises, else halve) per pose, the group's first lane
// doing the per-pose scalar work.

template <int G>
struct GL {
  static constexpr int PW = 32 / G;   // poses per warp
};

// Shared memory of one warp: transforms [ncap + 1][PW][12]; per-lane bond
// sums [ncap][32][6]; pose state [4][PW][7 + ncap] (pose, candidate, two
// gradients); then the staged ligand.
template <int G>
__host__ __device__ inline size_t gl_carve(int acap, int ncap, unsigned char* base, FkLigand* S, float** T,
                                           float** acc, float** st) {
  constexpr int PW = GL<G>::PW;
  const size_t tb = (size_t)(ncap + 1) * PW * 12 * sizeof(float);
  const size_t ab = (size_t)ncap * 32 * 6 * sizeof(float);
  const size_t sb = ((size_t)4 * PW * (7 + ncap) * sizeof(float) + 15) & ~(size_t)15;
  if (base) {
    *T = (float*)base;
    *acc = (float*)(base + tb);
    *st = (float*)(base + tb + ab);
  }
  return tb + ab + sb + fk_ligand_carve(acap, ncap, base ? base + tb + ab + sb : nullptr, S);
}

__device__ __forceinline__ float gl_sum(float v, int G) {
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// S of `pose` (7 + n floats, shared by the group) and dS/dpose into `grad`
// (written by the group's first lane). Every lane of the group returns S.
// All lanes of the warp call it.
template <int G>
__device__ float gl_eval(const GradArgs& a, const FkLigand& S, int N, int n, const float* pose, float* grad,
                         float* T, float* acc, int grp, int sub, int lane) {
  constexpr int PW = GL<G>::PW;
  const float rqn = rsqrtf(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
  const Quat q = {pose[3] * rqn, pose[4] * rqn, pose[5] * rqn, pose[6] * rqn};
  fk_transforms_group<G>(S, n, pose, q, pose + 7, a.origin, a.inv_h, T + 12 * grp, (size_t)PW * 12, sub);
  for (int b = 0; b < n; ++b)
#pragma unroll
    for (int e = 0; e < 6; ++e) acc[((size_t)b * 32 + lane) * 6 + e] = 0.f;
  __syncwarp();
  const float d0[3] = {a.origin[0] - pose[0], a.origin[1] - pose[1], a.origin[2] - pose[2]};
  float Sl = 0.f, gs[3] = {0.f, 0.f, 0.f}, Gp[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) Gp[e] = 0.f;
  // The atoms are listed by owner: the owner's transform stays in registers
  // across its atoms, and so do this lane's (F, tau) sums of the owner, added
  // to the shared per-owner row once per run (the same additions in the
  // same order as adding atom by atom to the row, which starts at zero).
  int cur = -1;
  float4 m0, m1, m2;
  float fa[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  auto flush = [&]() {
    if (cur >= 0 && cur < n) {
      float* ac = acc + ((size_t)cur * 32 + lane) * 6;
#pragma unroll
      for (int e = 0; e < 6; ++e) ac[e] += fa[e];
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) fa[e] = 0.f;
  };
  for (int i = sub; i < N; i += G) {
    const float4 X = S.sx[i];
    const int o = S.own[i];
    if (o != cur) {
      flush();
      fk_get(T + ((size_t)o * PW + grp) * 12, m0, m1, m2);
      cur = o;
    }
    const float u[3] = {fmaf(m0.x, X.x, fmaf(m0.y, X.y, fmaf(m0.z, X.z, m0.w))),
                        fmaf(m1.x, X.x, fmaf(m1.y, X.y, fmaf(m1.z, X.z, m1.w))),
                        fmaf(m2.x, X.x, fmaf(m2.y, X.y, fmaf(m2.z, X.z, m2.w)))};
    float gx, gy, gz;
    Sl -= grid_sample_grad(a.grid, u[0], u[1], u[2], __float_as_int(X.w), &gx, &gy, &gz);
    const float du[3] = {-gx, -gy, -gz};   // dS/du, per grid unit
#pragma unroll
    for (int r = 0; r < 3; ++r) gs[r] += du[r];
    const float dv[3] = {fmaf(a.h, u[0], d0[0]), fmaf(a.h, u[1], d0[1]), fmaf(a.h, u[2], d0[2])};   // x - t, A
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Gp[3 * r + c] = fmaf(du[r], dv[c], Gp[3 * r + c]);
    if (o < n) {
      fa[0] += du[0];
      fa[1] += du[1];
      fa[2] += du[2];
      fa[3] += u[1] * du[2] - u[2] * du[1];
      fa[4] += u[2] * du[0] - u[0] * du[2];
      fa[5] += u[0] * du[1] - u[1] * du[0];
    }
  }
  flush();
  // subtree sums, children first (this lane's own sums)
  for (int r = n - 1; r >= 0; --r) {
    const int b = S.ord[r], pb = S.par[b];
    if (pb < n) {
#pragma unroll
      for (int e = 0; e < 6; ++e) acc[((size_t)pb * 32 + lane) * 6 + e] += acc[((size_t)b * 32 + lane) * 6 + e];
    }
  }
  Sl = gl_sum(Sl, G);
#pragma unroll
  for (int r = 0; r < 3; ++r) gs[r] = gl_sum(gs[r], G);
#pragma unroll
  for (int e = 0; e < 9; ++e) Gp[e] = gl_sum(Gp[e], G);
  __syncwarp();
  if (sub == 0) {
    float R[9];
    qmat(q, R);
    // Gy = Gp R: sum du y^T with y = R^T (x - t)
    float Gy[9];
    mat3mul(Gp, R, Gy);
    const float dR[4][9] = {
        {0.f, -2.f * q.z, 2.f * q.y, 2.f * q.z, 0.f, -2.f * q.x, -2.f * q.y, 2.f * q.x, 0.f},
        {0.f, 2.f * q.y, 2.f * q.z, 2.f * q.y, -4.f * q.x, -2.f * q.w, 2.f * q.z, 2.f * q.w, -4.f * q.x},
        {-4.f * q.y, 2.f * q.x, 2.f * q.w, 2.f * q.x, 0.f, 2.f * q.z, -2.f * q.w, 2.f * q.z, -4.f * q.y},
        {-4.f * q.z, -2.f * q.w, 2.f * q.x, 2.f * q.w, -4.f * q.z, 2.f * q.y, 2.f * q.x, 2.f * q.y, 0.f}};
    float dq[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float s = 0.f;
#pragma unroll
      for (int e = 0; e < 9; ++e) s = fmaf(dR[k][e], Gy[e], s);
      dq[k] = s * a.inv_h;
    }
    const float proj = q.w * dq[0] + q.x * dq[1] + q.y * dq[2] + q.z * dq[3];
    const float qh[4] = {q.w, q.x, q.y, q.z};
#pragma unroll
    for (int r = 0; r < 3; ++r) grad[r] = gs[r] * a.inv_h;
#pragma unroll
    for (int k = 0; k < 4; ++k) grad[3 + k] = (dq[k] - qh[k] * proj) * rqn;
  }
  for (int b = sub; b < n; b += G) {   // torsion gradients, bonds over the group's lanes
    float F[3] = {0.f, 0.f, 0.f}, tau[3] = {0.f, 0.f, 0.f};
    for (int j = 0; j < G; ++j) {   // the group's lanes, in lane order
      const float* ac = acc + ((size_t)b * 32 + grp * G + j) * 6;
      F[0] += ac[0]; F[1] += ac[1]; F[2] += ac[2];
      tau[0] += ac[3]; tau[1] += ac[4]; tau[2] += ac[5];
    }
    float4 p0, p1, p2;
    fk_get(T + ((size_t)S.par[b] * PW + grp) * 12, p0, p1, p2);
    const float4 xv = S.sx[S.sb[b].y], k = S.ax[b];
    const float uv[3] = {fmaf(p0.x, xv.x, fmaf(p0.y, xv.y, fmaf(p0.z, xv.z, p0.w))),
                         fmaf(p1.x, xv.x, fmaf(p1.y, xv.y, fmaf(p1.z, xv.z, p1.w))),
                         fmaf(p2.x, xv.x, fmaf(p2.y, xv.y, fmaf(p2.z, xv.z, p2.w)))};
    float w[3] = {p0.x * k.x + p0.y * k.y + p0.z * k.z, p1.x * k.x + p1.y * k.y + p1.z * k.z,
                  p2.x * k.x + p2.y * k.y + p2.z * k.z};
    const float wn = rsqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    const float c0 = tau[0] - (uv[1] * F[2] - uv[2] * F[1]);
    const float c1 = tau[1] - (uv[2] * F[0] - uv[0] * F[2]);
    const float c2 = tau[2] - (uv[0] * F[1] - uv[1] * F[0]);
    grad[7 + b] = (w[0] * c0 + w[1] * c1 + w[2] * c2) * wn;
  }
  __syncwarp();
  return Sl;
}

template <int G, bool REFINE>
__global__ void __launch_bounds__(32, 16) grad_lane_kernel(const GradArgs a) {
  constexpr int PW = GL<G>::PW;
  extern __shared__ __align__(16) unsigned char gl_smem[];
  const int acap = a.max_atoms, ncap = a.max_rot;
  FkLigand S;
  float *T, *acc, *st;
  gl_carve<G>(acap, ncap, gl_smem, &S, &T, &acc, &st);
  const int lane = threadIdx.x & 31, grp = lane / G, sub = lane % G;
  const int wpl = (a.P + PW - 1) / PW;   // warps per ligand
  const size_t gw = blockIdx.x;
  if (gw >= (size_t)a.n_list * wpl) return;
  const int li = (int)(gw / wpl);
  const int l = a.list ? a.list[li] : li;
  const int p0 = (int)(gw % wpl) * PW + grp;
  const bool own = p0 < a.P;
  const int p = own ? p0 : a.P - 1;   // spare groups shadow the last pose and write nothing
  const size_t gp = (size_t)l * a.P + p;
  const int a0 = a.lig.atom_off[l];
  const int N = a.lig.atom_off[l + 1] - a0;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  const int plen = 7 + n;
  const size_t off = (size_t)a.P * (7 * (size_t)l + r0) + (size_t)p * plen;
  bool ok = a.pk.status[l] == 0 && lg_check(a.grid.check, N <= acap && n <= ncap, kChkItemShape);
  if (ok) ok = lg_check(a.grid.check, fk_load(a.pk, l, a0, N, r0, n, S, lane), kChkAtomIndex);
  if (!ok) {   // uniform over the warp (one ligand)
    if (own && sub == 0) a.out_scores[gp] = -INFINITY;
    if (!REFINE && own)
      for (int e = sub; e < plen; e += G) a.out_grads[off + e] = 0.f;
    return;
  }
  const int sl = 7 + ncap;
  float* pose = st + (size_t)(0 * PW + grp) * sl;
  float* cand = st + (size_t)(1 * PW + grp) * sl;
  float* grad = st + (size_t)(2 * PW + grp) * sl;
  float* grad_c = st + (size_t)(3 * PW + grp) * sl;
  const float* src = REFINE ? a.inout_poses : a.poses;
  for (int e = sub; e < plen; e += G) pose[e] = src[off + e];
  __syncwarp();
  float Sc = gl_eval<G>(a, S, N, n, pose, grad, T, acc, grp, sub, lane);
  if constexpr (!REFINE) {
    if (own) {
      if (sub == 0) a.out_scores[gp] = Sc;
      for (int e = sub; e < plen; e += G) a.out_grads[off + e] = grad[e];
    }
    return;
  } else {
    float s_t = a.step_t, s_q = a.step_q, s_th = a.step_theta;
    for (int s = 0; s < a.steps; ++s) {
      if (sub == 0) {
        float nt = 0.f, nq = 0.f, nth = 0.f;
        for (int e = 0; e < plen; ++e) {
          const float v = grad[e] * grad[e];
          if (e < 3) nt += v; else if (e < 7) nq += v; else nth += v;
        }
        nt = sqrtf(nt); nq = sqrtf(nq); nth = sqrtf(nth);
        const float kt = nt > 0.f ? s_t / nt : 0.f;
        const float kq = nq > 0.f ? s_q / nq : 0.f;
        const float kth = nth > 0.f ? s_th / nth : 0.f;
        const float rqn = 1.f / sqrtf(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
        float qq[4], qm = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          qq[k] = fmaf(kq, grad[3 + k], pose[3 + k] * rqn);
          qm += qq[k] * qq[k];
        }
        const float rqm = 1.f / sqrtf(qm);
        for (int e = 0; e < plen; ++e) {
          float v;
          if (e < 3) {
            v = fmaf(kt, grad[e], pose[e]);
            v = fminf(fmaxf(v, a.box_lo[e]), a.box_hi[e]);
          } else if (e < 7) {
            v = qq[e - 3] * rqm;
          } else {
            // wrap to [-pi, pi): one turn suffices from a wrapped angle;
            // other inputs take the general reduction
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
      }
      __syncwarp();
      // the candidate with its gradient: a kept step needs no second evaluation
      const float S2 = gl_eval<G>(a, S, N, n, cand, grad_c, T, acc, grp, sub, lane);
      const bool take = S2 > Sc;   // identical in every lane of the group (group sums)
      if (own && a.out_accept && sub == 0) a.out_accept[gp * a.steps + s] = take ? 1 : 0;
      if (take) {
        float* t = pose; pose = cand; cand = t;
        t = grad; grad = grad_c; grad_c = t;
        Sc = S2;
      } else {
        s_t *= 0.5f; s_q *= 0.5f; s_th *= 0.5f;
      }
      __syncwarp();
    }
    if (own) {
      const float sgn = pose[3] < 0.f ? -1.f : 1.f;
      for (int e = sub; e < plen; e += G) a.inout_poses[off + e] = (e >= 3 && e < 7) ? sgn * pose[e] : pose[e];
      if (sub == 0) a.out_scores[gp] = Sc;
    }
  }
}

template <int G, bool REFINE>
cudaError_t launch_gl(const GradArgs& a, cudaStream_t s) {
  const size_t smem = gl_carve<G>(a.max_atoms, a.max_rot, nullptr, nullptr, nullptr, nullptr, nullptr);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(grad_lane_kernel<G, REFINE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const size_t blocks = (size_t)a.n_list * ((a.P + GL<G>::PW - 1) / GL<G>::PW);
  grad_lane_kernel<G, REFINE><<<(unsigned)blocks, 32, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grad_lanes(const GradArgs& a, bool refine, cudaStream_t s) {
  if ((size_t)a.n_list * a.P == 0) return cudaSuccess;
  // lanes per pose: the fewest that fill a warp with this many poses
  const int G = a.P > 16 ? 1 : a.P > 8 ? 2 : 4;
  if (G == 1) return refine ? launch_gl<1, true>(a, s) : launch_gl<1, false>(a, s);
  if (G == 2) return refine ? launch_gl<2, true>(a, s) : launch_gl<2, false>(a, s);
  return refine ? launch_gl<4, true>(a, s) : launch_gl<4, false>(a, s);
}

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
