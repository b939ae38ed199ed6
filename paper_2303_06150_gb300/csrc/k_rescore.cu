// FP64 re-score of kept poses and re-ranking: FP64 arithmetic on the GPU is
// spent only on the K kept poses of each ligand, where near-ties between
// FP32 scores decide the ranking.
//
// Everything is recomputed in FP64 from the caller's FP32 inputs: the input
// centroid, the pose's atom positions, and the trilinear value from the
// eight FP32 node values of the caller's [z][y][x][c] grid. The positions
// follow the pose definition (torsions bond by bond in index order, each
// about its current axis; then R(q/|q|) and t) as forward kinematics in
// FP64, equal in exact arithmetic: bond b's transform is its parent's
// composed with the rotation by theta_b about b's input-frame axis through
// its moving endpoint v, and an atom's position is its owner's transform of
// its centred input coordinates (owners, parents and the bond order from
// fk_stage, as in the scoring kernels).
//
// Mapping. GB300 issues FP64 at a small fraction of its FP32 rate, so the
// FP64 instruction count decides the time. A warp holds kRsPoses poses of
// one ligand, a group of kRsLanes lanes per pose. The bond axes and pivots
// are computed once per warp, one lane per bond. Each pose's transforms are
// composed depth by depth, the group's lanes splitting a depth's bonds. Then
// the group's lanes split the atoms: one 3x4 transform each, then the
// trilinear value. Measured on GB300, re-scoring the 600,000 kept poses of
// the screening library:
//   warp per pose, every lane repeating the per-bond work     28 ms
//   torsions atom by atom, bond axes by every lane of a group  8.5 ms
//   forward kinematics, 4 poses per warp                       6.5 ms
//   the same, 8 poses per warp (4 lanes each)                  5.1 ms
// Positions are scaled by 1/h (one FP64 product) instead of divided by h;
// the two differ by FP64 rounding only.
// Re-ranking: one warp per ligand orders its K poses by FP64 score
// (descending; ties by the restart that produced them) and rewrites poses,
// scores and restart ids in that order.
#include <cmath>

#include "../../include/ligen.h"
#include "internal.h"
#include "fk_pose.cuh"

namespace ligen {
namespace {

constexpr int kResWarps = 4;
// lanes per pose: the warp's per-pose FP64 passes (root, sines and cosines,
// transforms by depth) serve 32 / kRsLanes poses. Measured on GB300, the
// re-score stage of a screening step: 8 lanes 6.6 ms, 4 lanes 5.2 ms,
// 2 lanes 5.6 ms.
constexpr int kRsLanes = 4;
constexpr int kRsPoses = 32 / kRsLanes;            // poses per warp (one ligand)
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

// The box and scaling of the FP64 trilinear value, once per thread.
struct Tri64 {
  double ox, oy, oz, inv_h;   // origin, 1 / h
  double mx, my, mz;          // points - 1 per axis: the box in grid units
};

// FP64 trilinear value of channel c at world point (x, y, z): the cell by a
// round-down conversion, then 7 interpolations (x, then y, then z) of the 8
// FP32 node values widened to FP64. Outside the box: the penalty.
__device__ __forceinline__ double trilinear64(const RescoreArgs& a, const Tri64& t, double x, double y, double z,
                                              int c) {
  const double u0 = (x - t.ox) * t.inv_h, u1 = (y - t.oy) * t.inv_h, u2 = (z - t.oz) * t.inv_h;
  if (!(u0 >= 0.0 && u0 <= t.mx && u1 >= 0.0 && u1 <= t.my && u2 >= 0.0 && u2 <= t.mz)) return a.penalty;
  const int i0 = min(__double2int_rd(u0), a.nx - 2);
  const int i1 = min(__double2int_rd(u1), a.ny - 2);
  const int i2 = min(__double2int_rd(u2), a.nz - 2);
  const double f0 = u0 - i0, f1 = u1 - i1, f2 = u2 - i2;
  const size_t sx = (size_t)a.nc, sy = sx * a.nx, sz = sy * a.ny;
  const size_t base = ((size_t)i2 * a.ny + i1) * a.nx + i0;
  if (!lg_check(a.check, c >= 0 && c < a.nc && base + (size_t)a.nx * a.ny + a.nx + 1 < (size_t)a.nx * a.ny * a.nz,
                kChkRescoreNode))
    return a.penalty;
  const float* v = a.values + base * sx + c;
  const double c000 = v[0], c100 = v[sx], c010 = v[sy], c110 = v[sy + sx];
  const double c001 = v[sz], c101 = v[sz + sx], c011 = v[sz + sy], c111 = v[sz + sy + sx];
  const double e00 = fma(f0, c100 - c000, c000), e10 = fma(f0, c110 - c010, c010);
  const double e01 = fma(f0, c101 - c001, c001), e11 = fma(f0, c111 - c011, c011);
  const double e0 = fma(f1, e10 - e00, e00), e1 = fma(f1, e11 - e01, e01);
  return fma(f2, e1 - e0, e0);
}

// Shared memory of one warp: the staged ligand (fk_stage), then per bond
// its unit axis and pivot v in the input frame (FP64, 6 each), then the
// transforms of the warp's poses (FP64, 12 each) [slot][pose][12], the
// centred input coordinates (FP64, 3 per atom), and the sine and cosine of
// every (pose, bond) [pose][bond][2].
__host__ __device__ inline size_t rs_warp_bytes(int acap, int ncap, unsigned char* base, FkLigand* S, double** B,
                                                double** T, double** Y, double** SC) {
  const size_t lb = fk_ligand_carve(acap, ncap, base, S);   // a multiple of 16
  const size_t bb = (size_t)ncap * 6 * sizeof(double);
  const size_t tb = (size_t)(ncap + 1) * kRsPoses * 12 * sizeof(double);
  const size_t yb = ((size_t)acap * 3 * sizeof(double) + 15) & ~(size_t)15;
  const size_t sb = (size_t)kRsPoses * ncap * 2 * sizeof(double);
  if (base) {
    *B = reinterpret_cast<double*>(base + lb);
    *T = reinterpret_cast<double*>(base + lb + bb);
    *Y = reinterpret_cast<double*>(base + lb + bb + tb);
    *SC = reinterpret_cast<double*>(base + lb + bb + tb + yb);
  }
  return lb + bb + tb + yb + sb;
}

__global__ void __launch_bounds__(32 * kResWarps) rescore_kernel(const RescoreArgs a) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int grp = lane / kRsLanes, sub = lane % kRsLanes;
  const int acap = a.max_atoms, ncap = a.max_rot;
  FkLigand S;
  double *B, *T, *Y, *SC;
  const size_t per = rs_warp_bytes(acap, ncap, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
  rs_warp_bytes(acap, ncap, rs_smem + (size_t)w * per, &S, &B, &T, &Y, &SC);
  const int wpl = (a.K + kRsPoses - 1) / kRsPoses;   // warps per ligand
  const size_t gw = (size_t)blockIdx.x * kResWarps + w;
  if (gw >= (size_t)a.lig.L * wpl) return;   // uniform over the warp
  const int l = (int)(gw / wpl);
  const int p0 = (int)(gw % wpl) * kRsPoses + grp;
  const bool own = p0 < a.K;
  const int p = own ? p0 : a.K - 1;          // spare groups shadow the last pose
  const size_t gp = (size_t)l * a.K + p;
  const int a0 = a.lig.atom_off[l];
  const int N = a.lig.atom_off[l + 1] - a0;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  bool ok = a.status[l] == 0 && lg_check(a.check, N <= acap && n <= ncap, kChkItemShape);   // uniform
  if (ok) ok = lg_check(a.check, fk_stage<true>(a.pk, a0, N, r0, n, S, lane), kChkAtomIndex);
  if (!ok) {
    if (own && sub == 0) a.s64[gp] = -INFINITY;
    return;
  }
  // FP64 centroid of the input coordinates
  double c0[3] = {0.0, 0.0, 0.0};
  for (int i = lane; i < N; i += 32)
    for (int k = 0; k < 3; ++k) c0[k] += (double)a.lig.xyz[3 * (a0 + i) + k];
  for (int k = 0; k < 3; ++k) c0[k] = warp_sum_d(c0[k]) / N;
  for (int i = lane; i < N; i += 32)   // centred coordinates, once for the warp's poses
    for (int k = 0; k < 3; ++k) Y[3 * i + k] = (double)a.lig.xyz[3 * (a0 + i) + k] - c0[k];
  // per bond, once for the warp's poses: unit axis u -> v and pivot v in the
  // input frame (fk_stage checked both ends against N)
  for (int b = lane; b < n; b += 32) {
    const uchar4 bi = S.sb[b];
    double pu[3], pv[3];
    for (int k = 0; k < 3; ++k) {
      pu[k] = (double)a.lig.xyz[3 * (a0 + bi.x) + k] - c0[k];
      pv[k] = (double)a.lig.xyz[3 * (a0 + bi.y) + k] - c0[k];
    }
    const double kx = pv[0] - pu[0], ky = pv[1] - pu[1], kz = pv[2] - pu[2];
    const double inv = rsqrt(kx * kx + ky * ky + kz * kz);
    double* bb = B + 6 * b;
    bb[0] = kx * inv; bb[1] = ky * inv; bb[2] = kz * inv;
    bb[3] = pv[0]; bb[4] = pv[1]; bb[5] = pv[2];
  }
  // the pose's transforms (input frame -> world, Angstrom): the root R(q/|q|)
  // and t, then bond by bond, parents first (depth by depth, the group's
  // lanes splitting the bonds of a depth): bond b's is its parent's composed
  // with the rotation by theta_b about b's axis through v
  const float* pose = a.poses + (size_t)a.K * (7 * (size_t)l + r0) + (size_t)p * (7 + n);
  const size_t stride = (size_t)kRsPoses * 12;
  double* Tg = T + 12 * grp;
  // The sines and cosines of all (pose, bond) pairs in one pass over the
  // warp's lanes, not inside the depth loop, where only a depth's bonds
  // keep lanes busy (measured on GB300: re-score 6.9 -> 6.5 ms; FP64 warp
  // instructions seem to cost about the same however few lanes are active).
  double* scg = SC + (size_t)grp * ncap * 2;
  for (int b = sub; b < n; b += kRsLanes) sincos((double)pose[7 + b], &scg[2 * b], &scg[2 * b + 1]);
  if (sub == 0) {
    const double qi = rsqrt((double)pose[3] * pose[3] + (double)pose[4] * pose[4] + (double)pose[5] * pose[5] +
                            (double)pose[6] * pose[6]);
    const double qw = pose[3] * qi, qx = pose[4] * qi, qy = pose[5] * qi, qz = pose[6] * qi;
    const double R[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                         2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                         2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
    double* Tr = Tg + (size_t)n * stride;
    for (int r = 0; r < 3; ++r) {
      Tr[4 * r] = R[3 * r];
      Tr[4 * r + 1] = R[3 * r + 1];
      Tr[4 * r + 2] = R[3 * r + 2];
      Tr[4 * r + 3] = (double)pose[r];
    }
  }
  __syncwarp();
  const int depths = n ? S.loff[LIGEN_MAX_ROT] : 0;
  for (int d = 0; d < depths; ++d) {
    for (int k = S.loff[d] + sub; k < S.loff[d + 1]; k += kRsLanes) {
      const int b = S.lord[k];
      const double* P = Tg + (size_t)S.par[b] * stride;
      const double* bb = B + 6 * b;
      const double kx = bb[0], ky = bb[1], kz = bb[2];
      const double sn = scg[2 * b], cs = scg[2 * b + 1];
      const double tc = 1.0 - cs;
      // c I + s [k]x + (1 - c) k k^T: the right-handed rotation about k
      const double Rb[9] = {tc * kx * kx + cs,      tc * kx * ky - sn * kz, tc * kx * kz + sn * ky,
                            tc * kx * ky + sn * kz, tc * ky * ky + cs,      tc * ky * kz - sn * kx,
                            tc * kx * kz - sn * ky, tc * ky * kz + sn * kx, tc * kz * kz + cs};
      double* Tb = Tg + (size_t)b * stride;
      for (int r = 0; r < 3; ++r) {
        const double p0r = P[4 * r], p1r = P[4 * r + 1], p2r = P[4 * r + 2];
        const double m0 = p0r * Rb[0] + p1r * Rb[3] + p2r * Rb[6];
        const double m1 = p0r * Rb[1] + p1r * Rb[4] + p2r * Rb[7];
        const double m2 = p0r * Rb[2] + p1r * Rb[5] + p2r * Rb[8];
        // v keeps its place: o_b = T_p(v) - M_b v
        const double tp = p0r * bb[3] + p1r * bb[4] + p2r * bb[5] + P[4 * r + 3];
        Tb[4 * r] = m0;
        Tb[4 * r + 1] = m1;
        Tb[4 * r + 2] = m2;
        Tb[4 * r + 3] = tp - (m0 * bb[3] + m1 * bb[4] + m2 * bb[5]);
      }
    }
    __syncwarp();
  }
  // the group's lanes split the atoms: owner's transform, FP64 trilinear value
  Tri64 tb;
  tb.ox = a.origin[0]; tb.oy = a.origin[1]; tb.oz = a.origin[2];
  tb.inv_h = 1.0 / a.h;
  tb.mx = a.nx - 1; tb.my = a.ny - 1; tb.mz = a.nz - 1;
  double Sg = 0.0;
  for (int i = sub; i < N; i += kRsLanes) {
    const double* M = Tg + (size_t)S.own[i] * stride;
    const double* y = Y + 3 * i;
    double x[3];
    for (int r = 0; r < 3; ++r) x[r] = M[4 * r] * y[0] + M[4 * r + 1] * y[1] + M[4 * r + 2] * y[2] + M[4 * r + 3];
    Sg -= trilinear64(a, tb, x[0], x[1], x[2], a.lig.type[a0 + i]);
  }
  Sg = group_sum_d(Sg);
  if (own && sub == 0) a.s64[gp] = Sg;
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
  const size_t smem =
      (size_t)kResWarps * rs_warp_bytes(a.max_atoms, a.max_rot, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
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
