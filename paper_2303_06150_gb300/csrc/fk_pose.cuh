// Forward kinematics of a pose, shared by the pose-per-lane scoring kernel
// and the pose-group gradient kernel.
//
// Moving sides of rotatable bonds are nested or disjoint, so the pose
// definition (torsions bond by bond in index order, each about its current
// axis, on the centred input coordinates; then R(q/|q|) and t) equals, in
// exact arithmetic, a chain of rigid transforms: bond b's transform is its
// parent's (the smallest moving side strictly containing b's) composed
// with the rotation by theta_b about b's axis in the input conformation, and
// an atom's position is its owner's transform (the smallest moving side
// holding it, or the ligand's root frame) applied to its input coordinates.
// The root frame carries the pose's rotation, translation and the change to
// grid units, so every transform maps input coordinates to grid units.
//
// fk_stage derives, per ligand, in shared memory: the centred input
// coordinates, the bond records and moving-atom lists (coalesced loads);
// each atom's owner; each bond's parent (the owner of its moving endpoint v,
// which no other bond's list holds); the bonds in decreasing moving-side
// size (a parent before its children) and grouped by depth in the bond
// tree; the bond axes. fk_table_kernel runs it once per ligand and writes
// the result out, with the atoms listed by owner; the scoring and gradient
// kernels stage it with fk_load (vector copies). Transforms are 12 floats:
// three rows (m0 m1 m2 | o).
#pragma once

#include "internal.h"

namespace ligen {

struct FkLigand {
  float4* sx;     // [acap] centred input coordinates (w = type)
  float4* ax;     // [ncap] unit bond axes in the input conformation
  uchar4* sb;     // [ncap] bond records (u, v, list length)
  uint8_t* sf;    // [ncap][fstride] moving-atom lists (moving side without v)
  uint8_t* own;   // [acap] owner of each atom: a bond, or the root slot n after fk_stage
  uint8_t* par;   // [ncap] parent of each bond: a bond, or the root slot n
  uint8_t* ord;   // [ncap] bonds, larger moving side first
  uint8_t* lord;  // [ncap] bonds by depth in the bond tree (root's children first)
  uint8_t* loff;  // [48] first entry of each depth in lord (loff[depths] = n);
                  // loff[LIGEN_MAX_ROT] = the number of depths; loff[kFkBad]: see fk_load
  int fstride;
};

// A moving side has at most N/2 atoms (the smaller side of the cut), so a
// list of a ligand of at most `acap` atoms fits the first acap/2 bytes of its
// kFragStride-byte slot, rounded to a whole 16-byte vector.
__host__ __device__ inline int fk_fstride(int acap) {
  const int s = ((acap / 2 + 15) / 16) * 16;
  return s < 16 ? 16 : (s > kFragStride ? kFragStride : s);
}

// Bytes of the staged ligand (16-byte multiple); carves it at `base` when S.
__host__ __device__ inline size_t fk_ligand_carve(int acap, int ncap, unsigned char* base, FkLigand* S) {
  const int fs = fk_fstride(acap);
  const int n16 = (ncap + 15) / 16 * 16;
  const int a16 = (acap + 15) / 16 * 16;
  size_t o = 0;
  const size_t osx = o;  o += (size_t)acap * sizeof(float4);
  const size_t oax = o;  o += (size_t)ncap * sizeof(float4);
  const size_t osb = o;  o += (size_t)n16 * sizeof(uchar4);
  const size_t osf = o;  o += (size_t)ncap * fs;
  const size_t oown = o; o += (size_t)a16;
  const size_t opar = o; o += (size_t)n16;
  const size_t oord = o; o += (size_t)n16;
  const size_t olord = o; o += (size_t)n16;
  const size_t oloff = o; o += 48;   // LIGEN_MAX_ROT + 1 entries (the last: the number of depths)
  if (S) {
    S->lord = base + olord;
    S->loff = base + oloff;
    S->sx = (float4*)(base + osx);
    S->ax = (float4*)(base + oax);
    S->sb = (uchar4*)(base + osb);
    S->sf = base + osf;
    S->own = base + oown;
    S->par = base + opar;
    S->ord = base + oord;
    S->fstride = fs;
  }
  return o;
}

// Stage ligand (a0, N, r0, n) for the warp (all 32 lanes call it); DEPTHS:
// also the bonds grouped by depth (lord, loff) for fk_transforms_group.
// Returns false, on every lane, when a bond endpoint or a moving atom is out
// of range (nothing out of range is written).
template <bool DEPTHS = false>
__device__ inline bool fk_stage(const Packed& pk, int a0, int N, int r0, int n, const FkLigand& S, int lane) {
  for (int i = lane; i < N; i += 32) {
    S.sx[i] = pk.xc[a0 + i];
    S.own[i] = (uint8_t)n;   // the root until a list claims the atom
  }
  for (int b = lane; b < n; b += 32) S.sb[b] = pk.binfo[r0 + b];
  {   // the first fstride bytes of every list (16-byte vectors)
    const int per = S.fstride / 16;
    const uint4* src = reinterpret_cast<const uint4*>(pk.frag + (size_t)r0 * kFragStride);
    uint4* dst = reinterpret_cast<uint4*>(S.sf);
    for (int v = lane; v < n * per; v += 32) dst[v] = src[(v / per) * (kFragStride / 16) + v % per];
  }
  __syncwarp();
  // owners: the bond with the shortest list holding the atom (lists of
  // nested moving sides have different lengths); the lanes of one bond
  // touch distinct atoms, bonds go one after another
  bool bad = false;
  for (int b = 0; b < n; ++b) {
    const int m = S.sb[b].z;
    bad |= m > S.fstride;
    for (int k = lane; k < m && k < S.fstride; k += 32) {
      const int i = S.sf[b * S.fstride + k];
      if (i >= N) { bad = true; continue; }
      const int o = S.own[i];
      if (o == n || m < S.sb[o].z) S.own[i] = (uint8_t)b;
    }
    __syncwarp();
  }
  if (lane < n) {   // parent (owner of v), order (longer list first), axis
    const uchar4 bi = S.sb[lane];
    bad |= bi.x >= N || bi.y >= N;
    const int u = bi.x < N ? bi.x : 0, v = bi.y < N ? bi.y : 0;
    S.par[lane] = S.own[v];
    int rank = 0;
    for (int b = 0; b < n; ++b) {
      const int mb = S.sb[b].z;
      rank += (mb > bi.z) || (mb == bi.z && b < lane);
    }
    S.ord[rank] = (uint8_t)lane;
    const float4 xv = S.sx[v], xu = S.sx[u];
    float kx = xv.x - xu.x, ky = xv.y - xu.y, kz = xv.z - xu.z;
    const float kn = rsqrtf(kx * kx + ky * ky + kz * kz);
    S.ax[lane] = make_float4(kx * kn, ky * kn, kz * kn, 0.f);
  }
  bad = __any_sync(0xffffffffu, bad);
  __syncwarp();
  if (DEPTHS && lane == 0 && !bad) {   // depths (parents first in ord), then bonds by depth
    uint8_t depth[LIGEN_MAX_ROT];
    int cnt[LIGEN_MAX_ROT + 1] = {};
    int dmax = -1;
    for (int r = 0; r < n; ++r) {
      const int b = S.ord[r], pb = S.par[b];
      depth[b] = (uint8_t)(pb == n ? 0 : depth[pb] + 1);
      ++cnt[depth[b]];
      dmax = depth[b] > dmax ? depth[b] : dmax;
    }
    int o = 0;
    for (int d = 0; d <= dmax; ++d) {
      S.loff[d] = (uint8_t)o;
      o += cnt[d];
    }
    S.loff[dmax + 1] = (uint8_t)n;
    for (int d = 0; d <= dmax; ++d) cnt[d] = S.loff[d];
    for (int r = 0; r < n; ++r) S.lord[cnt[depth[S.ord[r]]]++] = S.ord[r];
    S.loff[LIGEN_MAX_ROT] = (uint8_t)(dmax + 1);   // number of depths
  }
  __syncwarp();
  return !bad;
}

// Stage ligand l = (a0, N, r0, n) for the warp (all 32 lanes call it) from
// the forward-kinematics table (pk.fk_*, written by fk_table_kernel with
// fk_stage<true>): the contents fk_stage<true> builds, but for the
// moving-atom lists (nothing reads them after staging), with the atoms
// listed by owner (S.sx, S.own in the table's order) and S.sb[b].y the list
// position of bond b's v (S.sb[b].x unused). Vector copies, no per-bond
// passes. Returns false, on every lane, when the table marks the ligand's
// lists as malformed.
__device__ inline bool fk_load(const Packed& pk, int l, int a0, int N, int r0, int n, const FkLigand& S, int lane) {
  static_assert(kFkLoffBytes == 48 && kFkBad > LIGEN_MAX_ROT, "depth row of the table = the staged row");
  for (int i = lane; i < N; i += 32) {
    S.sx[i] = pk.fk_xs[a0 + i];
    S.own[i] = pk.fk_own[a0 + i];
  }
  for (int b = lane; b < n; b += 32) {
    const uchar4 bi = pk.binfo[r0 + b];
    const uchar4 t = pk.fk_bond[r0 + b];
    S.sb[b] = make_uchar4(0, t.w, bi.z, 0);
    S.ax[b] = pk.fk_ax[r0 + b];
    S.par[b] = t.x;
    S.ord[b] = t.y;
    S.lord[b] = t.z;
  }
  if (lane < kFkLoffBytes / 4)
    reinterpret_cast<uint32_t*>(S.loff)[lane] =
        reinterpret_cast<const uint32_t*>(pk.fk_loff + (size_t)l * kFkLoffBytes)[lane];
  __syncwarp();
  return S.loff[kFkBad] == 0;
}

__device__ __forceinline__ void fk_put(float* T, const float* m, const float* o) {
  float4* d = reinterpret_cast<float4*>(T);
  d[0] = make_float4(m[0], m[1], m[2], o[0]);
  d[1] = make_float4(m[3], m[4], m[5], o[1]);
  d[2] = make_float4(m[6], m[7], m[8], o[2]);
}

__device__ __forceinline__ void fk_get(const float* T, float4& r0, float4& r1, float4& r2) {
  const float4* d = reinterpret_cast<const float4*>(T);
  r0 = d[0];
  r1 = d[1];
  r2 = d[2];
}

// The n + 1 transforms of one pose: the root (slot n) from the translation
// t and the unit quaternion q (w, x, y, z), in grid units; then every bond,
// parents first, with the torsion angles theta[b * theta_stride], b = 0 ..
// n-1 (which may lie in slot b itself: it is read before the slot is
// written). Transform of slot s at T + s * slot_stride (16-byte aligned).
__device__ inline void fk_transforms(const FkLigand& S, int n, const float* t, Quat q, const float* theta,
                                     size_t theta_stride, const float* origin, float inv_h, float* T,
                                     size_t slot_stride) {
  {
    float R[9], o[3];
    qmat(q, R);
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] *= inv_h;
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = (t[k] - origin[k]) * inv_h;
    fk_put(T + (size_t)n * slot_stride, R, o);
  }
  for (int r = 0; r < n; ++r) {
    const int b = S.ord[r];
    float4 p0, p1, p2;
    fk_get(T + (size_t)S.par[b] * slot_stride, p0, p1, p2);
    const float Mp[9] = {p0.x, p0.y, p0.z, p1.x, p1.y, p1.z, p2.x, p2.y, p2.z};
    const float op[3] = {p0.w, p1.w, p2.w};
    float sn, cs;
    sincosf(theta[(size_t)b * theta_stride], &sn, &cs);
    const float4 k = S.ax[b];
    const float tc = 1.f - cs;
    // rotation by theta_b about k (right-handed): c I + s [k]x + (1 - c) k k^T
    const float Rb[9] = {fmaf(tc * k.x, k.x, cs),     fmaf(tc * k.x, k.y, -sn * k.z), fmaf(tc * k.x, k.z, sn * k.y),
                         fmaf(tc * k.x, k.y, sn * k.z), fmaf(tc * k.y, k.y, cs),     fmaf(tc * k.y, k.z, -sn * k.x),
                         fmaf(tc * k.x, k.z, -sn * k.y), fmaf(tc * k.y, k.z, sn * k.x), fmaf(tc * k.z, k.z, cs)};
    float Mb[9];
    mat3mul(Mp, Rb, Mb);
    // the axis point v keeps its place: o_b = T_p(x_v) - M_b x_v
    const float4 xv = S.sx[S.sb[b].y];
    float ob[3];
#pragma unroll
    for (int rr = 0; rr < 3; ++rr) {
      const float tp = fmaf(Mp[3 * rr], xv.x, fmaf(Mp[3 * rr + 1], xv.y, fmaf(Mp[3 * rr + 2], xv.z, op[rr])));
      ob[rr] = tp - fmaf(Mb[3 * rr], xv.x, fmaf(Mb[3 * rr + 1], xv.y, Mb[3 * rr + 2] * xv.z));
    }
    fk_put(T + (size_t)b * slot_stride, Mb, ob);
  }
}

// fk_transforms spread over a group of G lanes (sub = 0 .. G-1), all lanes
// of the warp calling it: the root by the group's first lane, then the
// bonds depth by depth (bonds of one depth are independent: a parent is one
// depth up), round-robin over the group. Same transforms, bit for bit.
template <int G>
__device__ inline void fk_transforms_group(const FkLigand& S, int n, const float* t, Quat q, const float* theta,
                                           const float* origin, float inv_h, float* T, size_t slot_stride,
                                           int sub) {
  if (sub == 0) {
    float R[9], o[3];
    qmat(q, R);
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] *= inv_h;
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = (t[k] - origin[k]) * inv_h;
    fk_put(T + (size_t)n * slot_stride, R, o);
  }
  __syncwarp();
  const int depths = n ? S.loff[LIGEN_MAX_ROT] : 0;
  for (int d = 0; d < depths; ++d) {
    for (int k = S.loff[d] + sub; k < S.loff[d + 1]; k += G) {
      const int b = S.lord[k];
      float4 p0, p1, p2;
      fk_get(T + (size_t)S.par[b] * slot_stride, p0, p1, p2);
      const float Mp[9] = {p0.x, p0.y, p0.z, p1.x, p1.y, p1.z, p2.x, p2.y, p2.z};
      const float op[3] = {p0.w, p1.w, p2.w};
      float sn, cs;
      sincosf(theta[b], &sn, &cs);
      const float4 k4 = S.ax[b];
      const float tc = 1.f - cs;
      const float Rb[9] = {fmaf(tc * k4.x, k4.x, cs),     fmaf(tc * k4.x, k4.y, -sn * k4.z),
                           fmaf(tc * k4.x, k4.z, sn * k4.y), fmaf(tc * k4.x, k4.y, sn * k4.z),
                           fmaf(tc * k4.y, k4.y, cs),     fmaf(tc * k4.y, k4.z, -sn * k4.x),
                           fmaf(tc * k4.x, k4.z, -sn * k4.y), fmaf(tc * k4.y, k4.z, sn * k4.x),
                           fmaf(tc * k4.z, k4.z, cs)};
      float Mb[9];
      mat3mul(Mp, Rb, Mb);
      const float4 xv = S.sx[S.sb[b].y];
      float ob[3];
#pragma unroll
      for (int rr = 0; rr < 3; ++rr) {
        const float tp = fmaf(Mp[3 * rr], xv.x, fmaf(Mp[3 * rr + 1], xv.y, fmaf(Mp[3 * rr + 2], xv.z, op[rr])));
        ob[rr] = tp - fmaf(Mb[3 * rr], xv.x, fmaf(Mb[3 * rr + 1], xv.y, Mb[3 * rr + 2] * xv.z));
      }
      fk_put(T + (size_t)b * slot_stride, Mb, ob);
    }
    __syncwarp();
  }
}

}  // namespace ligen
