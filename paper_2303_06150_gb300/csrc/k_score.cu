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
// (ligand, 32 poses), lane p scoring pose p on its own, with the torsions
// applied as forward kinematics instead of atom by atom.
//
// Moving sides are nested or disjoint, so the pose definition (bond by bond
// in index order, each about its current axis) equals, in exact
// arithmetic, a chain of rigid transforms: the transform of bond b is its
// parent's transform (the smallest moving side that strictly contains b's)
// composed with the rotation by theta_b about b's axis in the input
// conformation. An atom's position is then the transform of its owner (the
// smallest moving side holding it; the ligand's root frame when no torsion
// moves it) applied to its input coordinates. Every transform here also
// carries the pose's rotation R(q/|q|), its translation and the change to
// grid units, so an atom costs one 3x4 transform (9 FMA) and one sample.
//
// Per ligand, the warp stages in shared memory with coalesced loads: the
// centred input coordinates, the bond records and moving-atom lists; then
// works out each atom's owner, each bond's parent (the owner of its moving
// endpoint v, which no other bond's list holds), the order of the bonds
// (larger moving side first, so a parent comes before its children) and the
// bond axes. Per lane: the n + 1 transforms, 48 bytes each, in shared memory
// [slot][lane][12] (a 48-byte lane stride keeps 128-bit accesses free of
// bank conflicts). Shared memory thus grows with the bonds, and the caller
// launches ligands by rotatable-bond class. Lanes past the ligand's last
// pose shadow it and write nothing.
struct FkSmem {
  float* T;       // [ncap + 1][32][12] per-lane transforms (rows of M, then o)
  float4* sx;     // [acap] centred input coordinates (w = type)
  float4* ax;     // [ncap] unit bond axes in the input conformation
  uchar4* sb;     // [ncap] bond records (u, v, list length)
  uint8_t* sf;    // [ncap][fstride] moving-atom lists (moving side without v)
  uint8_t* own;   // [acap] owner of each atom (a bond, or ncap for the root)
  uint8_t* par;   // [ncap] parent of each bond (a bond, or the root)
  uint8_t* ord;   // [ncap] bonds, larger moving side first
  int fstride;
};

// A moving side has at most N/2 atoms (the smaller side of the cut), so a
// list of a ligand of at most `acap` atoms fits the first acap/2 bytes of its
// kFragStride-byte slot, rounded to a whole 16-byte vector.
__host__ __device__ inline int lane_fstride(int acap) {
  const int s = ((acap / 2 + 15) / 16) * 16;
  return s < 16 ? 16 : (s > kFragStride ? kFragStride : s);
}

__host__ __device__ inline size_t fk_carve(int acap, int ncap, unsigned char* base, FkSmem* S) {
  const int fs = lane_fstride(acap);
  const int n4 = (ncap + 15) / 16 * 16;
  const int a16 = (acap + 15) / 16 * 16;
  size_t o = 0;
  const size_t oT = o;   o += (size_t)(ncap + 1) * 32 * 12 * sizeof(float);
  const size_t osx = o;  o += (size_t)acap * sizeof(float4);
  const size_t oax = o;  o += (size_t)ncap * sizeof(float4);
  const size_t osb = o;  o += (size_t)n4 * sizeof(uchar4);
  const size_t osf = o;  o += (size_t)ncap * fs;
  const size_t oown = o; o += (size_t)a16;
  const size_t opar = o; o += (size_t)n4;
  const size_t oord = o; o += (size_t)n4;
  if (S) {
    S->T = (float*)(base + oT);
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

__device__ __forceinline__ void fk_store(float* T, int slot, int lane, const float* m, const float* o) {
  float4* d = reinterpret_cast<float4*>(T + ((size_t)slot * 32 + lane) * 12);
  d[0] = make_float4(m[0], m[1], m[2], o[0]);
  d[1] = make_float4(m[3], m[4], m[5], o[1]);
  d[2] = make_float4(m[6], m[7], m[8], o[2]);
}

// rows (m0 m1 m2 | o0), (m3 m4 m5 | o1), (m6 m7 m8 | o2)
__device__ __forceinline__ void fk_load(const float* T, int slot, int lane, float4& r0, float4& r1, float4& r2) {
  const float4* d = reinterpret_cast<const float4*>(T + ((size_t)slot * 32 + lane) * 12);
  r0 = d[0];
  r1 = d[1];
  r2 = d[2];
}

__global__ void __launch_bounds__(32, 16) score_lane_kernel(const ScoreArgs a) {
  extern __shared__ __align__(16) unsigned char lane_smem[];
  const int acap = a.max_atoms, ncap = a.max_rot;
  FkSmem S;
  fk_carve(acap, ncap, lane_smem, &S);
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
  if (!lg_check(a.grid.check, N <= acap && n <= ncap, kChkItemShape)) {
    if (own) a.out_scores[gp] = -INFINITY;
    return;
  }
  // ---- stage the ligand (coalesced, all lanes)
  for (int i = lane; i < N; i += 32) {
    S.sx[i] = a.pk.xc[a0 + i];
    S.own[i] = (uint8_t)ncap;   // the root frame until a list claims the atom
  }
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
  // ---- owners: the bond with the shortest list holding the atom (lists of
  // nested moving sides have different lengths; lanes of one bond touch
  // distinct atoms, bonds go one after another)
  bool bad = false;
  for (int b = 0; b < n; ++b) {
    const int m = S.sb[b].z;
    bad |= m > S.fstride;
    for (int k = lane; k < m && k < S.fstride; k += 32) {
      const int i = S.sf[b * S.fstride + k];
      if (i >= N) { bad = true; continue; }
      const int o = S.own[i];
      if (o == ncap || m < S.sb[o].z) S.own[i] = (uint8_t)b;
    }
    __syncwarp();
  }
  // ---- per bond: parent (owner of v), order (longer list first), axis
  if (lane < n) {
    const uchar4 bi = S.sb[lane];
    bad |= bi.x >= N || bi.y >= N;
    const int u = bi.x < N ? bi.x : 0, v = bi.y < N ? bi.y : 0;
    const int po = S.own[v];
    S.par[lane] = (uint8_t)(po == ncap ? n : po);   // root slot = n below
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
  if (!lg_check(a.grid.check, !__any_sync(0xffffffffu, bad), kChkAtomIndex)) {
    if (own) a.out_scores[gp] = -INFINITY;
    return;
  }
  __syncwarp();
  // ---- per lane: the root transform (pose rotation and translation, in grid
  // units), then every bond's, parents first; the root sits in slot n
  {
    const Quat q = qnormalize({q4[0], q4[1], q4[2], q4[3]});
    float R[9], o[3];
    qmat(q, R);
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] *= a.inv_h;
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = (t[k] - a.origin[k]) * a.inv_h;
    fk_store(S.T, n, lane, R, o);
  }
  for (int r = 0; r < n; ++r) {
    const int b = S.ord[r];
    const int pb = S.par[b];
    float4 p0r, p1r, p2r;
    fk_load(S.T, pb, lane, p0r, p1r, p2r);
    const float Mp[9] = {p0r.x, p0r.y, p0r.z, p1r.x, p1r.y, p1r.z, p2r.x, p2r.y, p2r.z};
    const float op[3] = {p0r.w, p1r.w, p2r.w};
    float sn, cs;
    sincosf(pose[7 + b], &sn, &cs);
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
    fk_store(S.T, b, lane, Mb, ob);
  }
  // ---- samples: unconditional loads, 8 gathers in flight per lane
  float acc = 0.f;
#pragma unroll 8
  for (int i = 0; i < N; ++i) {
    const float4 X = S.sx[i];
    const int o = S.own[i];
    float4 m0, m1, m2;
    fk_load(S.T, o == ncap ? n : o, lane, m0, m1, m2);
    const float ux = fmaf(m0.x, X.x, fmaf(m0.y, X.y, fmaf(m0.z, X.z, m0.w)));
    const float uy = fmaf(m1.x, X.x, fmaf(m1.y, X.y, fmaf(m1.z, X.z, m1.w)));
    const float uz = fmaf(m2.x, X.x, fmaf(m2.y, X.y, fmaf(m2.z, X.z, m2.w)));
    acc -= grid_sample_nb(a.grid, ux, uy, uz, __float_as_int(X.w));
  }
  if (own) a.out_scores[gp] = acc;
}

}  // namespace

size_t score_lane_smem_bytes(int acap, int ncap) { return fk_carve(acap, ncap, nullptr, nullptr); }

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
