// Device building blocks shared by the docking kernels: the restart random
// stream, quaternion algebra, the cube rotation table and the grid sampler.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace ligen {

// ------------------------------------------------------------------ RNG --
// SplitMix64 (Steele, Lea, Flood 2014): first output of a generator whose
// state is x.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Uniform k of restart r of ligand l: 24 high bits of
// SplitMix64(seed ^ ((l * 2^32 + r) * 8 + k)) scaled by 2^-24; exact in FP32.
__device__ __forceinline__ float restart_uniform(uint64_t seed, uint32_t lig, uint32_t r, uint32_t k) {
  uint64_t c = ((((uint64_t)lig << 32) + (uint64_t)r) << 3) + k;
  return (float)(uint32_t)(splitmix64(seed ^ c) >> 40) * (1.0f / 16777216.0f);
}

// ------------------------------------------------------------ rotations --
struct Quat {
  float w, x, y, z;
};

__device__ __forceinline__ Quat qmul(Quat a, Quat b) {
  return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
          a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
          a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
          a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}

__device__ __forceinline__ Quat qnormalize(Quat q) {
  float s = rsqrtf(q.w * q.w + q.x * q.x + q.y * q.y + q.z * q.z);
  return {q.w * s, q.x * s, q.y * s, q.z * s};
}

// Row-major rotation matrix of a unit quaternion.
__device__ __forceinline__ void qmat(Quat q, float* m) {
  float w = q.w, x = q.x, y = q.y, z = q.z;
  m[0] = 1.f - 2.f * (y * y + z * z); m[1] = 2.f * (x * y - w * z);       m[2] = 2.f * (x * z + w * y);
  m[3] = 2.f * (x * y + w * z);       m[4] = 1.f - 2.f * (x * x + z * z); m[5] = 2.f * (y * z - w * x);
  m[6] = 2.f * (x * z - w * y);       m[7] = 2.f * (y * z + w * x);       m[8] = 1.f - 2.f * (x * x + y * y);
}

// Shoemake (1992) uniform rotation from three uniforms:
// (sqrt(u0) cos 2pi u2, sqrt(1-u0) sin 2pi u1, sqrt(1-u0) cos 2pi u1, sqrt(u0) sin 2pi u2).
__device__ __forceinline__ Quat shoemake(float u0, float u1, float u2) {
  float r1 = sqrtf(1.0f - u0), r2 = sqrtf(u0);
  float s1, c1, s2, c2;
  sincospif(2.0f * u1, &s1, &c1);
  sincospif(2.0f * u2, &s2, &c2);
  return {r2 * c2, r1 * s1, r1 * c1, r2 * s2};
}

// The 24 proper rotations of the cube as unit quaternions (w, x, y, z):
//  0 identity; 1-3 half turns about x, y, z; 4-9 quarter turns +x, -x, +y,
//  -y, +z, -z; 10-17 third turns (120 deg) about the body diagonal
//  (sx, sy, sz) with m = k - 10 and s = -1 where bit 2 (x), 1 (y), 0 (z) of m
//  is set; 18-23 half turns about the face diagonals (1,1,0), (1,-1,0),
//  (0,1,1), (0,1,-1), (1,0,1), (1,0,-1).
#define LIGEN_H_ 0.5f
#define LIGEN_S_ 0.70710678118654752f
static __constant__ float kCubeQuat[24][4] = {
    {1, 0, 0, 0},
    {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1},
    {LIGEN_S_, LIGEN_S_, 0, 0}, {LIGEN_S_, -LIGEN_S_, 0, 0},
    {LIGEN_S_, 0, LIGEN_S_, 0}, {LIGEN_S_, 0, -LIGEN_S_, 0},
    {LIGEN_S_, 0, 0, LIGEN_S_}, {LIGEN_S_, 0, 0, -LIGEN_S_},
    {LIGEN_H_, LIGEN_H_, LIGEN_H_, LIGEN_H_}, {LIGEN_H_, LIGEN_H_, LIGEN_H_, -LIGEN_H_},
    {LIGEN_H_, LIGEN_H_, -LIGEN_H_, LIGEN_H_}, {LIGEN_H_, LIGEN_H_, -LIGEN_H_, -LIGEN_H_},
    {LIGEN_H_, -LIGEN_H_, LIGEN_H_, LIGEN_H_}, {LIGEN_H_, -LIGEN_H_, LIGEN_H_, -LIGEN_H_},
    {LIGEN_H_, -LIGEN_H_, -LIGEN_H_, LIGEN_H_}, {LIGEN_H_, -LIGEN_H_, -LIGEN_H_, -LIGEN_H_},
    {0, LIGEN_S_, LIGEN_S_, 0}, {0, LIGEN_S_, -LIGEN_S_, 0},
    {0, 0, LIGEN_S_, LIGEN_S_}, {0, 0, LIGEN_S_, -LIGEN_S_},
    {0, LIGEN_S_, 0, LIGEN_S_}, {0, LIGEN_S_, 0, -LIGEN_S_},
};
#undef LIGEN_H_
#undef LIGEN_S_

__device__ __forceinline__ Quat cube_quat(int k) {
  return {kCubeQuat[k][0], kCubeQuat[k][1], kCubeQuat[k][2], kCubeQuat[k][3]};
}

// Matrix of cube rotation k, exact: its entries are 0 or +-1, so the FP32
// matrix of the (rounded) quaternion is rounded to the nearest integer.
__device__ __forceinline__ void cube_mat(int k, float* g) {
  float m[9];
  qmat(cube_quat(k), m);
#pragma unroll
  for (int i = 0; i < 9; ++i) g[i] = rintf(m[i]);
}

// c = a * b for row-major 3x3 matrices.
__device__ __forceinline__ void mat3mul(const float* a, const float* b, float* c) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int col = 0; col < 3; ++col)
      c[3 * r + col] = a[3 * r] * b[col] + a[3 * r + 1] * b[3 + col] + a[3 * r + 2] * b[6 + col];
}

// Torsion increment j of a step of `step_deg` degrees: (cos, sin) of
// j * step_deg degrees. Every kernel uses this one definition, so the
// rotation applied after a decision is the one that was scored.
__device__ __forceinline__ void torsion_cs(int j, int step_deg, float* c, float* s) {
  sincospif((float)(j * step_deg) * (1.0f / 180.0f), s, c);
}

// Rotation of point x by the angle with cosine c and sine s about the line
// through v with unit direction k (right-handed): the component along k
// stays, the perpendicular part turns. Same arithmetic as the docking
// kernel's sweep.
__device__ __forceinline__ void rodrigues_apply(float* x, const float* v, const float* k, float c, float s) {
  const float dx = x[0] - v[0], dy = x[1] - v[1], dz = x[2] - v[2];
  const float kd = k[0] * dx + k[1] * dy + k[2] * dz;
  const float px = fmaf(k[0], kd, v[0]), py = fmaf(k[1], kd, v[1]), pz = fmaf(k[2], kd, v[2]);
  const float ex = fmaf(-k[0], kd, dx), ey = fmaf(-k[1], kd, dy), ez = fmaf(-k[2], kd, dz);
  const float qx = k[1] * dz - k[2] * dy, qy = k[2] * dx - k[0] * dz, qz = k[0] * dy - k[1] * dx;
  x[0] = fmaf(ex, c, fmaf(qx, s, px));
  x[1] = fmaf(ey, c, fmaf(qy, s, py));
  x[2] = fmaf(ez, c, fmaf(qz, s, pz));
}

// --------------------------------------------------------------- sampler --
// The grid is stored per cell and channel as the 8 coefficients of its
// trilinear polynomial, E(f) = a0 + ax fx + ay fy + az fz + axy fx fy +
// axz fx fz + ayz fy fz + axyz fx fy fz with f the position inside the cell.
// One 32-byte record per (cell, channel) makes one sample one aligned 32-byte
// load (one L2 sector) instead of eight scattered corner loads.
//
// Records are channel-major, [c][iz][iy][ix][8]. With the channel innermost
// instead, all lanes sampling atoms of one type would hit the same 32-byte
// position inside their 128-byte lines: measured on GB300, such 256-bit
// gathers run at two thirds of the rate of gathers at mixed positions (the
// L1 data banks serve one position per cycle). Channel-major puts the
// position at ix mod 4, which varies from lane to lane.
struct GridView {
  const float* coef;   // records at rec_index, 256-byte aligned
  int cx, cy, cz;      // record cells per axis (rec_cells of the format)
  int nc;
  float mx, my, mz;    // points - 1 per axis, as float: upper box bound in grid units
  float penalty;
  size_t n_rec;        // records in the buffer (checked builds compare with it)
  unsigned* check;     // checked builds: first out-of-range code, else NULL
};

// Checked builds (compiled with -DLIGEN_CHECKED=1): every data-dependent
// index is compared with its bound before use; a violation stores its code
// in *check (the first one wins) and the access is skipped, so the kernel
// carries on without touching memory out of range. Other builds compile the
// checks away.
#ifndef LIGEN_CHECKED
#define LIGEN_CHECKED 0
#endif
enum CheckCode : unsigned {
  kChkGridRecord = 1,   // grid record index or channel out of range
  kChkRescoreNode = 2,  // FP64 re-score: lattice node out of range
  kChkItemShape = 3,    // a ligand larger than the launch's shared-memory carve-up
  kChkAtomIndex = 4,    // a bond endpoint or moving-atom index >= the ligand's atoms
};
__device__ __forceinline__ bool lg_check(unsigned* check, bool ok, unsigned code) {
  if constexpr (LIGEN_CHECKED) {
    if (!ok && check) atomicCAS(check, 0u, code);
    return ok;
  }
  return true;
}

// Index (in records) of the record of channel c, cell (ix, iy, iz); the
// grid preparation writes records at the same indices.
__host__ __device__ __forceinline__ size_t rec_index(int cx, int cy, int cz, int c, int ix, int iy, int iz) {
  return (size_t)c * cz * cy * cx + (size_t)((iz * cy + iy) * cx + ix);
}
// Records to allocate for a grid of cx * cy * cz cells and nc channels.
__host__ __device__ __forceinline__ size_t rec_count(int cx, int cy, int cz, int nc) {
  return (size_t)cx * cy * cz * nc;
}

// Packed FP32 pairs (sm_100 family: fma.rn.f32x2, sub.rn.f32x2): one
// instruction for two independent operations, each element rounded exactly
// as the scalar operation, so results are bit-identical to scalar code.
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {   // a * b + c
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)), "l"(pk2(c.x, c.y)));
  return upk2(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {   // a - b
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)));
  return upk2(d);
}

// 256-bit read-only load (sm_100+): one 32-byte record in one instruction,
// not volatile (no side effect, so the compiler may batch it), and without
// allocating the line in L1 (L1::no_allocate): the samplers' 32-byte
// records are rarely read twice from L1 (~3% hits), and not allocating them
// keeps L1 for the kernels' other data. Measured on
// GB300 (8,000 screening ligands): FP32 docking 18.97 -> 18.35 ms, gradient
// refinement of their top 16 poses 9.27 -> 8.52 ms. The same hint on the
// 16-byte records made FP16 docking 1.2% slower, so they keep the default.
__device__ __forceinline__ void ld_global_v8_na(const float* p, float (&v)[8]) {
  asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
                 "=f"(v[7])
               : "l"(p));
}

// Energy of channel `c` at grid-unit position u (u = (x - origin) / spacing).
// Inside iff 0 <= u <= n - 1 on every axis; cell i = min(floor(u), n - 2),
// f = u - i. Outside: the penalty.
__device__ __forceinline__ float grid_sample(const GridView& g, float ux, float uy, float uz, int c) {
  bool inb = (ux >= 0.f) & (ux <= g.mx) & (uy >= 0.f) & (uy <= g.my) & (uz >= 0.f) & (uz <= g.mz);
  float e = g.penalty;
  if (inb) {
    float fx = fminf(floorf(ux), g.mx - 1.f);
    float fy = fminf(floorf(uy), g.my - 1.f);
    float fz = fminf(floorf(uz), g.mz - 1.f);
    int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    float dx = ux - fx, dy = uy - fy, dz = uz - fz;
    const size_t ri = rec_index(g.cx, g.cy, g.cz, c, ix, iy, iz);
    if (!lg_check(g.check, c >= 0 && c < g.nc && ri < g.n_rec, kChkGridRecord)) return g.penalty;
    const float* rec = g.coef + ri * 8;
    float a[8];
    ld_global_v8_na(rec, a);
    float t1 = fmaf(dz, a[7], a[4]);
    float t2 = fmaf(dy, t1, a[1]);
    t2 = fmaf(dz, a[5], t2);
    float t3 = fmaf(dz, a[6], a[2]);
    e = fmaf(dz, a[3], a[0]);
    e = fmaf(dy, t3, e);
    e = fmaf(dx, t2, e);
  }
  return e;
}

// Grid record formats of the docking kernel.
//   kRecF32:  32-byte records, the 8 FP32 coefficients of the cell's
//             trilinear polynomial (one 256-bit load, 7 FMA);
//   kRecF16, kRecBF16: 16-byte records, the 8 corner values of the cell in
//             FP16 or BF16 (one 128-bit load, FP32 interpolation).
// Records are channel-major in every format.
enum RecFormat { kRecF32 = 0, kRecF16 = 1, kRecBF16 = 2 };

__host__ __device__ constexpr int rec_bytes(int fmt) { return fmt == kRecF32 ? 32 : 16; }

// Extra record layers past the lattice's last node, 16-bit formats.
constexpr int kRecPad16 = 0;

// Cells per axis of the record grid of a lattice with n points per axis.
// FP32 coefficient records cover its n - 1 cells; the sampler clamps the
// cell index so that a point on an upper face (u = n - 1) uses the last cell
// at f = 1. The 16-bit corner records add one layer on each upper face (its
// corners repeat the face's node values, plus kRecPad16 spare layers), so
// their sampler needs no clamp: a point on an upper face samples that layer
// at f = 0 and gets the node value exactly. Measured on GB300: the padded,
// clamp-free FP16 sampler is 2.5% faster; the same padding made FP32 records
// 5.7% slower, so FP32 keeps n - 1 cells.
__host__ __device__ constexpr int rec_cells(int n, int fmt) { return fmt == kRecF32 ? n - 1 : n + kRecPad16; }

template <int FMT>
__device__ __forceinline__ float2 unpack2(unsigned int w) {
  if constexpr (FMT == kRecF16) {
    __half2 h = *reinterpret_cast<__half2*>(&w);
    return __half22float2(h);
  } else {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
    return __bfloat1622float2(h);
  }
}

// grid_sample for any record format (see RecFormat).
template <int FMT>
__device__ __forceinline__ float grid_sample_fmt(const GridView& g, float ux, float uy, float uz, int c) {
  if constexpr (FMT == kRecF32) {
    return grid_sample(g, ux, uy, uz, c);
  } else {
    bool inb = (ux >= 0.f) & (ux <= g.mx) & (uy >= 0.f) & (uy <= g.my) & (uz >= 0.f) & (uz <= g.mz);
    float e = g.penalty;
    if (inb) {
      float fx = floorf(ux);   // <= n - 1: the padding layer holds the upper faces
      float fy = floorf(uy);
      float fz = floorf(uz);
      int ix = (int)fx, iy = (int)fy, iz = (int)fz;
      float dx = ux - fx, dy = uy - fy, dz = uz - fz;
      const size_t ri = rec_index(g.cx, g.cy, g.cz, c, ix, iy, iz);
      if (!lg_check(g.check, c >= 0 && c < g.nc && ri < g.n_rec, kChkGridRecord)) return g.penalty;
      const uint4* rec = reinterpret_cast<const uint4*>(g.coef) + ri;
      const uint4 v = __ldg(rec);
      const float2 a = unpack2<FMT>(v.x), b = unpack2<FMT>(v.y);   // (c000, c100), (c010, c110)
      const float2 d = unpack2<FMT>(v.z), f = unpack2<FMT>(v.w);   // (c001, c101), (c011, c111)
      // 7 lerps v0 + d (v1 - v0), x-lerps and y-lerps in packed pairs
      // (measured: 1.5% faster FP16 docking; the FP32 sampler lost 1% the same way)
      const float2 dxx = make_float2(dx, dx);
      const float2 p0 = make_float2(a.x, b.x), q0 = make_float2(a.y, b.y);   // (c000, c010), (c100, c110)
      const float2 p1 = make_float2(d.x, f.x), q1 = make_float2(d.y, f.y);   // (c001, c011), (c101, c111)
      const float2 x0 = fma2(dxx, sub2(q0, p0), p0);                         // (x00, x10)
      const float2 x1 = fma2(dxx, sub2(q1, p1), p1);                         // (x01, x11)
      const float2 lo = make_float2(x0.x, x1.x), hi = make_float2(x0.y, x1.y);
      const float2 y = fma2(make_float2(dy, dy), sub2(hi, lo), lo);          // (y0, y1)
      e = fmaf(dz, y.y - y.x, y.x);
    }
    return e;
  }
}

// 16-bit record samplers with the channel's record base computed by the
// caller (chan_base16, once per atom): a sample then forms its address from
// a 32-bit in-channel cell index with one wide multiply-add instead of a
// 64-bit record index. Same records, same arithmetic, same results as
// grid_sample_fmt. Measured on GB300 (screen20k docking kernel): FP16
// 45.65 -> 45.11 ms, BF16 47.13 -> 46.06 ms. The same change to the FP32
// sampler made it 1.5% slower (more spills in the 8-CTA build), so FP32
// records keep grid_sample.
__device__ __forceinline__ const unsigned char* chan_base16(const GridView& g, int c) {
  return reinterpret_cast<const unsigned char*>(g.coef) + (size_t)c * g.cz * g.cy * g.cx * 16;
}

template <int FMT>
__device__ __forceinline__ float grid_sample16_cb(const GridView& g, const unsigned char* cb, float ux, float uy,
                                                  float uz, int c) {
  static_assert(FMT != kRecF32, "16-bit records only");
  const bool inb = (ux >= 0.f) & (ux <= g.mx) & (uy >= 0.f) & (uy <= g.my) & (uz >= 0.f) & (uz <= g.mz);
  float e = g.penalty;
  if (inb) {
    const float fx = floorf(ux), fy = floorf(uy), fz = floorf(uz);   // the padding layer holds the upper faces
    const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    const float dx = ux - fx, dy = uy - fy, dz = uz - fz;
    const unsigned li = (unsigned)((iz * g.cy + iy) * g.cx + ix);
    if constexpr (LIGEN_CHECKED) {
      const size_t ri = rec_index(g.cx, g.cy, g.cz, c, ix, iy, iz);
      if (!lg_check(g.check, c >= 0 && c < g.nc && ri < g.n_rec, kChkGridRecord)) return g.penalty;
    }
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(cb) + li);
    const float2 a = unpack2<FMT>(v.x), b = unpack2<FMT>(v.y);   // (c000, c100), (c010, c110)
    const float2 d = unpack2<FMT>(v.z), f = unpack2<FMT>(v.w);   // (c001, c101), (c011, c111)
    const float2 dxx = make_float2(dx, dx);
    const float2 p0 = make_float2(a.x, b.x), q0 = make_float2(a.y, b.y);
    const float2 p1 = make_float2(d.x, f.x), q1 = make_float2(d.y, f.y);
    const float2 x0 = fma2(dxx, sub2(q0, p0), p0);
    const float2 x1 = fma2(dxx, sub2(q1, p1), p1);
    const float2 lo = make_float2(x0.x, x1.x), hi = make_float2(x0.y, x1.y);
    const float2 y = fma2(make_float2(dy, dy), sub2(hi, lo), lo);
    e = fmaf(dz, y.y - y.x, y.x);
  }
  return e;
}

// Value and gradient (per grid unit) of channel `c` at grid-unit position u:
// the derivative of the cell's trilinear polynomial, zero outside the box.
__device__ __forceinline__ float grid_sample_grad(const GridView& g, float ux, float uy, float uz, int c,
                                                  float* gx, float* gy, float* gz) {
  bool inb = (ux >= 0.f) & (ux <= g.mx) & (uy >= 0.f) & (uy <= g.my) & (uz >= 0.f) & (uz <= g.mz);
  float e = g.penalty;
  *gx = *gy = *gz = 0.f;
  if (inb) {
    float fx = fminf(floorf(ux), g.mx - 1.f);
    float fy = fminf(floorf(uy), g.my - 1.f);
    float fz = fminf(floorf(uz), g.mz - 1.f);
    int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    float dx = ux - fx, dy = uy - fy, dz = uz - fz;
    const size_t ri = rec_index(g.cx, g.cy, g.cz, c, ix, iy, iz);
    if (!lg_check(g.check, c >= 0 && c < g.nc && ri < g.n_rec, kChkGridRecord)) return g.penalty;
    const float* rec = g.coef + ri * 8;
    float a[8];
    ld_global_v8_na(rec, a);
    float t1 = fmaf(dz, a[7], a[4]);
    float t2 = fmaf(dy, t1, a[1]);
    t2 = fmaf(dz, a[5], t2);
    float t3 = fmaf(dz, a[6], a[2]);
    e = fmaf(dz, a[3], a[0]);
    e = fmaf(dy, t3, e);
    e = fmaf(dx, t2, e);
    *gx = t2;                                              // ax + axy fy + axz fz + axyz fy fz
    *gy = fmaf(dx, t1, t3);                                // ay + axy fx + ayz fz + axyz fx fz
    *gz = fmaf(dx, fmaf(dy, a[7], a[5]), fmaf(dy, a[6], a[3]));  // az + axz fx + ayz fy + axyz fx fy
  }
  return e;
}

}  // namespace ligen
