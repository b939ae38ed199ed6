// Torsion rebuild of a pose by a group of W lanes (the scoring and gradient
// kernels): the centred input coordinates of ligand l are turned, bond by
// bond in index order, about each bond's current axis from its fixed
// endpoint u to its moving endpoint v (right-handed, Rodrigues), which is the
// pose definition of the docking output. The group's poses belong to one
// ligand, so every group of the warp runs the same bond loop in lockstep.
#pragma once

#include "internal.h"

namespace ligen {

// Per-bond values of the group's pose, bond b held by lane b % W (two bonds
// per lane, so at most 2 W bonds): sin and cos of the torsion and the bond
// record, read by shuffle inside the bond loops, so each lane computes two
// sincosf instead of n and the loops carry no global load of their own.
template <int W>
struct GroupBonds {
  static_assert(W >= 1 && W <= 32 && (W & (W - 1)) == 0, "a power-of-two group width");
  static_assert(LIGEN_MAX_ROT <= 2 * W, "two torsions per lane");
  float s_lo = 0.f, c_lo = 1.f, s_hi = 0.f, c_hi = 1.f;
  uchar4 b_lo = make_uchar4(0, 0, 0, 0), b_hi = make_uchar4(0, 0, 0, 0);

  // theta: the pose's n torsions; r0: the ligand's first bond.
  __device__ __forceinline__ void load(const Packed& pk, int r0, int n, const float* theta, int sub) {
    if (sub < n) {
      sincosf(theta[sub], &s_lo, &c_lo);
      b_lo = pk.binfo[r0 + sub];
    }
    if (sub + W < n) {
      sincosf(theta[W + sub], &s_hi, &c_hi);
      b_hi = pk.binfo[r0 + W + sub];
    }
  }
  // All lanes of the warp call these with the same b.
  __device__ __forceinline__ uchar4 bond(int b) const {
    const uchar4 mine = b < W ? b_lo : b_hi;
    const unsigned w = __shfl_sync(0xffffffffu, *reinterpret_cast<const unsigned*>(&mine), b % W, W);
    return *reinterpret_cast<const uchar4*>(&w);
  }
  __device__ __forceinline__ void sincos(int b, float* s, float* c) const {
    *s = __shfl_sync(0xffffffffu, b < W ? s_lo : s_hi, b % W, W);
    *c = __shfl_sync(0xffffffffu, b < W ? c_lo : c_hi, b % W, W);
  }
};

// y[0..N): the ligand's centred input coordinates (w = type), turned in
// place into the pose's body coordinates. Called by all lanes of the warp;
// lane `sub` of the group moves moving atoms sub, sub + W, ... of each bond.
template <int W>
__device__ __forceinline__ void group_torsions(const Packed& pk, int r0, int n, int N, const GroupBonds<W>& B,
                                               float4* y, unsigned* check, int sub) {
  for (int b = 0; b < n; ++b) {   // b is uniform over the warp (one ligand)
    float s, c;
    B.sincos(b, &s, &c);
    const uchar4 bi = B.bond(b);
    if (!lg_check(check, bi.x < N && bi.y < N && bi.z < N, kChkAtomIndex)) continue;
    const float4 pv = y[bi.y], pu = y[bi.x];
    float kx = pv.x - pu.x, ky = pv.y - pu.y, kz = pv.z - pu.z;
    const float kn = rsqrtf(kx * kx + ky * ky + kz * kz);
    kx *= kn; ky *= kn; kz *= kn;
    const uint8_t* fr = pk.frag + (size_t)(r0 + b) * kFragStride;
    for (int t = sub; t < bi.z; t += W) {
      const int i = fr[t];
      if (!lg_check(check, i < N, kChkAtomIndex)) continue;
      float4 v = y[i];
      const float dx = v.x - pv.x, dy = v.y - pv.y, dz = v.z - pv.z;
      const float kd = kx * dx + ky * dy + kz * dz;
      const float ex = dx - kx * kd, ey = dy - ky * kd, ez = dz - kz * kd;
      const float qx = ky * dz - kz * dy, qy = kz * dx - kx * dz, qz = kx * dy - ky * dx;
      v.x = pv.x + kx * kd + ex * c + qx * s;
      v.y = pv.y + ky * kd + ey * c + qy * s;
      v.z = pv.z + kz * kd + ez * c + qz * s;
      y[i] = v;
    }
    __syncwarp();
  }
}

}  // namespace ligen
