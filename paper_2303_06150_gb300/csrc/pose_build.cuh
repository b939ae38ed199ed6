// Torsion rebuild of a pose by a group of W lanes (the scoring and gradient
// kernels): the centred input coordinates of ligand l are turned, bond by
// bond in index order, about each bond's current axis from its fixed
// endpoint u to its moving endpoint v (right-handed, Rodrigues), which is the
// pose definition of the docking output. The group's poses belong to one
// ligand, so every group of the warp runs the same bond loop in lockstep.
#pragma once

#include "internal.h"

namespace ligen {

// Per-bond values of the group's pose, bond b held by lane b % W (K bonds
// per lane, K W >= the bond limit): sin and cos of the torsion and the bond
// record, read by shuffle inside the bond loops, so each lane computes K
// sincosf instead of n and the loops carry no global load of their own.
template <int W>
struct GroupBonds {
  static_assert(W >= 1 && W <= 32 && (W & (W - 1)) == 0, "a power-of-two group width");
  static constexpr int K = (LIGEN_MAX_ROT + W - 1) / W;   // bonds per lane
  float s[K], c[K];
  unsigned rec[K];   // uchar4 bond records

  // theta: the pose's n torsions; r0: the ligand's first bond.
  __device__ __forceinline__ void load(const Packed& pk, int r0, int n, const float* theta, int sub) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      s[k] = 0.f;
      c[k] = 1.f;
      rec[k] = 0u;
      if (sub + k * W < n) {
        sincosf(theta[k * W + sub], &s[k], &c[k]);
        const uchar4 r = pk.binfo[r0 + k * W + sub];
        rec[k] = *reinterpret_cast<const unsigned*>(&r);
      }
    }
  }
  // This lane's entry for bond b (b is warp-uniform, so the select is too).
  template <typename T>
  __device__ __forceinline__ static T mine(const T (&v)[K], int b) {
    const int k = b / W;
    T x = v[0];
#pragma unroll
    for (int kk = 1; kk < K; ++kk)
      if (k == kk) x = v[kk];
    return x;
  }
  // All lanes of the warp call these with the same b.
  __device__ __forceinline__ uchar4 bond(int b) const {
    const unsigned w = __shfl_sync(0xffffffffu, mine(rec, b), b % W, W);
    return *reinterpret_cast<const uchar4*>(&w);
  }
  __device__ __forceinline__ void sincos(int b, float* sn, float* cs) const {
    *sn = __shfl_sync(0xffffffffu, mine(s, b), b % W, W);
    *cs = __shfl_sync(0xffffffffu, mine(c, b), b % W, W);
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
