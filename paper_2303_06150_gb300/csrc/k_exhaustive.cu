// Exhaustive search (mode 1, small ligands): for every restart, every
// combination of a cube rotation k and torsion increments (j_0 .. j_{n-1})
// is scored and the best kept, ties going to the combination that comes
// first in lexicographic order of (k, j_0, .., j_{n-1}). It is the brute
// force the greedy search is an approximation of: per restart, greedy <=
// exhaustive. The result is written in the greedy kernel's per-restart
// format (score, k, increments), so top-K, pose compaction and the FP64
// re-score follow unchanged.
//
// One CTA per (ligand, restart). Threads take combination indices
// c = ((k * nt + j_0) * nt + j_1) * nt + ... in a strided loop. Each pose is
// rebuilt from the input conformation: the torsions are applied bond by bond
// in index order, each about its axis as moved by the earlier bonds (the
// axis endpoints are rotated first, then every atom), then the cube rotation
// and the restart's orientation and translation.
#include "../../include/ligen.h"
#include "internal.h"

namespace ligen {
namespace {

constexpr int kExThreads = 128;

template <int FMT>
__global__ void __launch_bounds__(kExThreads) exhaustive_kernel(const DockArgs a) {
  __shared__ float4 sx[LIGEN_MAX_ATOMS];
  __shared__ uint32_t member[kExMaxRot][LIGEN_MAX_ATOMS / 32];
  __shared__ int saxis[kExMaxRot][2];
  __shared__ float red_s[kExThreads / 32];
  __shared__ long long red_c[kExThreads / 32];

  const int l = blockIdx.x / a.R, r = blockIdx.x % a.R;
  if (a.pk.status[l] != 0) return;   // uniform over the CTA
  const int tid = threadIdx.x;
  const int a0 = a.lig.atom_off[l];
  const int N = a.lig.atom_off[l + 1] - a0;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;   // <= kExMaxRot (checked on the host)
  if (!lg_check(a.grid.check, N <= LIGEN_MAX_ATOMS && n <= kExMaxRot, kChkItemShape)) return;   // uniform

  for (int i = tid; i < N; i += kExThreads) sx[i] = a.pk.xc[a0 + i];
  for (int w = tid; w < kExMaxRot * (LIGEN_MAX_ATOMS / 32); w += kExThreads) (&member[0][0])[w] = 0u;
  __syncthreads();
  for (int b = 0; b < n; ++b) {
    const uchar4 bi = a.pk.binfo[r0 + b];
    if (tid == 0) {
      saxis[b][0] = bi.x;
      saxis[b][1] = bi.y;
      lg_check(a.grid.check, bi.x < N && bi.y < N, kChkAtomIndex);
    }
    for (int t = tid; t < bi.z; t += kExThreads) {
      const int i = a.pk.frag[(size_t)(r0 + b) * kFragStride + t];
      if (!lg_check(a.grid.check, i < N, kChkAtomIndex)) continue;
      atomicOr(&member[b][i >> 5], 1u << (i & 31));
    }
  }
  __syncthreads();

  // restart orientation and translation, as in the greedy kernel
  float u[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) u[k] = restart_uniform(a.seed, (uint32_t)l, (uint32_t)r, (uint32_t)k);
  const Quat qr = qnormalize(shoemake(u[0], u[1], u[2]));
  float Rm[9], M[9];
  qmat(qr, Rm);
#pragma unroll
  for (int i = 0; i < 9; ++i) M[i] = Rm[i] * a.inv_h;
  float o[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float t = a.center[k] + (2.0f * u[3 + k] - 1.0f) * a.jitter;
    o[k] = (t - a.origin[k]) * a.inv_h;
  }

  const int nt = a.n_theta;
  long long per_k = 1;
  for (int b = 0; b < n; ++b) per_k *= nt;
  const long long total = per_k * a.n_rigid;

  float best = -INFINITY;
  long long bestc = 0x7fffffffffffffffll;
  for (long long c = tid; c < total; c += kExThreads) {
    long long rem = c;
    int j[kExMaxRot];
#pragma unroll
    for (int b = kExMaxRot - 1; b >= 0; --b) {
      j[b] = 0;
      if (b < n) { j[b] = (int)(rem % nt); rem /= nt; }
    }
    const int k = (int)rem;
    // axis of each bond after the earlier bonds: its moving end pv and unit direction kd
    float pv[kExMaxRot][3], kd[kExMaxRot][3], cs[kExMaxRot], sn[kExMaxRot];
#pragma unroll
    for (int b = 0; b < kExMaxRot; ++b) {
      if (b >= n) break;
      const int iu = saxis[b][0], iv = saxis[b][1];
      float pu[3] = {sx[iu].x, sx[iu].y, sx[iu].z};
      float pw[3] = {sx[iv].x, sx[iv].y, sx[iv].z};
#pragma unroll
      for (int e = 0; e < kExMaxRot; ++e) {
        if (e >= b) break;
        if (member[e][iu >> 5] >> (iu & 31) & 1u) rodrigues_apply(pu, pv[e], kd[e], cs[e], sn[e]);
        if (member[e][iv >> 5] >> (iv & 31) & 1u) rodrigues_apply(pw, pv[e], kd[e], cs[e], sn[e]);
      }
      const float d0 = pw[0] - pu[0], d1 = pw[1] - pu[1], d2 = pw[2] - pu[2];
      const float inv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
      kd[b][0] = d0 * inv; kd[b][1] = d1 * inv; kd[b][2] = d2 * inv;
      pv[b][0] = pw[0]; pv[b][1] = pw[1]; pv[b][2] = pw[2];
      torsion_cs(j[b], a.step_deg, &cs[b], &sn[b]);
    }
    float G[9], Mk[9];
    cube_mat(k, G);
    mat3mul(M, G, Mk);
    float acc = 0.f;
    for (int i = 0; i < N; ++i) {
      const float4 X = sx[i];
      float y[3] = {X.x, X.y, X.z};
#pragma unroll
      for (int b = 0; b < kExMaxRot; ++b) {
        if (b >= n) break;
        if (member[b][i >> 5] >> (i & 31) & 1u) rodrigues_apply(y, pv[b], kd[b], cs[b], sn[b]);
      }
      const float ux = fmaf(Mk[0], y[0], fmaf(Mk[1], y[1], fmaf(Mk[2], y[2], o[0])));
      const float uy = fmaf(Mk[3], y[0], fmaf(Mk[4], y[1], fmaf(Mk[5], y[2], o[1])));
      const float uz = fmaf(Mk[6], y[0], fmaf(Mk[7], y[1], fmaf(Mk[8], y[2], o[2])));
      acc -= grid_sample_fmt<FMT>(a.grid, ux, uy, uz, __float_as_int(X.w));
    }
    if (acc > best) { best = acc; bestc = c; }   // c ascends per thread: ties keep the first
  }
  // block argmax: higher score, then lower combination index
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, best, off);
    const long long oc = __shfl_xor_sync(0xffffffffu, bestc, off);
    if (os > best || (os == best && oc < bestc)) { best = os; bestc = oc; }
  }
  if ((tid & 31) == 0) { red_s[tid >> 5] = best; red_c[tid >> 5] = bestc; }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < kExThreads / 32; ++w)
      if (red_s[w] > best || (red_s[w] == best && red_c[w] < bestc)) { best = red_s[w]; bestc = red_c[w]; }
    if (bestc >= total) bestc = 0;   // only if every score is NaN; keeps the indices in range
    const size_t lr = (size_t)l * a.R + r;
    if (a.samples) atomicAdd(&a.samples[blockIdx.x % kSampleSlots], (unsigned long long)(total * N));
    a.res_score[lr] = best;
    long long rem = bestc;
    uint8_t* cnt = a.res_cnt + (size_t)r0 * a.R + (size_t)r * n;
    for (int b = n - 1; b >= 0; --b) { cnt[b] = (uint8_t)(rem % nt); rem /= nt; }
    a.res_k[lr] = (uint8_t)rem;
  }
}

}  // namespace

cudaError_t launch_exhaustive(const DockArgs& a, cudaStream_t s) {
  const long long blocks = (long long)a.lig.L * a.R;
  if (blocks == 0) return cudaSuccess;
  if (a.fmt == kRecF32)
    exhaustive_kernel<kRecF32><<<(unsigned)blocks, kExThreads, 0, s>>>(a);
  else if (a.fmt == kRecF16)
    exhaustive_kernel<kRecF16><<<(unsigned)blocks, kExThreads, 0, s>>>(a);
  else
    exhaustive_kernel<kRecBF16><<<(unsigned)blocks, kExThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ligen
