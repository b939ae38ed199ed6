// Docking kernel: restarts -> rigid stage -> torsion sweeps -> final score.
//
// Mapping. A work item is one ligand over `rpc` consecutive restarts; each
// restart is owned by a group of G adjacent lanes (G = 2, 4, 8, 16 or 32), so
// a warp runs 32/G restarts of the same ligand in lockstep (identical atom counts,
// bonds and fragment sizes: no divergence). Inside a group the lanes split
// the *candidates* of a stage (cube rotations in the rigid stage, torsion
// increments in the sweep) and each lane sums its candidates' atom terms on
// its own, so a stage needs no per-candidate reduction, only a log2(G)-step
// shuffle argmax across the group. A lane holds SLOTS increments, so SLOTS
// independent 256-bit gathers are in flight per moving atom.
//
// Shared memory per CTA: the ligand (centred coordinates + type, bond axes,
// moving-atom lists) and the current coordinates of every restart, in grid
// units, as [atom][restart] planes so that the restarts of a warp read
// consecutive words. The sweep caches nothing: the moving side of a bond is
// re-sampled for each increment j, the fixed side is a constant of the
// decision and is not sampled at all (the argmax is over moving-side sums).
//
// Work distribution. Either one CTA per work item (grid = items), or a
// persistent grid whose CTAs take items from a device counter (atomicAdd,
// no waiting) until the list is exhausted; items may come from a ligand list
// (a bucket of similar ligands) instead of the whole library.
#include "../../include/ligen.h"
#include "internal.h"

namespace ligen {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct SmemLayout {
  float4* sx;       // [max_atoms]
  float* cx;        // [max_atoms][rpc]
  float* cy;
  float* cz;
  uchar4* sb;       // [max_rot]
  uint16_t* soff;   // [max_rot]
  uint8_t* scnt;    // [max_rot][rpc]
  uint8_t* sfrag;   // [max_frag]
  uint32_t* stouch; // [max_rot] bonds whose sweep a turn of this bond affects
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

__host__ __device__ inline size_t carve(int max_atoms, int max_rot, int max_frag, int rpc,
                                        unsigned char* base, SmemLayout* L) {
  size_t off[9];
  const size_t bytes[9] = {(size_t)max_atoms * 16, (size_t)max_atoms * rpc * 4, (size_t)max_atoms * rpc * 4,
                           (size_t)max_atoms * rpc * 4, (size_t)max_rot * 4, (size_t)max_rot * 2,
                           (size_t)max_rot * rpc, (size_t)max_frag, (size_t)max_rot * 4};
  size_t o = 0;
  for (int i = 0; i < 9; ++i) { off[i] = o; o = align16(o + bytes[i]); }
  if (L) {
    L->sx = (float4*)(base + off[0]); L->cx = (float*)(base + off[1]);
    L->cy = (float*)(base + off[2]);  L->cz = (float*)(base + off[3]);
    L->sb = (uchar4*)(base + off[4]); L->soff = (uint16_t*)(base + off[5]);
    L->scnt = base + off[6];          L->sfrag = base + off[7];
    L->stouch = (uint32_t*)(base + off[8]);
  }
  return o;
}

// Increment a lane evaluates in the sweep slot that starts at `base`: its
// own j, or, for a lane past the last increment, a valid j of the same slot,
// so that its loads repeat another lane's addresses in the same instruction
// and coalesce with them at no cost (the selection skips such lanes). With
// 36 increments on 8 lanes x 5 slots the last slot's 4 spare lanes used to
// load 4 new positions; measured on GB300: 2.5% faster docking with FP16
// records, 3.3% with FP32.
__device__ __forceinline__ int slot_j(int j, int base, int nt) {
  if (j < nt) return j;
  return base < nt ? base + (j - base) % (nt - base) : j % nt;
}

// Argmax over the G lanes of a group: higher score wins, lower index on ties.
template <int G>
__device__ __forceinline__ void group_argmax(float& s, int& idx) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    float os = __shfl_xor_sync(kFull, s, o);
    int oi = __shfl_xor_sync(kFull, idx, o);
    if (os > s || (os == s && oi < idx)) { s = os; idx = oi; }
  }
}

// One work item: ligand l, restarts [chunk * rpc, chunk * rpc + rpc).
// COUNT: also add the samples the item's restarts needed to a.samples (a
// separate instantiation, so the plain kernel carries no counting).
template <int G, int SLOTS, int FMT, bool COUNT>
__device__ __forceinline__ void dock_item(const DockArgs& a, const SmemLayout& S, int l, int chunk) {
  const int rpc = a.rpc;
  const int tid = threadIdx.x;
  const int a0 = a.lig.atom_off[l];
  const int N = a.lig.atom_off[l + 1] - a0;
  const int r0 = a.lig.rot_off[l];
  const int n = a.lig.rot_off[l + 1] - r0;
  if (!lg_check(a.grid.check, N <= a.max_atoms && n <= a.max_rot, kChkItemShape)) return;   // uniform

  for (int i = tid; i < N; i += blockDim.x) S.sx[i] = a.pk.xc[a0 + i];
  for (int b = tid; b < n; b += blockDim.x) {
    S.sb[b] = a.pk.binfo[r0 + b];
    S.stouch[b] = a.pk.touch[r0 + b];
  }
  for (int i = tid; i < n * rpc; i += blockDim.x) S.scnt[i] = 0;
  __syncthreads();
  if (tid == 0) {
    int o = 0;
    for (int b = 0; b < n; ++b) { S.soff[b] = (uint16_t)o; o += S.sb[b].z; }
  }
  __syncthreads();
  const int n_frag = n > 0 ? S.soff[n - 1] + S.sb[n - 1].z : 0;
  if (!lg_check(a.grid.check, n_frag <= a.max_frag, kChkItemShape)) return;   // uniform
  for (int b = 0; b < n; ++b) {
    const int m = S.sb[b].z;
    for (int i = tid; i < m; i += blockDim.x)
      S.sfrag[S.soff[b] + i] = a.pk.frag[(size_t)(r0 + b) * kFragStride + i];
  }
  __syncthreads();
  if constexpr (LIGEN_CHECKED) {   // every axis end and moving atom is an atom of the ligand
    bool bad = false;
    for (int b = tid; b < n; b += blockDim.x) bad |= S.sb[b].x >= N || S.sb[b].y >= N;
    for (int t = tid; t < n_frag; t += blockDim.x) bad |= S.sfrag[t] >= N;
    if (__syncthreads_or(bad)) {
      if (tid == 0) lg_check(a.grid.check, false, kChkAtomIndex);
      return;
    }
  }

  const int rr = tid / G, sub = tid % G;
  const int r_raw = chunk * rpc + rr;
  const bool active = r_raw < a.R;
  const int r = active ? r_raw : a.R - 1;   // idle groups shadow a real restart
  const GridView& grid = a.grid;

  // ---- restart initialisation: q_r (Shoemake), t_r = centre + jitter
  float u[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) u[k] = restart_uniform(a.seed, (uint32_t)l, (uint32_t)r, (uint32_t)k);
  const Quat qr = qnormalize(shoemake(u[0], u[1], u[2]));
  float Rm[9];
  qmat(qr, Rm);
  float M[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) M[i] = Rm[i] * a.inv_h;   // body (Angstrom) -> grid units
  float o[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float t = a.center[k] + (2.0f * u[3 + k] - 1.0f) * a.jitter;
    o[k] = (t - a.origin[k]) * a.inv_h;
  }

  // ---- rigid stage: lane `sub` scores cube rotations sub, sub+G, ...
  float best = -INFINITY;
  int kb = 0;
  for (int k = sub; k < a.n_rigid; k += G) {
    float Gk[9], Mk[9];
    cube_mat(k, Gk);
    mat3mul(M, Gk, Mk);
    float acc = 0.f;
#pragma unroll 4
    for (int i = 0; i < N; ++i) {
      const float4 X = S.sx[i];
      const float ux = fmaf(Mk[0], X.x, fmaf(Mk[1], X.y, fmaf(Mk[2], X.z, o[0])));
      const float uy = fmaf(Mk[3], X.x, fmaf(Mk[4], X.y, fmaf(Mk[5], X.z, o[1])));
      const float uz = fmaf(Mk[6], X.x, fmaf(Mk[7], X.y, fmaf(Mk[8], X.z, o[2])));
      const int c = __float_as_int(X.w);
      if constexpr (FMT == kRecF32) acc -= grid_sample(grid, ux, uy, uz, c);
      else acc -= grid_sample16_cb<FMT>(grid, chan_base16(grid, c), ux, uy, uz, c);
    }
    if (acc > best) { best = acc; kb = k; }
  }
  group_argmax<G>(best, kb);
  const int D = 1 + a.passes * n;
  int16_t* trace = nullptr;
  if (a.trace && active)
    trace = a.trace + (size_t)a.R * ((size_t)l + (size_t)a.passes * r0) + (size_t)r * D;
  if (trace && sub == 0) trace[0] = (int16_t)kb;
  {
    float Gk[9], Mk[9];
    cube_mat(kb, Gk);
    mat3mul(M, Gk, Mk);
    for (int i = sub; i < N; i += G) {
      const float4 X = S.sx[i];
      S.cx[i * rpc + rr] = fmaf(Mk[0], X.x, fmaf(Mk[1], X.y, fmaf(Mk[2], X.z, o[0])));
      S.cy[i * rpc + rr] = fmaf(Mk[3], X.x, fmaf(Mk[4], X.y, fmaf(Mk[5], X.z, o[1])));
      S.cz[i * rpc + rr] = fmaf(Mk[6], X.x, fmaf(Mk[7], X.y, fmaf(Mk[8], X.z, o[2])));
    }
  }
  __syncwarp();

  // ---- torsion sweep: lane `sub` scores increments j = base + sub + G*s
  const int nt = a.n_theta;
  const int per_chunk = G * SLOTS;
  const int nchunks = (nt + per_chunk - 1) / per_chunk;
  float cs[SLOTS], sn[SLOTS];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) torsion_cs(slot_j(sub + G * s, G * s, a.n_theta), a.step_deg, &cs[s], &sn[s]);

  // Clean bonds. A bond's decision reads only the positions of its moving
  // atoms and of its axis ends, and its sweep scores the whole circle of
  // increments. After a sweep, the bond sits at the best increment of that
  // circle: kept (j = 0) or turned to j*, which moves none of the axis ends.
  // Until a later turn moves one of the atoms it reads (the packer's touch
  // masks), a new sweep would score the same circle from its maximum, so
  // the bond is clean and its decision is 0 without sampling. After a kept
  // torsion the new sweep would repeat the last one exactly; after a turn it
  // scores rotated copies of the same positions, equal in exact arithmetic,
  // so only a near-tie, where either choice is valid, could go another way
  // in floating point. A clean restart in a warp that sweeps samples nothing
  // for that bond; a bond clean for the whole warp is skipped, and so is the
  // rest of the sweep once every bond of every restart of the warp is clean.
  uint32_t dirty = n >= 32 ? 0xffffffffu : ((1u << n) - 1u);   // bonds that must be swept
  long long needed = COUNT ? (long long)a.n_rigid * N : 0;   // samples this restart needs
  for (int p = 0; p < a.passes; ++p) {
    for (int b = 0; b < n; ++b) {
      if (__all_sync(kFull, dirty == 0u)) {
        if (trace && sub == 0)
          for (int d = p * n + b; d < a.passes * n; ++d) trace[1 + d] = 0;
        p = a.passes;   // leaves both loops
        break;
      }
      const bool live = (dirty >> b) & 1u;
      if (!__any_sync(kFull, live)) {
        if (trace && sub == 0) trace[1 + p * n + b] = 0;
        continue;
      }
      const uchar4 bi = S.sb[b];
      const int vi = bi.y, m = bi.z, off = S.soff[b];
      const float vx = S.cx[vi * rpc + rr], vy = S.cy[vi * rpc + rr], vz = S.cz[vi * rpc + rr];
      float kx = vx - S.cx[bi.x * rpc + rr];
      float ky = vy - S.cy[bi.x * rpc + rr];
      float kz = vz - S.cz[bi.x * rpc + rr];
      const float kn = rsqrtf(kx * kx + ky * ky + kz * kz);
      kx *= kn; ky *= kn; kz *= kn;
      float bs = -INFINITY;
      int jb = 0;
      for (int ch = 0; ch < nchunks; ++ch) {
        const int jbase = ch * per_chunk;
        if (ch > 0) {
#pragma unroll
          for (int s = 0; s < SLOTS; ++s) torsion_cs(slot_j(jbase + sub + G * s, jbase + G * s, nt), a.step_deg, &cs[s], &sn[s]);
        }
        float acc[SLOTS];
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) acc[s] = 0.f;
        // A clean bond samples nothing: its candidates all sum to 0, so it
        // keeps j = 0, the decision a sweep would reach.
        const int m_live = live ? m : 0;
        if (COUNT && ch == 0) needed += (long long)(nt - 1) * m_live;
        for (int t = 0; t < m_live; ++t) {
          const int i = S.sfrag[off + t];
          const int c = __float_as_int(S.sx[i].w);
          const unsigned char* cb = FMT == kRecF32 ? nullptr : chan_base16(grid, c);   // 16-bit records
          const float dx = S.cx[i * rpc + rr] - vx;
          const float dy = S.cy[i * rpc + rr] - vy;
          const float dz = S.cz[i * rpc + rr] - vz;
          const float kd = kx * dx + ky * dy + kz * dz;
          const float px = fmaf(kx, kd, vx), py = fmaf(ky, kd, vy), pz = fmaf(kz, kd, vz);
          const float ex = fmaf(-kx, kd, dx), ey = fmaf(-ky, kd, dy), ez = fmaf(-kz, kd, dz);
          const float qx = ky * dz - kz * dy, qy = kz * dx - kx * dz, qz = kx * dy - ky * dx;
          if constexpr (FMT != kRecF32) {
            // two increments per packed instruction (measured: 0.5% faster
            // with 16-bit records, 1% slower with FP32 records)
            float ux[SLOTS], uy[SLOTS], uz[SLOTS];
#pragma unroll
            for (int s = 0; s + 1 < SLOTS; s += 2) {
              const float2 cc = make_float2(cs[s], cs[s + 1]), ss = make_float2(sn[s], sn[s + 1]);
              const float2 X = fma2(make_float2(ex, ex), cc, fma2(make_float2(qx, qx), ss, make_float2(px, px)));
              const float2 Y = fma2(make_float2(ey, ey), cc, fma2(make_float2(qy, qy), ss, make_float2(py, py)));
              const float2 Z = fma2(make_float2(ez, ez), cc, fma2(make_float2(qz, qz), ss, make_float2(pz, pz)));
              ux[s] = X.x; ux[s + 1] = X.y; uy[s] = Y.x; uy[s + 1] = Y.y; uz[s] = Z.x; uz[s + 1] = Z.y;
            }
            if constexpr (SLOTS % 2 == 1) {
              ux[SLOTS - 1] = fmaf(ex, cs[SLOTS - 1], fmaf(qx, sn[SLOTS - 1], px));
              uy[SLOTS - 1] = fmaf(ey, cs[SLOTS - 1], fmaf(qy, sn[SLOTS - 1], py));
              uz[SLOTS - 1] = fmaf(ez, cs[SLOTS - 1], fmaf(qz, sn[SLOTS - 1], pz));
            }
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) acc[s] -= grid_sample16_cb<FMT>(grid, cb, ux[s], uy[s], uz[s], c);
          } else {
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) {
              const float ux = fmaf(ex, cs[s], fmaf(qx, sn[s], px));
              const float uy = fmaf(ey, cs[s], fmaf(qy, sn[s], py));
              const float uz = fmaf(ez, cs[s], fmaf(qz, sn[s], pz));
              acc[s] -= grid_sample_fmt<FMT>(grid, ux, uy, uz, c);
            }
          }
        }
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
          const int j = jbase + sub + G * s;
          if (j < nt && acc[s] > bs) { bs = acc[s]; jb = j; }
        }
      }
      if (nchunks > 1) {
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) torsion_cs(slot_j(sub + G * s, G * s, a.n_theta), a.step_deg, &cs[s], &sn[s]);
      }
      group_argmax<G>(bs, jb);
      if (jb != 0) {
        float c, s;
        torsion_cs(jb, a.step_deg, &c, &s);
        for (int t = sub; t < m; t += G) {
          const int i = S.sfrag[off + t];
          const float dx = S.cx[i * rpc + rr] - vx;
          const float dy = S.cy[i * rpc + rr] - vy;
          const float dz = S.cz[i * rpc + rr] - vz;
          const float kd = kx * dx + ky * dy + kz * dz;
          const float px = fmaf(kx, kd, vx), py = fmaf(ky, kd, vy), pz = fmaf(kz, kd, vz);
          const float ex = fmaf(-kx, kd, dx), ey = fmaf(-ky, kd, dy), ez = fmaf(-kz, kd, dz);
          const float qx = ky * dz - kz * dy, qy = kz * dx - kx * dz, qz = kx * dy - ky * dx;
          S.cx[i * rpc + rr] = fmaf(ex, c, fmaf(qx, s, px));
          S.cy[i * rpc + rr] = fmaf(ey, c, fmaf(qy, s, py));
          S.cz[i * rpc + rr] = fmaf(ez, c, fmaf(qz, s, pz));
        }
      }
      __syncwarp();
      if (sub == 0) {
        S.scnt[b * rpc + rr] = (uint8_t)((S.scnt[b * rpc + rr] + jb) % nt);
        if (trace) trace[1 + p * n + b] = (int16_t)jb;
      }
      // a turn dirties the bonds it touches; the bond itself is clean either way
      dirty = ((jb != 0) ? (dirty | S.stouch[b]) : dirty) & ~(1u << b);
    }
  }

  // ---- final score of the restart's pose (all atoms)
  float acc = 0.f;
  for (int i = sub; i < N; i += G)
    acc -= grid_sample_fmt<FMT>(grid, S.cx[i * rpc + rr], S.cy[i * rpc + rr], S.cz[i * rpc + rr],
                       __float_as_int(S.sx[i].w));
#pragma unroll
  for (int off = 1; off < G; off <<= 1) acc += __shfl_xor_sync(kFull, acc, off);
  if constexpr (COUNT) {   // one add per warp, spread over the counter slots
    long long v = (active && sub == 0) ? needed : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((tid & 31) == 0) atomicAdd(&a.samples[blockIdx.x % kSampleSlots], (unsigned long long)v);
  }
  if (a.coords && active) {   // debug output: the positions the final score sampled
    float* cd = a.coords + 3 * ((size_t)a.R * a0 + (size_t)r * N);
    for (int i = sub; i < N; i += G) {
      cd[3 * i] = S.cx[i * rpc + rr];
      cd[3 * i + 1] = S.cy[i * rpc + rr];
      cd[3 * i + 2] = S.cz[i * rpc + rr];
    }
  }
  if (active && sub == 0) {
    const size_t lr = (size_t)l * a.R + r;
    a.res_score[lr] = acc;
    a.res_k[lr] = (uint8_t)kb;
    uint8_t* cnt = a.res_cnt + (size_t)r0 * a.R + (size_t)r * n;
    for (int b = 0; b < n; ++b) cnt[b] = S.scnt[b * rpc + rr];
  }
}

// MINB: resident CTAs asked of the register allocator (1: no request).
// 8-lane shapes come in four builds: 8 CTAs (64 registers, some spill to
// local memory), 7 (72 registers), 6 (~80) and unconstrained (~100, 4 CTAs).
// More CTAs pay only while their shared memory leaves L1 room for the
// spills and the gathers: measured on GB300, the screening library (~20 KB
// per CTA) docks fastest with 8 CTAs, the bimodal one (27.6 KB per CTA) with
// 7 (8 leave under 48 KB of L1 and run 60% slower; 6 CTAs 9%, the
// unconstrained build 42%).
// launch_dock takes the largest count whose CTAs fit kCtaSmemBudget.
template <int G, int SLOTS, int FMT, bool COUNT, int MINB>
__global__ void __launch_bounds__(128, MINB) dock_kernel(const DockArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int next_item;
  SmemLayout S;
  carve(a.max_atoms, a.max_rot, a.max_frag, a.rpc, smem, &S);
  int item = blockIdx.x;
  while (true) {
    if (a.queue) {   // persistent: take the next item from the device counter
      if (threadIdx.x == 0) next_item = atomicAdd(a.queue, 1);
      __syncthreads();
      item = next_item;
      __syncthreads();
    }
    if (item >= a.n_items) break;
    const int li = item / a.chunks;
    const int l = a.list ? a.list[li] : li;
    if (a.pk.status[l] == 0)   // uniform over the CTA
      dock_item<G, SLOTS, FMT, COUNT>(a, S, l, item - li * a.chunks);
    if (!a.queue) break;
    __syncthreads();   // shared memory is reused by the next item
  }
}

}  // namespace

size_t dock_smem_bytes(int max_atoms, int max_rot, int max_frag, int rpc) {
  return carve(max_atoms, max_rot, max_frag, rpc, nullptr, nullptr);
}

namespace {

using KernelFn = void (*)(DockArgs);


// Instantiated (G, SLOTS, record format) shapes; G * SLOTS increments per
// chunk of the sweep. The 16-bit record formats exist for 4 and 8 lanes.
struct Shape {
  int G, SLOTS, FMT;
  KernelFn fn[2][4];   // [counts the samples needed][build: 8, 7, 6 CTAs, unconstrained]
};
#define LG_BUILDS(G, S, F, C)                                                                         \
  {dock_kernel<G, S, F, C, G == 8 ? 8 : 1>, dock_kernel<G, S, F, C, G == 8 ? 7 : 1>,                   \
   dock_kernel<G, S, F, C, G == 8 ? 6 : 1>, dock_kernel<G, S, F, C, 1>}
// The counting kernel only serves untimed calls: one build for all four.
#define LG_COUNTING(G, S, F)                                                                          \
  {dock_kernel<G, S, F, true, 1>, dock_kernel<G, S, F, true, 1>, dock_kernel<G, S, F, true, 1>,        \
   dock_kernel<G, S, F, true, 1>}
#define LG_SHAPE(G, S, F) {G, S, F, {LG_BUILDS(G, S, F, false), LG_COUNTING(G, S, F)}}
const Shape kShapes[] = {
    LG_SHAPE(2, 6, kRecF32),
    LG_SHAPE(2, 18, kRecF32),
    LG_SHAPE(4, 3, kRecF32),
    LG_SHAPE(4, 9, kRecF32),
    LG_SHAPE(8, 2, kRecF32),
    LG_SHAPE(8, 5, kRecF32),
    LG_SHAPE(4, 3, kRecF16),
    LG_SHAPE(4, 9, kRecF16),
    LG_SHAPE(8, 2, kRecF16),
    LG_SHAPE(8, 5, kRecF16),
    LG_SHAPE(4, 3, kRecBF16),
    LG_SHAPE(4, 9, kRecBF16),
    LG_SHAPE(8, 2, kRecBF16),
    LG_SHAPE(8, 5, kRecBF16),
    // one restart per half-warp or warp: a gather request covers 16 or 32
    // consecutive increments of one atom of one restart (36 increments as
    // 3 x 16 or 2 x 32 slots, the spare lanes repeating a valid increment)
    LG_SHAPE(16, 3, kRecF32),
    LG_SHAPE(32, 2, kRecF32),
    LG_SHAPE(16, 3, kRecF16),
    LG_SHAPE(32, 2, kRecF16),
};
#undef LG_SHAPE
#undef LG_COUNTING
#undef LG_BUILDS

// Shared memory the resident CTAs may take together (of the SM's 256 KB of
// L1 and shared memory), and the build for a CTA of `smem` bytes: the one
// asking for as many CTAs as fit that budget. 192 KB puts the screening
// library (~20 KB per CTA) at 8 CTAs and the bimodal one (27.6 KB, with the
// host's upper bound on the moving lists) at 7, the best of the measured
// builds for each.
constexpr size_t kCtaSmemBudget = 192 * 1024;
int build_for(size_t smem) {
  const size_t fit = smem ? kCtaSmemBudget / smem : 8;
  return fit >= 8 ? 0 : fit >= 7 ? 1 : fit >= 6 ? 2 : 3;
}

// The instantiation for G lanes, n_theta increments and record format: the
// fewest slots that cover n_theta in one chunk, else the largest (several
// chunks).
const Shape* pick_shape(int G, int n_theta, int fmt) {
  const Shape* best = nullptr;
  for (const Shape& sh : kShapes) {
    if (sh.G != G || sh.FMT != fmt) continue;
    if (sh.G * sh.SLOTS >= n_theta) {
      if (!best || best->G * best->SLOTS < n_theta || sh.SLOTS < best->SLOTS) best = &sh;
    } else if (!best || (best->G * best->SLOTS < n_theta && sh.SLOTS > best->SLOTS)) {
      best = &sh;
    }
  }
  return best;
}

}  // namespace

bool dock_lanes_supported(int G) { return G == 2 || G == 4 || G == 8 || G == 16 || G == 32; }

bool dock_shape_supported(int G, int fmt) { return pick_shape(G, 36, fmt) != nullptr; }

cudaError_t launch_dock(const DockArgs& a, int grid_ctas, cudaStream_t s, bool set_attr) {
  if (a.n_items == 0) return cudaSuccess;
  const Shape* sh = pick_shape(a.lanes, a.n_theta, a.fmt);
  if (!sh) return cudaErrorInvalidValue;
  const size_t smem = dock_smem_bytes(a.max_atoms, a.max_rot, a.max_frag, a.rpc);
  const KernelFn fn = sh->fn[a.samples != nullptr][build_for(smem)];
  if (set_attr) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const unsigned blocks = a.queue ? (unsigned)grid_ctas : (unsigned)a.n_items;
  fn<<<blocks, a.rpc * a.lanes, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t dock_set_smem_limit(int lanes, int n_theta, int fmt, size_t smem) {
  const Shape* sh = pick_shape(lanes, n_theta, fmt);
  if (!sh) return cudaErrorInvalidValue;
  for (int c = 0; c < 2; ++c)
    for (int o = 0; o < 4; ++o) {
      const cudaError_t e = cudaFuncSetAttribute(sh->fn[c][o], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

cudaError_t dock_occupancy(int lanes, int n_theta, int fmt, int rpc, size_t smem, int* blocks_per_sm) {
  const Shape* sh = pick_shape(lanes, n_theta, fmt);
  if (!sh) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sh->fn[0][build_for(smem)], rpc * lanes,
                                                       smem);
}

}  // namespace ligen
