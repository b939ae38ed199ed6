// Ligand packer: one warp per ligand.
//
// Converts the CSR library into what the docking kernel stages in shared
// memory: centred SoA-friendly coordinates (float4, type in w), and for every
// rotatable bond its axis (fixed endpoint u, moving endpoint v) and the list
// of moving atoms. Cutting rotatable bond (a, b) splits the tree in two; the
// moving side is the smaller part, and on a tie the part without atom 0.
// Invalid ligands (not a tree, ids or types out of range, too large) get
// status LIGEN_ERR_BAD_LIGAND; nothing traps.
#include "../../include/ligen.h"
#include "internal.h"

namespace ligen {
namespace {

constexpr int kPackWarps = 4;
constexpr int kMaxN = LIGEN_MAX_ATOMS;

struct PackScratch {
  int32_t deg[kMaxN];
  int32_t cursor[kMaxN];
  int16_t adj_off[kMaxN + 1];
  int16_t parent[kMaxN];
  uint16_t size[kMaxN];
  uint8_t adj[2 * kMaxN];
  uint8_t tin[kMaxN];
  uint8_t order[kMaxN];
  uint8_t stack[kMaxN];
  // per rotatable bond: moving side = atoms with preorder index in [lo, hi)
  // (child side moves) or outside it; fixed endpoint u, moving endpoint v
  // per rotatable bond, as atom bit masks: the atoms a turn moves (moving
  // side without v) and the atoms its sweep reads (moving side and u)
  uint32_t moved[LIGEN_MAX_ROT][kMaxN / 32];
  uint32_t reads[LIGEN_MAX_ROT][kMaxN / 32];
};

__device__ __forceinline__ int rot_class(int n) {
  const int edges[11] = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
  int c = 10;
#pragma unroll
  for (int k = 10; k >= 0; --k)
    if (n <= edges[k]) c = k;
  return c;
}

__device__ __forceinline__ int atom_class(int N) {
  return N <= 32 ? 0 : N <= 64 ? 1 : N <= 128 ? 2 : 3;
}

__global__ void __launch_bounds__(32 * kPackWarps) pack_kernel(const LigandsDev lig, int nc, const Packed out) {
  __shared__ PackScratch scratch[kPackWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.x * kPackWarps + warp;
  if (l >= lig.L) return;
  PackScratch& S = scratch[warp];
  const int a0 = lig.atom_off[l];
  const int N = lig.atom_off[l + 1] - a0;
  const int e0 = a0 - l;
  const int r0 = lig.rot_off[l];
  const int n = lig.rot_off[l + 1] - r0;
  const unsigned full = 0xffffffffu;

  bool bad = (N < 1) | (N > kMaxN) | (n < 0) | (n > LIGEN_MAX_ROT);
  if (!bad) {
    // centroid and centred coordinates
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int i = lane; i < N; i += 32) {
      sx += lig.xyz[3 * (a0 + i)];
      sy += lig.xyz[3 * (a0 + i) + 1];
      sz += lig.xyz[3 * (a0 + i) + 2];
      bad |= lig.type[a0 + i] >= nc;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(full, sx, o);
      sy += __shfl_xor_sync(full, sy, o);
      sz += __shfl_xor_sync(full, sz, o);
    }
    const float inv = 1.0f / (float)N;
    sx *= inv; sy *= inv; sz *= inv;
    for (int i = lane; i < N; i += 32) {
      float4 v;
      v.x = lig.xyz[3 * (a0 + i)] - sx;
      v.y = lig.xyz[3 * (a0 + i) + 1] - sy;
      v.z = lig.xyz[3 * (a0 + i) + 2] - sz;
      v.w = __int_as_float((int)lig.type[a0 + i]);
      out.xc[a0 + i] = v;
    }
    for (int e = lane; e < N - 1; e += 32) {
      int a = lig.bonds[2 * (e0 + e)], b = lig.bonds[2 * (e0 + e) + 1];
      bad |= (a < 0) | (a >= N) | (b < 0) | (b >= N);
    }
    for (int b = lane; b < n; b += 32) {
      int e = lig.rot_edge[r0 + b];
      bad |= (e < 0) | (e >= N - 1);
    }
  }
  bad = __any_sync(full, bad);

  if (!bad) {
    // adjacency lists (CSR in shared memory)
    for (int i = lane; i < N; i += 32) { S.deg[i] = 0; S.parent[i] = -1; S.size[i] = 1; }
    __syncwarp();
    for (int e = lane; e < N - 1; e += 32) {
      atomicAdd(&S.deg[lig.bonds[2 * (e0 + e)]], 1);
      atomicAdd(&S.deg[lig.bonds[2 * (e0 + e) + 1]], 1);
    }
    __syncwarp();
    if (lane == 0) {
      int o = 0;
      for (int i = 0; i < N; ++i) { S.adj_off[i] = (int16_t)o; S.cursor[i] = o; o += S.deg[i]; }
      S.adj_off[N] = (int16_t)o;
    }
    __syncwarp();
    for (int e = lane; e < N - 1; e += 32) {
      int a = lig.bonds[2 * (e0 + e)], b = lig.bonds[2 * (e0 + e) + 1];
      S.adj[atomicAdd(&S.cursor[a], 1)] = (uint8_t)b;
      S.adj[atomicAdd(&S.cursor[b], 1)] = (uint8_t)a;
    }
    __syncwarp();
    // depth-first preorder from atom 0 (lane 0); each atom is pushed once
    int ok = 1;
    if (lane == 0) {
      int sp = 0, t = 0;
      S.stack[sp++] = 0;
      S.parent[0] = 0;
      while (sp > 0) {
        int x = S.stack[--sp];
        S.tin[x] = (uint8_t)t;
        S.order[t++] = (uint8_t)x;
        for (int q = S.adj_off[x]; q < S.adj_off[x + 1]; ++q) {
          int y = S.adj[q];
          if (S.parent[y] < 0) {
            S.parent[y] = (int16_t)x;
            S.stack[sp++] = (uint8_t)y;
          } else if (y != S.parent[x] && !(x == 0 && y == 0)) {
            ok = 0;   // reached an atom twice: a cycle
          }
        }
      }
      ok &= (t == N);
      // subtree sizes, children before parents
      if (ok)
        for (int q = N - 1; q >= 1; --q) {
          int x = S.order[q];
          S.size[S.parent[x]] += S.size[x];
        }
    }
    bad = !__shfl_sync(full, ok, 0);
    __syncwarp();
  }

  if (!bad) {
    for (int b = 0; b < n; ++b) {
      const int gb = r0 + b;
      const int e = lig.rot_edge[gb];
      const int pa = lig.bonds[2 * (e0 + e)], pb = lig.bonds[2 * (e0 + e) + 1];
      const int child = (pb != 0 && S.parent[pb] == pa) ? pb : pa;
      const int par = (child == pb) ? pa : pb;
      const int sz = S.size[child];
      const bool child_moves = 2 * sz <= N;   // smaller side; tie: side without atom 0
      const int v = child_moves ? child : par;
      const int u = child_moves ? par : child;
      const int lo = S.tin[child], hi = lo + sz;
      int cnt = 0;
      const int words = (N + 31) >> 5;   // mask words holding atoms; the rest are zero
      if (out.fbits && lane >= words && lane < kMaxN / 32) out.fbits[(size_t)gb * 8 + lane] = 0u;
      for (int base = 0; base < 32 * words; base += 32) {
        const int i = base + lane;
        bool mv = false;
        if (i < N) {
          const bool in_sub = (S.tin[i] >= lo) & (S.tin[i] < hi);
          mv = child_moves ? in_sub : !in_sub;
        }
        const unsigned word = __ballot_sync(full, mv);
        if (out.fbits && lane == 0) out.fbits[(size_t)gb * 8 + (base >> 5)] = word;
        const bool mx = mv & (i != v);
        const unsigned bx = __ballot_sync(full, mx);
        if (lane == 0) {
          S.moved[b][base >> 5] = bx;
          S.reads[b][base >> 5] = word | (((u >> 5) == (base >> 5)) ? 1u << (u & 31) : 0u);
        }
        if (mx) out.frag[(size_t)gb * kFragStride + cnt + __popc(bx & ((1u << lane) - 1u))] = (uint8_t)i;
        cnt += __popc(bx);
      }
      if (lane == 0) {
        out.binfo[gb] = make_uchar4((uint8_t)u, (uint8_t)v, (uint8_t)cnt, 0);
        if (out.axis) { out.axis[2 * gb] = u; out.axis[2 * gb + 1] = v; }
      }
    }
    __syncwarp();
    // touch[b'] bit b: turning bond b' moves an atom that bond b's sweep reads
    // (its moving side, v included, or its fixed endpoint u). Turning b'
    // moves its moving side except v_b', which lies on its own axis.
    if (out.touch) {
      const int words = (N + 31) >> 5;
      for (int bp = lane; bp < n; bp += 32) {   // one lane per turning bond
        uint32_t bits = 1u << bp;
        for (int b = 0; b < n; ++b) {
          uint32_t hit = 0u;
          for (int w = 0; w < words; ++w) hit |= S.moved[bp][w] & S.reads[b][w];
          if (hit) bits |= 1u << b;
        }
        out.touch[r0 + bp] = bits;
      }
    }
  } else {
    for (int b = 0; b < n && b < LIGEN_MAX_ROT; ++b) {
      const int gb = r0 + b;
      if (out.fbits && lane < 8) out.fbits[(size_t)gb * 8 + lane] = 0u;
      if (lane == 0) {
        out.binfo[gb] = make_uchar4(0, 0, 0, 0);
        if (out.axis) { out.axis[2 * gb] = -1; out.axis[2 * gb + 1] = -1; }
        if (out.touch) out.touch[gb] = 0u;
      }
    }
  }
  if (lane == 0) {
    out.status[l] = bad ? LIGEN_ERR_BAD_LIGAND : 0;
    if (out.bucket) out.bucket[l] = atom_class(N) * 11 + rot_class(n);
  }
}

}  // namespace

cudaError_t launch_pack(const LigandsDev& lig, int nc, const Packed& out, cudaStream_t s) {
  if (lig.L == 0) return cudaSuccess;
  const int blocks = (lig.L + kPackWarps - 1) / kPackWarps;
  pack_kernel<<<blocks, 32 * kPackWarps, 0, s>>>(lig, nc, out);
  return cudaGetLastError();
}

}  // namespace ligen
