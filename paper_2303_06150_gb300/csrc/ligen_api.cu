// C ABI of the docking library: argument checks, memory-space detection,
// workspace management, host staging and the launch sequence
//   [H2D] -> grid preparation -> ligand packer -> docking -> top-K -> [D2H].
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ligen.h"
#include "internal.h"

using namespace ligen;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(LIGEN_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LG_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// 1 = host memory (pageable or pinned), 0 = device or managed memory.
int is_host(const void* p) {
  if (!p) return -1;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 0 : 1;
}

// Memory space shared by a set of pointers (NULL entries ignored); -1 if mixed.
int space_of(std::initializer_list<const void*> ptrs) {
  int s = -2;
  for (const void* p : ptrs) {
    if (!p) continue;
    int h = is_host(p);
    if (s == -2) s = h;
    else if (s != h) return -1;
  }
  return s == -2 ? 0 : s;
}


// ------------------------------------------------------------ workspace --
struct Workspace {
  char* base = nullptr;
  size_t cap = 0;
};

std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

// Bump allocator over one workspace; every region is 256-byte aligned.
struct Arena {
  size_t used = 0;
  char* base = nullptr;
  size_t take(size_t bytes) {
    size_t at = used;
    used = (used + bytes + 255) & ~(size_t)255;
    return at;
  }
  template <class T>
  T* at(size_t off) const { return reinterpret_cast<T*>(base + off); }
};

// Upper bound on any one workspace (0: none), ligen_set_workspace_limit.
std::atomic<size_t> g_ws_limit{0};

int get_workspace(cudaStream_t s, size_t bytes, char** out) {
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  const size_t limit = g_ws_limit.load();
  if (limit && bytes > limit)
    return fail(LIGEN_ERR_OOM, "workspace of %zu bytes exceeds the limit of %zu bytes", bytes, limit);
  std::lock_guard<std::mutex> lk(g_ws_mu);
  Workspace& w = g_ws[{dev, s}];
  if (w.cap < bytes) {
    if (w.base) {
      LG_CUDA(cudaStreamSynchronize(s));
      cudaFree(w.base);
      w.base = nullptr;
      w.cap = 0;
    }
    size_t want = bytes + bytes / 8 + (1 << 20);
    if (limit && want > limit) want = limit;
    cudaError_t e = cudaMalloc(&w.base, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      w.base = nullptr;
      return fail(LIGEN_ERR_OOM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    w.cap = want;
  }
  *out = w.base;
  return LIGEN_OK;
}

// ------------------------------------------------------------ checking --
struct LibShape {
  int64_t atoms = 0, rot = 0;
  int max_atoms = 0, max_rot = 0;
  int64_t max_frag = 0;
  int64_t trace_len = 0;   // sum over ligands of 1 + passes * n_l (times R later)
};

int check_ligands(const ligen_ligands_t* g, int passes, LibShape* sh) {
  if (!g) return fail(LIGEN_ERR_INVALID_ARG, "ligands is NULL");
  if (g->n_ligands < 0) return fail(LIGEN_ERR_INVALID_ARG, "n_ligands < 0");
  if (g->n_ligands == 0) return LIGEN_OK;
  if (!g->h_atom_off || !g->h_rot_off)
    return fail(LIGEN_ERR_INVALID_ARG, "h_atom_off and h_rot_off (host copies) are required");
  if (!g->atom_off || !g->rot_off || !g->xyz || !g->type)
    return fail(LIGEN_ERR_INVALID_ARG, "atom_off, rot_off, xyz and type are required");
  if (g->h_atom_off[0] != 0 || g->h_rot_off[0] != 0)
    return fail(LIGEN_ERR_INVALID_ARG, "offsets must start at 0");
  for (int l = 0; l < g->n_ligands; ++l) {
    int N = g->h_atom_off[l + 1] - g->h_atom_off[l];
    int n = g->h_rot_off[l + 1] - g->h_rot_off[l];
    if (N < 1) return fail(LIGEN_ERR_INVALID_ARG, "ligand %d has %d atoms", l, N);
    if (n < 0) return fail(LIGEN_ERR_INVALID_ARG, "rot_off decreases at ligand %d", l);
    if (N > LIGEN_MAX_ATOMS) return fail(LIGEN_ERR_UNSUPPORTED, "ligand %d has %d atoms (max %d)", l, N, LIGEN_MAX_ATOMS);
    if (n > LIGEN_MAX_ROT) return fail(LIGEN_ERR_UNSUPPORTED, "ligand %d has %d rotatable bonds (max %d)", l, n, LIGEN_MAX_ROT);
    sh->max_atoms = N > sh->max_atoms ? N : sh->max_atoms;
    sh->max_rot = n > sh->max_rot ? n : sh->max_rot;
    int64_t frag = (int64_t)n * (N / 2);
    sh->max_frag = frag > sh->max_frag ? frag : sh->max_frag;
    sh->trace_len += 1 + (int64_t)passes * n;
  }
  sh->atoms = g->h_atom_off[g->n_ligands];
  sh->rot = g->h_rot_off[g->n_ligands];
  if (sh->atoms - g->n_ligands > 0 && !g->bonds) return fail(LIGEN_ERR_INVALID_ARG, "bonds is NULL");
  if (sh->rot > 0 && !g->rot_edge) return fail(LIGEN_ERR_INVALID_ARG, "rot_edge is NULL");
  if (sh->atoms > INT32_MAX / 4) return fail(LIGEN_ERR_UNSUPPORTED, "library too large");
  return LIGEN_OK;
}

int check_grid(const ligen_grid_t* g) {
  if (!g) return fail(LIGEN_ERR_INVALID_ARG, "grid is NULL");
  if (!g->data) return fail(LIGEN_ERR_INVALID_ARG, "grid data is NULL");
  if (g->nx < 2 || g->ny < 2 || g->nz < 2) return fail(LIGEN_ERR_INVALID_ARG, "grid needs >= 2 points per axis");
  if (g->nc < 1 || g->nc > LIGEN_MAX_CHANNELS)
    return fail(LIGEN_ERR_UNSUPPORTED, "grid channels %d outside 1..%d", g->nc, LIGEN_MAX_CHANNELS);
  if (g->dtype != LIGEN_F32) return fail(LIGEN_ERR_UNSUPPORTED, "grid dtype %d not supported", g->dtype);
  if (!(g->spacing > 0.f) || !std::isfinite(g->spacing)) return fail(LIGEN_ERR_INVALID_ARG, "grid spacing must be > 0");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(g->origin[k])) return fail(LIGEN_ERR_INVALID_ARG, "grid origin not finite");
  double cells = (double)(g->nx - 1) * (g->ny - 1) * (g->nz - 1);
  if (cells * g->nc > 2.0e9) return fail(LIGEN_ERR_UNSUPPORTED, "grid too large");
  return LIGEN_OK;
}

int check_params(const ligen_params_t* p) {
  if (!p) return fail(LIGEN_ERR_INVALID_ARG, "params is NULL");
  if (p->restarts < 1 || p->restarts > 65536) return fail(LIGEN_ERR_INVALID_ARG, "restarts must be 1..65536");
  if (p->n_rigid < 1 || p->n_rigid > LIGEN_N_RIGID) return fail(LIGEN_ERR_INVALID_ARG, "n_rigid must be 1..24");
  if (p->torsion_step_deg < 2 || p->torsion_step_deg > 360 || 360 % p->torsion_step_deg != 0)
    return fail(LIGEN_ERR_INVALID_ARG, "torsion_step_deg must divide 360 and be >= 2");
  if (p->passes < 0 || p->passes > 1000) return fail(LIGEN_ERR_INVALID_ARG, "passes must be 0..1000");
  if (p->top_k < 1 || p->top_k > p->restarts) return fail(LIGEN_ERR_INVALID_ARG, "top_k must be 1..restarts");
  if (p->mode != 0 && p->mode != 1) return fail(LIGEN_ERR_INVALID_ARG, "mode must be 0 (greedy) or 1 (exhaustive)");
  if (p->batching != LIGEN_BATCH_PLAIN && p->batching != LIGEN_BATCH_BUCKETS &&
      p->batching != LIGEN_BATCH_BUCKETS_STATIC && p->batching != LIGEN_BATCH_QUEUE)
    return fail(LIGEN_ERR_INVALID_ARG, "batching must be LIGEN_BATCH_PLAIN, _BUCKETS, _BUCKETS_STATIC or _QUEUE");
  if (p->grid_format != LIGEN_GRID_F32 && p->grid_format != LIGEN_GRID_F16 && p->grid_format != LIGEN_GRID_BF16)
    return fail(LIGEN_ERR_INVALID_ARG, "grid_format must be LIGEN_GRID_F32, _F16 or _BF16");
  if (p->rescore_fp64 != 0 && p->rescore_fp64 != 1) return fail(LIGEN_ERR_INVALID_ARG, "rescore_fp64 must be 0 or 1");
  if (p->scores_f64 && !p->rescore_fp64) return fail(LIGEN_ERR_INVALID_ARG, "scores_f64 needs rescore_fp64 = 1");
  if (!std::isfinite(p->jitter) || p->jitter < 0.f) return fail(LIGEN_ERR_INVALID_ARG, "jitter must be >= 0");
  if (!std::isfinite(p->out_penalty)) return fail(LIGEN_ERR_INVALID_ARG, "out_penalty not finite");
  return LIGEN_OK;
}

// Exhaustive mode: small ligands only (see ligen_params_t.mode).
int check_exhaustive(const ligen_ligands_t* g, const ligen_params_t* p) {
  if (p->trace) return fail(LIGEN_ERR_INVALID_ARG, "trace is not written in exhaustive mode (mode 1)");
  if (p->coords) return fail(LIGEN_ERR_INVALID_ARG, "coords are not written in exhaustive mode (mode 1)");
  if ((int64_t)g->n_ligands * p->restarts > INT32_MAX)
    return fail(LIGEN_ERR_UNSUPPORTED, "exhaustive mode: ligands * restarts exceeds 2^31 - 1");
  const int nt = 360 / p->torsion_step_deg;
  for (int l = 0; l < g->n_ligands; ++l) {
    const int n = g->h_rot_off[l + 1] - g->h_rot_off[l];
    if (n > kExMaxRot)
      return fail(LIGEN_ERR_UNSUPPORTED, "exhaustive mode: ligand %d has %d rotatable bonds (max %d)", l, n,
                  kExMaxRot);
    long long combos = p->n_rigid;
    for (int b = 0; b < n; ++b) combos *= nt;
    if (combos > kExMaxCombos)
      return fail(LIGEN_ERR_UNSUPPORTED, "exhaustive mode: ligand %d needs %lld poses per restart (max %lld)", l,
                  combos, kExMaxCombos);
  }
  return LIGEN_OK;
}

// ------------------------------------------------------ staged library --
// Ligand arrays on the device: the caller's pointers, or workspace copies.
struct LigandPlan {
  size_t off_atom_off, off_xyz, off_type, off_bonds, off_rot_off, off_rot_edge;
  bool host;
};

void plan_ligands(Arena& ar, const ligen_ligands_t* g, const LibShape& sh, bool host, LigandPlan* p) {
  p->host = host;
  if (!host) return;
  p->off_atom_off = ar.take(4 * (size_t)(g->n_ligands + 1));
  p->off_xyz = ar.take(12 * (size_t)sh.atoms);
  p->off_type = ar.take((size_t)sh.atoms);
  p->off_bonds = ar.take(8 * (size_t)(sh.atoms - g->n_ligands));
  p->off_rot_off = ar.take(4 * (size_t)(g->n_ligands + 1));
  p->off_rot_edge = ar.take(4 * (size_t)sh.rot);
}

int stage_ligands(const Arena& ar, const ligen_ligands_t* g, const LibShape& sh, const LigandPlan& p,
                  cudaStream_t s, LigandsDev* d) {
  d->L = g->n_ligands;
  if (!p.host) {
    d->atom_off = g->atom_off; d->xyz = g->xyz; d->type = g->type; d->bonds = g->bonds;
    d->rot_off = g->rot_off; d->rot_edge = g->rot_edge;
    return LIGEN_OK;
  }
  auto cp = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(ar.base + off, src, bytes, cudaMemcpyHostToDevice, s);
  };
  LG_CUDA(cp(p.off_atom_off, g->atom_off, 4 * (size_t)(g->n_ligands + 1)));
  LG_CUDA(cp(p.off_xyz, g->xyz, 12 * (size_t)sh.atoms));
  LG_CUDA(cp(p.off_type, g->type, (size_t)sh.atoms));
  LG_CUDA(cp(p.off_bonds, g->bonds, 8 * (size_t)(sh.atoms - g->n_ligands)));
  LG_CUDA(cp(p.off_rot_off, g->rot_off, 4 * (size_t)(g->n_ligands + 1)));
  LG_CUDA(cp(p.off_rot_edge, g->rot_edge, 4 * (size_t)sh.rot));
  d->atom_off = ar.at<int32_t>(p.off_atom_off);
  d->xyz = ar.at<float>(p.off_xyz);
  d->type = ar.at<uint8_t>(p.off_type);
  d->bonds = ar.at<int32_t>(p.off_bonds);
  d->rot_off = ar.at<int32_t>(p.off_rot_off);
  d->rot_edge = ar.at<int32_t>(p.off_rot_edge);
  return LIGEN_OK;
}

size_t grid_values_bytes(const ligen_grid_t* g) {
  return (size_t)g->nx * g->ny * g->nz * g->nc * sizeof(float);
}
size_t grid_coef_bytes(const ligen_grid_t* g, int fmt = kRecF32) {
  return rec_count(rec_cells(g->nx, fmt), rec_cells(g->ny, fmt), rec_cells(g->nz, fmt), g->nc) * rec_bytes(fmt);
}

GridView make_view(const ligen_grid_t* g, const float* coef, float penalty, int fmt = kRecF32) {
  GridView v;
  v.coef = coef;
  v.cx = rec_cells(g->nx, fmt); v.cy = rec_cells(g->ny, fmt); v.cz = rec_cells(g->nz, fmt);
  v.n_rec = rec_count(v.cx, v.cy, v.cz, g->nc);
  v.check = nullptr;
  v.nc = g->nc;
  v.mx = (float)(g->nx - 1); v.my = (float)(g->ny - 1); v.mz = (float)(g->nz - 1);
  v.penalty = penalty;
  return v;
}

// Checked builds (LIGEN_CHECKED): one device word per call collects the
// first out-of-range code any kernel of the call records (lg_check); the
// call waits for its work and turns a nonzero word into LIGEN_ERR_CHECK.
// Other builds take no word and wait for nothing.
struct CallCheck {
  size_t off = 0;
  unsigned* d = nullptr;
  void plan(Arena& ar) {
    if (LIGEN_CHECKED) off = ar.take(16);
  }
  int arm(Arena& ar, cudaStream_t s) {
    if (!LIGEN_CHECKED) return LIGEN_OK;
    d = ar.at<unsigned>(off);
    LG_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned), s));
    return LIGEN_OK;
  }
  int verdict(cudaStream_t s) {
    if (!LIGEN_CHECKED) return LIGEN_OK;
    unsigned h = 0;
    LG_CUDA(cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
    if (h) return fail(LIGEN_ERR_CHECK, "checked build: an out-of-range index was caught and skipped (code %u)", h);
    return LIGEN_OK;
  }
};

struct Timer {
  float* out;
  cudaStream_t s;
  cudaEvent_t ev[LIGEN_N_STAGES + 1] = {};
  int n = 0;
  Timer(float* o, cudaStream_t st) : out(o), s(st) {
    if (!out) return;
    for (auto& e : ev) cudaEventCreate(&e);
  }
  void mark() {
    if (out && n <= LIGEN_N_STAGES) cudaEventRecord(ev[n++], s);
  }
  void finish() {
    if (!out) return;
    while (n <= LIGEN_N_STAGES) mark();
    cudaEventSynchronize(ev[LIGEN_N_STAGES]);
    for (int i = 0; i < LIGEN_N_STAGES; ++i) cudaEventElapsedTime(&out[i], ev[i], ev[i + 1]);
  }
  ~Timer() {
    if (!out) return;
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

// Default launch shape: 8 lanes per restart, up to 16 restarts per CTA
// (measured on GB300: faster than 2 or 4 lanes for both small and large
// ligands; fewer registers and half the shared memory of 4 lanes per CTA).
constexpr int kDefaultLanes = 8;

int dock_restarts_per_cta(int R, int lanes) {
  const int per_warp = 32 / lanes;
  const int cap = 128 / lanes;
  int rpc = ((R + per_warp - 1) / per_warp) * per_warp;
  return rpc < cap ? rpc : cap;
}

// ------------------------------------------------------------- buckets --
// Paper §3: ligands are classified by atom count and rotamer count. Atom
// classes on warp multiples (<=32, <=64, <=128, larger); rotamer classes with
// upper edges 0,1,2,3,4,6,8,12,16,24,32 (finer at low counts).
int atom_class_of(int N) { return N <= 32 ? 0 : N <= 64 ? 1 : N <= 128 ? 2 : 3; }
int rot_class_of(int n) {
  static const int edges[11] = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
  for (int c = 0; c < 11; ++c)
    if (n <= edges[c]) return c;
  return 10;
}

constexpr int kMaxDev = 64;

struct TuneEntry {
  int lanes = kDefaultLanes;
  int rpc = 128 / kDefaultLanes;
};
std::mutex g_tune_mu;
TuneEntry g_tune[kMaxDev][LIGEN_N_BUCKETS];

bool valid_shape(int lanes, int rpc) {
  return dock_lanes_supported(lanes) && rpc >= 1 && rpc % (32 / lanes) == 0 && rpc * lanes <= 128;
}

// One persistent launch: ligands order[beg..end) with one kernel shape.
struct Group {
  int lanes = 0, rpc = 0;
  int beg = 0, end = 0;
  int max_atoms = 0, max_rot = 0, max_frag = 0;
  double cost = 0.0;
};

// Host plan of the bucketed layout: groups keyed by (atom class, tuned
// shape); inside a group ligands go by decreasing estimated cost
// (R * (n_rigid * N + passes * n * n_theta * N / 4)), and the groups by
// decreasing total cost, so the longest work starts first. `single`: one
// group of every ligand (the single-queue layout), default shape, in the
// same cost order. Four times the per-restart cost is an integer, so the
// order (group, cost descending, ligand index) comes from a stable
// counting sort in O(L) (the call waits for it before its first launch).
void plan_groups(const ligen_ligands_t* g, const ligen_params_t* p, int dev, std::vector<int32_t>& order,
                 std::vector<Group>& groups, bool single = false) {
  const int L = g->n_ligands;
  const int nt = 360 / p->torsion_step_deg;
  // the group key (atom class, lanes, restarts per CTA) of every bucket,
  // groups numbered in key order
  std::tuple<int, int, int> bkey[LIGEN_N_BUCKETS];
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int b = 0; b < LIGEN_N_BUCKETS; ++b) {
      TuneEntry t = single ? TuneEntry() : g_tune[dev][b];
      if (!dock_shape_supported(t.lanes, p->grid_format)) t = TuneEntry();   // default shape
      bkey[b] = std::make_tuple(single ? 0 : b / 11, t.lanes, t.rpc);
    }
  }
  std::vector<std::tuple<int, int, int>> keys(bkey, bkey + LIGEN_N_BUCKETS);
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  int bgid[LIGEN_N_BUCKETS];
  for (int b = 0; b < LIGEN_N_BUCKETS; ++b)
    bgid[b] = (int)(std::lower_bound(keys.begin(), keys.end(), bkey[b]) - keys.begin());
  const int G = (int)keys.size();
  std::vector<uint32_t> inv(L);   // 2^32 - 1 - 4 x cost: ascending = cost descending
  std::vector<uint8_t> gid(L);
  for (int l = 0; l < L; ++l) {
    const int N = g->h_atom_off[l + 1] - g->h_atom_off[l];
    const int n = g->h_rot_off[l + 1] - g->h_rot_off[l];
    const uint64_t c4 = 4ull * N * p->n_rigid + (uint64_t)p->passes * n * nt * (N + 4);
    inv[l] = 0xffffffffu - (uint32_t)std::min<uint64_t>(c4, 0xffffffffull);
    gid[l] = (uint8_t)bgid[atom_class_of(N) * 11 + rot_class_of(n)];
  }
  // LSD: the cost key's low and high 16 bits, then the group (each pass stable)
  std::vector<int32_t> a(L), b(L);
  for (int l = 0; l < L; ++l) a[l] = l;
  auto pass = [&](int buckets, auto digit) {
    std::vector<int> cnt((size_t)buckets + 1, 0);
    for (int i = 0; i < L; ++i) ++cnt[digit(a[i]) + 1];
    for (int k = 0; k < buckets; ++k) cnt[k + 1] += cnt[k];
    for (int i = 0; i < L; ++i) b[cnt[digit(a[i])]++] = a[i];
    a.swap(b);
  };
  pass(1 << 16, [&](int l) { return (int)(inv[l] & 0xffffu); });
  pass(1 << 16, [&](int l) { return (int)(inv[l] >> 16); });
  pass(G, [&](int l) { return (int)gid[l]; });
  order.assign(a.begin(), a.end());
  groups.clear();
  for (int i = 0; i < L;) {
    const int k = gid[order[i]];
    Group gr;
    gr.lanes = std::get<1>(keys[k]);
    gr.rpc = std::get<2>(keys[k]);
    gr.beg = i;
    uint64_t c4sum = 0;
    for (; i < L && gid[order[i]] == k; ++i) {
      const int l = order[i];
      const int N = g->h_atom_off[l + 1] - g->h_atom_off[l];
      const int n = g->h_rot_off[l + 1] - g->h_rot_off[l];
      gr.max_atoms = std::max(gr.max_atoms, N);
      gr.max_rot = std::max(gr.max_rot, n);
      gr.max_frag = std::max(gr.max_frag, n * (N / 2));
      c4sum += 0xffffffffu - inv[l];
    }
    gr.end = i;
    gr.cost = 0.25 * (double)c4sum;
    groups.push_back(gr);
  }
  std::stable_sort(groups.begin(), groups.end(), [](const Group& x, const Group& y) { return x.cost > y.cost; });
}

// Side streams and events for the forked launches, per (device, calling
// stream): calls in flight on different streams fork onto different side
// streams and record different events (calls on one stream are ordered).
struct Fork {
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t start = nullptr;
};
std::mutex g_fork_mu;
std::map<std::pair<int, cudaStream_t>, Fork> g_fork;
std::map<std::pair<int, cudaStream_t>, Fork> g_fence;   // capture streams for uncapturable streams

int get_fork(int dev, cudaStream_t s, int n, Fork** out, bool fence = false) {
  std::lock_guard<std::mutex> lk(g_fork_mu);
  Fork& f = (fence ? g_fence : g_fork)[{dev, s}];
  if (!f.start) LG_CUDA(cudaEventCreateWithFlags(&f.start, cudaEventDisableTiming));
  while ((int)f.streams.size() < n) {
    cudaStream_t st;
    cudaEvent_t ev;
    LG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    LG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    f.streams.push_back(st);
    f.done.push_back(ev);
  }
  *out = &f;
  return LIGEN_OK;
}

// Instantiated graphs of the bucketed launch sequence, keyed by everything
// the launches capture by value (pointers, sizes, shapes, grid sizes).
struct GraphEntry {
  std::string key;
  cudaGraphExec_t exec;
};
std::mutex g_graph_mu;
std::map<std::pair<int, cudaStream_t>, std::vector<GraphEntry>> g_graphs;
constexpr size_t kGraphsPerStream = 16;

void append_key(std::string& k, const void* p, size_t n) { k.append((const char*)p, n); }

std::string launch_key(const std::vector<DockArgs>& args, const std::vector<int>& ctas) {
  std::string k;
  for (size_t i = 0; i < args.size(); ++i) {
    const DockArgs& a = args[i];
    const void* ptrs[] = {a.lig.atom_off, a.lig.xyz, a.lig.type, a.lig.bonds, a.lig.rot_off, a.lig.rot_edge,
                          a.pk.xc, a.pk.binfo, a.pk.frag, a.pk.status, a.grid.coef, a.res_score, a.res_k,
                          a.res_cnt, a.trace, a.list, a.queue, a.samples, a.pk.touch, a.grid.check,
                          a.coords};
    append_key(k, ptrs, sizeof ptrs);
    const int ints[] = {a.lig.L, a.grid.cx, a.grid.cy, a.grid.cz, a.grid.nc, a.R, a.n_rigid, a.step_deg,
                        a.n_theta, a.passes, a.lanes, a.fmt, a.rpc, a.chunks, a.n_items, a.max_atoms,
                        a.max_rot, a.max_frag, ctas[i]};
    append_key(k, ints, sizeof ints);
    const float fl[] = {a.origin[0], a.origin[1], a.origin[2], a.inv_h, a.center[0], a.center[1], a.center[2],
                        a.jitter, a.grid.penalty, a.grid.mx, a.grid.my, a.grid.mz};
    append_key(k, fl, sizeof fl);
    append_key(k, &a.seed, sizeof a.seed);
  }
  return k;
}

// Issue the groups' launches: one CTA per work item (static) forked from
// `s` onto side streams and joined back, so one group's last wave overlaps
// the next group's CTAs; persistent launches one after another on `s`.
// Measured on GB300 (bimodal200k, docking kernel per call): persistent
// groups forked 840 ms, in order on one stream 832 ms; static groups forked
// 829.5 ms, on one stream 830.7 ms. A persistent group's CTAs hold their
// slots until its queue is empty, so side by side the groups only share the
// SMs worse.
int issue_groups(const std::vector<DockArgs>& args, const std::vector<int>& ctas, int dev, bool persistent,
                 cudaStream_t s) {
  if (persistent) {
    for (size_t i = 0; i < args.size(); ++i) {
      if (args[i].queue) LG_CUDA(cudaMemsetAsync(args[i].queue, 0, sizeof(int), s));
      LG_CUDA(launch_dock(args[i], ctas[i], s, false));
    }
    return LIGEN_OK;
  }
  Fork* f = nullptr;
  int rc = get_fork(dev, s, (int)args.size(), &f);
  if (rc != LIGEN_OK) return rc;
  LG_CUDA(cudaEventRecord(f->start, s));
  for (size_t i = 0; i < args.size(); ++i) {
    cudaStream_t st = f->streams[i];
    LG_CUDA(cudaStreamWaitEvent(st, f->start, 0));
    if (args[i].queue) LG_CUDA(cudaMemsetAsync(args[i].queue, 0, sizeof(int), st));
    LG_CUDA(launch_dock(args[i], ctas[i], st, false));
    LG_CUDA(cudaEventRecord(f->done[i], st));
    LG_CUDA(cudaStreamWaitEvent(s, f->done[i], 0));
  }
  return LIGEN_OK;
}

// issue(stream) replayed from a cached CUDA graph keyed by `key` (every
// pointer, size and shape the launches capture by value) and by the calling
// stream, captured on its first use: on `s`, or, where `s` cannot be
// captured (the legacy or per-thread default stream), on a side stream
// (capture runs nothing, so it needs no ordering with `s`). Every call then
// launches the graph on `s` itself. When `s` is already capturing, the
// launches are issued into the caller's graph.
template <class F>
int run_graphed(int dev, cudaStream_t s, const std::string& key, F&& issue) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  LG_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return issue(s);
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto& e : g_graphs[{dev, s}])
      if (e.key == key) exec = e.exec;
  }
  if (!exec) {
    cudaStream_t cap = s;
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) {
      Fork* f = nullptr;
      int rc = get_fork(dev, s, 1, &f, true);
      if (rc != LIGEN_OK) return rc;
      cap = f->streams[0];
    }
    LG_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    int rc = issue(cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    if (rc != LIGEN_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    std::lock_guard<std::mutex> lk(g_graph_mu);
    auto& v = g_graphs[{dev, s}];
    if (v.size() >= kGraphsPerStream) {
      cudaGraphExecDestroy(v.front().exec);
      v.erase(v.begin());
    }
    v.push_back({key, exec});
  }
  LG_CUDA(cudaGraphLaunch(exec, s));
  return LIGEN_OK;
}

// The bucketed layout: one persistent launch per group, sized by Eq. 1
// (b blocks per SM from the occupancy query, times the SM count), or with
// `persistent` false one CTA per work item; run from a cached CUDA graph
// (run_graphed).
int run_bucketed(const DockArgs& base, const std::vector<Group>& groups, int32_t* d_order, int* d_queue,
                 bool persistent, cudaStream_t s) {
  int dev = 0, nsm = 0;
  LG_CUDA(cudaGetDevice(&dev));
  LG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // one dynamic shared-memory limit per kernel shape: the largest its groups need
  std::map<int, size_t> limit;
  for (const Group& gr : groups) {
    const size_t smem = dock_smem_bytes(gr.max_atoms, gr.max_rot, gr.max_frag, gr.rpc);
    size_t& l = limit[gr.lanes];
    l = std::max(l, smem);
  }
  for (const auto& kv : limit) LG_CUDA(dock_set_smem_limit(kv.first, base.n_theta, base.fmt, kv.second));
  std::vector<DockArgs> args;
  std::vector<int> ctas;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const Group& gr = groups[gi];
    DockArgs a = base;
    a.lanes = gr.lanes;
    a.rpc = gr.rpc;
    a.chunks = (a.R + a.rpc - 1) / a.rpc;
    a.list = d_order + gr.beg;
    a.n_items = (gr.end - gr.beg) * a.chunks;
    a.queue = persistent ? d_queue + gi : nullptr;
    a.max_atoms = gr.max_atoms;
    a.max_rot = gr.max_rot;
    a.max_frag = gr.max_frag;
    const size_t smem = dock_smem_bytes(a.max_atoms, a.max_rot, a.max_frag, a.rpc);
    int b = 0;
    LG_CUDA(dock_occupancy(a.lanes, a.n_theta, a.fmt, a.rpc, smem, &b));
    if (b < 1) return fail(LIGEN_ERR_UNSUPPORTED, "no CTA of shape (%d lanes, %d restarts) fits an SM", a.lanes, a.rpc);
    ctas.push_back(persistent ? (int)std::min<int64_t>((int64_t)b * nsm, a.n_items) : a.n_items);
    args.push_back(a);
  }
  return run_graphed(dev, s, launch_key(args, ctas),
                     [&](cudaStream_t st) { return issue_groups(args, ctas, dev, persistent, st); });
}

// ------------------------------------------------------------- scoring --
// Calls with at least kLanePosesMin poses per ligand score one pose per lane
// (launch_score_lanes), ligands grouped by rotatable-bond count: that
// kernel keeps n + 1 rigid transforms per lane (1.5 KB per warp each) in
// shared memory, so ligands with few bonds are not charged for the most
// flexible one. Fewer poses per ligand leave most lanes of such a warp
// idle; those calls keep the group-per-pose kernel (launch_score).
constexpr int kLanePosesMin = 16;
constexpr int kScoreClasses = 9;
constexpr int kScoreRotCap[kScoreClasses] = {0, 2, 4, 6, 8, 12, 16, 24, 32};

int score_class_of(int n) {
  int c = 0;
  while (c + 1 < kScoreClasses && n > kScoreRotCap[c]) ++c;
  return c;
}

struct ScorePlan {
  int n[kScoreClasses] = {};        // ligands per class
  int start[kScoreClasses] = {};    // first entry of the class in `list`
  std::vector<int32_t> list;        // ligand ids, class by class, ascending within a class
};

// (Within a class, ligands in decreasing atom count instead of index order
// measured the same on GB300: 0.169 against 0.166 ms for the 600,000 kept
// screening poses, 8.87 against 8.75 ms for their refinement.)
void plan_score(const int32_t* h_rot_off, int L, ScorePlan* sp) {
  int cnt[kScoreClasses] = {};
  for (int l = 0; l < L; ++l) ++cnt[score_class_of(h_rot_off[l + 1] - h_rot_off[l])];
  int o = 0;
  for (int c = 0; c < kScoreClasses; ++c) {
    sp->n[c] = cnt[c];
    sp->start[c] = o;
    o += cnt[c];
  }
  sp->list.assign(L, 0);
  int fill[kScoreClasses];
  std::copy(sp->start, sp->start + kScoreClasses, fill);
  for (int l = 0; l < L; ++l) sp->list[fill[score_class_of(h_rot_off[l + 1] - h_rot_off[l])]++] = l;
}

// Regions of the forward-kinematics table (Packed::fk_*) in an arena.
struct FkRegions {
  size_t xs = 0, own = 0, bond = 0, ax = 0, loff = 0;
};

FkRegions take_fk(Arena& ar, const LibShape& sh, int L) {
  FkRegions r;
  r.xs = ar.take(16 * (size_t)sh.atoms);
  r.own = ar.take((size_t)sh.atoms);
  r.bond = ar.take(4 * (size_t)sh.rot);
  r.ax = ar.take(16 * (size_t)sh.rot);
  r.loff = ar.take((size_t)kFkLoffBytes * L);
  return r;
}

void set_fk(const Arena& ar, const FkRegions& r, Packed* pk) {
  pk->fk_xs = ar.at<float4>(r.xs);
  pk->fk_own = ar.at<uint8_t>(r.own);
  pk->fk_bond = ar.at<uchar4>(r.bond);
  pk->fk_ax = ar.at<float4>(r.ax);
  pk->fk_loff = ar.at<uint8_t>(r.loff);
}

// The launches launch(i, stream), i = 0 .. n-1, forked from `s` onto side
// streams and joined back (on `s` itself when n == 1), so that the classes'
// launches run side by side and one's ragged last wave overlaps another's
// work. Measured on GB300 against the same launches one after another on
// `s`: scoring the 600,000 kept screening poses (7 classes) 0.251 -> 0.166
// ms, refining the top 16 poses of 20,000 ligands (50 steps) 13.4 -> 8.75
// ms, their gradients 0.87 -> 0.70 ms.
template <class F>
int run_forked(int n, cudaStream_t s, F&& launch) {
  if (n == 1) {
    LG_CUDA(launch(0, s));
    return LIGEN_OK;
  }
  if (n < 1) return LIGEN_OK;
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  Fork* f = nullptr;
  int rc = get_fork(dev, s, n, &f);
  if (rc != LIGEN_OK) return rc;
  LG_CUDA(cudaEventRecord(f->start, s));
  for (int i = 0; i < n; ++i) {
    cudaStream_t st = f->streams[i];
    LG_CUDA(cudaStreamWaitEvent(st, f->start, 0));
    LG_CUDA(launch(i, st));
    LG_CUDA(cudaEventRecord(f->done[i], st));
    LG_CUDA(cudaStreamWaitEvent(s, f->done[i], 0));
  }
  return LIGEN_OK;
}

// The plan's non-empty classes, most bonds (longest warps) first.
int used_classes(const ScorePlan& sp, int* used) {
  int nu = 0;
  for (int c = kScoreClasses - 1; c >= 0; --c)
    if (sp.n[c]) used[nu++] = c;
  return nu;
}

std::string score_key(const ScoreArgs& b, const int32_t* d_list, const int* used, int nu, const LaunchCfg* cfg,
                      const ScorePlan& sp) {
  std::string k;
  const void* ptrs[] = {b.lig.atom_off, b.lig.rot_off, b.pk.xc,     b.pk.binfo,  b.pk.frag,    b.pk.status,
                        b.pk.fk_xs,     b.pk.fk_own,   b.pk.fk_bond, b.pk.fk_ax, b.pk.fk_loff, b.grid.coef,
                        b.grid.check,   b.poses,       b.out_scores, d_list};
  append_key(k, ptrs, sizeof ptrs);
  const int ints[] = {b.lig.L, b.grid.cx, b.grid.cy, b.grid.cz, b.grid.nc, b.P, b.max_atoms, nu};
  append_key(k, ints, sizeof ints);
  const float fl[] = {b.grid.mx, b.grid.my, b.grid.mz, b.grid.penalty, b.origin[0], b.origin[1], b.origin[2], b.inv_h};
  append_key(k, fl, sizeof fl);
  append_key(k, &b.grid.n_rec, sizeof b.grid.n_rec);
  for (int i = 0; i < nu; ++i) {
    const int c = used[i];
    const int ci[] = {c, sp.start[c], sp.n[c], (int)cfg[i].blocks};
    append_key(k, ci, sizeof ci);
    append_key(k, &cfg[i].smem, sizeof cfg[i].smem);
  }
  return k;
}

// Every ligand of base.lig scored: class by class, the classes' launches
// side by side (d_list = the plan's list on the device; base.max_atoms the
// call's largest ligand) and replayed from a cached CUDA graph, or in one
// group-per-pose launch.
int run_score(const ScoreArgs& base, const ScorePlan& sp, const int32_t* d_list, cudaStream_t s) {
  if (base.P < kLanePosesMin) {   // reads the moving-atom lists
    if (!base.pk.frag) return fail(LIGEN_ERR_CUDA, "internal: scoring without the moving-atom lists");
    LG_CUDA(launch_score(base, s));
    return LIGEN_OK;
  }
  if (!base.pk.fk_xs || !base.pk.fk_own || !base.pk.fk_bond || !base.pk.fk_ax || !base.pk.fk_loff)
    return fail(LIGEN_ERR_CUDA, "internal: pose-per-lane scoring without the forward-kinematics table");
  int used[kScoreClasses];
  const int nu = used_classes(sp, used);
  ScoreArgs args[kScoreClasses];
  LaunchCfg cfg[kScoreClasses];
  for (int i = 0; i < nu; ++i) {
    const int c = used[i];
    args[i] = base;
    args[i].list = d_list + sp.start[c];
    args[i].n_list = sp.n[c];
    args[i].max_rot = kScoreRotCap[c];
    LG_CUDA(score_lanes_config(args[i], &cfg[i]));
  }
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  return run_graphed(dev, s, score_key(base, d_list, used, nu, cfg, sp), [&](cudaStream_t gs) {
    return run_forked(nu, gs, [&](int i, cudaStream_t st) { return launch_score_lanes(args[i], cfg[i], st); });
  });
}

}  // namespace

// Inputs prepared once for repeated scoring (ligen_prepare_scoring): the
// FP32 grid records, the packed library and the scoring plan, in one
// device allocation owned by the handle.
struct ligen_prepared {
  int dev = 0;
  char* mem = nullptr;
  LigandsDev lig{};
  Packed pk{};
  float* coef = nullptr;
  ligen_grid_t grid{};          // dimensions, origin, spacing (data not kept)
  LibShape sh;
  std::vector<int32_t> h_atom_off, h_rot_off;
  ScorePlan plan;
  int32_t* d_list = nullptr;
};

extern "C" {

int ligen_abi_version(void) { return LIGEN_ABI_VERSION; }

int ligen_set_workspace_limit(int64_t bytes) {
  g_ws_limit.store(bytes > 0 ? (size_t)bytes : 0);
  return LIGEN_OK;
}

const char* ligen_last_error(void) { return g_err.c_str(); }

int ligen_release_workspaces(void) {
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> gl(g_graph_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
      if (it->first.first == dev) {
        for (auto& e : it->second) cudaGraphExecDestroy(e.exec);
        it = g_graphs.erase(it);
      } else {
        ++it;
      }
    }
  }
  {   // side streams and events of the forked launches (a captured graph keeps no reference to them)
    std::lock_guard<std::mutex> fl(g_fork_mu);
    for (auto* m : {&g_fork, &g_fence}) {
      for (auto it = m->begin(); it != m->end();) {
        if (it->first.first == dev) {
          for (cudaStream_t st : it->second.streams) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
          }
          for (cudaEvent_t ev : it->second.done) cudaEventDestroy(ev);
          if (it->second.start) cudaEventDestroy(it->second.start);
          it = m->erase(it);
        } else {
          ++it;
        }
      }
    }
  }
  std::lock_guard<std::mutex> lk(g_ws_mu);
  for (auto it = g_ws.begin(); it != g_ws.end();) {
    if (it->first.first == dev) {
      cudaStreamSynchronize(it->first.second);
      cudaFree(it->second.base);
      it = g_ws.erase(it);
    } else {
      ++it;
    }
  }
  return LIGEN_OK;
}

// Docking of one library into n_sites grids (n_sites = 1: ligen_dock_batch).
// The library is staged and packed once; per site the grid records are built
// in one shared buffer, then docking, top-K and the optional FP64 re-score
// write that site's slice of every output.
static int dock_impl(const ligen_ligands_t* ligands, const ligen_grid_t* grids, int n_sites,
                     const ligen_params_t* params, float* out_poses, float* out_scores) {
  g_err.clear();
  int rc;
  if ((rc = check_params(params)) != LIGEN_OK) return rc;
  LibShape sh;
  if ((rc = check_ligands(ligands, params->passes, &sh)) != LIGEN_OK) return rc;
  if (!grids || n_sites < 1) return fail(LIGEN_ERR_INVALID_ARG, "grids is NULL or n_sites < 1");
  for (int g = 0; g < n_sites; ++g) {
    if ((rc = check_grid(&grids[g])) != LIGEN_OK) return rc;
    if (grids[g].nc != grids[0].nc) return fail(LIGEN_ERR_INVALID_ARG, "all sites need the same channel count");
  }
  const int L = ligands->n_ligands;
  if (L == 0) return LIGEN_OK;   // nothing to dock; outputs may be empty (NULL)
  if (!out_poses || !out_scores) return fail(LIGEN_ERR_INVALID_ARG, "out_poses and out_scores are required");
  cudaStream_t s = (cudaStream_t)params->stream;
  const int R = params->restarts, K = params->top_k, P = params->passes;
  const bool exhaustive = params->mode == 1;
  if (exhaustive && (rc = check_exhaustive(ligands, params)) != LIGEN_OK) return rc;

  const int lhost = space_of({ligands->atom_off, ligands->xyz, ligands->type, ligands->bonds,
                              ligands->rot_off, ligands->rot_edge});
  int ghost = -2;
  for (int g = 0; g < n_sites; ++g) {
    const int gh = space_of({grids[g].data});
    if (ghost == -2) ghost = gh;
    else if (gh != ghost) return fail(LIGEN_ERR_INVALID_ARG, "site grids mix host and device memory");
  }
  const int ohost = space_of({out_poses, out_scores, params->status, params->trace, params->top_restart,
                              params->scores_f64, params->coords});
  if (lhost < 0) return fail(LIGEN_ERR_INVALID_ARG, "ligand arrays mix host and device memory");
  if (ohost < 0) return fail(LIGEN_ERR_INVALID_ARG, "output arrays mix host and device memory");

  const size_t pose_floats = (size_t)K * (7 * (size_t)L + sh.rot);
  const size_t trace_elems = (size_t)R * sh.trace_len;
  const size_t coord_elems = 3 * (size_t)R * sh.atoms;
  const int fmt = params->grid_format;
  size_t gval_max = 0, coef_max = 0;
  for (int g = 0; g < n_sites; ++g) {
    gval_max = std::max(gval_max, grid_values_bytes(&grids[g]));
    coef_max = std::max(coef_max, grid_coef_bytes(&grids[g], fmt));
  }
  Arena ar;
  LigandPlan lp;
  plan_ligands(ar, ligands, sh, lhost == 1, &lp);
  const size_t o_gval = ghost ? ar.take(gval_max) : 0;
  const size_t o_coef = ar.take(coef_max);
  const size_t o_xc = ar.take(16 * (size_t)sh.atoms);
  const size_t o_binfo = ar.take(4 * (size_t)sh.rot);
  const size_t o_frag = ar.take((size_t)kFragStride * sh.rot);
  const size_t o_touch = ar.take(4 * (size_t)sh.rot);
  const size_t o_status = ar.take(4 * (size_t)L);
  const size_t o_rs = ar.take(4 * (size_t)L * R);
  const size_t o_rk = ar.take((size_t)L * R);
  const size_t o_rc = ar.take((size_t)sh.rot * R);
  size_t o_poses = 0, o_scores = 0, o_trace = 0, o_top = 0, o_coords = 0;
  if (ohost == 1) {
    o_poses = ar.take(4 * pose_floats);
    o_scores = ar.take(4 * (size_t)L * K);
    if (params->trace) o_trace = ar.take(2 * trace_elems);
    if (params->coords) o_coords = ar.take(4 * coord_elems);
    if (params->top_restart) o_top = ar.take(4 * (size_t)L * K);
  }
  const bool rescore = params->rescore_fp64 == 1;
  size_t o_itop = 0, o_tmp_poses = 0, o_tmp_top = 0, o_s64 = 0, o_out64 = 0;
  if (rescore) {
    if (!params->top_restart) o_itop = ar.take(4 * (size_t)L * K);   // restart ids for tie-breaks
    o_tmp_poses = ar.take(4 * pose_floats);
    o_tmp_top = ar.take(4 * (size_t)L * K);
    o_s64 = ar.take(8 * (size_t)L * K);
    if (params->scores_f64 && ohost) o_out64 = ar.take(8 * (size_t)L * K);
  }
  const bool buckets = params->batching != LIGEN_BATCH_PLAIN && !exhaustive;
  std::vector<int32_t> order;
  std::vector<Group> groups;
  size_t o_order = 0, o_queue = 0;
  int plan_dev = 0;
  if (buckets) {   // the plan itself is made after the first launches (below)
    LG_CUDA(cudaGetDevice(&plan_dev));
    if (plan_dev >= kMaxDev) return fail(LIGEN_ERR_UNSUPPORTED, "device ordinal %d >= %d", plan_dev, kMaxDev);
    o_order = ar.take(4 * (size_t)L);
    o_queue = ar.take(sizeof(int) * LIGEN_N_BUCKETS);   // at most one group per bucket
  }
  const size_t o_samples = params->samples ? ar.take(8 * (size_t)kSampleSlots) : 0;
  CallCheck chk;
  chk.plan(ar);
  if ((rc = get_workspace(s, ar.used, &ar.base)) != LIGEN_OK) return rc;
  if ((rc = chk.arm(ar, s)) != LIGEN_OK) return rc;
  unsigned long long* d_samples = nullptr;
  if (params->samples) {
    d_samples = ar.at<unsigned long long>(o_samples);
    LG_CUDA(cudaMemsetAsync(d_samples, 0, 8 * (size_t)kSampleSlots, s));
  }

  // stage times accumulate over the sites
  float stage_acc[LIGEN_N_STAGES] = {0.f, 0.f, 0.f, 0.f, 0.f};
  float* stage_out = params->stage_ms;
  LigandsDev lig;
  Packed pk{};
  pk.xc = ar.at<float4>(o_xc);
  pk.binfo = ar.at<uchar4>(o_binfo);
  pk.frag = ar.at<uint8_t>(o_frag);
  pk.touch = ar.at<uint32_t>(o_touch);
  pk.status = ar.at<int32_t>(o_status);
  const cudaMemcpyKind back = ohost ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;

  for (int site = 0; site < n_sites; ++site) {
    const ligen_grid_t* grid = &grids[site];
    float* site_poses = out_poses + (size_t)site * pose_floats;
    float* site_scores = out_scores + (size_t)site * L * K;
    int16_t* site_trace = params->trace ? params->trace + (size_t)site * trace_elems : nullptr;
    float* site_coords = params->coords ? params->coords + (size_t)site * coord_elems : nullptr;
    int32_t* site_top = params->top_restart ? params->top_restart + (size_t)site * L * K : nullptr;
    double* site_s64 = params->scores_f64 ? params->scores_f64 + (size_t)site * L * K : nullptr;
    float site_ms[LIGEN_N_STAGES];
    Timer tm(stage_out ? site_ms : nullptr, s);
    tm.mark();
    if (site == 0) {
      if ((rc = stage_ligands(ar, ligands, sh, lp, s, &lig)) != LIGEN_OK) return rc;
    }
    const float* gvals = (const float*)grid->data;
    if (ghost) {
      LG_CUDA(cudaMemcpyAsync(ar.base + o_gval, grid->data, grid_values_bytes(grid), cudaMemcpyHostToDevice, s));
      gvals = ar.at<float>(o_gval);
    }
    tm.mark();
    float* coef = ar.at<float>(o_coef);
    LG_CUDA(launch_grid_prep_fmt(gvals, grid->nx, grid->ny, grid->nz, grid->nc, fmt, coef, s));
    tm.mark();
    if (site == 0) LG_CUDA(launch_pack(lig, grid->nc, pk, s));
    tm.mark();

    float* d_poses = ohost ? ar.at<float>(o_poses) : site_poses;
    float* d_scores = ohost ? ar.at<float>(o_scores) : site_scores;
    int16_t* d_trace = site_trace ? (ohost ? ar.at<int16_t>(o_trace) : site_trace) : nullptr;
    float* d_coords = site_coords ? (ohost ? ar.at<float>(o_coords) : site_coords) : nullptr;
    int32_t* d_top = site_top ? (ohost ? ar.at<int32_t>(o_top) : site_top) : nullptr;
    if (rescore && !d_top) d_top = ar.at<int32_t>(o_itop);

    DockArgs da{};
    da.lig = lig;
    da.pk = pk;
    da.grid = make_view(grid, coef, params->out_penalty, fmt);
    da.grid.check = chk.d;
    const float h = grid->spacing;
    const int np[3] = {grid->nx, grid->ny, grid->nz};
    for (int k = 0; k < 3; ++k) {
      da.origin[k] = grid->origin[k];
      da.center[k] = (float)((double)grid->origin[k] + (double)h * (np[k] - 1) / 2.0);
    }
    da.inv_h = (float)(1.0 / (double)h);
    da.jitter = params->jitter;
    da.seed = params->seed;
    da.R = R;
    da.n_rigid = params->n_rigid;
    da.step_deg = params->torsion_step_deg;
    da.n_theta = 360 / params->torsion_step_deg;
    da.passes = P;
    da.lanes = kDefaultLanes;
    da.fmt = fmt;
    da.rpc = dock_restarts_per_cta(R, da.lanes);
    da.chunks = (R + da.rpc - 1) / da.rpc;
    da.list = nullptr;
    da.n_items = L * da.chunks;
    da.queue = nullptr;
    da.max_atoms = sh.max_atoms;
    da.max_rot = sh.max_rot;
    da.max_frag = (int)sh.max_frag;
    da.res_score = ar.at<float>(o_rs);
    da.res_k = ar.at<uint8_t>(o_rk);
    da.res_cnt = ar.at<uint8_t>(o_rc);
    da.trace = d_trace;
    da.coords = d_coords;
    da.samples = d_samples;
    if (exhaustive) {
      LG_CUDA(launch_exhaustive(da, s));
    } else if (buckets) {
      // Uploaded on every call: any other call on this stream may have
      // carved the workspace differently and overwritten this region (a
      // grid of another record format, for one). Pageable source: the copy
      // is staged before cudaMemcpyAsync returns.
      // planned here, on the first site, while the grid records and the
      // packer run on the device
      if (groups.empty()) plan_groups(ligands, params, plan_dev, order, groups, params->batching == LIGEN_BATCH_QUEUE);
      int32_t* d_order = ar.at<int32_t>(o_order);
      LG_CUDA(cudaMemcpyAsync(d_order, order.data(), 4 * order.size(), cudaMemcpyHostToDevice, s));
      if ((rc = run_bucketed(da, groups, d_order, ar.at<int>(o_queue),
                             params->batching != LIGEN_BATCH_BUCKETS_STATIC, s)) != LIGEN_OK)
        return rc;
    } else {
      LG_CUDA(launch_dock(da, 0, s, true));
    }
    tm.mark();

    TopkArgs ta{};
    ta.L = L; ta.R = R; ta.K = K; ta.step_deg = params->torsion_step_deg;
    ta.rot_off = lig.rot_off;
    ta.status = pk.status;
    ta.res_score = da.res_score; ta.res_k = da.res_k; ta.res_cnt = da.res_cnt;
    ta.seed = params->seed;
    for (int k = 0; k < 3; ++k) ta.center[k] = da.center[k];
    ta.jitter = params->jitter;
    ta.out_poses = d_poses;
    ta.out_scores = d_scores;
    ta.top_restart = d_top;
    LG_CUDA(launch_topk(ta, s));
    double* d_out64 = nullptr;
    if (rescore) {
      d_out64 = site_s64 ? (ohost ? ar.at<double>(o_out64) : site_s64) : nullptr;
      LG_CUDA(cudaMemcpyAsync(ar.base + o_tmp_poses, d_poses, 4 * pose_floats, cudaMemcpyDeviceToDevice, s));
      LG_CUDA(cudaMemcpyAsync(ar.base + o_tmp_top, d_top, 4 * (size_t)L * K, cudaMemcpyDeviceToDevice, s));
      RescoreArgs rsa{};
      rsa.lig = lig;
      rsa.pk = pk;
      rsa.status = pk.status;
      rsa.values = gvals;
      rsa.nx = grid->nx; rsa.ny = grid->ny; rsa.nz = grid->nz; rsa.nc = grid->nc;
      for (int k = 0; k < 3; ++k) rsa.origin[k] = grid->origin[k];
      rsa.h = grid->spacing;
      rsa.penalty = params->out_penalty;
      rsa.K = K;
      rsa.max_atoms = sh.max_atoms;
      rsa.max_rot = sh.max_rot;
      rsa.poses = d_poses;
      rsa.scores = d_scores;
      rsa.top_restart = site_top ? d_top : nullptr;
      rsa.out_s64 = d_out64;
      rsa.s64 = ar.at<double>(o_s64);
      rsa.tmp_poses = ar.at<float>(o_tmp_poses);
      rsa.tmp_top = ar.at<int32_t>(o_tmp_top);
      rsa.check = chk.d;
      LG_CUDA(launch_rescore(rsa, s));
    }

    if (site == 0 && params->status)
      LG_CUDA(cudaMemcpyAsync(params->status, pk.status, 4 * (size_t)L, back, s));
    if (ohost) {
      LG_CUDA(cudaMemcpyAsync(site_poses, d_poses, 4 * pose_floats, back, s));
      LG_CUDA(cudaMemcpyAsync(site_scores, d_scores, 4 * (size_t)L * K, back, s));
      if (d_trace) LG_CUDA(cudaMemcpyAsync(site_trace, d_trace, 2 * trace_elems, back, s));
      if (d_coords) LG_CUDA(cudaMemcpyAsync(site_coords, d_coords, 4 * coord_elems, back, s));
      if (site_top) LG_CUDA(cudaMemcpyAsync(site_top, d_top, 4 * (size_t)L * K, back, s));
      if (d_out64) LG_CUDA(cudaMemcpyAsync(site_s64, d_out64, 8 * (size_t)L * K, back, s));
    }
    tm.mark();
    tm.finish();
    if (stage_out)
      for (int k = 0; k < LIGEN_N_STAGES; ++k) stage_acc[k] += site_ms[k];
    // The next site reuses the staging and record buffers; stream order
    // keeps its writes behind this site's reads, so no host wait is needed.
  }
  if (stage_out)
    for (int k = 0; k < LIGEN_N_STAGES; ++k) stage_out[k] = stage_acc[k];
  if (params->samples) {
    unsigned long long h[kSampleSlots];
    LG_CUDA(cudaMemcpyAsync(h, d_samples, sizeof h, cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
    unsigned long long total = 0;
    for (int k = 0; k < kSampleSlots; ++k) total += h[k];
    *params->samples = (int64_t)total;
  }
  if (ohost) LG_CUDA(cudaStreamSynchronize(s));
  return chk.verdict(s);
}

int ligen_dock_batch(const ligen_ligands_t* ligands, const ligen_grid_t* grid, const ligen_params_t* params,
                     float* out_poses, float* out_scores) {
  g_err.clear();
  if (!grid) return fail(LIGEN_ERR_INVALID_ARG, "grid is NULL");
  return dock_impl(ligands, grid, 1, params, out_poses, out_scores);
}

int ligen_dock_sites(const ligen_ligands_t* ligands, const ligen_grid_t* grids, int32_t n_sites,
                     const ligen_params_t* params, float* out_poses, float* out_scores) {
  return dock_impl(ligands, grids, n_sites, params, out_poses, out_scores);
}

int ligen_score_poses(const ligen_ligands_t* ligands, const ligen_grid_t* grid, int32_t poses_per_ligand,
                      const float* poses, float out_penalty, float* out_scores, void* stream) {
  g_err.clear();
  int rc;
  LibShape sh;
  if ((rc = check_ligands(ligands, 0, &sh)) != LIGEN_OK) return rc;
  if ((rc = check_grid(grid)) != LIGEN_OK) return rc;
  if (poses_per_ligand < 0) return fail(LIGEN_ERR_INVALID_ARG, "poses_per_ligand < 0");
  if (!std::isfinite(out_penalty)) return fail(LIGEN_ERR_INVALID_ARG, "out_penalty not finite");
  const int L = ligands->n_ligands;
  if (L == 0 || poses_per_ligand == 0) return LIGEN_OK;
  if (!poses || !out_scores) return fail(LIGEN_ERR_INVALID_ARG, "poses and out_scores are required");
  cudaStream_t s = (cudaStream_t)stream;
  const int lhost = space_of({ligands->atom_off, ligands->xyz, ligands->type, ligands->bonds,
                              ligands->rot_off, ligands->rot_edge});
  const int ghost = space_of({grid->data});
  const int ohost = space_of({poses, out_scores});
  if (lhost < 0 || ohost < 0) return fail(LIGEN_ERR_INVALID_ARG, "arrays mix host and device memory");
  const size_t pose_floats = (size_t)poses_per_ligand * (7 * (size_t)L + sh.rot);
  const size_t nscores = (size_t)poses_per_ligand * L;
  ScorePlan plan;
  if (poses_per_ligand >= kLanePosesMin) plan_score(ligands->h_rot_off, L, &plan);   // pose-per-lane launches
  Arena ar;
  LigandPlan lp;
  plan_ligands(ar, ligands, sh, lhost == 1, &lp);
  const size_t o_gval = ghost ? ar.take(grid_values_bytes(grid)) : 0;
  const size_t o_coef = ar.take(grid_coef_bytes(grid));
  const size_t o_xc = ar.take(16 * (size_t)sh.atoms);
  const size_t o_binfo = ar.take(4 * (size_t)sh.rot);
  const size_t o_frag = ar.take((size_t)kFragStride * sh.rot);
  const size_t o_status = ar.take(4 * (size_t)L);
  const size_t o_list = ar.take(4 * plan.list.size());
  const bool lanes = poses_per_ligand >= kLanePosesMin;
  const FkRegions o_fk = lanes ? take_fk(ar, sh, L) : FkRegions{};
  size_t o_poses = 0, o_scores = 0;
  if (ohost) {
    o_poses = ar.take(4 * pose_floats);
    o_scores = ar.take(4 * nscores);
  }
  CallCheck chk;
  chk.plan(ar);
  if ((rc = get_workspace(s, ar.used, &ar.base)) != LIGEN_OK) return rc;
  if ((rc = chk.arm(ar, s)) != LIGEN_OK) return rc;
  LigandsDev lig;
  if ((rc = stage_ligands(ar, ligands, sh, lp, s, &lig)) != LIGEN_OK) return rc;
  const float* gvals = (const float*)grid->data;
  if (ghost) {
    LG_CUDA(cudaMemcpyAsync(ar.base + o_gval, grid->data, grid_values_bytes(grid), cudaMemcpyHostToDevice, s));
    gvals = ar.at<float>(o_gval);
  }
  const float* d_poses = poses;
  if (ohost) {
    LG_CUDA(cudaMemcpyAsync(ar.base + o_poses, poses, 4 * pose_floats, cudaMemcpyHostToDevice, s));
    d_poses = ar.at<float>(o_poses);
  }
  if (!plan.list.empty())   // pageable source: staged before the call returns
    LG_CUDA(cudaMemcpyAsync(ar.base + o_list, plan.list.data(), 4 * plan.list.size(), cudaMemcpyHostToDevice, s));
  float* coef = ar.at<float>(o_coef);
  LG_CUDA(launch_grid_prep(gvals, grid->nx, grid->ny, grid->nz, grid->nc, coef, s));
  Packed pk{};
  pk.xc = ar.at<float4>(o_xc);
  pk.binfo = ar.at<uchar4>(o_binfo);
  pk.frag = ar.at<uint8_t>(o_frag);
  pk.status = ar.at<int32_t>(o_status);
  LG_CUDA(launch_pack(lig, grid->nc, pk, s));
  if (lanes) {
    set_fk(ar, o_fk, &pk);
    LG_CUDA(launch_fk_table(lig, pk, sh.max_atoms, sh.max_rot, s));
  }
  ScoreArgs sa{};
  sa.lig = lig;
  sa.pk = pk;
  sa.grid = make_view(grid, coef, out_penalty);
  sa.grid.check = chk.d;
  for (int k = 0; k < 3; ++k) sa.origin[k] = grid->origin[k];
  sa.inv_h = (float)(1.0 / (double)grid->spacing);
  sa.P = poses_per_ligand;
  sa.max_atoms = sh.max_atoms;
  sa.max_rot = sh.max_rot;
  sa.poses = d_poses;
  sa.out_scores = ohost ? ar.at<float>(o_scores) : out_scores;
  if ((rc = run_score(sa, plan, ar.at<int32_t>(o_list), s)) != LIGEN_OK) return rc;
  if (ohost) {
    LG_CUDA(cudaMemcpyAsync(out_scores, sa.out_scores, 4 * nscores, cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
  }
  return chk.verdict(s);
}

int ligen_prepare_scoring(const ligen_ligands_t* ligands, const ligen_grid_t* grid, void* stream,
                          ligen_prepared_t** out) {
  g_err.clear();
  if (!out) return fail(LIGEN_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int rc;
  LibShape sh;
  if ((rc = check_ligands(ligands, 0, &sh)) != LIGEN_OK) return rc;
  if ((rc = check_grid(grid)) != LIGEN_OK) return rc;
  const int L = ligands->n_ligands;
  cudaStream_t s = (cudaStream_t)stream;
  const int lhost = L ? space_of({ligands->atom_off, ligands->xyz, ligands->type, ligands->bonds,
                                  ligands->rot_off, ligands->rot_edge}) : 0;
  const int ghost = space_of({grid->data});
  if (lhost < 0) return fail(LIGEN_ERR_INVALID_ARG, "ligand arrays mix host and device memory");
  // Persistent regions (the handle's own allocation).
  Arena keep;
  const size_t k_atom_off = keep.take(4 * (size_t)(L + 1));
  const size_t k_rot_off = keep.take(4 * (size_t)(L + 1));
  const size_t k_coef = keep.take(grid_coef_bytes(grid));
  const size_t k_xc = keep.take(16 * (size_t)sh.atoms);
  const size_t k_binfo = keep.take(4 * (size_t)sh.rot);
  const size_t k_frag = keep.take((size_t)kFragStride * sh.rot);   // the group-per-pose kernel reads the lists
  const size_t k_status = keep.take(4 * (size_t)L);
  const size_t k_list = keep.take(4 * (size_t)L);
  const FkRegions k_fk = take_fk(keep, sh, L);
  const size_t limit = g_ws_limit.load();
  if (limit && keep.used > limit)
    return fail(LIGEN_ERR_OOM, "prepared inputs of %zu bytes exceed the limit of %zu bytes", keep.used, limit);
  // Staging of host inputs (the calling stream's workspace, this call only).
  Arena tmp;
  LigandPlan lp;
  plan_ligands(tmp, ligands, sh, lhost == 1, &lp);
  const size_t o_gval = ghost ? tmp.take(grid_values_bytes(grid)) : 0;
  CallCheck chk;
  chk.plan(tmp);
  if (tmp.used && (rc = get_workspace(s, tmp.used, &tmp.base)) != LIGEN_OK) return rc;
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  auto* h = new ligen_prepared();
  h->dev = dev;
  cudaError_t e = cudaMalloc(&h->mem, keep.used);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(LIGEN_ERR_OOM, "prepared inputs of %zu bytes: %s", keep.used, cudaGetErrorString(e));
  }
  keep.base = h->mem;
  auto bail = [&](int code) { cudaFree(h->mem); delete h; return code; };
  if ((rc = chk.arm(tmp, s)) != LIGEN_OK) return bail(rc);
  h->grid = *grid;
  h->grid.data = nullptr;
  h->sh = sh;
  h->h_atom_off.assign(ligands->h_atom_off, ligands->h_atom_off + L + 1);
  h->h_rot_off.assign(ligands->h_rot_off, ligands->h_rot_off + L + 1);
  plan_score(h->h_rot_off.data(), L, &h->plan);
  LigandsDev lig;
  if ((rc = stage_ligands(tmp, ligands, sh, lp, s, &lig)) != LIGEN_OK) return bail(rc);
  const float* gvals = (const float*)grid->data;
  if (ghost) {
    const cudaError_t ge =
        cudaMemcpyAsync(tmp.base + o_gval, grid->data, grid_values_bytes(grid), cudaMemcpyHostToDevice, s);
    if (ge != cudaSuccess) return bail(cuda_fail(ge, "grid upload"));
    gvals = tmp.at<float>(o_gval);
  }
  const cudaMemcpyKind kind = lhost ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  h->lig.L = L;
  h->lig.atom_off = keep.at<int32_t>(k_atom_off);
  h->lig.rot_off = keep.at<int32_t>(k_rot_off);
  h->coef = keep.at<float>(k_coef);
  h->pk.xc = keep.at<float4>(k_xc);
  h->pk.binfo = keep.at<uchar4>(k_binfo);
  h->pk.frag = keep.at<uint8_t>(k_frag);
  h->pk.status = keep.at<int32_t>(k_status);
  set_fk(keep, k_fk, &h->pk);
  h->d_list = keep.at<int32_t>(k_list);
  cudaError_t ce = cudaSuccess;
  if (L) {
    ce = cudaMemcpyAsync((void*)h->lig.atom_off, ligands->atom_off, 4 * (size_t)(L + 1), kind, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync((void*)h->lig.rot_off, ligands->rot_off, 4 * (size_t)(L + 1), kind, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(h->d_list, h->plan.list.data(), 4 * (size_t)L, cudaMemcpyHostToDevice, s);
  }
  if (ce == cudaSuccess) ce = launch_grid_prep(gvals, grid->nx, grid->ny, grid->nz, grid->nc, h->coef, s);
  if (ce == cudaSuccess && L) ce = launch_pack(lig, grid->nc, h->pk, s);
  if (ce == cudaSuccess && L) ce = launch_fk_table(lig, h->pk, sh.max_atoms, sh.max_rot, s);
  if (ce != cudaSuccess) return bail(cuda_fail(ce, "preparing the scoring inputs"));
  // Host inputs are copied through the workspace asynchronously: wait for
  // the copies, so the caller may reuse its host buffers on return.
  if (lhost || ghost) {
    if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamSynchronize"));
  }
  if ((rc = chk.verdict(s)) != LIGEN_OK) return bail(rc);
  *out = h;
  return LIGEN_OK;
}

int ligen_score_prepared(const ligen_prepared_t* prep, int32_t poses_per_ligand, const float* poses,
                         float out_penalty, float* out_scores, void* stream) {
  g_err.clear();
  if (!prep) return fail(LIGEN_ERR_INVALID_ARG, "prep is NULL");
  if (poses_per_ligand < 0) return fail(LIGEN_ERR_INVALID_ARG, "poses_per_ligand < 0");
  if (!std::isfinite(out_penalty)) return fail(LIGEN_ERR_INVALID_ARG, "out_penalty not finite");
  const int L = prep->lig.L;
  if (L == 0 || poses_per_ligand == 0) return LIGEN_OK;
  if (!poses || !out_scores) return fail(LIGEN_ERR_INVALID_ARG, "poses and out_scores are required");
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  if (dev != prep->dev) return fail(LIGEN_ERR_INVALID_ARG, "prepared on device %d, called on device %d", prep->dev, dev);
  cudaStream_t s = (cudaStream_t)stream;
  const int ohost = space_of({poses, out_scores});
  if (ohost < 0) return fail(LIGEN_ERR_INVALID_ARG, "poses and out_scores mix host and device memory");
  const size_t pose_floats = (size_t)poses_per_ligand * (7 * (size_t)L + prep->sh.rot);
  const size_t nscores = (size_t)poses_per_ligand * L;
  Arena ar;
  size_t o_poses = 0, o_scores = 0;
  if (ohost) {
    o_poses = ar.take(4 * pose_floats);
    o_scores = ar.take(4 * nscores);
  }
  CallCheck chk;
  chk.plan(ar);
  int rc;
  if (ar.used && (rc = get_workspace(s, ar.used, &ar.base)) != LIGEN_OK) return rc;
  if ((rc = chk.arm(ar, s)) != LIGEN_OK) return rc;
  const float* d_poses = poses;
  if (ohost) {
    LG_CUDA(cudaMemcpyAsync(ar.base + o_poses, poses, 4 * pose_floats, cudaMemcpyHostToDevice, s));
    d_poses = ar.at<float>(o_poses);
  }
  ScoreArgs sa{};
  sa.lig = prep->lig;
  sa.pk = prep->pk;
  sa.grid = make_view(&prep->grid, prep->coef, out_penalty);
  sa.grid.check = chk.d;
  for (int k = 0; k < 3; ++k) sa.origin[k] = prep->grid.origin[k];
  sa.inv_h = (float)(1.0 / (double)prep->grid.spacing);
  sa.P = poses_per_ligand;
  sa.max_atoms = prep->sh.max_atoms;
  sa.max_rot = prep->sh.max_rot;
  sa.poses = d_poses;
  sa.out_scores = ohost ? ar.at<float>(o_scores) : out_scores;
  if ((rc = run_score(sa, prep->plan, prep->d_list, s)) != LIGEN_OK) return rc;
  if (ohost) {
    LG_CUDA(cudaMemcpyAsync(out_scores, sa.out_scores, 4 * nscores, cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
  }
  return chk.verdict(s);
}

int ligen_release_prepared(ligen_prepared_t* prep) {
  g_err.clear();
  if (!prep) return LIGEN_OK;
  int cur = 0;
  LG_CUDA(cudaGetDevice(&cur));
  if (cur != prep->dev) LG_CUDA(cudaSetDevice(prep->dev));
  cudaError_t e = cudaFree(prep->mem);
  if (cur != prep->dev) cudaSetDevice(cur);
  delete prep;
  if (e != cudaSuccess) return cuda_fail(e, "cudaFree(prepared inputs)");
  return LIGEN_OK;
}

// Shared body of ligen_pose_grad and ligen_refine_poses: stage inputs, build
// the grid records, pack the ligands, run the gradient kernel, copy back.
static int grad_call(const ligen_ligands_t* ligands, const ligen_grid_t* grid, int32_t poses_per_ligand,
                     const float* poses_in, float* poses_inout, float out_penalty, float* out_scores,
                     float* out_grads, int refine, int32_t steps, float step_t, float step_q, float step_theta,
                     int8_t* out_accept, void* stream) {
  g_err.clear();
  int rc;
  LibShape sh;
  if ((rc = check_ligands(ligands, 0, &sh)) != LIGEN_OK) return rc;
  if ((rc = check_grid(grid)) != LIGEN_OK) return rc;
  if (poses_per_ligand < 0) return fail(LIGEN_ERR_INVALID_ARG, "poses_per_ligand < 0");
  if (!std::isfinite(out_penalty)) return fail(LIGEN_ERR_INVALID_ARG, "out_penalty not finite");
  if (refine) {
    if (steps < 0 || steps > 100000) return fail(LIGEN_ERR_INVALID_ARG, "steps must be 0..100000");
    if (!(step_t >= 0.f) || !(step_q >= 0.f) || !(step_theta >= 0.f) || !std::isfinite(step_t) ||
        !std::isfinite(step_q) || !std::isfinite(step_theta))
      return fail(LIGEN_ERR_INVALID_ARG, "step sizes must be finite and >= 0");
  }
  const int L = ligands->n_ligands;
  if (L == 0 || poses_per_ligand == 0) return LIGEN_OK;
  const float* pin = refine ? poses_inout : poses_in;
  if (!pin || !out_scores || (!refine && !out_grads))
    return fail(LIGEN_ERR_INVALID_ARG, "poses and outputs are required");
  cudaStream_t s = (cudaStream_t)stream;
  const int lhost = space_of({ligands->atom_off, ligands->xyz, ligands->type, ligands->bonds,
                              ligands->rot_off, ligands->rot_edge});
  const int ghost = space_of({grid->data});
  const int ohost = space_of({pin, out_scores, out_grads, out_accept});
  if (lhost < 0 || ohost < 0) return fail(LIGEN_ERR_INVALID_ARG, "arrays mix host and device memory");
  const size_t pose_floats = (size_t)poses_per_ligand * (7 * (size_t)L + sh.rot);
  const size_t nposes = (size_t)poses_per_ligand * L;
  Arena ar;
  LigandPlan lp;
  plan_ligands(ar, ligands, sh, lhost == 1, &lp);
  const size_t o_gval = ghost ? ar.take(grid_values_bytes(grid)) : 0;
  const size_t o_coef = ar.take(grid_coef_bytes(grid));
  const size_t o_xc = ar.take(16 * (size_t)sh.atoms);
  const size_t o_binfo = ar.take(4 * (size_t)sh.rot);
  const size_t o_frag = ar.take((size_t)kFragStride * sh.rot);
  const size_t o_status = ar.take(4 * (size_t)L);
  ScorePlan plan;   // ligands by rotatable-bond class for the pose-group kernel
  const bool lanes = poses_per_ligand >= kGradLanePosesMin;
  if (lanes) plan_score(ligands->h_rot_off, L, &plan);
  const size_t o_list = ar.take(4 * plan.list.size());
  const FkRegions o_fk = lanes ? take_fk(ar, sh, L) : FkRegions{};
  size_t o_poses = 0, o_scores = 0, o_grads = 0, o_acc = 0;
  if (ohost) {
    o_poses = ar.take(4 * pose_floats);
    o_scores = ar.take(4 * nposes);
    if (!refine) o_grads = ar.take(4 * pose_floats);
    if (out_accept) o_acc = ar.take(nposes * (size_t)steps);
  }
  CallCheck chk;
  chk.plan(ar);
  if ((rc = get_workspace(s, ar.used, &ar.base)) != LIGEN_OK) return rc;
  if ((rc = chk.arm(ar, s)) != LIGEN_OK) return rc;
  LigandsDev lig;
  if ((rc = stage_ligands(ar, ligands, sh, lp, s, &lig)) != LIGEN_OK) return rc;
  const float* gvals = (const float*)grid->data;
  if (ghost) {
    LG_CUDA(cudaMemcpyAsync(ar.base + o_gval, grid->data, grid_values_bytes(grid), cudaMemcpyHostToDevice, s));
    gvals = ar.at<float>(o_gval);
  }
  float* d_poses = const_cast<float*>(pin);
  if (ohost) {
    LG_CUDA(cudaMemcpyAsync(ar.base + o_poses, pin, 4 * pose_floats, cudaMemcpyHostToDevice, s));
    d_poses = ar.at<float>(o_poses);
  }
  float* coef = ar.at<float>(o_coef);
  LG_CUDA(launch_grid_prep(gvals, grid->nx, grid->ny, grid->nz, grid->nc, coef, s));
  Packed pk{};
  pk.xc = ar.at<float4>(o_xc);
  pk.binfo = ar.at<uchar4>(o_binfo);
  pk.frag = ar.at<uint8_t>(o_frag);
  pk.status = ar.at<int32_t>(o_status);
  LG_CUDA(launch_pack(lig, grid->nc, pk, s));
  if (lanes) {
    set_fk(ar, o_fk, &pk);
    LG_CUDA(launch_fk_table(lig, pk, sh.max_atoms, sh.max_rot, s));
  }
  GradArgs ga{};
  ga.lig = lig;
  ga.pk = pk;
  ga.grid = make_view(grid, coef, out_penalty);
  ga.grid.check = chk.d;
  for (int k = 0; k < 3; ++k) ga.origin[k] = grid->origin[k];
  ga.inv_h = (float)(1.0 / (double)grid->spacing);
  ga.P = poses_per_ligand;
  ga.max_atoms = sh.max_atoms;
  ga.poses = d_poses;
  ga.inout_poses = d_poses;
  ga.out_scores = ohost ? ar.at<float>(o_scores) : out_scores;
  ga.out_grads = refine ? nullptr : (ohost ? ar.at<float>(o_grads) : out_grads);
  ga.steps = steps;
  ga.step_t = step_t;
  ga.step_q = step_q;
  ga.step_theta = step_theta;
  const int np[3] = {grid->nx, grid->ny, grid->nz};
  for (int k = 0; k < 3; ++k) {
    ga.box_lo[k] = grid->origin[k];
    ga.box_hi[k] = (float)((double)grid->origin[k] + (double)grid->spacing * (np[k] - 1));
  }
  ga.out_accept = out_accept ? (ohost ? ar.at<int8_t>(o_acc) : out_accept) : nullptr;
  ga.h = grid->spacing;
  if (!lanes) {
    LG_CUDA(launch_grad(ga, refine != 0, s));
  } else {   // pose groups on forward kinematics, class by class
    LG_CUDA(cudaMemcpyAsync(ar.base + o_list, plan.list.data(), 4 * plan.list.size(), cudaMemcpyHostToDevice, s));
    if (!pk.fk_xs || !pk.fk_own || !pk.fk_bond || !pk.fk_ax || !pk.fk_loff)
      return fail(LIGEN_ERR_CUDA, "internal: pose-group gradients without the forward-kinematics table");
    int used[kScoreClasses];
    const int nu = used_classes(plan, used);
    rc = run_forked(nu, s, [&](int i, cudaStream_t st) {
      const int c = used[i];
      GradArgs gc = ga;
      gc.list = ar.at<int32_t>(o_list) + plan.start[c];
      gc.n_list = plan.n[c];
      gc.max_rot = kScoreRotCap[c];
      return launch_grad_lanes(gc, refine != 0, st);
    });
    if (rc != LIGEN_OK) return rc;
  }
  if (ohost) {
    LG_CUDA(cudaMemcpyAsync(out_scores, ga.out_scores, 4 * nposes, cudaMemcpyDeviceToHost, s));
    if (refine) LG_CUDA(cudaMemcpyAsync(poses_inout, d_poses, 4 * pose_floats, cudaMemcpyDeviceToHost, s));
    else LG_CUDA(cudaMemcpyAsync(out_grads, ga.out_grads, 4 * pose_floats, cudaMemcpyDeviceToHost, s));
    if (out_accept)
      LG_CUDA(cudaMemcpyAsync(out_accept, ga.out_accept, nposes * (size_t)steps, cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
  }
  return chk.verdict(s);
}

int ligen_pose_grad(const ligen_ligands_t* ligands, const ligen_grid_t* grid, int32_t poses_per_ligand,
                    const float* poses, float out_penalty, float* out_scores, float* out_grads, void* stream) {
  return grad_call(ligands, grid, poses_per_ligand, poses, nullptr, out_penalty, out_scores, out_grads, 0, 0, 0.f,
                   0.f, 0.f, nullptr, stream);
}

int ligen_refine_poses(const ligen_ligands_t* ligands, const ligen_grid_t* grid, int32_t poses_per_ligand,
                       float* poses, float out_penalty, int32_t steps, float step_t, float step_q, float step_theta,
                       float* out_scores, int8_t* out_accept, void* stream) {
  return grad_call(ligands, grid, poses_per_ligand, nullptr, poses, out_penalty, out_scores, nullptr, 1, steps,
                   step_t, step_q, step_theta, out_accept, stream);
}

int ligen_pack_ligands(const ligen_ligands_t* ligands, int32_t n_channels, uint32_t* frag_bits, int32_t* axis,
                       int32_t* bucket, int32_t* status, void* stream) {
  g_err.clear();
  int rc;
  LibShape sh;
  if ((rc = check_ligands(ligands, 0, &sh)) != LIGEN_OK) return rc;
  if (n_channels < 1 || n_channels > LIGEN_MAX_CHANNELS)
    return fail(LIGEN_ERR_INVALID_ARG, "n_channels must be 1..%d", LIGEN_MAX_CHANNELS);
  const int L = ligands->n_ligands;
  if (L == 0) return LIGEN_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int lhost = space_of({ligands->atom_off, ligands->xyz, ligands->type, ligands->bonds,
                              ligands->rot_off, ligands->rot_edge});
  const int ohost = space_of({frag_bits, axis, bucket, status});
  if (lhost < 0 || ohost < 0) return fail(LIGEN_ERR_INVALID_ARG, "arrays mix host and device memory");
  Arena ar;
  LigandPlan lp;
  plan_ligands(ar, ligands, sh, lhost == 1, &lp);
  const size_t o_xc = ar.take(16 * (size_t)sh.atoms);
  const size_t o_binfo = ar.take(4 * (size_t)sh.rot);
  const size_t o_frag = ar.take((size_t)kFragStride * sh.rot);
  const size_t o_status = ar.take(4 * (size_t)L);
  const size_t o_bucket = ar.take(4 * (size_t)L);
  const size_t o_bits = ar.take(32 * (size_t)sh.rot);
  const size_t o_axis = ar.take(8 * (size_t)sh.rot);
  if ((rc = get_workspace(s, ar.used, &ar.base)) != LIGEN_OK) return rc;
  LigandsDev lig;
  if ((rc = stage_ligands(ar, ligands, sh, lp, s, &lig)) != LIGEN_OK) return rc;
  Packed pk{};
  pk.xc = ar.at<float4>(o_xc);
  pk.binfo = ar.at<uchar4>(o_binfo);
  pk.frag = ar.at<uint8_t>(o_frag);
  pk.status = ar.at<int32_t>(o_status);
  pk.bucket = ar.at<int32_t>(o_bucket);
  pk.fbits = ar.at<uint32_t>(o_bits);
  pk.axis = ar.at<int32_t>(o_axis);
  LG_CUDA(launch_pack(lig, n_channels, pk, s));
  const cudaMemcpyKind k = ohost ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (frag_bits && sh.rot) LG_CUDA(cudaMemcpyAsync(frag_bits, pk.fbits, 32 * (size_t)sh.rot, k, s));
  if (axis && sh.rot) LG_CUDA(cudaMemcpyAsync(axis, pk.axis, 8 * (size_t)sh.rot, k, s));
  if (bucket) LG_CUDA(cudaMemcpyAsync(bucket, pk.bucket, 4 * (size_t)L, k, s));
  if (status) LG_CUDA(cudaMemcpyAsync(status, pk.status, 4 * (size_t)L, k, s));
  if (ohost) LG_CUDA(cudaStreamSynchronize(s));
  return LIGEN_OK;
}

int ligen_pack_touch(const ligen_ligands_t* ligands, int32_t n_channels, uint32_t* touch, void* stream) {
  g_err.clear();
  int rc;
  LibShape sh;
  if ((rc = check_ligands(ligands, 0, &sh)) != LIGEN_OK) return rc;
  if (n_channels < 1 || n_channels > LIGEN_MAX_CHANNELS)
    return fail(LIGEN_ERR_INVALID_ARG, "n_channels must be 1..%d", LIGEN_MAX_CHANNELS);
  const int L = ligands->n_ligands;
  if (L == 0 || sh.rot == 0) return LIGEN_OK;
  if (!touch) return fail(LIGEN_ERR_INVALID_ARG, "touch is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int lhost = space_of({ligands->atom_off, ligands->xyz, ligands->type, ligands->bonds,
                              ligands->rot_off, ligands->rot_edge});
  const int ohost = space_of({touch});
  if (lhost < 0) return fail(LIGEN_ERR_INVALID_ARG, "ligand arrays mix host and device memory");
  Arena ar;
  LigandPlan lp;
  plan_ligands(ar, ligands, sh, lhost == 1, &lp);
  const size_t o_xc = ar.take(16 * (size_t)sh.atoms);
  const size_t o_binfo = ar.take(4 * (size_t)sh.rot);
  const size_t o_frag = ar.take((size_t)kFragStride * sh.rot);
  const size_t o_status = ar.take(4 * (size_t)L);
  const size_t o_touch = ar.take(4 * (size_t)sh.rot);
  if ((rc = get_workspace(s, ar.used, &ar.base)) != LIGEN_OK) return rc;
  LigandsDev lig;
  if ((rc = stage_ligands(ar, ligands, sh, lp, s, &lig)) != LIGEN_OK) return rc;
  Packed pk{};
  pk.xc = ar.at<float4>(o_xc);
  pk.binfo = ar.at<uchar4>(o_binfo);
  pk.frag = ar.at<uint8_t>(o_frag);
  pk.status = ar.at<int32_t>(o_status);
  pk.touch = ar.at<uint32_t>(o_touch);
  LG_CUDA(launch_pack(lig, n_channels, pk, s));
  LG_CUDA(cudaMemcpyAsync(touch, pk.touch, 4 * (size_t)sh.rot, ohost ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                          s));
  if (ohost) LG_CUDA(cudaStreamSynchronize(s));
  return LIGEN_OK;
}

int64_t ligen_bucket_size(int32_t max_atoms, int32_t* b, int32_t* sm, int32_t* t, int32_t* ws) {
  g_err.clear();
  if (max_atoms < 1 || max_atoms > LIGEN_MAX_ATOMS)
    return fail(LIGEN_ERR_INVALID_ARG, "max_atoms must be 1..%d", LIGEN_MAX_ATOMS);
  int dev = 0, nsm = 0, warp = 0, blocks = 0;
  LG_CUDA(cudaGetDevice(&dev));
  LG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  LG_CUDA(cudaDeviceGetAttribute(&warp, cudaDevAttrWarpSize, dev));
  const int rpc = dock_restarts_per_cta(256, kDefaultLanes);
  const size_t smem = dock_smem_bytes(max_atoms, LIGEN_MAX_ROT, LIGEN_MAX_ROT * (max_atoms / 2), rpc);
  LG_CUDA(dock_set_smem_limit(kDefaultLanes, 36, kRecF32, smem));
  LG_CUDA(dock_occupancy(kDefaultLanes, 36, kRecF32, rpc, smem, &blocks));
  const int threads = rpc * kDefaultLanes;
  if (b) *b = blocks;
  if (sm) *sm = nsm;
  if (t) *t = threads;
  if (ws) *ws = warp;
  return (int64_t)blocks * nsm * threads / warp;
}

int ligen_tune_set(int32_t bucket, int32_t lanes, int32_t restarts_per_cta) {
  g_err.clear();
  if (bucket < 0 || bucket >= LIGEN_N_BUCKETS) return fail(LIGEN_ERR_INVALID_ARG, "bucket must be 0..%d", LIGEN_N_BUCKETS - 1);
  if (!valid_shape(lanes, restarts_per_cta))
    return fail(LIGEN_ERR_INVALID_ARG, "shape (%d lanes, %d restarts) is not supported", lanes, restarts_per_cta);
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  if (dev >= kMaxDev) return fail(LIGEN_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDev);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[dev][bucket].lanes = lanes;
  g_tune[dev][bucket].rpc = restarts_per_cta;
  return LIGEN_OK;
}

int ligen_tune_get(int32_t bucket, int32_t* lanes, int32_t* restarts_per_cta) {
  g_err.clear();
  if (bucket < 0 || bucket >= LIGEN_N_BUCKETS) return fail(LIGEN_ERR_INVALID_ARG, "bucket must be 0..%d", LIGEN_N_BUCKETS - 1);
  if (!lanes || !restarts_per_cta) return fail(LIGEN_ERR_INVALID_ARG, "NULL output");
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  if (dev >= kMaxDev) return fail(LIGEN_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDev);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  *lanes = g_tune[dev][bucket].lanes;
  *restarts_per_cta = g_tune[dev][bucket].rpc;
  return LIGEN_OK;
}

int ligen_autotune(const ligen_ligands_t* ligands, const ligen_grid_t* grid, const ligen_params_t* params,
                   int32_t sample, int32_t* out_lanes, int32_t* out_rpc, float* out_ms_per_ligand) {
  g_err.clear();
  int rc;
  if ((rc = check_params(params)) != LIGEN_OK) return rc;
  if (params->mode != 0) return fail(LIGEN_ERR_UNSUPPORTED, "autotuning times the greedy search (mode 0)");
  LibShape sh;
  if ((rc = check_ligands(ligands, params->passes, &sh)) != LIGEN_OK) return rc;
  if ((rc = check_grid(grid)) != LIGEN_OK) return rc;
  if (sample < 1) return fail(LIGEN_ERR_INVALID_ARG, "sample must be >= 1");
  if (!out_lanes || !out_rpc) return fail(LIGEN_ERR_INVALID_ARG, "out_lanes and out_rpc are required");
  for (int b = 0; b < LIGEN_N_BUCKETS; ++b) {
    out_lanes[b] = 0;
    out_rpc[b] = 0;
    if (out_ms_per_ligand) out_ms_per_ligand[b] = 0.f;
  }
  const int L = ligands->n_ligands;
  if (L == 0) return LIGEN_OK;
  if (space_of({ligands->atom_off, ligands->xyz, ligands->type, ligands->bonds, ligands->rot_off,
                ligands->rot_edge}) != 0 || space_of({grid->data}) != 0)
    return fail(LIGEN_ERR_INVALID_ARG, "ligen_autotune takes device memory only");
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  if (dev >= kMaxDev) return fail(LIGEN_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDev);
  cudaStream_t s = (cudaStream_t)params->stream;
  const int R = params->restarts;

  // up to `sample` ligands of each bucket, bucket by bucket
  std::vector<std::vector<int32_t>> members(LIGEN_N_BUCKETS);
  for (int l = 0; l < L; ++l) {
    const int N = ligands->h_atom_off[l + 1] - ligands->h_atom_off[l];
    const int n = ligands->h_rot_off[l + 1] - ligands->h_rot_off[l];
    auto& m = members[atom_class_of(N) * 11 + rot_class_of(n)];
    if ((int)m.size() < sample) m.push_back(l);
  }
  std::vector<int32_t> order;
  std::vector<Group> bucket(LIGEN_N_BUCKETS);
  for (int b = 0; b < LIGEN_N_BUCKETS; ++b) {
    bucket[b].beg = (int)order.size();
    for (int32_t l : members[b]) {
      order.push_back(l);
      const int N = ligands->h_atom_off[l + 1] - ligands->h_atom_off[l];
      const int n = ligands->h_rot_off[l + 1] - ligands->h_rot_off[l];
      bucket[b].max_atoms = std::max(bucket[b].max_atoms, N);
      bucket[b].max_rot = std::max(bucket[b].max_rot, n);
      bucket[b].max_frag = std::max(bucket[b].max_frag, n * (N / 2));
    }
    bucket[b].end = (int)order.size();
  }

  Arena ar;
  const int fmt = params->grid_format;
  const size_t o_coef = ar.take(grid_coef_bytes(grid, fmt));
  const size_t o_xc = ar.take(16 * (size_t)sh.atoms);
  const size_t o_binfo = ar.take(4 * (size_t)sh.rot);
  const size_t o_frag = ar.take((size_t)kFragStride * sh.rot);
  const size_t o_touch = ar.take(4 * (size_t)sh.rot);
  const size_t o_status = ar.take(4 * (size_t)L);
  const size_t o_rs = ar.take(4 * (size_t)L * R);
  const size_t o_rk = ar.take((size_t)L * R);
  const size_t o_rc = ar.take((size_t)sh.rot * R);
  const size_t o_order = ar.take(4 * order.size());
  CallCheck chk;
  chk.plan(ar);
  if ((rc = get_workspace(s, ar.used, &ar.base)) != LIGEN_OK) return rc;
  if ((rc = chk.arm(ar, s)) != LIGEN_OK) return rc;

  LigandsDev lig;
  lig.L = L;
  lig.atom_off = ligands->atom_off; lig.xyz = ligands->xyz; lig.type = ligands->type;
  lig.bonds = ligands->bonds; lig.rot_off = ligands->rot_off; lig.rot_edge = ligands->rot_edge;
  float* coef = ar.at<float>(o_coef);
  LG_CUDA(launch_grid_prep_fmt((const float*)grid->data, grid->nx, grid->ny, grid->nz, grid->nc, fmt, coef, s));
  Packed pk{};
  pk.xc = ar.at<float4>(o_xc);
  pk.binfo = ar.at<uchar4>(o_binfo);
  pk.frag = ar.at<uint8_t>(o_frag);
  pk.touch = ar.at<uint32_t>(o_touch);
  pk.status = ar.at<int32_t>(o_status);
  LG_CUDA(launch_pack(lig, grid->nc, pk, s));
  int32_t* d_order = ar.at<int32_t>(o_order);
  LG_CUDA(cudaMemcpyAsync(d_order, order.data(), 4 * order.size(), cudaMemcpyHostToDevice, s));

  DockArgs base{};
  base.lig = lig;
  base.pk = pk;
  base.grid = make_view(grid, coef, params->out_penalty, fmt);
  base.grid.check = chk.d;
  const float h = grid->spacing;
  const int np[3] = {grid->nx, grid->ny, grid->nz};
  for (int k = 0; k < 3; ++k) {
    base.origin[k] = grid->origin[k];
    base.center[k] = (float)((double)grid->origin[k] + (double)h * (np[k] - 1) / 2.0);
  }
  base.inv_h = (float)(1.0 / (double)h);
  base.jitter = params->jitter;
  base.seed = params->seed;
  base.R = R;
  base.n_rigid = params->n_rigid;
  base.step_deg = params->torsion_step_deg;
  base.n_theta = 360 / params->torsion_step_deg;
  base.passes = params->passes;
  base.fmt = fmt;
  base.res_score = ar.at<float>(o_rs);
  base.res_k = ar.at<uint8_t>(o_rk);
  base.res_cnt = ar.at<uint8_t>(o_rc);

  static const int kCand[][2] = {{4, 32}, {4, 16}, {8, 16}, {8, 8}, {2, 64}, {16, 8}, {32, 4}};
  cudaEvent_t e0, e1;
  LG_CUDA(cudaEventCreate(&e0));
  LG_CUDA(cudaEventCreate(&e1));
  int result = LIGEN_OK;
  for (int b = 0; b < LIGEN_N_BUCKETS && result == LIGEN_OK; ++b) {
    const int cnt = bucket[b].end - bucket[b].beg;
    if (cnt == 0) continue;
    float best_ms = 0.f;
    int best = -1;
    for (int c = 0; c < (int)(sizeof kCand / sizeof kCand[0]); ++c) {
      if (!valid_shape(kCand[c][0], kCand[c][1]) || !dock_shape_supported(kCand[c][0], fmt)) continue;
      DockArgs a = base;
      a.lanes = kCand[c][0];
      a.rpc = kCand[c][1];
      a.chunks = (R + a.rpc - 1) / a.rpc;
      a.list = d_order + bucket[b].beg;
      a.n_items = cnt * a.chunks;
      a.queue = nullptr;
      a.max_atoms = bucket[b].max_atoms;
      a.max_rot = bucket[b].max_rot;
      a.max_frag = bucket[b].max_frag;
      float ms = 0.f;
      for (int rep = 0; rep < 3; ++rep) {   // first run warms up
        cudaError_t e = cudaEventRecord(e0, s);
        if (e == cudaSuccess) e = launch_dock(a, 0, s, true);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e != cudaSuccess) {
          result = cuda_fail(e, "autotune launch");
          break;
        }
        if (rep == 1 || (rep == 2 && t < ms)) ms = t;
      }
      if (result != LIGEN_OK) break;
      if (best < 0 || ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    if (result != LIGEN_OK || best < 0) break;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[dev][b].lanes = kCand[best][0];
      g_tune[dev][b].rpc = kCand[best][1];
    }
    out_lanes[b] = kCand[best][0];
    out_rpc[b] = kCand[best][1];
    if (out_ms_per_ligand) out_ms_per_ligand[b] = best_ms / cnt;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != LIGEN_OK) return result;
  return chk.verdict(s);
}

int ligen_probe_gather(const float* records, int64_t n_records, int32_t bytes_per_load, int32_t loads_per_thread,
                       float* sink, double* loads_done, float* ms_out, void* stream) {
  g_err.clear();
  if (!records || !sink || !ms_out || !loads_done) return fail(LIGEN_ERR_INVALID_ARG, "NULL argument");
  if (bytes_per_load != 4 && bytes_per_load != 8 && bytes_per_load != 16 && bytes_per_load != 32)
    return fail(LIGEN_ERR_INVALID_ARG, "bytes_per_load must be 4, 8, 16 or 32");
  if (n_records < 1 || n_records > (int64_t)UINT32_MAX) return fail(LIGEN_ERR_INVALID_ARG, "n_records out of range");
  if ((uintptr_t)records % 32 != 0) return fail(LIGEN_ERR_INVALID_ARG, "records must be 32-byte aligned");
  const int iters = loads_per_thread / probe_streams();
  if (iters < 1) return fail(LIGEN_ERR_INVALID_ARG, "loads_per_thread must be >= %d", probe_streams());
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  LG_CUDA(cudaGetDevice(&dev));
  LG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * (2048 / probe_threads());
  cudaEvent_t e0, e1;
  LG_CUDA(cudaEventCreate(&e0));
  LG_CUDA(cudaEventCreate(&e1));
  LG_CUDA(launch_probe(records, (uint32_t)n_records, bytes_per_load, 1, 7, sink, blocks, s));   // warm the cache
  LG_CUDA(cudaEventRecord(e0, s));
  LG_CUDA(launch_probe(records, (uint32_t)n_records, bytes_per_load, iters, 11, sink, blocks, s));
  LG_CUDA(cudaEventRecord(e1, s));
  LG_CUDA(cudaEventSynchronize(e1));
  LG_CUDA(cudaEventElapsedTime(ms_out, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *loads_done = (double)blocks * probe_threads() * iters * probe_streams();
  return LIGEN_OK;
}

int ligen_probe_stream(const void* buffer, int64_t n_bytes, int32_t passes, float* sink, double* bytes_done,
                       float* ms_out, void* stream) {
  g_err.clear();
  if (!buffer || !sink || !bytes_done || !ms_out) return fail(LIGEN_ERR_INVALID_ARG, "NULL argument");
  if (n_bytes < 16 || n_bytes % 16 != 0) return fail(LIGEN_ERR_INVALID_ARG, "n_bytes must be a positive multiple of 16");
  if ((uintptr_t)buffer % 16 != 0) return fail(LIGEN_ERR_INVALID_ARG, "buffer must be 16-byte aligned");
  if (passes < 1) return fail(LIGEN_ERR_INVALID_ARG, "passes must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  LG_CUDA(cudaGetDevice(&dev));
  LG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * (2048 / probe_threads());
  const uint64_t n_vec = (uint64_t)n_bytes / 16;
  cudaEvent_t e0, e1;
  LG_CUDA(cudaEventCreate(&e0));
  LG_CUDA(cudaEventCreate(&e1));
  LG_CUDA(launch_stream_probe(buffer, n_vec, 1, sink, blocks, s));   // brings the buffer into L2
  LG_CUDA(cudaEventRecord(e0, s));
  LG_CUDA(launch_stream_probe(buffer, n_vec, passes, sink, blocks, s));
  LG_CUDA(cudaEventRecord(e1, s));
  LG_CUDA(cudaEventSynchronize(e1));
  LG_CUDA(cudaEventElapsedTime(ms_out, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *bytes_done = (double)n_bytes * passes;
  return LIGEN_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------
// ligen_dock_batch_static: the docking call for callers that must not
// allocate device memory. Its scratch is the file-scope device array below,
// of LIGEN_STATIC_SCRATCH_BYTES; every device that loads this library holds
// it until the process exits. Host code reaches the array only through
// cudaGetSymbolAddress (the array's name is a host-side stand-in, not a
// device address); the address is looked up once per device, with that
// device current, on the first call made on it.
static __device__ __align__(256) unsigned char g_static_scratch[LIGEN_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
char* g_static_base[kMaxDevices] = {};

int static_scratch_base(char** out) {
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(LIGEN_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    if (!p || (uintptr_t)p % 256 != 0) return fail(LIGEN_ERR_CUDA, "static scratch address not 256-byte aligned");
    g_static_base[dev] = (char*)p;
  }
  *out = g_static_base[dev];
  return LIGEN_OK;
}

}  // namespace

extern "C" int ligen_dock_batch_static(const ligen_ligands_t* ligands, const ligen_grid_t* grid,
                                       const ligen_params_t* params, float* out_poses, float* out_scores) {
  g_err.clear();
  int rc;
  if ((rc = check_params(params)) != LIGEN_OK) return rc;
  if (params->mode != 0) return fail(LIGEN_ERR_UNSUPPORTED, "ligen_dock_batch_static runs the greedy search (mode 0)");
  // The call runs the plain launch over FP32 grid records and nothing else;
  // every setting it would not honour is refused rather than ignored.
  if (params->grid_format != LIGEN_GRID_F32)
    return fail(LIGEN_ERR_UNSUPPORTED, "ligen_dock_batch_static samples FP32 grid records only (grid_format 0)");
  if (params->batching != LIGEN_BATCH_PLAIN)
    return fail(LIGEN_ERR_UNSUPPORTED, "ligen_dock_batch_static runs the plain launch only (batching 0)");
  if (params->rescore_fp64 != 0 || params->scores_f64)
    return fail(LIGEN_ERR_UNSUPPORTED, "ligen_dock_batch_static has no FP64 re-score (rescore_fp64 0, scores_f64 NULL)");
  if (params->stage_ms || params->samples || params->coords)
    return fail(LIGEN_ERR_UNSUPPORTED,
                "ligen_dock_batch_static reports neither stage_ms, samples nor coords (all NULL)");
  LibShape sh;
  if ((rc = check_ligands(ligands, params->passes, &sh)) != LIGEN_OK) return rc;
  if ((rc = check_grid(grid)) != LIGEN_OK) return rc;
  const int L = ligands->n_ligands;
  if (L == 0) return LIGEN_OK;
  if (!out_poses || !out_scores) return fail(LIGEN_ERR_INVALID_ARG, "out_poses and out_scores are required");
  const int R = params->restarts, K = params->top_k;

  // Scratch plan (the same regions as the device path of ligen_dock_batch);
  // checked against the static maximum before any device call.
  Arena ar;
  const size_t o_coef = ar.take(grid_coef_bytes(grid));
  const size_t o_xc = ar.take(16 * (size_t)sh.atoms);
  const size_t o_binfo = ar.take(4 * (size_t)sh.rot);
  const size_t o_frag = ar.take((size_t)kFragStride * sh.rot);
  const size_t o_touch = ar.take(4 * (size_t)sh.rot);
  const size_t o_status = ar.take(4 * (size_t)L);
  const size_t o_rs = ar.take(4 * (size_t)L * R);
  const size_t o_rk = ar.take((size_t)L * R);
  const size_t o_rc = ar.take((size_t)sh.rot * R);
  CallCheck chk;
  chk.plan(ar);
  if (ar.used > (size_t)LIGEN_STATIC_SCRATCH_BYTES)
    return fail(LIGEN_ERR_UNSUPPORTED,
                "this batch needs %zu bytes of scratch; ligen_dock_batch_static has %zu "
                "(use fewer ligands or restarts, a smaller grid, or ligen_dock_batch)",
                ar.used, (size_t)LIGEN_STATIC_SCRATCH_BYTES);

  const int lhost = space_of({ligands->atom_off, ligands->xyz, ligands->type, ligands->bonds,
                              ligands->rot_off, ligands->rot_edge});
  const int ghost = space_of({grid->data});
  const int ohost = space_of({out_poses, out_scores, params->status, params->trace, params->top_restart});
  if (lhost != 0 || ghost != 0 || ohost != 0)
    return fail(LIGEN_ERR_INVALID_ARG, "ligen_dock_batch_static takes device memory only "
                                       "(ligands, grid and outputs)");
  if ((rc = static_scratch_base(&ar.base)) != LIGEN_OK) return rc;
  cudaStream_t s = (cudaStream_t)params->stream;
  if ((rc = chk.arm(ar, s)) != LIGEN_OK) return rc;

  // Every scratch region is written in full before it is read within this
  // call, so nothing is cleared between calls.
  LigandsDev lig;
  lig.L = L;
  lig.atom_off = ligands->atom_off; lig.xyz = ligands->xyz; lig.type = ligands->type;
  lig.bonds = ligands->bonds; lig.rot_off = ligands->rot_off; lig.rot_edge = ligands->rot_edge;
  float* coef = ar.at<float>(o_coef);
  LG_CUDA(launch_grid_prep((const float*)grid->data, grid->nx, grid->ny, grid->nz, grid->nc, coef, s));
  Packed pk{};
  pk.xc = ar.at<float4>(o_xc);
  pk.binfo = ar.at<uchar4>(o_binfo);
  pk.frag = ar.at<uint8_t>(o_frag);
  pk.touch = ar.at<uint32_t>(o_touch);
  pk.status = ar.at<int32_t>(o_status);
  LG_CUDA(launch_pack(lig, grid->nc, pk, s));

  DockArgs da{};
  da.lig = lig;
  da.pk = pk;
  da.grid = make_view(grid, coef, params->out_penalty);
  da.grid.check = chk.d;
  const float h = grid->spacing;
  const int np[3] = {grid->nx, grid->ny, grid->nz};
  for (int k = 0; k < 3; ++k) {
    da.origin[k] = grid->origin[k];
    da.center[k] = (float)((double)grid->origin[k] + (double)h * (np[k] - 1) / 2.0);
  }
  da.inv_h = (float)(1.0 / (double)h);
  da.jitter = params->jitter;
  da.seed = params->seed;
  da.R = R;
  da.n_rigid = params->n_rigid;
  da.step_deg = params->torsion_step_deg;
  da.n_theta = 360 / params->torsion_step_deg;
  da.passes = params->passes;
  da.lanes = kDefaultLanes;
  da.rpc = dock_restarts_per_cta(R, da.lanes);
  da.chunks = (R + da.rpc - 1) / da.rpc;
  da.list = nullptr;
  da.n_items = L * da.chunks;
  da.queue = nullptr;
  da.max_atoms = sh.max_atoms;
  da.max_rot = sh.max_rot;
  da.max_frag = (int)sh.max_frag;
  da.res_score = ar.at<float>(o_rs);
  da.res_k = ar.at<uint8_t>(o_rk);
  da.res_cnt = ar.at<uint8_t>(o_rc);
  da.trace = params->trace;
  LG_CUDA(launch_dock(da, 0, s, true));

  TopkArgs ta{};
  ta.L = L; ta.R = R; ta.K = K; ta.step_deg = params->torsion_step_deg;
  ta.rot_off = lig.rot_off;
  ta.status = pk.status;
  ta.res_score = da.res_score; ta.res_k = da.res_k; ta.res_cnt = da.res_cnt;
  ta.seed = params->seed;
  for (int k = 0; k < 3; ++k) ta.center[k] = da.center[k];
  ta.jitter = params->jitter;
  ta.out_poses = out_poses;
  ta.out_scores = out_scores;
  ta.top_restart = params->top_restart;
  LG_CUDA(launch_topk(ta, s));
  if (params->status)
    LG_CUDA(cudaMemcpyAsync(params->status, pk.status, 4 * (size_t)L, cudaMemcpyDeviceToDevice, s));
  return chk.verdict(s);
}
