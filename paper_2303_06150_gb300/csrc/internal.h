// Internal interface between the C ABI (ligen_api.cu) and the kernel
// translation units. Not installed; not part of the ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace ligen {

constexpr int kFragStride = 128;   // bytes per rotatable bond in the moving-atom lists

// Device-resident ligand library (CSR, see ligen_ligands_t).
struct LigandsDev {
  int L;
  const int32_t* atom_off;
  const float* xyz;
  const uint8_t* type;
  const int32_t* bonds;
  const int32_t* rot_off;
  const int32_t* rot_edge;
};

// Packer outputs.
struct Packed {
  float4* xc;        // [sum N] centred input coordinates; w = atom type (int bits)
  uchar4* binfo;     // [sum n] (fixed u, moving v, moving atoms excluding v, 0)
  uint8_t* frag;     // [sum n][kFragStride] moving atoms excluding v, ascending
  int32_t* status;   // [L] 0 or LIGEN_ERR_BAD_LIGAND
  int32_t* bucket;   // [L] optional
  uint32_t* fbits;   // [sum n][8] optional: full moving side as a bit mask
  int32_t* axis;     // [sum n][2] optional: (u, v)
  uint32_t* touch;   // [sum n] optional: bit b of touch[b'] set when turning bond b'
                     // moves an atom bond b's sweep reads (bit b' always set)
  // Forward-kinematics table (fk_table_kernel; read by the pose-per-lane
  // scoring and pose-group gradient kernels), optional. A ligand's atoms
  // are listed by owner (bond 0's, bond 1's, ..., then the root frame's;
  // input order within an owner):
  float4* fk_xs;     // [sum N] centred input coordinates (w = type) in that order
  uint8_t* fk_own;   // [sum N] owner of each listed atom: a bond, or n (the root frame)
  uchar4* fk_bond;   // [sum n] (parent of bond j, j-th bond parents first, j-th bond by depth,
                     //          list position of bond j's moving endpoint v)
  float4* fk_ax;     // [sum n] unit bond axes in the input conformation
  uint8_t* fk_loff;  // [L][kFkLoffBytes] first entry of each depth, depth count, malformed flag
};

constexpr int kFkLoffBytes = 48;
constexpr int kFkBad = 47;   // byte of a ligand's fk_loff row: 1 when its lists are malformed

// Sample counters are spread over this many slots (summed on the host) so
// that CTAs do not all add to one address.
constexpr int kSampleSlots = 64;

struct DockArgs {
  LigandsDev lig;
  Packed pk;
  GridView grid;
  float origin[3];
  float inv_h;
  float center[3];
  float jitter;
  uint64_t seed;
  int R, n_rigid, step_deg, n_theta, passes;
  int lanes;          // G: lanes per restart (2, 4, 8, 16 or 32)
  int fmt;            // grid record format (RecFormat)
  int rpc;            // restarts per work item (a multiple of 32 / lanes)
  int chunks;         // work items per ligand: ceil(R / rpc)
  const int32_t* list;  // ligands to dock (NULL: 0 .. n_items / chunks - 1)
  int n_items;        // work items: (list length or L) * chunks
  int* queue;         // persistent mode: device counter of taken items (zeroed
                      // before the launch); NULL: one CTA per item
  int max_atoms, max_rot, max_frag;   // shared-memory carve-up bounds
  float* res_score;   // [L][R]
  uint8_t* res_k;     // [L][R]
  uint8_t* res_cnt;   // [sum n][R] torsion increments (mod n_theta) per restart
  int16_t* trace;     // optional
  unsigned long long* samples;   // optional [kSampleSlots]: atom samples the search needed
  float* coords;      // optional: final grid-unit positions, [3 R atom_off[l] + 3 (r N_l + i) + k]
};

// Exhaustive search (mode 1): at most kExMaxRot rotatable bonds per ligand
// and kExMaxCombos combinations (n_rigid * n_theta^n) per restart.
constexpr int kExMaxRot = 4;
constexpr long long kExMaxCombos = 1ll << 27;
cudaError_t launch_exhaustive(const DockArgs& a, cudaStream_t s);

struct TopkArgs {
  int L, R, K, step_deg;
  const int32_t* rot_off;
  const int32_t* status;
  const float* res_score;
  const uint8_t* res_k;
  const uint8_t* res_cnt;
  uint64_t seed;
  float center[3];
  float jitter;
  float* out_poses;
  float* out_scores;
  int32_t* top_restart;   // optional
};

struct ScoreArgs {
  LigandsDev lig;
  Packed pk;
  GridView grid;
  float origin[3];
  float inv_h;
  int P;              // poses per ligand
  int max_atoms;      // largest ligand of the launch (shared-memory carve-up)
  int max_rot;        // most rotatable bonds of a ligand of the launch
  const float* poses;
  float* out_scores;
  const int32_t* list;  // pose-per-lane launch: ligands to score (NULL: 0 .. n_list - 1)
  int n_list;
};

struct GradArgs {
  LigandsDev lig;
  Packed pk;
  GridView grid;
  float origin[3];
  float inv_h;
  int P;              // poses per ligand
  int max_atoms;
  const float* poses;       // gradient: input poses
  float* inout_poses;       // refinement: poses, refined in place
  float* out_scores;        // [L][P]
  float* out_grads;         // gradient: same packing as poses
  int steps;                // refinement iterations
  float step_t, step_q, step_theta;
  float box_lo[3], box_hi[3];
  int8_t* out_accept;       // refinement: [L * P][steps], optional
  const int32_t* list;      // pose-group launch: ligands (NULL: 0 .. n_list - 1)
  int n_list;
  int max_rot;              // pose-group launch: most rotatable bonds of a ligand of the launch
  float h;                  // grid spacing (Angstrom)
};

struct RescoreArgs {
  LigandsDev lig;
  Packed pk;
  const int32_t* status;
  const float* values;      // caller's grid [z][y][x][c], FP32
  int nx, ny, nz, nc;
  double origin[3];
  double h;
  double penalty;
  int K;                    // kept poses per ligand
  int max_atoms;            // largest ligand (shared-memory carve-up)
  int max_rot;              // most rotatable bonds of a ligand (shared-memory carve-up)
  float* poses;             // outputs, re-ranked in place
  float* scores;            // [L][K], FP64 scores rounded to FP32
  int32_t* top_restart;     // [L][K] or NULL
  double* out_s64;          // [L][K] or NULL: FP64 scores, re-ranked
  double* s64;              // scratch [L][K]
  const float* tmp_poses;   // copy of the poses before re-ranking
  const int32_t* tmp_top;   // copy of top_restart before re-ranking, or NULL
  unsigned* check;          // checked builds: first out-of-range code, else NULL
};

cudaError_t launch_grid_prep(const float* values, int nx, int ny, int nz, int nc, float* coef,
                             cudaStream_t s);
// Records in format `fmt` (RecFormat) for the docking kernel.
cudaError_t launch_grid_prep_fmt(const float* values, int nx, int ny, int nz, int nc, int fmt, void* rec,
                                 cudaStream_t s);
cudaError_t launch_pack(const LigandsDev& lig, int nc, const Packed& out, cudaStream_t s);
// The forward-kinematics table of every ligand (pk.fk_*), after launch_pack;
// max_atoms / max_rot: the library's largest ligand.
cudaError_t launch_fk_table(const LigandsDev& lig, const Packed& pk, int max_atoms, int max_rot, cudaStream_t s);
size_t dock_smem_bytes(int max_atoms, int max_rot, int max_frag, int rpc);
bool dock_lanes_supported(int lanes);
bool dock_shape_supported(int lanes, int fmt);
// grid_ctas: CTAs of a persistent launch (ignored when a.queue is NULL).
// set_attr: set the kernel's dynamic shared-memory limit first (false when
// dock_occupancy already did, e.g. before a stream capture).
cudaError_t launch_dock(const DockArgs& a, int grid_ctas, cudaStream_t s, bool set_attr);
// The kernel of (lanes, n_theta) accepts up to `smem` bytes of dynamic
// shared memory from now on (a per-kernel setting: set the largest value any
// pending launch of that kernel needs).
cudaError_t dock_set_smem_limit(int lanes, int n_theta, int fmt, size_t smem);
// Resident CTAs per SM for a launch with `smem` bytes (within the limit).
cudaError_t dock_occupancy(int lanes, int n_theta, int fmt, int rpc, size_t smem, int* blocks_per_sm);
cudaError_t launch_topk(const TopkArgs& a, cudaStream_t s);
cudaError_t launch_score(const ScoreArgs& a, cudaStream_t s);
// Pose-per-lane scoring of the ligands a.list[0 .. n_list) (all of them at
// most a.max_atoms atoms and a.max_rot bonds), 32 poses per warp: the launch
// shape (sets the kernel's shared-memory limit; no stream work, so it is
// called before a graph capture), then the launch.
struct LaunchCfg {
  unsigned blocks = 0;
  size_t smem = 0;
};
cudaError_t score_lanes_config(const ScoreArgs& a, LaunchCfg* c);
cudaError_t launch_score_lanes(const ScoreArgs& a, const LaunchCfg& c, cudaStream_t s);
cudaError_t launch_rescore(const RescoreArgs& a, cudaStream_t s);
size_t grad_smem_bytes(int max_atoms);
// refine = false: dS/dpose of every pose; true: gradient refinement in place.
cudaError_t launch_grad(const GradArgs& a, bool refine, cudaStream_t s);
// The same on forward kinematics, a group of lanes per pose, for the ligands
// a.list[0 .. n_list) (at most a.max_atoms atoms and a.max_rot bonds each);
// calls with at least kGradLanePosesMin poses per ligand.
constexpr int kGradLanePosesMin = 4;
cudaError_t launch_grad_lanes(const GradArgs& a, bool refine, cudaStream_t s);
cudaError_t launch_probe(const float* rec, uint32_t n_rec, int bytes, int iters, uint64_t seed, float* sink,
                         int blocks, cudaStream_t s);
int probe_streams();
int probe_threads();
cudaError_t launch_stream_probe(const void* buf, uint64_t n_vec, int passes, float* sink, int blocks,
                                cudaStream_t s);

}  // namespace ligen
