/*
 * ligen.h — C ABI of the GB300 docking pose search.
 *
 * The library docks a library of ligands into one pocket grid. For every
 * ligand it runs R restarts; each restart tries the 24 rotations of the cube
 * about the ligand's centroid (rigid stage), then sweeps every rotatable bond
 * through its torsion increments (one pass after another, bonds in index
 * order), keeping at every stage the candidate with the highest score; each
 * ligand keeps its best K restarts. A pose's score is S = -sum_i E_i where E_i
 * is the trilinear sample of atom i's channel in the grid (a fixed penalty
 * outside the box). Paper §2 names the docking task; §3 states that its cost
 * follows the ligand's atoms and its rotamers (rotatable atom subsets), which
 * is what the per-ligand launch data here is organised around.
 *
 * Conventions for every call:
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy
 *     default stream) unless an output lives in host memory, in which case
 *     the call synchronises the stream before returning.
 *   - Each structure's arrays live in ONE memory space: all device memory
 *     (cudaMalloc / managed) or all host memory (pageable or pinned). The
 *     library detects the space per structure; host inputs are copied to the
 *     device inside the call and host outputs are copied back. The caller
 *     keeps ownership of every pointer it passes.
 *   - The library owns one internal device workspace per (device, stream),
 *     grown on demand and released by ligen_release_workspaces(). Two calls
 *     in flight on different streams use different workspaces; calls on the
 *     same stream are ordered by the stream, so several host threads that
 *     share a stream must not call into the library at the same time (their
 *     copies into the shared workspace could interleave). No workspace
 *     content is assumed to survive from one call to the next.
 *   - Argument errors are detected on the host and returned immediately,
 *     before any device work (message in ligen_last_error()). Errors in a
 *     single ligand's data (not a tree, index or type out of range) do not
 *     fail the call: that ligand's status entry is set to
 *     LIGEN_ERR_BAD_LIGAND, its scores to -INFINITY, its poses to zero
 *     (identity quaternion); the device never traps.
 *   - Limits: atoms per ligand 1..256, rotatable bonds per ligand 0..32,
 *     channels 1..64, grid points per axis >= 2.
 */
#ifndef LIGEN_H
#define LIGEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LIGEN_ABI_VERSION 5
#define LIGEN_MAX_ATOMS 256
#define LIGEN_MAX_ROT 32
#define LIGEN_MAX_CHANNELS 64
#define LIGEN_N_RIGID 24

typedef enum {
  LIGEN_OK = 0,
  LIGEN_ERR_INVALID_ARG = -1,  /* a host-checkable argument is wrong */
  LIGEN_ERR_UNSUPPORTED = -2,  /* valid but beyond the documented limits */
  LIGEN_ERR_OOM = -3,          /* workspace allocation failed */
  LIGEN_ERR_CUDA = -4,         /* a CUDA runtime call or launch failed */
  LIGEN_ERR_TIMEOUT = -5,      /* a bounded device wait expired */
  LIGEN_ERR_BAD_LIGAND = -6,   /* per-ligand status value only */
  LIGEN_ERR_CHECK = -7         /* bounds-checked builds only (LIGEN_CHECKED=1): a
                                  kernel caught a data-dependent index out of range
                                  and skipped the access; results are invalid */
} ligen_status;

typedef enum { LIGEN_F32 = 0 } ligen_dtype;

/* A ligand library in CSR form.
 *   h_atom_off, h_rot_off  HOST copies of atom_off and rot_off (always host).
 *   atom_off [L+1]   ligand l owns atoms atom_off[l] .. atom_off[l+1]-1
 *   xyz      [sum N][3] input conformation, Angstrom, row per atom
 *   type     [sum N]    grid channel of each atom (< grid nc)
 *   bonds    [sum N - L][2] tree edges as LOCAL atom ids (0..N_l-1);
 *                       ligand l's N_l - 1 rows start at row atom_off[l] - l
 *   rot_off  [L+1]   ligand l owns rotatable bonds rot_off[l] .. rot_off[l+1]-1
 *   rot_edge [sum n] each rotatable bond as a LOCAL row id into the ligand's
 *                    bond rows; rotatable bond b of ligand l is torsion b. */
typedef struct ligen_ligands {
  int32_t n_ligands;
  int32_t reserved;
  const int32_t* h_atom_off;
  const int32_t* h_rot_off;
  const int32_t* atom_off;
  const float* xyz;
  const uint8_t* type;
  const int32_t* bonds;
  const int32_t* rot_off;
  const int32_t* rot_edge;
} ligen_ligands_t;

/* Pocket grid: data[z][y][x][c] (channel innermost), node (i, j, k) at
 * origin + spacing * (i, j, k). A point is inside the box when
 * 0 <= (p - origin) / spacing <= n - 1 on every axis. */
typedef struct ligen_grid {
  int32_t nx, ny, nz, nc;
  float origin[3];
  float spacing;
  int32_t dtype;   /* ligen_dtype */
  int32_t reserved;
  const void* data;
} ligen_grid_t;

/* Search settings and optional outputs of ligen_dock_batch.
 *   restarts          R >= 1
 *   n_rigid           1..24: the rigid stage tries cube rotations 0..n_rigid-1
 *   torsion_step_deg  2..360 and a divisor of 360; 360/step candidates per bond
 *   passes            >= 0 sweeps over all rotatable bonds
 *   top_k             1..R poses kept per ligand
 *   mode              0 = greedy search; 1 = exhaustive search (small
 *                     ligands): every restart scores every combination of
 *                     cube rotation 0..n_rigid-1 and torsion increments and
 *                     keeps the best (ties: the first combination in the
 *                     order (k, j_0, .., j_{n-1})); passes and batching are
 *                     ignored, trace must be NULL; every ligand needs at
 *                     most 4 rotatable bonds and n_rigid * (360/step)^n <=
 *                     2^27, else LIGEN_ERR_UNSUPPORTED
 *   seed              restart random stream (SplitMix64 counter hash)
 *   jitter            restart translation = grid centre + U[-jitter, jitter]^3 A
 *   out_penalty       energy of an atom outside the grid box
 *   stream            cudaStream_t or NULL
 * Optional outputs (NULL to skip), same memory space as out_scores:
 *   status      [L]  0 or LIGEN_ERR_BAD_LIGAND
 *   trace       per ligand l, per restart r, D_l = 1 + passes * n_l int16:
 *               the chosen cube rotation, then the chosen increment of every
 *               (pass, bond); ligand l starts at R * (l + passes * rot_off[l]),
 *               restart r at + r * D_l
 *   top_restart [L][K] restart index of each kept pose
 * Optional host-side timing: stage_ms (HOST, [LIGEN_N_STAGES]) receives the
 * device time of each stage measured with CUDA events on `stream`; passing it
 * makes the call synchronise the stream. */
#define LIGEN_N_STAGES 5 /* h2d, grid prep, pack, dock, top-k + d2h */

/* How the docking work of a call is laid out on the GPU (same results).
 *   LIGEN_BATCH_PLAIN    one launch over the library, one CTA per (ligand,
 *                        restart chunk), shared memory sized for the largest
 *                        ligand of the call;
 *   LIGEN_BATCH_BUCKETS  paper §3: ligands are grouped by atom class x
 *                        rotamer class (the bucket ids of ligen_pack_ligands)
 *                        and ordered largest-cost first; each atom class runs
 *                        as one persistent launch (CTAs take work items from a
 *                        device counter) with shared memory sized for that
 *                        class, Eq. 1's b x SM CTAs (b from the occupancy query)
 *                        and the lanes-per-restart / restarts-per-CTA shape
 *                        of the tuning table (ligen_tune_set, ligen_autotune);
 *                        the classes run one after another (a class's
 *                        CTAs keep their SMs until its queue is empty) and
 *                        the whole sequence is captured once into a CUDA
 *                        graph and replayed while the call's shape is
 *                        unchanged;
 *   LIGEN_BATCH_BUCKETS_STATIC  the same groups, shapes and graph, but each
 *                        group is a plain launch of one CTA per work item
 *                        (no device counter), the groups side by side on
 *                        forked streams: the static
 *                        per-bucket launches the persistent form is
 *                        compared against;
 *   LIGEN_BATCH_QUEUE    the whole library in ONE persistent launch: one
 *                        device work queue over every ligand in the
 *                        buckets' largest-cost-first order, the default
 *                        kernel shape, shared memory sized for the
 *                        library's largest ligand, Eq. 1's b x SM CTAs,
 *                        captured into a CUDA graph like the buckets. */
#define LIGEN_BATCH_PLAIN 0
#define LIGEN_BATCH_BUCKETS 1
#define LIGEN_BATCH_BUCKETS_STATIC 2
#define LIGEN_BATCH_QUEUE 3
#define LIGEN_N_BUCKETS 44 /* 4 atom classes x 11 rotamer classes */

/* How the docking kernel stores the grid it samples (built from the
 * caller's FP32 grid inside the call; coordinates and sums stay FP32).
 *   LIGEN_GRID_F32   32 bytes per (cell, channel): the FP32 coefficients of
 *                    the cell's trilinear polynomial;
 *   LIGEN_GRID_F16   16 bytes: the 8 corner values in FP16;
 *   LIGEN_GRID_BF16  16 bytes: the 8 corner values in BF16.
 * The 16-bit formats run with 4, 8, 16 or 32 lanes per restart. */
#define LIGEN_GRID_F32 0
#define LIGEN_GRID_F16 1
#define LIGEN_GRID_BF16 2

typedef struct ligen_params {
  int32_t restarts;
  int32_t n_rigid;
  int32_t torsion_step_deg;
  int32_t passes;
  int32_t top_k;
  int32_t mode;
  uint64_t seed;
  float jitter;
  float out_penalty;
  void* stream;
  int32_t* status;
  int16_t* trace;
  int32_t* top_restart;
  float* stage_ms;
  int32_t batching;     /* LIGEN_BATCH_PLAIN, _BUCKETS, _BUCKETS_STATIC or _QUEUE */
  int32_t grid_format;  /* LIGEN_GRID_F32, LIGEN_GRID_F16 or LIGEN_GRID_BF16 */
  int32_t rescore_fp64; /* 1: re-score the K kept poses of every ligand in
                           FP64 on the GPU (from the caller's FP32 grid
                           values and coordinates) and re-rank them by that
                           score (ties: lower restart); out_scores then
                           holds the FP64 scores rounded to FP32 */
  int32_t reserved3;
  double* scores_f64;   /* optional [L][K], same memory space as out_scores:
                           the FP64 scores (needs rescore_fp64 = 1) */
  int64_t* samples;     /* optional, HOST, 1 value: the atom samples the
                           search needed, summed over all sites: per restart
                           n_rigid * N for the rigid stage plus, for every
                           torsion decision that had to be swept (not a clean
                           bond, see the docking kernel), (360/step - 1) *
                           (moving atoms - 1); exhaustive mode: every
                           combination's N. Counting makes the call wait
                           for its work. */
  float* coords;        /* optional debug output, same memory space as
                           out_scores: the final FP32 atom positions of every
                           restart as the docking kernel holds them, in grid
                           units u = (x - origin) / spacing, ligand l's block
                           at 3 * R * atom_off[l], restart r at + 3 * r * N_l,
                           atom i at + 3 * i (x, y, z); [n_sites][...] for
                           ligen_dock_sites. Greedy mode only. */
} ligen_params_t;

/* Dock every ligand (paper §2, the dock task; cost per §3 follows atoms and
 * rotamers).
 *   out_scores [L][K]  scores of the kept poses, best first (ties: lower
 *                      restart index first)
 *   out_poses  ligand l's K poses start at float K * (7 * l + rot_off[l]);
 *              each pose is 7 + n_l floats: translation t[3] (Angstrom, the
 *              image of the input centroid), unit quaternion q = (w, x, y, z)
 *              with w >= 0, torsion angles theta[n_l] in radians in [-pi, pi).
 *              Atom positions of a pose: x_i = R(q) (T_theta(X0)_i - c0) + t,
 *              where c0 is the input centroid and T_theta turns, bond by bond
 *              in index order, the moving side of rotatable bond b by
 *              theta_b about the axis from its fixed endpoint to its moving
 *              endpoint (right-handed). The moving side is the smaller part
 *              of the tree cut at the bond; on a tie, the part without atom 0.
 * Returns LIGEN_OK or an error code. */
int ligen_dock_batch(const ligen_ligands_t* ligands, const ligen_grid_t* grid,
                     const ligen_params_t* params, float* out_poses, float* out_scores);

/* Dock one library into n_sites docking sites (paper §2: the library is
 * ranked per docking site; §5 screens twelve sites of one target, and the
 * footprint grows with the number of sites). grids[n_sites] are the sites'
 * pocket grids: same channel count, each its own box and spacing, all in
 * host memory or all in device memory. The library is staged and packed once;
 * the grid records of one site at a time live in one buffer sized for the
 * largest site, so device memory grows with the largest grid, not with the
 * number of sites.
 * Outputs are site-major: site g's scores start at out_scores + g * L * K,
 * its poses at out_poses + g * K * (7 * L + total rotatable bonds); trace,
 * top_restart and scores_f64 (when given) are likewise [n_sites][...] with
 * the per-site sizes of ligen_dock_batch; status is written once ([L]; a
 * ligand's status does not depend on the site, given equal channel counts).
 * stage_ms sums the stages over the sites. Site g's outputs are those of
 * ligen_dock_batch(ligands, &grids[g], params, ...), bit for bit: the same
 * seed, restarts and search run in every site.
 * Returns LIGEN_OK or an error code; n_sites < 1, NULL grids or channel
 * counts that differ are LIGEN_ERR_INVALID_ARG. */
int ligen_dock_sites(const ligen_ligands_t* ligands, const ligen_grid_t* grids, int32_t n_sites,
                     const ligen_params_t* params, float* out_poses, float* out_scores);

/* ligen_dock_batch for callers that must not allocate device memory: a
 * host framework whose caching allocator already owns the device's memory,
 * or a latency-bound service that cannot take the device-wide
 * synchronisation a cudaMalloc/cudaFree implies. The paper has no
 * counterpart. Same search and outputs as ligen_dock_batch with default
 * layout settings (bit for bit: the same kernels on the same inputs), with
 * these differences:
 *   - Its scratch is one file-scope device array of LIGEN_STATIC_SCRATCH_BYTES
 *     inside this library (every GPU that loads the library holds it until
 *     the process exits); the call itself allocates nothing. A batch whose
 *     scratch would exceed it is rejected with LIGEN_ERR_UNSUPPORTED before
 *     any device work. With L ligands, A atoms and B rotatable bonds in
 *     total, R restarts and an nx x ny x nz x nc grid, the scratch is the sum
 *     of these ten regions, EACH rounded up to a multiple of 256 bytes:
 *       (nx-1)(ny-1)(nz-1) nc * 32   grid records
 *       16 A                         packed coordinates
 *       4 B, 128 B, 4 B              bond records, moving-atom lists, masks
 *       4 L                          ligand status
 *       4 L R, L R, B R              per-restart scores, rotations, torsions
 *     plus, in bounds-checked builds (LIGEN_CHECKED) only, one more 256-byte
 *     region for the error word. A batch is accepted iff that sum is at most
 *     LIGEN_STATIC_SCRATCH_BYTES.
 *   - Ligands, grid and every output must be device memory
 *     (LIGEN_ERR_INVALID_ARG otherwise).
 *   - Only the plain launch over FP32 grid records runs: grid_format other
 *     than LIGEN_GRID_F32, batching other than LIGEN_BATCH_PLAIN,
 *     rescore_fp64 != 0, scores_f64, stage_ms or samples not NULL, or
 *     mode != 0 are rejected with LIGEN_ERR_UNSUPPORTED (never ignored).
 *     status, trace and top_restart are written as by ligen_dock_batch.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *   - All calls share the one array: two calls that overlap on the GPU (for
 *     instance on different streams without ordering) race and corrupt each
 *     other's results. Each call writes every scratch region before reading
 *     it, so the contents left by the previous call do not matter. */
#define LIGEN_STATIC_SCRATCH_BYTES (32u << 20)
int ligen_dock_batch_static(const ligen_ligands_t* ligands, const ligen_grid_t* grid,
                            const ligen_params_t* params, float* out_poses, float* out_scores);

/* Tuning table of the bucketed layout, one per device (the current one):
 * for bucket b (atom_class * 11 + rotamer_class, 0 .. LIGEN_N_BUCKETS-1) the
 * lanes per restart (2, 4, 8, 16 or 32) and restarts per CTA (a multiple of
 * 32/lanes, lanes * restarts <= 128). Defaults: 8 lanes, 16 restarts. The
 * 16-bit grid formats run with 4 to 32 lanes; other shapes fall back to the
 * default. The table keeps one shape per bucket whatever the record format;
 * shapes tuned on one format can be far from the best on another (measured
 * on GB300, the bimodal library's static per-bucket launches on FP16
 * records with the FP32-tuned shapes: 1224 ms, against 836 ms for the plain
 * FP16 launch), so tune with the format the bucketed calls will use. */
int ligen_tune_set(int32_t bucket, int32_t lanes, int32_t restarts_per_cta);
int ligen_tune_get(int32_t bucket, int32_t* lanes, int32_t* restarts_per_cta);

/* Autotuner: for every bucket present in `ligands` (at most `sample`
 * ligands of each), dock with every candidate shape (lanes per restart x
 * restarts per CTA: 2 x 64, 4 x 16, 4 x 32, 8 x 8, 8 x 16, 16 x 8, 32 x 4;
 * those the record format does not run are skipped), time the docking
 * kernel with CUDA events on
 * params->stream, and store the fastest shape per ligand in the tuning table.
 * Writes the chosen shapes to out_lanes / out_rpc ([LIGEN_N_BUCKETS], HOST,
 * 0 for absent buckets) and each bucket's best time per ligand in
 * out_ms_per_ligand (HOST, nullable). Ligands and grid in device memory.
 * Synchronises the stream. */
int ligen_autotune(const ligen_ligands_t* ligands, const ligen_grid_t* grid, const ligen_params_t* params,
                   int32_t sample, int32_t* out_lanes, int32_t* out_rpc, float* out_ms_per_ligand);

/* Score given poses: the scoring half of the dock task of paper §2 (the
 * task that estimates the ligand's placement in the docking site). The
 * search of ligen_dock_batch keeps the candidates that maximise this score;
 * here the caller supplies the poses. It is not §2's third task, which rates
 * the interaction strength of an already docked ligand.
 * Same pose packing as ligen_dock_batch with K = poses_per_ligand:
 * out_scores[l][p] = S of pose p of ligand l, or -INFINITY for an invalid
 * ligand. `poses` and `out_scores` share one memory space. With 16 or more
 * poses per ligand the ligands are scored by rotatable-bond class (0, 2, 4,
 * 6, 8, 12, 16, 24, 32 bonds at most), one pose per lane, the classes'
 * launches on forked streams, the sequence captured once into a CUDA graph
 * per (stream, call shape) and replayed on `stream` (for the legacy or
 * per-thread default stream, which cannot be captured, the capture is made
 * on a side stream); on a stream that is being captured the launches go
 * into the caller's graph. ligen_release_workspaces() frees the cached
 * graphs. */
int ligen_score_poses(const ligen_ligands_t* ligands, const ligen_grid_t* grid,
                      int32_t poses_per_ligand, const float* poses, float out_penalty,
                      float* out_scores, void* stream);

/* Scoring inputs prepared once for many ligen_score_prepared calls: a
 * caller that scores batch after batch of poses of one library against one
 * grid (a refinement loop, a rescoring service) pays the grid records and
 * the ligand packer once instead of on every call. The paper has no
 * counterpart; it is the scoring of ligen_score_poses split into its
 * per-input and per-pose parts.
 *   ligen_prepare_scoring  builds, on `stream`, the FP32 grid records, the
 *          packed library, the forward-kinematics table (each atom's
 *          owning bond, each bond's parent, the bonds parents first and by
 *          depth, the bond axes) and the scoring plan in one device allocation
 *          owned by the returned handle (*out; NULL on error). Ligands and
 *          grid may be host or device memory; the handle keeps no pointer
 *          to them (host inputs: the call waits for their copies).
 *          LIGEN_ERR_OOM when the allocation fails or exceeds the
 *          ligen_set_workspace_limit cap.
 *   ligen_score_prepared   ligen_score_poses on the prepared inputs (same
 *          poses packing, outputs, results, launches and graphs); `poses` and `out_scores`
 *          in one memory space. Stream-ordered after the preparation when
 *          on the same stream; otherwise the caller orders the streams.
 *          Must run on the device the handle was prepared on.
 *   ligen_release_prepared frees the handle (NULL: no-op). Its cudaFree
 *          waits for the device, so release after the last call that uses
 *          it, and never during a stream capture. */
typedef struct ligen_prepared ligen_prepared_t;
int ligen_prepare_scoring(const ligen_ligands_t* ligands, const ligen_grid_t* grid, void* stream,
                          ligen_prepared_t** out);
int ligen_score_prepared(const ligen_prepared_t* prep, int32_t poses_per_ligand, const float* poses,
                         float out_penalty, float* out_scores, void* stream);
int ligen_release_prepared(ligen_prepared_t* prep);

/* Gradient of the pose score with respect to translation, rotation and
 * torsions (the differentiable form of the score; no paper counterpart).
 * For pose p of ligand l (packing as ligen_score_poses), out_scores[l][p] =
 * S and out_grads holds dS/dpose in the pose's own slot: dS/dt[3], dS/dq[4]
 * (through q/|q|, so orthogonal to q), dS/dtheta[n_l]. E is differentiated inside the cell that
 * holds the atom (one-sided at cell faces); atoms outside the box contribute
 * no gradient. Atom coordinates are rebuilt from the pose, never stored.
 * Invalid ligands: S = -INFINITY, zero gradient. `poses`, `out_scores` and
 * `out_grads` share one memory space. */
int ligen_pose_grad(const ligen_ligands_t* ligands, const ligen_grid_t* grid, int32_t poses_per_ligand,
                    const float* poses, float out_penalty, float* out_scores, float* out_grads, void* stream);

/* Gradient refinement of poses in place: for every pose, `steps` iterations
 * of normalised-step projected ascent. An iteration moves t by step_t (A)
 * along dS/dt / |dS/dt| (then clamps t to the grid box), q^ = q/|q| by step_q
 * along dS/dq / |dS/dq| (then renormalises), theta by step_theta (rad) along
 * dS/dtheta / |dS/dtheta| (then wraps to [-pi, pi)); a block with a zero
 * gradient does not move. The move is kept when it raises S; otherwise the
 * three step sizes are halved. On return the pose has w >= 0 and
 * out_scores[l][p] holds its S. out_accept (nullable, [L * P][steps], same
 * memory space) records 1 for kept moves. */
int ligen_refine_poses(const ligen_ligands_t* ligands, const ligen_grid_t* grid, int32_t poses_per_ligand,
                       float* poses, float out_penalty, int32_t steps, float step_t, float step_q, float step_theta,
                       float* out_scores, int8_t* out_accept, void* stream);

/* The ligand packer on its own, for inspection (paper §3: ligands are
 * classified by atom count and rotamer count).
 *   frag_bits [sum n][8]  bit i of word i/32 set when atom i is on the moving
 *                         side of the rotatable bond
 *   axis      [sum n][2]  (fixed endpoint u, moving endpoint v), local ids
 *   bucket    [L]  atom_class * 11 + rotamer_class, atom classes <=32, <=64,
 *                  <=128, larger; rotamer classes with upper edges
 *                  0,1,2,3,4,6,8,12,16,24,32
 *   status    [L]  0 or LIGEN_ERR_BAD_LIGAND
 * Any output may be NULL. Outputs share one memory space. */
int ligen_pack_ligands(const ligen_ligands_t* ligands, int32_t n_channels, uint32_t* frag_bits,
                       int32_t* axis, int32_t* bucket, int32_t* status, void* stream);

/* The packer's bond interaction masks, which the docking kernel uses to
 * skip sweeps that cannot change the pose (no counterpart in the paper).
 *   touch [sum n]  for ligand l's bond b' (entry rot_off[l] + b'), bit b is
 *                  set when turning b' moves an atom that bond b's sweep
 *                  reads: an atom of b's moving side (v_b included) or b's
 *                  fixed end u_b. Turning b' moves its moving side except
 *                  v_b'. Bit b' is always set. 0 for an invalid ligand.
 * `touch` may be host or device memory. */
int ligen_pack_touch(const ligen_ligands_t* ligands, int32_t n_channels, uint32_t* touch, void* stream);

/* Paper Eq. 1: ligands per bucket l = b * SM * t / ws for the docking
 * kernel instance used for ligands of up to max_atoms atoms, with b from the
 * CUDA occupancy query, SM the device's multiprocessor count, t the kernel's
 * threads per block and ws the warp size. Writes the four factors when the
 * pointers are not NULL. Returns l (> 0) or an error code. */
int64_t ligen_bucket_size(int32_t max_atoms, int32_t* b, int32_t* sm, int32_t* t, int32_t* ws);

/* Measurement utility (the paper has no counterpart): the achievable rate of
 * the docking kernel's memory access pattern on this device. Every thread of
 * a full-device launch makes `loads_per_thread` aligned loads of
 * `bytes_per_load` (4, 8, 16 or 32) bytes, each from the start of a uniformly
 * random 32-byte record of `records` (DEVICE, n_records * 8 floats, 32-byte
 * aligned; 32-byte loads skip L1 allocation as the FP32 sampler's do), and
 * discards the values (`sink`, DEVICE, 1 float, is written
 * only to keep the loads alive). *loads_done receives the number of loads
 * made and *ms_out their device time (CUDA events on `stream`; the call
 * synchronises). With 32-byte loads over a buffer that fits in L2 this is
 * the docking kernel's gather ceiling. Returns LIGEN_OK or an error code. */
int ligen_probe_gather(const float* records, int64_t n_records, int32_t bytes_per_load, int32_t loads_per_thread,
                       float* sink, double* loads_done, float* ms_out, void* stream);

/* Measurement utility (no paper counterpart): streaming read bandwidth of
 * the L2. A full-device launch reads `buffer` (DEVICE, n_bytes, 16-byte
 * aligned, n_bytes a multiple of 16) `passes` times with coalesced 16-byte
 * loads that bypass L1 (ld.global.cg); after one untimed pass the buffer is
 * L2-resident when it fits. *bytes_done receives the bytes read in the timed
 * passes and *ms_out their device time (CUDA events on `stream`; the call
 * synchronises). `sink` (DEVICE, 1 float) keeps the loads alive. Returns
 * LIGEN_OK or an error code. */
int ligen_probe_stream(const void* buffer, int64_t n_bytes, int32_t passes, float* sink, double* bytes_done,
                       float* ms_out, void* stream);

/* Release every cached workspace of the calling thread's current device,
 * with the cached CUDA graphs and the side streams and events of the forked
 * launches (created per calling stream on first use). Waits for the work on
 * those streams. No other library call may run on that device meanwhile
 * (from any thread): they share these caches. */
int ligen_release_workspaces(void);

/* Caps every internal workspace at `bytes` (<= 0: no cap, the default), for
 * the whole process. A call whose workspace would exceed the cap fails with
 * LIGEN_ERR_OOM before any device work, as it does when cudaMalloc fails;
 * workspaces already allocated are kept. Lets a caller bound the library's
 * device memory, and tests inject an allocation failure without exhausting
 * the GPU. */
int ligen_set_workspace_limit(int64_t bytes);

/* Message of the last error on the calling thread ("" if none). */
const char* ligen_last_error(void);

int ligen_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LIGEN_H */
