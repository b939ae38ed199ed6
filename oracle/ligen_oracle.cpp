// ORACLE — plain, slow, single-threaded FP64 reference of the docking pose
// search. This is TEST INFRASTRUCTURE: only the tests, the smoke check and the
// benchmark's CPU-baseline leg may load it. The CUDA library never links,
// includes or calls anything here, and this file includes nothing of it.
//
// What it computes. The paper (§2) names the docking task: estimate the 3D
// placement of a ligand's atoms in a docking site. §3 states that the work
// grows with the ligand's atoms and its *rotamers*, the rotatable subsets of
// atoms that change shape without changing chemistry. The paper does not spell
// the search out, so this file fixes one reading of it and writes every step
// out in the most direct form:
//
//   for every restart r:    random orientation q_r and translation t_r
//   rigid stage:            try the 24 rotations g_k of the cube, keep the best
//   sweep, pass by pass:    for every rotatable bond b in index order, try the
//                           torsion increments j * step (j = 0 .. 360/step-1)
//                           of its moving fragment, keep the best
//   result:                 the restart's final pose and score; the ligand
//                           keeps the top K restarts.
//
// Each candidate pose is rebuilt from its parameters (t, q, theta) and every
// atom is re-scored: no caching, no incremental update.
//
// Parity status: every function below is pinned by CPU tests against values
// fixed by mathematics or by independent library routines (scipy rotations and
// interpolation, networkx components, brute-force enumeration, published
// SplitMix64 outputs, the paper's Eq. 1 and Table 1).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;

struct Vec {
  double x, y, z;
};
Vec add(Vec a, Vec b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
Vec sub(Vec a, Vec b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
Vec scale(Vec a, double s) { return {a.x * s, a.y * s, a.z * s}; }
double dot(Vec a, Vec b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
Vec cross(Vec a, Vec b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

}  // namespace

extern "C" {

// One ligand, host arrays.
//   xyz   [N][3] input conformation (Angstrom)
//   type  [N]    grid channel of each atom
//   bonds [N-1][2] tree edges, local atom ids
//   rot_edge [n] rows of `bonds` that are rotatable
struct or_ligand {
  int32_t n_atoms;
  int32_t n_rot;
  const double* xyz;
  const uint8_t* type;
  const int32_t* bonds;
  const int32_t* rot_edge;
};

// Pocket grid: values[z][y][x][c], node (i,j,k) at origin + spacing*(i,j,k).
struct or_grid {
  int32_t nx, ny, nz, nc;
  double origin[3];
  double spacing;
  const double* v;
};

struct or_params {
  int32_t restarts;
  int32_t n_rigid;    // first n_rigid of the 24 cube rotations (24 = all)
  int32_t step_deg;   // torsion increment; 360 / step_deg candidates per bond
  int32_t passes;     // sweeps over all rotatable bonds
  int32_t top_k;
  int32_t reserved;
  uint64_t seed;
  double jitter;      // translation jitter half-width (Angstrom)
  double penalty;     // energy of an atom outside the grid box
};

// ---------------------------------------------------------------- RNG -----
// SplitMix64 (Steele, Lea, Flood 2014): the first output of a SplitMix64
// generator whose state is x.
uint64_t or_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Uniform number k (0..7) of restart `restart` of ligand `lig`:
// counter c = (lig * 2^32 + restart) * 8 + k, z = SplitMix64(seed XOR c),
// u = (z >> 40) * 2^-24, a 24-bit value in [0, 1).
double or_uniform(uint64_t seed, int64_t lig, int64_t restart, int32_t k) {
  uint64_t c = ((uint64_t)lig << 32) + (uint64_t)restart;
  c = c * 8u + (uint64_t)k;
  uint64_t z = or_splitmix64(seed ^ c);
  return (double)(z >> 40) * (1.0 / 16777216.0);
}

// ---------------------------------------------------------- rotations -----
// Quaternions are (w, x, y, z).

// Shoemake (1992) uniform random rotation from three uniforms:
// q = (sqrt(u0) cos 2pi u2, sqrt(1-u0) sin 2pi u1, sqrt(1-u0) cos 2pi u1,
//      sqrt(u0) sin 2pi u2).
void or_shoemake(const double* u, double* q) {
  double r1 = std::sqrt(1.0 - u[0]);
  double r2 = std::sqrt(u[0]);
  double a = 2.0 * kPi * u[1];
  double b = 2.0 * kPi * u[2];
  q[0] = r2 * std::cos(b);
  q[1] = r1 * std::sin(a);
  q[2] = r1 * std::cos(a);
  q[3] = r2 * std::sin(b);
}

// Hamilton product a * b (apply b first, then a).
void or_quat_mul(const double* a, const double* b, double* o) {
  double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
  o[0] = w; o[1] = x; o[2] = y; o[3] = z;
}

// Rotation matrix (row-major) of q / |q|.
void or_quat_to_mat(const double* qin, double* m) {
  double n = std::sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
  double w = qin[0] / n, x = qin[1] / n, y = qin[2] / n, z = qin[3] / n;
  m[0] = 1 - 2 * (y * y + z * z); m[1] = 2 * (x * y - w * z);     m[2] = 2 * (x * z + w * y);
  m[3] = 2 * (x * y + w * z);     m[4] = 1 - 2 * (x * x + z * z); m[5] = 2 * (y * z - w * x);
  m[6] = 2 * (x * z - w * y);     m[7] = 2 * (y * z + w * x);     m[8] = 1 - 2 * (x * x + y * y);
}

// The 24 proper rotations of the cube, as (axis, angle), in this order:
//   0      identity
//   1-3    180 deg about x, y, z
//   4-9    +90, -90 about x; +90, -90 about y; +90, -90 about z
//   10-17  120 deg about the body diagonal (sx, sy, sz), m = k - 10,
//          sx = -1 if m & 4, sy = -1 if m & 2, sz = -1 if m & 1 (else +1)
//   18-23  180 deg about the face diagonals (1,1,0), (1,-1,0), (0,1,1),
//          (0,1,-1), (1,0,1), (1,0,-1)
void or_octahedral(int32_t k, double* q) {
  double ax[3] = {1, 0, 0};
  double ang = 0.0;
  if (k == 0) {
    ang = 0.0;
  } else if (k <= 3) {
    ax[0] = (k == 1); ax[1] = (k == 2); ax[2] = (k == 3);
    ang = kPi;
  } else if (k <= 9) {
    int a = (k - 4) / 2;
    ax[0] = (a == 0); ax[1] = (a == 1); ax[2] = (a == 2);
    ang = ((k - 4) % 2 == 0) ? kPi / 2 : -kPi / 2;
  } else if (k <= 17) {
    int m = k - 10;
    ax[0] = (m & 4) ? -1 : 1; ax[1] = (m & 2) ? -1 : 1; ax[2] = (m & 1) ? -1 : 1;
    ang = 2.0 * kPi / 3.0;
  } else {
    static const double d[6][3] = {{1, 1, 0}, {1, -1, 0}, {0, 1, 1}, {0, 1, -1}, {1, 0, 1}, {1, 0, -1}};
    ax[0] = d[k - 18][0]; ax[1] = d[k - 18][1]; ax[2] = d[k - 18][2];
    ang = kPi;
  }
  double n = std::sqrt(ax[0] * ax[0] + ax[1] * ax[1] + ax[2] * ax[2]);
  double s = std::sin(ang / 2) / n;
  q[0] = std::cos(ang / 2);
  q[1] = ax[0] * s; q[2] = ax[1] * s; q[3] = ax[2] * s;
}

// Rodrigues rotation of point p by angle theta about the line through `a`
// with direction `dir` (right-handed, dir need not be unit).
void or_rodrigues(const double* p, const double* a, const double* dir, double theta, double* out) {
  Vec k = {dir[0], dir[1], dir[2]};
  k = scale(k, 1.0 / std::sqrt(dot(k, k)));
  Vec v = sub({p[0], p[1], p[2]}, {a[0], a[1], a[2]});
  double c = std::cos(theta), s = std::sin(theta);
  Vec r = add(add(scale(v, c), scale(cross(k, v), s)), scale(k, dot(k, v) * (1.0 - c)));
  out[0] = a[0] + r.x; out[1] = a[1] + r.y; out[2] = a[2] + r.z;
}

// ---------------------------------------------------------- fragments -----
// Checks that the bonds form a tree on N atoms and that the rotatable edge
// ids and atom types are in range. Returns 0 when valid, 1 otherwise.
int32_t or_validate(const or_ligand* L, int32_t n_channels) {
  int N = L->n_atoms;
  if (N < 1) return 1;
  for (int i = 0; i < N; ++i)
    if (L->type[i] >= n_channels) return 1;
  for (int e = 0; e < N - 1; ++e)
    for (int s = 0; s < 2; ++s)
      if (L->bonds[2 * e + s] < 0 || L->bonds[2 * e + s] >= N) return 1;
  for (int r = 0; r < L->n_rot; ++r)
    if (L->rot_edge[r] < 0 || L->rot_edge[r] >= N - 1) return 1;
  // connected with N-1 edges <=> tree
  std::vector<char> seen(N, 0);
  std::vector<int> stack{0};
  seen[0] = 1;
  int count = 1;
  while (!stack.empty()) {
    int x = stack.back();
    stack.pop_back();
    for (int e = 0; e < N - 1; ++e) {
      int a = L->bonds[2 * e], b = L->bonds[2 * e + 1];
      int y = (a == x) ? b : (b == x) ? a : -1;
      if (y >= 0 && !seen[y]) {
        seen[y] = 1;
        ++count;
        stack.push_back(y);
      }
    }
  }
  return count == N ? 0 : 1;
}

// Moving fragment of each rotatable bond. Cutting rotatable edge (a, b)
// splits the tree in two; the moving side is the smaller one, and on a tie
// the side that does not contain atom 0. mask[r][i] = 1 when atom i moves;
// axis[r] = (u, v) with u the fixed endpoint and v the moving endpoint.
// Returns 0, or 1 when the ligand is not a valid tree.
int32_t or_fragments(const or_ligand* L, uint8_t* mask, int32_t* axis) {
  int N = L->n_atoms;
  if (or_validate(L, 256)) return 1;
  for (int r = 0; r < L->n_rot; ++r) {
    int cut = L->rot_edge[r];
    int a = L->bonds[2 * cut], b = L->bonds[2 * cut + 1];
    // component of a once the edge is removed
    std::vector<char> side(N, 0);
    std::vector<int> stack{a};
    side[a] = 1;
    while (!stack.empty()) {
      int x = stack.back();
      stack.pop_back();
      for (int e = 0; e < N - 1; ++e) {
        if (e == cut) continue;
        int p = L->bonds[2 * e], q = L->bonds[2 * e + 1];
        int y = (p == x) ? q : (q == x) ? p : -1;
        if (y >= 0 && !side[y]) {
          side[y] = 1;
          stack.push_back(y);
        }
      }
    }
    int na = 0;
    for (int i = 0; i < N; ++i) na += side[i];
    int nb = N - na;
    bool a_moves = (na < nb) || (na == nb && !side[0]);
    for (int i = 0; i < N; ++i) mask[(size_t)r * N + i] = a_moves ? side[i] : !side[i];
    axis[2 * r] = a_moves ? b : a;
    axis[2 * r + 1] = a_moves ? a : b;
  }
  return 0;
}

// ---------------------------------------------------------- bucketing -----
// Paper §3: atom classes sit on warp-size multiples (its example: up to 32,
// up to 64, the rest). Classes here: <=32, <=64, <=128, larger.
int32_t or_atom_class(int32_t n_atoms) {
  if (n_atoms <= 32) return 0;
  if (n_atoms <= 64) return 1;
  if (n_atoms <= 128) return 2;
  return 3;
}

// Paper §3: rotamer classes split the range unevenly, finer at low counts.
// Upper edges: 0,1,2,3,4,6,8,12,16,24,32 (11 classes; 33+ shares the last).
int32_t or_rot_class(int32_t n_rot) {
  static const int edges[11] = {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
  for (int c = 0; c < 11; ++c)
    if (n_rot <= edges[c]) return c;
  return 10;
}

int32_t or_bucket_id(int32_t n_atoms, int32_t n_rot) {
  return or_atom_class(n_atoms) * 11 + or_rot_class(n_rot);
}

// Paper Eq. 1: ligands per bucket l = b * SM * t / ws.
int64_t or_eq1_bucket_size(int64_t b, int64_t sm, int64_t t, int64_t ws) {
  return b * sm * t / ws;
}

// ------------------------------------------------------------ scoring -----
// Trilinear sample of channel c at point x. u = (x - origin) / spacing per
// axis; the point is inside iff 0 <= u <= n-1 on every axis; the cell is
// i = min(floor(u), n-2) and f = u - i; the value is the sum over the 8
// corners of V * prod((1-f) or f). Sets *inbox; returns 0 when outside.
double or_trilinear(const or_grid* g, int32_t c, const double* x, int32_t* inbox) {
  int n[3] = {g->nx, g->ny, g->nz};
  double u[3];
  int i[3];
  double f[3];
  for (int a = 0; a < 3; ++a) {
    u[a] = (x[a] - g->origin[a]) / g->spacing;
    if (!(u[a] >= 0.0 && u[a] <= n[a] - 1)) {
      *inbox = 0;
      return 0.0;
    }
    i[a] = std::min((int)std::floor(u[a]), n[a] - 2);
    f[a] = u[a] - i[a];
  }
  *inbox = 1;
  double e = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
        size_t node = (((size_t)(i[2] + dz) * g->ny + (i[1] + dy)) * g->nx + (i[0] + dx));
        e += w * g->v[node * g->nc + c];
      }
  return e;
}

// Gradient (d/dx, d/dy, d/dz, per Angstrom) of the trilinear sample inside its
// cell: the derivative of the corner-weighted sum with the weight of the
// differentiated axis replaced by -1 (corner 0) or +1 (corner 1), over the
// spacing. Zero outside the box. Returns the value as or_trilinear does.
double or_trilinear_grad(const or_grid* g, int32_t c, const double* x, double* grad, int32_t* inbox) {
  int n[3] = {g->nx, g->ny, g->nz};
  double u[3], f[3];
  int i[3];
  grad[0] = grad[1] = grad[2] = 0.0;
  for (int a = 0; a < 3; ++a) {
    u[a] = (x[a] - g->origin[a]) / g->spacing;
    if (!(u[a] >= 0.0 && u[a] <= n[a] - 1)) {
      *inbox = 0;
      return 0.0;
    }
    i[a] = std::min((int)std::floor(u[a]), n[a] - 2);
    f[a] = u[a] - i[a];
  }
  *inbox = 1;
  double e = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double wx = dx ? f[0] : 1 - f[0], wy = dy ? f[1] : 1 - f[1], wz = dz ? f[2] : 1 - f[2];
        double sx = dx ? 1.0 : -1.0, sy = dy ? 1.0 : -1.0, sz = dz ? 1.0 : -1.0;
        size_t node = (((size_t)(i[2] + dz) * g->ny + (i[1] + dy)) * g->nx + (i[0] + dx));
        double v = g->v[node * g->nc + c];
        e += wx * wy * wz * v;
        grad[0] += sx * wy * wz * v / g->spacing;
        grad[1] += wx * sy * wz * v / g->spacing;
        grad[2] += wx * wy * sz * v / g->spacing;
      }
  return e;
}

// Score of a set of atom positions: S = -sum_i E_i, with E_i the trilinear
// value of atom i's channel, or `penalty` when the atom is outside the box.
// Also returns D = max(|S|, sum_i |E_i|), if E is not null each E_i, and if
// Gs is not null the position sensitivity Gs = sum_i |grad E_i| |x_i - origin|:
// a relative perturbation eps of every atom's grid coordinate moves S by at
// most about eps * Gs.
double or_score_coords(const or_ligand* L, const or_grid* g, const double* xyz, double penalty,
                       double* D, double* E, double* Gs) {
  double s = 0.0, a = 0.0, sens = 0.0;
  for (int i = 0; i < L->n_atoms; ++i) {
    int32_t inb = 0;
    double gr[3];
    double e = or_trilinear_grad(g, L->type[i], xyz + 3 * i, gr, &inb);
    if (!inb) e = penalty;
    if (E) E[i] = e;
    s -= e;
    a += std::fabs(e);
    double r[3] = {xyz[3 * i] - g->origin[0], xyz[3 * i + 1] - g->origin[1], xyz[3 * i + 2] - g->origin[2]};
    sens += std::sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]) *
            std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  }
  if (D) *D = std::max(std::fabs(s), a);
  if (Gs) *Gs = sens;
  return s;
}

// Atom positions of pose (t, q, theta) = pose[0..2], pose[3..6], pose[7..]:
// x_i = R(q/|q|) (T_theta(X0)_i - c0) + t, with c0 the unweighted centroid of
// the input conformation X0 and T_theta the torsion rotations applied bond by
// bond in index order, bond b turning its moving atoms by theta_b about the
// current axis from its fixed endpoint u to its moving endpoint v.
void or_pose_coords(const or_ligand* L, const uint8_t* mask, const int32_t* axis,
                    const double* pose, double* out) {
  int N = L->n_atoms;
  std::vector<double> y(L->xyz, L->xyz + 3 * N);
  for (int b = 0; b < L->n_rot; ++b) {
    int u = axis[2 * b], v = axis[2 * b + 1];
    double pv[3] = {y[3 * v], y[3 * v + 1], y[3 * v + 2]};
    double dir[3] = {y[3 * v] - y[3 * u], y[3 * v + 1] - y[3 * u + 1], y[3 * v + 2] - y[3 * u + 2]};
    for (int i = 0; i < N; ++i) {
      if (!mask[(size_t)b * N + i]) continue;
      double o[3];
      or_rodrigues(&y[3 * i], pv, dir, pose[7 + b], o);
      y[3 * i] = o[0]; y[3 * i + 1] = o[1]; y[3 * i + 2] = o[2];
    }
  }
  double c0[3] = {0, 0, 0};
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < 3; ++a) c0[a] += L->xyz[3 * i + a];
  for (int a = 0; a < 3; ++a) c0[a] /= N;
  double m[9];
  or_quat_to_mat(pose + 3, m);
  for (int i = 0; i < N; ++i) {
    double d[3] = {y[3 * i] - c0[0], y[3 * i + 1] - c0[1], y[3 * i + 2] - c0[2]};
    for (int r = 0; r < 3; ++r)
      out[3 * i + r] = m[3 * r] * d[0] + m[3 * r + 1] * d[1] + m[3 * r + 2] * d[2] + pose[r];
  }
}

// Score of pose (t, q, theta): or_pose_coords, then or_score_coords. The
// ligand must be valid (or_validate); mask and axis come from or_fragments.
double or_score_pose(const or_ligand* L, const or_grid* g, const uint8_t* mask, const int32_t* axis,
                     const double* pose, double penalty, double* D, double* E, double* Gs) {
  std::vector<double> x(3 * (size_t)L->n_atoms);
  or_pose_coords(L, mask, axis, pose, x.data());
  return or_score_coords(L, g, x.data(), penalty, D, E, Gs);
}

// Analytic gradient of S(pose) = -sum_i E(x_i) with respect to the pose
// parameters (t[3], q[4], theta[n]); returns S.
//   x_i = R(q^) y_i + t, y_i = T_theta(X0)_i - c0, q^ = q / |q|.
//   dS/dx_i = g_i = -grad E(x_i) (zero outside the box, one-sided at cell
//   faces: the derivative inside the cell that holds x_i);
//   dS/dt = sum_i g_i;
//   dS/dq^_k = sum_i g_i . (dR/dq^_k) y_i, with R written as the polynomial
//   in (w, x, y, z) of or_quat_to_mat, and dS/dq = (I - q^ q^T) dS/dq^ / |q|;
//   dS/dtheta_b = sum_{i in M_b} g_i . (w_b x (x_i - x_v)), w_b the unit axis
//   of bond b from x_u to x_v in the final pose: torsions commute, so theta_b
//   may be taken as the last rotation applied.
double or_pose_grad(const or_ligand* L, const or_grid* g, const uint8_t* mask, const int32_t* axis,
                    const double* pose, double penalty, double* grad) {
  const int N = L->n_atoms, n = L->n_rot;
  std::vector<double> x(3 * (size_t)N);
  or_pose_coords(L, mask, axis, pose, x.data());
  // body coordinates y_i = R^T (x_i - t)
  double qn = std::sqrt(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
  double w = pose[3] / qn, qx = pose[4] / qn, qy = pose[5] / qn, qz = pose[6] / qn;
  double m[9];
  or_quat_to_mat(pose + 3, m);
  // dR/dq^ for R(w,x,y,z) = [[1-2(y2+z2), 2(xy-wz), 2(xz+wy)], [2(xy+wz), 1-2(x2+z2), 2(yz-wx)],
  //                          [2(xz-wy), 2(yz+wx), 1-2(x2+y2)]]
  const double dR[4][9] = {
      {0, -2 * qz, 2 * qy, 2 * qz, 0, -2 * qx, -2 * qy, 2 * qx, 0},
      {0, 2 * qy, 2 * qz, 2 * qy, -4 * qx, -2 * w, 2 * qz, 2 * w, -4 * qx},
      {-4 * qy, 2 * qx, 2 * w, 2 * qx, 0, 2 * qz, -2 * w, 2 * qz, -4 * qy},
      {-4 * qz, -2 * w, 2 * qx, 2 * w, -4 * qz, 2 * qy, 2 * qx, 2 * qy, 0}};
  for (int a = 0; a < 7 + n; ++a) grad[a] = 0.0;
  double S = 0.0, dqh[4] = {0, 0, 0, 0};
  std::vector<double> gi(3 * (size_t)N);
  for (int i = 0; i < N; ++i) {
    int32_t inb = 0;
    double gr[3];
    double e = or_trilinear_grad(g, L->type[i], &x[3 * i], gr, &inb);
    if (!inb) e = penalty;
    S -= e;
    for (int a = 0; a < 3; ++a) {
      gi[3 * i + a] = -gr[a];
      grad[a] += -gr[a];
    }
    double d[3] = {x[3 * i] - pose[0], x[3 * i + 1] - pose[1], x[3 * i + 2] - pose[2]};
    double y[3];
    for (int r = 0; r < 3; ++r) y[r] = m[r] * d[0] + m[3 + r] * d[1] + m[6 + r] * d[2];
    for (int k = 0; k < 4; ++k)
      for (int r = 0; r < 3; ++r)
        dqh[k] += gi[3 * i + r] * (dR[k][3 * r] * y[0] + dR[k][3 * r + 1] * y[1] + dR[k][3 * r + 2] * y[2]);
  }
  const double qh[4] = {w, qx, qy, qz};
  double proj = 0.0;
  for (int k = 0; k < 4; ++k) proj += qh[k] * dqh[k];
  for (int k = 0; k < 4; ++k) grad[3 + k] = (dqh[k] - qh[k] * proj) / qn;
  for (int b = 0; b < n; ++b) {
    const int u = axis[2 * b], v = axis[2 * b + 1];
    double om[3] = {x[3 * v] - x[3 * u], x[3 * v + 1] - x[3 * u + 1], x[3 * v + 2] - x[3 * u + 2]};
    double len = std::sqrt(om[0] * om[0] + om[1] * om[1] + om[2] * om[2]);
    for (int a = 0; a < 3; ++a) om[a] /= len;
    double acc = 0.0;
    for (int i = 0; i < N; ++i) {
      if (!mask[(size_t)b * N + i]) continue;
      double d[3] = {x[3 * i] - x[3 * v], x[3 * i + 1] - x[3 * v + 1], x[3 * i + 2] - x[3 * v + 2]};
      double c[3] = {om[1] * d[2] - om[2] * d[1], om[2] * d[0] - om[0] * d[2], om[0] * d[1] - om[1] * d[0]};
      acc += gi[3 * i] * c[0] + gi[3 * i + 1] * c[1] + gi[3 * i + 2] * c[2];
    }
    grad[7 + b] = acc;
  }
  return S;
}

// Gradient refinement of one pose: `steps` iterations of normalised-step
// projected ascent. Each iteration proposes
//   t' = clamp_box(t + st * g_t / |g_t|)
//   q' = (q^ + sq * g_q / |g_q|) / |.|            (q^ = q / |q|)
//   theta' = wrap(theta + sth * g_theta / |g_theta|)
// from the gradient g at the current pose (a block with a zero gradient does
// not move), and accepts it when S(pose') > S(pose); otherwise st, sq and sth
// are halved and the pose is kept. The final quaternion is made w >= 0.
// accept[s] = 1 when step s was accepted; gap[s] = S(pose') - S(pose).
// Returns the final score.
double or_refine_pose(const or_ligand* L, const or_grid* g, const uint8_t* mask, const int32_t* axis,
                      double* pose, double penalty, int32_t steps, double st, double sq, double sth,
                      int8_t* accept, double* gap) {
  const int n = L->n_rot, plen = 7 + n;
  std::vector<double> grad(plen), cand(plen);
  const double lo[3] = {g->origin[0], g->origin[1], g->origin[2]};
  const double hi[3] = {g->origin[0] + g->spacing * (g->nx - 1), g->origin[1] + g->spacing * (g->ny - 1),
                        g->origin[2] + g->spacing * (g->nz - 1)};
  double S = or_pose_grad(L, g, mask, axis, pose, penalty, grad.data());
  for (int s = 0; s < steps; ++s) {
    double nt = 0, nq = 0, nth = 0;
    for (int a = 0; a < 3; ++a) nt += grad[a] * grad[a];
    for (int a = 3; a < 7; ++a) nq += grad[a] * grad[a];
    for (int a = 7; a < plen; ++a) nth += grad[a] * grad[a];
    nt = std::sqrt(nt); nq = std::sqrt(nq); nth = std::sqrt(nth);
    double qn = std::sqrt(pose[3] * pose[3] + pose[4] * pose[4] + pose[5] * pose[5] + pose[6] * pose[6]);
    for (int a = 0; a < 3; ++a) {
      double v = pose[a] + (nt > 0 ? st * grad[a] / nt : 0.0);
      cand[a] = std::min(std::max(v, lo[a]), hi[a]);
    }
    double qq[4], qm = 0;
    for (int a = 0; a < 4; ++a) {
      qq[a] = pose[3 + a] / qn + (nq > 0 ? sq * grad[3 + a] / nq : 0.0);
      qm += qq[a] * qq[a];
    }
    qm = std::sqrt(qm);
    for (int a = 0; a < 4; ++a) cand[3 + a] = qq[a] / qm;
    for (int a = 7; a < plen; ++a) {
      double v = pose[a] + (nth > 0 ? sth * grad[a] / nth : 0.0);
      v = std::fmod(v + kPi, 2.0 * kPi);
      if (v < 0) v += 2.0 * kPi;
      cand[a] = v - kPi;
    }
    double S2 = or_score_pose(L, g, mask, axis, cand.data(), penalty, nullptr, nullptr, nullptr);
    if (gap) gap[s] = S2 - S;
    if (S2 > S) {
      for (int a = 0; a < plen; ++a) pose[a] = cand[a];
      S = or_pose_grad(L, g, mask, axis, pose, penalty, grad.data());
      if (accept) accept[s] = 1;
    } else {
      st *= 0.5; sq *= 0.5; sth *= 0.5;
      if (accept) accept[s] = 0;
    }
  }
  if (pose[3] < 0)
    for (int a = 3; a < 7; ++a) pose[a] = -pose[a];
  return S;
}

// Torsion angle of `count` increments of step_deg degrees, wrapped to
// [-180, 180) degrees, in radians.
double or_torsion_angle(int32_t count, int32_t step_deg) {
  int deg = (int)(((int64_t)count * step_deg) % 360);
  if (deg < 0) deg += 360;
  if (deg >= 180) deg -= 360;
  return deg * kPi / 180.0;
}

// Initial orientation and translation of a restart: q_r from Shoemake with
// uniforms 0..2, t_r = grid centre + (2 u_k - 1) * jitter for k = 3, 4, 5.
void or_restart_init(const or_grid* g, const or_params* P, int64_t lig, int64_t restart,
                     double* q, double* t) {
  double u[6];
  for (int k = 0; k < 6; ++k) u[k] = or_uniform(P->seed, lig, restart, k);
  or_shoemake(u, q);
  int n[3] = {g->nx, g->ny, g->nz};
  for (int a = 0; a < 3; ++a)
    t[a] = g->origin[a] + g->spacing * (n[a] - 1) / 2.0 + (2.0 * u[3 + a] - 1.0) * P->jitter;
}

// Greedy search of one ligand, restarts [r_begin, r_end).
// Per restart (index j = r - r_begin), with n = L->n_rot, D = 1 + passes*n:
//   score[j]             final score
//   pose[j][7+n]         final pose (t, q with w >= 0, theta wrapped)
//   trace[j][D]          chosen k, then chosen increment per (pass, bond)
//   gap[j][D], dn[j][D]  best minus second-best score of each decision, and
//                        D = max(|S|, sum |E|) of its best candidate
//   gs[j][D]             position sensitivity Gs of the best candidate
// Ties go to the lowest index. Returns 0, or 1 for an invalid ligand.
int32_t or_dock_ligand(const or_ligand* L, const or_grid* g, const or_params* P, int64_t lig,
                       int32_t r_begin, int32_t r_end, double* score, double* pose,
                       int16_t* trace, double* gap, double* dn, double* gs) {
  int N = L->n_atoms, n = L->n_rot;
  if (or_validate(L, g->nc)) return 1;
  std::vector<uint8_t> mask((size_t)n * N);
  std::vector<int32_t> axis(2 * (size_t)n + 2);
  or_fragments(L, mask.data(), axis.data());
  int nt = 360 / P->step_deg;
  int dlen = 1 + P->passes * n;
  int plen = 7 + n;
  std::vector<double> cand(plen);
  for (int r = r_begin; r < r_end; ++r) {
    int j = r - r_begin;
    double qr[4], tr[3];
    or_restart_init(g, P, lig, r, qr, tr);
    std::vector<int> count(n, 0);
    auto fill = [&](const double* q) {
      cand[0] = tr[0]; cand[1] = tr[1]; cand[2] = tr[2];
      for (int a = 0; a < 4; ++a) cand[3 + a] = q[a];
      for (int b = 0; b < n; ++b) cand[7 + b] = or_torsion_angle(count[b], P->step_deg);
    };
    // rigid stage: q = q_r * g_k
    double best = -INFINITY, second = -INFINITY, bestD = 0.0, bestG = 0.0, q[4];
    int kbest = 0;
    for (int k = 0; k < P->n_rigid; ++k) {
      double gk[4], qk[4], D, Gs;
      or_octahedral(k, gk);
      or_quat_mul(qr, gk, qk);
      fill(qk);
      double s = or_score_pose(L, g, mask.data(), axis.data(), cand.data(), P->penalty, &D, nullptr, &Gs);
      if (s > best) {
        second = best;
        best = s; bestD = D; bestG = Gs; kbest = k;
      } else if (s > second) {
        second = s;
      }
    }
    {
      double gk[4];
      or_octahedral(kbest, gk);
      or_quat_mul(qr, gk, q);
    }
    trace[(size_t)j * dlen] = (int16_t)kbest;
    gap[(size_t)j * dlen] = best - second;
    dn[(size_t)j * dlen] = bestD;
    gs[(size_t)j * dlen] = bestG;
    double cur = best;
    // torsion sweep
    for (int p = 0; p < P->passes; ++p) {
      for (int b = 0; b < n; ++b) {
        int base = count[b];
        double bs = -INFINITY, sc = -INFINITY, bD = 0.0, bG = 0.0;
        int jb = 0;
        for (int t = 0; t < nt; ++t) {
          count[b] = base + t;
          fill(q);
          double D, Gs;
          double s = or_score_pose(L, g, mask.data(), axis.data(), cand.data(), P->penalty, &D, nullptr, &Gs);
          if (s > bs) {
            sc = bs;
            bs = s; bD = D; bG = Gs; jb = t;
          } else if (s > sc) {
            sc = s;
          }
        }
        count[b] = (base + jb) % nt;
        size_t d = (size_t)j * dlen + 1 + (size_t)p * n + b;
        trace[d] = (int16_t)jb;
        gap[d] = bs - sc;
        dn[d] = bD;
        gs[d] = bG;
        cur = bs;
      }
    }
    // final pose, canonical quaternion (w >= 0)
    double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double sg = (q[0] < 0) ? -1.0 : 1.0;
    double qc[4] = {sg * q[0] / qn, sg * q[1] / qn, sg * q[2] / qn, sg * q[3] / qn};
    fill(qc);
    score[j] = cur;
    for (int a = 0; a < plen; ++a) pose[(size_t)j * plen + a] = cand[a];
  }
  return 0;
}

// Exhaustive search of one ligand (tiny ligands only): for every restart in
// [r_begin, r_end) and every combination (k, j_1..j_n), score the pose
// (t_r, q_r * g_k, theta = j * step) and keep the maximum (lowest combination
// in lexicographic order on ties). Outputs as or_dock_ligand's score/pose.
int32_t or_dock_exhaustive(const or_ligand* L, const or_grid* g, const or_params* P, int64_t lig,
                           int32_t r_begin, int32_t r_end, double* score, double* pose) {
  int N = L->n_atoms, n = L->n_rot;
  if (or_validate(L, g->nc)) return 1;
  std::vector<uint8_t> mask((size_t)n * N);
  std::vector<int32_t> axis(2 * (size_t)n + 2);
  or_fragments(L, mask.data(), axis.data());
  int nt = 360 / P->step_deg;
  int plen = 7 + n;
  std::vector<double> cand(plen), bestp(plen);
  for (int r = r_begin; r < r_end; ++r) {
    double qr[4], tr[3];
    or_restart_init(g, P, lig, r, qr, tr);
    double best = -INFINITY;
    for (int k = 0; k < P->n_rigid; ++k) {
      double gk[4], q[4];
      or_octahedral(k, gk);
      or_quat_mul(qr, gk, q);
      std::vector<int> j(n, 0);
      while (true) {
        cand[0] = tr[0]; cand[1] = tr[1]; cand[2] = tr[2];
        for (int a = 0; a < 4; ++a) cand[3 + a] = q[a];
        for (int b = 0; b < n; ++b) cand[7 + b] = or_torsion_angle(j[b], P->step_deg);
        double s = or_score_pose(L, g, mask.data(), axis.data(), cand.data(), P->penalty, nullptr, nullptr,
                                 nullptr);
        if (s > best) {
          best = s;
          bestp = cand;
        }
        int b = n - 1;
        while (b >= 0 && ++j[b] == nt) j[b--] = 0;
        if (b < 0) break;
      }
    }
    double qn = std::sqrt(bestp[3] * bestp[3] + bestp[4] * bestp[4] + bestp[5] * bestp[5] + bestp[6] * bestp[6]);
    double sg = (bestp[3] < 0) ? -1.0 : 1.0;
    for (int a = 3; a < 7; ++a) bestp[a] = sg * bestp[a] / qn;
    score[r - r_begin] = best;
    for (int a = 0; a < plen; ++a) pose[(size_t)(r - r_begin) * plen + a] = bestp[a];
  }
  return 0;
}

// Top K of R restart scores: descending score, lower restart index first on
// ties. Writes the K restart indices.
void or_top_k(int32_t R, const double* scores, int32_t K, int32_t* out) {
  std::vector<int32_t> idx(R);
  for (int i = 0; i < R; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return scores[a] > scores[b]; });
  for (int i = 0; i < K && i < R; ++i) out[i] = idx[i];
}

}  // extern "C"
