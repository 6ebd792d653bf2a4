// ce_mppi_oracle.cpp -- plain FP64 CPU oracle of one CE-MPPI replanning iteration.
//
// TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
// baseline leg of the benchmark to check the CUDA path.  It shares no code with
// the CUDA library.  Each function restates one definition of the paper
// (Liu, Chang, Chen, "Clustering-Embedded Model Predictive Path Integral
// Control"), cited by section and equation number in the order the equations
// are displayed:
//   Eq. 3  u^(k) = u + eps^(k)            Eq. 12 d = p(x_N) - pbar
//   Eq. 4  rollout x_{j+1} = f(x_j,u_j)    Eq. 13 z = d / (|d| + eps)
//   Eq. 5  S = phi(x_N) + sum_j l(x_j,u_j) Eq. 14 static selection argmin Sbar
//   Eq. 6  MPPI weights                    Eq. 15 g = unit terminal displacement
//   Eq. 7  MPPI update                     Eq. 16 cluster mean direction vhat_c
//   Eq. 8  trajectory tau                  Eq. 17 obstacle velocity estimate
//   Eq. 9  feasible set V                  Eq. 18 dynamic selection argmin dot
//   Eq. 10 colliding set C_col             Eq. 19 within-cluster weights
//   Eq. 11 reference point pbar            Eq. 20 within-cluster update
//   Eq. 21 unicycle model, Eq. 22-23 quadratic stage/terminal cost (Sec. III-A),
//   Eq. 24 arm stage cost (Sec. III-C).
// Everything is double precision except the DBSCAN neighbour predicate, which
// the library defines in FP32 (round-to-nearest, no fused multiply-add); this
// file must be compiled with -ffp-contract=off so that the compiler keeps it so.
//
// Parity pins for every function live in tests/test_oracle_pins.py.

#include "ce_mppi_oracle.h"

#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 multiplies
// with the multipliers 0xD2511F53 / 0xCD9E8D57; the key is bumped by the Weyl
// constants 0x9E3779B9 / 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0];
  const uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void philox10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k);
    if (r < 9) {
      k[0] += 0x9E3779B9u;
      k[1] += 0xBB67AE85u;
    }
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Uniform in (0,1) from the top 23 bits of a word: ((w >> 9) + 1/2) / 2^23
// (exactly representable in FP32 as well, so both precisions see one value).
double unit23(uint32_t w) { return ((double)(w >> 9) + 0.5) / 8388608.0; }

bool is_arm(int dyn) { return dyn == ORC_ARM || dyn == ORC_ARM12; }
int dim_n(int dyn) {
  return dyn == ORC_DI ? 4 : dyn == ORC_UNICYCLE ? 3 : dyn == ORC_ARM ? 6 : 12;
}
int dim_m(int dyn) { return is_arm(dyn) ? 6 : 2; }
int dim_p(int dyn) { return is_arm(dyn) ? 3 : 2; }

double clip(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

// UR5e-like standard DH table: d and a from the workload description, alpha
// from the published UR convention.
const double kD[6] = {0.1625, 0.0, 0.0, 0.1333, 0.0997, 0.0996};
const double kA[6] = {0.0, -0.425, -0.3922, 0.0, 0.0, 0.0};
const double kAlpha[6] = {kPi / 2, 0.0, 0.0, kPi / 2, -kPi / 2, 0.0};

// Collision of the robot at state x against all obstacles at one horizon time.
// Returns the lowest colliding obstacle index or -1; tracks min |clearance|.
int collide_at(const orc_params* P, const double* x, const double* obs_j,
               const double* radius, int n_obs, double* min_abs) {
  const int p = dim_p(P->dyn);
  double centres[24 * 3];
  const int npts = orc_robot_points(P, x, centres);
  int first = -1;
  for (int o = 0; o < n_obs; ++o) {
    for (int s = 0; s < npts; ++s) {
      double d2 = 0.0;
      for (int i = 0; i < p; ++i) {
        const double di = centres[s * 3 + i] - obs_j[o * p + i];
        d2 += di * di;
      }
      const double clear = std::sqrt(d2) - (radius[o] + P->robot_radius);
      if (min_abs && std::fabs(clear) < *min_abs) *min_abs = std::fabs(clear);
      if (clear < 0.0 && first < 0) first = o;
    }
  }
  return first;
}

// Geodesic angle between two rotations, acos((tr(Rg^T R) - 1) / 2).
double rot_angle(const double* R, const double* Rg) {
  double tr = 0.0;
  for (int i = 0; i < 9; ++i) tr += Rg[i] * R[i];
  return std::acos(clip((tr - 1.0) / 2.0, -1.0, 1.0));
}

// Stage cost l(x_j, u_j) (Eq. 5 with Eq. 22 / Eq. 24 / the double-integrator
// cost); obs_j is the obstacle set at horizon time j (arm collision term).
double stage_cost(const orc_params* P, const double* x, const double* u,
                  const double* obs_j, const double* radius, int n_obs) {
  const double* w = P->w;
  const double* g = P->goal;
  if (P->dyn == ORC_DI) {
    const double ex = x[0] - g[0], ey = x[1] - g[1];
    return w[0] * (ex * ex + ey * ey) + w[1] * (u[0] * u[0] + u[1] * u[1]);
  }
  if (P->dyn == ORC_UNICYCLE) {
    double c = 0.0;
    for (int i = 0; i < 3; ++i) c += w[i] * (x[i] - g[i]) * (x[i] - g[i]);
    return c;
  }
  double O[21], R[9];
  orc_arm_fk(x, O, R);
  double e2 = 0.0;
  for (int i = 0; i < 3; ++i) e2 += (O[18 + i] - g[i]) * (O[18 + i] - g[i]);
  const int icol = collide_at(P, x, obs_j, radius, n_obs, nullptr) >= 0 ? 1 : 0;
  return w[0] * std::sqrt(e2) + w[1] * rot_angle(R, g + 3) + w[2] * icol;
}

// Terminal cost phi(x_N) (Eq. 5 with Eq. 23 / the arm stage cost at x_N).
double terminal_cost(const orc_params* P, const double* x, const double* obs_N,
                     const double* radius, int n_obs) {
  const double* w = P->w;
  const double* g = P->goal;
  if (P->dyn == ORC_DI) {
    const double ex = x[0] - g[0], ey = x[1] - g[1];
    return w[2] * (ex * ex + ey * ey);
  }
  if (P->dyn == ORC_UNICYCLE) {
    double c = 0.0;
    for (int i = 0; i < 3; ++i) c += w[3 + i] * (x[i] - g[i]) * (x[i] - g[i]);
    return c;
  }
  const double zero_u[6] = {0, 0, 0, 0, 0, 0};
  return stage_cost(P, x, zero_u, obs_N, radius, n_obs);
}

}  // namespace

extern "C" {

int orc_dims(int dyn, int* n, int* m, int* p) {
  if (dyn < 0 || dyn > 2) return -1;
  *n = dim_n(dyn);
  *m = dim_m(dyn);
  *p = dim_p(dyn);
  return 0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  philox10(ctr, key, out);
}

// Gaussian perturbations (Sec. II-A, eps ~ N(0, Sigma)): normal number i of
// rollout k comes from Philox block i/4 with counter (k, i/4, counter_lo,
// counter_hi) and key (seed_lo, seed_hi); Box-Muller maps the word pairs
// (w0,w1) and (w2,w3) to normals (r cos, r sin) with r = sqrt(-2 ln u1).
void orc_normals(uint64_t seed, uint64_t counter, int k, int n, double* out) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int b = 0; 4 * b < n; ++b) {
    const uint32_t ctr[4] = {(uint32_t)k, (uint32_t)b, (uint32_t)counter,
                             (uint32_t)(counter >> 32)};
    uint32_t wv[4];
    philox10(ctr, key, wv);
    double z[4];
    for (int pair = 0; pair < 2; ++pair) {
      const double u1 = unit23(wv[2 * pair]);
      const double u2 = unit23(wv[2 * pair + 1]);
      const double r = std::sqrt(-2.0 * std::log(u1));
      z[2 * pair] = r * std::cos(2.0 * kPi * u2);
      z[2 * pair + 1] = r * std::sin(2.0 * kPi * u2);
    }
    for (int s = 0; s < 4 && 4 * b + s < n; ++s) out[4 * b + s] = z[s];
  }
}

// Eq. 17: v_obs = 1/(H-1) sum_{h=0}^{H-2} (o_{t-h} - o_{t-h-1}) / Delta t,
// with o_{t-h} = hist[H-1-h].  Fewer than two observations give v = 0.
void orc_obstacle_velocity(const orc_params* P, const double* hist, int n_obs, double* v) {
  const int p = dim_p(P->dyn);
  const int H = P->hist_len;
  for (int o = 0; o < n_obs; ++o) {
    for (int i = 0; i < p; ++i) {
      double acc = 0.0;
      for (int h = 0; h <= H - 2; ++h) {
        const double o_th = hist[((H - 1 - h) * n_obs + o) * p + i];
        const double o_th1 = hist[((H - 2 - h) * n_obs + o) * p + i];
        acc += (o_th - o_th1) / P->obs_dt;
      }
      v[o * p + i] = H >= 2 ? acc / (double)(H - 1) : 0.0;
    }
  }
}

// Obstacle positions over the horizon: the newest observation carried forward
// at the estimated velocity, o_j = o_t + v_obs * (j dt), j = 0..T.
void orc_tracks(const orc_params* P, const double* hist, int n_obs, double* tracks) {
  const int p = dim_p(P->dyn);
  std::vector<double> v((size_t)n_obs * p);
  orc_obstacle_velocity(P, hist, n_obs, v.data());
  const double* newest = hist + (size_t)(P->hist_len - 1) * n_obs * p;
  for (int j = 0; j <= P->T; ++j)
    for (int o = 0; o < n_obs; ++o)
      for (int i = 0; i < p; ++i)
        tracks[((size_t)j * n_obs + o) * p + i] =
            newest[o * p + i] + v[o * p + i] * (j * P->dt);
}

// x_{t+1} = f(x_t, u_t).  Double integrator: explicit Euler on (p, v) with
// acceleration input.  Unicycle: Eq. 21 (heading advanced after the position,
// from the old heading).  Arm: joint-velocity integrator q' = q + u dt.
// 12-D arm (joint positions and velocities, the UR5e state of Sec. III-C):
// explicit Euler with joint-acceleration input, q' = q + qdot dt,
// qdot' = qdot + u dt.
void orc_step(const orc_params* P, const double* x, const double* u, double* xn) {
  const double dt = P->dt;
  if (P->dyn == ORC_DI) {
    xn[0] = x[0] + x[2] * dt;
    xn[1] = x[1] + x[3] * dt;
    xn[2] = x[2] + u[0] * dt;
    xn[3] = x[3] + u[1] * dt;
  } else if (P->dyn == ORC_UNICYCLE) {
    xn[0] = x[0] + u[0] * std::cos(x[2]) * dt;
    xn[1] = x[1] + u[0] * std::sin(x[2]) * dt;
    xn[2] = x[2] + u[1] * dt;
  } else if (P->dyn == ORC_ARM) {
    for (int i = 0; i < 6; ++i) xn[i] = x[i] + u[i] * dt;
  } else {
    for (int i = 0; i < 6; ++i) {
      xn[i] = x[i] + x[6 + i] * dt;
      xn[6 + i] = x[6 + i] + u[i] * dt;
    }
  }
}

// Task-space position p(x): planar position, or the arm's end-effector.
void orc_task_pos(const orc_params* P, const double* x, double* pos) {
  if (is_arm(P->dyn)) {
    double O[21], R[9];
    orc_arm_fk(x, O, R);
    for (int i = 0; i < 3; ++i) pos[i] = O[18 + i];
  } else {
    pos[0] = x[0];
    pos[1] = x[1];
  }
}

// Standard Denavit-Hartenberg chain: T_i = T_{i-1} Rz(q_i) Tz(d_i) Tx(a_i) Rx(alpha_i).
void orc_arm_fk(const double* q, double* O, double* R) {
  double T[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
  O[0] = O[1] = O[2] = 0.0;
  for (int i = 0; i < 6; ++i) {
    const double ct = std::cos(q[i]), st = std::sin(q[i]);
    const double ca = std::cos(kAlpha[i]), sa = std::sin(kAlpha[i]);
    const double A[16] = {ct, -st * ca, st * sa,  kA[i] * ct,
                          st, ct * ca,  -ct * sa, kA[i] * st,
                          0,  sa,       ca,       kD[i],
                          0,  0,        0,        1};
    double N[16];
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        double s = 0.0;
        for (int e = 0; e < 4; ++e) s += T[r * 4 + e] * A[e * 4 + c];
        N[r * 4 + c] = s;
      }
    std::memcpy(T, N, sizeof(T));
    for (int r = 0; r < 3; ++r) O[(i + 1) * 3 + r] = T[r * 4 + 3];
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) R[r * 3 + c] = T[r * 4 + c];
}

// Collision geometry: the planar robot is one disc; the arm carries four
// spheres per link at fractions 0, 1/3, 2/3, 1 of the segment O_{i-1} -> O_i.
int orc_robot_points(const orc_params* P, const double* x, double* centres) {
  if (!is_arm(P->dyn)) {
    centres[0] = x[0];
    centres[1] = x[1];
    centres[2] = 0.0;
    return 1;
  }
  double O[21], R[9];
  orc_arm_fk(x, O, R);
  int s = 0;
  for (int link = 1; link <= 6; ++link)
    for (int f = 0; f < 4; ++f, ++s)
      for (int i = 0; i < 3; ++i)
        centres[s * 3 + i] =
            O[(link - 1) * 3 + i] + (f / 3.0) * (O[link * 3 + i] - O[(link - 1) * 3 + i]);
  return s;
}

// Algorithm 1 [Rollouts]: perturb (Eq. 3, clipped to the input box), simulate
// (Eq. 4), accumulate the cost (Eq. 5) and the collision indicator over tau
// (Eq. 8, times 1..T unless check_j0).
void orc_rollouts(const orc_params* P, const double* x0, const double* U,
                  const double* tracks, const double* radius, int n_obs,
                  double* S, int* col, int* hit, int* hit_j, double* pN,
                  double* eps_eff, double* min_abs_clear, double* traj) {
  const int n = dim_n(P->dyn), m = dim_m(P->dyn), p = dim_p(P->dyn);
  const int K = P->K, T = P->T;
  std::vector<double> nz((size_t)T * m);
  for (int k = 0; k < K; ++k) {
    orc_normals(P->seed, P->counter, k, T * m, nz.data());
    double x[12], xn[12], u[6];
    for (int i = 0; i < n; ++i) x[i] = x0[i];
    if (traj)
      for (int i = 0; i < n; ++i) traj[((size_t)k * (T + 1)) * n + i] = x[i];
    double min_abs = std::numeric_limits<double>::infinity();
    int first_o = -1, first_j = -1;
    if (P->check_j0) {
      const int o = collide_at(P, x, tracks, radius, n_obs, &min_abs);
      if (o >= 0) { first_o = o; first_j = 0; }
    }
    double cost = 0.0;
    for (int j = 0; j < T; ++j) {
      for (int d = 0; d < m; ++d) {
        const double nominal = U[j * m + d];
        u[d] = clip(nominal + P->sigma[d] * nz[(size_t)j * m + d], P->u_min[d], P->u_max[d]);
        if (eps_eff) eps_eff[((size_t)k * T + j) * m + d] = u[d] - nominal;
      }
      cost += stage_cost(P, x, u, tracks + (size_t)j * n_obs * p, radius, n_obs);
      orc_step(P, x, u, xn);
      for (int i = 0; i < n; ++i) x[i] = xn[i];
      if (traj)
        for (int i = 0; i < n; ++i) traj[((size_t)k * (T + 1) + j + 1) * n + i] = x[i];
      const int o = collide_at(P, x, tracks + (size_t)(j + 1) * n_obs * p, radius, n_obs,
                               &min_abs);
      if (o >= 0 && first_o < 0) { first_o = o; first_j = j + 1; }
    }
    cost += terminal_cost(P, x, tracks + (size_t)T * n_obs * p, radius, n_obs);
    // 2-D robots: w[7] I_col(tau) (Eq. 8), a collision penalty for standard
    // MPPI (zero by default: CE-MPPI prunes colliding rollouts instead)
    if (!is_arm(P->dyn) && first_o >= 0) cost += P->w[7];
    if (S) S[k] = cost;
    if (col) col[k] = first_o >= 0 ? 1 : 0;
    if (hit) hit[k] = first_o;
    if (hit_j) hit_j[k] = first_j;
    if (min_abs_clear) min_abs_clear[k] = min_abs;
    if (pN) {
      double pos[3];
      orc_task_pos(P, x, pos);
      for (int i = 0; i < p; ++i) pN[(size_t)k * p + i] = pos[i];
    }
  }
}

// Eq. 9 and Eq. 10: V = {k | I_col = 0}, C_col = {k | I_col = 1}.
void orc_prune(const int* col, int K, int* idxV, int* nV, int* idxC, int* nC) {
  int a = 0, b = 0;
  for (int k = 0; k < K; ++k) {
    if (col[k]) idxC[b++] = k;
    else idxV[a++] = k;
  }
  *nV = a;
  *nC = b;
}

// Eq. 11, restricted (as the method overview states) to the colliding rollouts
// near the closest obstacle: o* is the obstacle, among those some rollout hits
// first, with the least clearance |p(x_0) - o_t| - r_o (ties: lowest index);
// pbar is the mean p(x_N) of the colliding rollouts whose first hit is o*.
// ref_mode 1 takes the literal mean over all of C_col.
int orc_reference_point(const orc_params* P, const double* x0, const double* tracks,
                        const double* radius, int n_obs, const int* idxC, int nC,
                        const int* hit, const double* pN, double* pbar) {
  const int p = dim_p(P->dyn);
  double pos0[3];
  orc_task_pos(P, x0, pos0);
  std::vector<char> was_hit(n_obs, 0);
  for (int i = 0; i < nC; ++i)
    if (hit[idxC[i]] >= 0) was_hit[hit[idxC[i]]] = 1;
  int o_star = -1;
  double best = std::numeric_limits<double>::infinity();
  for (int o = 0; o < n_obs; ++o) {
    if (!was_hit[o]) continue;
    double d2 = 0.0;
    for (int i = 0; i < p; ++i) {
      const double di = pos0[i] - tracks[o * p + i];
      d2 += di * di;
    }
    const double clear = std::sqrt(d2) - radius[o];
    if (clear < best) { best = clear; o_star = o; }
  }
  double acc[3] = {0, 0, 0};
  int cnt = 0;
  for (int i = 0; i < nC; ++i) {
    const int k = idxC[i];
    if (P->ref_mode == 0 && hit[k] != o_star) continue;
    for (int c = 0; c < p; ++c) acc[c] += pN[(size_t)k * p + c];
    ++cnt;
  }
  for (int c = 0; c < p; ++c) pbar[c] = cnt > 0 ? acc[c] / cnt : 0.0;
  return o_star;
}

// Eq. 12-13: z = d / (|d| + eps), d = p(x_N) - pbar; Eq. 15:
// g = (p(x_N) - p(x_0)) / (|p(x_N) - p(x_0)| + eps).
void orc_features(const orc_params* P, const double* x0, const double* pbar,
                  const int* idxV, int nV, const double* pN, double* z, double* g) {
  const int p = dim_p(P->dyn);
  double pos0[3];
  orc_task_pos(P, x0, pos0);
  for (int i = 0; i < nV; ++i) {
    const double* pk = pN + (size_t)idxV[i] * p;
    double d[3], e[3], nd = 0.0, ne = 0.0;
    for (int c = 0; c < p; ++c) {
      d[c] = pk[c] - pbar[c];
      e[c] = pk[c] - pos0[c];
      nd += d[c] * d[c];
      ne += e[c] * e[c];
    }
    nd = std::sqrt(nd);
    ne = std::sqrt(ne);
    for (int c = 0; c < p; ++c) {
      if (z) z[(size_t)i * p + c] = d[c] / (nd + P->norm_eps);
      if (g) g[(size_t)i * p + c] = e[c] / (ne + P->norm_eps);
    }
  }
}

// DBSCAN (Sec. II-B2) with the library's conventions: a and b are neighbours
// when the FP32 sum of squared coordinate differences, accumulated in
// coordinate order without fused multiply-add, is <= eps2; a point is core when
// it has at least min_pts neighbours (itself included); clusters are the
// connected components of the core points; a non-core point joins the cluster
// of its lowest-index core neighbour, or is noise (-1).  Components are found
// by breadth-first expansion from the lowest unlabelled core point, so cluster
// ids follow the smallest core member.
int orc_dbscan(const float* z, int n, int p, float eps2, int min_pts, int* labels) {
  auto nb = [&](int a, int b) -> bool {
    float s = 0.0f;
    for (int c = 0; c < p; ++c) {
      const float dc = z[(size_t)a * p + c] - z[(size_t)b * p + c];
      const float sq = dc * dc;
      s = s + sq;
    }
    return s <= eps2;
  };
  std::vector<char> core(n, 0);
  for (int a = 0; a < n; ++a) {
    int count = 0;
    for (int b = 0; b < n; ++b) count += nb(a, b) ? 1 : 0;
    core[a] = count >= min_pts;
  }
  for (int a = 0; a < n; ++a) labels[a] = -1;
  int M = 0;
  std::vector<int> queue;
  for (int a = 0; a < n; ++a) {
    if (!core[a] || labels[a] >= 0) continue;
    const int c = M++;
    labels[a] = c;
    queue.assign(1, a);
    for (size_t qi = 0; qi < queue.size(); ++qi) {
      const int u = queue[qi];
      for (int b = 0; b < n; ++b)
        if (core[b] && labels[b] < 0 && nb(u, b)) {
          labels[b] = c;
          queue.push_back(b);
        }
    }
  }
  for (int a = 0; a < n; ++a) {
    if (core[a]) continue;
    for (int b = 0; b < n; ++b)
      if (core[b] && nb(a, b)) {
        labels[a] = labels[b];
        break;
      }
  }
  return M;
}

// Algorithm 1 [Cluster stats] and [Selection]: Sbar_c (mean cost), v_c the mean
// of g over the cluster and vhat_c = v_c / (|v_c| + eps) (Eq. 16); the obstacle
// is dynamic when |v_obs| > v_static_thresh, with vhat_obs = v_obs/(|v_obs|+eps)
// (Eq. 17).  Static: argmin Sbar_c (Eq. 14).  Dynamic: argmin vhat_c . vhat_obs
// (Eq. 18).  Ties go to the lowest cluster id.
int orc_select(const orc_params* P, const int* labels, int nV, const int* idxV,
               const double* S, const double* g, int M, const double* v_obs,
               int* dynamic, int* cnt, double* Sbar, double* vhat) {
  const int p = dim_p(P->dyn);
  if (M <= 0) return -1;
  std::vector<double> vsum((size_t)M * p, 0.0);
  for (int c = 0; c < M; ++c) { cnt[c] = 0; Sbar[c] = 0.0; }
  for (int i = 0; i < nV; ++i) {
    const int c = labels[i];
    if (c < 0) continue;
    cnt[c] += 1;
    Sbar[c] += S[idxV[i]];
    for (int q = 0; q < p; ++q) vsum[(size_t)c * p + q] += g[(size_t)i * p + q];
  }
  for (int c = 0; c < M; ++c) {
    Sbar[c] /= cnt[c];
    double nrm = 0.0;
    for (int q = 0; q < p; ++q) {
      vsum[(size_t)c * p + q] /= cnt[c];
      nrm += vsum[(size_t)c * p + q] * vsum[(size_t)c * p + q];
    }
    nrm = std::sqrt(nrm);
    for (int q = 0; q < p; ++q) vhat[(size_t)c * p + q] = vsum[(size_t)c * p + q] / (nrm + P->norm_eps);
  }
  double vn = 0.0;
  for (int q = 0; q < p; ++q) vn += v_obs[q] * v_obs[q];
  vn = std::sqrt(vn);
  *dynamic = vn > P->v_static_thresh ? 1 : 0;
  int best = 0;
  if (!*dynamic) {
    for (int c = 1; c < M; ++c)
      if (Sbar[c] < Sbar[best]) best = c;
  } else {
    double bestdot = std::numeric_limits<double>::infinity();
    for (int c = 0; c < M; ++c) {
      double dot = 0.0;
      for (int q = 0; q < p; ++q) dot += vhat[(size_t)c * p + q] * (v_obs[q] / (vn + P->norm_eps));
      if (dot < bestdot) { bestdot = dot; best = c; }
    }
  }
  return best;
}

// Eq. 6 / Eq. 19 (weights normalised over the member list) and Eq. 7 / Eq. 20
// (u_j += sum_k w_k eps_kj).  exp(-S/lambda) is evaluated as
// exp(-(S - S_min)/lambda): the common factor exp(-S_min/lambda) cancels in the
// ratio, so the weights are the same numbers without underflow.
double orc_update(const orc_params* P, const double* U, const double* S,
                  const double* eps_eff, const int* members, int n_members,
                  double* w, double* U_new) {
  const int m = dim_m(P->dyn), T = P->T;
  double s_min = std::numeric_limits<double>::infinity();
  for (int i = 0; i < n_members; ++i) s_min = std::fmin(s_min, S[members[i]]);
  for (int k = 0; k < P->K; ++k) w[k] = 0.0;
  double Z = 0.0;
  for (int i = 0; i < n_members; ++i) Z += std::exp(-(S[members[i]] - s_min) / P->lambda);
  for (int i = 0; i < n_members; ++i)
    w[members[i]] = std::exp(-(S[members[i]] - s_min) / P->lambda) / Z;
  for (int j = 0; j < T; ++j)
    for (int d = 0; d < m; ++d) {
      double acc = 0.0;
      for (int i = 0; i < n_members; ++i) {
        const int k = members[i];
        acc += w[k] * eps_eff[((size_t)k * T + j) * m + d];
      }
      U_new[j * m + d] = U[j * m + d] + acc;
    }
  return s_min;
}

// Algorithm 1 [Execute]: drop u_t, shift, repeat the last control.
void orc_shift(const orc_params* P, const double* U_new, double* U_next) {
  const int m = dim_m(P->dyn), T = P->T;
  for (int j = 0; j < T; ++j) {
    const int src = j + 1 < T ? j + 1 : T - 1;
    for (int d = 0; d < m; ++d) U_next[j * m + d] = U_new[src * m + d];
  }
}

// Algorithm 1, one iteration.  Fallbacks: no colliding rollout -> standard
// MPPI over all K (as the paper states); every rollout colliding -> standard
// MPPI over all K; DBSCAN returning only noise -> standard MPPI over V.
void orc_replan(const orc_params* P, const double* x0, const double* U,
                const double* hist, const double* radius, int n_obs,
                double* U_new, orc_diag* diag,
                double* S_out, int* col_out, int* hit_out, double* pN_out,
                double* eps_out, double* min_abs_out, int* labels_out, double* w_out) {
  const int m = dim_m(P->dyn), p = dim_p(P->dyn);
  const int K = P->K, T = P->T;
  std::vector<double> tracks((size_t)(T + 1) * n_obs * p), vel((size_t)n_obs * p);
  orc_tracks(P, hist, n_obs, tracks.data());
  orc_obstacle_velocity(P, hist, n_obs, vel.data());
  std::vector<double> S(K), pN((size_t)K * p), eps((size_t)K * T * m), mac(K), w(K);
  std::vector<int> col(K), hit(K), idxV(K), idxC(K), labels(K, -1);
  orc_rollouts(P, x0, U, tracks.data(), radius, n_obs, S.data(), col.data(), hit.data(),
               nullptr, pN.data(), eps.data(), mac.data(), nullptr);
  int nV = 0, nC = 0;
  orc_prune(col.data(), K, idxV.data(), &nV, idxC.data(), &nC);
  orc_diag dg;
  std::memset(&dg, 0, sizeof(dg));
  dg.n_col = nC;
  dg.n_valid = nV;
  dg.o_star = -1;
  dg.sel_label = -1;
  std::vector<int> members;
  if (P->mppi_only || nC == 0 || nV == 0) {
    dg.mode = P->mppi_only ? ORC_MODE_MPPI : nC == 0 ? ORC_MODE_NOCOL : ORC_MODE_ALLCOL;
    for (int k = 0; k < K; ++k) members.push_back(k);
  } else {
    dg.o_star = orc_reference_point(P, x0, tracks.data(), radius, n_obs, idxC.data(), nC,
                                    hit.data(), pN.data(), dg.pbar);
    std::vector<double> z((size_t)nV * p), g((size_t)nV * p);
    orc_features(P, x0, dg.pbar, idxV.data(), nV, pN.data(), z.data(), g.data());
    std::vector<float> zf((size_t)nV * p);
    for (size_t i = 0; i < zf.size(); ++i) zf[i] = (float)z[i];
    const float eps_f = (float)P->dbscan_eps;  // eps^2 as the FP32 product of FP32 eps
    const float eps2 = eps_f * eps_f;
    const int M = orc_dbscan(zf.data(), nV, p, eps2, P->min_pts, labels.data());
    dg.n_clusters = M;
    if (M == 0) {
      dg.mode = ORC_MODE_ALLNOISE;
      members.assign(idxV.begin(), idxV.begin() + nV);
    } else {
      for (int q = 0; q < p; ++q) dg.v_obs[q] = vel[(size_t)dg.o_star * p + q];
      std::vector<int> cnt(M);
      std::vector<double> Sbar(M), vhat((size_t)M * p);
      const int cs = orc_select(P, labels.data(), nV, idxV.data(), S.data(), g.data(), M,
                                dg.v_obs, &dg.dynamic, cnt.data(), Sbar.data(), vhat.data());
      dg.sel_label = cs;
      dg.mode = dg.dynamic ? ORC_MODE_DYNAMIC : ORC_MODE_STATIC;
      for (int i = 0; i < nV; ++i)
        if (labels[i] == cs) members.push_back(idxV[i]);
    }
  }
  dg.S_min = orc_update(P, U, S.data(), eps.data(), members.data(), (int)members.size(),
                        w.data(), U_new);
  if (diag) *diag = dg;
  if (S_out) std::memcpy(S_out, S.data(), sizeof(double) * K);
  if (col_out) std::memcpy(col_out, col.data(), sizeof(int) * K);
  if (hit_out) std::memcpy(hit_out, hit.data(), sizeof(int) * K);
  if (pN_out) std::memcpy(pN_out, pN.data(), sizeof(double) * K * p);
  if (eps_out) std::memcpy(eps_out, eps.data(), sizeof(double) * K * T * m);
  if (min_abs_out) std::memcpy(min_abs_out, mac.data(), sizeof(double) * K);
  if (labels_out) std::memcpy(labels_out, labels.data(), sizeof(int) * K);
  if (w_out) std::memcpy(w_out, w.data(), sizeof(double) * K);
}

double orc_replan_many(const orc_params* Ps, const double* const* x0s,
                       const double* const* Us, const double* const* hists,
                       const double* const* radii, const int* n_obs, int n,
                       int n_threads, double* const* U_news) {
  const auto t0 = std::chrono::steady_clock::now();
  if (n_threads < 1) n_threads = 1;
  std::vector<std::thread> pool;
  for (int t = 0; t < n_threads; ++t)
    pool.emplace_back([=]() {
      for (int i = t; i < n; i += n_threads)
        orc_replan(&Ps[i], x0s[i], Us[i], hists[i], radii[i], n_obs[i], U_news[i], nullptr,
                   nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    });
  for (auto& th : pool) th.join();
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // extern "C"
