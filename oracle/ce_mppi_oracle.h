/*
 * ce_mppi_oracle.h -- plain FP64 CPU oracle of one CE-MPPI replanning iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA path; it is
 * not part of the product.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table
 * or constant with the CUDA library: everything here is written from the
 * paper's definitions (Liu, Chang, Chen, "Clustering-Embedded Model Predictive
 * Path Integral Control", Sec. II and Sec. III) and, for the random numbers,
 * from the published Philox4x32-10 definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11).
 *
 * Every stage is a separate function with explicit inputs, so a test can feed a
 * stage the GPU's own outputs of the previous stage (stage hand-off parity).
 *
 * Layouts (all row-major, C order):
 *   x0        [n]            state (n = 4 double integrator, 3 unicycle, 6 arm)
 *   U         [T][m]         nominal control sequence
 *   hist      [H][n_obs][p]  obstacle position observations, oldest first
 *   radius    [n_obs]        obstacle radii
 *   tracks    [T+1][n_obs][p] predicted obstacle centres over the horizon
 *   eps_eff   [K][T][m]      effective (post-clip) perturbations
 *   pN        [K][p]         terminal task-space positions p(x_T)
 *   z, g      [nV][p]        clustering feature / unit displacement (V order)
 */
#ifndef CE_MPPI_ORACLE_H
#define CE_MPPI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_DI = 0, ORC_UNICYCLE = 1, ORC_ARM = 2, ORC_ARM12 = 3 };
enum { ORC_MODE_NOCOL = 0, ORC_MODE_ALLCOL = 1, ORC_MODE_ALLNOISE = 2,
       ORC_MODE_STATIC = 3, ORC_MODE_DYNAMIC = 4, ORC_MODE_MPPI = 5 };

typedef struct {
  int dyn;             /* ORC_DI / ORC_UNICYCLE / ORC_ARM / ORC_ARM12         */
  int K, T;            /* rollouts, horizon N                                 */
  double dt;           /* model time step                                     */
  double obs_dt;       /* spacing of obstacle observations (Delta t, Eq. 17)  */
  double lambda;       /* temperature                                         */
  double dbscan_eps;   /* DBSCAN radius on the feature z                      */
  int min_pts;         /* DBSCAN minPts, the point itself included            */
  double sigma[6], u_min[6], u_max[6];
  double goal[16];     /* 2-D: goal state; arm: p_g[3] then R_g[9] row-major  */
  double w[8];         /* cost weights, meaning per dynamics (see .cpp)       */
  int hist_len;        /* H observations supplied                             */
  double robot_radius; /* 2-D robot radius / arm link-sphere radius           */
  double norm_eps;     /* epsilon of the unit-vector normalisations           */
  double v_static_thresh; /* |v_o*| at or below this counts as static          */
  uint64_t seed;       /* Philox key                                          */
  uint64_t counter;    /* replan counter (upper Philox counter words)         */
  int ref_mode;        /* 0: colliding rollouts whose first hit is o*; 1: all */
  int check_j0;        /* 1: also test x_0 for collision                      */
  int mppi_only;       /* 1: standard MPPI (Eq. 6-7 over all K), no clustering */
} orc_params;

typedef struct {
  int mode;            /* ORC_MODE_*                                          */
  int n_col, n_valid, n_clusters, sel_label, o_star, dynamic;
  double pbar[3], v_obs[3], S_min;
} orc_diag;

int orc_dims(int dyn, int* n, int* m, int* p);

/* Philox4x32-10 block function: out = bijection(ctr) under key.             */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* The first n standard normal deviates of rollout k (Box-Muller on Philox).  */
void orc_normals(uint64_t seed, uint64_t counter, int k, int n, double* out);

/* Obstacle velocity estimate, Eq. (17): v[n_obs][p].                         */
void orc_obstacle_velocity(const orc_params* P, const double* hist, int n_obs, double* v);
/* Constant-velocity prediction over the horizon: tracks[T+1][n_obs][p].      */
void orc_tracks(const orc_params* P, const double* hist, int n_obs, double* tracks);

/* Model pieces (Eq. 4, Sec. III-A2, Sec. III-C1).                            */
void orc_step(const orc_params* P, const double* x, const double* u, double* xn);
void orc_task_pos(const orc_params* P, const double* x, double* pos);
/* Standard DH forward kinematics: frame origins O[7][3], EE rotation R[9].   */
void orc_arm_fk(const double* q, double* O, double* R);
/* Robot collision points at state x: centres [npts][3], returns npts.        */
int orc_robot_points(const orc_params* P, const double* x, double* centres);

/* Rollouts + cost + collision (Algorithm 1, [Rollouts]; Eq. 3-5).
 * Outputs (any may be NULL): S[K], col[K], hit[K] (first-hit obstacle or -1),
 * hit_j[K], pN[K][p], eps_eff[K][T][m], min_abs_clear[K], traj[K][T+1][n].  */
void orc_rollouts(const orc_params* P, const double* x0, const double* U,
                  const double* tracks, const double* radius, int n_obs,
                  double* S, int* col, int* hit, int* hit_j, double* pN,
                  double* eps_eff, double* min_abs_clear, double* traj);

/* Pruning (Sec. II-B1): V and C_col in ascending k.                          */
void orc_prune(const int* col, int K, int* idxV, int* nV, int* idxC, int* nC);

/* Reference point (Sec. II-B2, Eq. 11): returns o_star, writes pbar[p].      */
int orc_reference_point(const orc_params* P, const double* x0, const double* tracks,
                        const double* radius, int n_obs, const int* idxC, int nC,
                        const int* hit, const double* pN, double* pbar);
/* Features z (Eq. 12-13) and g (Eq. 15) for k in V.                          */
void orc_features(const orc_params* P, const double* x0, const double* pbar,
                  const int* idxV, int nV, const double* pN, double* z, double* g);

/* DBSCAN on FP32 features with the FP32 neighbour predicate; labels[n] are
 * -1 (noise) or 0..M-1 ordered by the smallest core member.  Returns M.     */
int orc_dbscan(const float* z, int n, int p, float eps2, int min_pts, int* labels);

/* Cluster statistics and selection (Sec. II-B3, Eq. 14, 16, 18).
 * cnt/Sbar/vhat are [M], [M], [M][p]; returns c* (or -1 when M == 0).       */
int orc_select(const orc_params* P, const int* labels, int nV, const int* idxV,
               const double* S, const double* g, int M, const double* v_obs,
               int* dynamic, int* cnt, double* Sbar, double* vhat);

/* Softmin weights over a member list (Eq. 6 / Eq. 19) and the update
 * (Eq. 7 / Eq. 20): U_new = U + sum_k w_k eps_eff_k.  w[K] is written for
 * every k (zero outside the list).  Returns S_min of the list.               */
double orc_update(const orc_params* P, const double* U, const double* S,
                  const double* eps_eff, const int* members, int n_members,
                  double* w, double* U_new);

/* Receding-horizon shift and warm start (Algorithm 1, [Execute]).           */
void orc_shift(const orc_params* P, const double* U_new, double* U_next);

/* One full CE-MPPI iteration (Algorithm 1).  U_new[T][m] is the updated
 * nominal before the shift.  Optional per-rollout outputs as orc_rollouts;
 * labels_V[K] (V order, first nV used), w[K].                                */
void orc_replan(const orc_params* P, const double* x0, const double* U,
                const double* hist, const double* radius, int n_obs,
                double* U_new, orc_diag* diag,
                double* S, int* col, int* hit, double* pN, double* eps_eff,
                double* min_abs_clear, int* labels_V, double* w);

/* Threaded throughput helper: runs n independent replans on n_threads host
 * threads (the CPU baseline).  Entry i of each pointer array holds instance
 * i's input or output with the shapes above.  Returns wall seconds.          */
double orc_replan_many(const orc_params* Ps, const double* const* x0s,
                       const double* const* Us, const double* const* hists,
                       const double* const* radii, const int* n_obs, int n,
                       int n_threads, double* const* U_news);

#ifdef __cplusplus
}
#endif
#endif
