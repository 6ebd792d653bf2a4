/*
 * ce_mppi.h -- C ABI of the B300 (sm_103a) CE-MPPI replanning library.
 *
 * One call of ce_mppi_replan* runs one iteration of Clustering-Embedded MPPI
 * (Liu, Chang, Chen, "Clustering-Embedded Model Predictive Path Integral
 * Control", Algorithm 1) entirely on the GPU:
 *
 *   sample K perturbed control sequences around the nominal (Sec. II-A, Eq. 3)
 *   -> forward-simulate each over the horizon T with cost (Eq. 4-5) and
 *      collision flags against predicted obstacle tracks (Sec. II-B1, Eq. 8)
 *   -> prune colliding rollouts (Eq. 9-10); reference point from the colliding
 *      rollouts near the closest obstacle (Eq. 11)
 *   -> DBSCAN on the direction feature z (Eq. 12-13, Sec. II-B2)
 *   -> select a cluster: least mean cost when the obstacle is static (Eq. 14),
 *      most opposite to its motion when it moves (Eq. 15-18)
 *   -> softmin-weighted update over the selected cluster (Eq. 19-20); with no
 *      colliding rollout, the standard MPPI update over all K (Eq. 6-7)
 *   -> receding-horizon shift of the nominal (Algorithm 1, [Execute]).
 *
 * Conventions
 *   - All arithmetic is FP32.  All arrays are row-major (C order).
 *   - Dimensions by dynamics: double integrator n=4 (px,py,vx,vy), m=2
 *     (ax,ay), p=2; unicycle n=3 (x,y,theta), m=2 (v,omega), p=2 (Sec. III-A,
 *     Eq. 21); arm n=6 (joint angles), m=6 (joint velocities), p=3 (end
 *     effector position, Sec. III-C).
 *   - Every call returns a ce_status_t and never throws; on failure
 *     ce_mppi_last_error() returns a thread-local message.  Parameters are
 *     validated before anything is launched.
 *   - A handle owns all of its device memory (nominal sequence, replan counter,
 *     scratch); it is allocated in ce_mppi_create and freed in ce_mppi_destroy.
 *     Host pointers passed to a call are read or written only during the call.
 *     Device pointers passed to a *_dev call must stay valid until the work
 *     queued on the handle's stream has completed.
 *   - A handle is not thread-safe: one host thread drives it at a time.
 */
#ifndef CE_MPPI_H
#define CE_MPPI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CE_DYN_DOUBLE_INT_2D = 0, /* p += v dt; v += a dt                        */
  CE_DYN_UNICYCLE = 1,      /* Sec. III-A, Eq. 21                          */
  CE_DYN_ARM6_KIN = 2,      /* q += qdot dt, UR5e-like standard DH chain   */
  CE_DYN_ARM12_DI = 3       /* 12-D (q, qdot), joint accelerations: q += qdot dt, */
                            /* qdot += u dt (the UR5e state of Sec. III-C) */
} ce_dyn_t;

typedef enum {
  CE_MPPI_OK = 0,
  CE_MPPI_ERR_INVALID_ARG = 1, /* a parameter or size is out of range         */
  CE_MPPI_ERR_NO_MEMORY = 2,   /* device or host allocation failed            */
  CE_MPPI_ERR_CUDA = 3,        /* a CUDA runtime call failed                  */
  CE_MPPI_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up          */
  CE_MPPI_ERR_BUSY = 5         /* result not ready yet                        */
} ce_status_t;

/* Which update a replan applied (Algorithm 1). */
typedef enum {
  CE_MODE_NOCOL = 0,    /* no colliding rollout: standard MPPI over all K (Eq. 6-7) */
  CE_MODE_ALLCOL = 1,   /* every rollout collides: standard MPPI over all K         */
  CE_MODE_ALLNOISE = 2, /* DBSCAN found no cluster: standard MPPI over V            */
  CE_MODE_STATIC = 3,   /* cluster of least mean cost (Eq. 14)                      */
  CE_MODE_DYNAMIC = 4,  /* cluster most opposite to the obstacle motion (Eq. 18)    */
  CE_MODE_MPPI = 5      /* standard MPPI requested (mppi_only): Eq. 6-7 over all K  */
} ce_mode_t;

typedef struct {
  int dyn;               /* ce_dyn_t                                               */
  int K;                 /* rollouts, 1 .. 1<<20                                   */
  int T;                 /* horizon N, 1 .. 256                                    */
  float dt;              /* model step (s), > 0                                    */
  float obs_dt;          /* spacing of the obstacle observations (Delta t of Eq. 17) */
  float lambda;          /* temperature, > 0                                       */
  float dbscan_eps;      /* DBSCAN radius on the unit feature z, (0.02, 2]         */
  int min_pts;           /* DBSCAN minPts, the point itself included, >= 1         */
  float sigma[6];        /* per control dimension noise std, >= 0                  */
  float u_min[6], u_max[6]; /* input box, u_min <= u_max                           */
  float goal[16];        /* 2-D: goal state (n entries); arm: p_g[3], R_g[9]        */
  float w[8];            /* cost weights: DI (pos, ctrl, terminal);                */
                         /* unicycle Q[3], H[3] (Eq. 22-23); arm (w_p, w_R, w_c);   */
                         /* 2-D robots: w[7] is added once to S of a colliding    */
                         /* rollout (I_col of Eq. 8; 0 for CE-MPPI, which prunes) */
  int n_obs_max;         /* largest obstacle count a replan may pass, >= 0         */
  int hist_len;          /* H, observations per replan, >= 1                       */
  float robot_radius;    /* 2-D robot disc radius / arm link-sphere radius (m)     */
  float norm_eps;        /* epsilon of the normalisations of Eq. 13, 15-17, > 0    */
  float v_static_thresh; /* |v_o*| <= this selects by cost (Eq. 14), else Eq. 18   */
  unsigned long long seed; /* Philox4x32-10 key of the perturbations               */
  int ref_mode;          /* 0: colliding rollouts whose first hit is the closest   */
                         /*    hit obstacle (the method overview); 1: all of C_col */
  int check_j0;          /* 1: the current state x_0 also counts for collisions    */
  int mppi_only;         /* 1: standard MPPI (Eq. 6-7 over all K), no pruning or   */
                         /*    clustering (the paper's comparison baseline)        */
  int noise_regen;       /* 0: the rollouts store eps' (K*T*m floats) for the      */
                         /*    update; 1: nothing is stored, the update draws the  */
                         /*    same Philox numbers again for the rollouts of       */
                         /*    nonzero weight (less memory; peek of EPS refused).  */
                         /*    Cheaper when few weights are nonzero; an update over */
                         /*    many rollouts (the no-collision fallback with close  */
                         /*    costs) draws them all again, slower than reading    */
                         /*    stored ones                                          */
  int uf_limit;          /* parent reads allowed per union-find operation of the   */
                         /*    grid DBSCAN (0: the default, 2^20, never reached by */
                         /*    valid data).  When one runs out, the replan reports */
                         /*    CE_MPPI_ERR_TIMEOUT in diag.status and takes the    */
                         /*    all-noise fallback; 1 makes every union give up (a  */
                         /*    hook for testing that failure path), >= 0           */
} ce_mppi_params;

/* Per-replan diagnostics. */
typedef struct {
  int mode;        /* ce_mode_t; -1 when the replan was refused (status != 0 and  */
                   /* nothing updated, nominal and counter kept: a non-finite     */
                   /* device input, INVALID_ARG; or a rollout CTA whose bounded   */
                   /* wait for its copy of the obstacle tracks ran out, TIMEOUT)  */
  int n_col;       /* |C_col|                                                     */
  int n_valid;     /* |V|                                                         */
  int n_clusters;  /* M_t                                                         */
  int sel_label;   /* c*, or -1                                                   */
  int o_star;      /* index of the reference obstacle, or -1                      */
  int dynamic;     /* 1 when the selection used the obstacle motion              */
  int status;      /* 0, or a ce_status_t raised on the device                   */
  float S_min;     /* least cost among the rollouts of the update                 */
  float pbar[3];   /* reference point (Eq. 11)                                    */
  float v_obs[3];  /* velocity estimate of the reference obstacle (Eq. 17)        */
  unsigned long long counter; /* replan counter this replan used                  */
  int col_tests;   /* obstacle tests per rollout over the horizon after the reach */
                   /* culling of the track builder: 2-D robots one per obstacle  */
                   /* of a pair of steps (at most ceil(T/2) * n_obs; the exact   */
                   /* tests of a pair that may collide come on top), the arm     */
                   /* one per obstacle and step (T * n_obs)                      */
} ce_mppi_diag;

/* Inputs and outputs of one replan, all in device memory. */
typedef struct {
  const float* x0;         /* [n] current state                                    */
  const float* obs_hist;   /* [H][n_obs][p] obstacle centres, oldest first         */
  const float* obs_radius; /* [n_obs] obstacle radii                               */
  int n_obs;               /* 0 .. n_obs_max                                       */
  long long obs_step;      /* floats obs_hist advances per replan (0: fixed), for  */
                           /* recorded observation streams replayed by a batch     */
  float* u_out;            /* [T][m] updated nominal before the shift, or NULL     */
  float* x_next;           /* [n] f(x0, u_0), or NULL; may alias x0 (closed loop)   */
  ce_mppi_diag* diag;      /* or NULL                                              */
} ce_mppi_request;

typedef struct ce_mppi_handle ce_mppi_handle;
typedef struct ce_mppi_batch ce_mppi_batch;

/* Allocate a planner.  stream is a cudaStream_t (NULL: the legacy default
 * stream).  The nominal sequence starts at zero, the replan counter at 0.
 * Errors: INVALID_ARG (bad parameter), NO_MEMORY, CUDA.                        */
ce_status_t ce_mppi_create(const ce_mppi_params* params, void* stream, ce_mppi_handle** out);
/* Wait for the handle's queued work and free everything it owns.              */
ce_status_t ce_mppi_destroy(ce_mppi_handle* h);

/* Nominal control sequence U_t [T][m] (host memory).  Blocking.               */
ce_status_t ce_mppi_set_nominal(ce_mppi_handle* h, const float* U);
ce_status_t ce_mppi_get_nominal(ce_mppi_handle* h, float* U);
/* Replan counter: the upper Philox counter words of the next replan.  Blocking. */
ce_status_t ce_mppi_set_counter(ce_mppi_handle* h, unsigned long long counter);
ce_status_t ce_mppi_get_counter(ce_mppi_handle* h, unsigned long long* counter);

/* One replan from host buffers: copies x0 [n], obs_hist [H][n_obs][p] and
 * obs_radius [n_obs] to the device, runs Algorithm 1, copies the updated
 * nominal (before the shift) to u_out [T][m] and the diagnostics to diag
 * (nullable), and returns when done.  Afterwards the handle's nominal is the
 * shifted sequence and its counter has advanced by one.  The inputs are
 * checked first as by ce_mppi_check_inputs (NaN or infinity: INVALID_ARG,
 * nothing launched).
 * Errors: INVALID_ARG, CUDA, TIMEOUT (device-side wait limit reached).       */
ce_status_t ce_mppi_replan(ce_mppi_handle* h, const float* x0, const float* obs_hist,
                           const float* obs_radius, int n_obs, float* u_out,
                           ce_mppi_diag* diag);

/* Check the host inputs of one replan for a planner created with params,
 * without a GPU and without launching anything: params as ce_mppi_create
 * validates them; x0 [n] non-NULL and finite; 0 <= n_obs <= n_obs_max;
 * obs_hist [H][n_obs][p] and obs_radius [n_obs] non-NULL when n_obs > 0, every
 * value finite and every radius >= 0.  ce_mppi_replan and the server's submit
 * calls apply the same check before they copy anything.  Device-buffer replans
 * (ce_mppi_replan_dev, batches) cannot be checked on the host: their obstacle
 * track kernel reports a non-finite x0, observation or radius as INVALID_ARG
 * in diag->status instead.  Errors: INVALID_ARG.                             */
ce_status_t ce_mppi_check_inputs(const ce_mppi_params* params, const float* x0,
                                 const float* obs_hist, const float* obs_radius, int n_obs);

/* One replan from device buffers, queued on the handle's stream; returns
 * without waiting.  Device-side faults of the bounded waits are reported in
 * diag->status.  A NaN or infinity in x0, the observation window or the
 * radii (or a negative radius) is found by the first kernel of the replan:
 * diag->status = INVALID_ARG, diag->mode = -1, u_out receives the current
 * nominal, and the nominal, the counter and x_next are left unchanged.
 * Errors: INVALID_ARG, CUDA.                                                  */
ce_status_t ce_mppi_replan_dev(ce_mppi_handle* h, const ce_mppi_request* req);

/* Batches: n handles replanned together by one replan chain for all of them
 * (instances of different K, T and obstacle count): the track kernel, the
 * rollout kernel, and one kernel running pruning, DBSCAN, selection and the
 * update as a thread-block cluster per instance (plus the tiled update kernel
 * for the arms).  The requests are fixed at creation (use obs_step to replay
 * recorded observation streams).  With n_branches > 1 the instances are split
 * (balanced by K*T) into that many branches whose chains run concurrently on
 * streams of their own.  n_branches = 0 autotunes: the branch count (1, 2,
 * 4, 8) and the CTAs per instance of the clustering kernel (1, 2, 4, 8) are
 * chosen by timing the batch itself (a warm-up and three replans per
 * candidate; the planners' nominals, counters and the requests' x0 are
 * restored after each, u_out / x_next / diag receive the trial results) and
 * cached per (dynamics, log2 largest K, largest T / 16, log2 n).  With
 * use_graph != 0 the whole batch (fork, branches, join) is captured once as a
 * CUDA graph and replayed by ce_mppi_batch_run.  stream is the cudaStream_t
 * the batch runs on.  Every handle must have the same dynamics kind.  Results
 * are bitwise those of replanning each handle alone.  Errors: INVALID_ARG,
 * NO_MEMORY, CUDA.                                                            */
ce_status_t ce_mppi_batch_create(ce_mppi_handle* const* hs, const ce_mppi_request* reqs,
                                 int n, void* stream, int use_graph, int n_branches,
                                 ce_mppi_batch** out);
/* The batch's branch count and clustering-kernel CTAs per instance (0: chosen
 * per launch from the occupancy of the device).  Errors: INVALID_ARG.        */
ce_status_t ce_mppi_batch_config(const ce_mppi_batch* b, int* n_branches, int* post_ctas);
/* Set the clustering-kernel CTAs per instance of the batch's later launches
 * made without a graph (ce_mppi_batch_run_part; ce_mppi_batch_run of a batch
 * created with use_graph = 0): 1, 2, 4 or 8 CTAs (one thread-block cluster
 * per instance), or 0 to choose per launch from the occupancy of the device
 * as if the batch ran alone.  A batch whose clustering runs beside other work
 * (the halves of a software pipeline) may give the SMs to that work with
 * fewer CTAs.  The results do not depend on it (the stage sums run in an
 * order fixed by K alone).  Errors: INVALID_ARG (NULL batch, another value,
 * or a batch that replays a captured graph, whose launches are fixed).      */
ce_status_t ce_mppi_batch_set_post_ctas(ce_mppi_batch* b, int post_ctas);
/* Queue one replan of every instance of the batch; returns without waiting.  */
ce_status_t ce_mppi_batch_run(ce_mppi_batch* b);
/* A batch fed from host buffers (the counterpart of ce_mppi_replan for many
 * planners): as ce_mppi_batch_create, but the requests are the batch's own --
 * one device staging block (inputs, then outputs) mirrored in pinned host
 * memory, owned and freed by the batch.  n_obs[i] fixes instance i's obstacle
 * count (0 .. its n_obs_max).  Errors: INVALID_ARG, NO_MEMORY, CUDA.          */
ce_status_t ce_mppi_batch_create_host(ce_mppi_handle* const* hs, const int* n_obs, int n,
                                      void* stream, int use_graph, int n_branches,
                                      ce_mppi_batch** out);
/* One replan of every instance of a host-buffer batch, blocking: the inputs
 * of instance i follow those of instance i-1 in x0s ([n] each), hists
 * ([H][n_obs[i]][p] each) and radii ([n_obs[i]] each); they are checked as by
 * ce_mppi_check_inputs, packed and copied in one transfer; the batch runs as
 * ce_mppi_batch_run; the updated nominals (u_outs, [T][m] each), the next
 * states (x_nexts, [n] each, nullable) and the diagnostics (diags, nullable)
 * come back in one transfer.  Afterwards every handle's nominal is shifted and
 * its counter advanced.  Errors: INVALID_ARG (not a host-buffer batch, a
 * refused input: nothing launched), CUDA, TIMEOUT.                            */
ce_status_t ce_mppi_batch_run_host(ce_mppi_batch* b, const float* x0s, const float* hists,
                                   const float* radii, float* u_outs, float* x_nexts,
                                   ce_mppi_diag* diags);
/* Queue one half of a replan of every instance, without a graph, on stream (a
 * cudaStream_t; NULL: the batch's stream): part 0 = obstacle tracks and the
 * rollouts (Algorithm 1 [Rollouts]); part 1 = pruning, reference point,
 * features, DBSCAN, selection, weights and the update with its shift.  Part 1
 * must follow part 0 of the same replan in stream order, and part 0 of the
 * next replan must follow part 1.  Between the two, the instances' state is
 * held on the device, so the halves of two batches of independent instances
 * can be interleaved (one batch's rollouts over the other's clustering), for
 * example on two streams inside the caller's own CUDA graph.  Part 0 may also
 * be queued as its two launches: part 2 = the obstacle tracks alone, part 3
 * = the rollouts alone (after part 2 of the same replan); the tracks of the
 * next replan need only part 1 of the previous one, so they can run beside
 * other work instead of at the head of the rollouts.  Part 2 is launched as
 * a programmatic dependent of the kernel before it in stream order (part 1's
 * update kernel, which lets it be scheduled early; the track kernel waits for
 * that grid's completion before it reads the state), so queue it directly
 * behind part 1, not behind a wait on another stream's launch-completion
 * event (its grid would then wait for that kernel's completion).  The results
 * are bitwise those of ce_mppi_batch_run.  Errors: INVALID_ARG, CUDA.        */
ce_status_t ce_mppi_batch_run_part(ce_mppi_batch* b, int part, void* stream);
/* ce_mppi_batch_run_part with, for part 1, an event `started` (a cudaEvent_t
 * created with cudaEventDisableTiming, or NULL) that the clustering kernel's
 * launch records as its launch-completion event: it fires once every CTA of
 * that kernel has begun execution (best effort: the runtime may fire it only
 * when the kernel completes).  A stream that waits on it before launching the
 * other half's rollouts lets the clustering kernel's CTAs, each of which
 * needs a whole SM, take their SMs first; without it, whichever grid the
 * device dispatches first may fill every SM and the two run one after the
 * other.  Recorded in stream capture it becomes a launch-completion edge of
 * the caller's graph.  `started` must be NULL for part 0.  The results do not
 * depend on it.  Errors: INVALID_ARG, CUDA.                                  */
ce_status_t ce_mppi_batch_run_part_ev(ce_mppi_batch* b, int part, void* stream, void* started);
/* Run one replan of the batch stage by stage (no graph) with CUDA events
 * between the stage launches, wait for it, and write the device time of each
 * stage in milliseconds to stage_ms[6]: tracks, rollouts, prune + reference
 * point + features, DBSCAN, cluster statistics + selection + weights, update.
 * The replan advances the instances like ce_mppi_batch_run.                   */
ce_status_t ce_mppi_batch_profile(ce_mppi_batch* b, float* stage_ms);
ce_status_t ce_mppi_batch_destroy(ce_mppi_batch* b);

/* ---- continuous-batching server ------------------------------------------
 * Controller sessions are admitted against a device-memory budget and keep
 * their planner state (nominal, replan counter, scratch) on the device.  A
 * worker thread batches the queued replan requests of one dynamics kind as
 * soon as one of n_streams in-flight slots is free: one input transfer, one
 * launch per stage for the whole batch, one output transfer; batches on
 * different slots overlap.  A session is in at most one batch at a time; a
 * request submitted while the session's previous one is still queued replaces
 * it, and every ticket of the replaced request receives the newer result.
 * Each replan's result is bitwise the result of replanning that session alone.
 * Thread-safe: any number of host threads may submit and poll.               */
typedef struct ce_mppi_server ce_mppi_server;
typedef struct {
  size_t mem_budget_bytes; /* device bytes all sessions together may hold     */
  int max_sessions;        /* session slots, 1 .. 65536                        */
  int max_batch;           /* most replans in one batch, >= 1                  */
  int n_streams;           /* batches in flight at once, 1 .. 16 (>= 2 overlaps) */
  int device;              /* CUDA device ordinal                              */
} ce_server_params;
typedef struct {
  unsigned long long replans, batches, sessions_opened, sessions_rejected, superseded;
  size_t mem_in_use;       /* device bytes held by open sessions               */
  int sessions_open;
  double mean_batch;       /* replans per batch                                */
  double p50_latency_s, p99_latency_s, mean_latency_s; /* submit -> result ready */
} ce_server_stats;

/* Start a server (and its worker thread) on `device`.
 * Errors: INVALID_ARG, NO_MEMORY, CUDA.                                      */
ce_status_t ce_mppi_server_create(const ce_server_params* params, ce_mppi_server** out);
/* Stop the worker, finish the batches in flight, free every session.        */
ce_status_t ce_mppi_server_destroy(ce_mppi_server* s);
/* Admit a session with its own planner parameters; NO_MEMORY when the budget
 * or the slots are exhausted (the session is rejected, nothing is held).     */
ce_status_t ce_mppi_server_open(ce_mppi_server* s, const ce_mppi_params* params, int* session);
/* Close a session; its memory is released once its batch in flight is done. */
ce_status_t ce_mppi_server_close(ce_mppi_server* s, int session);
/* Queue a replan from host buffers (x0 [n], obs_hist [H][n_obs][p],
 * obs_radius [n_obs]), copied before the call returns.  ticket (nullable)
 * receives an id for ce_mppi_server_poll; with NULL the result is dropped and
 * only counted in the statistics.                                            */
ce_status_t ce_mppi_server_submit(ce_mppi_server* s, int session, const float* x0,
                                  const float* obs_hist, const float* obs_radius, int n_obs,
                                  unsigned long long* ticket);
/* Queue n replans at once without tickets (results only counted in the
 * statistics): session ids sids[n]; the inputs of request i follow those of
 * request i-1 in x0s (n floats each), hists ([H][n_obs[i]][p] each) and radii
 * (n_obs[i] each).  For load generators.  Requests are taken in order: on an
 * INVALID_ARG for request i (no such session, bad obstacle count, NULL
 * obstacle arrays), requests 0 .. i-1 stay queued and the rest are not.      */
ce_status_t ce_mppi_server_submit_many(ce_mppi_server* s, int n, const int* sids,
                                       const float* x0s, const float* hists,
                                       const float* radii, const int* n_obs);
/* BUSY until the ticket's replan is done; then copies the updated nominal
 * (u_out [T][m]), the diagnostics and the latency (seconds from submit to
 * result) and forgets the ticket.                                            */
ce_status_t ce_mppi_server_poll(ce_mppi_server* s, unsigned long long ticket, float* u_out,
                                ce_mppi_diag* diag, double* latency_s);
/* Counters and latency percentiles since the last reset (reset != 0 clears). */
ce_status_t ce_mppi_server_stats(ce_mppi_server* s, ce_server_stats* out, int reset);

/* Internal buffers of the last replan, copied to host memory (blocking), for
 * diagnostics and stage-by-stage checks.  bytes must equal the buffer size.  */
typedef enum {
  CE_BUF_S = 0,       /* float [K]      trajectory costs S (Eq. 5)                  */
  CE_BUF_HIT = 1,     /* int   [K]      first-hit obstacle, -1 when collision-free  */
  CE_BUF_PN = 2,      /* float [p][K]   terminal task positions p(x_T)              */
  CE_BUF_EPS = 3,     /* float [T*m][K] effective perturbations u^(k) - u (Eq. 3)   */
  CE_BUF_IDXV = 4,    /* int   [K]      V in ascending k (first n_valid used)       */
  CE_BUF_IDXC = 5,    /* int   [K]      C_col in ascending k (first n_col used)     */
  CE_BUF_Z = 6,       /* float [p][K]   feature z of V (Eq. 13), V order            */
  CE_BUF_G = 7,       /* float [p][K]   unit displacement g of V (Eq. 15)           */
  CE_BUF_LABEL = 8,   /* int   [K]      DBSCAN label of V, -1 noise                 */
  CE_BUF_W = 9,       /* float [K]      normalised update weights (Eq. 6 / Eq. 19)  */
  CE_BUF_HITJ = 10,   /* int   [K]      horizon step of the first hit, -1 if none   */
  CE_BUF_DBCYC = 11   /* long long [16] SM clock stamps (SM cycles) that thread 0 of  */
                      /* the clustering kernel's first CTA leaves: [0..8] the DBSCAN */
                      /* phases, [9] kernel start, [10] after pruning, [11] after   */
                      /* DBSCAN, [12] after the statistics, selection and weights, */
                      /* [13] after the partial sums of a dense update (rank 0     */
                      /* alone from here), [14] after the update and its shift;    */
                      /* [15] unused                                                */
} ce_buf_t;
ce_status_t ce_mppi_peek(ce_mppi_handle* h, int which, void* host_dst, size_t bytes);

/* ---- stage entry points (device buffers, queued on stream) ---------------- */

/* Philox4x32-10 words of the perturbation stream: out[k][b][4] for rollouts
 * k < K and blocks b < nblk, counter (k, b, counter_lo, counter_hi), key
 * (seed_lo, seed_hi) (Salmon et al., SC'11).                                  */
ce_status_t ce_mppi_philox_dev(unsigned long long seed, unsigned long long counter, int K,
                               int nblk, unsigned int* out, void* stream);
/* The first n standard normals of rollouts k < K: out[k][n]: normal i is
 * element i % 4 of block i / 4; Box-Muller on the uniforms ((w >> 9) + 1/2)
 * 2^-23 of the word pairs (w0,w1) and (w2,w3): r = sqrt(-2 ln u1),
 * (r cos 2 pi u2, r sin 2 pi u2).  FP32: -2 ln u1 as ce_mppi_neg2ln_dev, the
 * sine and cosine from the special-function unit, so each normal is within
 * ~5e-6 of exact (absolute; the largest radius is 5.77).  These are the
 * normals the rollouts draw.                                                 */
ce_status_t ce_mppi_normals_dev(unsigned long long seed, unsigned long long counter, int K,
                                int n, float* out, void* stream);
/* -2 ln u, the squared Box-Muller radius, for every uniform the rollouts can
 * draw: out[m] for u = (m + 1/2) 2^-23, m = 0 .. 2^23 - 1 (out: 2^23 floats,
 * device).  FP32: a Taylor series in u - 1 for u > 7/8, the special-function
 * unit's base-2 logarithm elsewhere; relative error under 2^-20 (checked
 * against the exact values).  Errors: INVALID_ARG (NULL out), CUDA.          */
ce_status_t ce_mppi_neg2ln_dev(float* out, void* stream);
/* DBSCAN (Sec. II-B2) of n points z stored as [p][ld] (SoA, p = 2 or 3):
 * neighbours when the FP32 sum of squared coordinate differences (coordinate
 * order, no fused multiply-add) is <= fl32(eps^2); core when at least min_pts
 * neighbours (itself included); clusters are connected components of the core
 * points; a non-core point takes the cluster of its lowest-index core
 * neighbour, else -1.  Cluster ids 0..M-1 follow the smallest core member.
 * labels [n] and n_clusters [1] are device outputs.  workspace is device memory
 * of at least ce_mppi_dbscan_workspace_bytes(n) bytes.                        */
size_t ce_mppi_dbscan_workspace_bytes(int n);
ce_status_t ce_mppi_dbscan_dev(const float* z, int n, int ld, int p, float eps, int min_pts,
                               int* labels, int* n_clusters, void* workspace, size_t ws_bytes,
                               void* stream);

/* DBSCAN exactly as ce_mppi_dbscan_dev, for callers that cannot allocate
 * device memory (no workspace argument).  It makes no allocation call: its
 * scratch is a fixed __device__ array of about 0.6 MB compiled into the
 * library, which every GPU that loads the library keeps until the process
 * exits.  Limits: n <= 16384 points (larger n is rejected with INVALID_ARG).
 * The first call on a device looks up the scratch's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the one scratch array and nothing in it needs to
 * start cleared; calls that can run at the same time on the GPU (different
 * streams, or different host threads) race on it and must be serialised by
 * the caller.  The paper has no counterpart: this is a deployment variant of
 * the clustering stage.  Errors: INVALID_ARG, CUDA.                           */
ce_status_t ce_mppi_dbscan_noalloc_dev(const float* z, int n, int ld, int p, float eps,
                                       int min_pts, int* labels, int* n_clusters,
                                       void* stream);

/* Host helper: forward kinematics of the arm model (standard DH, UR5e-like),
 * frame origins O[7][3] and end-effector rotation R[3][3], FP64, for turning a
 * joint-space goal into the pose goal of ce_mppi_params.                      */
ce_status_t ce_mppi_arm_fk(const double* q, double* O, double* R);

/* Thread-local message of the last failed call on this thread.               */
const char* ce_mppi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CE_MPPI_H */
