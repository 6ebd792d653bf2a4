// ce_mppi_api.cu -- host side of the C ABI declared in include/ce_mppi.h:
// parameter validation, device memory of a planner, the stage chain on a
// stream, batches (one launch per stage for many instances) with optional
// CUDA-graph capture, and the stage entry points used for checking.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "ce_mppi_host.h"

using namespace cem;

namespace {

thread_local std::string g_err;

ce_status_t fail(ce_status_t s, const std::string& msg) {
  g_err = msg;
  return s;
}

ce_status_t cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return CE_MPPI_ERR_CUDA;
}

#define CE_CUDA(call)                                         \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

void dims_of(int dyn, int* n, int* m, int* p) {
  *n = dyn == CE_DYN_DOUBLE_INT_2D ? 4 : dyn == CE_DYN_UNICYCLE ? 3 : dyn == CE_DYN_ARM6_KIN ? 6 : 12;
  *m = is_arm(dyn) ? 6 : 2;
  *p = is_arm(dyn) ? 3 : 2;
}

bool finite(float v) { return std::isfinite(v); }

// DBSCAN grid: cell side 0.99 eps / sqrt(p) (any two points of a cell are
// neighbours), G cells per axis over [-1, 1], reach R cells.
void dbscan_grid(float eps, int p, float* cell_inv, int* G, int* R, int* ncells) {
  const double ci = std::sqrt((double)p) / (0.99 * (double)eps);
  *cell_inv = (float)ci;
  *G = (int)std::floor(2.0 * ci) + 1;
  *R = (int)std::ceil((double)eps * ci);
  *ncells = p == 3 ? (*G) * (*G) * (*G) : (*G) * (*G);
}

float eps_squared(float eps) {
  volatile float e = eps;
  return e * e;  // FP32 product of the FP32 radius (the predicate's eps^2)
}

std::mutex g_cfg_mu;
std::vector<int> g_cfg_devices;   // devices whose kernel attributes are set

}  // namespace

namespace cem {
void set_last_error(const char* msg) { g_err = msg; }

void ensure_configured() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  if (std::find(g_cfg_devices.begin(), g_cfg_devices.end(), dev) != g_cfg_devices.end()) return;
  configure_rollout();
  configure_cluster(g_cfg_devices.empty());
  g_cfg_devices.push_back(dev);
}
}  // namespace cem

namespace {

ce_status_t validate(const ce_mppi_params* P) {
  if (!P) return fail(CE_MPPI_ERR_INVALID_ARG, "params is NULL");
  if (P->dyn < 0 || P->dyn > 3) return fail(CE_MPPI_ERR_INVALID_ARG, "dyn must be 0, 1, 2 or 3");
  if (P->K < 1 || P->K > (1 << 20)) return fail(CE_MPPI_ERR_INVALID_ARG, "K must be in [1, 2^20]");
  if (P->T < 1 || P->T > kMaxT) return fail(CE_MPPI_ERR_INVALID_ARG, "T must be in [1, 256]");
  if (!(P->dt > 0) || !finite(P->dt)) return fail(CE_MPPI_ERR_INVALID_ARG, "dt must be > 0");
  if (!(P->obs_dt > 0) || !finite(P->obs_dt))
    return fail(CE_MPPI_ERR_INVALID_ARG, "obs_dt must be > 0");
  if (!(P->lambda > 0) || !finite(P->lambda))
    return fail(CE_MPPI_ERR_INVALID_ARG, "lambda must be > 0");
  if (!(P->dbscan_eps > 0.02f) || !(P->dbscan_eps <= 2.0f))
    return fail(CE_MPPI_ERR_INVALID_ARG, "dbscan_eps must be in (0.02, 2]");
  if (P->min_pts < 1) return fail(CE_MPPI_ERR_INVALID_ARG, "min_pts must be >= 1");
  if (P->hist_len < 1) return fail(CE_MPPI_ERR_INVALID_ARG, "hist_len must be >= 1");
  if (P->n_obs_max < 0 || P->n_obs_max > kMaxObs)
    return fail(CE_MPPI_ERR_INVALID_ARG, "n_obs_max must be in [0, 4096]");
  if (!(P->robot_radius >= 0) || !finite(P->robot_radius))
    return fail(CE_MPPI_ERR_INVALID_ARG, "robot_radius must be >= 0");
  if (!(P->norm_eps > 0) || !finite(P->norm_eps))
    return fail(CE_MPPI_ERR_INVALID_ARG, "norm_eps must be > 0");
  if (!(P->v_static_thresh >= 0) || !finite(P->v_static_thresh))
    return fail(CE_MPPI_ERR_INVALID_ARG, "v_static_thresh must be >= 0");
  if (P->ref_mode < 0 || P->ref_mode > 1) return fail(CE_MPPI_ERR_INVALID_ARG, "ref_mode must be 0 or 1");
  if (P->check_j0 < 0 || P->check_j0 > 1) return fail(CE_MPPI_ERR_INVALID_ARG, "check_j0 must be 0 or 1");
  if (P->mppi_only < 0 || P->mppi_only > 1)
    return fail(CE_MPPI_ERR_INVALID_ARG, "mppi_only must be 0 or 1");
  if (P->noise_regen < 0 || P->noise_regen > 1)
    return fail(CE_MPPI_ERR_INVALID_ARG, "noise_regen must be 0 or 1");
  if (P->uf_limit < 0) return fail(CE_MPPI_ERR_INVALID_ARG, "uf_limit must be >= 0");
  int n, m, p;
  dims_of(P->dyn, &n, &m, &p);
  for (int i = 0; i < m; ++i) {
    if (!(P->sigma[i] >= 0) || !finite(P->sigma[i]))
      return fail(CE_MPPI_ERR_INVALID_ARG, "sigma must be finite and >= 0");
    if (!finite(P->u_min[i]) || !finite(P->u_max[i]) || P->u_min[i] > P->u_max[i])
      return fail(CE_MPPI_ERR_INVALID_ARG, "u_min must be <= u_max, both finite");
  }
  for (int i = 0; i < 16; ++i)
    if (!finite(P->goal[i])) return fail(CE_MPPI_ERR_INVALID_ARG, "goal must be finite");
  for (int i = 0; i < 8; ++i)
    if (!finite(P->w[i])) return fail(CE_MPPI_ERR_INVALID_ARG, "weights must be finite");
  float ci;
  int G, R, nc;
  dbscan_grid(P->dbscan_eps, p, &ci, &G, &R, &nc);
  if (nc > kMaxCells)
    return fail(CE_MPPI_ERR_INVALID_ARG,
                "dbscan_eps too small for the DBSCAN grid (p=3 needs eps >= 0.19)");
  const size_t smem = track_bytes(P->T, P->n_obs_max) + (size_t)P->T * m * 4;
  if (smem > (size_t)kMaxSmemTracks)
    return fail(CE_MPPI_ERR_INVALID_ARG, "(T+1) * n_obs_max too large for shared memory");
  return CE_MPPI_OK;
}

}  // namespace

namespace {
void fill_scalars(InstDesc& d, const ce_mppi_params* P, const ce_mppi_handle* h);
}  // namespace

namespace cem {
void run_chain(int dyn, const KArgs& base, const int2* troll, int n_roll, const int2* tupd,
               int n_upd, int smem_roll, int max_cells, cudaStream_t s, const int* pre_roll,
               const int* pre_upd) {
  KArgs a = base;
  launch_tracks(a, s);
  a.tiles = troll;
  a.tprefix = pre_roll;
  a.n_tiles = n_roll;
  launch_rollout(dyn, a, smem_roll, s, true);
  // The fused kernel applies the update when few weights are nonzero; a dense
  // one (many nonzero weights: the arms' small costs, a no-collision replan
  // with close costs) is left to the tiled update kernel that follows over the
  // whole GPU, which skips the replans already done.
  const bool fused = launch_post(a, max_cells, s);
  if (!fused) {
    launch_prune(a, s);
    launch_dbscan(a, max_cells, s);
    launch_select(a, s);
  }
  a.tiles = tupd;
  a.tprefix = pre_upd;
  a.n_tiles = n_upd;
  launch_update(a, s);
}

ce_status_t validate_params(const ce_mppi_params* P) { return validate(P); }

bool same_layout(const ce_mppi_handle* h, const ce_mppi_params* P) {
  float ci;
  int G, R, nc;
  int n, m, p;
  dims_of(P->dyn, &n, &m, &p);
  dbscan_grid(P->dbscan_eps, p, &ci, &G, &R, &nc);
  return P->dyn == h->P.dyn && P->K == h->P.K && P->T == h->P.T &&
         P->n_obs_max == h->P.n_obs_max && P->hist_len == h->P.hist_len && nc == h->ncells &&
         P->noise_regen == h->P.noise_regen;
}

ce_status_t handle_retarget(ce_mppi_handle* h, const ce_mppi_params* P) {
  if (!same_layout(h, P)) return fail(CE_MPPI_ERR_INVALID_ARG, "different buffer layout");
  h->P = *P;
  fill_scalars(h->hdesc, P, h);
  float ci;
  dbscan_grid(P->dbscan_eps, h->p, &ci, &h->G, &h->R, &h->ncells);
  CE_CUDA(cudaMemsetAsync(h->hdesc.U, 0, sizeof(float) * P->T * h->m, h->stream));
  CE_CUDA(cudaMemsetAsync(h->hdesc.counter, 0, 8, h->stream));
  CE_CUDA(cudaMemcpyAsync(h->ddesc, &h->hdesc, sizeof(InstDesc), cudaMemcpyHostToDevice, h->stream));
  CE_CUDA(cudaStreamSynchronize(h->stream));
  return CE_MPPI_OK;
}
}  // namespace cem

namespace {

void tiles_of(const ce_mppi_handle* h, int inst, std::vector<int2>& roll, std::vector<int2>& upd) {
  const int per = is_arm(h->P.dyn) ? kArmWarps : kRolloutThreads;
  for (int t = 0; t * per < h->P.K; ++t) roll.push_back(make_int2(inst, t));
  // update tiles: (column block, rollout chunk) enumerated as kc * ncb + cb
  const int TM = h->P.T * h->m;
  const bool arm = is_arm(h->P.dyn);
  const int cper = 32, kch = arm ? kUpdChunkArm : kUpdChunk2D;   // (as k_update)
  const int ncb = (TM + cper - 1) / cper, nkc = (h->P.K + kch - 1) / kch;
  for (int t = 0; t < ncb * nkc; ++t) upd.push_back(make_int2(inst, t));
}

Req to_req(const ce_mppi_request* q, unsigned long long counter0) {
  Req r;
  std::memset(&r, 0, sizeof(r));
  r.x0 = q->x0;
  r.obs_hist = q->obs_hist;
  r.obs_radius = q->obs_radius;
  r.n_obs = q->n_obs;
  r.obs_step = q->obs_step;
  r.counter0 = counter0;
  r.u_out = q->u_out;
  r.x_next = q->x_next;
  r.diag = q->diag;
  return r;
}

// Parameter-derived fields of a descriptor (everything but the buffers).
void fill_scalars(InstDesc& d, const ce_mppi_params* P, const ce_mppi_handle* h) {
  const int K = P->K, Kp = h->Kp;
  float ci;
  int G, R, nc;
  dbscan_grid(P->dbscan_eps, h->p, &ci, &G, &R, &nc);
  d.dyn = P->dyn; d.K = K; d.Kp = Kp; d.T = P->T; d.m = h->m; d.n = h->n; d.p = h->p;
  d.n_obs_max = P->n_obs_max; d.H = P->hist_len; d.min_pts = P->min_pts; d.ref_mode = P->ref_mode;
  d.check_j0 = P->check_j0; d.G = G; d.R = R; d.regen = P->noise_regen;
  d.mppi_only = P->mppi_only;
  d.gsz = is_arm(P->dyn) ? 1 : 32;
  d.uf_limit = P->uf_limit > 0 ? P->uf_limit : kUfLimit;
  d.eps_ld_c = is_arm(P->dyn) ? 1 : Kp;
  d.eps_ld_k = is_arm(P->dyn) ? h->TMp : 1;
  d.dt = P->dt; d.obs_dt = P->obs_dt; d.inv_lambda = 1.0f / P->lambda;
  d.eps2 = eps_squared(P->dbscan_eps); d.cell_inv = ci; d.robot_radius = P->robot_radius;
  d.norm_eps = P->norm_eps; d.v_static_thresh = P->v_static_thresh;
  for (int i = 0; i < 6; ++i) { d.sigma[i] = P->sigma[i]; d.u_min[i] = P->u_min[i]; d.u_max[i] = P->u_max[i]; }
  for (int i = 0; i < 16; ++i) d.goal[i] = P->goal[i];
  for (int i = 0; i < 8; ++i) d.w[i] = P->w[i];
  d.seed_lo = (unsigned)P->seed; d.seed_hi = (unsigned)(P->seed >> 32);
  d.TMp = h->TMp;
}

// Host inputs of one replan: x0 [n], obs_hist [H][n_obs][p], obs_radius
// [n_obs], every value finite and every radius >= 0 (checked before anything
// is copied or launched).
ce_status_t check_inputs_dims(int n, int p, int H, int n_obs_max, const float* x0,
                              const float* obs_hist, const float* obs_radius, int n_obs) {
  if (!x0) return fail(CE_MPPI_ERR_INVALID_ARG, "x0 is NULL");
  if (n_obs < 0 || n_obs > n_obs_max)
    return fail(CE_MPPI_ERR_INVALID_ARG, "n_obs must be in [0, n_obs_max]");
  if (n_obs > 0 && (!obs_hist || !obs_radius))
    return fail(CE_MPPI_ERR_INVALID_ARG, "obs_hist / obs_radius is NULL");
  for (int i = 0; i < n; ++i)
    if (!finite(x0[i])) return fail(CE_MPPI_ERR_INVALID_ARG, "x0 holds a NaN or an infinity");
  const size_t nh = (size_t)H * n_obs * p;
  for (size_t i = 0; i < nh; ++i)
    if (!finite(obs_hist[i]))
      return fail(CE_MPPI_ERR_INVALID_ARG, "obs_hist holds a NaN or an infinity");
  for (int i = 0; i < n_obs; ++i)
    if (!finite(obs_radius[i]) || !(obs_radius[i] >= 0.0f))
      return fail(CE_MPPI_ERR_INVALID_ARG, "obs_radius must be finite and >= 0");
  return CE_MPPI_OK;
}

ce_status_t check_req(const ce_mppi_handle* h, const ce_mppi_request* q) {
  if (!q) return fail(CE_MPPI_ERR_INVALID_ARG, "request is NULL");
  if (!q->x0) return fail(CE_MPPI_ERR_INVALID_ARG, "x0 is NULL");
  if (q->n_obs < 0 || q->n_obs > h->P.n_obs_max)
    return fail(CE_MPPI_ERR_INVALID_ARG, "n_obs must be in [0, n_obs_max]");
  if (q->n_obs > 0 && (!q->obs_hist || !q->obs_radius))
    return fail(CE_MPPI_ERR_INVALID_ARG, "obs_hist / obs_radius is NULL");
  return CE_MPPI_OK;
}

}  // namespace

namespace cem {
ce_status_t check_host_inputs(const ce_mppi_handle* h, const float* x0, const float* obs_hist,
                              const float* obs_radius, int n_obs) {
  return check_inputs_dims(h->n, h->p, h->P.hist_len, h->P.n_obs_max, x0, obs_hist, obs_radius,
                           n_obs);
}
}  // namespace cem

extern "C" {

const char* ce_mppi_last_error(void) { return g_err.c_str(); }

ce_status_t ce_mppi_create(const ce_mppi_params* P, void* stream, ce_mppi_handle** out) {
  if (!out) return fail(CE_MPPI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  ce_status_t st = validate(P);
  if (st != CE_MPPI_OK) return st;
  cem::ensure_configured();
  ce_mppi_handle* h = new (std::nothrow) ce_mppi_handle();
  if (!h) return fail(CE_MPPI_ERR_NO_MEMORY, "host allocation failed");
  h->P = *P;
  h->stream = static_cast<cudaStream_t>(stream);
  dims_of(P->dyn, &h->n, &h->m, &h->p);
  const int K = P->K, T = P->T, m = h->m, n = h->n, p = h->p;
  h->Kp = (K + 31) & ~31;
  h->TMp = (T * m + 3) & ~3;
  float ci;
  dbscan_grid(P->dbscan_eps, p, &ci, &h->G, &h->R, &h->ncells);
  const int Kp = h->Kp, nobs = P->n_obs_max, H = P->hist_len;
  const size_t A = 256;
  // carve one allocation
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes, A); return o; };
  const size_t o_ctr = take(8), o_ctl = take(sizeof(Ctl));
  const size_t o_U = take(sizeof(float) * T * m), o_Unew = take(sizeof(float) * T * m);
  // + 16: the packed 2-D table's header may round up 16 bytes past the rows'
  const size_t o_trk = take(std::max(track_bytes(T, nobs), track_pair_bytes(T, nobs)) + 16);
  const size_t o_S = take(4 * Kp), o_w = take(4 * Kp), o_Sv = take(4 * Kp),
               o_cmin = take(4 * Kp), o_nzk = take(4 * kSparseMax), o_nze = take(4 * kSparseMax),
               o_zpart = take(4 * kPruneRanges);
  const size_t o_pN = take(4 * 3 * Kp), o_z = take(4 * 3 * Kp), o_g = take(4 * 3 * Kp),
               o_zs = take(4 * 3 * Kp);
  const size_t eps_elems = P->noise_regen ? 0
                          : is_arm(P->dyn) ? (size_t)Kp * h->TMp : (size_t)T * m * Kp;
  const size_t o_eps = take(4 * eps_elems);
  size_t o_int[8];
  for (int i = 0; i < 8; ++i) o_int[i] = take(4 * Kp);
  const int gsz = is_arm(P->dyn) ? 1 : 32, ngroups = (K + gsz - 1) / gsz;
  const size_t o_gcnt = take(sizeof(int2) * ngroups), o_gS = take(sizeof(float4) * ngroups);
  const size_t o_osum = take(sizeof(long long) * 4 * (size_t)std::max(nobs, 1));
  const size_t o_bbox = take(sizeof(float) * 6 * h->ncells);
  const size_t o_ang = take(sizeof(int) * 2 * kAngBuckets);
  const int kch_min = std::min(kUpdChunkArm, kUpdChunk2D);   // most rollout chunks of an update
  const size_t o_upart = take(sizeof(float) * (size_t)((K + kch_min - 1) / kch_min) * h->TMp);
  // host-path staging: inputs then outputs
  const size_t in_x0 = 0, in_hist = align_up(4 * n, 16),
               in_rad = align_up(in_hist + 4 * (size_t)H * nobs * p, 16),
               in_end = align_up(in_rad + 4 * (size_t)nobs, 16);
  const size_t out_u = 0, out_diag = align_up(4 * (size_t)T * m, 16),
               out_end = align_up(out_diag + sizeof(ce_mppi_diag), 16);
  const size_t o_in = take(in_end), o_out = take(out_end);
  h->dbytes = off;
  h->in_bytes = in_end;
  h->out_bytes = out_end;
  cudaError_t e = cudaMalloc(&h->dmem, h->dbytes);
  if (e != cudaSuccess) { delete h; return fail(CE_MPPI_ERR_NO_MEMORY, "device allocation failed"); }
  e = cudaHostAlloc((void**)&h->h_stage, in_end + out_end, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    cudaFree(h->dmem);
    delete h;
    return fail(CE_MPPI_ERR_NO_MEMORY, "pinned host allocation failed");
  }
  char* b = static_cast<char*>(h->dmem);
  InstDesc& d = h->hdesc;
  std::memset(&d, 0, sizeof(d));
  fill_scalars(d, P, h);
  d.counter = reinterpret_cast<unsigned long long*>(b + o_ctr);
  d.ctl = reinterpret_cast<Ctl*>(b + o_ctl);
  d.U = reinterpret_cast<float*>(b + o_U);
  d.Unew = reinterpret_cast<float*>(b + o_Unew);
  d.tracks = reinterpret_cast<float4*>(b + o_trk);
  d.S = reinterpret_cast<float*>(b + o_S);
  d.w_k = reinterpret_cast<float*>(b + o_w);
  d.Sv = reinterpret_cast<float*>(b + o_Sv);
  d.cmin = reinterpret_cast<float*>(b + o_cmin);
  d.nzk = reinterpret_cast<int*>(b + o_nzk);
  d.nze = reinterpret_cast<float*>(b + o_nze);
  d.zpart = reinterpret_cast<float*>(b + o_zpart);
  d.pN = reinterpret_cast<float*>(b + o_pN);
  d.z = reinterpret_cast<float*>(b + o_z);
  d.g = reinterpret_cast<float*>(b + o_g);
  d.zs = reinterpret_cast<float*>(b + o_zs);
  d.eps = P->noise_regen ? nullptr : reinterpret_cast<float*>(b + o_eps);
  int** ints[8] = {&d.hit, &d.hitj, &d.idxV, &d.idxC, &d.label, &d.cell, &d.sorted, &d.parent};
  for (int i = 0; i < 8; ++i) *ints[i] = reinterpret_cast<int*>(b + o_int[i]);
  d.gcnt = reinterpret_cast<int2*>(b + o_gcnt);
  d.gS = reinterpret_cast<float4*>(b + o_gS);
  d.osum = reinterpret_cast<long long*>(b + o_osum);
  d.bbox = reinterpret_cast<float*>(b + o_bbox);
  d.ang = reinterpret_cast<int*>(b + o_ang);
  d.upart = reinterpret_cast<float*>(b + o_upart);
  d.TMp = h->TMp;
  h->d_x0 = reinterpret_cast<float*>(b + o_in + in_x0);
  h->d_hist = reinterpret_cast<float*>(b + o_in + in_hist);
  h->d_rad = reinterpret_cast<float*>(b + o_in + in_rad);
  h->d_uout = reinterpret_cast<float*>(b + o_out + out_u);
  h->d_diag = reinterpret_cast<ce_mppi_diag*>(b + o_out + out_diag);
  std::vector<int2> roll, upd;
  tiles_of(h, 0, roll, upd);
  h->n_roll = (int)roll.size();
  h->n_upd = (int)upd.size();
  h->smem_roll = is_arm(P->dyn)
                     ? (int)(track_bytes(T, nobs) + (size_t)T * m * 4)
                     : (int)((((size_t)T * m * 4 + 15) & ~(size_t)15) + track_smem_2d(T, nobs));
  auto cleanup = [&]() {
    cudaFree(h->dmem);
    cudaFree(h->ddesc);
    cudaFree(h->dtiles);
    cudaFreeHost(h->h_stage);
    delete h;
  };
  if ((e = cudaMalloc(&h->ddesc, sizeof(InstDesc))) != cudaSuccess ||
      (e = cudaMalloc(&h->dtiles, sizeof(int2) * (roll.size() + upd.size()))) != cudaSuccess) {
    cleanup();
    return fail(CE_MPPI_ERR_NO_MEMORY, "device allocation failed");
  }
  std::vector<int2> all(roll);
  all.insert(all.end(), upd.begin(), upd.end());
  if ((e = cudaMemsetAsync(h->dmem, 0, h->dbytes, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->ddesc, &d, sizeof(InstDesc), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->dtiles, all.data(), sizeof(int2) * all.size(), cudaMemcpyHostToDevice,
                           h->stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "create");
  }
  *out = h;
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_destroy(ce_mppi_handle* h) {
  if (!h) return CE_MPPI_OK;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->dmem);
  cudaFree(h->ddesc);
  cudaFree(h->dtiles);
  cudaFreeHost(h->h_stage);
  delete h;
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_set_nominal(ce_mppi_handle* h, const float* U) {
  if (!h || !U) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  CE_CUDA(cudaStreamSynchronize(h->stream));
  CE_CUDA(cudaMemcpy(h->hdesc.U, U, sizeof(float) * h->P.T * h->m, cudaMemcpyHostToDevice));
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_get_nominal(ce_mppi_handle* h, float* U) {
  if (!h || !U) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  CE_CUDA(cudaStreamSynchronize(h->stream));
  CE_CUDA(cudaMemcpy(U, h->hdesc.U, sizeof(float) * h->P.T * h->m, cudaMemcpyDeviceToHost));
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_set_counter(ce_mppi_handle* h, unsigned long long c) {
  if (!h) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL handle");
  CE_CUDA(cudaStreamSynchronize(h->stream));
  CE_CUDA(cudaMemcpy(h->hdesc.counter, &c, 8, cudaMemcpyHostToDevice));
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_get_counter(ce_mppi_handle* h, unsigned long long* c) {
  if (!h || !c) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  CE_CUDA(cudaStreamSynchronize(h->stream));
  CE_CUDA(cudaMemcpy(c, h->hdesc.counter, 8, cudaMemcpyDeviceToHost));
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_replan_dev(ce_mppi_handle* h, const ce_mppi_request* q) {
  if (!h) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL handle");
  ce_status_t st = check_req(h, q);
  if (st != CE_MPPI_OK) return st;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.D = h->ddesc;
  a.R = nullptr;
  a.r0 = to_req(q, 0);
  a.r0.obs_step = 0;  // a single replan reads obs_hist as given
  a.n_inst = 1;
  a.n_conc = 1;
  run_chain(h->P.dyn, a, h->dtiles, h->n_roll, h->dtiles + h->n_roll, h->n_upd, h->smem_roll,
            h->ncells, h->stream);
  CE_CUDA(cudaGetLastError());
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_check_inputs(const ce_mppi_params* P, const float* x0,
                                 const float* obs_hist, const float* obs_radius, int n_obs) {
  ce_status_t st = validate(P);
  if (st != CE_MPPI_OK) return st;
  int n, m, p;
  dims_of(P->dyn, &n, &m, &p);
  return check_inputs_dims(n, p, P->hist_len, P->n_obs_max, x0, obs_hist, obs_radius, n_obs);
}

ce_status_t ce_mppi_replan(ce_mppi_handle* h, const float* x0, const float* obs_hist,
                           const float* obs_radius, int n_obs, float* u_out, ce_mppi_diag* diag) {
  if (!h || !x0 || !u_out) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  ce_status_t st0 = check_inputs_dims(h->n, h->p, h->P.hist_len, h->P.n_obs_max, x0, obs_hist,
                                      obs_radius, n_obs);
  if (st0 != CE_MPPI_OK) return st0;
  const int n = h->n, p = h->p, H = h->P.hist_len, TM = h->P.T * h->m;
  unsigned char* hin = h->h_stage;
  unsigned char* hout = h->h_stage + h->in_bytes;
  const size_t hist_off = (char*)h->d_hist - (char*)h->d_x0, rad_off = (char*)h->d_rad - (char*)h->d_x0;
  std::memcpy(hin, x0, sizeof(float) * n);
  if (n_obs > 0) {
    std::memcpy(hin + hist_off, obs_hist, sizeof(float) * (size_t)H * n_obs * p);
    std::memcpy(hin + rad_off, obs_radius, sizeof(float) * n_obs);
  }
  CE_CUDA(cudaMemcpyAsync(h->d_x0, hin, h->in_bytes, cudaMemcpyHostToDevice, h->stream));
  ce_mppi_request q;
  std::memset(&q, 0, sizeof(q));
  q.x0 = h->d_x0;
  q.obs_hist = h->d_hist;
  q.obs_radius = h->d_rad;
  q.n_obs = n_obs;
  q.u_out = h->d_uout;
  q.diag = h->d_diag;
  ce_status_t st = ce_mppi_replan_dev(h, &q);
  if (st != CE_MPPI_OK) return st;
  CE_CUDA(cudaMemcpyAsync(hout, h->d_uout, h->out_bytes, cudaMemcpyDeviceToHost, h->stream));
  CE_CUDA(cudaStreamSynchronize(h->stream));
  std::memcpy(u_out, hout, sizeof(float) * TM);
  ce_mppi_diag dg;
  std::memcpy(&dg, hout + ((char*)h->d_diag - (char*)h->d_uout), sizeof(dg));
  if (diag) *diag = dg;
  if (dg.status == CE_MPPI_ERR_TIMEOUT)
    return fail(CE_MPPI_ERR_TIMEOUT, "device-side bounded wait gave up");
  if (dg.status != 0) return fail((ce_status_t)dg.status, "input refused on the device");
  return CE_MPPI_OK;
}

namespace {

void free_batch(ce_mppi_batch* b) {
  for (auto& br : b->branches) {
    cudaFree(br.dtiles_roll);
    cudaFree(br.dtiles_upd);
    if (br.stream) cudaStreamDestroy(br.stream);
    if (br.done) cudaEventDestroy(br.done);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->ddesc);
  cudaFree(b->dreq);
  cudaFree(b->dtiles_roll);
  cudaFree(b->dtiles_upd);
  if (b->d_stage) cudaFree(b->d_stage);
  if (b->h_stage) cudaFreeHost(b->h_stage);
  delete b;
}

// Queue one replan of every instance: the branches fork from `s`, run their
// chains concurrently on their own streams and join back into `s`.
void run_branches(ce_mppi_batch* b, cudaStream_t s) {
  if (b->branches.size() == 1) {
    const auto& br = b->branches[0];
    KArgs a;
    std::memset(&a, 0, sizeof(a));
    a.D = b->ddesc;
    a.R = b->dreq;
    a.n_inst = br.n;
    a.n_conc = (int)b->hs.size();
    a.post_ctas = b->post_ctas;
    run_chain(b->dyn, a, br.dtiles_roll, br.n_roll, br.dtiles_upd, br.n_upd, br.smem_roll,
              br.max_cells, s);
    return;
  }
  cudaEventRecord(b->fork, s);
  for (auto& br : b->branches) {
    cudaStreamWaitEvent(br.stream, b->fork, 0);
    KArgs a;
    std::memset(&a, 0, sizeof(a));
    a.D = b->ddesc + br.off;
    a.R = b->dreq + br.off;
    a.n_inst = br.n;
    a.n_conc = (int)b->hs.size();
    a.post_ctas = b->post_ctas;
    run_chain(b->dyn, a, br.dtiles_roll, br.n_roll, br.dtiles_upd, br.n_upd, br.smem_roll,
              br.max_cells, br.stream);
    cudaEventRecord(br.done, br.stream);
  }
  for (auto& br : b->branches) cudaStreamWaitEvent(s, br.done, 0);
}

}  // namespace

namespace {
ce_status_t batch_create_with(ce_mppi_handle* const* hs, const ce_mppi_request* reqs, int n,
                              void* stream, int use_graph, int n_branches, int post_ctas,
                              ce_mppi_batch** out);
ce_status_t batch_autotune(ce_mppi_handle* const* hs, const ce_mppi_request* reqs, int n,
                           void* stream, int* n_branches, int* post_ctas);
}  // namespace

ce_status_t ce_mppi_batch_create(ce_mppi_handle* const* hs, const ce_mppi_request* reqs, int n,
                                 void* stream, int use_graph, int n_branches,
                                 ce_mppi_batch** out) {
  if (!out) return fail(CE_MPPI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!hs || !reqs || n < 1) return fail(CE_MPPI_ERR_INVALID_ARG, "empty batch");
  if (n_branches < 0 || n_branches > 64) return fail(CE_MPPI_ERR_INVALID_ARG, "n_branches in [0, 64]");
  int post_ctas = 0;
  if (n_branches == 0) {
    ce_status_t st = batch_autotune(hs, reqs, n, stream, &n_branches, &post_ctas);
    if (st != CE_MPPI_OK) return st;
  }
  return batch_create_with(hs, reqs, n, stream, use_graph, n_branches, post_ctas, out);
}

ce_status_t ce_mppi_batch_config(const ce_mppi_batch* b, int* n_branches, int* post_ctas) {
  if (!b || !n_branches || !post_ctas) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  *n_branches = (int)b->branches.size();
  *post_ctas = b->post_ctas;
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_batch_set_post_ctas(ce_mppi_batch* b, int post_ctas) {
  if (!b) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL batch");
  if (post_ctas != 0 && post_ctas != 1 && post_ctas != 2 && post_ctas != 4 && post_ctas != 8)
    return fail(CE_MPPI_ERR_INVALID_ARG, "post_ctas must be 0, 1, 2, 4 or 8");
  if (b->exec) return fail(CE_MPPI_ERR_INVALID_ARG, "the batch replays a captured graph");
  b->post_ctas = post_ctas;
  return CE_MPPI_OK;
}

}  // extern "C"

namespace {

// The batch autotuner: the branch count and the fused kernel's CTAs per
// instance, chosen by timing the batch itself (one warm-up and three timed
// replans per candidate, every planner's nominal, counter and state restored
// after each) and cached per shape: (dynamics, log2 of the largest K, largest
// T / 16, log2 of the instance count).
struct TuneKey {
  int dyn, lk, lt, ln;
  bool operator<(const TuneKey& o) const {
    return std::tie(dyn, lk, lt, ln) < std::tie(o.dyn, o.lk, o.lt, o.ln);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;

int ceil_log2(long long v) {
  int l = 0;
  while ((1ll << l) < v) ++l;
  return l;
}

ce_status_t batch_autotune(ce_mppi_handle* const* hs, const ce_mppi_request* reqs, int n,
                           void* stream, int* n_branches, int* post_ctas) {
  int maxK = 0, maxT = 0;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL handle in batch");
    maxK = std::max(maxK, hs[i]->P.K);
    maxT = std::max(maxT, hs[i]->P.T);
  }
  const TuneKey key{hs[0]->P.dyn, ceil_log2(maxK), (maxT + 15) / 16, ceil_log2(n)};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *n_branches = it->second.first;
      *post_ctas = it->second.second;
      return CE_MPPI_OK;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // device copies of the state a replan changes: nominal, counter, x0 (x_next
  // may alias it)
  size_t bytes = 0;
  std::vector<size_t> offU(n), offX(n);
  for (int i = 0; i < n; ++i) {
    offU[i] = bytes;
    bytes += align_up(4 * (size_t)hs[i]->P.T * hs[i]->m + 8, 16);
    offX[i] = bytes;
    bytes += align_up(4 * (size_t)hs[i]->n, 16);
  }
  char* save = nullptr;
  cudaError_t e = cudaMalloc(&save, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "autotune scratch");
  auto copy_state = [&](bool to_save) {
    for (int i = 0; i < n; ++i) {
      const InstDesc& d = hs[i]->hdesc;
      const size_t ub = 4 * (size_t)hs[i]->P.T * hs[i]->m;
      char* su = save + offU[i];
      char* sx = save + offX[i];
      float* x0 = const_cast<float*>(reqs[i].x0);
      if (to_save) {
        cudaMemcpyAsync(su, d.U, ub, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(su + ub, d.counter, 8, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(sx, x0, 4 * (size_t)hs[i]->n, cudaMemcpyDeviceToDevice, s);
      } else {
        cudaMemcpyAsync(d.U, su, ub, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(d.counter, su + ub, 8, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(x0, sx, 4 * (size_t)hs[i]->n, cudaMemcpyDeviceToDevice, s);
      }
    }
  };
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  float best_ms = 1e30f;
  int best_nb = 1, best_cl = 0;
  const int nbs[4] = {1, 2, 4, 8}, cls[4] = {1, 2, 4, 8};
  for (int a = 0; a < 4; ++a) {
    if (nbs[a] > n) break;
    for (int c = 0; c < 4; ++c) {
      ce_mppi_batch* b = nullptr;
      if (batch_create_with(hs, reqs, n, stream, 0, nbs[a], cls[c], &b) != CE_MPPI_OK) continue;
      copy_state(true);
      run_branches(b, s);   // warm-up
      cudaEventRecord(ev[0], s);
      for (int r = 0; r < 3; ++r) run_branches(b, s);
      cudaEventRecord(ev[1], s);
      copy_state(false);
      float ms = 0.f;
      e = cudaEventSynchronize(ev[1]);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      free_batch(b);
      if (e != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (ms < best_ms) { best_ms = ms; best_nb = nbs[a]; best_cl = cls[c]; }
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  cudaStreamSynchronize(s);
  cudaFree(save);
  *n_branches = best_nb;
  *post_ctas = best_cl;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {best_nb, best_cl};
  return CE_MPPI_OK;
}

ce_status_t batch_create_with(ce_mppi_handle* const* hs, const ce_mppi_request* reqs, int n,
                              void* stream, int use_graph, int n_branches, int post_ctas,
                              ce_mppi_batch** out) {
  *out = nullptr;
  const int dyn = hs[0] ? hs[0]->P.dyn : -1;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL handle in batch");
    if (hs[i]->P.dyn != dyn) return fail(CE_MPPI_ERR_INVALID_ARG, "mixed dynamics in one batch");
    ce_status_t st = check_req(hs[i], &reqs[i]);
    if (st != CE_MPPI_OK) return st;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(CE_MPPI_ERR_INVALID_ARG, "a handle appears twice");
  }
  n_branches = std::min(n_branches, n);
  ce_mppi_batch* b = new (std::nothrow) ce_mppi_batch();
  if (!b) return fail(CE_MPPI_ERR_NO_MEMORY, "host allocation failed");
  b->hs.assign(hs, hs + n);
  b->stream = static_cast<cudaStream_t>(stream);
  b->dyn = dyn;
  b->post_ctas = post_ctas;
  // balance the branches by rollout work (largest instances first)
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (long long)hs[x]->P.K * hs[x]->P.T > (long long)hs[y]->P.K * hs[y]->P.T;
  });
  std::vector<std::vector<int>> members(n_branches);
  std::vector<long long> load(n_branches, 0);
  for (int i : order) {
    const int bb = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    members[bb].push_back(i);
    load[bb] += (long long)hs[i]->P.K * hs[i]->P.T;
  }
  std::vector<InstDesc> descs;
  std::vector<Req> rq;
  std::vector<int2> roll, upd;   // whole-batch tiles (stage-by-stage profile)
  b->branches.resize(n_branches);
  std::vector<std::vector<int2>> broll(n_branches), bupd(n_branches);
  for (int bb = 0; bb < n_branches; ++bb) {
    auto& br = b->branches[bb];
    br.off = (int)descs.size();
    br.n = (int)members[bb].size();
    for (int li = 0; li < br.n; ++li) {
      ce_mppi_handle* h = hs[members[bb][li]];
      unsigned long long c0 = 0;
      cudaStreamSynchronize(h->stream);
      cudaMemcpy(&c0, h->hdesc.counter, 8, cudaMemcpyDeviceToHost);
      descs.push_back(h->hdesc);
      rq.push_back(to_req(&reqs[members[bb][li]], c0));
      tiles_of(h, (int)descs.size() - 1, roll, upd);
      tiles_of(h, li, broll[bb], bupd[bb]);
      br.smem_roll = std::max(br.smem_roll, h->smem_roll);
      br.max_cells = std::max(br.max_cells, h->ncells);
      b->smem_roll = std::max(b->smem_roll, h->smem_roll);
      b->max_cells = std::max(b->max_cells, h->ncells);
    }
    br.n_roll = (int)broll[bb].size();
    br.n_upd = (int)bupd[bb].size();
  }
  b->n_roll = (int)roll.size();
  b->n_upd = (int)upd.size();
  cudaError_t e;
  bool ok = (e = cudaMalloc(&b->ddesc, sizeof(InstDesc) * n)) == cudaSuccess &&
            (e = cudaMalloc(&b->dreq, sizeof(Req) * n)) == cudaSuccess &&
            (e = cudaMalloc(&b->dtiles_roll, sizeof(int2) * roll.size())) == cudaSuccess &&
            (e = cudaMalloc(&b->dtiles_upd, sizeof(int2) * upd.size())) == cudaSuccess;
  for (int bb = 0; ok && bb < n_branches; ++bb) {
    auto& br = b->branches[bb];
    ok = (e = cudaMalloc(&br.dtiles_roll, sizeof(int2) * broll[bb].size())) == cudaSuccess &&
         (e = cudaMalloc(&br.dtiles_upd, sizeof(int2) * bupd[bb].size())) == cudaSuccess &&
         (e = cudaMemcpy(br.dtiles_roll, broll[bb].data(), sizeof(int2) * broll[bb].size(),
                         cudaMemcpyHostToDevice)) == cudaSuccess &&
         (e = cudaMemcpy(br.dtiles_upd, bupd[bb].data(), sizeof(int2) * bupd[bb].size(),
                         cudaMemcpyHostToDevice)) == cudaSuccess;
    if (ok && n_branches > 1)
      ok = (e = cudaStreamCreateWithFlags(&br.stream, cudaStreamNonBlocking)) == cudaSuccess &&
           (e = cudaEventCreateWithFlags(&br.done, cudaEventDisableTiming)) == cudaSuccess;
  }
  if (ok && n_branches > 1)
    ok = (e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) == cudaSuccess;
  if (ok)
    ok = (e = cudaMemcpy(b->ddesc, descs.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice)) == cudaSuccess &&
         (e = cudaMemcpy(b->dreq, rq.data(), sizeof(Req) * n, cudaMemcpyHostToDevice)) == cudaSuccess &&
         (e = cudaMemcpy(b->dtiles_roll, roll.data(), sizeof(int2) * roll.size(), cudaMemcpyHostToDevice)) == cudaSuccess &&
         (e = cudaMemcpy(b->dtiles_upd, upd.data(), sizeof(int2) * upd.size(), cudaMemcpyHostToDevice)) == cudaSuccess;
  if (!ok) {
    free_batch(b);
    return cuda_fail(e, "batch set-up");
  }
  if (use_graph) {
    // capture on a private non-blocking stream (the legacy default stream
    // cannot be captured); the graph is launched on the batch's stream.
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) {
      free_batch(b);
      return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      cudaStreamDestroy(cap);
      free_batch(b);
      return cuda_fail(e, "cudaStreamBeginCapture");
    }
    run_branches(b, cap);
    e = cudaStreamEndCapture(cap, &b->graph);
    cudaStreamDestroy(cap);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
      free_batch(b);
      return cuda_fail(e, "graph capture");
    }
  }
  *out = b;
  return CE_MPPI_OK;
}

}  // namespace

extern "C" {

ce_status_t ce_mppi_batch_run(ce_mppi_batch* b) {
  if (!b) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL batch");
  if (b->exec) {
    CE_CUDA(cudaGraphLaunch(b->exec, b->stream));
    return CE_MPPI_OK;
  }
  run_branches(b, b->stream);
  CE_CUDA(cudaGetLastError());
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_batch_run_part(ce_mppi_batch* b, int part, void* stream) {
  return ce_mppi_batch_run_part_ev(b, part, stream, nullptr);
}

ce_status_t ce_mppi_batch_run_part_ev(ce_mppi_batch* b, int part, void* stream, void* started) {
  if (!b) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL batch");
  if (part < 0 || part > 3) return fail(CE_MPPI_ERR_INVALID_ARG, "part must be 0, 1, 2 or 3");
  if (part != 1 && started) return fail(CE_MPPI_ERR_INVALID_ARG, "started event is for part 1");
  cudaEvent_t ev = static_cast<cudaEvent_t>(started);
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : b->stream;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.D = b->ddesc;
  a.R = b->dreq;
  a.n_inst = (int)b->hs.size();
  a.n_conc = a.n_inst;
  a.post_ctas = b->post_ctas;
  if (part != 1) {
    if (part != 3) launch_tracks(a, s, part == 2);
    if (part != 2) {
      a.tiles = b->dtiles_roll;
      a.n_tiles = b->n_roll;
      launch_rollout(b->dyn, a, b->smem_roll, s, part == 0);
    }
  } else {
    const bool fused = launch_post(a, b->max_cells, s, ev);   // (as in a whole replan's chain)
    if (!fused) {
      launch_prune(a, s, ev);
      launch_dbscan(a, b->max_cells, s);
      launch_select(a, s);
    }
    a.tiles = b->dtiles_upd;
    a.n_tiles = b->n_upd;
    launch_update(a, s);
  }
  CE_CUDA(cudaGetLastError());
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_batch_profile(ce_mppi_batch* b, float* stage_ms) {
  if (!b || !stage_ms) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  cudaEvent_t ev[7];
  for (int i = 0; i < 7; ++i) CE_CUDA(cudaEventCreate(&ev[i]));
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.D = b->ddesc;
  a.R = b->dreq;
  a.n_inst = (int)b->hs.size();
  a.n_conc = a.n_inst;
  cudaStream_t s = b->stream;
  cudaEventRecord(ev[0], s);
  launch_tracks(a, s);
  cudaEventRecord(ev[1], s);
  a.tiles = b->dtiles_roll;
  a.n_tiles = b->n_roll;
  launch_rollout(b->dyn, a, b->smem_roll, s, true);
  cudaEventRecord(ev[2], s);
  launch_prune(a, s);
  cudaEventRecord(ev[3], s);
  launch_dbscan(a, b->max_cells, s);
  cudaEventRecord(ev[4], s);
  launch_select(a, s);
  cudaEventRecord(ev[5], s);
  a.tiles = b->dtiles_upd;
  a.n_tiles = b->n_upd;
  launch_update(a, s);
  cudaEventRecord(ev[6], s);
  cudaError_t e = cudaEventSynchronize(ev[6]);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&stage_ms[i], ev[i], ev[i + 1]);
  for (int i = 0; i < 7; ++i) cudaEventDestroy(ev[i]);
  if (e != cudaSuccess) return cuda_fail(e, "batch profile");
  CE_CUDA(cudaGetLastError());
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_batch_destroy(ce_mppi_batch* b) {
  if (!b) return CE_MPPI_OK;
  cudaStreamSynchronize(b->stream);
  for (auto& br : b->branches)
    if (br.stream) cudaStreamSynchronize(br.stream);
  free_batch(b);
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_batch_create_host(ce_mppi_handle* const* hs, const int* n_obs, int n,
                                      void* stream, int use_graph, int n_branches,
                                      ce_mppi_batch** out) {
  if (!out) return fail(CE_MPPI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!hs || !n_obs || n < 1) return fail(CE_MPPI_ERR_INVALID_ARG, "empty batch");
  // staging layout per instance: inputs x0 [n], obs_hist [H][n_obs][p],
  // obs_radius [n_obs]; outputs u_out [T][m], x_next [n], diag (16-byte aligned)
  std::vector<size_t> in_off(n), out_off(n);
  size_t in_b = 0, out_b = 0;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL handle in batch");
    const ce_mppi_handle* h = hs[i];
    if (n_obs[i] < 0 || n_obs[i] > h->P.n_obs_max)
      return fail(CE_MPPI_ERR_INVALID_ARG, "n_obs must be in [0, n_obs_max]");
    in_off[i] = in_b;
    in_b += align_up(4 * ((size_t)h->n + (size_t)h->P.hist_len * n_obs[i] * h->p + n_obs[i]), 16);
    out_off[i] = out_b;
    out_b += align_up(4 * ((size_t)h->P.T * h->m + h->n), 16) + align_up(sizeof(ce_mppi_diag), 16);
  }
  unsigned char* d_stage = nullptr;
  unsigned char* h_stage = nullptr;
  cudaError_t e = cudaMalloc(&d_stage, in_b + out_b);
  if (e != cudaSuccess) return fail(CE_MPPI_ERR_NO_MEMORY, "device allocation failed");
  e = cudaHostAlloc((void**)&h_stage, in_b + out_b, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    cudaFree(d_stage);
    return fail(CE_MPPI_ERR_NO_MEMORY, "pinned host allocation failed");
  }
  std::memset(h_stage, 0, in_b + out_b);
  std::vector<ce_mppi_request> reqs(n);
  for (int i = 0; i < n; ++i) {
    const ce_mppi_handle* h = hs[i];
    float* in = reinterpret_cast<float*>(d_stage + in_off[i]);
    float* o = reinterpret_cast<float*>(d_stage + in_b + out_off[i]);
    std::memset(&reqs[i], 0, sizeof(ce_mppi_request));
    reqs[i].x0 = in;
    reqs[i].obs_hist = in + h->n;
    reqs[i].obs_radius = in + h->n + (size_t)h->P.hist_len * n_obs[i] * h->p;
    reqs[i].n_obs = n_obs[i];
    reqs[i].u_out = o;
    reqs[i].x_next = o + (size_t)h->P.T * h->m;
    reqs[i].diag = reinterpret_cast<ce_mppi_diag*>(
        d_stage + in_b + out_off[i] + align_up(4 * ((size_t)h->P.T * h->m + h->n), 16));
  }
  // (the staging holds valid zeros: the tuner's trial replans read them)
  if ((e = cudaMemset(d_stage, 0, in_b + out_b)) != cudaSuccess) {
    cudaFree(d_stage);
    cudaFreeHost(h_stage);
    return cuda_fail(e, "staging set-up");
  }
  ce_status_t st = ce_mppi_batch_create(hs, reqs.data(), n, stream, use_graph, n_branches, out);
  if (st != CE_MPPI_OK) {
    cudaFree(d_stage);
    cudaFreeHost(h_stage);
    return st;
  }
  ce_mppi_batch* b = *out;
  b->d_stage = d_stage;
  b->h_stage = h_stage;
  b->in_bytes = in_b;
  b->out_bytes = out_b;
  b->n_obs.assign(n_obs, n_obs + n);
  b->in_off = in_off;
  b->out_off = out_off;
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_batch_run_host(ce_mppi_batch* b, const float* x0s, const float* hists,
                                   const float* radii, float* u_outs, float* x_nexts,
                                   ce_mppi_diag* diags) {
  if (!b || !b->h_stage) return fail(CE_MPPI_ERR_INVALID_ARG, "not a host-buffer batch");
  const int n = (int)b->hs.size();
  if (!x0s || !u_outs) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  // inputs: checked (as ce_mppi_check_inputs), then packed into the pinned block
  size_t ox = 0, oh = 0, orr = 0;
  for (int i = 0; i < n; ++i) {
    const ce_mppi_handle* h = b->hs[i];
    const int no = b->n_obs[i];
    const size_t nh = (size_t)h->P.hist_len * no * h->p;
    ce_status_t st = check_host_inputs(h, x0s + ox, no > 0 ? hists + oh : nullptr,
                                       no > 0 ? radii + orr : nullptr, no);
    if (st != CE_MPPI_OK) return st;
    float* in = reinterpret_cast<float*>(b->h_stage + b->in_off[i]);
    std::memcpy(in, x0s + ox, 4 * (size_t)h->n);
    if (no > 0) {
      std::memcpy(in + h->n, hists + oh, 4 * nh);
      std::memcpy(in + h->n + nh, radii + orr, 4 * (size_t)no);
    }
    ox += h->n;
    oh += nh;
    orr += no;
  }
  // one copy in, the batch's launches (or graph), one copy out
  CE_CUDA(cudaMemcpyAsync(b->d_stage, b->h_stage, b->in_bytes, cudaMemcpyHostToDevice, b->stream));
  ce_status_t st = ce_mppi_batch_run(b);
  if (st != CE_MPPI_OK) return st;
  CE_CUDA(cudaMemcpyAsync(b->h_stage + b->in_bytes, b->d_stage + b->in_bytes, b->out_bytes,
                          cudaMemcpyDeviceToHost, b->stream));
  CE_CUDA(cudaStreamSynchronize(b->stream));
  size_t ou = 0, on = 0;
  int bad = 0;
  for (int i = 0; i < n; ++i) {
    const ce_mppi_handle* h = b->hs[i];
    const size_t TM = (size_t)h->P.T * h->m;
    const float* o = reinterpret_cast<const float*>(b->h_stage + b->in_bytes + b->out_off[i]);
    std::memcpy(u_outs + ou, o, 4 * TM);
    if (x_nexts) std::memcpy(x_nexts + on, o + TM, 4 * (size_t)h->n);
    ce_mppi_diag dg;
    std::memcpy(&dg, b->h_stage + b->in_bytes + b->out_off[i] + align_up(4 * (TM + h->n), 16),
                sizeof(dg));
    if (diags) diags[i] = dg;
    if (dg.status != 0 && !bad) bad = dg.status;
    ou += TM;
    on += h->n;
  }
  if (bad == CE_MPPI_ERR_TIMEOUT) return fail(CE_MPPI_ERR_TIMEOUT, "device-side bounded wait gave up");
  if (bad) return fail((ce_status_t)bad, "input refused on the device");
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_peek(ce_mppi_handle* h, int which, void* dst, size_t bytes) {
  if (!h || !dst) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  const InstDesc& d = h->hdesc;
  const size_t K = h->P.K, Kp = h->Kp, p = h->p, TM = (size_t)h->P.T * h->m;
  CE_CUDA(cudaStreamSynchronize(h->stream));
  auto want = [&](size_t b) -> ce_status_t {
    return bytes == b ? CE_MPPI_OK : fail(CE_MPPI_ERR_INVALID_ARG, "peek: wrong byte count");
  };
  const void* src1 = nullptr;
  switch (which) {
    case CE_BUF_S: src1 = d.S; break;
    case CE_BUF_HIT: src1 = d.hit; break;
    case CE_BUF_IDXV: src1 = d.idxV; break;
    case CE_BUF_IDXC: src1 = d.idxC; break;
    case CE_BUF_LABEL: src1 = d.label; break;
    case CE_BUF_W: src1 = d.w_k; break;
    case CE_BUF_HITJ: src1 = d.hitj; break;
    default: break;
  }
  if (src1) {
    if (want(4 * K) != CE_MPPI_OK) return CE_MPPI_ERR_INVALID_ARG;
    CE_CUDA(cudaMemcpy(dst, src1, 4 * K, cudaMemcpyDeviceToHost));
    if (which == CE_BUF_W) {   // the device keeps exp(-(S - S_min)/lambda) and 1/Z
      float iz = 0.f;
      CE_CUDA(cudaMemcpy(&iz, &d.ctl->invZ, sizeof(float), cudaMemcpyDeviceToHost));
      float* wv = static_cast<float*>(dst);
      for (size_t k = 0; k < K; ++k) wv[k] *= iz;
    }
    return CE_MPPI_OK;
  }
  if (which == CE_BUF_PN || which == CE_BUF_Z || which == CE_BUF_G) {
    if (want(4 * p * K) != CE_MPPI_OK) return CE_MPPI_ERR_INVALID_ARG;
    const float* s = which == CE_BUF_PN ? d.pN : (which == CE_BUF_Z ? d.z : d.g);
    CE_CUDA(cudaMemcpy2D(dst, 4 * K, s, 4 * Kp, 4 * K, p, cudaMemcpyDeviceToHost));
    return CE_MPPI_OK;
  }
  if (which == CE_BUF_DBCYC) {
    if (want(sizeof(long long) * 16) != CE_MPPI_OK) return CE_MPPI_ERR_INVALID_ARG;
    CE_CUDA(cudaMemcpy(dst, d.ctl->dbcyc, sizeof(long long) * 16, cudaMemcpyDeviceToHost));
    return CE_MPPI_OK;
  }
  if (which == CE_BUF_EPS) {
    if (!d.eps) return fail(CE_MPPI_ERR_INVALID_ARG, "peek: eps' is not stored (noise_regen)");
    if (want(4 * K * TM) != CE_MPPI_OK) return CE_MPPI_ERR_INVALID_ARG;
    float* o = static_cast<float*>(dst);
    if (is_arm(h->P.dyn)) {
      CE_CUDA(cudaMemcpy2D(o, 4 * TM, d.eps, 4 * (size_t)h->TMp, 4 * TM, K, cudaMemcpyDeviceToHost));
    } else {
      std::vector<float> tmp(TM * K);
      CE_CUDA(cudaMemcpy2D(tmp.data(), 4 * K, d.eps, 4 * Kp, 4 * K, TM, cudaMemcpyDeviceToHost));
      for (size_t c = 0; c < TM; ++c)
        for (size_t k = 0; k < K; ++k) o[k * TM + c] = tmp[c * K + k];
    }
    return CE_MPPI_OK;
  }
  return fail(CE_MPPI_ERR_INVALID_ARG, "peek: unknown buffer");
}

ce_status_t ce_mppi_philox_dev(unsigned long long seed, unsigned long long counter, int K, int nblk,
                               unsigned int* out, void* stream) {
  if (K < 0 || nblk < 0 || (!out && K * nblk > 0)) return fail(CE_MPPI_ERR_INVALID_ARG, "bad sizes");
  if ((long long)K * nblk == 0) return CE_MPPI_OK;
  launch_philox(seed, counter, K, nblk, out, static_cast<cudaStream_t>(stream));
  CE_CUDA(cudaGetLastError());
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_normals_dev(unsigned long long seed, unsigned long long counter, int K, int n,
                                float* out, void* stream) {
  if (K < 0 || n < 0 || (!out && K * n > 0)) return fail(CE_MPPI_ERR_INVALID_ARG, "bad sizes");
  if ((long long)K * n == 0) return CE_MPPI_OK;
  launch_normals(seed, counter, K, n, out, static_cast<cudaStream_t>(stream));
  CE_CUDA(cudaGetLastError());
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_neg2ln_dev(float* out, void* stream) {
  if (!out) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL output");
  launch_neg2ln(out, static_cast<cudaStream_t>(stream));
  CE_CUDA(cudaGetLastError());
  return CE_MPPI_OK;
}

size_t ce_mppi_dbscan_workspace_bytes(int n) { return n < 0 ? 0 : dbscan_ws_bytes(n); }

ce_status_t ce_mppi_dbscan_dev(const float* z, int n, int ld, int p, float eps, int min_pts,
                               int* labels, int* n_clusters, void* ws, size_t ws_bytes,
                               void* stream) {
  if (p != 2 && p != 3) return fail(CE_MPPI_ERR_INVALID_ARG, "p must be 2 or 3");
  if (n < 0 || ld < n || min_pts < 1) return fail(CE_MPPI_ERR_INVALID_ARG, "bad sizes");
  if (!(eps > 0.02f) || !(eps <= 2.0f)) return fail(CE_MPPI_ERR_INVALID_ARG, "eps must be in (0.02, 2]");
  if (!n_clusters || (n > 0 && (!z || !labels || !ws)))
    return fail(CE_MPPI_ERR_INVALID_ARG, "NULL pointer");
  if (ws_bytes < dbscan_ws_bytes(n)) return fail(CE_MPPI_ERR_INVALID_ARG, "workspace too small");
  float ci;
  int G, R, nc;
  dbscan_grid(eps, p, &ci, &G, &R, &nc);
  if (nc > kMaxCells) return fail(CE_MPPI_ERR_INVALID_ARG, "eps too small for the DBSCAN grid");
  cem::ensure_configured();
  launch_dbscan_standalone(z, n, ld, p, eps_squared(eps), ci, G, R, min_pts, labels, n_clusters,
                           ws, static_cast<cudaStream_t>(stream));
  CE_CUDA(cudaGetLastError());
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_arm_fk(const double* q, double* O, double* R) {
  if (!q || !O || !R) return fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  const double d[6] = {0.1625, 0.0, 0.0, 0.1333, 0.0997, 0.0996};
  const double a[6] = {0.0, -0.425, -0.3922, 0.0, 0.0, 0.0};
  const double ca[6] = {0, 1, 1, 0, 0, 1}, sa[6] = {1, 0, 0, 1, -1, 0};
  double T[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
  O[0] = O[1] = O[2] = 0.0;
  for (int i = 0; i < 6; ++i) {
    const double ct = std::cos(q[i]), st = std::sin(q[i]);
    const double A[12] = {ct, -st * ca[i], st * sa[i], a[i] * ct,
                          st, ct * ca[i], -ct * sa[i], a[i] * st,
                          0, sa[i], ca[i], d[i]};
    double N[12];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 4; ++c) {
        double s = (c == 3) ? T[r * 4 + 3] : 0.0;
        for (int e = 0; e < 3; ++e) s += T[r * 4 + e] * A[e * 4 + c];
        N[r * 4 + c] = s;
      }
    std::memcpy(T, N, sizeof(T));
    for (int r = 0; r < 3; ++r) O[(i + 1) * 3 + r] = T[r * 4 + 3];
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) R[r * 3 + c] = T[r * 4 + c];
  return CE_MPPI_OK;
}

}  // extern "C"
