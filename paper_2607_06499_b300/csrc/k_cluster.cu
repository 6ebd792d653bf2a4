// k_cluster.cu -- pruning, reference point and features, grid-binned DBSCAN,
// cluster statistics and selection, and the softmin-weighted update of the
// CE-MPPI replan (Algorithm 1 after [Rollouts]).
//
// Every reduction here is deterministic: float sums run in an order fixed by
// K alone (thread t takes elements t, t + blockDim, ...; fixed shuffle trees),
// and per-cluster sums use exact int64 fixed-point atomics, so a replan gives
// the same bits alone and inside any batch.
#include <algorithm>
#include <cooperative_groups.h>

#include "ce_mppi_internal.cuh"

namespace cg = cooperative_groups;

namespace cem {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Block-wide exclusive scan of one flag per thread; returns the exclusive
// prefix of this thread and writes the block total to *total.
__device__ __forceinline__ int block_scan_flag(bool f, int* wsum, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned b = __ballot_sync(FULL, f);
  if (lane == 0) wsum[wid] = __popc(b);
  __syncthreads();
  if (wid == 0) {
    const int v = lane < nw ? wsum[lane] : 0;
    int s = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) wsum[lane] = s - v;
    if (lane == 31) wsum[32] = s;
  }
  __syncthreads();
  const int r = wsum[wid] + __popc(b & ((1u << lane) - 1u));
  *total = wsum[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void task_pos0(const InstDesc& d, const float* x0, float* p0) {
  if (is_arm(d.dyn)) {
    float q[6], O[7][3], R[9];
    for (int i = 0; i < 6; ++i) q[i] = x0[i];
    arm_fk(q, O, R);
    p0[0] = O[6][0]; p0[1] = O[6][1]; p0[2] = O[6][2];
  } else {
    p0[0] = x0[0]; p0[1] = x0[1]; p0[2] = 0.0f;
  }
}

}  // namespace

// ========================================================================= prune
// Eq. 9-10 (stable ballot/prefix-sum compaction of V and C_col), the closest
// hit obstacle o* and the reference point pbar (Eq. 11), the features z
// (Eq. 12-13) and g (Eq. 15) of V, and the velocity estimate of o* (Eq. 17).
// One thread-block cluster of CL CTAs per instance (CL = 1 .. 8, chosen at
// launch), CTAs independent of each other: the rollout kernel has left, per
// group of rollouts, the sizes of V and C_col and the extremes of S, and per
// obstacle hit first, the count and the exact fixed-point sums of p(x_T).  So
// every CTA finds the instance's totals, its warps' list offsets, o* and pbar
// from those records, then reads its warps' contiguous rollout ranges once
// (coalesced) and writes V, C_col, S in V order and the features.
__device__ __forceinline__ void prune_stage(const KArgs& a, bool fused) {
  (void)fused;
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int inst = blockIdx.x / CL;
  const InstDesc& d = desc_of(a, inst);
  const Req r = req_of(a, inst);
  Ctl* ctl = d.ctl;
  __shared__ unsigned long long best;
  __shared__ float p0s[3];
  __shared__ int wv[32], wc[32];            // counts of each warp's range
  __shared__ float wred[32][3];             // per-warp extremes of S
  __shared__ int wlow[32][4];               // per-warp totals: V, C_col, V and C_col below rank
  __shared__ long long wsum4[32][4];        // per-warp sums for pbar over all of C_col
  __shared__ float tv[8];
  const int K = d.K, Kp = d.Kp, p = d.p, n_obs = r.n_obs, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int gsz = d.gsz, ng = (K + gsz - 1) / gsz;
  if (tid == 0) {
    best = ~0ull;
    task_pos0(d, r.x0, p0s);
  }
  // warp ranges: contiguous, multiples of 32 rollouts (aligned to the groups)
  const int L = (((K + CL * nw - 1) / (CL * nw)) + 31) & ~31;
  const int beg = min(K, (rank * nw + wid) * L), end = min(K, beg + L);
  const int g_rank = min(ng, rank * nw * L / gsz);   // first group of this rank
  // ---- totals, the lower ranks' counts, the extremes of S (from the group
  //      records, every CTA alike); this warp's counts
  {
    int tvv = 0, tcc = 0, lvv = 0, lcc = 0;
    float vmax = 0.f, vmin = INFINITY, amin = INFINITY;
    int mvv = 0, mcc = 0;
    const int gb = beg / gsz, ge = (end + gsz - 1) / gsz;
    {
      // (the first records of both loops below are loaded together)
      const int gi = tid, gj = gb + lane;
      int2 c0 = make_int2(0, 0), c1 = make_int2(0, 0);
      float4 e0 = make_float4(0.f, INFINITY, INFINITY, 0.f);
      if (gi < ng) { c0 = __ldcg(d.gcnt + gi); e0 = __ldcg(d.gS + gi); }
      if (gj < ge) c1 = __ldcg(d.gcnt + gj);
      tvv += c0.x;
      tcc += c0.y;
      if (gi < g_rank) { lvv += c0.x; lcc += c0.y; }
      vmax = fmaxf(vmax, e0.x);
      vmin = fminf(vmin, e0.y);
      amin = fminf(amin, e0.z);
      mvv += c1.x;
      mcc += c1.y;
    }
    for (int gi = tid + blockDim.x; gi < ng; gi += blockDim.x) {
      const int2 c = __ldcg(d.gcnt + gi);
      const float4 e = __ldcg(d.gS + gi);
      tvv += c.x;
      tcc += c.y;
      if (gi < g_rank) { lvv += c.x; lcc += c.y; }
      vmax = fmaxf(vmax, e.x);
      vmin = fminf(vmin, e.y);
      amin = fminf(amin, e.z);
    }
    for (int gi = gb + 32 + lane; gi < ge; gi += 32) {
      const int2 c = __ldcg(d.gcnt + gi);
      mvv += c.x;
      mcc += c.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tvv += __shfl_xor_sync(FULL, tvv, o);
      tcc += __shfl_xor_sync(FULL, tcc, o);
      lvv += __shfl_xor_sync(FULL, lvv, o);
      lcc += __shfl_xor_sync(FULL, lcc, o);
      mvv += __shfl_xor_sync(FULL, mvv, o);
      mcc += __shfl_xor_sync(FULL, mcc, o);
      vmax = fmaxf(vmax, __shfl_xor_sync(FULL, vmax, o));
      vmin = fminf(vmin, __shfl_xor_sync(FULL, vmin, o));
      amin = fminf(amin, __shfl_xor_sync(FULL, amin, o));
    }
    if (lane == 0) {
      wlow[wid][0] = tvv; wlow[wid][1] = tcc; wlow[wid][2] = lvv; wlow[wid][3] = lcc;
      wv[wid] = mvv; wc[wid] = mcc;
      wred[wid][0] = vmax; wred[wid][1] = vmin; wred[wid][2] = amin;
    }
  }
  // ---- o*: least clearance |p(x_0) - o_t| - r_o among the obstacles some
  //      rollout hit first (count > 0); ties to the lowest index
  __syncthreads();   // (p0s)
  {
    const float* hn = hist_of(r, d) + (size_t)(d.H - 1) * n_obs * p;   // newest observation
    for (int o = tid; o < n_obs; o += blockDim.x) {
      // (count, centre and radius loaded together)
      const long long cnt = __ldcg(d.osum + 4 * (size_t)o);
      const float ox = hn[o * p], oy = hn[o * p + 1], oz = p == 3 ? hn[o * p + 2] : 0.f;
      const float orad = r.obs_radius[o];
      if (cnt == 0) continue;
      const float dx = p0s[0] - ox, dy = p0s[1] - oy;
      const float dz = p == 3 ? p0s[2] - oz : 0.f;
      const float clear = sqrtf(dx * dx + dy * dy + dz * dz) - orad;
      atomicMin(&best, ((unsigned long long)float_key(clear) << 32) | (unsigned)o);
    }
  }
  __syncthreads();
  if (wid == 0) {
    int t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] = lane < nw ? wlow[lane][q] : 0;
    float e0 = lane < nw ? wred[lane][0] : 0.f, e1 = lane < nw ? wred[lane][1] : INFINITY,
          e2 = lane < nw ? wred[lane][2] : INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) t[q] += __shfl_xor_sync(FULL, t[q], o);
      e0 = fmaxf(e0, __shfl_xor_sync(FULL, e0, o));
      e1 = fminf(e1, __shfl_xor_sync(FULL, e1, o));
      e2 = fminf(e2, __shfl_xor_sync(FULL, e2, o));
    }
    // exclusive scan of the warps' counts, after the lower ranks'
    const int v = lane < nw ? wv[lane] : 0, c = lane < nw ? wc[lane] : 0;
    int sv = v, sc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int yv = __shfl_up_sync(FULL, sv, o), yc = __shfl_up_sync(FULL, sc, o);
      if (lane >= o) { sv += yv; sc += yc; }
    }
    if (lane < nw) { wv[lane] = t[2] + sv - v; wc[lane] = t[3] + sc - c; }
    if (lane == 0) {
      tv[0] = e0; tv[1] = e1; tv[2] = e2;
      tv[3] = __int_as_float(t[0]);
      tv[4] = __int_as_float(t[1]);
    }
  }
  __syncthreads();
  const int nV = __float_as_int(tv[3]), nC = __float_as_int(tv[4]);
  const int o_star = nC > 0 ? (int)(best & 0xffffffffull) : -1;
  if (tid == 0 && rank == 0) {
    ctl->S_absmax_V = tv[0];
    ctl->S_min_V = tv[1];
    ctl->S_min_all = tv[2];
  }
  // the fallbacks (no clustering): the lists are still written, not the features
  const bool fallback = nC == 0 || nV == 0 || d.mppi_only;
  if (fallback && tid == 0 && rank == 0) {
    ctl->nV = nV; ctl->nC = nC; ctl->M = 0; ctl->sel = -1; ctl->o_star = -1;
    ctl->dynamic = 0;
    ctl->mode = d.mppi_only ? CE_MODE_MPPI : nC == 0 ? CE_MODE_NOCOL : CE_MODE_ALLCOL;
    for (int i = 0; i < 3; ++i) { ctl->pbar[i] = 0.f; ctl->v_obs[i] = 0.f; ctl->p0[i] = p0s[i]; }
  }
  // ---- pbar (Eq. 11): the mean p(x_T) of the colliding rollouts whose first
  //      hit is o* (ref_mode 0) or of all of them (ref_mode 1), from the exact
  //      fixed-point sums
  float pbar[3] = {0.f, 0.f, 0.f};
  if (!fallback && d.ref_mode == 0) {
    const long long* os = d.osum + 4 * (size_t)o_star;
    const float cnt = (float)__ldcg(os);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < p) pbar[c] = __ll2float_rn(__ldcg(os + 1 + c)) * kPosFixedInv / cnt;
  } else if (!fallback) {
    long long s4[4] = {0, 0, 0, 0};
    for (int o = tid; o < n_obs; o += blockDim.x)
#pragma unroll
      for (int q = 0; q < 4; ++q) s4[q] += __ldcg(d.osum + 4 * (size_t)o + q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < 4; ++q) s4[q] += __shfl_xor_sync(FULL, s4[q], o);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < 4; ++q) wsum4[wid][q] = s4[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      s4[q] = 0;
      for (int w2 = 0; w2 < nw; ++w2) s4[q] += wsum4[w2][q];   // (exact: any order)
    }
    const float cnt = (float)s4[0];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < p) pbar[c] = __ll2float_rn(s4[1 + c]) * kPosFixedInv / cnt;
  }
  // ---- the pass over the warp's rollouts: lists, S in V order, features
  const float ne = d.norm_eps;
  const unsigned lt = (1u << lane) - 1u;
  int bv = wv[wid], bc = wc[wid];
  // the first hit, cost and p(x_T) of the next 32 rollouts are loaded before
  // this step's work
  int nh = -1;
  float nSk = 0.f, npk[3] = {0.f, 0.f, 0.f};
  auto pfetch = [&](int k) {
    nh = -1;
    if (k < end) {
      nh = __ldg(d.hit + k);
      nSk = __ldg(d.S + k);
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (c < p) npk[c] = __ldg(d.pN + (size_t)c * Kp + k);
    }
  };
  pfetch(beg + lane);
  for (int s0 = beg; s0 < end; s0 += 32) {
    const int k = s0 + lane;
    const int h = nh;
    const float Sk = nSk, pk3[3] = {npk[0], npk[1], npk[2]};
    pfetch(s0 + 32 + lane);
    const bool in = k < end;
    const bool isV = in && h < 0, isC = h >= 0;
    const unsigned mv = __ballot_sync(FULL, isV), mc = __ballot_sync(FULL, isC);
    if (isV) {
      const int i = bv + __popc(mv & lt);
      d.idxV[i] = k;
      d.Sv[i] = Sk;
    }
    if (isV && !fallback) {
      const int i = bv + __popc(mv & lt);
      float dv[3] = {0.f, 0.f, 0.f}, ev[3] = {0.f, 0.f, 0.f}, nd = 0.f, nn = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (c >= p) continue;
        const float pk = pk3[c];
        dv[c] = pk - pbar[c];
        ev[c] = pk - p0s[c];
        nd += dv[c] * dv[c];
        nn += ev[c] * ev[c];
      }
      const float izd = 1.0f / (sqrtf(nd) + ne), izn = 1.0f / (sqrtf(nn) + ne);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (c >= p) continue;
        d.z[(size_t)c * Kp + i] = dv[c] * izd;
        d.g[(size_t)c * Kp + i] = ev[c] * izn;
      }
    }
    if (isC) d.idxC[bc + __popc(mc & lt)] = k;
    bv += __popc(mv);
    bc += __popc(mc);
  }
  if (tid == 0 && rank == 0 && !fallback) {
    const int H = d.H;
    const float inv = H >= 2 ? 1.0f / ((float)(H - 1) * d.obs_dt) : 0.0f;
    const float* h = hist_of(r, d);
    // the observations first, then the stores (see the selection's prefetch)
    float hn[3] = {0.f, 0.f, 0.f}, ho[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c < p) {
        hn[c] = h[((size_t)(H - 1) * n_obs + o_star) * p + c];
        ho[c] = h[(size_t)o_star * p + c];
      }
    ctl->nV = nV; ctl->nC = nC; ctl->M = 0; ctl->sel = -1; ctl->o_star = o_star;
    ctl->dynamic = 0; ctl->mode = CE_MODE_STATIC;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ctl->pbar[c] = c < p ? pbar[c] : 0.f;
      ctl->p0[c] = p0s[c];
      ctl->v_obs[c] = c < p ? (hn[c] - ho[c]) * inv : 0.f;
    }
  }
}

__global__ void __maxnreg__(64) k_prune(KArgs a) { prune_stage(a, false); }

// ========================================================================= DBSCAN
// Grid-binned DBSCAN over n points z ([p][ld], coordinates in [-1, 1]).  The
// cell side s = 0.99 eps / sqrt(p) makes any two points of one cell neighbours
// (in the FP32 predicate too), so the core points of a cell are connected and
// the union-find runs over cells: two cells join when some core pair between
// them is within eps.  Shared memory: 4 int arrays of G^p (+1) entries.
struct DbWork {
  int* labels_tmp;  // [n] list of the points of sparse cells (the labels buffer)
  int* cell;     // [n] cell id of each point
  int* sorted;   // [n] point ids in cell order
  float* zs;     // [p][ld_s] coordinates in cell order
  int ld_s;
  int* core;     // [n] core flag
  float* bbox;   // [ncells][6] core bounding box (min xyz, max xyz)
  int* ahist;    // [kAngBuckets] angle-bucket counts (zero at entry), angular method
  int* amin;     // [kAngBuckets] least core index per bucket (INT_MAX at entry)
};

// The 125 neighbour-cell offsets of a 3-D point (reach R = 2 cells), nearest
// first: by the least possible distance between points of the two cells, so
// that core counting meets min_pts early.  Entry = (dx+2) | (dy+2) << 3 |
// (dz+2) << 6.
__device__ const unsigned short kNbOrder3[125] = {
    146, 82, 138, 145, 147, 154, 210, 74, 81, 83, 90, 137, 139, 153, 155, 202, 209, 211, 218, 73,
    75, 89, 91, 201, 203, 217, 219, 18, 130, 144, 148, 162, 274, 10, 17, 19, 26, 66, 80, 84,
    98, 129, 131, 136, 140, 152, 156, 161, 163, 194, 208, 212, 226, 266, 273, 275, 282, 9, 11, 25,
    27, 65, 67, 72, 76, 88, 92, 97, 99, 193, 195, 200, 204, 216, 220, 225, 227, 265, 267, 281,
    283, 2, 16, 20, 34, 128, 132, 160, 164, 258, 272, 276, 290, 1, 3, 8, 12, 24, 28, 33,
    35, 64, 68, 96, 100, 192, 196, 224, 228, 257, 259, 264, 268, 280, 284, 289, 291, 0, 4, 32,
    36, 256, 260, 288, 292};

template <int p>
__device__ __forceinline__ bool nb_pred_t(const float* za, const float* zb, float eps2) {
  const float dx = __fsub_rn(za[0], zb[0]);
  float s = __fmul_rn(dx, dx);
  const float dy = __fsub_rn(za[1], zb[1]);
  s = __fadd_rn(s, __fmul_rn(dy, dy));
  if (p == 3) {
    const float dz = __fsub_rn(za[2], zb[2]);
    s = __fadd_rn(s, __fmul_rn(dz, dz));
  }
  return s <= eps2;
}

__device__ __forceinline__ int cell_coord(float v, float cell_inv, int G) {
  const float f = floorf((v + 1.0f) * cell_inv);
  return (int)fminf(fmaxf(f, 0.0f), (float)(G - 1));
}

// Union-find over cell ids with a bounded budget of parent reads: each read
// spends one unit of `budget`; once it is spent the search stops at the node
// reached (always a valid cell id) with budget 0, and the caller reports
// CE_MPPI_ERR_TIMEOUT.  (The default budget, 2^20 reads per operation, is
// never reached by a valid parent forest; a tiny one is a test hook.)
__device__ __forceinline__ int cfind(int* par, int x, int& budget) {
  while (budget > 0) {
    --budget;
    const int p = par[x];
    if (p == x) return x;
    const int gp = par[p];
    if (gp != p) atomicMin(&par[x], gp);
    x = gp;
  }
  return x;
}

// Join the sets of a and b (the larger root points to the smaller); false
// when the budget ran out first.
__device__ __forceinline__ bool cunion(int* par, int a, int b, int budget) {
  while (budget > 0) {
    a = cfind(par, a, budget);
    b = cfind(par, b, budget);
    if (budget <= 0) return false;
    if (a == b) return true;
    if (a > b) { const int t = a; a = b; b = t; }
    --budget;
    const int old = atomicCAS(&par[b], b, a);
    if (old == b) return true;
    b = old;
  }
  return false;
}

// True when a and b are known to share a root (false when the budget ran out:
// the caller then searches and unions, which reports the timeout).
__device__ __forceinline__ bool cjoined(int* par, int a, int b, int limit) {
  int budget = limit;
  const int ra = cfind(par, a, budget);
  const int rb = cfind(par, b, budget);
  return budget > 0 && ra == rb;
}

// Inverse of float_key.
__device__ __forceinline__ float key_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Squared distances from point a to the nearest and to the farthest point of
// the box given by keys bb[q] (min, stride S) and bb[3S + q] (max).
template <int p>
__device__ __forceinline__ void box_dist2(const float* za, const uint32_t* bb, int S,
                                          float* near2, float* far2) {
  float sn = 0.f, sf = 0.f;
#pragma unroll
  for (int q = 0; q < p; ++q) {
    const float lo = key_float(bb[q * S]), hi = key_float(bb[(3 + q) * S]);
    const float e = za[q] < lo ? lo - za[q] : (za[q] > hi ? za[q] - hi : 0.f);
    const float f = fmaxf(fabsf(za[q] - lo), fabsf(za[q] - hi));
    sn += e * e;
    sf += f * f;
  }
  *near2 = sn;
  *far2 = sf;
}

// Per-cell boxes (and, for core points, the smallest point id) over the
// positions [pb, pe) in cell order, merged by atomics into box / opar / omin
// (which may be another CTA's shared memory).  Warp w takes a contiguous range of
// positions, 32 at a time; a step whose lanes all fall in one cell is reduced
// across the warp and merged into a running accumulator that is written
// (shared-memory atomics) only when the cell changes, so a cell of thousands of
// points costs a handful of atomics; mixed steps reduce per cell group.
template <int p, bool CORE>
__device__ __forceinline__ void cell_boxes(int pb, int pe, const DbWork& w, const int* map,
                                           uint32_t* box, int S, int* opar, int* omin) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int L = (((pe - pb + nwarp - 1) / nwarp) + 31) & ~31;
  const int beg = min(pe, pb + wid * L), end = min(pe, beg + L);
  int run = -1;
  uint32_t rlo[3], rhi[3], rmn = 0xffffffffu;
  auto flush = [&]() {
    if (run >= 0 && lane == 0) {
#pragma unroll
      for (int q = 0; q < p; ++q) {
        atomicMin(&box[q * S + run], rlo[q]);
        atomicMax(&box[(3 + q) * S + run], rhi[q]);
      }
      if (CORE) {
        opar[run] = run;
        atomicMin(&omin[run], (int)rmn);
      }
    }
  };
  for (int s0 = beg; s0 < end; s0 += 32) {
    const int pos = s0 + lane;
    int o = -1;
    uint32_t kk[3] = {0u, 0u, 0u}, idx = 0xffffffffu;
    if (pos < end) {
      const int i = w.sorted[pos];
      const bool keep = !CORE || w.core[i];
      // from here on, sorted marks the non-core points by their complement
      if (CORE && !keep) w.sorted[pos] = ~i;
      if (keep) {
        o = map[w.cell[i]];
        idx = (uint32_t)i;
#pragma unroll
        for (int q = 0; q < p; ++q) kk[q] = float_key(w.zs[(size_t)q * w.ld_s + pos]);
      }
    }
    const int k0 = __shfl_sync(FULL, o, 0);
    if (__all_sync(FULL, o == k0)) {
      if (k0 < 0) continue;
      uint32_t lo[3], hi[3];
#pragma unroll
      for (int q = 0; q < p; ++q) {
        lo[q] = __reduce_min_sync(FULL, kk[q]);
        hi[q] = __reduce_max_sync(FULL, kk[q]);
      }
      const uint32_t mn = CORE ? __reduce_min_sync(FULL, idx) : 0u;
      if (k0 == run) {
#pragma unroll
        for (int q = 0; q < p; ++q) { rlo[q] = min(rlo[q], lo[q]); rhi[q] = max(rhi[q], hi[q]); }
        rmn = min(rmn, mn);
      } else {
        flush();
        run = k0;
#pragma unroll
        for (int q = 0; q < p; ++q) { rlo[q] = lo[q]; rhi[q] = hi[q]; }
        rmn = mn;
      }
    } else {
      flush();
      run = -1;
      const unsigned peers = __match_any_sync(FULL, o);
      if (o >= 0) {
        const int leader = __ffs(peers) - 1;
        uint32_t lo[3], hi[3];
#pragma unroll
        for (int q = 0; q < p; ++q) {
          lo[q] = __reduce_min_sync(peers, kk[q]);
          hi[q] = __reduce_max_sync(peers, kk[q]);
        }
        const uint32_t mn = CORE ? __reduce_min_sync(peers, idx) : 0u;
        if (lane == leader) {
#pragma unroll
          for (int q = 0; q < p; ++q) {
            atomicMin(&box[q * S + o], lo[q]);
            atomicMax(&box[(3 + q) * S + o], hi[q]);
          }
          if (CORE) {
            opar[o] = o;
            atomicMin(&omin[o], (int)mn);
          }
        }
      }
    }
  }
  flush();
}

// Shared memory of dbscan_block: map[nc] (cell -> occupied-cell id), lcnt[nc]
// (this CTA's points per cell), then per occupied cell: ostart[kMaxOcc + 1],
// ocell, ofill, opar, omin (kMaxOcc each), obox[6][kMaxOcc] (all points) and
// ocbox[6][kMaxOcc] (core points) as keys.
// (the per-occupied-cell tables hold min(kMaxOcc, nc) entries)
__host__ __device__ __forceinline__ int dbscan_occ_cap(int nc) { return nc < kMaxOcc ? nc : kMaxOcc; }
__host__ __device__ __forceinline__ size_t dbscan_smem_bytes(int nc) {
  return (2 * (size_t)nc + 1 + 17 * (size_t)dbscan_occ_cap(nc)) * 4;
}

// One thread-block cluster of CL CTAs (CL = 1 .. 8) per point set.  CTA r owns
// the index slice [i0, i1) and the cell-order position slice [pb, pe) of n.
// The cell-level tables (occupied cells, offsets, boxes, union-find parents,
// component minima) are computed identically in every CTA or merged into
// rank 0's shared memory (distributed shared memory atomics) and copied back;
// the union-find runs on rank 0's parents.  Phases, separated by cluster
// barriers: 1 cells and per-CTA counts; 2 occupied cells and offsets; 3
// scatter into cell order, cell boxes; 4 core flags; 5 core boxes; 6 union of
// cells; 7 components; 8 canonical ids and core labels; 9 border points.
template <int p>
__device__ __forceinline__ void dbscan_block(const float* __restrict__ z, int ld, int n,
                                             float eps2, float cell_inv, int G, int R, int min_pts,
                                             DbWork w, int* labels, int* M_out, int* status,
                                             int* smem, long long* cyc, int uf_limit) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
  const int nc = p == 3 ? G * G * G : G * G;
  const float far_ok = eps2 * 0.9999f;              // whole box within eps
  const float near_no = eps2 * 1.0001f + 1e-12f;    // whole box beyond eps
  const int S = dbscan_occ_cap(nc);
  int* map = smem;                  // [nc]
  int* lcnt = map + nc;             // [nc]
  int* ostart = lcnt + nc;          // [S + 1]
  int* ocell = ostart + S + 1;      // [S]
  int* ofill = ocell + S;           // [S] scatter cursor, later canonical id of a root
  int* opar = ofill + S;            // [S] union-find parent (-1: no core point)
  int* omin = opar + S;             // [S] smallest core id of the cell / component
  uint32_t* obox = reinterpret_cast<uint32_t*>(omin + S);   // [6][S]
  uint32_t* ocbox = obox + 6 * S;                           // [6][S]
  // rank 0's tables (this CTA's own when CL == 1)
  int* opar0 = cluster.map_shared_rank(opar, 0);
  int* omin0 = cluster.map_shared_rank(omin, 0);
  uint32_t* obox0 = cluster.map_shared_rank(obox, 0);
  uint32_t* ocbox0 = cluster.map_shared_rank(ocbox, 0);
  __shared__ int wsum[33];
  __shared__ int bad, n_occ_s, n_root_s;
  auto stamp = [&](int k) {
    if (cyc && tid == 0 && rank == 0) cyc[k] = clock64();
  };
  // slices: index [i0, i1) and cell-order position [pb, pe) (32-aligned)
  const int chunk = (((n + CL - 1) / CL) + 31) & ~31;
  const int i0 = min(n, rank * chunk), i1 = min(n, i0 + chunk);
  const int pb = i0, pe = i1;
  stamp(0);
  if (tid == 0) bad = 0;
  for (int c = tid; c < nc; c += blockDim.x) lcnt[c] = 0;
  __syncthreads();
  // 1. cell of each point of the slice; per-cell counts (one atomic per cell
  //    per warp)
  for (int b0 = i0; b0 < i1; b0 += blockDim.x) {
    const int i = b0 + tid;
    int ci = -1;
    if (i < i1) {
      int mul = 1;
      ci = 0;
      for (int c = 0; c < p; ++c) {
        const float v = z[(size_t)c * ld + i];
        if (!(v >= -1.0f && v <= 1.0f)) bad = 1;
        ci += cell_coord(v, cell_inv, G) * mul;
        mul *= G;
      }
      w.cell[i] = ci;
    }
    if (ci >= 0) atomicAdd(&lcnt[ci], 1);
  }
  cluster.sync();   // (1) every CTA's counts
  stamp(1);
  // 2. counts of the whole set per cell; occupied cells in cell order: id,
  //    offsets, reset of the per-cell summaries; map becomes cell -> occupied
  //    id.  Identical in every CTA.
  // (the ranks' flags read once, by warp 0, and shared through this CTA)
  __shared__ int anybad_s;
  if (tid < 32) {
    const int f = lane < CL ? *cluster.map_shared_rank(&bad, lane) : 0;
    const unsigned any = __reduce_or_sync(FULL, (unsigned)f);
    if (lane == 0) anybad_s = (int)any;
  }
  for (int c = tid; c < nc; c += blockDim.x) {
    int t = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < CL) t += cluster.map_shared_rank(lcnt, q)[c];
    map[c] = t;
  }
  __syncthreads();
  {
    int base = 0, off = 0;
    for (int c0 = 0; c0 < nc; c0 += blockDim.x) {
      const int c = c0 + tid;
      const int cnt = c < nc ? map[c] : 0;
      int tot;
      const int rk = block_scan_flag(cnt > 0, wsum, &tot);
      // offsets: block exclusive sum of cnt over this chunk
      int s = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, s, o);
        if (lane >= o) s += y;
      }
      if (lane == 31) wsum[wid] = s;
      __syncthreads();
      if (wid == 0) {
        const int v = lane < nwarp ? wsum[lane] : 0;
        int t = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(FULL, t, o);
          if (lane >= o) t += y;
        }
        if (lane < nwarp) wsum[lane] = t - v;
        if (lane == nwarp - 1) wsum[32] = t;
      }
      __syncthreads();
      const int excl = off + wsum[wid] + s - cnt;
      const int chunk_tot = wsum[32];
      __syncthreads();
      if (c < nc) {
        if (cnt > 0) {
          const int o = base + rk;
          if (o < S) {
            ocell[o] = c;
            ostart[o] = excl;
            ofill[o] = excl;
            opar[o] = -1;
            omin[o] = 0x7fffffff;
            for (int q = 0; q < 3; ++q) {
              obox[q * S + o] = 0xffffffffu; obox[(3 + q) * S + o] = 0u;
              ocbox[q * S + o] = 0xffffffffu; ocbox[(3 + q) * S + o] = 0u;
            }
          }
          map[c] = o;
        } else {
          map[c] = -1;
        }
      }
      base += tot;
      off += chunk_tot;
    }
    if (tid == 0) {
      n_occ_s = base;
      if (base <= S) ostart[base] = n;
    }
  }
  __syncthreads();
  const int n_occ = n_occ_s;
  const int anybad = anybad_s;   // (set before the barriers above)
  if (anybad || n_occ > S) {
    for (int i = i0 + tid; i < i1; i += blockDim.x) labels[i] = -1;
    if (tid == 0 && rank == 0) { *M_out = 0; atomicCAS(status, 0, CE_MPPI_ERR_INVALID_ARG); }
    cluster.sync();   // no CTA leaves while another reads its counts
    return;
  }
  // this CTA's write cursor in each occupied cell: after the lower ranks' points
  for (int o = tid; o < n_occ; o += blockDim.x) {
    int lo = 0;
    const int co = ocell[o];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < rank) lo += cluster.map_shared_rank(lcnt, q)[co];
    ofill[o] = ostart[o] + lo;
  }
  __syncthreads();
  stamp(2);
  // 3. scatter the slice into cell order (a shared-memory cursor atomic per
  //    point: the order inside a cell does not enter the result)
  for (int b0 = i0; b0 < i1; b0 += blockDim.x) {
    const int i = b0 + tid;
    const int o = i < i1 ? map[w.cell[i]] : -1;
    if (o >= 0) {
      const int pos = atomicAdd(&ofill[o], 1);
      w.sorted[pos] = i;
#pragma unroll
      for (int q = 0; q < p; ++q) w.zs[(size_t)q * w.ld_s + pos] = z[(size_t)q * ld + i];
    }
  }
  cluster.sync();   // (2) the cell order is complete; no more reads of lcnt
  //    bounding boxes of all points of each cell: the position slice of each
  //    CTA merged into rank 0, then copied back
  cell_boxes<p, false>(pb, pe, w, map, obox0, S, nullptr, nullptr);
  cluster.sync();   // (3)
  if (rank != 0)
    for (int e = tid; e < 6 * n_occ; e += blockDim.x) {
      const int q = e / n_occ, o = e - q * n_occ;
      obox[q * S + o] = obox0[q * S + o];
    }
  __syncthreads();
  stamp(3);
  // 4. core flags of the slice.  A cell with >= min_pts points is all core.
  //    The points of the other cells are listed, then one warp per listed
  //    point counts its neighbours cell by cell: a box entirely within eps
  //    counts whole, a box entirely beyond eps is skipped, other cells are
  //    scanned 32 points per step; the count stops at min_pts.
  {
    int n_sparse = 0;
    for (int b0 = i0; b0 < i1; b0 += blockDim.x) {
      const int i = b0 + tid;
      bool sparse = false;
      if (i < i1) {
        const int oi = map[w.cell[i]];
        const bool dense = (ostart[oi + 1] - ostart[oi]) >= min_pts;
        w.core[i] = dense ? 1 : 0;
        sparse = !dense;
      }
      int tot;
      const int rk = block_scan_flag(sparse, wsum, &tot);
      if (sparse) w.labels_tmp[i0 + n_sparse + rk] = i;
      n_sparse += tot;
    }
    __syncthreads();
    const int side = 2 * R + 1, nofs = p == 3 ? side * side * side : side * side;
    for (int is = wid; is < n_sparse; is += nwarp) {
      const int i = w.labels_tmp[i0 + is];
      const int ci = w.cell[i];
      float za[3];
#pragma unroll
      for (int c = 0; c < p; ++c) za[c] = z[(size_t)c * ld + i];
      const int cx = ci % G, cy = (ci / G) % G, cz = p == 3 ? ci / (G * G) : 0;
      int count = 0;
      // the lanes screen 32 neighbour cells at a time: boxes within eps count
      // whole, boxes beyond eps are skipped, the rest are scanned by the warp
      for (int of0 = 0; of0 < nofs && count < min_pts; of0 += 32) {
        const int of = of0 + lane;
        int whole = 0, ob = -1;
        bool scan = false;
        if (of < nofs) {
          int nx, ny, nz = 0;
          if (p == 3 && R == 2) {   // nearest cells first
            const int code = __ldg(&kNbOrder3[of]);
            nx = cx + (code & 7) - 2;
            ny = cy + ((code >> 3) & 7) - 2;
            nz = cz + (code >> 6) - 2;
          } else {
            nx = cx + of % side - R;
            ny = cy + (of / side) % side - R;
            if (p == 3) nz = cz + of / (side * side) - R;
          }
          if (nx >= 0 && ny >= 0 && nz >= 0 && nx < G && ny < G && (p != 3 || nz < G)) {
            ob = map[(nz * G + ny) * G + nx];
            if (ob >= 0) {
              float n2, f2;
              box_dist2<p>(za, obox + ob, S, &n2, &f2);
              if (f2 <= far_ok) whole = ostart[ob + 1] - ostart[ob];
              else scan = n2 <= near_no;
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) whole += __shfl_xor_sync(FULL, whole, o);
        count += whole;
        unsigned sm = __ballot_sync(FULL, scan);
        while (sm && count < min_pts) {
          const int src = __ffs(sm) - 1;
          sm &= sm - 1;
          const int obs = __shfl_sync(FULL, ob, src);
          for (int pb0 = ostart[obs]; pb0 < ostart[obs + 1] && count < min_pts; pb0 += 32) {
            const int pp = pb0 + lane;
            bool hit = false;
            if (pp < ostart[obs + 1]) {
              float zb[3];
#pragma unroll
              for (int c = 0; c < p; ++c) zb[c] = w.zs[(size_t)c * w.ld_s + pp];
              hit = nb_pred_t<p>(za, zb, eps2);
            }
            count += __popc(__ballot_sync(FULL, hit));
          }
        }
      }
      if (lane == 0) w.core[i] = count >= min_pts ? 1 : 0;
    }
  }
  cluster.sync();   // (4) core flags of every slice
  stamp(4);
  // 5. per-cell core summary (parent, smallest core id, box of the core
  //    points) merged into rank 0, then copied back
  cell_boxes<p, true>(pb, pe, w, map, ocbox0, S, opar0, omin0);
  cluster.sync();   // (5)
  if (rank != 0)
    for (int e = tid; e < 8 * n_occ; e += blockDim.x) {
      const int q = e / n_occ, o = e - q * n_occ;
      if (q < 6) ocbox[q * S + o] = ocbox0[q * S + o];
      else if (q == 6) opar[o] = opar0[o];
      else omin[o] = omin0[o];
    }
  __syncthreads();
  stamp(5);
  // 6. cell-level union over rank 0's parents, one warp per occupied cell A
  //    with core points (cells dealt round the cluster's warps): the lanes
  //    screen the neighbour offsets in parallel (B > A with core points, core
  //    boxes within eps, not yet joined) and the warp searches each surviving
  //    pair for a core pair within eps (non-core positions hold ~index).  In
  //    2-D, two rounds: touching cells (offsets within 1) first, then the
  //    cells two apart, most of which are joined by then and need no search.
  //    (Spreading one cell's candidates over several warps measured slower:
  //    the concurrent unions contend on rank 0's parents.)
  const int side = 2 * R + 1, nofs = p == 3 ? side * side * side : side * side;
  for (int ring = p == 3 ? R : 1; ring <= R; ++ring) {   // (3-D: one round)
    if (ring > 1) cluster.sync();   // the touching cells' unions are done
    for (int A = rank * nwarp + wid; A < n_occ; A += CL * nwarp) {
      if (opar[A] < 0) continue;
      const int cA = ocell[A];
      const int ax = cA % G, ay = (cA / G) % G, az = p == 3 ? cA / (G * G) : 0;
      float alo[3], ahi[3];
      for (int q = 0; q < 3; ++q) { alo[q] = key_float(ocbox[q * S + A]); ahi[q] = key_float(ocbox[(3 + q) * S + A]); }
      for (int of0 = 0; of0 < nofs; of0 += 32) {
        const int of = of0 + lane;
        bool cand = false;
        int B = -1;
        if (of < nofs) {
          const int ox = of % side - R, oy = (of / side) % side - R;
          const int oz = p == 3 ? of / (side * side) - R : 0;
          const int bx = ax + ox, by = ay + oy, bz = az + oz;
          const int cheb = max(max(abs(ox), abs(oy)), abs(oz));
          const bool in_ring = p == 3 || (ring < R ? cheb <= ring : cheb >= ring);
          if (in_ring && bx >= 0 && by >= 0 && bz >= 0 && bx < G && by < G && (p != 3 || bz < G)) {
            B = map[(bz * G + by) * G + bx];
            if (B > A && opar[B] >= 0) {
              float s2 = 0.f;
              for (int q = 0; q < p; ++q) {
                const float g1 = key_float(ocbox[q * S + B]) - ahi[q];
                const float g2 = alo[q] - key_float(ocbox[(3 + q) * S + B]);
                const float gq = fmaxf(fmaxf(g1, g2), 0.f);
                s2 += gq * gq;
              }
              cand = s2 <= near_no;
            }
          }
        }
        unsigned cm = __ballot_sync(FULL, cand);
        while (cm) {
          const int src = __ffs(cm) - 1;
          cm &= cm - 1;
          const int Bc = __shfl_sync(FULL, B, src);
          int joined = 0;
          if (lane == 0) joined = cjoined(opar0, A, Bc, uf_limit);
          if (__shfl_sync(FULL, joined, 0)) continue;   // warp-uniform decision
          // the smaller cell's core points within eps of the other cell's core
          // box are found 32 at a time (lane-parallel screening); each of them
          // in turn (warp-uniform) is tested against 32 points of the other
          // cell per step
          int X = A, Y = Bc;
          if (ostart[Bc + 1] - ostart[Bc] < ostart[A + 1] - ostart[A]) { X = Bc; Y = A; }
          bool found = false;
          for (int px0 = ostart[X]; px0 < ostart[X + 1] && !found; px0 += 32) {
            const int pxl = px0 + lane;
            bool cnd = false;
            float zx[3] = {0.f, 0.f, 0.f};
            if (pxl < ostart[X + 1] && w.sorted[pxl] >= 0) {
#pragma unroll
              for (int q = 0; q < p; ++q) zx[q] = w.zs[(size_t)q * w.ld_s + pxl];
              float n2, f2;
              box_dist2<p>(zx, ocbox + Y, S, &n2, &f2);
              cnd = n2 <= near_no;
            }
            unsigned cb = __ballot_sync(FULL, cnd);
            // a long search stops once other warps have joined the two cells
            if (cb && px0 > ostart[X]) {
              int jn = 0;
              if (lane == 0) jn = cjoined(opar0, A, Bc, uf_limit);
              if (__shfl_sync(FULL, jn, 0)) break;
            }
            while (cb && !found) {
              const int src = __ffs(cb) - 1;
              cb &= cb - 1;
              float za[3];
#pragma unroll
              for (int q = 0; q < p; ++q) za[q] = __shfl_sync(FULL, zx[q], src);
              for (int py0 = ostart[Y]; py0 < ostart[Y + 1]; py0 += 32) {
                const int py = py0 + lane;
                bool hit = false;
                if (py < ostart[Y + 1] && w.sorted[py] >= 0) {
                  float zb[3];
#pragma unroll
                  for (int q = 0; q < p; ++q) zb[q] = w.zs[(size_t)q * w.ld_s + py];
                  hit = nb_pred_t<p>(za, zb, eps2);
                }
                if (__any_sync(FULL, hit)) { found = true; break; }
              }
            }
          }
          if (found && lane == 0 && !cunion(opar0, A, Bc, uf_limit))
            atomicCAS(status, 0, CE_MPPI_ERR_TIMEOUT);
          __syncwarp();
        }
      }
    }
  }
  cluster.sync();   // (6)
  stamp(6);
  // 7. components (rank 0): compress to the root; component minimum core id;
  //    then every CTA copies parents and minima
  if (rank == 0) {
    for (int o = tid; o < n_occ; o += blockDim.x)
      if (opar[o] >= 0) {
        int budget = uf_limit;
        opar[o] = cfind(opar, o, budget);
        if (budget <= 0) atomicCAS(status, 0, CE_MPPI_ERR_TIMEOUT);
      }
    __syncthreads();
    for (int o = tid; o < n_occ; o += blockDim.x)
      if (opar[o] >= 0 && opar[o] != o) atomicMin(&omin[opar[o]], omin[o]);
  }
  cluster.sync();   // (7)
  if (rank != 0)
    for (int e = tid; e < 2 * n_occ; e += blockDim.x) {
      if (e < n_occ) opar[e] = opar0[e];
      else omin[e - n_occ] = omin0[e - n_occ];
    }
  __syncthreads();
  // 8. canonical ids: a component's id is the rank of its smallest core index
  //    among the components' (computed identically in every CTA from the
  //    roots), then the labels of the slice's core points and the list of its
  //    other points (into cell: a chunk only overwrites entries already read)
  {
    if (tid == 0) n_root_s = 0;
    __syncthreads();
    for (int o = tid; o < n_occ; o += blockDim.x)
      if (opar[o] == o) ocell[atomicAdd(&n_root_s, 1)] = o;   // ocell is free now
    __syncthreads();
    const int nr = n_root_s;
    for (int t = tid; t < nr; t += blockDim.x) {
      const int ro = ocell[t], key = omin[ro];
      int id = 0;
      for (int u = 0; u < nr; ++u) id += omin[ocell[u]] < key;
      ofill[ro] = id;
    }
    __syncthreads();
    int n_border = 0;
    for (int b0 = i0; b0 < i1; b0 += blockDim.x) {
      const int i = b0 + tid;
      const bool valid = i < i1;
      const bool isc = valid && w.core[i], isb = valid && !w.core[i];
      if (isc) labels[i] = ofill[opar[map[w.cell[i]]]];
      const int rk_tot = __syncthreads_count(isb);   // (also orders the cell reads first)
      const unsigned bb = __ballot_sync(FULL, isb);
      if (lane == 0) wsum[wid] = __popc(bb);
      __syncthreads();
      if (wid == 0) {
        const int v = lane < nwarp ? wsum[lane] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(FULL, x, o);
          if (lane >= o) x += y;
        }
        wsum[lane] = x - v;
      }
      __syncthreads();
      if (isb) w.cell[i0 + n_border + wsum[wid] + __popc(bb & ((1u << lane) - 1u))] = i;
      n_border += rk_tot;
      __syncthreads();
    }
    if (tid == 0) wsum[32] = n_border;
    if (tid == 0 && rank == 0) *M_out = nr;
  }
  cluster.sync();   // (8) core labels of every slice; no distributed shared memory after
  stamp(7);
  // 9. the other points: one warp per point finds its lowest-index core
  //    neighbour among the core points of the cells within reach.  The lanes
  //    screen the neighbour cells (core box within eps); the candidates are
  //    visited in ascending order of a lower bound of their smallest core id
  //    (the cell's own, or its component's for a root cell), and the visit
  //    stops once that bound reaches the best id found.  No core neighbour:
  //    noise.
  const int n_border = wsum[32];
  for (int ib = wid; ib < n_border; ib += nwarp) {
    const int a = w.cell[i0 + ib];
    float za[3];
    for (int q = 0; q < p; ++q) za[q] = z[(size_t)q * ld + a];
    int cc[3];
    for (int q = 0; q < p; ++q) cc[q] = cell_coord(za[q], cell_inv, G);
    int best = 0x7fffffff;
    for (int of0 = 0; of0 < nofs; of0 += 32) {
      const int of = of0 + lane;
      int ob = -1, lb = 0x7fffffff;
      if (of < nofs) {
        const int bx = cc[0] + of % side - R, by = cc[1] + (of / side) % side - R;
        const int bz = p == 3 ? cc[2] + of / (side * side) - R : 0;
        if (bx >= 0 && by >= 0 && bz >= 0 && bx < G && by < G && (p != 3 || bz < G)) {
          ob = map[(bz * G + by) * G + bx];
          if (ob >= 0 && opar[ob] >= 0) {
            float n2, f2;
            box_dist2<p>(za, ocbox + ob, S, &n2, &f2);
            if (n2 <= near_no) lb = omin[ob];
          }
        }
      }
      for (int it = 0; it < 32; ++it) {
        // candidate with the smallest bound (ties: lowest lane)
        const int mlb = __reduce_min_sync(FULL, lb);
        if (mlb >= best) break;
        const int src = __ffs(__ballot_sync(FULL, lb == mlb)) - 1;
        const int obs = __shfl_sync(FULL, ob, src);
        if (lane == src) lb = 0x7fffffff;
        const int e = ostart[obs + 1];
        for (int pb0 = ostart[obs]; pb0 < e; pb0 += 32) {
          const int pp = pb0 + lane;
          int cand = 0x7fffffff;
          if (pp < e) {
            const int sid = w.sorted[pp];
            if (sid >= 0 && sid < best) {
              float zb[3];
#pragma unroll
              for (int q = 0; q < p; ++q) zb[q] = w.zs[(size_t)q * w.ld_s + pp];
              if (nb_pred_t<p>(za, zb, eps2)) cand = sid;
            }
          }
          best = min(best, __reduce_min_sync(FULL, cand));
        }
      }
    }
    if (lane == 0) labels[a] = best == 0x7fffffff ? -1 : labels[best];
  }
  stamp(8);
}

// ========================================================================= angular DBSCAN
// For p = 2 the features z = d / (|d| + eps_n) of Eq. 13 lie on or just inside
// the unit circle, so DBSCAN can work on their angles.  A point's angle (FP32
// atan2) puts it in one of kAngBuckets equal buckets around the circle.  With
// r_lo <= |z| <= r_hi over the set, two points at true angle difference phi
// have squared distance (r_a - r_b)^2 + 4 r_a r_b sin^2(phi/2), so
//   phi <= Phi_lo = 2 asin(sqrt(eps^2 - (r_hi - r_lo)^2) / (2 r_hi))  => neighbours,
//   phi >  Phi_hi = 2 asin(eps / (2 r_lo))                            => not.
// With margins for the FP32 predicate's rounding (|s - d^2| <= 4 2^-24 d^2,
// taken as 1e-6 relative), for atan2f and the bucket mapping (1.5e-5 rad per
// point), two points whose buckets are D apart (circularly) are neighbours
// for sure when D <= D_lo and cannot be when D > D_hi; only the few buckets
// in between (the band, D_hi - D_lo ~ 3) need the exact FP32 predicate.  So:
//   * core counting is a difference of the bucket prefix sums over the
//     window |D| <= D_lo, plus exact tests in the band when that count is
//     below minPts;
//   * core buckets within D_lo of each other are connected (all their core
//     points are pairwise neighbours): runs of core buckets whose gaps are
//     <= D_lo are connected sets; with D_hi <= 2 D_lo + 1 an edge can only
//     join two runs that are adjacent around the circle, across a gap of at
//     most D_hi, and only between their end buckets -- the exact predicate
//     decides those few pairs;
//   * a border point's lowest-index core neighbour is the least index over
//     the core points of the window (per-bucket minima) and of the band (exact
//     tests).
// The partition is the one the definition gives (every decision is either
// proven by the bounds or taken by the exact predicate).  Used when the set
// allows it (|z| >= 0.5 everywhere, D_lo >= 4, D_hi <= 2 D_lo + 1, windows
// shorter than the circle); otherwise the grid DBSCAN runs.
constexpr int kAngSmemInts = 5 * kAngBuckets + 2;
constexpr double kAngSlack = 1.5e-5;   // rad per point: atan2f error + bucket mapping

__device__ __forceinline__ int ang_wrap(int b) { return b & (kAngBuckets - 1); }

__device__ __forceinline__ int ang_bucket(float x, float y) {
  const float th = atan2f(y, x);   // [-pi, pi]
  const float f = (th + 3.14159265358979f) * ((float)kAngBuckets / 6.28318530717959f);
  return min(max((int)floorf(f), 0), kAngBuckets - 1);
}

// Block-wide scan of a[0 .. kAngBuckets) in place (blockDim.x * 4 ==
// kAngBuckets): exclusive sum (MAX = false) or exclusive max with identity
// -1 (MAX = true).  Returns the total (sum or max).
template <bool MAX>
__device__ __forceinline__ int ang_scan(int* a, int* wsum) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int b0 = 4 * tid;
  const int v0 = a[b0], v1 = a[b0 + 1], v2 = a[b0 + 2], v3 = a[b0 + 3];
  auto op = [](int x, int y) { return MAX ? max(x, y) : x + y; };
  const int id = MAX ? -1 : 0;
  const int t = op(op(v0, v1), op(v2, v3));
  int x = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x = op(x, y);
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const int w = wsum[lane];
    int s = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s = op(s, y);
    }
    const int sp = __shfl_up_sync(FULL, s, 1);
    wsum[lane] = lane ? sp : id;   // exclusive over warps
    if (lane == 31) wsum[32] = s;
  }
  __syncthreads();
  const int xp = __shfl_up_sync(FULL, x, 1);
  int e = lane ? op(wsum[wid], xp) : wsum[wid];   // exclusive before this thread
  a[b0] = e;
  e = op(e, v0);
  a[b0 + 1] = e;
  e = op(e, v1);
  a[b0 + 2] = e;
  a[b0 + 3] = op(e, v2);
  const int total = wsum[32];
  __syncthreads();
  return total;
}

// Positions (in bucket order) of the circular bucket range [b0, b1]
// (b1 - b0 < kAngBuckets): one or two contiguous ranges of st[] (the bucket
// starts, st[kAngBuckets] = n).
__device__ __forceinline__ void ang_range(const int* st, int b0, int b1, int* p0, int* p1,
                                          int* q0, int* q1) {
  *q0 = *q1 = 0;
  if (b1 < 0) {
    b0 += kAngBuckets;
    b1 += kAngBuckets;
  } else if (b0 >= kAngBuckets) {
    b0 -= kAngBuckets;
    b1 -= kAngBuckets;
  }
  if (b0 < 0) {
    *p0 = st[b0 + kAngBuckets]; *p1 = st[kAngBuckets];
    *q0 = st[0]; *q1 = st[b1 + 1];
  } else if (b1 >= kAngBuckets) {
    *p0 = st[b0]; *p1 = st[kAngBuckets];
    *q0 = st[0]; *q1 = st[b1 + 1 - kAngBuckets];
  } else {
    *p0 = st[b0]; *p1 = st[b1 + 1];
  }
}

__device__ __forceinline__ int ang_count(const int* st, int b0, int b1) {
  int p0, p1, q0, q1;
  ang_range(st, b0, b1, &p0, &p1, &q0, &q1);
  return (p1 - p0) + (q1 - q0);
}

// Up to four position ranges walked as one index space, so that a warp loads
// the points of every range in the same steps (one memory round trip covers
// the whole band of a sparse point).
struct AngRanges {
  int a[4], e[4];
  int tot;
  __device__ __forceinline__ void set(const int* st, int b0, int b1, int c0, int c1) {
    ang_range(st, b0, b1, &a[0], &e[0], &a[1], &e[1]);
    ang_range(st, c0, c1, &a[2], &e[2], &a[3], &e[3]);
    tot = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) tot += e[k] - a[k];
  }
  __device__ __forceinline__ int pos(int t) const {   // t < tot
    int base = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int len = e[k] - a[k];
      if (t < base + len) return a[k] + t - base;
      base += len;
    }
    return -1;
  }
};

// Thresholds from the radius range and eps^2; false when the angular method
// does not apply to this set.  FP32 (FP64 is slow on this GPU): every input
// and result is widened by 1e-5 relative toward the safe side, far above the
// few-ulp errors of sqrtf / asinf, so D_lo stays a proven-neighbour distance
// and D_hi a proven-apart one.
__device__ __forceinline__ bool ang_thresholds(float rmin2, float rmax2, float eps2, int* Dlo,
                                               int* Dhi) {
  const float r_lo = sqrtf(rmin2) * (1.0f - 1e-5f);
  const float r_hi = sqrtf(rmax2) * (1.0f + 1e-5f);
  if (!(r_lo >= 0.5f) || !(r_hi <= 2.0f)) return false;
  const float e_lo2 = eps2 * (1.0f - 1e-5f), e_hi2 = eps2 * (1.0f + 1e-5f);
  const float dr = (r_hi - r_lo) * (1.0f + 1e-5f);
  const float s_lo = sqrtf(fmaxf(0.0f, e_lo2 - dr * dr)) / (2.0f * r_hi) * (1.0f - 1e-5f);
  const float s_hi = sqrtf(e_hi2) / (2.0f * r_lo) * (1.0f + 1e-5f);
  if (!(s_hi < 1.0f)) return false;
  const float phi_lo = 2.0f * asinf(fminf(1.0f, s_lo)) * (1.0f - 1e-5f);
  const float phi_hi = 2.0f * asinf(s_hi) * (1.0f + 1e-5f);
  const float beta = 6.2831853f / (float)kAngBuckets;
  *Dlo = (int)floorf((phi_lo - 2.0f * (float)kAngSlack) / beta) - 1;
  *Dhi = (int)floorf((phi_hi + 2.0f * (float)kAngSlack) / beta) + 1;
  return *Dlo >= 4 && *Dhi <= 2 * *Dlo + 1 && 2 * *Dhi + 2 < kAngBuckets;
}

// The angular DBSCAN of n points z ([2][ld], slice [i0, i1) of this CTA) by
// one thread-block cluster.  Pass 1 (buckets, counts, radius range) has run:
// w.cell holds each point's bucket, w.core its offset inside the bucket,
// w.ahist the counts, and the cluster barrier after it has been taken.  Dlo /
// Dhi from ang_thresholds.  Shared memory (ints): hcnt, st (+1), cur, gmin,
// aux of kAngBuckets.
__device__ __forceinline__ void dbscan_angular(const float* __restrict__ z, int ld, int n,
                                               float eps2, int min_pts, int Dlo, int Dhi,
                                               DbWork w, int* labels, int* M_out, int* smem,
                                               long long* cyc, int i0, int i1) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
  constexpr int NB = kAngBuckets;
  int* hcnt = smem;             // [NB] the CTA's base in each bucket, boundary list, component minima
  int* st = hcnt + NB;          // [NB + 1] bucket starts in bucket order
  int* cur = st + NB + 1;       // [NB] run flags, then the component of each bucket
  int* gmin = cur + NB;         // [NB] least core index per bucket, whole set
  int* aux = gmin + NB;         // [NB] scans, then the canonical id of each component
  int* lst = reinterpret_cast<int*>(w.zs + 2 * (size_t)w.ld_s);   // (z's unused third row)
  // the coordinates in bucket order as (x, y) pairs: one scattered store per
  // point in the scatter, one load per point in the exact tests
  float2* zs2 = reinterpret_cast<float2*>(w.zs);
  __shared__ int wsum[33];
  __shared__ int n_list, n_cs_s;
  auto stamp = [&](int k) {
    if (cyc && tid == 0 && rank == 0) cyc[k] = clock64();
  };
  // ---- 2. bucket starts (every CTA alike, from the instance's count table),
  //    scatter of the slice into bucket order at the offsets pass 1 handed out
  {
    int v[NB / kBlock];   // (blockDim.x * 4 == NB, as the scans assume)
#pragma unroll
    for (int q = 0; q < NB / kBlock; ++q) v[q] = __ldcg(&w.ahist[tid + q * kBlock]);
#pragma unroll
    for (int q = 0; q < NB / kBlock; ++q) st[tid + q * kBlock] = v[q];
  }
  __syncthreads();
  ang_scan<false>(st, wsum);
  if (tid == 0) st[NB] = n;
  __syncthreads();
  for (int b0 = i0; b0 < i1; b0 += 2 * (int)blockDim.x) {
    int cb[2] = {0, 0}, co[2] = {0, 0};
    float zx[2] = {0.f, 0.f}, zy[2] = {0.f, 0.f};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = b0 + u * blockDim.x + tid;
      if (i < i1) { cb[u] = w.cell[i]; co[u] = w.core[i]; zx[u] = z[i]; zy[u] = z[(size_t)ld + i]; }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = b0 + u * blockDim.x + tid;
      if (i < i1) {
        const int pos = st[cb[u]] + hcnt[cb[u]] + co[u];
        w.sorted[pos] = i;
        zs2[pos] = make_float2(zx[u], zy[u]);
      }
    }
  }
  cluster.sync();   // (2) bucket order complete in global memory
  stamp(2);
  // ---- 3. core flags: window count, exact tests in the band when short
  if (tid == 0) n_list = 0;
  for (int b = tid; b < NB; b += blockDim.x) gmin[b] = 0x7fffffff;   // (the CTA's minima)
  __syncthreads();
  for (int b0 = i0; b0 < i1; b0 += 2 * (int)blockDim.x) {
    int cb[2] = {0, 0};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = b0 + u * blockDim.x + tid;
      if (i < i1) cb[u] = w.cell[i];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = b0 + u * blockDim.x + tid;
      bool need = false;
      if (i < i1) {
        // core for sure with minPts points within D_lo; not core for sure
        // with fewer than minPts within D_hi; the exact tests decide between
        const int b = cb[u];
        const int c = ang_count(st, b - Dlo, b + Dlo);
        w.core[i] = c >= min_pts ? 1 : 0;
        need = c < min_pts && ang_count(st, b - Dhi, b + Dhi) >= min_pts;
      }
      const unsigned bl = __ballot_sync(FULL, need);
      int base = 0;
      if (bl && lane == __ffs(bl) - 1) base = atomicAdd(&n_list, __popc(bl));
      base = __shfl_sync(FULL, base, bl ? __ffs(bl) - 1 : 0);   // (from the lane that added)
      if (need) lst[i0 + base + __popc(bl & ((1u << lane) - 1u))] = i;
    }
  }
  __syncthreads();
  const int nl = n_list;
  // a warp's entries are li = wid + j nwarp; lane j loads entry j's index,
  // bucket and coordinates for 32 entries at a time, then the warp takes
  // the entries in turn (their band tests)
  for (int lb = wid; lb < nl; lb += 32 * nwarp) {
    const int lj = lb + lane * nwarp;
    int ei = 0, eb = 0;
    float ex = 0.f, ey = 0.f;
    if (lj < nl) ei = lst[i0 + lj];
    if (lj < nl) { eb = w.cell[ei]; ex = z[ei]; ey = z[(size_t)ld + ei]; }
    const int ne = min(32, (nl - lb + nwarp - 1) / nwarp);
  for (int jj = 0; jj < ne; ++jj) {
    const int i = __shfl_sync(FULL, ei, jj);
    const int b = __shfl_sync(FULL, eb, jj);
    const float za[2] = {__shfl_sync(FULL, ex, jj), __shfl_sync(FULL, ey, jj)};
    int count = ang_count(st, b - Dlo, b + Dlo);
    // the two band ranges, (b + Dlo, b + Dhi] and [b - Dhi, b - Dlo)
    AngRanges br;
    br.set(st, b + Dlo + 1, b + Dhi, b - Dhi, b - Dlo - 1);
    for (int t0 = 0; t0 < br.tot && count < min_pts; t0 += 32) {
      const int t = t0 + lane;
      bool hit = false;
      if (t < br.tot) {
        const int q = br.pos(t);
        const float2 zq = zs2[q];
        const float zb[2] = {zq.x, zq.y};
        hit = nb_pred_t<2>(za, zb, eps2);
      }
      count += __popc(__ballot_sync(FULL, hit));
    }
    if (lane == 0) w.core[i] = count >= min_pts ? 1 : 0;
  }
  }
  __syncthreads();
  // least core index per bucket: the slice's in shared memory, then one
  // global atomic per occupied bucket
  for (int b0 = i0; b0 < i1; b0 += 2 * (int)blockDim.x) {
    int cf[2] = {0, 0}, cb[2] = {0, 0};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = b0 + u * blockDim.x + tid;
      if (i < i1) { cf[u] = w.core[i]; cb[u] = w.cell[i]; }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = b0 + u * blockDim.x + tid;
      if (i < i1 && cf[u]) atomicMin(&gmin[cb[u]], i);
    }
  }
  __syncthreads();
  for (int b = tid; b < NB; b += blockDim.x)
    if (gmin[b] != 0x7fffffff) atomicMin(&w.amin[b], gmin[b]);
  cluster.sync();   // (3) core flags and bucket minima of every CTA
  stamp(3);
  // ---- 4. components over the core buckets (every CTA alike)
  {
    int v[NB / kBlock];
#pragma unroll
    for (int q = 0; q < NB / kBlock; ++q) v[q] = __ldcg(&w.amin[tid + q * kBlock]);
#pragma unroll
    for (int q = 0; q < NB / kBlock; ++q) {
      const int b = tid + q * kBlock;
      gmin[b] = v[q];
      aux[b] = v[q] != 0x7fffffff ? b : -1;   // (for the previous-core-bucket scan)
    }
  }
  __syncthreads();
  const int last_core = ang_scan<true>(aux, wsum);   // aux[b] = largest core bucket < b
  // run starts (flag 1) and the boundaries an edge may cross (flag 2, listed
  // in hcnt, free since barrier 2, and checked below)
  if (tid == 0) n_list = 0;
  __syncthreads();
  for (int b = tid; b < NB; b += blockDim.x) {
    int f = 0;
    if (gmin[b] != 0x7fffffff) {
      const int prev = aux[b] >= 0 ? aux[b] : last_core - NB;   // (wraps to the last)
      const int gap = b - prev;
      if (gap > Dlo) {
        f = 1;
        if (gap <= Dhi) {
          f = 2;   // to be checked
          hcnt[atomicAdd(&n_list, 1)] = b;
        }
      }
    }
    cur[b] = f;
  }
  __syncthreads();
  // a boundary is closed when some core point of the buckets before it and
  // some core point after it, at most Dhi buckets apart, are neighbours: the
  // core points of buckets [b - Dhi, prev] (X) against those of [b, prev + Dhi]
  // (Y), 32 x 32 pairs per step (X in the lanes, Y broadcast by shuffles).
  // Pairs more than Dhi buckets apart are proven non-neighbours, so testing
  // them too changes nothing.
  {
    const int nbd = n_list;
    for (int bi = wid; bi < nbd; bi += nwarp) {
      const int b = hcnt[bi];
      const int prev = aux[b] >= 0 ? aux[b] : last_core - NB;
      AngRanges X, Y;
      X.set(st, b - Dhi, prev, 0, -1);
      Y.set(st, b, prev + Dhi, 0, -1);
      bool found = false;
      for (int x0 = 0; x0 < X.tot && !found; x0 += 32) {
        float xa[2] = {0.f, 0.f};
        bool xv = false;
        if (x0 + lane < X.tot) {
          const int q = X.pos(x0 + lane);
          xv = w.core[w.sorted[q]] != 0;
          const float2 zq = zs2[q];
          xa[0] = zq.x;
          xa[1] = zq.y;
        }
        for (int y0 = 0; y0 < Y.tot && !found; y0 += 32) {
          float ya[2] = {0.f, 0.f};
          bool yv = false;
          if (y0 + lane < Y.tot) {
            const int q = Y.pos(y0 + lane);
            yv = w.core[w.sorted[q]] != 0;
            const float2 zq = zs2[q];
            ya[0] = zq.x;
            ya[1] = zq.y;
          }
          bool hit = false;
          for (int j = 0; j < 32; ++j) {
            const float yb[2] = {__shfl_sync(FULL, ya[0], j), __shfl_sync(FULL, ya[1], j)};
            const bool vj = __shfl_sync(FULL, yv, j);
            hit |= xv && vj && nb_pred_t<2>(xa, yb, eps2);
          }
          found = __any_sync(FULL, hit);
        }
      }
      if (lane == 0 && found) cur[ang_wrap(b)] = 3;   // closed
    }
  }
  __syncthreads();
  // component starts: open run starts (flag 1, or 2 left unclosed)
  for (int b = tid; b < NB; b += blockDim.x) aux[b] = (cur[b] == 1 || cur[b] == 2) ? 1 : 0;
  __syncthreads();
  ang_scan<false>(aux, wsum);   // aux[b] = component starts before b
  if (tid == 0) n_cs_s = 0;
  __syncthreads();
  for (int b = tid; b < NB; b += blockDim.x) {
    const bool cs = cur[b] == 1 || cur[b] == 2;
    if (cs) atomicAdd(&n_cs_s, 1);
  }
  __syncthreads();
  const int n_cs = n_cs_s;
  // component of each core bucket: starts up to and including b, minus one;
  // core buckets before the first start belong to the last component (wrap)
  for (int b = tid; b < NB; b += blockDim.x) {
    int c = -1;
    if (gmin[b] != 0x7fffffff) {
      const bool cs = cur[b] == 1 || cur[b] == 2;
      const int upto = aux[b] + (cs ? 1 : 0);
      c = n_cs == 0 ? 0 : (upto >= 1 ? upto - 1 : n_cs - 1);
    }
    cur[b] = c;   // (run flags no longer needed)
  }
  __syncthreads();
  // least core index of each component (hcnt is free now), canonical ids
  const int n_comp = last_core >= 0 ? max(n_cs, 1) : 0;
  for (int c = tid; c < n_comp; c += blockDim.x) hcnt[c] = 0x7fffffff;
  __syncthreads();
  for (int b = tid; b < NB; b += blockDim.x)
    if (cur[b] >= 0) atomicMin(&hcnt[cur[b]], gmin[b]);
  __syncthreads();
  for (int c = tid; c < n_comp; c += blockDim.x) {
    const int key = hcnt[c];
    int id = 0;
    for (int u = 0; u < n_comp; ++u) id += hcnt[u] < key;
    aux[c] = id;   // canonical id of component c
  }
  __syncthreads();
  stamp(4);
  // ---- 5. labels of the slice: core points from their bucket's component;
  //    the others from their lowest-index core neighbour (window minima, then
  //    exact tests in the band), else noise
  if (tid == 0) n_list = 0;
  __syncthreads();
  for (int b0 = i0; b0 < i1; b0 += 2 * (int)blockDim.x) {
    int cf[2] = {0, 0}, cb[2] = {0, 0};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = b0 + u * blockDim.x + tid;
      if (i < i1) { cf[u] = w.core[i]; cb[u] = w.cell[i]; }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = b0 + u * blockDim.x + tid;
      bool border = false;
      if (i < i1) {
        if (cf[u]) labels[i] = aux[cur[cb[u]]];
        else border = true;
      }
      const unsigned bl = __ballot_sync(FULL, border);
      int base = 0;
      if (bl && lane == __ffs(bl) - 1) base = atomicAdd(&n_list, __popc(bl));
      base = __shfl_sync(FULL, base, bl ? __ffs(bl) - 1 : 0);   // (from the lane that added)
      if (border) lst[i0 + base + __popc(bl & ((1u << lane) - 1u))] = i;
    }
  }
  __syncthreads();
  const int nb_pts = n_list;
  for (int lb = wid; lb < nb_pts; lb += 32 * nwarp) {   // (32 entries' loads at a time)
    const int lj = lb + lane * nwarp;
    int ei = 0, eb = 0;
    float ex = 0.f, ey = 0.f;
    if (lj < nb_pts) ei = lst[i0 + lj];
    if (lj < nb_pts) { eb = w.cell[ei]; ex = z[ei]; ey = z[(size_t)ld + ei]; }
    const int ne = min(32, (nb_pts - lb + nwarp - 1) / nwarp);
  for (int jj = 0; jj < ne; ++jj) {
    const int i = __shfl_sync(FULL, ei, jj);
    const int b = __shfl_sync(FULL, eb, jj);
    const float za[2] = {__shfl_sync(FULL, ex, jj), __shfl_sync(FULL, ey, jj)};
    int best = 0x7fffffff;
    for (int d0 = -Dlo; d0 <= Dlo; d0 += 32) {
      const int dd = d0 + lane;
      if (dd <= Dlo) best = min(best, gmin[ang_wrap(b + dd)]);
    }
    best = __reduce_min_sync(FULL, best);
    // a core point of a band bucket has an index >= that bucket's least core
    // index: when none is below best, the band cannot lower it
    int bmin = 0x7fffffff;
    {
      const int nbb = Dhi - Dlo;   // band buckets on each side
      if (lane < 2 * nbb) {
        const int dd = lane < nbb ? Dlo + 1 + lane : -(Dlo + 1 + (lane - nbb));
        bmin = gmin[ang_wrap(b + dd)];
      }
      for (int l2 = lane + 32; l2 < 2 * nbb; l2 += 32) {
        const int dd = l2 < nbb ? Dlo + 1 + l2 : -(Dlo + 1 + (l2 - nbb));
        bmin = min(bmin, gmin[ang_wrap(b + dd)]);
      }
      bmin = __reduce_min_sync(FULL, bmin);
    }
    AngRanges br;
    br.set(st, b + Dlo + 1, b + Dhi, b - Dhi, b - Dlo - 1);
    if (bmin >= best) br.tot = 0;
    for (int t0 = 0; t0 < br.tot; t0 += 32) {
      const int t = t0 + lane;
      int cand = 0x7fffffff;
      if (t < br.tot) {
        const int q = br.pos(t);
        const int sid = w.sorted[q];
        const float2 zq = zs2[q];
        const float zb[2] = {zq.x, zq.y};
        if (sid < best && w.core[sid] && nb_pred_t<2>(za, zb, eps2)) cand = sid;
      }
      best = min(best, __reduce_min_sync(FULL, cand));
    }
    if (lane == 0) labels[i] = best == 0x7fffffff ? -1 : aux[cur[w.cell[best]]];
  }
  }
  if (tid == 0 && rank == 0) *M_out = n_comp;
  stamp(5);
}


// DBSCAN of 2-D points: pass 1 (angle buckets, per-CTA counts, radius range,
// the coordinate check), then the angular method when the set allows it, else
// the grid method.  Same interface as dbscan_block<2>.
__device__ __forceinline__ void dbscan2(const float* __restrict__ z, int ld, int n, float eps2,
                                        float cell_inv, int G, int R, int min_pts, DbWork w,
                                        int* labels, int* M_out, int* status, int* smem,
                                        long long* cyc, int uf_limit) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31;
  __shared__ unsigned s_rmin, s_rmax;   // squared radii as float bits (>= 0: ordered as ints)
  __shared__ int s_bad;
  if (cyc && tid == 0 && rank == 0) cyc[0] = clock64();
  const int chunk = (((n + CL - 1) / CL) + 31) & ~31;
  const int i0 = min(n, rank * chunk), i1 = min(n, i0 + chunk);
  if (tid == 0) {
    s_rmin = 0x7f800000u;   // +inf
    s_rmax = 0u;
    s_bad = 0;
  }
  __syncthreads();
  // ---- 1. bucket of each point of the slice, counts, radius range.  The
  //    counts are taken per CTA in shared memory (a point's offset inside
  //    its bucket among the slice's points, kept in w.core until the core
  //    flags replace it); then one global atomic per occupied bucket adds the
  //    CTA's count to the instance's table and returns the CTA's base in the
  //    bucket, kept in the first kAngBuckets ints of shared memory (the
  //    angular method's scatter adds it; its boundary list reuses the space
  //    later).
  int* lbase = smem;
  for (int b = tid; b < kAngBuckets; b += blockDim.x) lbase[b] = 0;
  __syncthreads();
  {
    float rmn = INFINITY, rmx = 0.f;
    bool bad = false;
    // two points per thread and step: their loads, then their count atomics,
    // in flight together
    const int B = blockDim.x;
    for (int b0 = i0; b0 < i1; b0 += 2 * B) {
      float xs[2] = {0.f, 0.f}, ys[2] = {0.f, 0.f};
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int i = b0 + u * B + tid;
        if (i < i1) { xs[u] = z[i]; ys[u] = z[(size_t)ld + i]; }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int i = b0 + u * B + tid;
        if (i < i1) {
          const float x = xs[u], y = ys[u];
          bad |= !(x >= -1.0f && x <= 1.0f && y >= -1.0f && y <= 1.0f);
          const int b = ang_bucket(x, y);
          w.cell[i] = b;
          w.core[i] = atomicAdd(&lbase[b], 1);
          const float r2 = x * x + y * y;
          rmn = fminf(rmn, r2);
          rmx = fmaxf(rmx, r2);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rmn = fminf(rmn, __shfl_xor_sync(FULL, rmn, o));
      rmx = fmaxf(rmx, __shfl_xor_sync(FULL, rmx, o));
    }
    if (lane == 0) {
      atomicMin(&s_rmin, __float_as_uint(rmn));
      atomicMax(&s_rmax, __float_as_uint(rmx));
    }
    if (bad) s_bad = 1;
  }
  __syncthreads();
  {
    int c[kAngBuckets / kBlock], bs[kAngBuckets / kBlock];
#pragma unroll
    for (int q = 0; q < kAngBuckets / kBlock; ++q) {
      c[q] = lbase[tid + q * kBlock];
      bs[q] = c[q] > 0 ? atomicAdd(&w.ahist[tid + q * kBlock], c[q]) : 0;
    }
#pragma unroll
    for (int q = 0; q < kAngBuckets / kBlock; ++q) lbase[tid + q * kBlock] = bs[q];
  }
  cluster.sync();   // (1) every CTA's counts and radius range (the table is complete)
  if (cyc && tid == 0 && rank == 0) cyc[1] = clock64();
  // the ranks' scalars are read once (lanes of warp 0) and the thresholds
  // (FP64 arithmetic, slow on this GPU) computed by one thread for the CTA
  __shared__ int s_dec[4];   // any bad coordinate, angular method, Dlo, Dhi
  if (tid < 32) {
    unsigned rmin_u = 0x7f800000u, rmax_u = 0u;
    int bad = 0;
    if (lane < CL) {
      rmin_u = *cluster.map_shared_rank(&s_rmin, lane);
      rmax_u = *cluster.map_shared_rank(&s_rmax, lane);
      bad = *cluster.map_shared_rank(&s_bad, lane);
    }
    rmin_u = __reduce_min_sync(FULL, rmin_u);
    rmax_u = __reduce_max_sync(FULL, rmax_u);
    bad = __reduce_or_sync(FULL, (unsigned)bad);
    if (lane == 0) {
      int Dlo = 0, Dhi = 0;
      const bool ok = !bad && n > 0 &&
                      ang_thresholds(__uint_as_float(rmin_u), __uint_as_float(rmax_u), eps2,
                                     &Dlo, &Dhi);
      s_dec[0] = bad;
      s_dec[1] = ok;
      s_dec[2] = Dlo;
      s_dec[3] = Dhi;
    }
  }
  __syncthreads();
  const int anybad = s_dec[0];
  if (anybad) {   // coordinates outside [-1, 1]: refused, as the grid method does
    for (int i = i0 + tid; i < i1; i += blockDim.x) labels[i] = -1;
    if (tid == 0 && rank == 0) { *M_out = 0; atomicCAS(status, 0, CE_MPPI_ERR_INVALID_ARG); }
    cluster.sync();   // no CTA leaves while another reads its scalars
    return;
  }
  const bool ang = s_dec[1] != 0;
  const int Dlo = s_dec[2], Dhi = s_dec[3];
  if (cyc && tid == 0 && rank == 0) cyc[15] = ang ? 1 : 2;
  if (ang) {
    dbscan_angular(z, ld, n, eps2, min_pts, Dlo, Dhi, w, labels, M_out, smem, cyc, i0, i1);
    if (cyc && tid == 0 && rank == 0) cyc[6] = cyc[7] = cyc[8] = cyc[5];
  } else {
    cluster.sync();   // the scalars are no longer read: the grid method reuses the memory
    dbscan_block<2>(z, ld, n, eps2, cell_inv, G, R, min_pts, w, labels, M_out, status, smem,
                    cyc, uf_limit);
  }
}

__device__ __forceinline__ DbWork db_work_of(const InstDesc& d) {
  DbWork w;
  w.cell = d.cell;
  w.sorted = d.sorted;
  w.zs = d.zs;
  w.ld_s = d.Kp;
  w.core = d.parent;
  w.bbox = d.bbox;
  w.labels_tmp = d.label;
  w.ahist = d.ang;
  w.amin = d.ang + kAngBuckets;
  return w;
}

// The angular method's two bucket tables start at zero counts and INT_MAX
// minima; this CTA's share of them is reset here (the caller's cluster barrier
// orders it before the method's atomics).
__device__ __forceinline__ void ang_reset(const DbWork& w) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  for (int b = rank * blockDim.x + threadIdx.x; b < kAngBuckets; b += CL * blockDim.x) {
    w.ahist[b] = 0;
    w.amin[b] = 0x7fffffff;
  }
}

// One cluster per instance; rank 0 publishes the cluster count and the mode.
__device__ __forceinline__ void dbscan_stage(const KArgs& a, int* smem_i) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int inst = blockIdx.x / CL;
  const InstDesc& d = desc_of(a, inst);
  Ctl* ctl = d.ctl;
  const int mode = ctl->mode;
  if (mode != CE_MODE_STATIC) return;   // fallback replans skip clustering (whole cluster)
  const int nV = ctl->nV;
  const DbWork w = db_work_of(d);
  __shared__ int M;
  if (d.p == 3)
    dbscan_block<3>(d.z, d.Kp, nV, d.eps2, d.cell_inv, d.G, d.R, d.min_pts, w, d.label, &M,
                    &ctl->status, smem_i, ctl->dbcyc, d.uf_limit);
  else
    dbscan2(d.z, d.Kp, nV, d.eps2, d.cell_inv, d.G, d.R, d.min_pts, w, d.label, &M,
            &ctl->status, smem_i, ctl->dbcyc, d.uf_limit);
  __syncthreads();
  if (threadIdx.x == 0 && cluster.block_rank() == 0) {
    // a union-find that gave up leaves labels that cannot be trusted: the
    // replan takes the all-noise fallback (every status raise of the stage
    // happened before its last cluster barrier)
    if (__ldcg(&ctl->status) != 0) M = 0;
    ctl->M = M;
    if (M == 0) ctl->mode = CE_MODE_ALLNOISE;
  }
}

__global__ void __maxnreg__(64) k_dbscan(KArgs a) {
  extern __shared__ int smem_i[];
  cg::cluster_group cluster = cg::this_cluster();
  ang_reset(db_work_of(desc_of(a, blockIdx.x / cluster.num_blocks())));
  cluster.sync();   // (the tables are reset before any CTA counts)
  dbscan_stage(a, smem_i);
}

__global__ void __maxnreg__(64) k_dbscan_standalone(const float* z, int n, int ld, int p,
                                                              float eps2, float cell_inv, int G,
                                                              int R, int min_pts, int* labels,
                                                              int* n_clusters, DbWork w) {
  extern __shared__ int smem_i[];
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ int M;
  __shared__ int status;
  w.labels_tmp = labels;
  if (threadIdx.x == 0) status = 0;
  ang_reset(w);
  cluster.sync();   // rank 0's status is cleared and the bucket tables reset before use
  int* st0 = cluster.map_shared_rank(&status, 0);
  if (p == 3)
    dbscan_block<3>(z, ld, n, eps2, cell_inv, G, R, min_pts, w, labels, &M, st0, smem_i,
                    nullptr, kUfLimit);
  else
    dbscan2(z, ld, n, eps2, cell_inv, G, R, min_pts, w, labels, &M, st0, smem_i, nullptr,
            kUfLimit);
  cluster.sync();   // every CTA's status updates have landed
  if (threadIdx.x == 0 && cluster.block_rank() == 0) *n_clusters = status ? -status : M;
}

// ========================================================================= select
// Algorithm 1 [Cluster stats], [Selection], [Within-cluster weighting]:
// per-cluster count, mean cost Sbar_c (Eq. 14), mean direction vhat_c
// (Eq. 16) and least cost, by exact int64 fixed-point sums (and min keys);
// c* by Eq. 14 (static) or Eq. 18 (dynamic, |v_o*| > threshold); then the
// softmin weights over the update set (Eq. 19, or Eq. 6 over all K / over V
// in the fallbacks) with the set's least cost subtracted before exp.  The
// weights are left unnormalised (the update multiplies by 1/Z); the nonzero
// ones are also listed by ascending k when there are at most kSparseMax.
constexpr int kWin = 512;   // clusters per statistics window
constexpr int kUpdProdMax = 4096;   // products staged per pass of the listed update
constexpr int kSlots = 2;   // per-warp label cache of the cluster statistics

// One thread-block cluster of CL CTAs per instance.  Each CTA sums the
// statistics of a window of clusters over its slice of V in its own shared
// memory; rank 0 adds the CTAs' sums through distributed shared memory (exact
// integers: order-free) and evaluates the criterion.
// The weights pass splits its domain into kPruneRanges fixed ranges whose
// normaliser partials are added in range order, so Z does not depend on CL.
struct SelSmem {
  unsigned long long accS[kWin], accG[3][kWin];
  int accN[kWin];
  unsigned int accM[kWin];
  int lk[kSparseMax];
  float le[kSparseMax];
  // the fused kernel's rank 0: the sorted list, the nominal before and after
  // the listed update, and what the finalize needs, read at the start of the
  // selection so that the update and the finalize make no global round trip
  int sk[kSparseMax];
  float se[kSparseMax];
  float Us[kMaxT * kMaxM], Un[kMaxT * kMaxM];
  float x0s[12];
  ce_mppi_diag dg;
  unsigned long long ctr;
  float invZ;
  int nnz;
};

// fused: called after the DBSCAN stage in the same kernel; with few nonzero
// weights rank 0 then also applies the update and finalizes the replan.
__device__ __forceinline__ void update_sparse_finalize(const KArgs& a, const InstDesc& d, int inst,
                                                       SelSmem& sm);
__device__ void finalize(const InstDesc& d, const Req& r);

__device__ __forceinline__ void select_stage(const KArgs& a, SelSmem& sm, bool fused) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
  const int inst = blockIdx.x / CL;
  const InstDesc& d = desc_of(a, inst);
  Ctl* ctl = d.ctl;
  unsigned long long* accS = sm.accS;
  unsigned long long (*accG)[kWin] = sm.accG;
  int* accN = sm.accN;
  unsigned int* accM = sm.accM;
  int* lk = sm.lk;
  float* le = sm.le;
  __shared__ float red[33];
  __shared__ unsigned long long bestkey;
  __shared__ int lcount, lnz;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int K = d.K, Kp = d.Kp, p = d.p;
  const int mode0 = ctl->mode;
  const int nV = ctl->nV, M = ctl->M;
  int sel = -1, dynamic = 0;
  if (tid == 0) { lcount = 0; lnz = 0; }
  if (fused && rank == 0) {
    // (loads that complete while the selection runs)
    const Req rq = req_of(a, inst);
    for (int c = tid; c < d.T * d.m; c += blockDim.x) sm.Us[c] = d.U[c];
    if (tid < d.n) sm.x0s[tid] = rq.x0[tid];
    if (tid == 0) {
      // every load first, then the stores (a store between them would hold
      // the next load back until its own value arrived)
      const int nC = ctl->nC, os = ctl->o_star, stt = ctl->status, ct = ctl->col_tests;
      float pb[3], vo[3];
      for (int i = 0; i < 3; ++i) { pb[i] = ctl->pbar[i]; vo[i] = ctl->v_obs[i]; }
      const unsigned long long cr = *d.counter;
      ce_mppi_diag& g = sm.dg;
      g.n_col = nC; g.n_valid = nV; g.n_clusters = M; g.o_star = os; g.status = stt;
      for (int i = 0; i < 3; ++i) { g.pbar[i] = pb[i]; g.v_obs[i] = vo[i]; }
      g.col_tests = ct;
      sm.ctr = cr;
    }
  }
  // the weights of the rollouts outside the update set are zero; with a
  // selection the window barriers below order these stores before the
  // members' weights (and the list count's reset before other CTAs' adds),
  // otherwise the barrier after this block does
  const bool over_all0 = mode0 == CE_MODE_NOCOL || mode0 == CE_MODE_ALLCOL || mode0 == CE_MODE_MPPI;
  if (!over_all0) {
    const int chunk = (((K + CL - 1) / CL) + 31) & ~31;
    const int kb = min(K, rank * chunk), ke = min(K, kb + chunk);
    for (int k = kb + tid; k < ke; k += blockDim.x) d.w_k[k] = 0.f;
  }
  if (mode0 == CE_MODE_STATIC) {
    // fixed-point scales: S in [-Smax, Smax], g in [-1, 1], at most nV terms
    const float sm = ctl->S_absmax_V;
    const int lgN = 32 - __clz(nV + 1);
    int eS = 60 - lgN - (sm > 0.f ? ilogbf(sm) + 1 : 0);
    eS = max(-100, min(eS, 100));
    const int eG = 60 - lgN - 1;
    const float vx = ctl->v_obs[0], vy = ctl->v_obs[1], vz = ctl->v_obs[2];
    const float vn = sqrtf(vx * vx + vy * vy + vz * vz);
    dynamic = vn > d.v_static_thresh;
    const float ivn = 1.0f / (vn + d.norm_eps);
    const float vh[3] = {vx * ivn, vy * ivn, vz * ivn};
    if (tid == 0) bestkey = ~0ull;
    // each warp owns a contiguous range of V and keeps per-lane partial sums
    // for up to kSlots labels (warp-uniform slot labels); a slot is reduced
    // across the warp and added to rank 0's accumulators only when evicted or
    // at the end -- exact int64 sums and min keys, so the result does not
    // depend on the order.
    const int Lr = (((nV + CL * nw - 1) / (CL * nw)) + 31) & ~31;
    const int beg = min(nV, (rank * nw + wid) * Lr), end = min(nV, beg + Lr);
    for (int w0 = 0; w0 < M; w0 += kWin) {
      // each CTA accumulates its slice of V in its own shared memory; rank 0
      // adds the CTAs' sums after the window (exact integers: order-free)
      for (int c = tid; c < kWin; c += blockDim.x) {
        accS[c] = 0ull; accN[c] = 0; accM[c] = 0xffffffffu;
        accG[0][c] = accG[1][c] = accG[2][c] = 0ull;
      }
      __syncthreads();
      int cl[kSlots];
      long long aS[kSlots], aG[kSlots][3];
      int aN[kSlots];
      uint32_t aM[kSlots];
#pragma unroll
      for (int sl = 0; sl < kSlots; ++sl) {
        cl[sl] = -1; aS[sl] = 0; aN[sl] = 0; aM[sl] = 0xffffffffu;
        aG[sl][0] = aG[sl][1] = aG[sl][2] = 0;
      }
      auto flush = [&](int sl) {
        if (cl[sl] < 0) return;   // (an empty slot: warp-uniform)
        long long s = aS[sl], g0 = aG[sl][0], g1 = aG[sl][1], g2 = aG[sl][2];
        int nn = aN[sl];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          s += __shfl_xor_sync(FULL, s, o);
          g0 += __shfl_xor_sync(FULL, g0, o);
          g1 += __shfl_xor_sync(FULL, g1, o);
          g2 += __shfl_xor_sync(FULL, g2, o);
          nn += __shfl_xor_sync(FULL, nn, o);
        }
        const uint32_t mk = __reduce_min_sync(FULL, aM[sl]);
        if (lane == 0) {
          const int c = cl[sl] - w0;
          atomicAdd(&accS[c], (unsigned long long)s);
          atomicAdd(&accG[0][c], (unsigned long long)g0);
          atomicAdd(&accG[1][c], (unsigned long long)g1);
          atomicAdd(&accG[2][c], (unsigned long long)g2);
          atomicAdd(&accN[c], nn);
          atomicMin(&accM[c], mk);
        }
        cl[sl] = -1; aS[sl] = 0; aN[sl] = 0; aM[sl] = 0xffffffffu;
        aG[sl][0] = aG[sl][1] = aG[sl][2] = 0;
      };
      // the loads of the next 32 positions are issued before this step's work
      int nL = -1;
      float nS = 0.f, nG[3] = {0.f, 0.f, 0.f};
      auto fetch = [&](int i) {
        nL = -1;
        if (i < end) {
          nL = __ldg(d.label + i);
          nS = __ldg(d.Sv + i);
          if (dynamic)   // (directions only enter the dynamic criterion)
#pragma unroll
            for (int q = 0; q < 3; ++q)
              if (q < p) nG[q] = __ldg(d.g + (size_t)q * Kp + i);
        }
      };
      fetch(beg + lane);
      for (int s0 = beg; s0 < end; s0 += 32) {
        int L = nL;
        const float Si = nS, Gi[3] = {nG[0], nG[1], nG[2]};
        fetch(s0 + 32 + lane);
        long long vS = 0, vG[3] = {0, 0, 0};
        uint32_t vM = 0xffffffffu;
        if (L >= w0 && L < w0 + kWin) {
          vS = __float2ll_rn(ldexpf(Si, eS));
          vM = float_key(Si);
#pragma unroll
          for (int q = 0; q < 3; ++q)
            if (q < p) vG[q] = __float2ll_rn(ldexpf(Gi[q], eG));
        } else {
          L = -1;
        }
        // accumulate the lanes whose label is cached; while some are not,
        // cache the first missing label in an empty slot (or in a slot
        // flushed for it, in turn); each round retires at least one lane's
        // label, so 33 rounds suffice
        bool done = L < 0;
        for (int round = 0; round <= 32; ++round) {
#pragma unroll
          for (int sl = 0; sl < kSlots; ++sl)
            if (!done && L == cl[sl]) {
              aS[sl] += vS; aN[sl] += 1; aM[sl] = min(aM[sl], vM);
              aG[sl][0] += vG[0]; aG[sl][1] += vG[1]; aG[sl][2] += vG[2];
              done = true;
            }
          const unsigned pend = __ballot_sync(FULL, !done);
          if (!pend) break;
          int vic = -1;
#pragma unroll
          for (int sl = kSlots - 1; sl >= 0; --sl)
            if (cl[sl] < 0) vic = sl;
          if (vic < 0) {
            vic = round % kSlots;
#pragma unroll
            for (int sl = 0; sl < kSlots; ++sl)
              if (sl == vic) flush(sl);
          }
          const int Lm = __shfl_sync(FULL, L, __ffs(pend) - 1);
#pragma unroll
          for (int sl = 0; sl < kSlots; ++sl)
            if (sl == vic) cl[sl] = Lm;
        }
      }
#pragma unroll
      for (int sl = 0; sl < kSlots; ++sl) flush(sl);
      cluster.sync();   // every CTA's sums of the window are final
      if (rank == 0)
        for (int c = tid; c < kWin && w0 + c < M; c += blockDim.x) {
          unsigned long long tS = 0ull, tG[3] = {0ull, 0ull, 0ull};
          int tN = 0;
          unsigned int tM = 0xffffffffu;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (q < CL) {   // (loads of all ranks in flight together)
              tS += *cluster.map_shared_rank(&accS[c], q);
#pragma unroll
              for (int e = 0; e < 3; ++e) tG[e] += *cluster.map_shared_rank(&accG[e][c], q);
              tN += *cluster.map_shared_rank(&accN[c], q);
              tM = min(tM, *cluster.map_shared_rank(&accM[c], q));
            }
          }
          const float n = (float)tN;
          float crit;
          if (!dynamic) {
            crit = ldexpf(__ll2float_rn((long long)tS), -eS) / n;
          } else {
            float v[3], nn = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              v[q] = q < p ? ldexpf(__ll2float_rn((long long)tG[q]), -eG) / n : 0.f;
              nn += v[q] * v[q];
            }
            const float iv = 1.0f / (sqrtf(nn) + d.norm_eps);
            crit = (v[0] * iv) * vh[0] + (v[1] * iv) * vh[1] + (v[2] * iv) * vh[2];
          }
          d.cmin[w0 + c] = key_float(tM);
          atomicMin(&bestkey, ((unsigned long long)float_key(crit) << 32) | (unsigned)(w0 + c));
        }
      cluster.sync();   // rank 0 has read every CTA's sums (they may be cleared)
    }
    sel = (int)(*cluster.map_shared_rank(&bestkey, 0) & 0xffffffffull);   // (final since the last window)
  }
  // the update set (all K / V / the selected cluster) and its least cost
  const int mode = mode0 == CE_MODE_STATIC ? (dynamic ? CE_MODE_DYNAMIC : CE_MODE_STATIC) : mode0;
  const bool over_all = mode == CE_MODE_NOCOL || mode == CE_MODE_ALLCOL || mode == CE_MODE_MPPI;
  const bool over_V = mode == CE_MODE_ALLNOISE;
  const float smin = over_all ? ctl->S_min_all : over_V ? ctl->S_min_V : d.cmin[sel];
  const float il = d.inv_lambda;
  // weights: the domain (K, or V) in kPruneRanges fixed ranges, m_z per warp
  const int dom = over_all ? K : nV;
  const int Lz = (((dom + kPruneRanges - 1) / kPruneRanges) + 31) & ~31;
  const int m_z = kPruneRanges / (CL * nw);
  const int v0 = (rank * nw + wid) * m_z;
  if (mode0 != CE_MODE_STATIC) cluster.sync();   // the zeros and the count's reset land first
  {
    const int zb = min(dom, v0 * Lz), ze = min(dom, zb + m_z * Lz);
    int jr = 0;
    float z = 0.f, zc = 0.f;
    // the loads of the next 32 positions are issued before this step's work
    // (label, rollout index and cost together, members or not)
    int nLab = -1, nIdx = 0;
    float nS = 0.f;
    auto wfetch = [&](int i) {
      if (i < ze) {
        if (over_all) {
          nS = __ldg(d.S + i);
        } else {
          nLab = __ldg(d.label + i);
          nIdx = __ldg(d.idxV + i);
          nS = __ldg(d.Sv + i);
        }
      }
    };
    wfetch(zb + lane);
    for (int s0 = zb; s0 < ze; s0 += 32) {
      const int i = s0 + lane;
      const int lab = nLab, kv = nIdx;
      const float Sf = nS;
      wfetch(s0 + 32 + lane);
      bool mem = false;
      int k = 0;
      float Sk = 0.f;
      if (i < ze) {
        if (over_all) {
          mem = true; k = i; Sk = Sf;
        } else {
          mem = over_V || lab == sel;
          if (mem) { k = kv; Sk = Sf; }
        }
      }
      float e = 0.f;
      if (mem) {
        e = expf(-(Sk - smin) * il);
        kahan_add(z, zc, e);
        d.w_k[k] = e;
      }
      // nonzero weights into rank 0's list (warp-aggregated)
      const bool nz = e != 0.f;
      const unsigned b = __ballot_sync(FULL, nz);
      if (b) {
        int base = 0;
        if (lane == __ffs(b) - 1) {
          base = atomicAdd(cluster.map_shared_rank(&lcount, 0), __popc(b));
          atomicAdd(&lnz, __popc(b));
        }
        base = __shfl_sync(FULL, base, __ffs(b) - 1) + __popc(b & ((1u << lane) - 1u));
        if (nz && base < kSparseMax) {
          *cluster.map_shared_rank(&lk[base], 0) = k;
          *cluster.map_shared_rank(&le[base], 0) = e;
        }
      }
      if (s0 + 32 - zb == (jr + 1) * Lz) {
        const float t = warp_sum(z);
        if (lane == 0) d.zpart[v0 + jr] = t;
        ++jr;
        z = zc = 0.f;
      }
    }
    for (; jr < m_z; ++jr) {   // a range cut by the domain's end, and ranges past it
      const float t = warp_sum(z);
      if (lane == 0) d.zpart[v0 + jr] = t;
      z = zc = 0.f;
    }
  }
  __syncthreads();
  if (tid == 0 && lnz) atomicAdd(&ctl->nnz_all, lnz);
  cluster.sync();   // the list, the range partials and the nonzero count are complete
  if (fused && tid == 0 && rank == 0) ctl->dbcyc[12] = clock64();   // (stage clock stamp)
  if (rank != 0) return;
  // the update kernel that follows may be scheduled now (the other ranks
  // have left): its CTAs wait for this grid's completion (pdl_wait)
  pdl_trigger();
  if (fused && tid == 0) ctl->dbcyc[13] = clock64();
  // rank 0: Z in range order, the list by ascending k, the control block
  if (wid == 0) {
    constexpr int per = kPruneRanges / 32;
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < per; ++j) t += __ldcg(d.zpart + per * lane + j);
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  const int nl = lcount;
  if (nl <= kSparseMax) {
    // rank by counting (keys are distinct)
    int rk = 0, kk = 0;
    float ee = 0.f;
    if (tid < nl) {
      kk = lk[tid];
      ee = le[tid];
      for (int j = 0; j < nl; ++j) rk += lk[j] < kk;
    }
    if (tid < nl) {
      d.nzk[rk] = kk;
      d.nze[rk] = ee;
      if (fused) { sm.sk[rk] = kk; sm.se[rk] = ee; }
    }
  }
  __syncthreads();
  if (tid == 0) {
    ctl->mode = mode;
    ctl->sel = sel;
    ctl->dynamic = dynamic;
    ctl->S_min = smin;
    ctl->invZ = 1.0f / red[32];
    ctl->nnz = nl <= kSparseMax ? nl : -1;
    if (fused) {
      sm.invZ = 1.0f / red[32];
      sm.nnz = nl <= kSparseMax ? nl : -1;
      sm.dg.mode = mode; sm.dg.sel_label = sel; sm.dg.dynamic = dynamic; sm.dg.S_min = smin;
    }
  }
  if (fused) {
    __syncthreads();
    // (a dense update is left to the tiled update kernel over the whole GPU)
    if (nl <= kSparseMax) update_sparse_finalize(a, d, inst, sm);
    if (tid == 0) ctl->dbcyc[14] = clock64();
  }
}

__global__ void __maxnreg__(64) k_select(KArgs a) {
  __shared__ SelSmem sm;
  select_stage(a, sm, false);
}

// ========================================================================= fused
// Prune, DBSCAN and selection of one instance in one cluster launch: the
// stages follow each other at cluster barriers instead of kernel boundaries,
// each instance at its own pace.  The selection's accumulators reuse the
// DBSCAN tables' shared memory.
// A replan whose inputs the track kernel refused (a NaN or infinity in a
// device buffer): the outputs get the current nominal and the diagnostics the
// status; the nominal, the counter and x_next are left as they are.
__device__ void refuse_replan(const InstDesc& d, const Req& r) {
  Ctl* ctl = d.ctl;
  const int TM = d.T * d.m;
  if (r.u_out)
    for (int c = threadIdx.x; c < TM; c += blockDim.x) r.u_out[c] = d.U[c];
  if (threadIdx.x == 0) {
    if (r.diag) {
      ce_mppi_diag g;
      memset(&g, 0, sizeof(g));
      g.mode = -1; g.n_col = 0; g.n_valid = 0; g.n_clusters = 0; g.sel_label = -1;
      g.o_star = -1; g.dynamic = 0; g.status = ctl->status; g.S_min = 0.f;
      for (int i = 0; i < 3; ++i) { g.pbar[i] = 0.f; g.v_obs[i] = 0.f; }
      g.counter = *d.counter;
      g.col_tests = 0;
      *r.diag = g;
    }
    ctl->updated = 1;
  }
}

__global__ void __maxnreg__(64) k_post(KArgs a) {
  extern __shared__ __align__(16) int smem_post[];
  cg::cluster_group cluster = cg::this_cluster();
  // launched as a programmatic dependent of the rollout kernel before it in
  // the stream, which lets it be scheduled once every rollout CTA has begun:
  // its CTAs take the SMs as the rollouts' last CTAs leave them and wait here
  // for that grid's completion (its records, the control block)
  pdl_wait();
  {
    // (the flag is the track kernel's, the same for every CTA of the cluster)
    const int inst = blockIdx.x / cluster.num_blocks();
    const InstDesc& d = desc_of(a, inst);
    if (d.ctl->rejected) {
      if (cluster.block_rank() == 0) refuse_replan(d, req_of(a, inst));
      return;
    }
  }
  // the angular DBSCAN's bucket tables (ordered before its atomics by the
  // prune stage's cluster barriers)
  ang_reset(db_work_of(desc_of(a, blockIdx.x / cluster.num_blocks())));
  // stage clock stamps of rank 0 (diagnostics): start, after prune, after DBSCAN
  long long* cyc = desc_of(a, blockIdx.x / cluster.num_blocks()).ctl->dbcyc;
  const bool st = threadIdx.x == 0 && cluster.block_rank() == 0;
  if (st) cyc[9] = clock64();
  prune_stage(a, true);
  cluster.sync();   // lists, features and the control block of the instance
  if (st) cyc[10] = clock64();
  dbscan_stage(a, smem_post);
  cluster.sync();   // labels, cluster count and mode; DBSCAN tables no longer read
  if (st) cyc[11] = clock64();
  select_stage(a, *reinterpret_cast<SelSmem*>(smem_post), true);
}

// ========================================================================= update
__device__ void finalize(const InstDesc& d, const Req& r);
// Eq. 20 / Eq. 7: U_new[c] = U[c] + sum_k w_k eps'[c][k] (Kahan, fixed order),
// then, in the last CTA of the instance, the outputs, the receding-horizon
// shift of the nominal, x_next = f(x0, u_0), the diagnostics and the counter.
// x <- f(x, u): one model step of the controller's own dynamics (the state
// x_next handed back with the replan).
__device__ __forceinline__ void step_model(const InstDesc& d, float* x, const float* u) {
  const float dt = d.dt;
  if (d.dyn == CE_DYN_DOUBLE_INT_2D) {
    x[0] += x[2] * dt; x[1] += x[3] * dt; x[2] += u[0] * dt; x[3] += u[1] * dt;
  } else if (d.dyn == CE_DYN_UNICYCLE) {
    float sn, cs;
    sincosf(x[2], &sn, &cs);
    x[0] += u[0] * cs * dt; x[1] += u[0] * sn * dt; x[2] += u[1] * dt;
  } else if (d.dyn == CE_DYN_ARM6_KIN) {
    for (int i = 0; i < 6; ++i) x[i] += u[i] * dt;
  } else {
    for (int i = 0; i < 6; ++i) { x[i] += x[6 + i] * dt; x[6 + i] += u[i] * dt; }
  }
}

__device__ void finalize(const InstDesc& d, const Req& r) {
  Ctl* ctl = d.ctl;
  const int T = d.T, m = d.m, TM = T * m;
  for (int c = threadIdx.x; c < TM; c += blockDim.x) {
    const float v = __ldcg(d.Unew + c);
    if (r.u_out) r.u_out[c] = v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < TM; c += blockDim.x) {
    const int j = c / m, dd = c - j * m;
    const int src = j + 1 < T ? j + 1 : T - 1;
    d.U[c] = __ldcg(d.Unew + src * m + dd);
  }
  if (threadIdx.x == 0) {
    if (r.x_next) {
      float x[12], u[6];
      for (int i = 0; i < d.n; ++i) x[i] = r.x0[i];
      for (int i = 0; i < m; ++i) u[i] = __ldcg(d.Unew + i);
      step_model(d, x, u);
      for (int i = 0; i < d.n; ++i) r.x_next[i] = x[i];
    }
    const unsigned long long c = *d.counter;
    if (r.diag) {
      ce_mppi_diag g;
      memset(&g, 0, sizeof(g));
      g.mode = ctl->mode; g.n_col = ctl->nC; g.n_valid = ctl->nV; g.n_clusters = ctl->M;
      g.sel_label = ctl->sel; g.o_star = ctl->o_star; g.dynamic = ctl->dynamic;
      g.status = ctl->status; g.S_min = ctl->S_min;
      for (int i = 0; i < 3; ++i) { g.pbar[i] = ctl->pbar[i]; g.v_obs[i] = ctl->v_obs[i]; }
      g.counter = c;
      g.col_tests = ctl->col_tests;
      *r.diag = g;
    }
    ctl->counter_used = c;
    *d.counter = c + 1;
    ctl->done = 0u;
  }
}

// The tiled update over the whole GPU (k_update).  2-D layout eps[T*m][Kp]:
// tile = (32 columns, kUpdChunk2D rollouts), a warp per four columns (one
// Philox block when eps' is drawn again) with lanes over k (coalesced).  Arm
// layout eps[Kp][T*m]: tile = (32 columns, kUpdChunkArm rollouts), lanes over
// the columns, each warp a contiguous block of rows.  Each tile writes its
// partial sums; the last tile of the instance adds them in chunk order
// (deterministic) and finalizes.
// The fused per-instance kernel's update when at most kSparseMax weights are
// nonzero (rank 0 of the cluster, all columns): U_new[c] = U[c] + (1/Z) sum_j
// w_j eps'[c][k_j] over the list in ascending k (Kahan), then the finalize --
// the list, 1/Z, the nominal and the finalize's inputs from shared memory
// (read at the start of the selection), U_new kept there too.
__device__ void finalize_fused(const InstDesc& d, const Req& r, const SelSmem& sm);
__device__ __forceinline__ void update_sparse_finalize(const KArgs& a, const InstDesc& d,
                                                       int inst, SelSmem& sm) {
  Ctl* ctl = d.ctl;
  const int TM = d.T * d.m, nnz = sm.nnz;
  const bool arm = is_arm(d.dyn);
  const float iz = sm.invZ;
  const unsigned long long ctr = sm.ctr;
  const int* nzk = sm.sk;
  const float* nze = sm.se;
  // the products w_j eps'_j[c] of JB list entries at a time are formed by all
  // threads at once (independent loads, or one Philox block of four columns
  // per thread), then each column's thread adds them in list order (Kahan)
  __shared__ float prod[kUpdProdMax];
  const bool regen = d.regen;
  const int NB = (TM + 3) >> 2;   // Philox blocks of a rollout's columns
  const int per = regen ? NB : TM;   // threads per list entry
  const int JB = max(1, min(kUpdProdMax / max(TM, 1), (int)blockDim.x / max(per, 1)));
  float s = 0.f, e = 0.f;   // column threadIdx.x (one pass)
  const bool one_pass = TM <= (int)blockDim.x && TM * JB <= kUpdProdMax;
  if (one_pass) {
    for (int j0 = 0; j0 < nnz; j0 += JB) {
      const int jn = min(JB, nnz - j0);
      if (regen) {
        for (int t = threadIdx.x; t < jn * NB; t += blockDim.x) {
          const int jj = t / NB, b = t - jj * NB, k = nzk[j0 + jj];
          const float wj = nze[j0 + jj];
          float x[4];
          eps_regen4(d, ctr, k, b, TM, x);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (4 * b + q < TM) prod[jj * TM + 4 * b + q] = wj * x[q];
        }
      } else {
        for (int t = threadIdx.x; t < jn * TM; t += blockDim.x) {
          const int jj = t / TM, c = t - jj * TM, k = nzk[j0 + jj];
          const float x = arm ? d.eps[(size_t)k * d.eps_ld_k + c] : d.eps[(size_t)c * d.eps_ld_c + k];
          prod[t] = nze[j0 + jj] * x;
        }
      }
      __syncthreads();
      if ((int)threadIdx.x < TM)
        for (int jj = 0; jj < jn; ++jj) kahan_add(s, e, prod[jj * TM + threadIdx.x]);
      __syncthreads();
    }
    if ((int)threadIdx.x < TM) {
      const float v = sm.Us[threadIdx.x] + s * iz;
      sm.Un[threadIdx.x] = v;
      d.Unew[threadIdx.x] = v;
    }
  } else {
    for (int c = threadIdx.x; c < TM; c += blockDim.x) {
      float sc = 0.f, ec = 0.f;
      for (int j = 0; j < nnz; ++j) {
        const int k = nzk[j];
        const float x = d.regen ? eps_regen(d, ctr, k, c)
                        : arm   ? d.eps[(size_t)k * d.eps_ld_k + c]
                                : d.eps[(size_t)c * d.eps_ld_c + k];
        kahan_add(sc, ec, nze[j] * x);
      }
      const float v = sm.Us[c] + sc * iz;
      sm.Un[c] = v;
      d.Unew[c] = v;
    }
  }
  __syncthreads();
  finalize_fused(d, req_of(a, inst), sm);
  if (threadIdx.x == 0) ctl->updated = 1;
}

// The finalize of the fused kernel's rank 0 from shared memory: the outputs,
// the receding-horizon shift, x_next = f(x0, u_0), the diagnostics (fields
// read at the start of the selection; mode, c*, S_min from the selection) and
// the counter.  The same values as finalize.
__device__ void finalize_fused(const InstDesc& d, const Req& r, const SelSmem& sm) {
  Ctl* ctl = d.ctl;
  const int T = d.T, m = d.m, TM = T * m;
  for (int c = threadIdx.x; c < TM; c += blockDim.x) {
    if (r.u_out) r.u_out[c] = sm.Un[c];
    const int j = c / m, dd = c - j * m;
    const int src = j + 1 < T ? j + 1 : T - 1;
    d.U[c] = sm.Un[src * m + dd];
  }
  if (threadIdx.x == 0) {
    if (r.x_next) {
      float x[12], u[6];
      for (int i = 0; i < d.n; ++i) x[i] = sm.x0s[i];
      for (int i = 0; i < m; ++i) u[i] = sm.Un[i];
      step_model(d, x, u);
      for (int i = 0; i < d.n; ++i) r.x_next[i] = x[i];
    }
    const unsigned long long c = sm.ctr;
    if (r.diag) {
      const ce_mppi_diag& f = sm.dg;
      ce_mppi_diag g;
      memset(&g, 0, sizeof(g));   // (padding bytes too: the outputs are compared bitwise)
      g.mode = f.mode; g.n_col = f.n_col; g.n_valid = f.n_valid; g.n_clusters = f.n_clusters;
      g.sel_label = f.sel_label; g.o_star = f.o_star; g.dynamic = f.dynamic;
      g.status = f.status; g.S_min = f.S_min;
      for (int i = 0; i < 3; ++i) { g.pbar[i] = f.pbar[i]; g.v_obs[i] = f.v_obs[i]; }
      g.counter = c;
      g.col_tests = f.col_tests;
      *r.diag = g;
    }
    ctl->counter_used = c;
    *d.counter = c + 1;
    ctl->done = 0u;
  }
}

__global__ void __launch_bounds__(kUpdateWarps * 32) k_update(KArgs a) {
  __shared__ float part[kUpdateWarps][32];
  __shared__ float wtile[kUpdChunkArm];   // arm, eps' stored: the warps' lists of
  __shared__ int rtile[kUpdChunkArm];     // nonzero weights and their rows
  __shared__ int last;
  // a track kernel launched behind this one (a pipelined half's next replan)
  // may be scheduled at once; it waits for this grid's completion
  pdl_trigger();
  const int2 tile = tile_of(a);
  const InstDesc& d = desc_of(a, tile.x);
  pdl_wait();   // (launched as a programmatic dependent of the clustering kernel)
  if (d.ctl->updated) return;   // done by the fused per-instance kernel
  if (d.ctl->rejected) {        // inputs refused by the track kernel: no update
    if (tile.y == 0) refuse_replan(d, req_of(a, tile.x));
    return;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int K = d.K, TM = d.T * d.m;
  const bool arm = is_arm(d.dyn);
  const int kch = arm ? kUpdChunkArm : kUpdChunk2D;
  const int cper = 32;   // columns per tile (2-D: four per warp; arm: one per lane)
  const int ncb = (TM + cper - 1) / cper;
  const int cb = tile.y % ncb, kc = tile.y / ncb;
  const int c0 = cb * cper, k0 = kc * kch, k1 = min(K, k0 + kch);
  const float* __restrict__ w = d.w_k;
  const float* __restrict__ eps = d.eps;
  const int nnz = d.ctl->nnz;
  const unsigned long long ctr = *d.counter;   // this replan's (finalize advances it)
  const bool regen = d.regen;
  if (nnz >= 0) {
    // few nonzero weights, listed by ascending k: the tiles of the first
    // rollout chunk sum over the list, the others contribute zeros
    if (!arm) {
      // warp wid: the four columns of one Philox block, lanes over the list
      const int cw = c0 + 4 * wid;
      if (cw < TM) {
        float s[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
        if (kc == 0)
          for (int j = lane; j < nnz; j += 32) {
            const int k = d.nzk[j];
            float x[4] = {0.f, 0.f, 0.f, 0.f};
            if (regen) {
              eps_regen4(d, ctr, k, cw >> 2, TM, x);
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (cw + q < TM) x[q] = eps[(size_t)(cw + q) * d.eps_ld_c + k];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) kahan_add(s[q], e[q], d.nze[j] * x[q]);
          }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float t = warp_sum(s[q]);
          if (lane == 0 && cw + q < TM) d.upart[(size_t)kc * d.TMp + cw + q] = t;
        }
      }
    } else {
      const int c = c0 + lane;
      float s = 0.f, e = 0.f;
      if (kc == 0 && c < TM)
        for (int j = wid; j < nnz; j += kUpdateWarps) {
          const int k = d.nzk[j];
          kahan_add(s, e, d.nze[j] * (d.regen ? eps_regen(d, ctr, k, c)
                                               : eps[(size_t)k * d.eps_ld_k + c]));
        }
      part[wid][lane] = s;
      __syncthreads();
      if (wid == 0 && c < TM) {
        float t = 0.f;
        for (int q = 0; q < kUpdateWarps; ++q) t += part[q][lane];
        d.upart[(size_t)kc * d.TMp + c] = t;
      }
    }
  } else if (!arm) {
    // dense: warp wid takes the four columns of one Philox block, lanes the
    // tile's rollouts (k in steps of 32, Kahan per column); eps' is read (or
    // drawn again, one Philox block for the four columns) only where the
    // weight is nonzero -- with the least cost subtracted, exp underflows to
    // exactly 0 for most rollouts at small lambda, and adding 0 keeps the
    // sums' bits as if they were read.  The same order either way.
    const int cw = c0 + 4 * wid;
    if (cw < TM) {
      float s[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
      if (regen) {
        for (int k = k0 + lane; k < k1; k += 32) {
          const float wk = w[k];
          if (wk == 0.f) continue;
          float x[4];
          eps_regen4(d, ctr, k, cw >> 2, TM, x);
#pragma unroll
          for (int q = 0; q < 4; ++q) kahan_add(s[q], e[q], wk * x[q]);
        }
      } else {
        // kUpdUnroll rollouts per lane in flight: their weights, then the
        // eps' of the nonzero ones, all loaded before the first add (the
        // adds keep the order of the plain loop)
        for (int kb = k0 + lane; kb < k1; kb += 32 * kUpdUnroll) {
          float wk[kUpdUnroll], x[kUpdUnroll][4];
#pragma unroll
          for (int u = 0; u < kUpdUnroll; ++u) {
            const int k = kb + 32 * u;
            wk[u] = k < k1 ? w[k] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < kUpdUnroll; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q)
              x[u][q] = (wk[u] != 0.f && cw + q < TM)
                            ? eps[(size_t)(cw + q) * d.eps_ld_c + kb + 32 * u] : 0.f;
#pragma unroll
          for (int u = 0; u < kUpdUnroll; ++u)
            if (wk[u] != 0.f)
#pragma unroll
              for (int q = 0; q < 4; ++q) kahan_add(s[q], e[q], wk[u] * x[u][q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float t = warp_sum(s[q]);
        if (lane == 0 && cw + q < TM) d.upart[(size_t)kc * d.TMp + cw + q] = t;
      }
    }
  } else {
    const int c = c0 + lane;
    float s = 0.f, e = 0.f;
    // warp wid takes the rows [k0 + wid R, k0 + (wid + 1) R) in order, lanes
    // the columns; rows of zero weight are neither read (or drawn) nor added
    constexpr int R = kUpdChunkArm / kUpdateWarps;
    const int r0 = wid * R, r1 = min(r0 + R, k1 - k0);
    if (!regen) {
      // the warp's rows of nonzero weight listed in ascending order (weight,
      // row) in its own segment of shared memory, padded with zero weights
      // to a multiple of kUpdArmUnroll; then kUpdArmUnroll rows at a time,
      // every load in bounds and issued before the first add (a padded entry
      // reads a listed row and is not added: the adds are those of the plain
      // loop over the nonzero rows)
      float* wl = wtile + r0;
      int* rl = rtile + r0;
      int n = 0;
      float wv[R / 32];   // the warp's weights, all loads in flight at once
#pragma unroll
      for (int j = 0; j < R / 32; ++j) {
        const int r = r0 + 32 * j + lane;
        wv[j] = r < r1 ? w[k0 + r] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < R / 32; ++j) {
        const unsigned nz = __ballot_sync(FULL, wv[j] != 0.f);
        if (wv[j] != 0.f) {
          const int pos = n + __popc(nz & ((1u << lane) - 1u));
          wl[pos] = wv[j];
          rl[pos] = r0 + 32 * j + lane;
        }
        n += __popc(nz);
      }
      __syncwarp();
      const int npad = (n + kUpdArmUnroll - 1) / kUpdArmUnroll * kUpdArmUnroll;
      for (int i = n + lane; i < npad; i += 32) {
        wl[i] = 0.f;
        rl[i] = rl[0];
      }
      __syncwarp();
      const int cc = min(c, TM - 1);
      for (int i = 0; i < npad; i += kUpdArmUnroll) {
        float x[kUpdArmUnroll];
#pragma unroll
        for (int u = 0; u < kUpdArmUnroll; ++u)
          x[u] = eps[(size_t)(k0 + rl[i + u]) * d.eps_ld_k + cc];
#pragma unroll
        for (int u = 0; u < kUpdArmUnroll; ++u) {
          const float wk = wl[i + u];
          if (wk != 0.f) kahan_add(s, e, wk * x[u]);
        }
      }
    } else if (c < TM) {
      for (int r = r0; r < r1; ++r) {
        const float wk = w[k0 + r];   // warp-uniform
        if (wk != 0.f) kahan_add(s, e, wk * eps_regen(d, ctr, k0 + r, c));
      }
    }
    part[wid][lane] = s;
    __syncthreads();
    if (wid == 0 && c < TM) {
      float t = 0.f;
      for (int q = 0; q < kUpdateWarps; ++q) t += part[q][lane];
      d.upart[(size_t)kc * d.TMp + c] = t;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ntile = (unsigned)(ncb * ((K + kch - 1) / kch));
    last = atomicAdd(&d.ctl->done, 1u) == ntile - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int nkc = (K + kch - 1) / kch;
  const float iz = __ldcg(&d.ctl->invZ);
  for (int c = threadIdx.x; c < TM; c += blockDim.x) {
    float t = 0.f;
    for (int q = 0; q < nkc; ++q) t += __ldcg(d.upart + (size_t)q * d.TMp + c);
    d.Unew[c] = d.U[c] + t * iz;
  }
  __threadfence();
  __syncthreads();
  finalize(d, req_of(a, tile.x));
}

// ========================================================================= launchers
// Cluster sizes of a per-instance kernel: the largest of 8, 4, 2 CTAs of which
// the device can hold n_conc clusters at once (queried once per kernel and
// size; clusters must fit in one GPC), else 1.
struct ClusterFit {
  int max_active[4] = {0, 0, 0, 0};   // clusters of 1, 2, 4, 8 CTAs
};

template <typename... Args>
static ClusterFit query_fit(void (*kern)(Args...), int threads, size_t smem) {
  ClusterFit f;
  for (int i = 0; i < 4; ++i) {
    const int cl = 1 << i;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cl);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    f.max_active[i] = n;
  }
  return f;
}

static int cluster_ctas(const ClusterFit& f, int n_conc) {
  for (int i = 3; i >= 1; --i)
    if (f.max_active[i] >= n_conc) return 1 << i;
  return 1;
}

static ClusterFit g_fit_prune, g_fit_select;
// DBSCAN: the fit depends on the shared memory of the launch (by grid size)
constexpr int kFitCells[3] = {256, 1024, kMaxCells};   // grid-size classes
static ClusterFit g_fit_db[3];
static size_t dbscan_smem(int nc);
static int fit_class(int nc) { return nc <= kFitCells[0] ? 0 : nc <= kFitCells[1] ? 1 : 2; }

template <typename... Args>
static void launch_clustered(void (*kern)(Args...), int cl, int n_inst, int threads, size_t smem,
                             cudaStream_t s, cudaEvent_t started, bool dependent, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_inst * cl));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[3];
  unsigned n = 0;
  if (dependent) {   // (the kernel waits for the grid before it: pdl_wait)
    at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
  }
  if (cl > 1) {   // (one CTA per instance: no cluster)
    at[n].id = cudaLaunchAttributeClusterDimension;
    at[n].val.clusterDim.x = (unsigned)cl;
    at[n].val.clusterDim.y = 1;
    at[n].val.clusterDim.z = 1;
    ++n;
  }
  if (started) {   // fires once every CTA has begun execution
    at[n].id = cudaLaunchAttributeLaunchCompletionEvent;
    at[n].val.launchCompletionEvent.event = started;
    at[n].val.launchCompletionEvent.flags = 0;
    ++n;
  }
  cfg.attrs = at;
  cfg.numAttrs = n;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

void launch_prune(const KArgs& a, cudaStream_t s, cudaEvent_t started) {
  const int cl = cluster_ctas(g_fit_prune, a.n_conc > 0 ? a.n_conc : a.n_inst);
  launch_clustered(k_prune, cl, a.n_inst, kBlock, 0, s, started, false, a);
}

// (2-D sets may take the angular method, whose tables are kAngSmemInts ints)
static size_t dbscan_smem(int nc) {
  return std::max(dbscan_smem_bytes(nc), sizeof(int) * (size_t)kAngSmemInts);
}

static ClusterFit g_fit_post[3];
static size_t post_smem(int nc) { return std::max(dbscan_smem(nc), sizeof(SelSmem)); }

bool launch_post(const KArgs& a, int max_cells, cudaStream_t s, cudaEvent_t started) {
  if (max_cells > kMaxCells) return false;
  const int fc = fit_class(max_cells);
  const size_t smem = post_smem(kFitCells[fc]);   // the class's size (a fit was queried for it)
  const ClusterFit& f = g_fit_post[fc];
  if (f.max_active[0] == 0) return false;   // (the launch would not fit)
  const int cl = a.post_ctas > 0 ? a.post_ctas : cluster_ctas(f, a.n_conc > 0 ? a.n_conc : a.n_inst);
  launch_clustered(k_post, cl, a.n_inst, kBlock, smem, s, started, true, a);
  return true;
}

// Kernel attributes of the current device (shared-memory limits); with
// `fits`, also the cluster-size fits (queried once per process, on the first
// device configured: the devices of one process are taken to be one model).
void configure_cluster(bool fits) {
  cudaFuncSetAttribute(k_dbscan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)dbscan_smem(kMaxCells));
  cudaFuncSetAttribute(k_dbscan_standalone, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)dbscan_smem(kMaxCells));
  cudaFuncSetAttribute(k_post, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)post_smem(kMaxCells));
  if (!fits) return;
  g_fit_prune = query_fit(k_prune, kBlock, 0);
  g_fit_select = query_fit(k_select, kBlock, 0);
  for (int c = 0; c < 3; ++c) g_fit_db[c] = query_fit(k_dbscan, kBlock, dbscan_smem(kFitCells[c]));
  for (int c = 0; c < 3; ++c) g_fit_post[c] = query_fit(k_post, kBlock, post_smem(kFitCells[c]));
}

void launch_dbscan(const KArgs& a, int max_cells, cudaStream_t s) {
  const int fc = fit_class(max_cells);
  const size_t smem = dbscan_smem(kFitCells[fc]);
  const int cl = cluster_ctas(g_fit_db[fc], a.n_conc > 0 ? a.n_conc : a.n_inst);
  launch_clustered(k_dbscan, cl, a.n_inst, kBlock, smem, s, nullptr, false, a);
}

void launch_select(const KArgs& a, cudaStream_t s) {
  const int cl = cluster_ctas(g_fit_select, a.n_conc > 0 ? a.n_conc : a.n_inst);
  launch_clustered(k_select, cl, a.n_inst, kBlock, 0, s, nullptr, false, a);
}

// A programmatic dependent of the kernel before it in the stream (the fused
// clustering kernel, or the selection kernel): scheduled once that kernel's
// rank-0 CTAs reach their tail, it waits for its completion (pdl_wait).
void launch_update(const KArgs& a, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)a.n_tiles);
  cfg.blockDim = dim3((unsigned)(kUpdateWarps * 32));
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_update, a);
}

void launch_dbscan_standalone(const float* z, int n, int ld, int p, float eps2, float cell_inv,
                              int G, int R, int min_pts, int* labels, int* n_clusters, void* ws,
                              cudaStream_t s) {
  const int nc = p == 3 ? G * G * G : G * G;
  const int ldn = (n + 31) & ~31;
  DbWork w;
  char* b = static_cast<char*>(ws);
  w.cell = reinterpret_cast<int*>(b); b += sizeof(int) * ldn;
  w.sorted = reinterpret_cast<int*>(b); b += sizeof(int) * ldn;
  w.core = reinterpret_cast<int*>(b); b += sizeof(int) * ldn;
  w.zs = reinterpret_cast<float*>(b); b += sizeof(float) * 3 * ldn;
  w.ld_s = ldn;
  w.bbox = reinterpret_cast<float*>(b); b += sizeof(float) * 6 * kMaxCells;
  w.ahist = reinterpret_cast<int*>(b); b += sizeof(int) * kAngBuckets;
  w.amin = reinterpret_cast<int*>(b);
  const int fc = fit_class(nc);
  const size_t smem = dbscan_smem(kFitCells[fc]);
  const int cl = cluster_ctas(g_fit_db[fc], 1);
  launch_clustered(k_dbscan_standalone, cl, 1, kBlock, smem, s, nullptr, false, z, n, ld, p, eps2, cell_inv, G, R,
                   min_pts, labels, n_clusters, w);
}

size_t dbscan_ws_bytes(int n) {
  const size_t ldn = (size_t)((n + 31) & ~31);
  return ldn * (3 * sizeof(int) + 3 * sizeof(float)) + (size_t)kMaxCells * 6 * sizeof(float) +
         2 * sizeof(int) * (size_t)kAngBuckets;
}

}  // namespace cem
