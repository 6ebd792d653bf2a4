// k_cluster.cu -- pruning, reference point and features, grid-binned DBSCAN,
// cluster statistics and selection, and the softmin-weighted update of the
// CE-MPPI replan (Algorithm 1 after [Rollouts]).
//
// Every reduction here is deterministic: float sums run in an order fixed by
// K alone (thread t takes elements t, t + blockDim, ...; fixed shuffle trees),
// and per-cluster sums use exact int64 fixed-point atomics, so a replan gives
// the same bits alone and inside any batch.
#include "ce_mppi_internal.cuh"

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

// Deterministic block sum (warp trees, then warp 0 over the warp partials).
__device__ __forceinline__ float block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float t = 0.0f;
  if (wid == 0) {
    t = warp_sum(lane < nw ? red[lane] : 0.0f);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  t = red[32];
  __syncthreads();
  return t;
}

__device__ __forceinline__ float block_max(float v, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    float t = lane < nw ? red[lane] : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmaxf(t, __shfl_xor_sync(FULL, t, o));
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  const float r = red[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void task_pos0(const InstDesc& d, const float* x0, float* p0) {
  if (d.dyn == CE_DYN_ARM6_KIN) {
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
__global__ void __launch_bounds__(kBlock) k_prune(KArgs a) {
  const int inst = blockIdx.x;
  const InstDesc& d = a.D[inst];
  const Req& r = req_of(a, inst);
  Ctl* ctl = d.ctl;
  __shared__ int wsum[33];
  __shared__ float red[33];
  __shared__ unsigned hitmask[kMaxObs / 32];
  __shared__ unsigned long long best;
  __shared__ float p0s[3];
  const int K = d.K, Kp = d.Kp, p = d.p, n_obs = r.n_obs, tid = threadIdx.x;
  for (int i = tid; i < (n_obs + 31) / 32; i += blockDim.x) hitmask[i] = 0u;
  if (tid == 0) {
    best = ~0ull;
    task_pos0(d, r.x0, p0s);
  }
  __syncthreads();
  int nV = 0, nC = 0;
  for (int k0 = 0; k0 < K; k0 += blockDim.x) {
    const int k = k0 + tid;
    const int h = k < K ? d.hit[k] : -1;
    const bool isV = k < K && h < 0, isC = k < K && h >= 0;
    if (isC) atomicOr(&hitmask[h >> 5], 1u << (h & 31));
    int tV, tC;
    const int rv = block_scan_flag(isV, wsum, &tV);
    const int rc = block_scan_flag(isC, wsum, &tC);
    if (isV) d.idxV[nV + rv] = k;
    if (isC) d.idxC[nC + rc] = k;
    nV += tV;
    nC += tC;
  }
  if (nC == 0 || nV == 0) {
    if (tid == 0) {
      ctl->nV = nV; ctl->nC = nC; ctl->M = 0; ctl->sel = -1; ctl->o_star = -1;
      ctl->dynamic = 0; ctl->mode = nC == 0 ? CE_MODE_NOCOL : CE_MODE_ALLCOL;
      for (int i = 0; i < 3; ++i) { ctl->pbar[i] = 0.f; ctl->v_obs[i] = 0.f; ctl->p0[i] = p0s[i]; }
    }
    return;
  }
  // o*: least clearance |p(x_0) - o_t| - r_o among obstacles hit first by some
  // rollout; ties to the lowest index (packed key, atomicMin).
  const int ts = track_stride(n_obs);
  (void)ts;
  for (int o = tid; o < n_obs; o += blockDim.x) {
    if (!((hitmask[o >> 5] >> (o & 31)) & 1u)) continue;
    const float4 t = d.tracks[o];   // horizon row 0 = newest observation
    const float dx = p0s[0] - t.x, dy = p0s[1] - t.y, dz = p0s[2] - t.z;
    const float clear = sqrtf(dx * dx + dy * dy + dz * dz) - r.obs_radius[o];
    atomicMin(&best, ((unsigned long long)float_key(clear) << 32) | (unsigned)o);
  }
  __syncthreads();
  const int o_star = (int)(best & 0xffffffffull);
  // pbar: mean terminal position of the colliding rollouts whose first hit is
  // o* (ref_mode 0) or of all colliding rollouts (ref_mode 1).
  float acc[3] = {0.f, 0.f, 0.f}, cmp[3] = {0.f, 0.f, 0.f};
  int cnt = 0;
  for (int i = tid; i < nC; i += blockDim.x) {
    const int k = d.idxC[i];
    if (d.ref_mode == 0 && d.hit[k] != o_star) continue;
    ++cnt;
    for (int c = 0; c < p; ++c) kahan_add(acc[c], cmp[c], d.pN[(size_t)c * Kp + k]);
  }
  const float ncnt = block_sum((float)cnt, red);
  float pbar[3] = {0.f, 0.f, 0.f};
  for (int c = 0; c < p; ++c) pbar[c] = block_sum(acc[c], red) / ncnt;
  // features of V
  const float ne = d.norm_eps;
  for (int i = tid; i < nV; i += blockDim.x) {
    const int k = d.idxV[i];
    float dv[3], ev[3], nd = 0.f, nn = 0.f;
    for (int c = 0; c < p; ++c) {
      const float pk = d.pN[(size_t)c * Kp + k];
      dv[c] = pk - pbar[c];
      ev[c] = pk - p0s[c];
      nd += dv[c] * dv[c];
      nn += ev[c] * ev[c];
    }
    const float izd = 1.0f / (sqrtf(nd) + ne), izn = 1.0f / (sqrtf(nn) + ne);
    for (int c = 0; c < p; ++c) {
      d.z[(size_t)c * Kp + i] = dv[c] * izd;
      d.g[(size_t)c * Kp + i] = ev[c] * izn;
    }
  }
  if (tid == 0) {
    const float* h = hist_of(r, d);
    const int H = d.H;
    const float inv = H >= 2 ? 1.0f / ((float)(H - 1) * d.obs_dt) : 0.0f;
    ctl->nV = nV; ctl->nC = nC; ctl->M = 0; ctl->sel = -1; ctl->o_star = o_star;
    ctl->dynamic = 0; ctl->mode = CE_MODE_STATIC;
    for (int c = 0; c < 3; ++c) {
      ctl->pbar[c] = c < p ? pbar[c] : 0.f;
      ctl->p0[c] = p0s[c];
      ctl->v_obs[c] = c < p ? (h[((size_t)(H - 1) * n_obs + o_star) * p + c] -
                               h[(size_t)o_star * p + c]) * inv
                            : 0.f;
    }
  }
}

// ========================================================================= DBSCAN
// Grid-binned DBSCAN over n points z ([p][ld], coordinates in [-1, 1]).  The
// cell side s = 0.99 eps / sqrt(p) makes any two points of one cell neighbours
// (in the FP32 predicate too), so the core points of a cell are connected and
// the union-find runs over cells: two cells join when some core pair between
// them is within eps.  Shared memory: 4 int arrays of G^p (+1) entries.
struct DbWork {
  int* cell;     // [n] cell id of each point
  int* sorted;   // [n] point ids in cell order
  float* zs;     // [p][ld_s] coordinates in cell order
  int ld_s;
  int* core;     // [n] core flag
  float* bbox;   // [ncells][6] core bounding box (min xyz, max xyz)
};

__device__ __forceinline__ bool nb_pred(const float* za, const float* zb, int p, float eps2) {
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

// squared distance from point a to the box [lo, hi] (per coordinate)
__device__ __forceinline__ float box_d2(const float* za, const float* bb, int p) {
  float s = 0.f;
  for (int c = 0; c < p; ++c) {
    const float lo = bb[c], hi = bb[3 + c];
    const float e = za[c] < lo ? lo - za[c] : (za[c] > hi ? za[c] - hi : 0.f);
    s += e * e;
  }
  return s;
}

__device__ int cfind(int* par, int x) {
  for (int it = 0; it < 1 << 20; ++it) {
    const int p = par[x];
    if (p == x) return x;
    const int gp = par[p];
    if (gp != p) atomicMin(&par[x], gp);
    x = gp;
  }
  return x;
}

__device__ bool cunion(int* par, int a, int b) {
  for (int it = 0; it < 1 << 20; ++it) {
    a = cfind(par, a);
    b = cfind(par, b);
    if (a == b) return true;
    if (a > b) { const int t = a; a = b; b = t; }
    const int old = atomicCAS(&par[b], b, a);
    if (old == b) return true;
    b = old;
  }
  return false;
}

__device__ void dbscan_block(const float* __restrict__ z, int ld, int n, int p, float eps2,
                             float cell_inv, int G, int R, int min_pts, DbWork w, int* labels,
                             int* M_out, int* status, int* smem) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
  const int nc = p == 3 ? G * G * G : G * G;
  int* start = smem;            // [nc + 1]
  int* fill = start + nc + 1;   // [nc]   scatter cursor, then min core id of the cell
  int* cpar = fill + nc;        // [nc]   cell union-find parent (-1: no core)
  int* aux = cpar + nc;         // [nc]   component minimum, then canonical id
  __shared__ int wsum[33];
  __shared__ int bad;
  if (tid == 0) bad = 0;
  for (int c = tid; c < nc; c += blockDim.x) start[c] = 0;
  __syncthreads();
  // 1. cell of each point; per-cell counts
  for (int i = tid; i < n; i += blockDim.x) {
    int ci = 0, mul = 1;
    for (int c = 0; c < p; ++c) {
      const float v = z[(size_t)c * ld + i];
      if (!(v >= -1.0f && v <= 1.0f)) bad = 1;
      ci += cell_coord(v, cell_inv, G) * mul;
      mul *= G;
    }
    w.cell[i] = ci;
    atomicAdd(&start[ci], 1);
  }
  __syncthreads();
  // 2. exclusive scan of the counts (each thread a contiguous run of cells)
  {
    const int per = (nc + blockDim.x - 1) / blockDim.x;
    const int c0 = min(tid * per, nc), c1 = min(c0 + per, nc);
    int loc = 0;
    for (int c = c0; c < c1; ++c) loc += start[c];
    // block exclusive scan of loc
    int s = loc;
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
    }
    __syncthreads();
    int run = wsum[wid] + s - loc;
    for (int c = c0; c < c1; ++c) {
      const int cnt = start[c];
      start[c] = run;
      fill[c] = run;
      run += cnt;
    }
    if (tid == 0) start[nc] = n;
  }
  __syncthreads();
  if (bad) {
    for (int i = tid; i < n; i += blockDim.x) labels[i] = -1;
    if (tid == 0) { *M_out = 0; atomicCAS(status, 0, CE_MPPI_ERR_INVALID_ARG); }
    return;
  }
  // 3. scatter into cell order
  for (int i = tid; i < n; i += blockDim.x) {
    const int pos = atomicAdd(&fill[w.cell[i]], 1);
    w.sorted[pos] = i;
    for (int c = 0; c < p; ++c) w.zs[(size_t)c * w.ld_s + pos] = z[(size_t)c * ld + i];
  }
  __syncthreads();
  // 4. core flags: a cell with >= min_pts points is all core; otherwise count
  //    neighbours over the (2R+1)^p surrounding cells, stopping at min_pts.
  for (int i = tid; i < n; i += blockDim.x) {
    const int ci = w.cell[i];
    int core = (start[ci + 1] - start[ci]) >= min_pts;
    if (!core) {
      float za[3];
      for (int c = 0; c < p; ++c) za[c] = z[(size_t)c * ld + i];
      const int cx = ci % G, cy = (ci / G) % G, cz = p == 3 ? ci / (G * G) : 0;
      int count = 0;
      const int zr = p == 3 ? R : 0;
      for (int oz = -zr; oz <= zr && !core; ++oz)
        for (int oy = -R; oy <= R && !core; ++oy)
          for (int ox = -R; ox <= R && !core; ++ox) {
            const int nx = cx + ox, ny = cy + oy, nz = cz + oz;
            if (nx < 0 || ny < 0 || nz < 0 || nx >= G || ny >= G || (p == 3 && nz >= G)) continue;
            const int nb = (nz * G + ny) * G + nx;
            for (int pos = start[nb]; pos < start[nb + 1]; ++pos) {
              float zb[3];
              for (int c = 0; c < p; ++c) zb[c] = w.zs[(size_t)c * w.ld_s + pos];
              if (nb_pred(za, zb, p, eps2) && ++count >= min_pts) { core = 1; break; }
            }
          }
    }
    w.core[i] = core;
  }
  __syncthreads();
  // 5. per-cell core summary: parent, min core id, bounding box of core points
  for (int c = tid; c < nc; c += blockDim.x) { cpar[c] = -1; fill[c] = 0x7fffffff; }
  __syncthreads();
  for (int c = wid; c < nc; c += nwarp) {
    const int s0 = start[c], s1 = start[c + 1];
    if (s0 == s1) continue;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    int mn = 0x7fffffff;
    for (int pos = s0 + lane; pos < s1; pos += 32) {
      const int i = w.sorted[pos];
      if (!w.core[i]) continue;
      mn = min(mn, i);
      for (int q = 0; q < p; ++q) {
        const float v = w.zs[(size_t)q * w.ld_s + pos];
        lo[q] = fminf(lo[q], v);
        hi[q] = fmaxf(hi[q], v);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(FULL, mn, o));
      for (int q = 0; q < 3; ++q) {
        lo[q] = fminf(lo[q], __shfl_xor_sync(FULL, lo[q], o));
        hi[q] = fmaxf(hi[q], __shfl_xor_sync(FULL, hi[q], o));
      }
    }
    if (lane == 0 && mn != 0x7fffffff) {
      cpar[c] = c;
      fill[c] = mn;
      for (int q = 0; q < 3; ++q) { w.bbox[c * 6 + q] = lo[q]; w.bbox[c * 6 + 3 + q] = hi[q]; }
    }
  }
  __syncthreads();
  // 6. cell-level union.  Occupied core cells are listed first; then one warp
  //    per cell A: the lanes screen the neighbour offsets in parallel (B > A,
  //    B has core points, core bounding boxes within eps, not yet joined) and
  //    the warp searches each surviving pair for a core pair within eps.
  int n_occ;
  {
    int base = 0;
    for (int c0 = 0; c0 < nc; c0 += blockDim.x) {
      const int c = c0 + tid;
      const bool occ = c < nc && cpar[c] >= 0;
      int tot;
      const int rk = block_scan_flag(occ, wsum, &tot);
      if (occ) aux[base + rk] = c;
      base += tot;
    }
    n_occ = base;
  }
  __syncthreads();
  {
    const int side = 2 * R + 1, nofs = p == 3 ? side * side * side : side * side;
    for (int ia = wid; ia < n_occ; ia += nwarp) {
      const int A = aux[ia];
      const int ax = A % G, ay = (A / G) % G, az = p == 3 ? A / (G * G) : 0;
      for (int of0 = 0; of0 < nofs; of0 += 32) {
        const int of = of0 + lane;
        bool cand = false;
        int B = -1;
        if (of < nofs) {
          const int ox = of % side - R, oy = (of / side) % side - R;
          const int oz = p == 3 ? of / (side * side) - R : 0;
          const int bx = ax + ox, by = ay + oy, bz = az + oz;
          if (bx >= 0 && by >= 0 && bz >= 0 && bx < G && by < G && (p != 3 || bz < G)) {
            B = (bz * G + by) * G + bx;
            if (B > A && cpar[B] >= 0) {
              float s2 = 0.f;
              for (int q = 0; q < p; ++q) {
                const float g1 = w.bbox[B * 6 + q] - w.bbox[A * 6 + 3 + q];
                const float g2 = w.bbox[A * 6 + q] - w.bbox[B * 6 + 3 + q];
                const float gq = fmaxf(fmaxf(g1, g2), 0.f);
                s2 += gq * gq;
              }
              cand = s2 <= eps2 * 1.0001f + 1e-12f;
            }
          }
        }
        unsigned cm = __ballot_sync(FULL, cand);
        while (cm) {
          const int src = __ffs(cm) - 1;
          cm &= cm - 1;
          const int Bc = __shfl_sync(FULL, B, src);
          int joined = 0;
          if (lane == 0) joined = cfind(cpar, A) == cfind(cpar, Bc);
          if (__shfl_sync(FULL, joined, 0)) continue;   // warp-uniform decision
          bool found = false;
          for (int pa = start[A]; pa < start[A + 1] && !found; pa += 32) {
            bool mine = false;
            const int posa = pa + lane;
            if (posa < start[A + 1] && w.core[w.sorted[posa]]) {
              float za[3];
              for (int q = 0; q < p; ++q) za[q] = w.zs[(size_t)q * w.ld_s + posa];
              if (box_d2(za, w.bbox + Bc * 6, p) <= eps2 * 1.0001f + 1e-12f) {
                for (int pb = start[Bc]; pb < start[Bc + 1]; ++pb) {
                  if (!w.core[w.sorted[pb]]) continue;
                  float zb[3];
                  for (int q = 0; q < p; ++q) zb[q] = w.zs[(size_t)q * w.ld_s + pb];
                  if (nb_pred(za, zb, p, eps2)) { mine = true; break; }
                }
              }
            }
            found = __any_sync(FULL, mine);
          }
          if (found && lane == 0 && !cunion(cpar, A, Bc)) atomicCAS(status, 0, CE_MPPI_ERR_TIMEOUT);
          __syncwarp();
        }
      }
    }
  }
  __syncthreads();
  // 7. components: root cell, component minimum core id
  for (int c = tid; c < nc; c += blockDim.x) aux[c] = 0x7fffffff;
  __syncthreads();
  for (int c = tid; c < nc; c += blockDim.x)
    if (cpar[c] >= 0) {
      const int rt = cfind(cpar, c);
      cpar[c] = rt;
      atomicMin(&aux[rt], fill[c]);
    }
  __syncthreads();
  // 8. canonical ids: rank of each component minimum in point order
  int M = 0;
  for (int i0 = 0; i0 < n; i0 += blockDim.x) {
    const int i = i0 + tid;
    bool first = false;
    int rt = -1;
    if (i < n && w.core[i]) {
      rt = cpar[w.cell[i]];
      first = aux[rt] == i;
    }
    int tot;
    const int rk = block_scan_flag(first, wsum, &tot);
    if (first) fill[rt] = M + rk;   // fill: canonical id of the root cell
    M += tot;
  }
  __syncthreads();
  // 9. labels: core -> its component; border -> component of the lowest-index
  //    core neighbour; else noise.
  for (int i = tid; i < n; i += blockDim.x) {
    const int ci = w.cell[i];
    if (w.core[i]) { labels[i] = fill[cpar[ci]]; continue; }
    float za[3];
    for (int c = 0; c < p; ++c) za[c] = z[(size_t)c * ld + i];
    const int cx = ci % G, cy = (ci / G) % G, cz = p == 3 ? ci / (G * G) : 0;
    int bestb = 0x7fffffff;
    const int zr = p == 3 ? R : 0;
    for (int oz = -zr; oz <= zr; ++oz)
      for (int oy = -R; oy <= R; ++oy)
        for (int ox = -R; ox <= R; ++ox) {
          const int nx = cx + ox, ny = cy + oy, nz = cz + oz;
          if (nx < 0 || ny < 0 || nz < 0 || nx >= G || ny >= G || (p == 3 && nz >= G)) continue;
          const int nb = (nz * G + ny) * G + nx;
          if (cpar[nb] < 0) continue;
          if (box_d2(za, w.bbox + nb * 6, p) > eps2 * 1.0001f + 1e-12f) continue;
          for (int pos = start[nb]; pos < start[nb + 1]; ++pos) {
            const int b = w.sorted[pos];
            if (b >= bestb || !w.core[b]) continue;
            float zb[3];
            for (int c = 0; c < p; ++c) zb[c] = w.zs[(size_t)c * w.ld_s + pos];
            if (nb_pred(za, zb, p, eps2)) bestb = b;
          }
        }
    labels[i] = bestb == 0x7fffffff ? -1 : fill[cpar[w.cell[bestb]]];
  }
  if (tid == 0) *M_out = M;
}

__device__ __forceinline__ DbWork db_work_of(const InstDesc& d) {
  DbWork w;
  w.cell = d.cell;
  w.sorted = d.sorted;
  w.zs = d.zs;
  w.ld_s = d.Kp;
  w.core = d.parent;
  w.bbox = d.bbox;
  return w;
}

__global__ void __launch_bounds__(kBlock) k_dbscan(KArgs a) {
  extern __shared__ int smem_i[];
  const int inst = blockIdx.x;
  const InstDesc& d = a.D[inst];
  Ctl* ctl = d.ctl;
  const int mode = ctl->mode;
  if (mode != CE_MODE_STATIC) return;   // fallback replans skip clustering
  const int nV = ctl->nV;
  const DbWork w = db_work_of(d);
  __shared__ int M;
  dbscan_block(d.z, d.Kp, nV, d.p, d.eps2, d.cell_inv, d.G, d.R, d.min_pts, w, d.label, &M,
               &ctl->status, smem_i);
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->M = M;
    if (M == 0) ctl->mode = CE_MODE_ALLNOISE;
  }
}

__global__ void __launch_bounds__(kBlock) k_dbscan_standalone(const float* z, int n, int ld, int p,
                                                              float eps2, float cell_inv, int G,
                                                              int R, int min_pts, int* labels,
                                                              int* n_clusters, DbWork w) {
  extern __shared__ int smem_i[];
  __shared__ int M;
  __shared__ int status;
  if (threadIdx.x == 0) status = 0;
  __syncthreads();
  dbscan_block(z, ld, n, p, eps2, cell_inv, G, R, min_pts, w, labels, &M, &status, smem_i);
  __syncthreads();
  if (threadIdx.x == 0) *n_clusters = status ? -status : M;
}

// ========================================================================= select
// Algorithm 1 [Cluster stats], [Selection], [Within-cluster weighting]:
// per-cluster count, mean cost Sbar_c (Eq. 14) and mean direction vhat_c
// (Eq. 16) by exact int64 fixed-point sums; c* by Eq. 14 (static) or Eq. 18
// (dynamic, |v_o*| > threshold); then the softmin weights over the update set
// (Eq. 19, or Eq. 6 over all K / over V in the fallbacks), normalised, with
// the minimum subtracted before exp.
constexpr int kWin = 512;   // clusters per statistics window

__global__ void __launch_bounds__(kBlock) k_select(KArgs a) {
  const int inst = blockIdx.x;
  const InstDesc& d = a.D[inst];
  Ctl* ctl = d.ctl;
  __shared__ unsigned long long accS[kWin], accG[3][kWin];
  __shared__ int accN[kWin];
  __shared__ float red[33];
  __shared__ unsigned long long bestkey;
  const int tid = threadIdx.x, lane = tid & 31;
  const int K = d.K, Kp = d.Kp, p = d.p;
  const int mode0 = ctl->mode;
  const int nV = ctl->nV, M = ctl->M;
  int sel = -1, dynamic = 0;
  if (mode0 == CE_MODE_STATIC) {
    // fixed-point scales: S in [-Smax, Smax], g in [-1, 1], at most nV terms
    float sm = 0.f;
    for (int i = tid; i < nV; i += blockDim.x) sm = fmaxf(sm, fabsf(d.S[d.idxV[i]]));
    sm = block_max(sm, red);
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
    for (int w0 = 0; w0 < M; w0 += kWin) {
      for (int c = tid; c < kWin; c += blockDim.x) {
        accS[c] = 0ull; accN[c] = 0;
        accG[0][c] = accG[1][c] = accG[2][c] = 0ull;
      }
      __syncthreads();
      for (int i0 = 0; i0 < nV; i0 += blockDim.x) {
        const int i = i0 + tid;
        int L = -1;
        long long vS = 0, vG[3] = {0, 0, 0};
        if (i < nV) {
          L = d.label[i];
          if (L >= w0 && L < w0 + kWin) {
            vS = __float2ll_rn(ldexpf(d.S[d.idxV[i]], eS));
            for (int q = 0; q < p; ++q) vG[q] = __float2ll_rn(ldexpf(d.g[(size_t)q * Kp + i], eG));
          } else {
            L = -1;
          }
        }
        // one atomic per distinct label present in the warp (exact integer sums)
        unsigned pending = __ballot_sync(FULL, L >= 0);
        while (pending) {
          const int Lw = __shfl_sync(FULL, L, __ffs(pending) - 1);
          const bool mine = L == Lw;
          const unsigned mm = __ballot_sync(FULL, mine);
          long long s = mine ? vS : 0, g0 = mine ? vG[0] : 0, g1 = mine ? vG[1] : 0,
                    g2 = mine ? vG[2] : 0;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(FULL, s, o);
            g0 += __shfl_xor_sync(FULL, g0, o);
            g1 += __shfl_xor_sync(FULL, g1, o);
            g2 += __shfl_xor_sync(FULL, g2, o);
          }
          if (lane == 0) {
            const int c = Lw - w0;
            atomicAdd(&accS[c], (unsigned long long)s);
            atomicAdd(&accG[0][c], (unsigned long long)g0);
            atomicAdd(&accG[1][c], (unsigned long long)g1);
            atomicAdd(&accG[2][c], (unsigned long long)g2);
            atomicAdd(&accN[c], __popc(mm));
          }
          pending &= ~mm;
        }
      }
      __syncthreads();
      for (int c = tid; c < kWin && w0 + c < M; c += blockDim.x) {
        const float n = (float)accN[c];
        float crit;
        if (!dynamic) {
          crit = ldexpf(__ll2float_rn((long long)accS[c]), -eS) / n;
        } else {
          float v[3], nn = 0.f;
          for (int q = 0; q < 3; ++q) {
            v[q] = q < p ? ldexpf(__ll2float_rn((long long)accG[q][c]), -eG) / n : 0.f;
            nn += v[q] * v[q];
          }
          const float iv = 1.0f / (sqrtf(nn) + d.norm_eps);
          crit = (v[0] * iv) * vh[0] + (v[1] * iv) * vh[1] + (v[2] * iv) * vh[2];
        }
        atomicMin(&bestkey, ((unsigned long long)float_key(crit) << 32) | (unsigned)(w0 + c));
      }
      __syncthreads();
    }
    sel = (int)(bestkey & 0xffffffffull);
  }
  // update set membership, S_min, normaliser, weights
  const int mode = mode0 == CE_MODE_STATIC ? (dynamic ? CE_MODE_DYNAMIC : CE_MODE_STATIC) : mode0;
  for (int k = tid; k < K; k += blockDim.x) d.w_k[k] = 0.f;
  __syncthreads();
  const bool over_all = mode == CE_MODE_NOCOL || mode == CE_MODE_ALLCOL;
  const int nIt = over_all ? K : nV;
  float smin = INFINITY;
  for (int i = tid; i < nIt; i += blockDim.x) {
    const bool mem = over_all || mode == CE_MODE_ALLNOISE || d.label[i] == sel;
    if (mem) smin = fminf(smin, d.S[over_all ? i : d.idxV[i]]);
  }
  smin = -block_max(-smin, red);
  const float il = d.inv_lambda;
  float z = 0.f, zc = 0.f;
  for (int i = tid; i < nIt; i += blockDim.x) {
    const bool mem = over_all || mode == CE_MODE_ALLNOISE || d.label[i] == sel;
    if (!mem) continue;
    const int k = over_all ? i : d.idxV[i];
    const float e = expf(-(d.S[k] - smin) * il);
    d.w_k[k] = e;
    kahan_add(z, zc, e);
  }
  const float Z = block_sum(z, red);
  const float iz = 1.0f / Z;
  for (int i = tid; i < nIt; i += blockDim.x) {
    const bool mem = over_all || mode == CE_MODE_ALLNOISE || d.label[i] == sel;
    if (!mem) continue;
    const int k = over_all ? i : d.idxV[i];
    d.w_k[k] = d.w_k[k] * iz;
  }
  if (tid == 0) {
    ctl->mode = mode;
    ctl->sel = sel;
    ctl->dynamic = dynamic;
    ctl->S_min = smin;
    ctl->invZ = iz;
  }
}

// ========================================================================= update
// Eq. 20 / Eq. 7: U_new[c] = U[c] + sum_k w_k eps'[c][k] (Kahan, fixed order),
// then, in the last CTA of the instance, the outputs, the receding-horizon
// shift of the nominal, x_next = f(x0, u_0), the diagnostics and the counter.
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
      float x[6], u[6];
      for (int i = 0; i < d.n; ++i) x[i] = r.x0[i];
      for (int i = 0; i < m; ++i) u[i] = __ldcg(d.Unew + i);
      const float dt = d.dt;
      if (d.dyn == CE_DYN_DOUBLE_INT_2D) {
        x[0] += x[2] * dt; x[1] += x[3] * dt; x[2] += u[0] * dt; x[3] += u[1] * dt;
      } else if (d.dyn == CE_DYN_UNICYCLE) {
        float sn, cs;
        sincosf(x[2], &sn, &cs);
        x[0] += u[0] * cs * dt; x[1] += u[0] * sn * dt; x[2] += u[1] * dt;
      } else {
        for (int i = 0; i < 6; ++i) x[i] += u[i] * dt;
      }
      for (int i = 0; i < d.n; ++i) r.x_next[i] = x[i];
    }
    const unsigned long long c = *d.counter;
    if (r.diag) {
      ce_mppi_diag g;
      g.mode = ctl->mode; g.n_col = ctl->nC; g.n_valid = ctl->nV; g.n_clusters = ctl->M;
      g.sel_label = ctl->sel; g.o_star = ctl->o_star; g.dynamic = ctl->dynamic;
      g.status = ctl->status; g.S_min = ctl->S_min;
      for (int i = 0; i < 3; ++i) { g.pbar[i] = ctl->pbar[i]; g.v_obs[i] = ctl->v_obs[i]; }
      g.counter = c;
      *r.diag = g;
    }
    ctl->counter_used = c;
    *d.counter = c + 1;
    ctl->done = 0u;
  }
}

// 2-D layout eps[T*m][Kp]: one warp per column, lanes over k (coalesced).
// Arm layout eps[Kp][T*m]: lanes over 32 columns, warps over k.
__global__ void __launch_bounds__(kUpdateWarps * 32) k_update(KArgs a) {
  __shared__ float part[kUpdateWarps][32];
  __shared__ int last;
  const int2 tile = a.tiles[blockIdx.x];
  const InstDesc& d = a.D[tile.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int K = d.K, TM = d.T * d.m;
  const float* __restrict__ w = d.w_k;
  const float* __restrict__ eps = d.eps;
  if (d.dyn != CE_DYN_ARM6_KIN) {
    const int c = tile.y + wid;
    if (c < TM) {
      float s = 0.f, sc = 0.f;
      const float* col = eps + (size_t)c * d.eps_ld_c;
      for (int k = lane; k < K; k += 32) kahan_add(s, sc, w[k] * col[k]);
      s = warp_sum(s);
      if (lane == 0) d.Unew[c] = d.U[c] + s;
    }
  } else {
    const int c = tile.y + lane;
    float s = 0.f, sc = 0.f;
    if (c < TM)
      for (int k = wid; k < K; k += kUpdateWarps) kahan_add(s, sc, w[k] * eps[(size_t)k * d.eps_ld_k + c]);
    part[wid][lane] = s;
    __syncthreads();
    if (wid == 0 && c < TM) {
      float t = 0.f;
      for (int q = 0; q < kUpdateWarps; ++q) t += part[q][lane];
      d.Unew[c] = d.U[c] + t;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int per = d.dyn != CE_DYN_ARM6_KIN ? kUpdateWarps : 32;
    const unsigned nblk = (unsigned)((TM + per - 1) / per);
    last = atomicAdd(&d.ctl->done, 1u) == nblk - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  finalize(d, req_of(a, tile.x));
}

// ========================================================================= launchers
void launch_prune(const KArgs& a, cudaStream_t s) { k_prune<<<a.n_inst, kBlock, 0, s>>>(a); }

static size_t dbscan_smem(int nc) { return (size_t)(4 * nc + 1) * sizeof(int); }

void configure_cluster() {
  cudaFuncSetAttribute(k_dbscan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)dbscan_smem(kMaxCells));
  cudaFuncSetAttribute(k_dbscan_standalone, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)dbscan_smem(kMaxCells));
}

void launch_dbscan(const KArgs& a, int max_cells, cudaStream_t s) {
  k_dbscan<<<a.n_inst, kBlock, dbscan_smem(max_cells), s>>>(a);
}

void launch_select(const KArgs& a, cudaStream_t s) { k_select<<<a.n_inst, kBlock, 0, s>>>(a); }

void launch_update(const KArgs& a, cudaStream_t s) {
  k_update<<<a.n_tiles, kUpdateWarps * 32, 0, s>>>(a);
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
  w.bbox = reinterpret_cast<float*>(b);
  (void)nc;
  k_dbscan_standalone<<<1, kBlock, dbscan_smem(nc), s>>>(z, n, ld, p, eps2, cell_inv, G, R,
                                                          min_pts, labels, n_clusters, w);
}

size_t dbscan_ws_bytes(int n) {
  const size_t ldn = (size_t)((n + 31) & ~31);
  return ldn * (3 * sizeof(int) + 3 * sizeof(float)) + (size_t)kMaxCells * 6 * sizeof(float);
}

}  // namespace cem
