// k_rollout.cu -- obstacle tracks and the fused sample + rollout + cost +
// collision kernels of the CE-MPPI replan (Algorithm 1, [Rollouts]).
//
// Noise: normal i of rollout k is element i % 4 of Philox4x32-10 block i / 4
// with counter (k, i / 4, replan_lo, replan_hi) and key (seed_lo, seed_hi),
// generated in registers (never stored as raw noise).  The effective
// perturbation eps' = clip(u + sigma z) - u (Sec. II-A, Eq. 3) is written once
// for the update stage.
#include "ce_mppi_internal.cuh"

namespace cem {

// ------------------------------------------------------------------ tracks
// Eq. 17 telescoped: v_o = (o_t - o_{t-H+1}) / ((H-1) Delta t); the predicted
// centre at horizon step j is o_t + v_o (j dt).  One CTA per instance.
//
// 2-D robots: row j of the table lists, in ascending obstacle index, only the
// obstacles that some rollout can reach at step j: every rollout's position
// lies in a disc of centre c_j and radius r_j fixed by x_0 and the input box
// (unicycle: c_j = p_0, r_j = j dt max|v|; double integrator: c_j = p_0 + j dt
// v_0, r_j = dt^2 j (j-1)/2 |a|max), so an obstacle farther than
// r_j + r_o + r_robot (+1 mm slack) from c_j cannot be hit at step j and is
// left out.  This changes no collision result.  The rows are pairs of steps
// (below): a pair's row lists the obstacles reachable at either step, with
// both centres and a widened radius for one test at the pair's end, so a
// rollout makes one test per entry per two steps and the exact tests only
// where that one passes (consecutive rows share ~97 % of their obstacles, so
// a pair's row is barely longer than one step's).  Rows are packed behind
// the row offsets (a count pass, a scan of the row counts, a write pass).
// Arm: every row holds every obstacle as (x, y, z, r_o + r_robot), rows of
// track_stride entries, then the row counts.
__global__ void __launch_bounds__(1024) k_tracks(KArgs a) {   // (launched with 1024 threads)
  // the rollout kernel that follows may be scheduled at once: its CTAs load
  // the nominal and then wait for this grid to complete (measured: 1.2 %
  // shorter pipelined steps than scheduling it after the table is written)
  pdl_trigger();
  const int inst = blockIdx.x;
  const InstDesc& d = desc_of(a, inst);
  const Req r = req_of(a, inst);
  // every parameter read into registers ahead of the kernel's first store
  // (a later read would wait behind the stores it might alias)
  const int n_obs = r.n_obs, p = d.p, H = d.H, T = d.T, dyn = d.dyn, dn = d.n;
  const float inv = H >= 2 ? 1.0f / ((float)(H - 1) * d.obs_dt) : 0.0f;
  const float dt = d.dt, robot = d.robot_radius;
  const float umin0 = d.u_min[0], umin1 = d.u_min[1], umax0 = d.u_max[0], umax1 = d.u_max[1];
  Ctl* const ctl = d.ctl;
  long long* const osum = d.osum;
  float4* const tracks = d.tracks;
  const bool arm = is_arm(dyn);
  const bool di = dyn == CE_DYN_DOUBLE_INT_2D;
  // (launched as a programmatic dependent of the previous replan's update
  // kernel, a pipelined half's next replan: the replan counter, the state and
  // the control block are that grid's until it completes; descriptor and
  // request above are the host's)
  pdl_wait();
  const float* h = hist_of(r, d);
  const float x0 = r.x0[0], y0 = r.x0[1];
  const float vx0 = di ? r.x0[2] : 0.f;
  const float vy0 = di ? r.x0[3] : 0.f;
  const int ts = track_stride(n_obs);
  int* counts = track_counts(tracks, T, n_obs);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {   // a new replan: clear the control block's flags
    ctl->status = 0;
    ctl->done = 0u;
    ctl->updated = 0;
    ctl->nnz_all = 0;
  }
  // 2-D robots: newest position, velocity and collision radius of the first
  // obstacles, staged in shared memory (their loads in flight together with
  // the input check's first ones)
  constexpr int kObsSmem = 1024;
  __shared__ float4 opv[kObsSmem];
  __shared__ float orr[kObsSmem];
  auto obstacle = [&](int o, float4* pv, float* R) {
    const float* newest = h + ((size_t)(H - 1) * n_obs + o) * 2;
    const float* oldest = h + (size_t)o * 2;
    *pv = make_float4(newest[0], newest[1], (newest[0] - oldest[0]) * inv,
                      (newest[1] - oldest[1]) * inv);
    *R = r.obs_radius[o] + robot;
  };
  {
    // device-buffer inputs are not seen by the host: a NaN or infinity in x0,
    // the observation window or the radii (or a negative radius) is reported
    // as INVALID_ARG in the replan's status, and the replan is refused (the
    // later stages leave the nominal and the counter as they are)
    const int nh = H * n_obs * p, tot = dn + nh + n_obs;
    auto input = [&](int i) {
      return i < dn ? r.x0[i] : i < dn + nh ? h[i - dn] : r.obs_radius[i - dn - nh];
    };
    const int i0 = threadIdx.x;
    const float v0 = i0 < tot ? input(i0) : 0.f;
    if (!arm)
      for (int o = threadIdx.x; o < min(n_obs, kObsSmem); o += blockDim.x)
        obstacle(o, &opv[o], &orr[o]);
    bool bad = i0 < tot && (!isfinite(v0) || (i0 >= dn + nh && !(v0 >= 0.0f)));
    for (int i = i0 + blockDim.x; i < tot; i += blockDim.x) {
      const float v = input(i);
      bad |= !isfinite(v) || (i >= dn + nh && !(v >= 0.0f));
    }
    const bool any_bad = __syncthreads_or(bad);   // (also orders the staged obstacles)
    if (threadIdx.x == 0) {
      ctl->rejected = any_bad ? 1 : 0;
      if (any_bad) raise_status(ctl, CE_MPPI_ERR_INVALID_ARG);
    }
  }
  // per-obstacle sums of the pruning stage, filled by the rollout kernel
  for (int e = threadIdx.x; e < 4 * n_obs; e += blockDim.x) osum[e] = 0;
  if (arm) {
    const int total = (T + 1) * n_obs;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int j = e / n_obs, o = e - j * n_obs;
      const float* newest = h + ((size_t)(H - 1) * n_obs + o) * p;
      const float* oldest = h + (size_t)o * p;
      const float tj = (float)j * dt;
      float c[3];
      for (int i = 0; i < 3; ++i) c[i] = newest[i] + ((newest[i] - oldest[i]) * inv) * tj;
      const float R = r.obs_radius[o] + robot;
      tracks[(size_t)j * ts + o] = make_float4(c[0], c[1], c[2], R);
    }
    for (int j = threadIdx.x; j <= T; j += blockDim.x) counts[j] = n_obs;
    if (threadIdx.x == 0) ctl->col_tests = T * n_obs;
    return;
  }
  const float m0 = fmaxf(fabsf(umin0), fabsf(umax0));
  const float m1 = fmaxf(fabsf(umin1), fabsf(umax1));
  const float amax = sqrtf(m0 * m0 + m1 * m1);
  __shared__ int roff[kMaxT + 2];
  int* off = reinterpret_cast<int*>(tracks);
  float4* ent = reinterpret_cast<float4*>(reinterpret_cast<char*>(tracks) + track_hdr_bytes(T));
  // the reach disc of time step j (centre, radius)
  auto disc = [&](int j, float* cx, float* cy, float* rj) {
    const float tj = (float)j * dt;
    *cx = x0;
    *cy = y0;
    if (di) {
      *cx = x0 + tj * vx0;
      *cy = y0 + tj * vy0;
      *rj = dt * dt * (0.5f * (float)j * (float)(j - 1 > 0 ? j - 1 : 0)) * amax;
    } else {
      *rj = tj * m0;
    }
  };
  const float v0n = sqrtf(vx0 * vx0 + vy0 * vy0);
  const int Q = (T + 1) / 2;   // pairs of steps
  // Row 0: time 0 (the current state, check_j0).  Row q + 1: the pair of
  // steps 2q, 2q + 1, whose end positions are those of times j1 = 2q + 1 and
  // j2 = 2q + 2 (j2 <= T, else one step): the obstacles reachable at either.
  // An entry is two float4: (o(j2), R'^2, index) and (o(j1), R^2, 0), where
  // R' = R + the position's largest move over step j1 + |o(j2) - o(j1)| +
  // slack: a rollout within R of o(j1) at time j1 is within R' of o(j2) at
  // time j2, so one test at the pair's end (against R') finds every pair
  // that may hold a collision, and only those are tested exactly.
  // The entry of obstacle o in row rw; true where it is kept.
  auto entry = [&](int rw, int o, float4* ea, float4* eb) -> bool {
    const int j1 = rw == 0 ? 0 : 2 * rw - 1;
    const bool two = rw > 0 && j1 + 1 <= T;
    const int j2 = two ? j1 + 1 : j1;
    float c1x, c1y, r1, c2x, c2y, r2;
    disc(j1, &c1x, &c1y, &r1);
    disc(j2, &c2x, &c2y, &r2);
    const float t1 = (float)j1 * dt, t2 = (float)j2 * dt;
    // the largest move of the position over step j1 (unicycle: max |v| dt;
    // double integrator: (|v0| + j1 dt |a|max) dt)
    const float smax = di ? (v0n + (float)j1 * dt * amax) * dt : m0 * dt;
    float4 pv;
    float R;
    if (o < kObsSmem) {
      pv = opv[o];
      R = orr[o];
    } else {
      obstacle(o, &pv, &R);
    }
    const float o1x = pv.x + pv.z * t1, o1y = pv.y + pv.w * t1;
    const float o2x = pv.x + pv.z * t2, o2y = pv.y + pv.w * t2;
    const float reach1 = r1 + R + 1e-3f * (1.0f + r1);
    const float reach2 = r2 + R + 1e-3f * (1.0f + r2);
    const float d1x = o1x - c1x, d1y = o1y - c1y, d2x = o2x - c2x, d2y = o2y - c2y;
    const bool keep = d1x * d1x + d1y * d1y <= reach1 * reach1 ||
                      d2x * d2x + d2y * d2y <= reach2 * reach2;
    const float mx = o2x - o1x, my = o2y - o1y;
    const float Rc = R + smax + sqrtf(mx * mx + my * my) + 1e-3f * (1.0f + r2);
    *ea = make_float4(o2x, o2y, rw == 0 ? R * R : Rc * Rc, __int_as_float(o));   // (row 0: an exact test only)
    *eb = make_float4(o1x, o1y, R * R, 0.f);
    return keep;
  };
  // exclusive scan of the Q + 1 row counts (warp 0), 32 at a time with a carry
  auto scan_rows = [&]() {
    if (wid != 0) return;
    int carry = 0;
    for (int j0 = 0; j0 <= Q; j0 += 32) {
      const int j = j0 + lane;
      const int v = j <= Q ? roff[j] : 0;
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (j <= Q) roff[j] = carry + x - v;
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) roff[Q + 1] = carry;
  };
  if (Q + 1 <= nw && n_obs <= 64) {
    // one row per warp, at most two obstacles per lane: the entries stay in
    // registers from the count to the write, computed once
    const int rw = wid;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 ea0 = z4, eb0 = z4, ea1 = z4, eb1 = z4;
    bool k0 = false, k1 = false;
    if (rw <= Q) {
      if (lane < n_obs) k0 = entry(rw, lane, &ea0, &eb0);
      if (32 + lane < n_obs) k1 = entry(rw, 32 + lane, &ea1, &eb1);
    }
    const unsigned b0 = __ballot_sync(0xffffffffu, k0), b1 = __ballot_sync(0xffffffffu, k1);
    if (rw <= Q && lane == 0) roff[rw] = __popc(b0) + __popc(b1);
    __syncthreads();
    scan_rows();
    __syncthreads();
    if (rw <= Q) {
      const unsigned lt = (1u << lane) - 1u;
      const int e0 = roff[rw] + __popc(b0 & lt), e1 = roff[rw] + __popc(b0) + __popc(b1 & lt);
      if (k0) {
        ent[2 * e0] = ea0;
        ent[2 * e0 + 1] = eb0;
      }
      if (k1) {
        ent[2 * e1] = ea1;
        ent[2 * e1 + 1] = eb1;
      }
    }
  } else {
    // pass 0 counts the kept entries of each row, pass 1 writes them
    for (int pass = 0; pass < 2; ++pass) {
      for (int rw = wid; rw <= Q; rw += nw) {
        int cnt = pass ? roff[rw] : 0;
        for (int o0 = 0; o0 < n_obs; o0 += 32) {
          const int o = o0 + lane;
          float4 ea = make_float4(0.f, 0.f, 0.f, 0.f), eb = ea;
          const bool keep = o < n_obs && entry(rw, o, &ea, &eb);
          const unsigned b = __ballot_sync(0xffffffffu, keep);
          if (pass && keep) {
            const int e = cnt + __popc(b & ((1u << lane) - 1u));
            ent[2 * e] = ea;
            ent[2 * e + 1] = eb;
          }
          cnt += __popc(b);
        }
        if (!pass && lane == 0) roff[rw] = cnt;
      }
      __syncthreads();
      if (!pass) scan_rows();
      __syncthreads();
    }
  }
  for (int j = threadIdx.x; j <= Q + 1; j += blockDim.x) off[j] = roff[j];
  // obstacle tests of a rollout at the pairs' ends (row 0 only with check_j0;
  // the exact tests of a pair that may hold a collision come on top)
  if (threadIdx.x == 0) ctl->col_tests = roff[Q + 1] - roff[1];
}

// A rollout CTA whose copy of the track table did not land in time: the
// replan reports TIMEOUT and is refused by the later stages (nominal and
// counter kept), so no rollout record of this launch is ever used.
__device__ __forceinline__ void give_up_replan(Ctl* c) {
  raise_status(c, CE_MPPI_ERR_TIMEOUT);
  atomicExch(&c->rejected, 2);
}

// Stage the instance's tracks and row counts (TMA bulk copy) and the nominal
// into shared memory.  Returns false (the replan given up) if the copy did
// not land in time.
__device__ __forceinline__ bool stage_tracks(const InstDesc& d, int n_obs, float4* trk,
                                             float* Us, uint64_t* bar) {
  const uint32_t bytes = n_obs > 0 ? (uint32_t)track_bytes(d.T, n_obs) : 0u;
  if (threadIdx.x == 0 && bytes > 0) mbar_init(bar, 1);
  for (int i = threadIdx.x; i < d.T * d.m; i += blockDim.x) Us[i] = d.U[i];
  pdl_wait();   // (the nominal is the previous replan's; the table is the track kernel's)
  __syncthreads();
  if (threadIdx.x == 0 && bytes > 0) {
    mbar_expect_tx(bar, bytes);
    bulk_g2s(trk, d.tracks, bytes, bar);
  }
  // the CTA decides together: on a timeout the copy may still be landing, so
  // every thread waits once more (bounded) before the CTA leaves
  const bool ok = __syncthreads_and(bytes == 0 || mbar_wait(bar, 0));
  if (!ok) {
    if (threadIdx.x == 0) give_up_replan(d.ctl);
    mbar_wait(bar, 0);
  }
  return ok;
}

// ------------------------------------------------------------------ 2-D robots
// One thread per rollout.  DYN 0: double integrator (p += v dt; v += a dt),
// cost |p-g|^2 w0 + |u|^2 w1, terminal w2 |p_T - g|^2.  DYN 1: unicycle
// (Eq. 21), cost Eq. 22-23 with Q = w[0..2], H = w[3..5].  Collision: first
// horizon step j (1..T, plus 0 when check_j0) and lowest obstacle index with
// |p_j - o_j|^2 < (r_o + r_robot)^2.
// Shared memory of the 2-D kernel: the nominal, the row offsets of the packed
// table, then an entry buffer of the rest of the launch's dynamic shared
// memory (at least one row of the largest obstacle count).  A table that fits
// arrives by one bulk copy; a larger one is staged in runs of whole rows,
// each run by one bulk copy, the CTA advancing the horizon run by run.
template <int DYN>
__global__ void __launch_bounds__(kRolloutThreads, kRolloutMinCtas) k_rollout2d(KArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // the clustering kernel that follows may be scheduled once every CTA of
  // this grid has begun (it waits for the grid's completion)
  pdl_trigger();
  __shared__ uint64_t bar;
  __shared__ int whole;
  const int2 tile = tile_of(a);
  const InstDesc& d = desc_of(a, tile.x);
  const Req r = req_of(a, tile.x);
  const int n_obs = r.n_obs, T = d.T, Kp = d.Kp;
  const uint32_t us_bytes = ((uint32_t)(T * d.m) * 4u + 15u) & ~15u;
  const uint32_t hdr = (uint32_t)track_hdr_bytes(T);
  float* Us = reinterpret_cast<float*>(smem_raw);
  const int* off = reinterpret_cast<const int*>(smem_raw + us_bytes);
  const float4* buf = reinterpret_cast<const float4*>(smem_raw + us_bytes + hdr);
  const float4* gent =
      reinterpret_cast<const float4*>(reinterpret_cast<const unsigned char*>(d.tracks) + hdr);
  uint32_t cap_b;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(cap_b));
  const int cap_e = (int)((cap_b - us_bytes - hdr) / 32u);   // entries of two float4
  const int Q = (T + 1) / 2;   // rows 1..Q: pairs of steps
  uint32_t phase = 0;
  for (int i = threadIdx.x; i < T * d.m; i += blockDim.x) Us[i] = d.U[i];
  pdl_wait();   // (the nominal is the previous replan's; the table is the track kernel's)
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    const int tot = reinterpret_cast<const int*>(d.tracks)[Q + 1];
    const bool all = tot <= cap_e;
    // everything at once, or the row offsets alone (the runs follow)
    const uint32_t bytes = hdr + (all ? (uint32_t)tot * 32u : 0u);
    mbar_expect_tx(&bar, bytes);
    bulk_g2s(smem_raw + us_bytes, d.tracks, bytes, &bar);
    whole = all;
  }
  __syncthreads();
  // A copy that did not land in time gives the replan up (TIMEOUT; the later
  // kernels refuse it): the thread's rollout is left out, no further copy is
  // issued on this barrier, and the thread waits once more (bounded) for the
  // copy that may still be landing before the CTA leaves.
  bool ok = mbar_wait(&bar, phase);
  uint32_t pend = phase;
  phase ^= 1u;
  const bool all = whole != 0;
  const int k = tile.y * kRolloutThreads + threadIdx.x;
  const bool act = k < d.K && ok;
  const unsigned long long ctr = *d.counter;
  // the Philox key in registers: the step loop's stores may alias the
  // descriptor, which would otherwise be read again for every block
  // (0.1344 -> 0.1336 ms per pipelined step over whole episodes)
  const uint2 key = make_uint2(d.seed_lo, d.seed_hi);

  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  if (act) {
    s0 = r.x0[0]; s1 = r.x0[1]; s2 = r.x0[2]; s3 = DYN == 0 ? r.x0[3] : 0.0f;
  }
  // parameters into registers (the output stores below may alias the descriptor)
  const float dt = d.dt;
  const float g0 = d.goal[0], g1 = d.goal[1], g2 = d.goal[2];
  const float sg0 = d.sigma[0], sg1 = d.sigma[1];
  const float lo0 = d.u_min[0], lo1 = d.u_min[1], hi0 = d.u_max[0], hi1 = d.u_max[1];
  const float w0 = d.w[0], w1 = d.w[1], w2 = d.w[2], w3 = d.w[3], w4 = d.w[4], w5 = d.w[5];
  float* __restrict__ eps = d.eps;
  float S = 0.0f, Sc = 0.0f;
  int first = -1, first_j = -1;
  float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  int j = 0;
  // the collision tests of pair q (steps 2q and, with two, 2q + 1): the
  // position after step 2q was (p1x, p1y), after step 2q + 1 it is (s0, s1).
  // One test per entry at the pair's end against the widened radius; only
  // where one passes, the exact tests of the two steps in turn (descending:
  // the lowest index wins).
  auto pair_test = [&](int q, float p1x, float p1y, bool two, int base) {
    if (first >= 0) return;
    const int e_lo = off[q + 1] - base, e_hi = off[q + 2] - base;
    bool may = !two;
    if (two) {
      // (unrolled by two: 0.1395 against 0.1414 ms per pipelined step with
      // four, 0.1462 with none, 0.1421 with eight)
#pragma unroll 2
      for (int e = e_lo; e < e_hi; ++e) {
        const float4 t = buf[2 * e];
        const float dx = s0 - t.x, dy = s1 - t.y;
        may |= dx * dx + dy * dy < t.z;
      }
    }
    if (may) {
      int h = n_obs;
      for (int e = e_hi - 1; e >= e_lo; --e) {
        const float4 t = buf[2 * e + 1];
        const float dx = p1x - t.x, dy = p1y - t.y;
        h = (dx * dx + dy * dy < t.z) ? __float_as_int(buf[2 * e].w) : h;
      }
      if (h < n_obs) {
        first = h;
        first_j = 2 * q + 1;
      } else if (two) {
        for (int e = e_hi - 1; e >= e_lo; --e) {
          const float4 t = buf[2 * e];
          const float dx = s0 - t.x, dy = s1 - t.y;
          h = (dx * dx + dy * dy < buf[2 * e + 1].z) ? __float_as_int(t.w) : h;
        }
        if (h < n_obs) {
          first = h;
          first_j = 2 * q + 2;
        }
      }
    }
  };
  // runs of rows [ra, rb): row 0 (the current state, only with check_j0),
  // row q + 1 the pair of steps 2q, 2q + 1
  for (int ra = 0; ra <= Q;) {
    int rb = Q + 1;
    if (!all) {
      // (large tables) the CTA agrees that every copy so far has landed
      // before the next one is issued; the previous run's entries are no
      // longer read
      if (!__syncthreads_and(ok)) break;
      rb = ra + 1;
      while (rb <= Q && off[rb + 1] - off[ra] <= cap_e) ++rb;
      if (off[rb] - off[ra] > cap_e) {
        // a row longer than the buffer (the launch's shared memory is sized
        // for the largest row, so this does not happen): the replan is
        // refused instead of copying past the buffer
        if (threadIdx.x == 0) {
          raise_status(d.ctl, CE_MPPI_ERR_INVALID_ARG);
          atomicExch(&d.ctl->rejected, 2);
        }
        ok = false;
        break;
      }
      if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)(off[rb] - off[ra]) * 32u;
        mbar_expect_tx(&bar, bytes);
        if (bytes > 0) bulk_g2s((void*)buf, gent + 2 * (size_t)off[ra], bytes, &bar);
      }
      ok = mbar_wait(&bar, phase);
      pend = phase;
      phase ^= 1u;
    }
    const int base = all ? 0 : off[ra];
    if (ra == 0 && d.check_j0 && act) {
      int h = n_obs;
      for (int e = off[1] - 1 - base; e >= off[0] - base; --e) {
        const float4 t = buf[2 * e];
        const float dx = s0 - t.x, dy = s1 - t.y;
        h = (dx * dx + dy * dy < t.z) ? __float_as_int(t.w) : h;
      }
      if (h < n_obs) { first = h; first_j = 0; }
    }
    const int jend = act ? min(2 * (rb - 1), T) : j;
    const bool store = !d.regen;
    float* ep = store ? eps + (size_t)(2 * j) * Kp + k : nullptr;   // eps' of step j (advances 2 Kp a step)
    // one horizon step's control, cost and motion with normals (z0, z1)
    auto advance = [&](int jj, float z0, float z1) {
      const float n0 = Us[2 * jj], n1 = Us[2 * jj + 1];
      const float u0 = sampled_control(n0, sg0, z0, lo0, hi0);
      const float u1 = sampled_control(n1, sg1, z1, lo1, hi1);
      if (store) {
        ep[0] = u0 - n0;
        ep[Kp] = u1 - n1;
        ep += 2 * (size_t)Kp;
      }
      if (DYN == 0) {
        const float ex = s0 - g0, ey = s1 - g1;
        kahan_add(S, Sc, w0 * (ex * ex + ey * ey) + w1 * (u0 * u0 + u1 * u1));
        s0 += s2 * dt;
        s1 += s3 * dt;
        s2 += u0 * dt;
        s3 += u1 * dt;
      } else {
        const float ex = s0 - g0, ey = s1 - g1, et = s2 - g2;
        kahan_add(S, Sc, w0 * ex * ex + w1 * ey * ey + w2 * et * et);
        // heading sine and cosine on the special-function unit: absolute
        // error ~2^-21 for |theta| up to a few radians, ~1e-6 m of position
        // over the horizon (the full-accuracy call is a long instruction
        // sequence in the kernel's innermost loop)
        float sn, cs;
        __sincosf(s2, &sn, &cs);
        const float vdt = u0 * dt;
        s0 += vdt * cs;
        s1 += vdt * sn;
        s2 += u1 * dt;
      }
    };
    // normals 2j, 2j+1 of step j are elements (2j) % 4, (2j) % 4 + 1 of
    // Philox block j / 2: a pair of steps per block (runs start on even steps)
    for (; j + 1 < jend; j += 2) {
      z4 = philox_normals(key, ctr, k, j >> 1);
      advance(j, z4.x, z4.y);
      const float p1x = s0, p1y = s1;
      advance(j + 1, z4.z, z4.w);
      pair_test(j >> 1, p1x, p1y, true, base);
    }
    if (j < jend) {   // an odd horizon's last step
      z4 = philox_normals(key, ctr, k, j >> 1);
      advance(j, z4.x, z4.y);
      pair_test(j >> 1, s0, s1, false, base);
      ++j;
    }
    ra = rb;
  }
  if (!ok) {
    give_up_replan(d.ctl);
    mbar_wait(&bar, pend);
  }
  if (act) {
    if (DYN == 0) {
      const float ex = s0 - g0, ey = s1 - g1;
      kahan_add(S, Sc, w2 * (ex * ex + ey * ey));
    } else {
      const float ex = s0 - g0, ey = s1 - g1, et = s2 - g2;
      kahan_add(S, Sc, w3 * ex * ex + w4 * ey * ey + w5 * et * et);
    }
    if (first >= 0) kahan_add(S, Sc, d.w[7]);   // collision penalty (0 for CE-MPPI)
    d.S[k] = S;
    d.hit[k] = first;
    d.hitj[k] = first_j;
    d.pN[k] = s0;
    d.pN[Kp + k] = s1;
  }
  // the pruning stage's inputs in aggregate (Eq. 9-11): for this warp's 32
  // rollouts the sizes of V and C_col and the extremes of S; for each
  // obstacle hit first, the count and the fixed-point sum of p(x_T)
  const int lane = threadIdx.x & 31;
  const bool isV = act && first < 0, isC = act && first >= 0;
  const unsigned mv = __ballot_sync(0xffffffffu, isV), mc = __ballot_sync(0xffffffffu, isC);
  float vmax = isV ? fabsf(S) : 0.f, vmin = isV ? S : INFINITY, amin = act ? S : INFINITY;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
    amin = fminf(amin, __shfl_xor_sync(0xffffffffu, amin, o));
  }
  const int g = k >> 5;   // (lane 0's k is a multiple of 32)
  if (lane == 0 && 32 * g < d.K) {
    d.gcnt[g] = make_int2(__popc(mv), __popc(mc));
    d.gS[g] = make_float4(vmax, vmin, amin, 0.f);
  }
  for (unsigned pend = mc; pend;) {   // one round per distinct obstacle
    const int leader = __ffs(pend) - 1;
    const int o = __shfl_sync(0xffffffffu, first, leader);
    const bool mine = isC && first == o;
    const unsigned grp = __ballot_sync(0xffffffffu, mine);
    long long sx = mine ? pos_fixed(s0) : 0ll, sy = mine ? pos_fixed(s1) : 0ll;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, off);
      sy += __shfl_xor_sync(0xffffffffu, sy, off);
    }
    if (lane == leader) {
      long long* os = d.osum + 4 * (size_t)o;
      atomicAdd(reinterpret_cast<unsigned long long*>(os), (unsigned long long)__popc(grp));
      atomicAdd(reinterpret_cast<unsigned long long*>(os + 1), (unsigned long long)sx);
      atomicAdd(reinterpret_cast<unsigned long long*>(os + 2), (unsigned long long)sy);
    }
    pend &= ~grp;
  }
}

// ------------------------------------------------------------------ 6-DoF arm
// One warp per rollout, lane l holds horizon step j = c*32 + l of chunk c:
// control u_j, state q_{j+1} = q_0 + dt sum_{i<=j} u_i (warp prefix sum),
// forward kinematics, 4 spheres per link against every obstacle, and the pose
// cost of Eq. 24 (w_p |p_ee - p_g| + w_R angle(R, R_g) + w_c I_col).
// S = sum_{j=0..T} l(q_j) (the terminal cost has the stage form).
// Two-level broad phase before the 24 sphere tests: an obstacle farther from
// the arm's bounding sphere (centre of the 7 frame origins, radius to the
// farthest) than its radius is skipped; then per link, an obstacle farther from
// the link's midpoint than half the link plus its radius is skipped.  Sphere
// centres lie on the link segments, so no colliding pair is skipped (a 1e-5
// relative slack covers FP32 rounding).  Entries are (x, y, z, r_o + r_robot).
__device__ __forceinline__ int arm_collide(const float O[7][3], const float4* tj, int n_obs) {
  float lc[6][3], lh[6], ac[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < 7; ++i)
#pragma unroll
    for (int q = 0; q < 3; ++q) ac[q] += O[i][q] * (1.0f / 7.0f);
  float ar2 = 0.f;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    const float dx = O[i][0] - ac[0], dy = O[i][1] - ac[1], dz = O[i][2] - ac[2];
    ar2 = fmaxf(ar2, dx * dx + dy * dy + dz * dz);
  }
  const float ar = sqrtf(ar2) * 1.00001f + 1e-6f;
#pragma unroll
  for (int l = 0; l < 6; ++l) {
    float s2 = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      lc[l][q] = 0.5f * (O[l][q] + O[l + 1][q]);
      const float e = O[l + 1][q] - O[l][q];
      s2 += e * e;
    }
    lh[l] = 0.5f * sqrtf(s2) * 1.00001f + 1e-6f;
  }
  for (int o = 0; o < n_obs; ++o) {
    const float4 t = tj[o];
    const float R = t.w;
    {
      const float dx = ac[0] - t.x, dy = ac[1] - t.y, dz = ac[2] - t.z;
      const float rr = ar + R;
      if (dx * dx + dy * dy + dz * dz >= rr * rr) continue;
    }
    const float R2 = R * R;
    bool any = false;
#pragma unroll
    for (int l = 0; l < 6; ++l) {
      const float dx = lc[l][0] - t.x, dy = lc[l][1] - t.y, dz = lc[l][2] - t.z;
      const float rr = lh[l] + R;
      if (dx * dx + dy * dy + dz * dz >= rr * rr) continue;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const float fr = (float)f * (1.0f / 3.0f);
        const float cx = O[l][0] + fr * (O[l + 1][0] - O[l][0]);
        const float cy = O[l][1] + fr * (O[l + 1][1] - O[l][1]);
        const float cz = O[l][2] + fr * (O[l + 1][2] - O[l][2]);
        const float ex = cx - t.x, ey = cy - t.y, ez = cz - t.z;
        any |= (ex * ex + ey * ey + ez * ez < R2);
      }
    }
    if (any) return o;
  }
  return n_obs;
}

__device__ __forceinline__ float arm_cost(const InstDesc& d, const float O[7][3],
                                          const float R[9], int collide) {
  const float ex = O[6][0] - d.goal[0], ey = O[6][1] - d.goal[1], ez = O[6][2] - d.goal[2];
  return d.w[0] * sqrtf(ex * ex + ey * ey + ez * ez) + d.w[1] * rot_angle(R, d.goal + 3) +
         (collide ? d.w[2] : 0.0f);
}

template <bool ACC>   // ACC: 12-D state with joint-acceleration input
__global__ void __launch_bounds__(kArmWarps * 32, 2) k_rollout_arm(KArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  pdl_trigger();   // (as in k_rollout2d: the clustering kernel may be scheduled)
  const int2 tile = tile_of(a);
  const InstDesc& d = desc_of(a, tile.x);
  const Req r = req_of(a, tile.x);
  const int n_obs = r.n_obs, T = d.T, ts = track_stride(n_obs);
  float4* trk = reinterpret_cast<float4*>(smem_raw);
  float* Us = reinterpret_cast<float*>(smem_raw + (n_obs > 0 ? track_bytes(T, n_obs) : 0));
  if (!stage_tracks(d, n_obs, trk, Us, &bar)) return;
  const int lane = threadIdx.x & 31;
  const int k = tile.y * kArmWarps + (threadIdx.x >> 5);
  if (k >= d.K) return;
  const unsigned long long ctr = *d.counter;
  const float dt = d.dt;

  constexpr bool acc = ACC;
  float q[6], qd[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    q[i] = r.x0[i];
    qd[i] = acc ? r.x0[6 + i] : 0.0f;
  }
  float O[7][3], R[9];
  // the shared initial state: its cost term (and optional collision test)
  arm_fk(q, O, R);
  const int c0 = arm_collide(O, trk, n_obs);
  float S = 0.0f, Sc = 0.0f;
  if (lane == 0) S = arm_cost(d, O, R, c0 < n_obs);
  int first = -1, first_j = -1;
  if (d.check_j0 && c0 < n_obs) { first = c0; first_j = 0; }
  float pN[3] = {0.f, 0.f, 0.f};
  for (int base = 0; base < T; base += 32) {
    const int j = base + lane;
    const bool act = j < T;
    float u[6];
    if (act) {
      // normals 6j .. 6j+5 live in Philox blocks (6j)/4 and (6j)/4 + 1
      const int n0 = 6 * j, b0 = n0 >> 2, off = n0 & 3;
      const float4 za = philox_normals(d, ctr, k, b0);
      const float4 zb = philox_normals(d, ctr, k, b0 + 1);
      const float zz[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const float z = off == 0 ? zz[i] : zz[i + 2];
        const float nom = Us[j * 6 + i];
        u[i] = sampled_control(nom, d.sigma[i], z, d.u_min[i], d.u_max[i]);
        if (!d.regen) d.eps[(size_t)k * d.eps_ld_k + n0 + i] = u[i] - nom;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 6; ++i) u[i] = 0.0f;
    }
    // inclusive warp prefix sums.  Velocity input: q_{j+1} = q + dt sum_{i<=j} u_i.
    // Acceleration input: qdot_j = qdot + dt sum_{i<j} u_i, then
    // q_{j+1} = q + dt sum_{i<=j} qdot_i.
    auto scan = [&](float v) {
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      return v;
    };
    const int last = min(31, T - 1 - base);
    float qj[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float su = scan(u[i]);
      if (!acc) {
        qj[i] = q[i] + su * dt;
      } else {
        const float vj = act ? qd[i] + (su - u[i]) * dt : 0.0f;
        qj[i] = q[i] + scan(vj) * dt;
        qd[i] = qd[i] + __shfl_sync(0xffffffffu, su, last) * dt;   // the next chunk's start
      }
    }
    int hit_here = n_obs;
    float cost = 0.0f;
    if (act) {
      arm_fk(qj, O, R);
      hit_here = arm_collide(O, trk + (size_t)(j + 1) * ts, n_obs);
      cost = arm_cost(d, O, R, hit_here < n_obs);
      if (j == T - 1) { pN[0] = O[6][0]; pN[1] = O[6][1]; pN[2] = O[6][2]; }
    }
    kahan_add(S, Sc, cost);
    const unsigned hm = __ballot_sync(0xffffffffu, hit_here < n_obs);
    if (first < 0 && hm) {
      const int l = __ffs(hm) - 1;
      first = __shfl_sync(0xffffffffu, hit_here, l);
      first_j = base + l + 1;
    }
    // carry the chunk's final state to the next chunk
#pragma unroll
    for (int i = 0; i < 6; ++i) q[i] = __shfl_sync(0xffffffffu, qj[i], last);
  }
  S = warp_sum(S);
  const int lt = (T - 1) & 31;
#pragma unroll
  for (int i = 0; i < 3; ++i) pN[i] = __shfl_sync(0xffffffffu, pN[i], lt);
  if (lane == 0) {
    d.S[k] = S;
    d.hit[k] = first;
    d.hitj[k] = first_j;
    d.pN[k] = pN[0];
    d.pN[d.Kp + k] = pN[1];
    d.pN[2 * d.Kp + k] = pN[2];
    // the pruning stage's inputs in aggregate (Eq. 9-11): this rollout's
    // group record, and its obstacle's count and fixed-point sums of p(x_T)
    const bool col = first >= 0;
    d.gcnt[k] = make_int2(col ? 0 : 1, col ? 1 : 0);
    d.gS[k] = make_float4(col ? 0.f : fabsf(S), col ? INFINITY : S, S, 0.f);
    if (col) {
      unsigned long long* os = reinterpret_cast<unsigned long long*>(d.osum + 4 * (size_t)first);
      atomicAdd(os, 1ull);
#pragma unroll
      for (int c = 0; c < 3; ++c) atomicAdd(os + 1 + c, (unsigned long long)pos_fixed(pN[c]));
    }
  }
}

// ------------------------------------------------------------------ test stages
__global__ void k_philox(unsigned long long seed, unsigned long long counter, int K, int nblk,
                         unsigned int* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)K * nblk) return;
  const int k = (int)(i / nblk), b = (int)(i % nblk);
  const uint4 w = philox10(make_uint4((uint32_t)k, (uint32_t)b, (uint32_t)counter,
                                      (uint32_t)(counter >> 32)),
                           make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  reinterpret_cast<uint4*>(out)[i] = w;
}

__global__ void k_normals(unsigned long long seed, unsigned long long counter, int K, int n,
                          float* out) {
  const int nb = (n + 3) / 4;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)K * nb) return;
  const int k = (int)(i / nb), b = (int)(i % nb);
  const uint4 w = philox10(make_uint4((uint32_t)k, (uint32_t)b, (uint32_t)counter,
                                      (uint32_t)(counter >> 32)),
                           make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const float4 z = normals4(w);
  const float zz[4] = {z.x, z.y, z.z, z.w};
  for (int s = 0; s < 4 && 4 * b + s < n; ++s) out[(size_t)k * n + 4 * b + s] = zz[s];
}

// -2 ln u of every uniform u = (m + 1/2) 2^-23, m < 2^23, as the rollouts
// compute it
__global__ void k_neg2ln(float* out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < (1 << 23)) out[m] = neg2ln(unit23((uint32_t)m << 9));
}

// ------------------------------------------------------------------ launchers
int rollout_threads(int dyn) { return is_arm(dyn) ? kArmWarps * 32 : kRolloutThreads; }

void launch_tracks(const KArgs& a, cudaStream_t s, bool after_update) {
  if (!after_update) {
    k_tracks<<<a.n_inst, 1024, 0, s>>>(a);
    return;
  }
  // scheduled while the update kernel before it in the stream runs (that
  // grid lets it be at its start); it waits for that grid's completion
  // before reading the state (pdl_wait)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)a.n_inst);
  cfg.blockDim = dim3(1024u);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_tracks, a);
}

void configure_rollout() {
  cudaFuncSetAttribute(k_rollout2d<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kMaxSmemTracks + 8192);
  cudaFuncSetAttribute(k_rollout2d<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kMaxSmemTracks + 8192);
  cudaFuncSetAttribute(k_rollout_arm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kMaxSmemTracks + 8192);
  cudaFuncSetAttribute(k_rollout_arm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kMaxSmemTracks + 8192);
}

// The rollout kernels are launched as programmatic dependents of the track
// kernel when it precedes them in the stream (dependent; see pdl_wait), else
// as plain launches (their pdl_wait then returns at once).
template <typename K>
static void launch_dependent(K kern, int grid, int block, int smem, cudaStream_t s,
                             const KArgs& a, bool dependent) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = dependent ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, a);
}

void launch_rollout(int dyn, const KArgs& a, int smem_bytes, cudaStream_t s, bool after_tracks) {
  if (dyn == CE_DYN_DOUBLE_INT_2D)
    launch_dependent(k_rollout2d<0>, a.n_tiles, kRolloutThreads, smem_bytes, s, a, after_tracks);
  else if (dyn == CE_DYN_UNICYCLE)
    launch_dependent(k_rollout2d<1>, a.n_tiles, kRolloutThreads, smem_bytes, s, a, after_tracks);
  else if (dyn == CE_DYN_ARM6_KIN)
    launch_dependent(k_rollout_arm<false>, a.n_tiles, kArmWarps * 32, smem_bytes, s, a,
                     after_tracks);
  else
    launch_dependent(k_rollout_arm<true>, a.n_tiles, kArmWarps * 32, smem_bytes, s, a,
                     after_tracks);
}

void launch_philox(unsigned long long seed, unsigned long long counter, int K, int nblk,
                   unsigned int* out, cudaStream_t s) {
  const long long n = (long long)K * nblk;
  k_philox<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(seed, counter, K, nblk, out);
}

void launch_neg2ln(float* out, cudaStream_t s) { k_neg2ln<<<(1 << 23) / 256, 256, 0, s>>>(out); }

void launch_normals(unsigned long long seed, unsigned long long counter, int K, int n,
                    float* out, cudaStream_t s) {
  const long long tot = (long long)K * ((n + 3) / 4);
  k_normals<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(seed, counter, K, n, out);
}

}  // namespace cem
