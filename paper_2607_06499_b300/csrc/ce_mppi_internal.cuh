// ce_mppi_internal.cuh -- device-side data layout and helpers shared by the
// CE-MPPI kernels (sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ce_mppi.h"

namespace cem {

constexpr int kMaxM = 6;
constexpr int kRolloutThreads = 128;    // 2-D rollouts: one rollout per thread
constexpr int kRolloutMinCtas = 6;      // 2-D rollouts: CTAs per SM the registers allow (80 a thread)
constexpr int kArmWarps = 8;            // arm rollouts: one warp per rollout
constexpr int kBlock = 1024;            // per-instance CTAs (prune, DBSCAN, select)
constexpr int kUpdateWarps = 8;         // update CTA: 8 warps, 32 columns per tile
constexpr int kUpdChunk2D = 1024;       // rollouts per update tile (2-D layout)
constexpr int kUpdChunkArm = 1024;      // rollouts per update tile (arm layout)
constexpr int kUpdUnroll = 4;           // stored eps': rollouts in flight per lane (2-D)
constexpr int kUpdArmUnroll = 32;       // stored eps': rows in flight per warp (arm)
constexpr int kMaxCells = 8192;         // DBSCAN grid cells (cell -> occupied map in smem)
constexpr int kMaxOcc = 2048;           // DBSCAN occupied cells held in shared memory
constexpr int kMaxObs = 4096;           // obstacle bitmap in shared memory
constexpr int kMaxT = 256;
constexpr int kMaxSmemTracks = 200 * 1024;
constexpr long long kSpinLimit = 1ll << 22;   // bounded waits (mbarrier)
constexpr int kUfLimit = 1 << 20;       // parent reads per union-find operation (default)
constexpr int kSparseMax = 256;         // nonzero update weights kept as a sorted list
constexpr int kPruneRanges = 256;       // fixed rollout ranges of the pbar sums
constexpr int kAngBuckets = 4096;       // angle buckets of the 2-D DBSCAN

// Per-instance control block written by the stages of one replan.
struct Ctl {
  int nV, nC, M, mode, sel, o_star, dynamic, status;
  float S_min, invZ;
  float S_absmax_V, S_min_V, S_min_all;   // over V / over all K (written by the prune stage)
  int nnz;                        // nonzero update weights listed (-1: more than kSparseMax)
  int updated;                    // the update was applied by the fused per-instance kernel
  int nnz_all;                    // nonzero weights of the replan (all CTAs of the instance)
  int rejected;                   // no update: 1 a non-finite input (track kernel), 2 a rollout CTA's copy timed out
  float pbar[3], v_obs[3], p0[3];
  unsigned int done;              // last-CTA ticket of the update stage
  int col_tests;                  // circle/sphere tests per rollout after reach culling
  unsigned long long counter_used;
  long long dbcyc[16];            // stage clock stamps of the last replan (see ce_mppi_peek)
};

// Static description of one planner instance: parameters and device buffers.
// Layout of the scratch buffers (Kp = K rounded up to a multiple of 32):
//   tracks float4 [(T+1)][track_stride]: 2-D (x, y, (r_o + r_robot)^2, index),
//          arm (x, y, z, r_o + r_robot); then the (T+1) row counts
//   S, w, Sv (S in V order), cmin (per-cluster least S) float [Kp];
//   hit, hitj, idxV, idxC, label, cell, sorted, parent int [Kp]
//   nzk int, nze float [kSparseMax]: nonzero update weights by ascending k
//   pN, z, g, zs float [p][Kp] (SoA)
//   eps    2-D: float [T*m][Kp] (k fastest); arm: float [Kp][T*m] (k slowest)
struct InstDesc {
  int dyn, K, Kp, T, m, n, p, n_obs_max, H, min_pts, ref_mode, check_j0;
  int regen;                      // eps' is not stored: the update draws it again
  int mppi_only;                  // standard MPPI: no pruning or clustering
  int uf_limit;                   // parent reads per DBSCAN union-find operation
  int G, R, eps_ld_c, eps_ld_k;   // DBSCAN grid size/reach; eps strides (column, rollout)
  float dt, obs_dt, inv_lambda, eps2, cell_inv, robot_radius, norm_eps, v_static_thresh;
  float sigma[6], u_min[6], u_max[6], goal[16], w[8];
  unsigned int seed_lo, seed_hi;
  unsigned long long* counter;
  float* U;      // [T][m] nominal
  float* Unew;   // [T][m] updated nominal before the shift
  float4* tracks;
  float *S, *w_k, *pN, *eps, *z, *g, *zs, *Sv, *cmin, *nze;
  float* zpart;  // [kPruneRanges] range partials of the softmin normaliser
  int* nzk;
  float* upart;  // [ceil(K/512)][TMp] partial sums of the update tiles
  int TMp;       // T*m rounded up to a multiple of 4
  int *hit, *hitj, *idxV, *idxC, *label, *cell, *sorted, *parent;
  int gsz;       // rollouts per group record: 32 (2-D, one warp), 1 (arm)
  int2* gcnt;    // [ceil(K / gsz)] per group: rollouts in V, in C_col
  float4* gS;    // [ceil(K / gsz)] per group: max |S| over V, min S over V, min S
  long long* osum;   // [n_obs_max][4] per obstacle hit first: count, fixed-point sum of p(x_T)
  float* bbox;   // [G^p][6] DBSCAN per-cell core bounding boxes
  int* ang;      // [2][kAngBuckets] angular DBSCAN: bucket counts, least core index
  Ctl* ctl;
};

// One replan's inputs and outputs (device pointers).
struct Req {
  const float* x0;
  const float* obs_hist;
  const float* obs_radius;
  int n_obs;
  int pad;
  long long obs_step;
  unsigned long long counter0;
  float* u_out;
  float* x_next;
  ce_mppi_diag* diag;
};

// Arguments common to every stage kernel.  Instance i of a launch uses the
// descriptor D[slot[i]] (D[i] when slot is null) and the request R[i] (r0 when
// R is null).  Tiled stages (rollouts, update) map blockIdx.x to a tile
// (instance, local tile index) from the explicit list `tiles`, or, when that is
// null, by searching the per-instance tile prefix counts tprefix[n_inst + 1].
struct KArgs {
  const InstDesc* D;
  const int* slot;
  const Req* R;
  Req r0;
  const int2* tiles;
  const int* tprefix;
  int n_inst;
  int n_tiles;
  int n_conc;   // instances whose per-instance stages run at the same time (sizes clusters)
  int post_ctas;    // CTAs per instance of the fused kernel (0: from the occupancy fit)
};

__device__ __forceinline__ const InstDesc& desc_of(const KArgs& a, int i) {
  return a.D[a.slot ? a.slot[i] : i];
}

__device__ __forceinline__ int2 tile_of(const KArgs& a) {
  const int b = blockIdx.x;
  if (a.tiles) return a.tiles[b];
  int lo = 0, hi = a.n_inst - 1;   // largest i with tprefix[i] <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.tprefix[mid] <= b) lo = mid; else hi = mid - 1;
  }
  return make_int2(lo, b - a.tprefix[lo]);
}

// Row stride (in float4) of the obstacle track table: odd, so that lanes
// reading different horizon rows hit different shared-memory banks.
// The two arm models share the kinematics, cost, collision and kernels.
__host__ __device__ __forceinline__ bool is_arm(int dyn) {
  return dyn == CE_DYN_ARM6_KIN || dyn == CE_DYN_ARM12_DI;
}

__host__ __device__ __forceinline__ int track_stride(int n_obs) { return n_obs | 1; }
// 2-D robots use a packed table instead: row offsets off[0..Q+1] (int, Q =
// (T + 1) / 2; T + 2 of them reserved, padded to 16 bytes), then the kept
// entries of rows 0..Q back to back (row r = entries [off[r], off[r+1]), an
// entry two float4): row 0 the current state's, row q + 1 the pair of steps
// 2q, 2q + 1.
__host__ __device__ __forceinline__ size_t track_hdr_bytes(int T) {
  return ((size_t)(T + 2) * 4 + 15) & ~(size_t)15;
}
__host__ __device__ __forceinline__ size_t track_pair_bytes(int T, int n_obs) {
  return track_hdr_bytes(T) + (size_t)(1 + (T + 1) / 2) * (size_t)(n_obs > 1 ? n_obs : 1) * 32;
}
// Shared memory the 2-D rollout kernel stages a packed table into (the row
// offsets, then an entry buffer): at least kTrackSmem2D, and at least one row
// of n_obs_max entries, so that every run of rows holds one row or more; a
// larger table is staged in runs of whole rows.
constexpr int kTrackSmem2D = 8 * 1024;
__host__ __device__ __forceinline__ size_t track_smem_2d(int T, int n_obs_max) {
  const size_t row = track_hdr_bytes(T) + (size_t)(n_obs_max > 1 ? n_obs_max : 1) * 32;
  return row > (size_t)kTrackSmem2D ? row : (size_t)kTrackSmem2D;
}
// Bytes of the track table: (T+1) rows of track_stride float4, then the
// (T+1) row counts (int), padded to 16 bytes.
__host__ __device__ __forceinline__ size_t track_bytes(int T, int n_obs) {
  return (size_t)(T + 1) * track_stride(n_obs) * 16 + (((size_t)(T + 1) * 4 + 15) & ~(size_t)15);
}
template <typename P>
__host__ __device__ __forceinline__ int* track_counts(P* tracks, int T, int n_obs) {
  return reinterpret_cast<int*>(reinterpret_cast<char*>(tracks) +
                                (size_t)(T + 1) * track_stride(n_obs) * 16);
}
template <typename P>
__host__ __device__ __forceinline__ const int* track_counts(const P* tracks, int T, int n_obs) {
  return reinterpret_cast<const int*>(reinterpret_cast<const char*>(tracks) +
                                      (size_t)(T + 1) * track_stride(n_obs) * 16);
}

__device__ __forceinline__ Req req_of(const KArgs& a, int i) {
  return a.R ? a.R[i] : a.r0;
}

__device__ __forceinline__ const float* hist_of(const Req& r, const InstDesc& d) {
  const unsigned long long c = *d.counter;
  return r.obs_hist + (long long)(c - r.counter0) * r.obs_step;
}

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl
// key increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// Four standard normals from one Philox block: Box-Muller on the 23-bit
// uniforms ((w >> 9) + 1/2) 2^-23 of the pairs (w0, w1) and (w2, w3); each
// uniform is exact in FP32 (24 significant bits).  The radius is
// sqrt(neg2ln(u1)), within 5e-7 of exact for every uniform (below).  The
// angle 2 pi u2 is taken in [-pi, pi)
// (u2 - 1 for u2 >= 1/2 is exact) and its sine and cosine come from the
// special-function unit: absolute error <= 2^-21.41 there, plus <= pi 2^-24
// from rounding the angle, so a normal is within r (2^-21.41 + pi 2^-24)
// <= 3.2e-6 of exact for the largest radius r = sqrt(-2 ln 2^-24) = 5.77,
// plus the radius' error.
// The uniform ((w >> 9) + 1/2) 2^-23 formed without an int-to-float
// conversion: 1 + (w >> 9) 2^-23 from the exponent bits of 1.0, minus
// (1 - 2^-24); the difference is exact (both operands lie in [1/2, 2]), so the
// value is the same float (checked for all 2^23 inputs).
__device__ __forceinline__ float unit23(uint32_t w) {
  return __uint_as_float((w >> 9) | 0x3f800000u) - 0.99999994039535522f;
}

// -2 ln u for the uniforms u = (m + 1/2) 2^-23 of unit23 (2^-24 <= u < 1).
// Near u = 1, where -ln u is small and an absolute error bound would not do,
// the Taylor series of -2 ln(1 + t) in t = u - 1 (exact for u >= 1/2):
// -2 (t - t^2/2 + t^3/3 - ... - t^8/8), Horner in FP32; for u > 7/8, |t| <
// 1/8 and the first omitted term is below 2 |t| 2^-27.  Elsewhere the
// special-function unit's base-2 logarithm times -2 ln 2: there |ln u| >=
// 0.133, so its small absolute error stays a small relative one.  Checked
// against the exact value for all 2^23 uniforms: relative error under 2^-20
// (6.9e-7 at most, on the logarithm's side just below 7/8), the radius
// sqrt(-2 ln u) within 5e-7.
// The library's full-accuracy logarithm cost 10 % of the 2-D rollout
// kernel's time.
__device__ __forceinline__ float neg2ln(float u) {
  const float t = u - 1.0f;
  float q = 0.25f;                 // -2 x -1/8
  q = fmaf(q, t, -0.285714298f);   // -2 x 1/7
  q = fmaf(q, t, 0.333333343f);    // -2 x -1/6
  q = fmaf(q, t, -0.4f);           // -2 x 1/5
  q = fmaf(q, t, 0.5f);            // -2 x -1/4
  q = fmaf(q, t, -0.666666687f);   // -2 x 1/3
  q = fmaf(q, t, 1.0f);            // -2 x -1/2
  q = fmaf(q, t, -2.0f);           // -2 x 1
  // both sides computed, then selected (no branch in the warp)
  const float near1 = q * t;
  const float far = __log2f(u) * -1.38629436f;   // -2 ln 2
  return u > 0.875f ? near1 : far;
}

__device__ __forceinline__ float4 normals4(uint4 w) {
  const float u1a = unit23(w.x), u2a = unit23(w.y);
  const float u1b = unit23(w.z), u2b = unit23(w.w);
  // sqrt(x) as x * rsqrt(x) (x >= 2^-23 > 0 here; rsqrtf is within 2 ulp)
  const float xa = neg2ln(u1a), xb = neg2ln(u1b);
  const float ra = xa * rsqrtf(xa), rb = xb * rsqrtf(xb);
  const float two_pi = 6.2831853071795865f;
  const float ta = two_pi * (u2a >= 0.5f ? u2a - 1.0f : u2a);
  const float tb = two_pi * (u2b >= 0.5f ? u2b - 1.0f : u2b);
  float sa, ca, sb, cb;
  __sincosf(ta, &sa, &ca);
  __sincosf(tb, &sb, &cb);
  return make_float4(ra * ca, ra * sa, rb * cb, rb * sb);
}

__device__ __forceinline__ float4 philox_normals(uint2 key, unsigned long long ctr, int k,
                                                 int b) {
  const uint4 c = make_uint4((uint32_t)k, (uint32_t)b, (uint32_t)ctr, (uint32_t)(ctr >> 32));
  return normals4(philox10(c, key));
}
__device__ __forceinline__ float4 philox_normals(const InstDesc& d, unsigned long long ctr,
                                                 int k, int b) {
  return philox_normals(make_uint2(d.seed_lo, d.seed_hi), ctr, k, b);
}

// The sampled control clip(u + sigma z) of Eq. 3 (the rollouts and the
// regenerating update share this one expression, so both round alike).
__device__ __forceinline__ float sampled_control(float nom, float sg, float z, float lo,
                                                 float hi) {
  return fminf(fmaxf(nom + sg * z, lo), hi);
}

// eps' of rollout k, column c (step c / m, input c % m) drawn again: normal
// c of rollout k is element c % 4 of Philox block c / 4 for every robot.
__device__ __forceinline__ float eps_regen(const InstDesc& d, unsigned long long ctr, int k,
                                           int c) {
  const float4 z4 = philox_normals(d, ctr, k, c >> 2);
  const int e = c & 3;
  const float z = e == 0 ? z4.x : e == 1 ? z4.y : e == 2 ? z4.z : z4.w;
  const int q = c % d.m;
  const float nom = d.U[c];
  return sampled_control(nom, d.sigma[q], z, d.u_min[q], d.u_max[q]) - nom;
}

// eps' of rollout k, columns 4b .. 4b+3 (those below TM) from one Philox
// block: column by column the values eps_regen gives (the same expression).
__device__ __forceinline__ void eps_regen4(const InstDesc& d, unsigned long long ctr, int k,
                                           int b, int TM, float* x) {
  const float4 z4 = philox_normals(d, ctr, k, b);
  const float zz[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int c = 4 * b + e;
    x[e] = 0.f;
    if (c < TM) {
      const int q = c % d.m;
      const float nom = d.U[c];
      x[e] = sampled_control(nom, d.sigma[q], zz[e], d.u_min[q], d.u_max[q]) - nom;
    }
  }
}

// ---------------------------------------------------------------- TMA bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Global -> shared bulk copy (non-multicast), completion counted on bar.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait for phase `parity` of bar; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void raise_status(Ctl* c, int code) { atomicCAS(&c->status, 0, code); }

// Programmatic dependent launch of the rollout kernel after the track kernel
// in the same stream: the track kernel lets the dependent grid be scheduled
// early; the rollout kernel waits, before it reads anything the track kernel
// writes, until that grid has completed and its writes are visible (at once
// when its launch has no such dependency).
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Task positions as 32.32 fixed point: sums over any number of rollouts are
// exact, so they do not depend on the order the atomics land in.
__device__ __forceinline__ long long pos_fixed(float v) { return __float2ll_rn(v * 4294967296.0f); }
constexpr float kPosFixedInv = 2.3283064365386963e-10f;   // 2^-32

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Deterministic warp sum (fixed butterfly order).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Order-preserving map of a float to an unsigned int (for packed argmin).
__device__ __forceinline__ uint32_t float_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// ---------------------------------------------------------------- models
// Standard DH chain of the UR5e-like arm (d, a from the workload description,
// alpha from the published UR convention): frame origins O[7][3], rotation R.
__device__ __forceinline__ float dh_d(int i) {
  return i == 0 ? 0.1625f : i == 3 ? 0.1333f : i == 4 ? 0.0997f : i == 5 ? 0.0996f : 0.0f;
}
__device__ __forceinline__ float dh_a(int i) { return i == 1 ? -0.425f : i == 2 ? -0.3922f : 0.0f; }
// cos/sin of alpha = (pi/2, 0, 0, pi/2, -pi/2, 0), exact
__device__ __forceinline__ float dh_ca(int i) { return (i == 0 || i == 3 || i == 4) ? 0.0f : 1.0f; }
__device__ __forceinline__ float dh_sa(int i) {
  return (i == 0 || i == 3) ? 1.0f : i == 4 ? -1.0f : 0.0f;
}

__device__ __forceinline__ void arm_fk(const float q[6], float O[7][3], float R[9]) {
  float T[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};  // 3x4, rows (R | t)
  O[0][0] = O[0][1] = O[0][2] = 0.0f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    // the joint's sine and cosine on the special-function unit: absolute
    // error ~2^-21.4 for |q| <= pi, growing in proportion to |q| beyond
    // (~1e-6 at 2 pi), so a frame origin moves by ~1e-6 m at most over the
    // ~1.3 m chain: below the 1e-5 m band of the collision parity and far
    // below the position tolerance (the full-accuracy call cost 4.3 % of
    // the arm's pipelined step)
    float st, ct;
    __sincosf(q[i], &st, &ct);
    const float ca = dh_ca(i), sa = dh_sa(i), ai = dh_a(i), di = dh_d(i);
    // A = [[ct, -st ca, st sa, a ct], [st, ct ca, -ct sa, a st], [0, sa, ca, d]]
    const float A00 = ct, A01 = -st * ca, A02 = st * sa, A03 = ai * ct;
    const float A10 = st, A11 = ct * ca, A12 = -ct * sa, A13 = ai * st;
    const float A21 = sa, A22 = ca, A23 = di;
    float N[12];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float t0 = T[r * 4 + 0], t1 = T[r * 4 + 1], t2 = T[r * 4 + 2], t3 = T[r * 4 + 3];
      N[r * 4 + 0] = t0 * A00 + t1 * A10;
      N[r * 4 + 1] = t0 * A01 + t1 * A11 + t2 * A21;
      N[r * 4 + 2] = t0 * A02 + t1 * A12 + t2 * A22;
      N[r * 4 + 3] = t0 * A03 + t1 * A13 + t2 * A23 + t3;
    }
#pragma unroll
    for (int e = 0; e < 12; ++e) T[e] = N[e];
    O[i + 1][0] = T[3];
    O[i + 1][1] = T[7];
    O[i + 1][2] = T[11];
  }
  R[0] = T[0]; R[1] = T[1]; R[2] = T[2];
  R[3] = T[4]; R[4] = T[5]; R[5] = T[6];
  R[6] = T[8]; R[7] = T[9]; R[8] = T[10];
}

// Geodesic angle between R and the goal rotation Rg: atan2(|axis|, tr - 1)
// with M = Rg^T R (well conditioned near 0 and pi, equal to acos((tr-1)/2)).
__device__ __forceinline__ float rot_angle(const float R[9], const float* Rg) {
  float M[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      M[r * 3 + c] = Rg[0 * 3 + r] * R[0 * 3 + c] + Rg[1 * 3 + r] * R[1 * 3 + c] +
                     Rg[2 * 3 + r] * R[2 * 3 + c];
  const float tr = M[0] + M[4] + M[8];
  const float ax = M[7] - M[5], ay = M[2] - M[6], az = M[3] - M[1];
  return atan2f(sqrtf(ax * ax + ay * ay + az * az), tr - 1.0f);
}

// ---------------------------------------------------------------- launchers
// Host-side launchers of each stage (defined in the .cu files).
// after_update: a programmatic dependent of the update kernel before it in
// the stream (a pipelined half's next replan, see ce_mppi_batch_run_part)
void launch_tracks(const KArgs& a, cudaStream_t s, bool after_update = false);
// after_tracks: the track kernel precedes in the stream, the rollouts are
// launched as its programmatic dependents (else as a plain launch: a
// programmatic edge would tie them to whatever kernel precedes instead)
void launch_rollout(int dyn, const KArgs& a, int smem_bytes, cudaStream_t s, bool after_tracks);
// (started: an optional launch-completion event of the launch)
void launch_prune(const KArgs& a, cudaStream_t s, cudaEvent_t started = nullptr);
void launch_dbscan(const KArgs& a, int max_cells, cudaStream_t s);
void launch_select(const KArgs& a, cudaStream_t s);
// prune + DBSCAN + selection (+ the update with few nonzero weights) as one
// clustered launch; false when the shared memory does not allow it
bool launch_post(const KArgs& a, int max_cells, cudaStream_t s, cudaEvent_t started = nullptr);
void launch_update(const KArgs& a, cudaStream_t s);
void launch_philox(unsigned long long seed, unsigned long long counter, int K, int nblk,
                   unsigned int* out, cudaStream_t s);
void launch_neg2ln(float* out, cudaStream_t s);
void launch_normals(unsigned long long seed, unsigned long long counter, int K, int n,
                    float* out, cudaStream_t s);
void launch_dbscan_standalone(const float* z, int n, int ld, int p, float eps2, float cell_inv,
                              int G, int R, int min_pts, int* labels, int* n_clusters,
                              void* ws, cudaStream_t s);
int rollout_threads(int dyn);
void configure_rollout();
void set_last_error(const char* msg);   // message returned by ce_mppi_last_error()
void configure_cluster(bool fits);
// Configure the kernels for the current device once (thread-safe; every entry
// point that launches calls it first).
void ensure_configured();
size_t dbscan_ws_bytes(int n);

}  // namespace cem
