// ce_mppi_host.h -- host-side objects of the library shared by the C-ABI
// implementation files (planner handle, batch) and the stage-chain launcher.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "ce_mppi_internal.cuh"

using cem::InstDesc;
using cem::Req;

struct ce_mppi_handle {
  ce_mppi_params P;
  int n, m, p, Kp, TMp, G, R, ncells;
  cudaStream_t stream;
  InstDesc hdesc;
  InstDesc* ddesc = nullptr;
  void* dmem = nullptr;
  size_t dbytes = 0;
  int2* dtiles = nullptr;   // rollout tiles then update tiles
  int n_roll = 0, n_upd = 0;
  int smem_roll = 0;
  // host-pointer path staging (device and pinned host)
  float *d_x0, *d_hist, *d_rad, *d_uout;
  ce_mppi_diag* d_diag;
  unsigned char* h_stage = nullptr;
  size_t in_bytes = 0, out_bytes = 0;
};

struct ce_mppi_batch {
  std::vector<ce_mppi_handle*> hs;
  cudaStream_t stream;
  int dyn;
  InstDesc* ddesc = nullptr;
  Req* dreq = nullptr;
  int2* dtiles_roll = nullptr;
  int2* dtiles_upd = nullptr;
  int n_roll = 0, n_upd = 0, smem_roll = 0, max_cells = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // concurrent branches: branch b owns descriptors/requests [off, off + n) of
  // ddesc/dreq and its own tiles; the branches run on their own streams
  struct Branch {
    int off = 0, n = 0, n_roll = 0, n_upd = 0, smem_roll = 0, max_cells = 0;
    int2* dtiles_roll = nullptr;
    int2* dtiles_upd = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
  };
  std::vector<Branch> branches;
  cudaEvent_t fork = nullptr;
  int post_ctas = 0;   // CTAs per instance of the fused kernel (0: occupancy fit)
  // host-buffer batches (ce_mppi_batch_create_host): the requests point into
  // one device staging block, inputs then outputs, mirrored in pinned memory
  unsigned char* h_stage = nullptr;
  unsigned char* d_stage = nullptr;
  size_t in_bytes = 0, out_bytes = 0;
  std::vector<int> n_obs;                  // per instance
  std::vector<size_t> in_off, out_off;     // per instance, in the staging block
};


namespace cem {
// Queue the six stages of one replan of the instances described by base.
// Tiles come from troll / tupd, or (when those are null) from the per-instance
// prefix counts pre_roll / pre_upd.
void run_chain(int dyn, const KArgs& base, const int2* troll, int n_roll, const int2* tupd,
               int n_upd, int smem_roll, int max_cells, cudaStream_t s,
               const int* pre_roll = nullptr, const int* pre_upd = nullptr);
ce_status_t validate_params(const ce_mppi_params* P);
// Host inputs of one replan of h (pointers, obstacle count, finite values,
// radii >= 0); sets the thread's last error when they are refused.
ce_status_t check_host_inputs(const ce_mppi_handle* h, const float* x0, const float* obs_hist,
                              const float* obs_radius, int n_obs);
// True when a planner created with P would have h's buffer layout.
bool same_layout(const ce_mppi_handle* h, const ce_mppi_params* P);
// Reuse h's buffers for parameters P of the same layout: new parameters,
// nominal and replan counter back to zero (blocking on h's stream).
ce_status_t handle_retarget(ce_mppi_handle* h, const ce_mppi_params* P);
}  // namespace cem
