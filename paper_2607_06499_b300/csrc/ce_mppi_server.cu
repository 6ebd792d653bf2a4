// ce_mppi_server.cu -- continuous-batching replan server.
//
// Controller sessions are admitted against a device-memory budget; each keeps
// its planner state (nominal sequence, replan counter, scratch) resident on the
// device.  Replan requests are staged on the host as they arrive; a worker
// thread forms a batch from every queued session of one dynamics kind as soon
// as one of its in-flight slots (a non-blocking stream with its own staging
// buffers) is free, copies the batch's inputs in one transfer, runs the replan
// chain once for the whole batch (instances addressed through the session
// slot table), and copies the results back in one transfer.  Batches on
// different slots overlap on the device, so requests that arrive while others
// run are picked up by the next free slot without waiting for them.  A session
// is in at most one batch at a time; a request that arrives while the
// session's previous one is still queued replaces it (both tickets get the
// newer result).  The kernels' reductions run in an order fixed by each
// instance alone, so a replan gives the same bits alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ce_mppi_host.h"

using namespace cem;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

struct Session {
  ce_mppi_handle* h = nullptr;
  bool open = false, queued = false, inflight = false, closing = false;
  int n_obs = 0;
  std::vector<float> in;                    // x0 [n] | hist [H][n_obs][p] | radius [n_obs]
  std::vector<unsigned long long> tickets;  // waiting on the queued request
  double t_submit = 0.0;
};

struct Result {
  bool done = false;
  int status = 0;
  std::vector<float> u;
  ce_mppi_diag diag;
  double latency = 0.0;
};

struct Flight {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool busy = false;
  unsigned char *h_in = nullptr, *d_in = nullptr, *h_out = nullptr, *d_out = nullptr;
  size_t in_cap = 0, out_cap = 0;
  int dyn = 0;
  std::vector<int> members;
  std::vector<std::vector<unsigned long long>> tickets;
  std::vector<double> t_submit;
  std::vector<size_t> out_off;
};

ce_status_t srv_fail(ce_status_t s, const char* msg) {
  set_last_error(msg);
  return s;
}

bool grow(unsigned char** h, unsigned char** d, size_t* cap, size_t need) {
  if (need <= *cap) return true;
  size_t nc = std::max(need, *cap * 2);
  if (*h) cudaFreeHost(*h);
  if (*d) cudaFree(*d);
  *h = nullptr;
  *d = nullptr;
  *cap = 0;
  if (cudaHostAlloc((void**)h, nc, cudaHostAllocDefault) != cudaSuccess) return false;
  if (cudaMalloc((void**)d, nc) != cudaSuccess) return false;
  *cap = nc;
  return true;
}

}  // namespace

struct ce_mppi_server {
  ce_server_params P;
  InstDesc* dslots = nullptr;
  cudaStream_t admin = nullptr;
  std::vector<Session> sessions;
  std::vector<int> free_slots;
  size_t mem_in_use = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false;
  std::vector<Flight> flights;
  std::deque<int> queue;
  std::unordered_map<unsigned long long, Result> results;
  unsigned long long next_ticket = 1;
  // statistics
  unsigned long long replans = 0, batches = 0, opened = 0, rejected = 0, superseded = 0;
  unsigned long long batch_members = 0;
  std::vector<double> lat;
  int worker_status = 0;

  void complete(Flight& f) {
    const double t = now_s();
    for (size_t i = 0; i < f.members.size(); ++i) {
      Session& s = sessions[f.members[i]];
      const ce_mppi_handle* h = s.h;
      const int TM = h->P.T * h->m;
      const float* u = reinterpret_cast<const float*>(f.h_out + f.out_off[i]);
      ce_mppi_diag dg;
      std::memcpy(&dg, f.h_out + f.out_off[i] + align16(sizeof(float) * TM), sizeof(dg));
      const double l = t - f.t_submit[i];
      if (lat.size() < (1u << 24)) lat.push_back(l);
      for (unsigned long long tk : f.tickets[i]) {
        auto it = results.find(tk);
        if (it == results.end()) continue;
        Result& r = it->second;
        r.u.assign(u, u + TM);
        r.diag = dg;
        r.status = dg.status;
        r.latency = t - f.t_submit[i];
        r.done = true;
      }
      s.inflight = false;
      ++replans;
      if (s.closing && !s.queued) release(f.members[i]);
    }
    f.busy = false;
    f.members.clear();
    f.tickets.clear();
    f.t_submit.clear();
    f.out_off.clear();
  }

  // Closed sessions' planners wait in a pool for a new session of the same
  // buffer layout (no device allocation or free while batches run); their
  // memory stays counted against the budget until the pool gives it back.
  std::vector<ce_mppi_handle*> pool;

  void release(int sid) {
    Session& s = sessions[sid];
    if (s.h) pool.push_back(s.h);
    s = Session();
    free_slots.push_back(sid);
  }

  // Free pooled planners until `need` more bytes fit in the budget.
  void shrink_pool(size_t need) {
    while (!pool.empty() && mem_in_use + need > P.mem_budget_bytes) {
      mem_in_use -= pool.back()->dbytes;
      ce_mppi_destroy(pool.back());
      pool.pop_back();
    }
  }

  // Take queued sessions of one dynamics kind into flight f (under the lock).
  bool form(Flight& f) {
    // a session closed while queued leaves its id behind (its planner may
    // already be pooled or its slot reused): drop such entries first
    while (!queue.empty()) {
      const Session& s = sessions[queue.front()];
      if (s.open && s.queued && s.h) break;
      queue.pop_front();
    }
    if (queue.empty()) return false;
    const int dyn = sessions[queue.front()].h->P.dyn;
    std::deque<int> rest;
    int smem = 0, cells = 0;
    size_t in_bytes = 0, out_bytes = 0;
    while (!queue.empty() && (int)f.members.size() < P.max_batch) {
      const int sid = queue.front();
      queue.pop_front();
      Session& s = sessions[sid];
      if (!s.open || !s.queued) continue;
      if (s.h->P.dyn != dyn || s.inflight) { rest.push_back(sid); continue; }
      f.members.push_back(sid);
      in_bytes += align16(sizeof(float) * s.in.size());
      out_bytes += align16(sizeof(float) * s.h->P.T * s.h->m) + align16(sizeof(ce_mppi_diag));
      smem = std::max(smem, s.h->smem_roll);
      cells = std::max(cells, s.h->ncells);
    }
    while (!rest.empty()) { queue.push_front(rest.back()); rest.pop_back(); }
    if (f.members.empty()) return false;
    const int n = (int)f.members.size();
    const size_t head = align16(sizeof(int) * (3 * (size_t)n + 2)) + align16(sizeof(Req) * n);
    if (!grow(&f.h_in, &f.d_in, &f.in_cap, head + in_bytes) ||
        !grow(&f.h_out, &f.d_out, &f.out_cap, out_bytes)) {
      worker_status = CE_MPPI_ERR_NO_MEMORY;
      for (int sid : f.members) queue.push_back(sid);
      f.members.clear();
      return false;
    }
    int* slots = reinterpret_cast<int*>(f.h_in);
    int* pre_roll = slots + n;
    int* pre_upd = pre_roll + n + 1;
    Req* reqs = reinterpret_cast<Req*>(f.h_in + align16(sizeof(int) * (3 * (size_t)n + 2)));
    size_t ioff = head, ooff = 0;
    pre_roll[0] = pre_upd[0] = 0;
    f.dyn = dyn;
    for (int i = 0; i < n; ++i) {
      Session& s = sessions[f.members[i]];
      ce_mppi_handle* h = s.h;
      slots[i] = f.members[i];
      const int per = is_arm(dyn) ? kArmWarps : kRolloutThreads;
      const int TM = h->P.T * h->m;
      const int cper = 32;   // (columns per update tile, as k_update)
      const int kch = is_arm(dyn) ? kUpdChunkArm : kUpdChunk2D;
      pre_roll[i + 1] = pre_roll[i] + (h->P.K + per - 1) / per;
      pre_upd[i + 1] = pre_upd[i] + ((TM + cper - 1) / cper) * ((h->P.K + kch - 1) / kch);
      std::memcpy(f.h_in + ioff, s.in.data(), sizeof(float) * s.in.size());
      const float* dbase = reinterpret_cast<const float*>(f.d_in + ioff);
      Req r;
      std::memset(&r, 0, sizeof(r));
      r.x0 = dbase;
      r.obs_hist = dbase + h->n;
      r.obs_radius = dbase + h->n + (size_t)h->P.hist_len * s.n_obs * h->p;
      r.n_obs = s.n_obs;
      r.u_out = reinterpret_cast<float*>(f.d_out + ooff);
      r.diag = reinterpret_cast<ce_mppi_diag*>(f.d_out + ooff + align16(sizeof(float) * TM));
      reqs[i] = r;
      f.out_off.push_back(ooff);
      ioff += align16(sizeof(float) * s.in.size());
      ooff += align16(sizeof(float) * TM) + align16(sizeof(ce_mppi_diag));
      f.tickets.push_back(std::move(s.tickets));
      s.tickets.clear();
      f.t_submit.push_back(s.t_submit);
      s.queued = false;
      s.inflight = true;
    }
    f.busy = true;
    launch_n = n;
    launch_in = ioff;
    launch_out = ooff;
    launch_smem = smem;
    launch_cells = cells;
    ++batches;
    batch_members += n;
    return true;
  }

  int launch_n = 0, launch_smem = 0, launch_cells = 0;
  size_t launch_in = 0, launch_out = 0;

  void launch(Flight& f, int n, size_t in_used, size_t out_used, int smem, int cells) {
    const int* pre_roll_h = reinterpret_cast<int*>(f.h_in) + n;
    const int* pre_upd_h = pre_roll_h + n + 1;
    const int n_roll = pre_roll_h[n], n_upd = pre_upd_h[n];
    cudaMemcpyAsync(f.d_in, f.h_in, in_used, cudaMemcpyHostToDevice, f.stream);
    KArgs a;
    std::memset(&a, 0, sizeof(a));
    a.D = dslots;
    a.slot = reinterpret_cast<const int*>(f.d_in);
    a.R = reinterpret_cast<const Req*>(f.d_in + align16(sizeof(int) * (3 * (size_t)n + 2)));
    a.n_inst = n;
    a.n_conc = n;
    const int* d_pre_roll = reinterpret_cast<const int*>(f.d_in) + n;
    run_chain(f.dyn, a, nullptr, n_roll, nullptr, n_upd, smem, cells, f.stream, d_pre_roll,
              d_pre_roll + n + 1);
    cudaMemcpyAsync(f.h_out, f.d_out, out_used, cudaMemcpyDeviceToHost, f.stream);
    cudaEventRecord(f.ev, f.stream);
    if (cudaGetLastError() != cudaSuccess) worker_status = CE_MPPI_ERR_CUDA;
  }

  void run() {
    cudaSetDevice(P.device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      bool progress = false, any_busy = false;
      for (Flight& f : flights)
        if (f.busy) {
          if (cudaEventQuery(f.ev) == cudaSuccess) {
            complete(f);
            progress = true;
          } else {
            any_busy = true;
          }
        }
      for (Flight& f : flights) {
        if (f.busy || queue.empty()) continue;
        if (!form(f)) continue;
        const int n = launch_n, smem = launch_smem, cells = launch_cells;
        const size_t in_used = launch_in, out_used = launch_out;
        lk.unlock();
        launch(f, n, in_used, out_used, smem, cells);
        lk.lock();
        progress = any_busy = true;
      }
      if (stop && !any_busy) break;
      if (!progress) {
        if (any_busy) cv.wait_for(lk, std::chrono::microseconds(20));
        else cv.wait_for(lk, std::chrono::milliseconds(5));
      }
    }
  }
};

extern "C" {

ce_status_t ce_mppi_server_create(const ce_server_params* P, ce_mppi_server** out) {
  if (!out || !P) return srv_fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (P->max_sessions < 1 || P->max_sessions > 65536 || P->max_batch < 1 || P->n_streams < 1 ||
      P->n_streams > 16)
    return srv_fail(CE_MPPI_ERR_INVALID_ARG,
                    "max_sessions in [1, 65536], max_batch >= 1, n_streams in [1, 16]");
  if (cudaSetDevice(P->device) != cudaSuccess) return srv_fail(CE_MPPI_ERR_CUDA, "cudaSetDevice");
  ce_mppi_server* s = new (std::nothrow) ce_mppi_server();
  if (!s) return srv_fail(CE_MPPI_ERR_NO_MEMORY, "host allocation failed");
  s->P = *P;
  s->sessions.resize(P->max_sessions);
  for (int i = P->max_sessions - 1; i >= 0; --i) s->free_slots.push_back(i);
  if (cudaMalloc(&s->dslots, sizeof(InstDesc) * P->max_sessions) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->admin, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(s->dslots);
    delete s;
    return srv_fail(CE_MPPI_ERR_NO_MEMORY, "device allocation failed");
  }
  s->flights.resize(P->n_streams);
  for (Flight& f : s->flights) {
    cudaStreamCreateWithFlags(&f.stream, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&f.ev, cudaEventDisableTiming);
  }
  s->worker = std::thread([s]() { s->run(); });
  *out = s;
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_server_destroy(ce_mppi_server* s) {
  if (!s) return CE_MPPI_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->queue.clear();
  }
  s->cv.notify_all();
  s->worker.join();
  for (Flight& f : s->flights) {
    cudaStreamSynchronize(f.stream);
    cudaStreamDestroy(f.stream);
    cudaEventDestroy(f.ev);
    cudaFreeHost(f.h_in);
    cudaFreeHost(f.h_out);
    cudaFree(f.d_in);
    cudaFree(f.d_out);
  }
  for (Session& ss : s->sessions)
    if (ss.h) ce_mppi_destroy(ss.h);
  for (ce_mppi_handle* h : s->pool) ce_mppi_destroy(h);
  cudaStreamDestroy(s->admin);
  cudaFree(s->dslots);
  delete s;
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_server_open(ce_mppi_server* s, const ce_mppi_params* params, int* session) {
  if (!s || !params || !session) return srv_fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  *session = -1;
  ce_status_t st = validate_params(params);
  if (st != CE_MPPI_OK) return st;
  int sid;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->free_slots.empty()) {
      ++s->rejected;
      return srv_fail(CE_MPPI_ERR_NO_MEMORY, "no free session slot");
    }
    sid = s->free_slots.back();
    s->free_slots.pop_back();
  }
  ce_mppi_handle* h = nullptr;
  bool reused = false;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t i = 0; i < s->pool.size(); ++i)
      if (same_layout(s->pool[i], params)) {
        h = s->pool[i];
        s->pool.erase(s->pool.begin() + i);
        reused = true;
        break;
      }
  }
  if (reused) st = handle_retarget(h, params);
  else st = ce_mppi_create(params, s->admin, &h);
  std::lock_guard<std::mutex> lk(s->mu);
  if (st == CE_MPPI_OK && !reused) {
    s->shrink_pool(h->dbytes);
    if (s->mem_in_use + h->dbytes > s->P.mem_budget_bytes) {
      ce_mppi_destroy(h);
      s->free_slots.push_back(sid);
      ++s->rejected;
      return srv_fail(CE_MPPI_ERR_NO_MEMORY, "device-memory budget exhausted");
    }
    s->mem_in_use += h->dbytes;
  }
  if (st != CE_MPPI_OK) {
    if (h && reused) s->pool.push_back(h);
    else if (h) ce_mppi_destroy(h);
    s->free_slots.push_back(sid);
    ++s->rejected;
    return st;
  }
  if (cudaMemcpyAsync(s->dslots + sid, &h->hdesc, sizeof(InstDesc), cudaMemcpyHostToDevice,
                      s->admin) != cudaSuccess ||
      cudaStreamSynchronize(s->admin) != cudaSuccess) {
    ce_mppi_destroy(h);
    s->free_slots.push_back(sid);
    return srv_fail(CE_MPPI_ERR_CUDA, "session upload failed");
  }
  Session& ss = s->sessions[sid];
  ss = Session();
  ss.h = h;
  ss.open = true;
  ss.in.assign(h->n + (size_t)params->hist_len * params->n_obs_max * h->p + params->n_obs_max, 0.f);
  ++s->opened;
  *session = sid;
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_server_close(ce_mppi_server* s, int sid) {
  if (!s) return srv_fail(CE_MPPI_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (sid < 0 || sid >= (int)s->sessions.size() || !s->sessions[sid].open)
    return srv_fail(CE_MPPI_ERR_INVALID_ARG, "no such session");
  Session& ss = s->sessions[sid];
  ss.open = false;
  for (unsigned long long tk : ss.tickets) {   // queued, never launched
    auto it = s->results.find(tk);
    if (it != s->results.end()) { it->second.done = true; it->second.status = CE_MPPI_ERR_INVALID_ARG; }
  }
  ss.tickets.clear();
  ss.queued = false;
  if (ss.inflight) ss.closing = true;   // freed when its batch completes
  else s->release(sid);
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_server_submit(ce_mppi_server* s, int sid, const float* x0,
                                  const float* obs_hist, const float* obs_radius, int n_obs,
                                  unsigned long long* ticket) {
  if (!s || !x0) return srv_fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  const double t = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (sid < 0 || sid >= (int)s->sessions.size() || !s->sessions[sid].open)
      return srv_fail(CE_MPPI_ERR_INVALID_ARG, "no such session");
    if (s->stop) return srv_fail(CE_MPPI_ERR_BUSY, "server is stopping");
    if (s->worker_status) return srv_fail((ce_status_t)s->worker_status, "server worker failed");
    Session& ss = s->sessions[sid];
    const ce_mppi_handle* h = ss.h;
    if (cem::check_host_inputs(h, x0, obs_hist, obs_radius, n_obs) != CE_MPPI_OK)
      return CE_MPPI_ERR_INVALID_ARG;   // (the message is set)
    const size_t nh = (size_t)h->P.hist_len * n_obs * h->p;
    ss.in.resize(h->n + nh + n_obs);
    std::memcpy(ss.in.data(), x0, sizeof(float) * h->n);
    if (n_obs > 0) {
      std::memcpy(ss.in.data() + h->n, obs_hist, sizeof(float) * nh);
      std::memcpy(ss.in.data() + h->n + nh, obs_radius, sizeof(float) * n_obs);
    }
    ss.n_obs = n_obs;
    if (ss.queued) {
      ++s->superseded;   // the newer inputs replace the queued ones
    } else {
      ss.queued = true;
      ss.t_submit = t;
      s->queue.push_back(sid);
    }
    if (ticket) {
      const unsigned long long tk = s->next_ticket++;
      s->results.emplace(tk, Result());
      ss.tickets.push_back(tk);
      *ticket = tk;
    }
  }
  s->cv.notify_one();
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_server_submit_many(ce_mppi_server* s, int n, const int* sids,
                                       const float* x0s, const float* hists,
                                       const float* radii, const int* n_obs) {
  if (!s || n < 0 || (n > 0 && (!sids || !x0s || !n_obs)))
    return srv_fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  const double t = now_s();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return srv_fail(CE_MPPI_ERR_BUSY, "server is stopping");
    if (s->worker_status) return srv_fail((ce_status_t)s->worker_status, "server worker failed");
    size_t ox = 0, oh = 0, orad = 0;
    for (int i = 0; i < n; ++i) {
      const int sid = sids[i];
      if (sid < 0 || sid >= (int)s->sessions.size() || !s->sessions[sid].open)
        return srv_fail(CE_MPPI_ERR_INVALID_ARG, "no such session");
      Session& ss = s->sessions[sid];
      const ce_mppi_handle* h = ss.h;
      const int no = n_obs[i];
      if (no < 0 || no > h->P.n_obs_max || (no > 0 && (!hists || !radii)))
        return srv_fail(CE_MPPI_ERR_INVALID_ARG, "bad obstacle count or NULL obstacle arrays");
      const size_t nh = (size_t)h->P.hist_len * no * h->p;
      if (cem::check_host_inputs(h, x0s + ox, no > 0 ? hists + oh : nullptr,
                                 no > 0 ? radii + orad : nullptr, no) != CE_MPPI_OK)
        return CE_MPPI_ERR_INVALID_ARG;   // (the message is set)
      ss.in.resize(h->n + nh + no);
      std::memcpy(ss.in.data(), x0s + ox, sizeof(float) * h->n);
      if (no > 0) {
        std::memcpy(ss.in.data() + h->n, hists + oh, sizeof(float) * nh);
        std::memcpy(ss.in.data() + h->n + nh, radii + orad, sizeof(float) * no);
      }
      ox += h->n;
      oh += nh;
      orad += no;
      ss.n_obs = no;
      if (ss.queued) {
        ++s->superseded;
      } else {
        ss.queued = true;
        ss.t_submit = t;
        s->queue.push_back(sid);
      }
    }
  }
  s->cv.notify_one();
  return CE_MPPI_OK;
}

ce_status_t ce_mppi_server_poll(ce_mppi_server* s, unsigned long long ticket, float* u_out,
                                ce_mppi_diag* diag, double* latency_s) {
  if (!s) return srv_fail(CE_MPPI_ERR_INVALID_ARG, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return srv_fail(CE_MPPI_ERR_INVALID_ARG, "unknown ticket");
  if (!it->second.done) return CE_MPPI_ERR_BUSY;
  const Result& r = it->second;
  if (u_out && !r.u.empty()) std::memcpy(u_out, r.u.data(), sizeof(float) * r.u.size());
  if (diag) *diag = r.diag;
  if (latency_s) *latency_s = r.latency;
  const int st = r.status;
  s->results.erase(it);
  return st ? srv_fail((ce_status_t)st, "replan failed on the device") : CE_MPPI_OK;
}

ce_status_t ce_mppi_server_stats(ce_mppi_server* s, ce_server_stats* out, int reset) {
  if (!s || !out) return srv_fail(CE_MPPI_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->replans = s->replans;
  out->batches = s->batches;
  out->sessions_opened = s->opened;
  out->sessions_rejected = s->rejected;
  out->superseded = s->superseded;
  out->mem_in_use = s->mem_in_use;
  out->mean_batch = s->batches ? (double)s->batch_members / (double)s->batches : 0.0;
  int open = 0;
  for (const Session& ss : s->sessions) open += ss.open ? 1 : 0;
  out->sessions_open = open;
  if (!s->lat.empty()) {
    std::vector<double> v(s->lat);
    auto pct = [&](double q) {
      const size_t k = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + k, v.end());
      return v[k];
    };
    out->p50_latency_s = pct(0.50);
    out->p99_latency_s = pct(0.99);
    double sum = 0.0;
    for (double x : s->lat) sum += x;
    out->mean_latency_s = sum / (double)s->lat.size();
  }
  if (reset) {
    s->replans = s->batches = s->batch_members = s->superseded = 0;
    s->lat.clear();
  }
  return CE_MPPI_OK;
}

}  // extern "C"
