// rb_serve.cu -- continuous-batching server for parameter queries.
//
// A host thread owns a table of device slots (capacity set by the memory budget). Each step it
//   1. admits waiting queries into free slots (mu, n written, u = 0, status = active),
//   2. advances every live slot by one Newton iteration (mixed precision: each slot climbs its
//      own precision ladder; FP64 contexts solve admitted queries to completion in one step),
//   3. recovers the pressure of the slots that converged in this step,
//   4. compacts finished slots on the device, copies their results to the host completion
//      table and frees the slots, recording submit-to-completion latency.
// Queries arriving while others are on the GPU join at the next step boundary, so their work
// overlaps with older queries' later iterations. Results do not depend on the mix: each slot's
// arithmetic uses only its own row of every operand.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <set>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "rb_ctx.h"

namespace rb {

using Clock = std::chrono::steady_clock;
constexpr int kSlotFree = -1;  // rb_query_info.status of an unused slot

struct Pending {
  uint64_t ticket;
  double mu[2];
  int n;
  Clock::time_point t0;
};

struct Done {
  std::vector<double> u, p;
  rb_query_info info;
};

struct ServeState {
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool running = false, stop_req = false, drain = true;
  int error = RB_OK;
  std::deque<Pending> queue;
  std::unordered_set<uint64_t> inflight;
  std::unordered_map<uint64_t, Done> done;
  uint64_t next_ticket = 1;
  // slots (host view)
  int cap = 0;
  std::vector<uint64_t> slot_ticket;
  std::vector<int> slot_iters;
  std::vector<int> slot_n;
  std::vector<int> live, live_n, live_it, perm;  // host scratch of one step
  std::vector<Clock::time_point> slot_t0;
  std::set<int> free_slots;   // lowest index first, so live slots stay packed at the front
  // device slot arrays
  double *d_mu = nullptr, *d_u = nullptr, *d_p = nullptr, *d_out = nullptr;
  int *d_n = nullptr, *d_idx = nullptr, *d_cnt = nullptr;
  rb_query_info *d_info = nullptr, *d_info_out = nullptr;
  // pinned staging
  double *h_mu = nullptr, *h_out = nullptr;
  int *h_n = nullptr, *h_idx = nullptr, *h_cnt = nullptr;
  rb_query_info *h_info = nullptr;
  cudaStream_t stream = nullptr;
  // statistics
  std::vector<double> lat;
  size_t completed = 0;
  Clock::time_point t_start, t_last;
};

// Admit K queries: slot idx[i] <- (mu_i, n_i), u = 0, status active (or rejected if n is bad).
__global__ void k_admit(int K, const int *idx, const double *mu_in, const int *n_in, int nm,
                        double *mu, int *nsz, double *u, rb_query_info *info) {
  for (int i = blockIdx.x; i < K; i += gridDim.x) {
    const int s = idx[i];
    for (int j = threadIdx.x; j < nm; j += blockDim.x) u[(size_t)s * nm + j] = 0.0;
    if (threadIdx.x == 0) {
      mu[2 * s] = mu_in[2 * i];
      mu[2 * s + 1] = mu_in[2 * i + 1];
      const int n = n_in[i];
      nsz[s] = n;
      rb_query_info q = {(n >= 1 && n <= nm) ? RB_Q_NOT_CONVERGED : RB_Q_REJECTED, 0, 0, 0, 0.0, 0.0};
      info[s] = q;
    }
  }
}

// Compact finished slots (any status but active-with-iterations-left) into out, then free them.
__global__ void k_collect(int cap, int max_iter, int nm, int m, const double *u, const double *p,
                          rb_query_info *info, int *cnt, int *idx_out, double *out,
                          rb_query_info *info_out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int s = w; s < cap; s += nw) {
    const rb_query_info q = info[s];
    const bool finished = q.status != kSlotFree &&
                          !(q.status == RB_Q_NOT_CONVERGED && q.iters < max_iter);
    if (!finished) continue;
    int slot = 0;
    if (lane == 0) slot = atomicAdd(cnt, 1);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    double *o = out + (size_t)slot * (nm + m);
    for (int j = lane; j < nm; j += 32) o[j] = u[(size_t)s * nm + j];
    for (int j = lane; j < m; j += 32) o[nm + j] = p ? p[(size_t)s * m + j] : 0.0;
    __syncwarp();
    if (lane == 0) {
      idx_out[slot] = s;
      info_out[slot] = q;
      info[s].status = kSlotFree;
    }
  }
}

__global__ void k_free_all(int cap, rb_query_info *info) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < cap; s += gridDim.x * blockDim.x) {
    rb_query_info q = {kSlotFree, 0, 0, 0, 0.0, 0.0};
    info[s] = q;
  }
}

static void release_state(rb_ctx *ctx, ServeState *S) {
  for (void *p : {(void *)S->d_mu, (void *)S->d_u, (void *)S->d_p, (void *)S->d_out,
                  (void *)S->d_n, (void *)S->d_idx, (void *)S->d_cnt, (void *)S->d_info,
                  (void *)S->d_info_out})
    ctx_free(ctx, p);
  for (void *p : {(void *)S->h_mu, (void *)S->h_out, (void *)S->h_n, (void *)S->h_idx,
                  (void *)S->h_cnt, (void *)S->h_info})
    if (p) cudaFreeHost(p);
  if (S->stream) cudaStreamDestroy(S->stream);
  S->d_mu = S->d_u = S->d_p = S->d_out = nullptr;
  S->h_mu = S->h_out = nullptr;
  S->stream = nullptr;
}

// Completion of one ticket (called with the lock held).
static void complete(ServeState *S, uint64_t ticket, Clock::time_point t0, const double *u,
                     const double *p, int nm, int m, const rb_query_info &info) {
  Done d;
  d.u.assign(u, u + nm);
  if (m > 0) d.p.assign(p, p + m);
  d.info = info;
  S->done[ticket] = std::move(d);
  S->inflight.erase(ticket);
  const auto t = Clock::now();
  S->lat.push_back(std::chrono::duration<double>(t - t0).count());
  S->completed += 1;
  S->t_last = t;
}

static int serve_step(rb_ctx *ctx, ServeState *S, bool &idle) {
  const DevOps &o = ctx->ops;
  const int nm = o.n_max, m = o.m > 0 && o.B ? o.m : 0;
  const bool mixed = ctx->cfg.precision == RB_PREC_MIXED;
  cudaStream_t st = S->stream;
  // 1. admission
  int K = 0;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    const bool any_live = (int)S->free_slots.size() < S->cap;
    if (S->queue.empty() && !any_live) {
      if (S->stop_req) return RB_OK;
      idle = true;
      S->cv.wait_for(lk, std::chrono::milliseconds(2));
      return RB_OK;
    }
    idle = false;
    if (S->stop_req && !S->drain) return RB_OK;
    if (!mixed) {  // FP64 steps finish every admitted query: admit into slots 0, 1, 2, ...
      S->free_slots.clear();
      for (int s = 0; s < S->cap; ++s) S->free_slots.insert(s);
    }
    while (!S->queue.empty() && !S->free_slots.empty()) {
      const Pending q = S->queue.front();
      S->queue.pop_front();
      const int s = *S->free_slots.begin();
      S->free_slots.erase(S->free_slots.begin());
      S->slot_ticket[s] = q.ticket;
      S->slot_iters[s] = 0;
      S->slot_n[s] = q.n;
      S->slot_t0[s] = q.t0;
      S->h_idx[K] = s;
      S->h_mu[2 * K] = q.mu[0];
      S->h_mu[2 * K + 1] = q.mu[1];
      S->h_n[K] = q.n;
      ++K;
    }
  }
  cudaError_t e = cudaSuccess;
  if (K > 0) {
    e = cudaMemcpyAsync(S->d_idx, S->h_idx, 4 * (size_t)K, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->d_out, S->h_mu, 16 * (size_t)K, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->d_cnt + 1, S->h_n, 4 * (size_t)K, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "serve admit copy");
    k_admit<<<std::min(K, ctx->sms * 4), 128, 0, st>>>(K, S->d_idx, S->d_out, S->d_cnt + 1, nm,
                                                        S->d_mu, S->d_n, S->d_u, S->d_info);
  }
  // 2. one Newton iteration for every live slot (the whole solve for FP64 contexts)
  int rc;
  if (mixed) {
    // one Newton iteration of every live slot, in size buckets (pressure of the slots that
    // converge in it included)
    S->live.clear();
    S->live_n.clear();
    S->live_it.clear();
    for (int s = 0; s < S->cap; ++s)
      if (S->slot_ticket[s]) {
        S->live.push_back(s);
        S->live_n.push_back(S->slot_n[s]);
        S->live_it.push_back(S->slot_iters[s]);
      }
    rc = mixed_serve_step(ctx, S->d_mu, S->d_n, S->d_u, m > 0 ? S->d_p : nullptr, S->d_info, S->live,
                          S->live_n, S->live_it, S->perm, st);
    if (rc != RB_OK) return rc;
    for (int s = 0; s < S->cap; ++s)
      if (S->slot_ticket[s]) S->slot_iters[s] += 1;
    if ((rc = mixed_error_word(ctx, st)) != RB_OK) return rc;
  } else if (K > 0) {  // the admitted queries occupy slots 0..K-1
    rc = solve_fp64(ctx, S->d_mu, nullptr, K, S->d_n, S->d_u, S->d_p, S->d_info, st);
    if (rc != RB_OK) return rc;
    if (m > 0 && (rc = solve_pressure(ctx, S->d_mu, nullptr, K, S->d_n, S->d_u, S->d_p, S->d_info, st)) != RB_OK)
      return rc;
  }
  // 4. collect finished slots
  cudaMemsetAsync(S->d_cnt, 0, 4, st);
  k_collect<<<std::max(1, std::min(S->cap / 8 + 1, ctx->sms * 8)), 256, 0, st>>>(
      S->cap, ctx->cfg.max_iter, nm, m, S->d_u, m ? S->d_p : nullptr, S->d_info, S->d_cnt,
      S->d_idx, S->d_out, S->d_info_out);
  e = cudaMemcpyAsync(S->h_cnt, S->d_cnt, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "serve collect");
  const int F = *S->h_cnt;
  if (F > 0) {
    e = cudaMemcpyAsync(S->h_idx, S->d_idx, 4 * (size_t)F, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->h_out, S->d_out, 8 * (size_t)F * (nm + m), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->h_info, S->d_info_out, sizeof(rb_query_info) * F, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "serve results");
    std::lock_guard<std::mutex> lk(S->mu);
    for (int i = 0; i < F; ++i) {
      const int s = S->h_idx[i];
      const double *row = S->h_out + (size_t)i * (nm + m);
      complete(S, S->slot_ticket[s], S->slot_t0[s], row, row + nm, nm, m, S->h_info[i]);
      S->slot_ticket[s] = 0;
      S->free_slots.insert(s);
    }
  }
  return RB_OK;
}

static void serve_loop(rb_ctx *ctx) {
  ServeState *S = ctx->serve;
  cudaSetDevice(ctx->device);
  int rc = RB_OK;
  for (;;) {
    bool idle = false;
    rc = serve_step(ctx, S, idle);
    std::lock_guard<std::mutex> lk(S->mu);
    if (rc != RB_OK) {
      S->error = rc;
      break;
    }
    const bool empty = S->queue.empty() && (int)S->free_slots.size() == S->cap;
    if (S->stop_req && (!S->drain || empty)) break;
  }
  // cancel whatever is left (stop without drain, or an error)
  std::lock_guard<std::mutex> lk(S->mu);
  const DevOps &o = ctx->ops;
  const int nm = o.n_max, m = o.m > 0 && o.B ? o.m : 0;
  std::vector<double> zu(nm, 0.0), zp(m, 0.0);
  rb_query_info rej = {RB_Q_REJECTED, 0, ctx->cfg.precision, 0, 0.0, 0.0};
  for (const Pending &q : S->queue) complete(S, q.ticket, q.t0, zu.data(), zp.data(), nm, m, rej);
  S->queue.clear();
  for (int s = 0; s < S->cap; ++s)
    if (S->slot_ticket[s]) {
      complete(S, S->slot_ticket[s], S->slot_t0[s], zu.data(), zp.data(), nm, m, rej);
      S->slot_ticket[s] = 0;
      S->free_slots.insert(s);
    }
  S->running = false;
  S->cv.notify_all();
}

bool serve_running(const rb_ctx *ctx) { return ctx->serve && ctx->serve->running; }

void serve_shutdown(rb_ctx *ctx) {
  ServeState *S = ctx->serve;
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop_req = true;
    S->drain = false;
  }
  S->cv.notify_all();
  if (S->th.joinable()) S->th.join();
  release_state(ctx, S);
  delete S;
  ctx->serve = nullptr;
}

}  // namespace rb

using namespace rb;

extern "C" {

int rb_serve_start(rb_ctx *ctx) {
  if (!ctx) return RB_ERR_ARG;
  if (!ctx->loaded) return set_error(ctx, RB_ERR_STATE, "no operators loaded");
  if (serve_running(ctx)) return set_error(ctx, RB_ERR_STATE, "server already running");
  if (ctx->cfg.pressure_method != RB_PRESSURE_RECOVER)
    return set_error(ctx, RB_ERR_STATE, "the server recovers the pressure; reconstruct it from "
                                        "the polled velocities with rb_reconstruct_pressure");
  serve_shutdown(ctx);  // reap a previous server
  cudaSetDevice(ctx->device);
  ServeState *S = new ServeState();
  ctx->serve = S;
  const DevOps &o = ctx->ops;
  const int nm = o.n_max, m = o.m > 0 && o.B ? o.m : 0;
  const bool mixed = ctx->cfg.precision == RB_PREC_MIXED;
  int rc = RB_OK;
  // operator layouts first, then as many slots as the remaining memory budget admits
  if (mixed && (rc = mixed_prepare(ctx, 1, ctx->stream)) != RB_OK) {
    serve_shutdown(ctx);
    return rc;
  }
  const size_t per_slot = (mixed ? mixed_slot_bytes(ctx) : 8 * (size_t)nm * nm) + 16 * (size_t)(nm + m) + 256;
  const size_t avail = ctx->budget > ctx->used ? ctx->budget - ctx->used : 0;
  const int limit = ctx->cfg.serve_slots > 0 ? std::min(ctx->cfg.serve_slots, 4096) : 4096;
  int cap = (int)std::min<size_t>((size_t)limit, (size_t)(0.8 * (double)avail) / per_slot);
  if (cap < 1) {
    serve_shutdown(ctx);
    return set_error(ctx, RB_ERR_OOM, "memory budget admits no serving slot");
  }
  S->cap = cap;
  void *p;
  auto dal = [&](void **dst, size_t bytes, const char *what) {
    if (rc == RB_OK) rc = ctx_alloc(ctx, dst, bytes, what);
  };
  dal(&p, 16 * (size_t)cap, "serve mu"); S->d_mu = (double *)p;
  dal(&p, 8 * (size_t)cap * nm, "serve u"); S->d_u = (double *)p;
  if (m) { dal(&p, 8 * (size_t)cap * m, "serve p"); S->d_p = (double *)p; }
  dal(&p, 8 * (size_t)cap * (nm + m + 2), "serve out"); S->d_out = (double *)p;
  dal(&p, 4 * (size_t)cap, "serve n"); S->d_n = (int *)p;
  dal(&p, 4 * (size_t)cap, "serve idx"); S->d_idx = (int *)p;
  dal(&p, 4 * (size_t)(cap + 1), "serve counters"); S->d_cnt = (int *)p;
  dal(&p, sizeof(rb_query_info) * cap, "serve info"); S->d_info = (rb_query_info *)p;
  dal(&p, sizeof(rb_query_info) * cap, "serve info out"); S->d_info_out = (rb_query_info *)p;
  bool pin_ok = rc == RB_OK &&
                cudaMallocHost(&S->h_mu, 16 * (size_t)cap) == cudaSuccess &&
                cudaMallocHost(&S->h_out, 8 * (size_t)cap * (nm + m)) == cudaSuccess &&
                cudaMallocHost(&S->h_n, 4 * (size_t)cap) == cudaSuccess &&
                cudaMallocHost(&S->h_idx, 4 * (size_t)cap) == cudaSuccess &&
                cudaMallocHost(&S->h_cnt, 4) == cudaSuccess &&
                cudaMallocHost(&S->h_info, sizeof(rb_query_info) * cap) == cudaSuccess &&
                cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) == cudaSuccess;
  if (rc == RB_OK && !pin_ok) rc = set_error(ctx, RB_ERR_OOM, "server staging");
  if (rc == RB_OK && mixed) rc = mixed_prepare(ctx, cap, S->stream);
  if (rc == RB_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    rc = set_error(ctx, RB_ERR_CUDA, "rb_serve_start: context stream");
  if (rc != RB_OK) {
    serve_shutdown(ctx);
    return rc;
  }
  k_free_all<<<std::max(1, std::min(cap / 256 + 1, ctx->sms * 4)), 256, 0, S->stream>>>(cap, S->d_info);
  cudaError_t e = cudaStreamSynchronize(S->stream);
  if (e != cudaSuccess) {
    serve_shutdown(ctx);
    return cuda_fail(ctx, e, "rb_serve_start");
  }
  S->slot_ticket.assign(cap, 0);
  S->slot_iters.assign(cap, 0);
  S->slot_n.assign(cap, 0);
  S->slot_t0.assign(cap, Clock::now());
  S->free_slots.clear();
  for (int s = 0; s < cap; ++s) S->free_slots.insert(s);
  S->t_start = S->t_last = Clock::now();
  S->running = true;
  S->th = std::thread(serve_loop, ctx);
  return RB_OK;
}

int rb_serve_stop(rb_ctx *ctx, int drain) {
  if (!ctx) return RB_ERR_ARG;
  ServeState *S = ctx->serve;
  if (!S) return set_error(ctx, RB_ERR_STATE, "server not started");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop_req = true;
    S->drain = drain != 0;
  }
  S->cv.notify_all();
  if (S->th.joinable()) S->th.join();
  return S->error;
}

int rb_serve_submit(rb_ctx *ctx, const double mu[2], int n, uint64_t *ticket) {
  if (!ctx) return RB_ERR_ARG;
  if (!mu || !ticket) return set_error(ctx, RB_ERR_ARG, "NULL argument");
  ServeState *S = ctx->serve;
  if (!S) return set_error(ctx, RB_ERR_STATE, "server not running");
  const int nn = n == 0 ? ctx->ops.n_max : n;
  if (nn < 1 || nn > ctx->ops.n_max) return set_error(ctx, RB_ERR_ARG, "n = %d out of range", n);
  std::lock_guard<std::mutex> lk(S->mu);
  if (!S->running || S->stop_req) return set_error(ctx, RB_ERR_STATE, "server not running");
  Pending q;
  q.ticket = S->next_ticket++;
  q.mu[0] = mu[0];
  q.mu[1] = mu[1];
  q.n = nn;
  q.t0 = Clock::now();
  S->queue.push_back(q);
  S->inflight.insert(q.ticket);
  *ticket = q.ticket;
  S->cv.notify_one();
  return RB_OK;
}

int rb_serve_poll(rb_ctx *ctx, uint64_t ticket, double *u_out, double *p_out, rb_query_info *info) {
  if (!ctx) return RB_ERR_ARG;
  ServeState *S = ctx->serve;
  if (!S) return set_error(ctx, RB_ERR_STATE, "server not started");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->done.find(ticket);
  if (it == S->done.end()) {
    if (S->inflight.count(ticket)) return RB_PENDING;
    return set_error(ctx, RB_ERR_ARG, "unknown or already polled ticket %llu", (unsigned long long)ticket);
  }
  if (u_out) memcpy(u_out, it->second.u.data(), 8 * it->second.u.size());
  if (p_out && !it->second.p.empty()) memcpy(p_out, it->second.p.data(), 8 * it->second.p.size());
  if (info) *info = it->second.info;
  S->done.erase(it);
  return RB_OK;
}

int rb_serve_slots(rb_ctx *ctx) {
  if (!ctx) return RB_ERR_ARG;
  if (!ctx->serve) return set_error(ctx, RB_ERR_STATE, "server not started");
  return ctx->serve->cap;
}

int rb_serve_stats(rb_ctx *ctx, double *p50_s, double *p99_s, double *solves_per_s) {
  if (!ctx) return RB_ERR_ARG;
  ServeState *S = ctx->serve;
  if (!S) return set_error(ctx, RB_ERR_STATE, "server not started");
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> v = S->lat;
  double a = 0, b = 0;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    a = v[(size_t)(0.50 * (v.size() - 1))];
    b = v[(size_t)(0.99 * (v.size() - 1))];
  }
  const double dt = std::chrono::duration<double>(S->t_last - S->t_start).count();
  if (p50_s) *p50_s = a;
  if (p99_s) *p99_s = b;
  if (solves_per_s) *solves_per_s = dt > 0 ? S->completed / dt : 0.0;
  return S->error;
}

}  // extern "C"
