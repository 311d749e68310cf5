// rb_runtime.cu -- host runtime of librb: context, operator residency on the device,
// solve dispatch and error reporting. Implements the C ABI declared in include/rb.h.
#include <cstdlib>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "rb_ctx.h"

// ---------------------------------------------------------------------------------------
// error reporting: one message per (context, thread)
namespace {
thread_local std::unordered_map<const rb_ctx *, std::string> t_err;
}

namespace rb {

int set_error(const rb_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err[ctx] = buf;
  return code;
}

int cuda_fail(const rb_ctx *ctx, cudaError_t e, const char *what) {
  return set_error(ctx, RB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ctx_alloc(rb_ctx *ctx, void **p, size_t bytes, const char *what) {
  *p = nullptr;
  if (bytes == 0) return RB_OK;
  if (ctx->used + bytes > ctx->budget)
    return set_error(ctx, RB_ERR_OOM, "%s: %zu bytes exceed the memory budget (%zu of %zu used)",
                     what, bytes, ctx->used, ctx->budget);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_error(ctx, RB_ERR_OOM, "%s: cudaMalloc(%zu): %s", what, bytes, cudaGetErrorString(e));
  }
  ctx->used += bytes;
  ctx->sizes[*p] = bytes;
  return RB_OK;
}

void ctx_free(rb_ctx *ctx, void *p) {
  if (!p) return;
  auto it = ctx->sizes.find(p);
  if (it != ctx->sizes.end()) {
    ctx->used -= it->second;
    ctx->sizes.erase(it);
  }
  cudaFree(p);
}

// grow-only device scratch
int Scratch::reserve(rb_ctx *ctx, size_t bytes, const char *what) {
  if (bytes <= cap) return RB_OK;
  ctx_free(ctx, ptr);
  ptr = nullptr;
  cap = 0;
  int rc = ctx_alloc(ctx, &ptr, bytes, what);
  if (rc == RB_OK) cap = bytes;
  return rc;
}

void Scratch::release(rb_ctx *ctx) {
  ctx_free(ctx, ptr);
  ptr = nullptr;
  cap = 0;
}

static void free_ops(rb_ctx *ctx) {
  drop_pressure_modes(ctx);
  for (void *p : ctx->op_allocs) ctx_free(ctx, p);
  ctx->op_allocs.clear();
  ctx->loaded = false;
  ctx->ops = DevOps{};
  mixed_release(ctx);
}

int op_alloc(rb_ctx *ctx, void **p, size_t bytes, const char *what) {
  int rc = ctx_alloc(ctx, p, bytes, what);
  if (rc == RB_OK && *p) ctx->op_allocs.push_back(*p);
  return rc;
}

static int upload(rb_ctx *ctx, void **dst, const void *src, size_t bytes, const char *what) {
  int rc = op_alloc(ctx, dst, bytes, what);
  if (rc != RB_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  return RB_OK;
}

// ---------------------------------------------------------------------------------------
// per-kernel event timing
static cudaEvent_t pool_event(rb_ctx *ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

int prof_begin(rb_ctx *ctx, int kind, cudaStream_t st) {
  if (!ctx->prof) return -1;
  ProfMark m{kind, pool_event(ctx), pool_event(ctx)};
  if (!m.a || !m.b) return -1;
  cudaEventRecord(m.a, st);
  ctx->marks.push_back(m);
  return (int)ctx->marks.size() - 1;
}

unsigned long long *prof_issued(rb_ctx *ctx, int kind) {
  return ctx->prof && ctx->d_issued ? ctx->d_issued + kind : nullptr;
}

void prof_end(rb_ctx *ctx, int mark, cudaStream_t st) {
  if (mark < 0 || mark >= (int)ctx->marks.size()) return;
  cudaEventRecord(ctx->marks[mark].b, st);
}

void prof_collect(rb_ctx *ctx) {
  for (auto &m : ctx->marks) {
    float ms = 0.f;
    if (cudaEventSynchronize(m.b) == cudaSuccess && cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
      ctx->prof_ms[m.kind] += ms;
      ctx->prof_n[m.kind] += 1;
    }
    ctx->event_pool.push_back(m.a);
    ctx->event_pool.push_back(m.b);
  }
  ctx->marks.clear();
}

// ---------------------------------------------------------------------------------------
// FP64 path: one fused kernel per batch (all Newton iterations in-kernel), then pressure.
int solve_fp64(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq, const int *d_n,
               double *d_u, double *d_p, rb_query_info *d_info, cudaStream_t st) {
  const DevOps &o = ctx->ops;
  NewtonParams p{};
  p.o = o;
  p.mu = d_mu;
  p.theta = d_theta;
  p.nsz = d_n;
  p.nq = nq;
  p.max_iter = ctx->cfg.max_iter;
  p.tol_upd = ctx->cfg.tol_update;
  p.tol_res = ctx->cfg.tol_res;
  p.u_out = d_u;
  p.info = d_info;
  const size_t smem_in = fp64_smem_bytes(o, true);
  p.j_in_smem = smem_in <= (size_t)ctx->max_smem ? 1 : 0;
  const size_t smem = fp64_smem_bytes(o, p.j_in_smem != 0);
  if (smem > (size_t)ctx->max_smem)
    return set_error(ctx, RB_ERR_ARG, "operator set too large for the FP64 kernel (%zu B smem)", smem);
  // resident CTAs per SM: 2048 threads / kThreads, and the shared memory of one SM
  const int per_sm =
      std::max(1, std::min(2048 / kThreads, (int)((size_t)ctx->smem_per_sm / (smem + 1024))));
  p.grid = std::max(1, std::min(nq, per_sm * ctx->sms));
  if (!p.j_in_smem) {
    int rc = ctx->jscratch.reserve(ctx, sizeof(double) * (size_t)p.grid * o.n_max * o.n_max,
                                   "FP64 Jacobian scratch");
    if (rc != RB_OK) return rc;
    p.jscratch = (double *)ctx->jscratch.ptr;
  }
  const int mk = prof_begin(ctx, RB_K_NEWTON_FP64, st);
  cudaError_t e = launch_newton_fp64(p, ctx->sms, st);
  prof_end(ctx, mk, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_newton_fp64 launch");
  return RB_OK;
}

int solve_pressure(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq,
                   const int *d_n, const double *d_u, double *d_p, rb_query_info *d_info,
                   cudaStream_t st) {
  const DevOps &o = ctx->ops;
  if (!d_p || o.m <= 0 || !o.B) return RB_OK;
  PressureParams pp{};
  pp.o = o;
  pp.mu = d_mu;
  pp.theta = d_theta;
  pp.nsz = d_n;
  pp.nq = nq;
  pp.u = d_u;
  pp.p_out = d_p;
  pp.info = d_info;
  if (pressure_smem_bytes(o) > (size_t)ctx->max_smem)
    return set_error(ctx, RB_ERR_ARG, "pressure system too large");
  const int mk = prof_begin(ctx, RB_K_PRESSURE, st);
  cudaError_t e = launch_pressure(pp, ctx->sms, st);
  prof_end(ctx, mk, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_pressure launch");
  return RB_OK;
}

int solve_device_impl(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq,
                      const int *d_n, double *d_u, double *d_p, rb_query_info *d_info,
                      cudaStream_t st, const int *h_n) {
  if (!ctx->loaded) return set_error(ctx, RB_ERR_STATE, "no operators loaded");
  if (serve_running(ctx))
    return set_error(ctx, RB_ERR_STATE, "the server owns this context's batch state; stop it first");
  // pressure by reconstruction (Sec. 4.2): the velocity solve without recovery, then p = P_hat u
  const bool recon = ctx->cfg.pressure_method == RB_PRESSURE_RECONSTRUCT && d_p;
  if (recon && !ctx->d_PT)
    return set_error(ctx, RB_ERR_STATE, "pressure reconstruction needs rb_load_pressure_modes");
  if (nq == 0) return RB_OK;
  if (recon) {
    int rc = solve_device_impl(ctx, d_mu, d_theta, nq, d_n, d_u, nullptr, d_info, st, h_n);
    if (rc != RB_OK) return rc;
    return reconstruct_impl(ctx, d_u, nq, d_n, d_p, st);
  }
  // per-query status is needed to gate pressure recovery
  rb_query_info *info = d_info;
  if (!info && d_p && ctx->ops.m > 0) {
    int rc = ctx->info_scratch.reserve(ctx, sizeof(rb_query_info) * (size_t)nq, "info scratch");
    if (rc != RB_OK) return rc;
    info = (rb_query_info *)ctx->info_scratch.ptr;
  }
  if (ctx->cfg.precision == RB_PREC_MIXED)  // pressure recovery included
    return solve_mixed(ctx, d_mu, d_theta, nq, d_n, h_n, d_u, d_p, info, st);
  int rc = solve_fp64(ctx, d_mu, d_theta, nq, d_n, d_u, d_p, info, st);
  if (rc != RB_OK) return rc;
  return solve_pressure(ctx, d_mu, d_theta, nq, d_n, d_u, d_p, info, st);
}

// host-buffer staging: one device block for mu/theta, n, u, p, info
int stage_solve(rb_ctx *ctx, const double *mu, const double *theta, int nq, const int *n,
                double *u_out, double *p_out, rb_query_info *info) {
  if (!ctx) return RB_ERR_ARG;
  if (!ctx->loaded) return set_error(ctx, RB_ERR_STATE, "no operators loaded");
  if (nq < 0 || (nq > 0 && (!(mu || theta) || !u_out)))
    return set_error(ctx, RB_ERR_ARG, "bad arguments to rb_solve");
  if (nq == 0) return RB_OK;
  const DevOps &o = ctx->ops;
  const int in_w = theta ? o.n_theta : 2;
  const bool recon = ctx->cfg.pressure_method == RB_PRESSURE_RECONSTRUCT;
  if (recon && p_out && !ctx->d_PT)
    return set_error(ctx, RB_ERR_STATE, "pressure reconstruction needs rb_load_pressure_modes");
  const int m = !p_out ? 0 : (recon ? ctx->m_r : (o.m > 0 ? o.m : 0));
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_in = al(sizeof(double) * (size_t)nq * in_w), b_n = al(sizeof(int) * (size_t)nq);
  const size_t b_u = al(sizeof(double) * (size_t)nq * o.n_max), b_p = al(sizeof(double) * (size_t)nq * m);
  const size_t b_i = al(sizeof(rb_query_info) * (size_t)nq);
  int rc = ctx->stage.reserve(ctx, b_in + b_n + b_u + b_p + b_i, "solve staging");
  if (rc != RB_OK) return rc;
  char *base = (char *)ctx->stage.ptr;
  double *d_in = (double *)base;
  int *d_n = n ? (int *)(base + b_in) : nullptr;
  double *d_u = (double *)(base + b_in + b_n);
  double *d_p = m ? (double *)(base + b_in + b_n + b_u) : nullptr;
  rb_query_info *d_info = (rb_query_info *)(base + b_in + b_n + b_u + b_p);
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(d_in, theta ? theta : mu, sizeof(double) * (size_t)nq * in_w,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n) e = cudaMemcpyAsync(d_n, n, sizeof(int) * (size_t)nq, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_solve upload");
  rc = solve_device_impl(ctx, theta ? nullptr : d_in, theta ? d_in : nullptr, nq, d_n, d_u, d_p,
                         d_info, st, n);
  if (rc != RB_OK) return rc;
  e = cudaMemcpyAsync(u_out, d_u, sizeof(double) * (size_t)nq * o.n_max, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && m) e = cudaMemcpyAsync(p_out, d_p, sizeof(double) * (size_t)nq * m, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && info) e = cudaMemcpyAsync(info, d_info, sizeof(rb_query_info) * (size_t)nq, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_solve");
  return mixed_solve_status(ctx, 1);
}

}  // namespace rb

using namespace rb;

// ---------------------------------------------------------------------------------------
extern "C" {

void rb_config_default(rb_config *cfg) {
  if (!cfg) return;
  cfg->precision = RB_PREC_FP64;
  cfg->tol_update = 1e-10;
  cfg->tol_res = 1e-10;
  cfg->max_iter = 50;
  cfg->mem_budget = 0;
  cfg->use_graph = 1;
  // RB_AUTOTUNE=0 starts from the untuned launch variants (for profilers, whose serialised
  // timing would skew the tuner's choices; RB_GEMM_PAIRS then fixes the GEMM variants)
  const char *at = getenv("RB_AUTOTUNE");
  cfg->autotune = (at && *at) ? (atoi(at) != 0) : 1;
  cfg->theta_family = RB_THETA_TRIG;
  cfg->serve_slots = 0;
  cfg->pressure_method = RB_PRESSURE_RECOVER;
}

int rb_create(rb_ctx **out, const rb_config *cfg, int device) {
  if (!out) return RB_ERR_ARG;
  *out = nullptr;
  rb_ctx *ctx = new rb_ctx();
  if (cfg) ctx->cfg = *cfg; else rb_config_default(&ctx->cfg);
  if (ctx->cfg.max_iter < 1 || ctx->cfg.precision < RB_PREC_FP64 || ctx->cfg.precision > RB_PREC_MIXED ||
      ctx->cfg.serve_slots < 0 || ctx->cfg.theta_family < RB_THETA_TRIG ||
      ctx->cfg.theta_family > RB_THETA_POLY || ctx->cfg.pressure_method < RB_PRESSURE_RECOVER ||
      ctx->cfg.pressure_method > RB_PRESSURE_RECONSTRUCT ||
      !(ctx->cfg.tol_update >= 0) || !(ctx->cfg.tol_res >= 0)) {
    delete ctx;
    return RB_ERR_ARG;
  }
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->cc_major, cudaDevAttrComputeCapabilityMajor, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return RB_ERR_CUDA;
  }
  ctx->budget = ctx->cfg.mem_budget ? ctx->cfg.mem_budget : (size_t)(0.8 * (double)free_b);
  *out = ctx;
  return RB_OK;
}

void rb_destroy(rb_ctx *ctx) {
  if (!ctx) return;
  serve_shutdown(ctx);
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_ops(ctx);
  ctx->stage.release(ctx);
  ctx->jscratch.release(ctx);
  ctx->info_scratch.release(ctx);
  ctx->eval_scratch.release(ctx);
  for (auto &kv : ctx->sizes) cudaFree(kv.first);
  ctx->sizes.clear();
  prof_collect(ctx);
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  ctx->event_pool.clear();
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  t_err.erase(ctx);
  delete ctx;
}

const char *rb_last_error(rb_ctx *ctx) {
  auto it = t_err.find(ctx);
  return it == t_err.end() ? "" : it->second.c_str();
}

int rb_load_operators(rb_ctx *ctx, const rb_operators *ops) {
  if (!ctx) return RB_ERR_ARG;
  if (!ops) return set_error(ctx, RB_ERR_ARG, "ops is NULL");
  if (serve_running(ctx)) return set_error(ctx, RB_ERR_STATE, "stop the server before reloading");
  serve_shutdown(ctx);
  const int n = ops->n_max;
  if (n < 1 || n > RB_N_MAX) return set_error(ctx, RB_ERR_ARG, "n_max %d out of range 1..%d", n, RB_N_MAX);
  if (ops->q_a < 1 || ops->q_c < 1 || ops->q_f < 1 || ops->q_a > RB_Q_MAX || ops->q_c > RB_Q_MAX ||
      ops->q_f > RB_Q_MAX || ops->q_b < 0 || ops->q_b > RB_Q_MAX)
    return set_error(ctx, RB_ERR_ARG, "affine term counts out of range 1..%d", RB_Q_MAX);
  if (ops->dtype_c != RB_F64 && ops->dtype_c != RB_F32 && ops->dtype_c != RB_BF16)
    return set_error(ctx, RB_ERR_ARG, "bad dtype_c");
  if (!ops->A || !ops->C || !ops->f) return set_error(ctx, RB_ERR_ARG, "A, C and f are required");
  const bool pres = ops->B != nullptr;
  if (pres && (ops->m < 1 || ops->m > RB_M_MAX || ops->q_b < 1 || !ops->As || !ops->Cs || !ops->fs))
    return set_error(ctx, RB_ERR_ARG, "pressure operators incomplete or m out of range 1..%d", RB_M_MAX);
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_ops(ctx);
  DevOps o{};
  o.n_max = n;
  o.m = pres ? ops->m : 0;
  o.q_a = ops->q_a;
  o.q_c = ops->q_c;
  o.q_f = ops->q_f;
  o.q_b = pres ? ops->q_b : 0;
  o.n_theta = o.q_a + o.q_c + o.q_f + o.q_b;
  o.theta_family = ctx->cfg.theta_family;
  const size_t nn = (size_t)n, ncube = nn * nn * nn;
  const int dt = ops->dtype_c;
  const size_t csz = dt == RB_F64 ? sizeof(double) : (dt == RB_F32 ? sizeof(float) : 2);
  int rc = RB_OK;
  void *p = nullptr;
  if ((rc = upload(ctx, &p, ops->A, sizeof(double) * o.q_a * nn * nn, "A")) != RB_OK) goto fail;
  o.A = (const double *)p;
  if ((rc = upload(ctx, &p, ops->f, sizeof(double) * o.q_f * nn, "f")) != RB_OK) goto fail;
  o.f = (const double *)p;
  if ((rc = upload(ctx, &p, ops->C, csz * o.q_c * ncube, "C")) != RB_OK) goto fail;
  ctx->d_C = p;
  ctx->c_dtype = dt;
  if ((rc = op_alloc(ctx, &p, sizeof(double) * o.q_c * ncube, "Dt (FP64)")) != RB_OK) goto fail;
  o.Dt = (const double *)p;
  {
    cudaError_t e = launch_build_dt(ctx->d_C, dt, (double *)o.Dt, n, o.q_c, ctx->sms, ctx->stream);
    if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "build Dt"); goto fail; }
  }
  if (pres) {
    const size_t m = (size_t)o.m;
    if ((rc = upload(ctx, &p, ops->B, sizeof(double) * o.q_b * m * m, "B")) != RB_OK) goto fail;
    o.B = (const double *)p;
    if ((rc = upload(ctx, &p, ops->As, sizeof(double) * o.q_a * m * nn, "As")) != RB_OK) goto fail;
    o.As = (const double *)p;
    if ((rc = upload(ctx, &p, ops->fs, sizeof(double) * o.q_f * m, "fs")) != RB_OK) goto fail;
    o.fs = (const double *)p;
    void *cs_store = nullptr;
    if ((rc = upload(ctx, &cs_store, ops->Cs, csz * o.q_c * nn * nn * m, "Cs")) != RB_OK) goto fail;
    if (dt != RB_F64) {
      if ((rc = op_alloc(ctx, &p, sizeof(double) * o.q_c * nn * nn * m, "Cs (FP64)")) != RB_OK) goto fail;
      cudaError_t e = launch_convert(cs_store, dt, (double *)p, o.q_c * nn * nn * m, ctx->sms, ctx->stream);
      if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "convert Cs"); goto fail; }
      o.Cs = (const double *)p;
    } else {
      o.Cs = (const double *)cs_store;
    }
  }
  {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "rb_load_operators"); goto fail; }
  }
  ctx->ops = o;
  ctx->loaded = true;
  return RB_OK;
fail:
  cudaStreamSynchronize(ctx->stream);
  free_ops(ctx);
  return rc;
}

int rb_solve(rb_ctx *ctx, const double *mu, int n_queries, const int *n, double *u_out,
             double *p_out, rb_query_info *info) {
  if (!ctx) return RB_ERR_ARG;
  if (!mu && n_queries > 0) return set_error(ctx, RB_ERR_ARG, "mu is NULL");
  cudaSetDevice(ctx->device);
  return stage_solve(ctx, mu, nullptr, n_queries, n, u_out, p_out, info);
}

int rb_solve_theta(rb_ctx *ctx, const double *theta, int n_queries, const int *n, double *u_out,
                   double *p_out, rb_query_info *info) {
  if (!ctx) return RB_ERR_ARG;
  if (!theta && n_queries > 0) return set_error(ctx, RB_ERR_ARG, "theta is NULL");
  cudaSetDevice(ctx->device);
  return stage_solve(ctx, nullptr, theta, n_queries, n, u_out, p_out, info);
}

int rb_solve_device(rb_ctx *ctx, const double *d_mu, int n_queries, const int *d_n, double *d_u,
                    double *d_p, rb_query_info *d_info, void *cuda_stream) {
  return rb_solve_device_sized(ctx, d_mu, n_queries, d_n, nullptr, d_u, d_p, d_info, cuda_stream);
}

int rb_solve_device_sized(rb_ctx *ctx, const double *d_mu, int n_queries, const int *d_n,
                          const int *h_n, double *d_u, double *d_p, rb_query_info *d_info,
                          void *cuda_stream) {
  if (!ctx) return RB_ERR_ARG;
  if (n_queries < 0 || (n_queries > 0 && (!d_mu || !d_u)) || (h_n && !d_n))
    return set_error(ctx, RB_ERR_ARG, "bad arguments to rb_solve_device");
  cudaSetDevice(ctx->device);
  return solve_device_impl(ctx, d_mu, nullptr, n_queries, d_n, d_u, d_p, d_info,
                           (cudaStream_t)cuda_stream, h_n);
}

int rb_solve_device_status(rb_ctx *ctx, int wait) {
  if (!ctx) return RB_ERR_ARG;
  cudaSetDevice(ctx->device);
  return mixed_solve_status(ctx, wait);
}

int rb_eval(rb_ctx *ctx, const double *mu, int n_queries, int n, const double *u, int precision,
            double *R_out, double *J_out) {
  if (!ctx) return RB_ERR_ARG;
  if (!ctx->loaded) return set_error(ctx, RB_ERR_STATE, "no operators loaded");
  if (n < 1 || n > ctx->ops.n_max || n_queries < 0 || (n_queries > 0 && (!mu || !u || !R_out)))
    return set_error(ctx, RB_ERR_ARG, "bad arguments to rb_eval");
  if (n_queries == 0) return RB_OK;
  cudaSetDevice(ctx->device);
  const size_t nq = (size_t)n_queries, nn = (size_t)n;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_mu = al(16 * nq), b_u = al(8 * nq * nn), b_R = al(8 * nq * nn), b_J = al(8 * nq * nn * nn);
  int rc = ctx->eval_scratch.reserve(ctx, b_mu + b_u + b_R + b_J, "eval scratch");
  if (rc != RB_OK) return rc;
  char *base = (char *)ctx->eval_scratch.ptr;
  double *d_mu = (double *)base, *d_u = (double *)(base + b_mu), *d_R = (double *)(base + b_mu + b_u);
  double *d_J = (double *)(base + b_mu + b_u + b_R);
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(d_mu, mu, 16 * nq, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_u, u, 8 * nq * nn, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_eval upload");
  if (precision == RB_PREC_FP64) {
    EvalParams p{ctx->ops, d_mu, n_queries, n, d_u, d_R, d_J};
    e = launch_eval_fp64(p, ctx->sms, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k_eval_fp64");
  } else {
    rc = eval_mixed(ctx, d_mu, n_queries, n, d_u, precision, d_R, d_J, st);
    if (rc != RB_OK) return rc;
  }
  e = cudaMemcpyAsync(R_out, d_R, 8 * nq * nn, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && J_out) e = cudaMemcpyAsync(J_out, d_J, 8 * nq * nn * nn, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_eval");
  return RB_OK;
}

int rb_tuning(rb_ctx *ctx, int i, int *out6, float *ms3) {
  if (!ctx) return RB_ERR_ARG;
  return mixed_tuning(ctx, i, out6, ms3);
}

int rb_profile(rb_ctx *ctx, int enable) {
  if (!ctx) return RB_ERR_ARG;
  cudaSetDevice(ctx->device);
  prof_collect(ctx);
  for (int k = 0; k < RB_K_COUNT; ++k) {
    ctx->prof_ms[k] = 0.0;
    ctx->prof_n[k] = 0;
  }
  if (enable && !ctx->d_issued) {
    void *p = nullptr;
    const int rc = ctx_alloc(ctx, &p, 8 * RB_K_COUNT, "profile counters");
    if (rc != RB_OK) return rc;
    ctx->d_issued = (unsigned long long *)p;
  }
  if (ctx->d_issued) {
    const cudaError_t e = cudaMemset(ctx->d_issued, 0, 8 * RB_K_COUNT);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "profile counters");
  }
  ctx->prof = enable != 0;
  return RB_OK;
}

int rb_profile_issued(rb_ctx *ctx, int kernel, double *flops) {
  if (!ctx || !flops) return RB_ERR_ARG;
  if (kernel < 0 || kernel >= RB_K_COUNT) return set_error(ctx, RB_ERR_ARG, "kernel id %d", kernel);
  cudaSetDevice(ctx->device);
  unsigned long long v = 0;
  if (ctx->d_issued) {
    const cudaError_t e = cudaMemcpy(&v, ctx->d_issued + kernel, 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "profile counters");
  }
  *flops = (double)v;
  return RB_OK;
}

int rb_profile_read(rb_ctx *ctx, int kernel, double *total_ms, long long *launches) {
  if (!ctx) return RB_ERR_ARG;
  if (kernel < 0 || kernel >= RB_K_COUNT) return set_error(ctx, RB_ERR_ARG, "kernel id %d", kernel);
  cudaSetDevice(ctx->device);
  prof_collect(ctx);
  if (total_ms) *total_ms = ctx->prof_ms[kernel];
  if (launches) *launches = ctx->prof_n[kernel];
  return RB_OK;
}

int rb_gepp_solve(rb_ctx *ctx, int n, int batch, const double *M, const double *rhs,
                  double *x_out, int *status) {
  if (!ctx) return RB_ERR_ARG;
  if (n < 1 || n > 4096 || batch < 0 || (batch > 0 && (!M || !rhs || !x_out || !status)))
    return set_error(ctx, RB_ERR_ARG, "bad arguments to rb_gepp_solve");
  if (batch == 0) return RB_OK;
  cudaSetDevice(ctx->device);
  const size_t nb = (size_t)batch, nn = (size_t)n;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_M = al(8 * nb * nn * nn), b_x = al(8 * nb * nn), b_s = al(4 * nb);
  int rc = ctx->eval_scratch.reserve(ctx, b_M + b_x + b_s, "gepp scratch");
  if (rc != RB_OK) return rc;
  char *base = (char *)ctx->eval_scratch.ptr;
  double *d_M = (double *)base, *d_x = (double *)(base + b_M);
  int *d_s = (int *)(base + b_M + b_x);
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(d_M, M, 8 * nb * nn * nn, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_x, rhs, 8 * nb * nn, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_gepp_solve upload");
  e = launch_gepp_fp64(d_M, d_x, n, batch, d_s, ctx->sms, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "k_gepp_fp64");
  e = cudaMemcpyAsync(x_out, d_x, 8 * nb * nn, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status, d_s, 4 * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "rb_gepp_solve");
  return RB_OK;
}

}  // extern "C"
