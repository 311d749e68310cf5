// rb_ctx.h -- the context object behind the opaque rb_ctx handle (internal).
#pragma once
#include <cuda_runtime.h>

#include <unordered_map>
#include <vector>

#include "rb_kernels.cuh"

struct rb_ctx;

namespace rb {

struct Scratch {
  void *ptr = nullptr;
  size_t cap = 0;
  int reserve(rb_ctx *ctx, size_t bytes, const char *what);
  void release(rb_ctx *ctx);
};

struct MixedState;   // low-precision layouts and per-batch state of the mixed path
struct ServeState;   // continuous-batching server

int set_error(const rb_ctx *ctx, int code, const char *fmt, ...);
int cuda_fail(const rb_ctx *ctx, cudaError_t e, const char *what);
int ctx_alloc(rb_ctx *ctx, void **p, size_t bytes, const char *what);
void ctx_free(rb_ctx *ctx, void *p);
int op_alloc(rb_ctx *ctx, void **p, size_t bytes, const char *what);

int solve_fp64(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq, const int *d_n,
               double *d_u, double *d_p, rb_query_info *d_info, cudaStream_t st);
// h_n: host copy of d_n if the caller has one (else read back when the batch needs bucketing)
int solve_mixed(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq, const int *d_n,
                const int *h_n, double *d_u, double *d_p, rb_query_info *d_info, cudaStream_t st);
int solve_pressure(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq,
                   const int *d_n, const double *d_u, double *d_p, rb_query_info *d_info,
                   cudaStream_t st);
int solve_device_impl(rb_ctx *ctx, const double *d_mu, const double *d_theta, int nq,
                      const int *d_n, double *d_u, double *d_p, rb_query_info *d_info,
                      cudaStream_t st, const int *h_n = nullptr);
int eval_mixed(rb_ctx *ctx, const double *d_mu, int nq, int n, const double *d_u, int precision,
               double *d_R, double *d_J, cudaStream_t st);
void mixed_release(rb_ctx *ctx);
// outcome of the asynchronous mixed solves enqueued so far (RB_OK, RB_PENDING, RB_ERR_TIMEOUT)
int mixed_solve_status(rb_ctx *ctx, int wait);
void serve_shutdown(rb_ctx *ctx);
bool serve_running(const rb_ctx *ctx);
// mixed-path pieces used by the server
int mixed_prepare(rb_ctx *ctx, int capacity, cudaStream_t st);
size_t mixed_slot_bytes(const rb_ctx *ctx);
int mixed_serve_step(rb_ctx *ctx, const double *d_mu, const int *d_n, double *d_u, double *d_p,
                     rb_query_info *d_info, const std::vector<int> &slots,
                     const std::vector<int> &slot_n, const std::vector<int> &slot_iters,
                     std::vector<int> &perm, cudaStream_t st);
int mixed_error_word(rb_ctx *ctx, cudaStream_t st);
int mixed_tuning(rb_ctx *ctx, int i, int *out6, float *ms3);
// pressure reconstruction (combined basis): p = P_hat u for every query
int reconstruct_impl(rb_ctx *ctx, const double *d_u, int nq, const int *d_n, double *d_p,
                     cudaStream_t st);
void drop_pressure_modes(rb_ctx *ctx);

// per-kernel event timing (active only while profiling is enabled)
struct ProfMark {
  int kind;
  cudaEvent_t a, b;
};
int prof_begin(rb_ctx *ctx, int kind, cudaStream_t st);  // returns a mark index or -1
void prof_end(rb_ctx *ctx, int mark, cudaStream_t st);
void prof_collect(rb_ctx *ctx);  // waits for recorded marks and accumulates them
// the device counter of the tensor FLOPs issued by kernels of `kind`, or null when not profiling
unsigned long long *prof_issued(rb_ctx *ctx, int kind);

}  // namespace rb

struct rb_ctx {
  rb_config cfg{};
  int device = 0, sms = 0, max_smem = 0, smem_per_sm = 0, cc_major = 0, cc_minor = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0, used = 0;
  std::unordered_map<void *, size_t> sizes;  // live allocations of this context
  // operators
  bool loaded = false;
  rb::DevOps ops{};
  std::vector<void *> op_allocs;
  void *d_C = nullptr;  // C in its storage type [q_c][n][n][n]
  int c_dtype = RB_F64;  // RB_F64, RB_F32 or RB_BF16
  double *d_PT = nullptr;  // pressure modes of a combined basis, transposed [n_max][m_r]
  int m_r = 0;
  // scratch
  rb::Scratch stage, jscratch, info_scratch, eval_scratch;
  rb::MixedState *mixed = nullptr;
  // profiling
  bool prof = false;
  std::vector<rb::ProfMark> marks;
  std::vector<cudaEvent_t> event_pool;
  double prof_ms[RB_K_COUNT] = {};
  long long prof_n[RB_K_COUNT] = {};
  unsigned long long *d_issued = nullptr;  // [RB_K_COUNT] tensor FLOPs issued (device counters)
  rb::ServeState *serve = nullptr;
};
