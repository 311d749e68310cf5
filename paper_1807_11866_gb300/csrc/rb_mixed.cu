// rb_mixed.cu -- mixed-precision batched path (placeholder until the tensor-core kernels land).
#include "rb_ctx.h"

namespace rb {
int solve_mixed(rb_ctx *ctx, const double *, const double *, int, const int *, double *, double *,
                rb_query_info *, cudaStream_t) {
  return set_error(ctx, RB_ERR_ARG, "mixed precision path not built");
}
int eval_mixed(rb_ctx *ctx, const double *, int, int, const double *, int, double *, double *,
               cudaStream_t) {
  return set_error(ctx, RB_ERR_ARG, "mixed precision path not built");
}
void mixed_release(rb_ctx *) {}
}  // namespace rb
