// rb_serve.cu -- continuous-batching server (placeholder).
#include "rb_ctx.h"

namespace rb {
void serve_shutdown(rb_ctx *) {}
}  // namespace rb

extern "C" {
int rb_serve_start(rb_ctx *ctx) { return ctx ? rb::set_error(ctx, RB_ERR_STATE, "server not built") : RB_ERR_ARG; }
int rb_serve_stop(rb_ctx *ctx, int) { return ctx ? RB_ERR_STATE : RB_ERR_ARG; }
int rb_serve_submit(rb_ctx *ctx, const double *, int, uint64_t *) { return ctx ? RB_ERR_STATE : RB_ERR_ARG; }
int rb_serve_poll(rb_ctx *ctx, uint64_t, double *, double *, rb_query_info *) { return ctx ? RB_ERR_STATE : RB_ERR_ARG; }
int rb_serve_stats(rb_ctx *ctx, double *, double *, double *) { return ctx ? RB_ERR_STATE : RB_ERR_ARG; }
}
