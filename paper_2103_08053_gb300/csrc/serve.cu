// serve.cu -- tc_submit / tc_poll (placeholder until the serving loop lands).
#include "api_internal.h"

using namespace tcg;

void tcg::serve_shutdown(tc_ctx*) {}

extern "C" {
tc_status tc_submit(tc_ctx* ctx, const tc_csr* g, uint64_t* ticket) {
    (void)g; (void)ticket;
    return ctx_fail(ctx, TC_ERR_UNSUPPORTED, "tc_submit: not built yet");
}
tc_status tc_poll(tc_ctx* ctx, uint64_t ticket, uint64_t* count) {
    (void)ticket; (void)count;
    return ctx_fail(ctx, TC_ERR_UNSUPPORTED, "tc_poll: not built yet");
}
tc_status tc_drain(tc_ctx* ctx) { return ctx_fail(ctx, TC_ERR_UNSUPPORTED, "tc_drain: not built yet"); }
}
