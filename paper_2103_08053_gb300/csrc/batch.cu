// batch.cu -- tc_count_batch (placeholder until the batched kernel lands).
#include "api_internal.h"

using namespace tcg;

void tcg::batch_release(tc_ctx*) {}

extern "C" tc_status tc_count_batch(tc_ctx* ctx, const tc_csr* gs, int32_t k, uint64_t* counts_host, void* stream) {
    (void)gs; (void)k; (void)counts_host; (void)stream;
    return ctx_fail(ctx, TC_ERR_UNSUPPORTED, "tc_count_batch: not built yet");
}
