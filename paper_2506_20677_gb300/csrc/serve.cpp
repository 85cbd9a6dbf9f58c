// Serving loop and batched sorts (filled in below).
#include "ctx.h"

extern "C" {

ahs_status ahs_sort_batch(ahs_ctx*, const void*, void*, const uint32_t*, uint32_t*, const uint64_t*,
                          uint32_t, ahs_key_type, void*, ahs_batch_info_t*) {
    return AHS_ERR_UNIMPLEMENTED;
}
ahs_status ahs_serve_start(ahs_ctx*, const ahs_serve_config_t*) { return AHS_ERR_UNIMPLEMENTED; }
ahs_status ahs_serve_submit(ahs_ctx*, const ahs_request_t*, uint64_t*) { return AHS_ERR_UNIMPLEMENTED; }
ahs_status ahs_serve_poll(ahs_ctx*, uint64_t, int32_t, ahs_result_t*) { return AHS_ERR_UNIMPLEMENTED; }
ahs_status ahs_serve_stats(ahs_ctx*, ahs_serve_stats_t*) { return AHS_ERR_UNIMPLEMENTED; }
ahs_status ahs_serve_stop(ahs_ctx*) { return AHS_OK; }

}
