// Batched multi-view rendering and the continuous-batching serving loop.
#include "aok_runtime.h"

using namespace aok;

namespace aok {
void batch_release(aok_ctx* ctx) { (void)ctx; }
}  // namespace aok

extern "C" {
int aok_render_batch(aok_ctx*, const aok_view*, uint32_t, void*) { return AOK_E_INVALID; }
int aok_set_launch(aok_ctx*, uint32_t, uint32_t, uint32_t) { return AOK_E_INVALID; }
int aok_get_launch(aok_ctx*, uint32_t*, uint32_t*, uint32_t*) { return AOK_E_INVALID; }
int aok_autotune(aok_ctx*, const aok_view*, uint32_t, void*, float*) { return AOK_E_INVALID; }
int aok_serve_start(aok_ctx*, uint32_t, uint32_t, uint32_t) { return AOK_E_INVALID; }
int aok_serve_stop(aok_ctx*) { return AOK_OK; }
int aok_serve_submit(aok_ctx*, const aok_request*, uint64_t*) { return AOK_E_INVALID; }
int aok_serve_poll(aok_ctx*, uint64_t, aok_frame*) { return AOK_E_INVALID; }
int aok_serve_wait(aok_ctx*, uint64_t, uint32_t, aok_frame*) { return AOK_E_INVALID; }
int aok_serve_release(aok_ctx*, uint64_t) { return AOK_E_INVALID; }
}
