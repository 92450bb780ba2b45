// Serving loop (placeholder until the continuous-batching scheduler lands).
#include "ctx.h"

namespace mm {
mm_status serve_start() { return MM_OK; }
void serve_stop() {}
}  // namespace mm

extern "C" {
mm_status mm_submit(const mm_problem *, mm_dtype, mm_mode, uint64_t *) { return MM_EUNSUPPORTED; }
mm_status mm_poll(uint64_t, mm_status *, double *, double *) { return MM_EUNSUPPORTED; }
mm_status mm_wait(uint64_t, double, mm_status *, double *, double *) { return MM_EUNSUPPORTED; }
mm_status mm_serve_stats(int64_t *, int64_t *, int64_t *, int64_t *) { return MM_EUNSUPPORTED; }
}
