// Uneven batches: one persistent launch over instances of different shapes.
#include <cuda_runtime.h>

#include "../../include/slos.h"
#include "plan.h"

namespace slos {
slos_status_t fail(slos_status_t st, const std::string &msg);
struct BatchedPlan {};
void batched_destroy(slos_plan_s *p) {
    delete p->batched;
    p->batched = nullptr;
}
}  // namespace slos

using namespace slos;

extern "C" {

slos_status_t slos_batched_plan(int, const int *, const int *, const int *const *, const slos_detection_t *,
                                slos_plan_t *out) {
    if (out) *out = nullptr;
    return fail(SLOS_ERR_UNSUPPORTED, "slos_batched_plan: not built yet");
}

slos_status_t slos_batched_query(slos_plan_t, int64_t *, int64_t *, size_t *) {
    return fail(SLOS_ERR_UNSUPPORTED, "slos_batched_query: not built yet");
}

slos_status_t slos_batched_forward(slos_plan_t, const void *, float *, void *, size_t, void *) {
    return fail(SLOS_ERR_UNSUPPORTED, "slos_batched_forward: not built yet");
}

slos_status_t slos_batched_autotune(slos_plan_t, const void *, float *, void *, size_t, const char *, void *) {
    return fail(SLOS_ERR_UNSUPPORTED, "slos_batched_autotune: not built yet");
}

}  // extern "C"
