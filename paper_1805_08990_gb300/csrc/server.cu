// Serving entry points (placeholder until the grouped scheduler lands).
#include "dme_internal.h"

using namespace dme;

extern "C" {

dme_status dme_server_create(size_t, int, dme_server_t* out) {
    if (out) *out = nullptr;
    set_error("serving is not available in this build");
    return DME_EINVAL;
}

dme_status dme_submit(dme_server_t, const dme_plan_desc*, const double*, const double*, const double*,
                      const double*, const double*, const double*, double, int, uint64_t*) {
    set_error("serving is not available in this build");
    return DME_EINVAL;
}

dme_status dme_poll(dme_server_t, uint64_t, double*, int64_t) {
    set_error("serving is not available in this build");
    return DME_EINVAL;
}

const char* dme_server_stats(dme_server_t) { return "{}"; }

dme_status dme_server_destroy(dme_server_t) { return DME_OK; }

}  // extern "C"
