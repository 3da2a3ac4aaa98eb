// Continuous-batching server (ttc_server_*): placeholder entry points until
// the request loop lands; every call reports TTC_ERR_INTERNAL.
#include "graph.cuh"

namespace ttc {
void set_last_error(const std::string &m);
}

extern "C" {

ttc_server *ttc_server_create(const ttc_server_opts *) {
    ttc::set_last_error("server not available in this build");
    return nullptr;
}
void ttc_server_destroy(ttc_server *) {}
ttc_status ttc_serve_load(ttc_server *, const uint32_t *, const uint32_t *, const int64_t *, uint64_t, uint64_t *) {
    return TTC_ERR_INTERNAL;
}
ttc_status ttc_serve_submit(ttc_server *, uint64_t, const ttc_delta *, uint64_t *) { return TTC_ERR_INTERNAL; }
ttc_status ttc_serve_poll(ttc_server *, uint64_t, uint64_t *, double *) { return TTC_ERR_INTERNAL; }
ttc_status ttc_serve_drain(ttc_server *, double) { return TTC_ERR_INTERNAL; }
ttc_status ttc_server_info(ttc_server *, ttc_server_stats *) { return TTC_ERR_INTERNAL; }
}
