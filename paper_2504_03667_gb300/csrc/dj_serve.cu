// Serving: placeholder entry points until the continuous-batching runtime lands.
#include <cstring>

#include "dj_internal.h"

using namespace dj;

extern "C" void dj_serve_opts_init(dj_serve_opts* o) {
  if (o) std::memset(o, 0, sizeof(*o));
}
extern "C" int dj_serve_create(const dj_serve_opts*, dj_server**) { return set_error(DJ_EUNSUPPORTED, "serving not built"); }
extern "C" int dj_serve_add_graph(dj_server*, const dj_graph*, int32_t*) { return set_error(DJ_EUNSUPPORTED, "serving not built"); }
extern "C" int dj_serve_submit(dj_server*, int32_t, int32_t, int32_t*, int32_t*, uint64_t*) { return set_error(DJ_EUNSUPPORTED, "serving not built"); }
extern "C" int dj_serve_poll(dj_server*, uint64_t, int*) { return set_error(DJ_EUNSUPPORTED, "serving not built"); }
extern "C" int dj_serve_wait(dj_server*, uint64_t, int64_t) { return set_error(DJ_EUNSUPPORTED, "serving not built"); }
extern "C" int dj_serve_result(dj_server*, uint64_t, int32_t*, int32_t*) { return set_error(DJ_EUNSUPPORTED, "serving not built"); }
extern "C" int dj_serve_stats_get(dj_server*, dj_serve_stats*) { return set_error(DJ_EUNSUPPORTED, "serving not built"); }
extern "C" int dj_serve_destroy(dj_server*) { return DJ_OK; }
extern "C" int dj_serve(const dj_graph* const*, int32_t, int64_t, const int32_t*, const int32_t*, const double*,
                        int32_t* const*, int32_t* const*, const dj_serve_opts*, dj_serve_stats*) {
  return set_error(DJ_EUNSUPPORTED, "serving not built");
}
