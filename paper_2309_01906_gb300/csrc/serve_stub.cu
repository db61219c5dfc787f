// placeholder translation unit for batching and serving entry points
#include "api_internal.h"

using namespace hp;

extern "C" {
hp_status hp_serve_create(size_t mem_budget_bytes, int max_slots, int n_streams, hp_server** out) {
  (void)mem_budget_bytes; (void)max_slots; (void)n_streams; (void)out;
  return fail(HP_EUNSUPPORTED, "serving is not built yet");
}
hp_status hp_serve_submit(hp_server* s, const hp_nest* shape, const void* const* in_dev, void* out_dev,
                          uint64_t* ticket) {
  (void)s; (void)shape; (void)in_dev; (void)out_dev; (void)ticket;
  return fail(HP_EUNSUPPORTED, "serving is not built yet");
}
hp_status hp_serve_poll(hp_server* s, uint64_t ticket, int timeout_us) {
  (void)s; (void)ticket; (void)timeout_us;
  return fail(HP_EUNSUPPORTED, "serving is not built yet");
}
hp_status hp_serve_stats(const hp_server* s, double* p50, double* p99, double* p999, double* nps) {
  (void)s; (void)p50; (void)p99; (void)p999; (void)nps;
  return fail(HP_EUNSUPPORTED, "serving is not built yet");
}
void hp_serve_destroy(hp_server* s) { (void)s; }
}
