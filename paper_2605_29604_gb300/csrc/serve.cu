// serve.cu -- continuous-batching request loop (mis_submit / mis_poll / mis_wait).
#include "graph.h"
#include "tcmis.h"

namespace tcmis {
void serve_release_graph(mis_graph* g) { (void)g; }
}  // namespace tcmis

using namespace tcmis;

extern "C" {
int mis_submit(mis_graph* g, uint64_t seed, uint8_t* out_status, mis_ticket* ticket) {
    (void)g; (void)seed; (void)out_status; (void)ticket;
    return set_error(MIS_EINTERNAL, "serving not available");
}
int mis_poll(mis_ticket t) { (void)t; return set_error(MIS_EINVAL, "unknown ticket"); }
int mis_wait(mis_ticket t, int64_t us) { (void)t; (void)us; return set_error(MIS_EINVAL, "unknown ticket"); }
int mis_serve_configure(const mis_options* opt) { (void)opt; return MIS_OK; }
void mis_serve_shutdown(void) {}
}
