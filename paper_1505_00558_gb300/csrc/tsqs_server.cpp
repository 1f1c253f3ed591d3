// tsqs_server.cpp -- placeholder until the serving loop lands (returns EINVAL).
#include "tsqs.h"
extern "C" {
int tsqs_plan_autotune(int, size_t, size_t, void *, tsqs_plan *) { return TSQS_EINVAL; }
tsqs_server *tsqs_server_create(size_t, int, int) { return nullptr; }
int tsqs_server_submit(tsqs_server *, void *, size_t, size_t, int, uint64_t *) { return TSQS_EINVAL; }
int tsqs_server_progress(tsqs_server *) { return 0; }
int tsqs_server_poll(tsqs_server *, uint64_t, tsqs_result *) { return TSQS_EINVAL; }
int tsqs_server_drain(tsqs_server *) { return 0; }
void tsqs_server_destroy(tsqs_server *) {}
}
