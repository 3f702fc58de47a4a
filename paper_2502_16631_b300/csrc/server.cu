// Serving loop (placeholder until the server lands).
#include "snap.h"
#include "runtime_internal.h"

extern "C" {
int snap_server_create(snap_server *, uint64_t, uint64_t, const snap_opts *) { return SNAP_EINVAL; }
int snap_server_destroy(snap_server) { return SNAP_EINVAL; }
int snap_server_submit(snap_server, snap_set, int, void *, uint64_t, uint64_t *) { return SNAP_EINVAL; }
int snap_server_wait(snap_server, uint64_t, uint32_t, int *, snap_stats *) { return SNAP_EINVAL; }
}
