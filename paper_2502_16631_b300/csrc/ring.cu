// Pageable images through the pinned ring (placeholder until the ring lands).
#include "snap.h"
#include "runtime_internal.h"

namespace snapk {
int ring_checkpoint(snap_set_s *, uint8_t *, uint64_t, int, uint64_t *, double, double, double) { return SNAP_EINVAL; }
int ring_restore(snap_set_s *, const uint8_t *, uint64_t, const ImageHeader &, double, double, double)
{
    return SNAP_EINVAL;
}
void ring_free(snap_set_s *) {}
}  // namespace snapk
