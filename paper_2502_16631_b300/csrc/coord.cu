// Two-phase coordination of one operation across ranks (host code only).
//
// Sec. 3.1: the lock action runs for every task before any task is
// checkpointed, and at exit each plugin learns whether the whole operation
// succeeded, so that a failure anywhere leaves every task's previous state
// in force.  Here each rank runs its local steps and, after the lock and
// after the run, combines its status with every other rank's through the
// caller's `agree` transport; a failure anywhere aborts everywhere.
#include "snap.h"
#include "runtime_internal.h"

namespace snapk {

int coordinate(const snap_coord_ops &o, void *ctx)
{
    int st = o.lock ? o.lock(ctx) : SNAP_OK;
    int g = o.agree(ctx, 0, st);
    if (g != SNAP_OK) return st != SNAP_OK ? st : SNAP_EPEER;
    st = o.run ? o.run(ctx) : SNAP_OK;
    g = o.agree(ctx, 1, st);
    if (g != SNAP_OK) {
        if (o.abort) o.abort(ctx);
        return st != SNAP_OK ? st : SNAP_EPEER;
    }
    if (o.commit) o.commit(ctx);
    return SNAP_OK;
}

}  // namespace snapk

extern "C" int snap_coordinate(const snap_coord_ops *ops, void *ctx)
{
    if (!ops || !ops->agree) return SNAP_EINVAL;
    return snapk::coordinate(*ops, ctx);
}
