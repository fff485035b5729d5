// qieo_oneshot.cu -- one-call forms of the public API, written only in terms of the
// public entry points (include/qieo.h).
#include "../../include/qieo.h"

extern "C" {

// A batched run without a batch handle: the members advance `generations` generations
// together (one launch per generation for all of them), exactly as qieo_batch_run on a
// batch of the same members. The call returns when that work has finished (freeing the
// temporary batch waits for it).
qieo_status qieo_run_batch(qieo_instance *const *instances, int32_t n, int32_t generations)
{
    qieo_batch *b = nullptr;
    qieo_status st = qieo_create_batch(instances, n, &b);
    if (st != QIEO_OK) return st;
    st = qieo_batch_run(b, generations);
    const qieo_status st2 = qieo_destroy_batch(b);
    return st != QIEO_OK ? st : st2;
}

}  // extern "C"
