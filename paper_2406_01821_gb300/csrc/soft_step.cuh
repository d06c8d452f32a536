// A soft step (forward + adjoint) on scratch the caller allocated once: for loops that run many
// steps of one shape (the evolution loop's fine-tuning), with no allocation per step, so that the
// steps can be captured in a CUDA graph.
#pragma once
#include "rs_internal.cuh"

namespace rs {

// Adam on the parameters after a step's gradients, applied by the gradient reduction itself:
// a always, b for pairs, t for thresholds; m and v hold two moments per condition.
struct SoftAdam {
    float *a = nullptr, *b = nullptr, *t = nullptr, *m = nullptr, *v = nullptr;
    int step = 0;
    float lr = 0.f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
};

// Bytes of scratch for a soft step over at most `cap_p` sets and `cap_c` conditions on a dataset
// of N samples.
size_t soft_scratch_bytes(int64_t cap_c, int cap_p, int64_t N);

// soft_step_known on `scratch` (soft_scratch_bytes(cap_c, cap_p, N) bytes, 256-byte aligned);
// a.b.P <= cap_p and the batch's condition capacity <= cap_c. `repeat`: the previous step on this
// scratch had the same structure (sets, rules, features, classes; only a, b, t differ), so its
// validation and set order are reused. `adam` (may be null): the update applied to the
// conditions of the batch's sets once their gradients are reduced (a.dloss must be given).
rs_status soft_step_scratch(Ctx *ctx, const SoftArgs &a, int maxR, int maxC, void *scratch, int64_t cap_c,
                            int cap_p, bool repeat, const SoftAdam *adam, cudaStream_t stream);

// Validation of a soft batch once, before a run of steps: the status word (RS_ERR_INVALID /
// RS_ERR_TOO_LARGE as rs_eval_soft_fwd gives them) and the largest rule and condition counts of a
// set, which size the steps. Waits for the stream.
rs_status soft_validate(Ctx *ctx, const SoftArgs &a, int *maxR, int *maxC, cudaStream_t stream);

}  // namespace rs
