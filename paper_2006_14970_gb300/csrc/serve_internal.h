// Level-granular serving support (api.cu, used by server.cu): a job's work-list plan over
// device buffers its owner holds, and launches that merge the ready level passes of
// several jobs into one work list.
#pragma once
#include "fgml.h"
#include "fgml_internal.h"

namespace fgml {

struct ServePlan;

// Bytes of each of the two intermediate-level buffers a w x h job needs (0: none).
size_t serve_level_bytes(int w, int h, int dtype, const fg_params &p);

// Whether the work list runs these parameters (Jacobi order, every level with sweeps).
bool serve_supported(const fg_params &p);

// Plans a w x h job. I and alpha rows must be on the 16-byte grid (pitches in elements;
// `padded`: rows readable up to the pitch); F and B receive the result (pitch d_pitch
// elements); lev0 and lev1 hold serve_level_bytes each. Tensor maps are encoded here,
// once per job.
fg_status serve_plan_create(int dtype, const fg_params &p, const void *I, long long I_pitch,
                            const void *A, long long A_pitch, bool padded, int w, int h, void *F,
                            void *B, long long d_pitch, void *lev0, void *lev1, ServePlan **out);
void serve_plan_destroy(ServePlan *plan);
// Level passes of the job after its coarse levels, and the pixels x sweeps of pass j.
int serve_plan_passes(const ServePlan *plan);
long long serve_plan_work(const ServePlan *plan, int j);

// One job's share of a launch: its coarse levels when `coarse` (its first launch), then
// passes [first, last), each waiting for the one before it inside the launch.
struct ServePart {
    const ServePlan *plan;
    int coarse;
    int first, last;
};

// Grows the work-list buffer of stream s's workspace to at least `worklist_bytes`.
fg_status serve_reserve(cudaStream_t s, size_t worklist_bytes);

// Enqueues on s: the coarse levels of the parts that start, then one work list over all
// parts' passes (their earlier passes must be complete).
fg_status serve_launch(int dtype, const fg_params &p, const ServePart *parts, int n, cudaStream_t s);

}  // namespace fgml
