// F32 form, d = 3, window widths {7}.
#include "launch.cuh"

namespace ml {
template ml_status run_layer_w<float, 3, 7>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_batch_w<3, 7>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
}  // namespace ml
