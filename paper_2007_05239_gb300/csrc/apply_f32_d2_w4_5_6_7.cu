// F32 form, d = 2, window widths {4, 5, 6, 7}.
#include "launch.cuh"

namespace ml {
template ml_status run_layer_w<float, 2, 4>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 2, 5>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 2, 6>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 2, 7>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_batch_w<2, 4>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<2, 5>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<2, 6>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<2, 7>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
}  // namespace ml
