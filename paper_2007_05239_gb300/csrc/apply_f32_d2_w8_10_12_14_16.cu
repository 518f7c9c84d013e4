// F32 form, d = 2, window widths {8, 10, 12, 14, 16}.
#include "launch.cuh"

namespace ml {
template ml_status run_layer_w<float, 2, 8>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 2, 10>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 2, 12>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 2, 14>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 2, 16>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_batch_w<2, 8>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<2, 10>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<2, 12>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<2, 14>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<2, 16>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
}  // namespace ml
