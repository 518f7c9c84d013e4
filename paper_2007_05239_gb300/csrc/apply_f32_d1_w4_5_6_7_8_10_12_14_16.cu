// F32 form, d = 1, window widths {4, 5, 6, 7, 8, 10, 12, 14, 16}.
#include "launch.cuh"

namespace ml {
template ml_status run_layer_w<float, 1, 4>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 1, 5>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 1, 6>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 1, 7>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 1, 8>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 1, 10>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 1, 12>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 1, 14>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<float, 1, 16>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_batch_w<1, 4>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<1, 5>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<1, 6>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<1, 7>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<1, 8>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<1, 10>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<1, 12>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<1, 14>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
template ml_status run_batch_w<1, 16>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &,
                                         cudaStream_t);
}  // namespace ml
