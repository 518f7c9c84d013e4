// F32 form, d = 2, window half-width m in {5, 6, 7, 8}.
#include "launch.cuh"

namespace ml {
template ml_status run_layer_m<float, 2, 5>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_m<float, 2, 6>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_m<float, 2, 7>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_m<float, 2, 8>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
}  // namespace ml
