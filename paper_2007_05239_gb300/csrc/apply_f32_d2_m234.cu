// F32 form, d = 2, window half-width m in {2, 3, 4}.
#include "launch.cuh"

namespace ml {
template ml_status run_layer_m<float, 2, 2>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_m<float, 2, 3>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_m<float, 2, 4>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
}  // namespace ml
