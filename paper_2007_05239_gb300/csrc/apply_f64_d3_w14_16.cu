// F64 form, d = 3, window widths {14, 16}.
#include "launch.cuh"

namespace ml {
template ml_status run_layer_w<double, 3, 14>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
template ml_status run_layer_w<double, 3, 16>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
}  // namespace ml
