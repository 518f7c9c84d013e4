// F32 form, d = 3, window half-width m in {4}.
#include "launch.cuh"

namespace ml {
template ml_status run_layer_m<float, 3, 4>(ml_plan_s *, const ApplyVec &, const ApplyOpts &,
                                              const LayerWork &, cudaStream_t);
}  // namespace ml
