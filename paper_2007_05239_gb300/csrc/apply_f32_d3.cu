// F32 form of one layer's fast summation for d = 3 (kernels in kernels.cuh).
#include "launch.cuh"

namespace ml {
ml_status run_layer_f32_d3(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                           cudaStream_t st)
{
    return run_layer_d<float, 3>(p, v, o, w, st);
}
}  // namespace ml
