// F32 form, d = 3: dispatch over the window half-width (kernels in kernels.cuh).
#include "launch.cuh"

namespace ml {
ML_DECL_LAYER_M(float, 3, 2)
ML_DECL_LAYER_M(float, 3, 3)
ML_DECL_LAYER_M(float, 3, 4)
ML_DECL_LAYER_M(float, 3, 5)
ML_DECL_LAYER_M(float, 3, 6)
ML_DECL_LAYER_M(float, 3, 7)
ML_DECL_LAYER_M(float, 3, 8)

ml_status run_layer_f32_d3(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                           cudaStream_t st)
{
    return run_layer_d<float, 3>(p, v, o, w, st);
}
}  // namespace ml
