// F32 form, d = 3: dispatch over the window width (kernels in kernels.cuh).
#include "launch.cuh"

namespace ml {
ML_DECL_LAYER_W(float, 3, 4)
ML_DECL_LAYER_W(float, 3, 5)
ML_DECL_LAYER_W(float, 3, 6)
ML_DECL_LAYER_W(float, 3, 7)
ML_DECL_LAYER_W(float, 3, 8)
ML_DECL_LAYER_W(float, 3, 10)
ML_DECL_LAYER_W(float, 3, 12)
ML_DECL_LAYER_W(float, 3, 14)
ML_DECL_LAYER_W(float, 3, 16)

ml_status run_layer_f32_d3(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                           cudaStream_t st)
{
    return run_layer_d<float, 3>(p, v, o, w, st);
}
}  // namespace ml
