// F32 form, d = 2: dispatch over the window width (kernels in kernels.cuh).
#include "launch.cuh"

namespace ml {
ML_DECL_LAYER_W(float, 2, 4)
ML_DECL_LAYER_W(float, 2, 5)
ML_DECL_LAYER_W(float, 2, 6)
ML_DECL_LAYER_W(float, 2, 7)
ML_DECL_LAYER_W(float, 2, 8)
ML_DECL_LAYER_W(float, 2, 10)
ML_DECL_LAYER_W(float, 2, 12)
ML_DECL_LAYER_W(float, 2, 14)
ML_DECL_LAYER_W(float, 2, 16)

ml_status run_layer_f32_d2(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                           cudaStream_t st)
{
    return run_layer_d<float, 2>(p, v, o, w, st);
}
}  // namespace ml
