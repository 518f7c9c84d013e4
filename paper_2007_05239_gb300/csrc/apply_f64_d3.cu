// F64 form, d = 3: dispatch over the window width (kernels in kernels.cuh).
#include "launch.cuh"

namespace ml {
ML_DECL_LAYER_W(double, 3, 4)
ML_DECL_LAYER_W(double, 3, 5)
ML_DECL_LAYER_W(double, 3, 6)
ML_DECL_LAYER_W(double, 3, 7)
ML_DECL_LAYER_W(double, 3, 8)
ML_DECL_LAYER_W(double, 3, 10)
ML_DECL_LAYER_W(double, 3, 12)
ML_DECL_LAYER_W(double, 3, 14)
ML_DECL_LAYER_W(double, 3, 16)

ml_status run_layer_f64_d3(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                           cudaStream_t st)
{
    return run_layer_d<double, 3>(p, v, o, w, st);
}
}  // namespace ml
