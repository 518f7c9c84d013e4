// F64 form, d = 1: dispatch over the window width (kernels in kernels.cuh).
#include "launch.cuh"

namespace ml {
ML_DECL_LAYER_W(double, 1, 4)
ML_DECL_LAYER_W(double, 1, 5)
ML_DECL_LAYER_W(double, 1, 6)
ML_DECL_LAYER_W(double, 1, 7)
ML_DECL_LAYER_W(double, 1, 8)
ML_DECL_LAYER_W(double, 1, 10)
ML_DECL_LAYER_W(double, 1, 12)
ML_DECL_LAYER_W(double, 1, 14)
ML_DECL_LAYER_W(double, 1, 16)

ml_status run_layer_f64_d1(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                           cudaStream_t st)
{
    return run_layer_d<double, 1>(p, v, o, w, st);
}
}  // namespace ml
