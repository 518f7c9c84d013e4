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

ML_DECL_BATCH_W(3, 4)
ML_DECL_BATCH_W(3, 5)
ML_DECL_BATCH_W(3, 6)
ML_DECL_BATCH_W(3, 7)
ML_DECL_BATCH_W(3, 8)
ML_DECL_BATCH_W(3, 10)
ML_DECL_BATCH_W(3, 12)
ML_DECL_BATCH_W(3, 14)
ML_DECL_BATCH_W(3, 16)

ml_status run_layer_f32_d3(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                           cudaStream_t st)
{
    return run_layer_d<float, 3>(p, v, o, w, st);
}

ml_status run_batch_f32_d3(ml_plan_s *const *L, int T, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st)
{
    switch (L[0]->W) {
    case 4: return run_batch_w<3, 4>(L, T, v, o, st);
    case 5: return run_batch_w<3, 5>(L, T, v, o, st);
    case 6: return run_batch_w<3, 6>(L, T, v, o, st);
    case 7: return run_batch_w<3, 7>(L, T, v, o, st);
    case 8: return run_batch_w<3, 8>(L, T, v, o, st);
    case 10: return run_batch_w<3, 10>(L, T, v, o, st);
    case 12: return run_batch_w<3, 12>(L, T, v, o, st);
    case 14: return run_batch_w<3, 14>(L, T, v, o, st);
    case 16: return run_batch_w<3, 16>(L, T, v, o, st);
    default: return fail(ML_ERR_ARG, "window width out of range");
    }
}
}  // namespace ml
