// F32 form, d = 1: dispatch over the window width (kernels in kernels.cuh).
#include "launch.cuh"

namespace ml {
ML_DECL_LAYER_W(float, 1, 4)
ML_DECL_LAYER_W(float, 1, 5)
ML_DECL_LAYER_W(float, 1, 6)
ML_DECL_LAYER_W(float, 1, 7)
ML_DECL_LAYER_W(float, 1, 8)
ML_DECL_LAYER_W(float, 1, 10)
ML_DECL_LAYER_W(float, 1, 12)
ML_DECL_LAYER_W(float, 1, 14)
ML_DECL_LAYER_W(float, 1, 16)

ML_DECL_BATCH_W(1, 4)
ML_DECL_BATCH_W(1, 5)
ML_DECL_BATCH_W(1, 6)
ML_DECL_BATCH_W(1, 7)
ML_DECL_BATCH_W(1, 8)
ML_DECL_BATCH_W(1, 10)
ML_DECL_BATCH_W(1, 12)
ML_DECL_BATCH_W(1, 14)
ML_DECL_BATCH_W(1, 16)

ml_status run_layer_f32_d1(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                           cudaStream_t st)
{
    return run_layer_d<float, 1>(p, v, o, w, st);
}

ml_status run_batch_f32_d1(ml_plan_s *const *L, int T, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st)
{
    switch (L[0]->W) {
    case 4: return run_batch_w<1, 4>(L, T, v, o, st);
    case 5: return run_batch_w<1, 5>(L, T, v, o, st);
    case 6: return run_batch_w<1, 6>(L, T, v, o, st);
    case 7: return run_batch_w<1, 7>(L, T, v, o, st);
    case 8: return run_batch_w<1, 8>(L, T, v, o, st);
    case 10: return run_batch_w<1, 10>(L, T, v, o, st);
    case 12: return run_batch_w<1, 12>(L, T, v, o, st);
    case 14: return run_batch_w<1, 14>(L, T, v, o, st);
    case 16: return run_batch_w<1, 16>(L, T, v, o, st);
    default: return fail(ML_ERR_ARG, "window width out of range");
    }
}
}  // namespace ml
