// One layer of the fast summation: spread -> fold -> forward transforms ->
// multiplier -> backward transforms -> interpolation + epilogue, launched on
// one stream.  Included by the per-precision translation units.
#pragma once

#include <algorithm>

#include "kernels.cuh"
#include "ml_internal.h"

namespace ml {

template <typename K>
static ml_status set_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
    }
    return ML_OK;
}

template <typename T, int D, int W, int NV>
static ml_status run_layer_dm(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                              cudaStream_t st)
{
    const GridGeom &g = p->g;
    const int nv = v.nv;
    const int tc = (int)g.tile_cells();
    const bool f32 = sizeof(T) == 4;
    // ---- spread
    SpreadArgs sa;
    sa.sub_bin = p->sub_bin.as<int>();
    sa.sub_start = p->sub_start.as<int>();
    sa.sub_count = p->sub_count.as<int>();
    sa.perm = p->perm.as<int>();
    sa.coords = p->coords.p;
    sa.wts = p->wts.as<double>();
    sa.offs = p->offs.as<int>();
    sa.sub_max = p->sub_max;
    sa.dinv = o.normalized ? p->dinv.as<double>() : nullptr;
    sa.X = v.X;
    sa.ldx = v.ldx;
    sa.nv = nv;
    sa.B = g.B;
    sa.Pt = g.Pt;
    sa.nb0 = g.nb[0];
    sa.nb1 = g.nb[1];
    sa.m2d = 0.25 * (double)W * (double)W;   // (W/2)^2
    sa.bd = p->kb_shape;
    sa.normd = p->kb_norm;
    sa.m2f = (float)sa.m2d;
    sa.bf = (float)sa.bd;
    sa.normf = (float)sa.normd;
    sa.scratch = w.scratch;
    if (p->nsub > 0) {
        ProfScope pr("spread", st);
        if (f32) {
            const size_t smem = (size_t)tc * nv * sizeof(int);
            ML_TRY(set_smem(k_spread_f32<D, W, NV>, smem));
            k_spread_f32<D, W, NV><<<p->nsub, 256, smem, st>>>(sa);
        } else {
            const size_t smem = (size_t)tc * nv * sizeof(double) * p->f64_warps +
                                (size_t)p->sub_max * (nv * sizeof(double) + sizeof(int));
            ML_TRY(set_smem(k_spread_f64<D, W, NV>, smem));
            k_spread_f64<D, W, NV><<<p->nsub, 32 * p->f64_warps, smem, st>>>(sa);
        }
        ML_CUDA(cudaGetLastError());
    }
    // ---- sum each group of subproblem tiles, then fold the group tiles into
    //      the active grid (work0)
    const int64_t tile_elems = (int64_t)tc * nv;
    T *gtile = static_cast<T *>(w.scratch) + (int64_t)p->nsub * tile_elems;
    if (p->ngroups > 0) {
        ProfScope pr("group_sum", st);
        dim3 grid((unsigned)((tile_elems + 255) / 256), (unsigned)p->ngroups);
        k_group_sum<T><<<grid, 256, 0, st>>>(static_cast<const T *>(w.scratch), p->grp_sub.as<int>(), tile_elems,
                                             gtile);
        ML_CUDA(cudaGetLastError());
    }
    FoldArgs fa;
    fa.bin_sub = p->bin_grp.as<int>();
    fa.scratch = gtile;
    fa.grid = w.work0;
    fa.nv = nv;
    fa.B = g.B;
    fa.Pt = g.Pt;
    fa.R = g.R;
    fa.nb0 = g.nb[0];
    fa.nb1 = g.nb[1];
    fa.nb2 = g.nb[2];
    fa.L0 = g.L[0];
    fa.L1 = g.L[1];
    fa.L2 = g.L[2];
    {
        ProfScope pr("fold", st);
        k_fold<T, D><<<(int)g.nbins(), 256, 0, st>>>(fa);
    }
    ML_CUDA(cudaGetLastError());
    // ---- transforms
    T *bufs[2] = {static_cast<T *>(w.work0), static_cast<T *>(w.work1)};
    int cur = 0;
    int64_t Kpow = 1;  // K^a
    for (int a = 0; a < D; ++a) {
        int64_t A = 1;
        for (int b = a + 1; b < D; ++b) A *= g.L[b];
        const int64_t C = Kpow * nv;
        dim3 grid((unsigned)((A * C + 63) / 64), (unsigned)((g.K + 31) / 32));
        ProfScope pr("axis", st);
        k_axis<T><<<grid, 256, 0, st>>>(bufs[cur], bufs[cur ^ 1], p->trig_f[a].as<T>(), (int)A, g.L[a], g.K, (int)C);
        cur ^= 1;
        Kpow *= g.K;
    }
    ML_CUDA(cudaGetLastError());
    {
        const int64_t slots = Kpow;
        const int blocks = (int)std::min<int64_t>((slots * nv + 255) / 256, 4096);
        ProfScope pr("mult", st);
        k_mult<T><<<blocks, 256, 0, st>>>(bufs[cur], p->mult_d.as<T>(), slots, nv);
    }
    for (int a = D - 1; a >= 0; --a) {
        Kpow /= g.K;
        int64_t A = 1;
        for (int b = a + 1; b < D; ++b) A *= g.L[b];
        const int64_t C = Kpow * nv;
        dim3 grid((unsigned)((A * C + 63) / 64), (unsigned)((g.L[a] + 31) / 32));
        ProfScope pr("axis", st);
        k_axis<T><<<grid, 256, 0, st>>>(bufs[cur], bufs[cur ^ 1], p->trig_b[a].as<T>(), (int)A, g.K, g.L[a], (int)C);
        cur ^= 1;
    }
    ML_CUDA(cudaGetLastError());
    // ---- interpolation + epilogue
    InterpArgs ia;
    ia.sub_bin = sa.sub_bin;
    ia.sub_start = sa.sub_start;
    ia.sub_count = sa.sub_count;
    ia.perm = sa.perm;
    ia.coords = sa.coords;
    ia.wts = sa.wts;
    ia.offs = sa.offs;
    ia.dinv = sa.dinv;
    ia.X = v.X;
    ia.ldx = v.ldx;
    ia.Y = v.Y;
    ia.ldy = v.ldy;
    ia.nv = nv;
    ia.B = g.B;
    ia.Pt = g.Pt;
    ia.nb0 = g.nb[0];
    ia.nb1 = g.nb[1];
    ia.L0 = g.L[0];
    ia.L1 = g.L[1];
    ia.L2 = g.L[2];
    ia.m2f = sa.m2f;
    ia.bf = sa.bf;
    ia.normf = sa.normf;
    ia.m2d = sa.m2d;
    ia.bd = sa.bd;
    ia.normd = sa.normd;
    ia.grid = bufs[cur];
    ia.alpha = o.alpha;
    ia.shift = o.shift;
    ia.self = o.self;
    ia.normalized = o.normalized;
    ia.accumulate = o.accumulate;
    ia.sorted_out = o.sorted_out;
    if (p->nsub > 0) {
        const size_t smem = (size_t)tc * nv * sizeof(T);
        ProfScope pr("interp", st);
        if (f32) {
            ML_TRY(set_smem(k_interp_f32<D, W, NV>, smem));
            k_interp_f32<D, W, NV><<<p->nsub, 256, smem, st>>>(ia);
        } else {
            ML_TRY(set_smem(k_interp_f64<D, W, NV>, smem));
            k_interp_f64<D, W, NV><<<p->nsub, 256, smem, st>>>(ia);
        }
        ML_CUDA(cudaGetLastError());
    }
    return ML_OK;
}

// Vector passes use NV = 1, 4 or 8 vectors; the wide passes exist for the
// small windows (W <= 8) where they matter for throughput.
template <typename T, int D, int W>
static ml_status run_layer_dmv(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                               cudaStream_t st)
{
    if constexpr (W <= 8) {
        if (v.nv == 8) return run_layer_dm<T, D, W, 8>(p, v, o, w, st);
        if (v.nv == 4) return run_layer_dm<T, D, W, 4>(p, v, o, w, st);
    }
    if (v.nv == 1) return run_layer_dm<T, D, W, 1>(p, v, o, w, st);
    return fail(ML_ERR_ARG, "unsupported vectors per pass");
}

// One layer pass for a given dimension and window width W (taps per
// dimension), instantiated per translation unit; the d = 3 instances are
// split over several files to keep each compile short.
template <typename T, int D, int W>
ml_status run_layer_w(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w, cudaStream_t st)
{
    return run_layer_dmv<T, D, W>(p, v, o, w, st);
}

#define ML_DECL_LAYER_W(T, D, W)                                                                       \
    extern template ml_status run_layer_w<T, D, W>(ml_plan_s *, const ApplyVec &, const ApplyOpts &, \
                                                   const LayerWork &, cudaStream_t);

// window widths with kernels: 4..8 and the even widths up to 16
template <typename T, int D>
static ml_status run_layer_d(ml_plan_s *p, const ApplyVec &v, const ApplyOpts &o, const LayerWork &w,
                             cudaStream_t st)
{
    switch (p->W) {
    case 4: return run_layer_w<T, D, 4>(p, v, o, w, st);
    case 5: return run_layer_w<T, D, 5>(p, v, o, w, st);
    case 6: return run_layer_w<T, D, 6>(p, v, o, w, st);
    case 7: return run_layer_w<T, D, 7>(p, v, o, w, st);
    case 8: return run_layer_w<T, D, 8>(p, v, o, w, st);
    case 10: return run_layer_w<T, D, 10>(p, v, o, w, st);
    case 12: return run_layer_w<T, D, 12>(p, v, o, w, st);
    case 14: return run_layer_w<T, D, 14>(p, v, o, w, st);
    case 16: return run_layer_w<T, D, 16>(p, v, o, w, st);
    default: return fail(ML_ERR_ARG, "window width out of range");
    }
}

}  // namespace ml
