// One layer of the fast summation: spread -> fold -> forward transforms ->
// multiplier -> backward transforms -> interpolation + epilogue, launched on
// one stream.  Included by the per-precision translation units.
#pragma once

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "ml_internal.h"

namespace ml {

// Allow `bytes` of dynamic shared memory for `kernel`: the default limit
// covers static plus dynamic shared memory up to 48 KB; above that the
// per-kernel maximum is raised (refused beyond the device's opt-in limit).
template <typename K>
static ml_status set_smem(K kernel, size_t bytes)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes", __FILE__, __LINE__);
    if (fa.sharedSizeBytes + bytes > 48 * 1024) {
        if (fa.sharedSizeBytes + bytes > 227 * 1024)
            return fail(ML_ERR_ARG, "a tile needs " + std::to_string(bytes) + " B of shared memory, beyond the limit");
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
    }
    return ML_OK;
}

// FP32 spreading: the box of cells written into each subproblem tile (int4,
// pack_box), 16-byte aligned after the subproblem and group tiles
static_assert(kGroupSubs <= kGroupSubsMax, "group size of the plan above the boxed group sum's limit");
static int4 *tile_boxes(void *scratch, int nsub, int ngroups, int64_t tile_bytes)
{
    const size_t off = ((size_t)(nsub + ngroups) * (size_t)tile_bytes + 15) & ~(size_t)15;
    return reinterpret_cast<int4 *>(static_cast<char *>(scratch) + off);
}

// One real trigonometric transform along an axis (k_axis): 32 x 64 tiles, or
// 16 x 32 tiles when the large ones would leave most SMs idle
template <typename T>
static void launch_axis(const T *in, T *out, const T *M, int64_t A, int J, int Ko, int64_t C, cudaStream_t st)
{
    const int64_t big = ((A * C + 63) / 64) * ((Ko + 31) / 32);
    if (big >= 2 * (int64_t)sm_count()) {
        k_axis<T><<<dim3((unsigned)((A * C + 63) / 64), (unsigned)((Ko + 31) / 32)), 256, 0, st>>>(in, out, M, (int)A, J,
                                                                                              Ko, (int)C);
    } else {
        k_axis_small<T><<<dim3((unsigned)((A * C + 31) / 32), (unsigned)((Ko + 15) / 16)), 128, 0, st>>>(
            in, out, M, (int)A, J, Ko, (int)C);
    }
}

// Offset of the row-product slots of the FP32 spreading after a tile of
// tile_bytes (16-byte aligned), or 0 when the path does not apply or the
// slots would not fit next to the tile (the plan limits its vectors per pass
// so that, where the slots fit for one vector, they fit for every pass width)
template <int D, int W, int NV>
static size_t row_spread_offset(size_t tile_bytes)
{
    if (!RowSpread<D, W, NV>::on) return 0;
    const size_t off = (tile_bytes + 15) & ~(size_t)15;
    return off + RowSpread<D, W, NV>::smem <= kRowSpreadBudget ? off : 0;
}

// Shared memory for the FP32 spreading's staged points (the nv inputs u of
// each of at most sub_max points, and their sorted indices when the layer
// has a spreading order) after `bytes`, when it fits the budget: returns the
// new total and sets *off (0: not staged; the kernel then reads the inputs
// twice).  Staging changes no result.
static size_t add_spread_staging(size_t bytes, int sub_max, int nv, bool with_index, int *off)
{
    const size_t o = (bytes + 15) & ~(size_t)15;
    const size_t need = (size_t)sub_max * sizeof(float) * (nv + (with_index ? 1 : 0));
    if (sub_max > 0 && o + need <= kRowSpreadBudget) {
        *off = (int)o;
        return o + need;
    }
    *off = 0;
    return bytes;
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
    SpreadArgs sa{};
    sa.sub_bin = p->sub_bin.as<int>();
    sa.sub_start = p->sub_start.as<int>();
    sa.sub_count = p->sub_count.as<int>();
    sa.perm = p->perm.as<int>();
    sa.sidx = p->sidx.as<int>();
    sa.coords = p->coords.p;
    sa.wts = p->wts.as<float2>();
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
    static_assert(sizeof(sa.kbp) == sizeof(p->kbp), "window polynomial table sizes");
    memcpy(sa.kbp, p->kbp, sizeof(sa.kbp));
    sa.scratch = w.scratch;
    // FP32: each subproblem tile records the box of cells it wrote (after
    // the tiles in the scratch, tile_boxes); the group sums read only those
    const int64_t tile_elems = (int64_t)tc * nv;
    int4 *sub_box = nullptr;
    if (f32 && p->ngroups > 0) {
        sub_box = tile_boxes(w.scratch, p->nsub, p->ngroups, tile_elems * (int64_t)sizeof(T));
        sa.sub_box = sub_box;
    }
    if (p->nsub > 0) {
        ProfScope pr("spread", st);
        if (f32) {
            size_t smem = (size_t)tc * nv * sizeof(int);
            const size_t roff = row_spread_offset<D, W, NV>(smem);
            if (roff) {
                sa.rows_off = (int)roff;
                smem = roff + RowSpread<D, W, NV>::smem;
            }
            smem = add_spread_staging(smem, p->sub_max, NV, sa.sidx != nullptr, &sa.stage_off);
            ML_TRY(set_smem(k_spread_f32<D, W, NV>, smem));
            k_spread_f32<D, W, NV><<<p->nsub, 256, smem, st>>>(sa);
        } else {
            const size_t smem = (size_t)tc * nv * sizeof(int2) + (size_t)p->sub_max * nv * sizeof(double);
            ML_TRY(set_smem(k_spread_f64<D, W, NV>, smem));
            k_spread_f64<D, W, NV><<<p->nsub, 256, smem, st>>>(sa);
        }
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess)
            return fail(ML_ERR_CUDA, std::string("spread launch failed (") + cudaGetErrorString(le) + "): d=" +
                                         std::to_string(D) + " W=" + std::to_string(W) + " nv=" + std::to_string(nv) +
                                         " bin=" + std::to_string(g.B) + " tile=" + std::to_string(tc) +
                                         " nsub=" + std::to_string(p->nsub) + " sub_max=" + std::to_string(p->sub_max));
    }
    // ---- sum each group of subproblem tiles, then fold the group tiles into
    //      the active grid (work0)
    T *gtile = static_cast<T *>(w.scratch) + (int64_t)p->nsub * tile_elems;
    if (p->ngroups > 0) {
        ProfScope pr("group_sum", st);
        if (sub_box) {
            const int plane = (D == 1 ? g.Pt : g.Pt * g.Pt) * nv;
            const int threads = std::min(512, std::max(64, (plane + 31) / 32 * 32));
            k_group_sum_box<D><<<dim3((unsigned)p->ngroups, D == 3 ? (unsigned)g.Pt : 1u), threads, 0, st>>>(
                reinterpret_cast<const float *>(w.scratch), p->grp_sub.as<int>(), sub_box, g.Pt, nv,
                reinterpret_cast<float *>(gtile));
        } else {
            const int chunks = (int)std::min<int64_t>((tile_elems + 255) / 256, 64);
            k_group_sum<T><<<(unsigned)((int64_t)p->ngroups * chunks), 256, 0, st>>>(
                static_cast<const T *>(w.scratch), p->grp_sub.as<int>(), tile_elems, chunks, gtile);
        }
        ML_CUDA(cudaGetLastError());
    }
    FoldArgs fa{};
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
        int64_t cells = 1;
        for (int a = 0; a < D; ++a) cells *= g.B;
        const int ch = fold_chunks(g.nbins(), cells * nv, sm_count());
        if (f32) k_fold<T, D><<<(int)(g.nbins() * ch), 256, 0, st>>>(fa, ch);
        else k_fold<T, D, float2><<<(int)(g.nbins() * ch), 256, 0, st>>>(fa, ch);
    }
    ML_CUDA(cudaGetLastError());
    // ---- transforms (FP64 form: double-word grids, matrices and multiplier)
    T *bufs[2] = {static_cast<T *>(w.work0), static_cast<T *>(w.work1)};
    int cur = 0;
    int64_t Kpow = 1;  // K^a
    for (int a = 0; a < D; ++a) {
        int64_t A = 1;
        for (int b = a + 1; b < D; ++b) A *= g.L[b];
        const int64_t C = Kpow * nv;
        ProfScope pr("axis", st);
        if (f32) {
            launch_axis<T>(bufs[cur], bufs[cur ^ 1], p->trig_f[a].as<T>(), A, g.L[a], g.K, C, st);
        } else {
            const int64_t outs = A * C * g.K;
            k_axis_dw<float2><<<(unsigned)((outs + 127) / 128), 128, 0, st>>>(
                reinterpret_cast<const float2 *>(bufs[cur]), reinterpret_cast<float2 *>(bufs[cur ^ 1]),
                p->trig_f[a].as<float2>(), (int)A, g.L[a], g.K, (int)C);
        }
        cur ^= 1;
        Kpow *= g.K;
    }
    ML_CUDA(cudaGetLastError());
    {
        const int64_t slots = Kpow;
        const int blocks = (int)std::min<int64_t>((slots * nv + 255) / 256, 4096);
        ProfScope pr("mult", st);
        if (f32)
            k_mult<T><<<blocks, 256, 0, st>>>(bufs[cur], p->mult_d.as<T>(), slots, nv);
        else
            k_mult_dw<float2><<<blocks, 256, 0, st>>>(reinterpret_cast<float2 *>(bufs[cur]), p->mult_d.as<float2>(), slots,
                                              nv);
    }
    for (int a = D - 1; a >= 0; --a) {
        Kpow /= g.K;
        int64_t A = 1;
        for (int b = a + 1; b < D; ++b) A *= g.L[b];
        const int64_t C = Kpow * nv;
        ProfScope pr("axis", st);
        if (f32) {
            launch_axis<T>(bufs[cur], bufs[cur ^ 1], p->trig_b[a].as<T>(), A, g.K, g.L[a], C, st);
        } else {
            const int64_t outs = A * C * g.L[a];
            k_axis_dw<float2><<<(unsigned)((outs + 127) / 128), 128, 0, st>>>(
                reinterpret_cast<const float2 *>(bufs[cur]), reinterpret_cast<float2 *>(bufs[cur ^ 1]),
                p->trig_b[a].as<float2>(), (int)A, g.K, g.L[a], (int)C);
        }
        cur ^= 1;
    }
    ML_CUDA(cudaGetLastError());
    // ---- interpolation + epilogue
    InterpArgs ia{};
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
    memcpy(ia.kbp, p->kbp, sizeof(ia.kbp));
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
    ia.sorted_final = o.sorted_final;
    ia.nsub = p->nsub;
    if (p->nsub > 0) {
        const size_t smem = (size_t)tc * nv * sizeof(T);
        ProfScope pr("interp", st);
        if (f32) {
            // two zero floats after the FP32 tile (read by the paired row loads)
            if constexpr (NV == 1 && W <= 5) {
                ML_TRY(set_smem(k_interp_f32_1v<D, W>, smem + 2 * sizeof(float)));
                k_interp_f32_1v<D, W><<<p->nsub, 256, smem + 2 * sizeof(float), st>>>(ia);
            } else {
                ML_TRY(set_smem(k_interp_f32<D, W, NV>, smem + 2 * sizeof(float)));
                k_interp_f32<D, W, NV><<<p->nsub, 256, smem + 2 * sizeof(float), st>>>(ia);
            }
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

// ------------------------------------------------------------------ batch
// All layers of a batch (see batchable) in one launch per stage.  The
// per-layer arguments live in one device blob owned by the first plan and
// are re-uploaded only when they change.
template <int D, int W, int NV>
ml_status run_batch_dm(ml_plan_s *const *L, int T, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st)
{
    using T_ = float;
    std::vector<SpreadArgs> sa(T);
    std::vector<GroupArgs> ga(T);
    std::vector<FoldArgs> fa(T);
    std::vector<AxisArgs> ax((size_t)2 * D * T);
    std::vector<MultArgs> ma(T);
    std::vector<InterpArgs> ia(T);
    int max_nsub = 0, max_ng = 0, max_nbins = 0;
    int64_t max_tile = 0, max_slots = 0;
    unsigned max_px[2 * D], max_ky[2 * D];
    for (int s = 0; s < 2 * D; ++s) max_px[s] = max_ky[s] = 1;
    for (int t = 0; t < T; ++t) {
        ml_plan_s *p = L[t];
        const ApplyVec &vt = o.layer_vecs ? o.layer_vecs[t] : v;
        const GridGeom &g = p->g;
        const int tc = (int)g.tile_cells();
        const int64_t tile_elems = (int64_t)tc * NV;
        T_ *scratch = p->scratch.as<T_>();
        T_ *gtile = scratch + (int64_t)p->nsub * tile_elems;
        T_ *bufs[2] = {p->work[0].as<T_>(), p->work[1].as<T_>()};
        SpreadArgs &a = sa[t];
        a = SpreadArgs{};
        a.sub_bin = p->sub_bin.as<int>();
        a.sub_start = p->sub_start.as<int>();
        a.sub_count = p->sub_count.as<int>();
        a.perm = p->perm.as<int>();
        a.sidx = p->sidx.as<int>();
        a.coords = p->coords.p;
        a.dinv = o.normalized ? p->dinv.as<double>() : nullptr;
        a.X = vt.X;
        a.ldx = vt.ldx;
        a.nv = NV;
        a.B = g.B;
        a.Pt = g.Pt;
        a.nb0 = g.nb[0];
        a.nb1 = g.nb[1];
        a.m2d = 0.25 * (double)W * (double)W;
        a.bd = p->kb_shape;
        a.normd = p->kb_norm;
        a.m2f = (float)a.m2d;
        a.bf = (float)a.bd;
        a.normf = (float)a.normd;
        memcpy(a.kbp, p->kbp, sizeof(a.kbp));
        a.scratch = scratch;
        a.nsub = p->nsub;
        a.sub_max = p->sub_max;
        ga[t] = GroupArgs{scratch, p->grp_sub.as<int>(), tile_elems, gtile, p->ngroups};
        FoldArgs &f = fa[t];
        f.nbins = (int)g.nbins();
        f.bin_sub = p->bin_grp.as<int>();
        f.scratch = gtile;
        f.grid = bufs[0];
        f.nv = NV;
        f.B = g.B;
        f.Pt = g.Pt;
        f.R = g.R;
        f.nb0 = g.nb[0];
        f.nb1 = g.nb[1];
        f.nb2 = g.nb[2];
        f.L0 = g.L[0];
        f.L1 = g.L[1];
        f.L2 = g.L[2];
        int cur = 0;
        int64_t Kpow = 1;
        for (int ad = 0; ad < D; ++ad) {
            int64_t A = 1;
            for (int b2 = ad + 1; b2 < D; ++b2) A *= g.L[b2];
            const int64_t C = Kpow * NV;
            ax[(size_t)ad * T + t] = AxisArgs{bufs[cur], bufs[cur ^ 1], p->trig_f[ad].p, (int)A, g.L[ad], g.K, (int)C};
            max_px[ad] = std::max(max_px[ad], (unsigned)((A * C + 63) / 64));
            max_ky[ad] = std::max(max_ky[ad], (unsigned)((g.K + 31) / 32));
            cur ^= 1;
            Kpow *= g.K;
        }
        ma[t] = MultArgs{bufs[cur], p->mult_d.p, Kpow};
        max_slots = std::max(max_slots, Kpow);
        for (int ad = D - 1; ad >= 0; --ad) {
            Kpow /= g.K;
            int64_t A = 1;
            for (int b2 = ad + 1; b2 < D; ++b2) A *= g.L[b2];
            const int64_t C = Kpow * NV;
            const int sidx = 2 * D - 1 - ad;
            ax[(size_t)sidx * T + t] = AxisArgs{bufs[cur], bufs[cur ^ 1], p->trig_b[ad].p, (int)A, g.K, g.L[ad], (int)C};
            max_px[sidx] = std::max(max_px[sidx], (unsigned)((A * C + 63) / 64));
            max_ky[sidx] = std::max(max_ky[sidx], (unsigned)((g.L[ad] + 31) / 32));
            cur ^= 1;
        }
        InterpArgs &ip = ia[t];
        ip = InterpArgs{};
        memcpy(ip.kbp, p->kbp, sizeof(ip.kbp));
        ip.sub_bin = a.sub_bin;
        ip.sub_start = a.sub_start;
        ip.sub_count = a.sub_count;
        ip.perm = a.perm;
        ip.coords = a.coords;
        ip.dinv = a.dinv;
        ip.X = vt.X;
        ip.ldx = vt.ldx;
        ip.Y = vt.Y;
        ip.ldy = vt.ldy;
        ip.nv = NV;
        ip.nsub = p->nsub;
        ip.B = g.B;
        ip.Pt = g.Pt;
        ip.nb0 = g.nb[0];
        ip.nb1 = g.nb[1];
        ip.L0 = g.L[0];
        ip.L1 = g.L[1];
        ip.L2 = g.L[2];
        ip.m2f = a.m2f;
        ip.bf = a.bf;
        ip.normf = a.normf;
        ip.m2d = a.m2d;
        ip.bd = a.bd;
        ip.normd = a.normd;
        ip.grid = bufs[cur];
        ip.alpha = o.alpha;
        ip.shift = 0.0;
        ip.self = o.self;
        ip.normalized = o.normalized;
        ip.accumulate = o.accumulate;
        max_nsub = std::max(max_nsub, p->nsub);
        max_ng = std::max(max_ng, p->ngroups);
        max_nbins = std::max(max_nbins, (int)g.nbins());
        max_tile = std::max(max_tile, (int64_t)tc);
    }
    // pack and upload
    // the row-product slots follow the largest tile (one offset for all layers)
    size_t spread_batch_smem = (size_t)max_tile * NV * sizeof(int);
    {
        const size_t roff = row_spread_offset<D, W, NV>(spread_batch_smem);
        if (roff) {
            for (int t = 0; t < T; ++t) sa[t].rows_off = (int)roff;
            spread_batch_smem = roff + RowSpread<D, W, NV>::smem;
        }
        int max_sub = 0, soff = 0;
        bool any_sidx = false;
        for (int t = 0; t < T; ++t) {
            max_sub = std::max(max_sub, L[t]->sub_max);
            any_sidx = any_sidx || sa[t].sidx != nullptr;
        }
        spread_batch_smem = add_spread_staging(spread_batch_smem, max_sub, NV, any_sidx, &soff);
        for (int t = 0; t < T; ++t) sa[t].stage_off = soff;
    }
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_sa = 0, o_ga = align(o_sa + sizeof(SpreadArgs) * T), o_fa = align(o_ga + sizeof(GroupArgs) * T),
                 o_ax = align(o_fa + sizeof(FoldArgs) * T), o_ma = align(o_ax + sizeof(AxisArgs) * ax.size()),
                 o_ia = align(o_ma + sizeof(MultArgs) * T), total = align(o_ia + sizeof(InterpArgs) * T);
    std::vector<unsigned char> blob(total, 0);
    memcpy(blob.data() + o_sa, sa.data(), sizeof(SpreadArgs) * T);
    memcpy(blob.data() + o_ga, ga.data(), sizeof(GroupArgs) * T);
    memcpy(blob.data() + o_fa, fa.data(), sizeof(FoldArgs) * T);
    memcpy(blob.data() + o_ax, ax.data(), sizeof(AxisArgs) * ax.size());
    memcpy(blob.data() + o_ma, ma.data(), sizeof(MultArgs) * T);
    memcpy(blob.data() + o_ia, ia.data(), sizeof(InterpArgs) * T);
    ml_plan_s *p0 = L[0];
    DevBuf &ddev = o.desc ? o.desc->dev : p0->batch_desc;
    std::vector<unsigned char> &dhost = o.desc ? o.desc->host : p0->batch_host;
    if (dhost != blob) {
        ML_TRY(ddev.ensure(total));
        ML_CUDA(cudaMemcpyAsync(ddev.p, blob.data(), total, cudaMemcpyHostToDevice, st));
        ML_CUDA(cudaStreamSynchronize(st));   // the host blob is reused at once
        dhost.swap(blob);
    }
    unsigned char *d = ddev.as<unsigned char>();
    {
        ProfScope pr("spread", st);
        const size_t smem = spread_batch_smem;
        ML_TRY(set_smem(k_spread_f32_batch<D, W, NV>, smem));
        k_spread_f32_batch<D, W, NV><<<dim3(max_nsub, T), 256, smem, st>>>(reinterpret_cast<SpreadArgs *>(d + o_sa));
        ML_CUDA(cudaGetLastError());
    }
    {
        ProfScope pr("group_sum", st);
        const int chunks = (int)std::min<int64_t>((max_tile * NV + 255) / 256, 64);
        dim3 grid((unsigned)((int64_t)max_ng * chunks), (unsigned)T);
        k_group_sum_batch<T_><<<grid, 256, 0, st>>>(reinterpret_cast<GroupArgs *>(d + o_ga), chunks);
    }
    {
        ProfScope pr("fold", st);
        int64_t max_cells = 1;
        for (int t = 0; t < T; ++t) {
            int64_t c = 1;
            for (int a = 0; a < D; ++a) c *= L[t]->g.B;
            max_cells = std::max(max_cells, c);
        }
        const int ch = fold_chunks((int64_t)max_nbins * T, max_cells * NV, sm_count());
        k_fold_batch<T_, D><<<dim3(max_nbins * ch, T), 256, 0, st>>>(reinterpret_cast<FoldArgs *>(d + o_fa), ch);
    }
    for (int sidx = 0; sidx < 2 * D; ++sidx) {
        if (sidx == D) {
            ProfScope pr("mult", st);
            const int blocks = (int)std::min<int64_t>((max_slots * NV + 255) / 256, 1024);
            k_mult_batch<T_><<<dim3(blocks, T), 256, 0, st>>>(reinterpret_cast<MultArgs *>(d + o_ma), NV);
        }
        ProfScope pr("axis", st);
        k_axis_batch<T_><<<dim3(max_px[sidx], max_ky[sidx], T), 256, 0, st>>>(
            reinterpret_cast<AxisArgs *>(d + o_ax) + (size_t)sidx * T);
    }
    ML_CUDA(cudaGetLastError());
    {
        ProfScope pr("interp", st);
        const size_t smem = (size_t)max_tile * NV * sizeof(float) + 2 * sizeof(float);   // tile + 2 zeros
        if (o.layer_vecs) {
            ML_TRY(set_smem(k_interp_f32_batch<D, W, NV>, smem));
            k_interp_f32_batch<D, W, NV><<<dim3(max_nsub, T), 256, smem, st>>>(
                reinterpret_cast<InterpArgs *>(d + o_ia));
        } else {
            // enough CTAs to fill the GPU: split the layers into groups whose
            // partial sums are added in a fixed order afterwards
            const int G = std::max(1, std::min(T, (sm_count() * 6 + max_nsub - 1) / max_nsub));
            const int LG = (T + G - 1) / G;
            const int Gu = (T + LG - 1) / LG;
            const int64_t n = p0->n;
            float *part = nullptr;
            if (Gu > 1) {
                ML_TRY(p0->batch_part.ensure((size_t)Gu * n * NV * sizeof(float)));
                part = p0->batch_part.as<float>();
            }
            ML_TRY(set_smem(k_interp_f32_sum<D, W, NV>, smem));
            k_interp_f32_sum<D, W, NV><<<dim3(max_nsub, Gu), 256, smem, st>>>(reinterpret_cast<InterpArgs *>(d + o_ia),
                                                                             T, LG, part, n);
            if (Gu > 1) {
                ML_CUDA(cudaGetLastError());
                const int blocks = (int)std::min<int64_t>((n * NV + 255) / 256, sm_count() * 16);
                k_sum_parts<NV><<<blocks, 256, 0, st>>>(part, Gu, n, v.Y, v.ldy);
            }
        }
        ML_CUDA(cudaGetLastError());
    }
    for (int t = 0; t < T; ++t) L[t]->applied += NV;
    return ML_OK;
}

template <int D, int W>
ml_status run_batch_w(ml_plan_s *const *L, int T, const ApplyVec &v, const ApplyOpts &o, cudaStream_t st)
{
    if constexpr (W <= 8) {
        if (v.nv == 8) return run_batch_dm<D, W, 8>(L, T, v, o, st);
        if (v.nv == 4) return run_batch_dm<D, W, 4>(L, T, v, o, st);
    }
    if (v.nv == 1) return run_batch_dm<D, W, 1>(L, T, v, o, st);
    return fail(ML_ERR_ARG, "unsupported vectors per pass");
}

#define ML_DECL_BATCH_W(D, W)                                                                             \
    extern template ml_status run_batch_w<D, W>(ml_plan_s *const *, int, const ApplyVec &, const ApplyOpts &, \
                                                cudaStream_t);

}  // namespace ml
