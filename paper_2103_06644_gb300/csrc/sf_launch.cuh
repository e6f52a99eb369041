// sf_launch.cuh -- kernel launch sequences of the library, as templates over
// the depth encoding DT.  Each fit_<dt>.cu includes this file once and
// instantiates it for its encoding through SF_DEFINE_LAUNCHERS.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "sf_host.h"
#include "sf_kernels.cuh"
#include "sf_delta.cuh"
#include "sf_refine.cuh"

namespace sfh {
namespace {

sf::Codec codec_of(const sf_ctx* c) {
    if (c->depth_type == SF_DEPTH_DISPARITY_U16) return sf::Codec{c->disp_q, c->disp_mul, c->disp_add, c->disp_frac};
    return sf::Codec{c->depth_scale, 0, 0, 0.f};
}

cudaEvent_t take_event(sf_ctx* c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one launch with events when profiling is on.
struct StageTimer {
    sf_ctx* c; int stage; cudaStream_t st; cudaEvent_t a = nullptr;
    StageTimer(sf_ctx* c_, int s_, cudaStream_t st_) : c(c_), stage(s_), st(st_) {
        if (c->profiling) { a = take_event(c); cudaEventRecord(a, st); }
    }
    ~StageTimer() {
        if (a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, st);
            c->recs.push_back({stage, a, b});
        }
    }
};

// Launch with programmatic dependent launch: the kernel may be scheduled while
// the previous kernel of the stream finishes (its blocks wait in
// wait_for_prior_grid before reading that kernel's results), which hides the
// gap between the two launches.  After a copy or memset it is an ordinary
// launch.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);  // errors surface through cudaGetLastError
}

// The horizontal pass for tiles of seg = 8, 16, 32, 64 or 128 columns (one
// kernel each: their register budgets and serial chains differ).
template <int DT, int M>
void launch_hpass(dim3 grid, size_t smem, cudaStream_t st, const void* depth, const sf_ctx* c, int bits, int raw_z,
                  int seg) {
    auto go = [&](auto kernel) {
        launch_pdl(kernel, grid, dim3(sf::kHThreads), smem, st, depth, c->W, c->H, c->r, codec_of(c),
                   (const unsigned*)c->vmax, bits, raw_z, c->Wp, c->plane_elems, (void*)c->planes);
    };
    if (seg <= 8) go(sf::hpass_kernel<DT, M, 1, 8>);
    else if (seg <= 16) go(sf::hpass_kernel<DT, M, 1, 16>);
    else if (seg <= 32) go(sf::hpass_kernel<DT, M, 1>);
    else if (seg <= 64) go(sf::hpass_kernel<DT, M, 2>);
    else go(sf::hpass_kernel<DT, M, 4>);
}

template <int DT, int M>
void set_hpass_smem_one(int smem) {
    cudaFuncSetAttribute(sf::hpass_kernel<DT, M, 1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(sf::hpass_kernel<DT, M, 1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(sf::hpass_kernel<DT, M, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(sf::hpass_kernel<DT, M, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(sf::hpass_kernel<DT, M, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// Blocks per frame of the range pass: one wave of 256-thread blocks (8 per
// SM) over all frames, at most one block per 16 x 256 elements.
int range_blocks(const sf_ctx* c, size_t fe, int nfr) {
    const size_t per_frame = (size_t)c->sms * 8 / (size_t)std::max(1, nfr);
    return (int)std::max<size_t>(1, std::min((fe + 4095) / 4096, per_frame));
}

// One wave of resident blocks of a kernel (persistent grid-stride kernels).
template <typename K>
int resident_blocks(const sf_ctx* c, K kernel, int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0) != cudaSuccess || nb < 1) nb = 4;
    return nb * c->sms;
}

sf::Calib calib_of(const sf_ctx* c) {
    return sf::Calib{c->tx, c->ty, (float)(1.0 / c->K.fx), (float)(1.0 / c->K.fy)};
}

template <int DT, int M, bool U4 = false>
sf_status launch_pass(sf_ctx* c, int nfr, const void* depth, float* normals, float* offsets, float* curv,
                      int32_t* counts, cudaStream_t st) {
    const size_t fe = (size_t)c->W * c->H;
    constexpr int B = sf::base_method(M);  // range and horizontal pass depend on the moments only
    const int raw_z = sf::fixed_quantum<DT, B>() ? 1 : 0;
    const int bits = quant_bits(M, c->k);
    SF_CUDA(cudaMemsetAsync(c->vmax, 0, sizeof(unsigned) * nfr, st));
    if (!raw_z) {
        StageTimer t(c, 0, st);
        const int blocks = range_blocks(c, fe, nfr);
        sf::range_kernel<DT, B><<<dim3(blocks, nfr), 256, 0, st>>>(depth, fe, codec_of(c), c->vmax);
    }
    {
        StageTimer t(c, 1, st);
        const int seg = horizontal_seg(c, nfr);
        dim3 grid((c->W + seg - 1) / seg, (c->H + sf::kHThreads - 1) / sf::kHThreads, nfr);
        const int IW = seg + 2 * c->r;
        const size_t smem = sizeof(int) * sf::kHThreads * (size_t)(IW | 1);
        launch_hpass<DT, B>(grid, smem, st, depth, c, bits, raw_z, seg);
    }
    const sf::Calib cal = calib_of(c);
    const bool fb = c->precision_mode > 0 && c->flags;
    // the implicit |(a,b,c)| = 1 fits queue their exact moments with each flagged window
    constexpr bool kRich = !U4 && (M == SF_METHOD_DISPARITY || M == SF_METHOD_STANDARD);
    if (fb) SF_CUDA(cudaMemsetAsync(c->flag_count, 0, 3 * sizeof(unsigned), st));
    {
        StageTimer t(c, 2, st);
        const int band = vertical_band(c, nfr);
        dim3 grid((c->W + sf::kVThreads - 1) / sf::kVThreads, (c->H + band - 1) / band, nfr);
        const float tau = c->precision_mode == 2 ? INFINITY : c->tau;
        if constexpr (kRich) {
            if (fb)
                launch_pdl(sf::vpass_kernel<DT, M, U4, true>, grid, dim3(sf::kVThreads), 0, st, depth, c->W, c->H,
                           c->r, codec_of(c), c->vmax, bits, raw_z, c->Wp, c->plane_elems, c->planes, cal,
                           c->min_valid, c->require_center, band, normals, offsets, curv, counts, tau, c->flags,
                           c->flag_count, c->moments_q, (unsigned)c->moments_cap);
            else
                launch_pdl(sf::vpass_kernel<DT, M, U4>, grid, dim3(sf::kVThreads), 0, st, depth, c->W, c->H, c->r,
                           codec_of(c), c->vmax, bits, raw_z, c->Wp, c->plane_elems, c->planes, cal, c->min_valid,
                           c->require_center, band, normals, offsets, curv, counts, tau,
                           (unsigned long long*)nullptr, c->flag_count, (void*)nullptr, 0u);
        } else {
            launch_pdl(sf::vpass_kernel<DT, M, U4>, grid, dim3(sf::kVThreads), 0, st, depth, c->W, c->H, c->r,
                       codec_of(c), c->vmax, bits, raw_z, c->Wp, c->plane_elems, c->planes, cal, c->min_valid,
                       c->require_center, band, normals, offsets, curv, counts, tau, fb ? c->flags : nullptr,
                       c->flag_count, (void*)nullptr, 0u);
        }
    }
    {
        if (fb) {
            StageTimer t2(c, 3, st);
            if constexpr (kRich) {
                // mode 1: refine the queued windows, then re-sum those that need it;
                // mode 2: re-sum and refine every window
                const bool all = c->precision_mode == 2;
                static const int nb_refine = resident_blocks(c, sf::refine_kernel<DT, M>, 128);
                static const int nb_resum = resident_blocks(c, sf::resum_kernel<DT, M>, 128);
                if (!all)
                    sf::refine_kernel<DT, M><<<nb_refine, 128, 0, st>>>(
                        depth, c->W, c->H, c->r, codec_of(c), c->vmax, bits, c->plane_elems, nfr, c->planes,
                        c->rays64, c->flags, c->flag_count, c->queue_c, c->moments_q, (unsigned)c->moments_cap,
                        normals, offsets, curv);
                sf::resum_kernel<DT, M><<<nb_resum, 128, 0, st>>>(
                    depth, c->W, c->H, c->r, codec_of(c), c->vmax, bits, c->plane_elems, nfr, c->planes, c->rays64,
                    c->flags, c->flag_count, all ? nullptr : c->queue_c, c->moments_q, (unsigned)c->moments_cap,
                    normals, offsets, curv);
            } else {
                sf::resolve_kernel<DT, M, U4><<<c->sms * 8, 128, 0, st>>>(
                    c->W, c->H, c->r, codec_of(c), c->vmax, bits, c->Wp, c->plane_elems, nfr, c->planes, cal,
                    c->rays64, c->flags, c->flag_count, normals, offsets, curv);
            }
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SF_OK;
}

template <int DT>
sf_status launch_pass_for(sf_ctx* c, int nfr, const void* depth, float* normals, float* offsets, float* curv,
                          int32_t* counts, cudaStream_t st) {
    switch (c->method) {
        case SF_METHOD_DISPARITY:
            return c->constraint == SF_CONSTRAINT_UNIT4
                       ? launch_pass<DT, SF_METHOD_DISPARITY, true>(c, nfr, depth, normals, offsets, curv, counts, st)
                       : launch_pass<DT, SF_METHOD_DISPARITY>(c, nfr, depth, normals, offsets, curv, counts, st);
        case SF_METHOD_STANDARD:
            return c->constraint == SF_CONSTRAINT_UNIT4
                       ? launch_pass<DT, SF_METHOD_STANDARD, true>(c, nfr, depth, normals, offsets, curv, counts, st)
                       : launch_pass<DT, SF_METHOD_STANDARD>(c, nfr, depth, normals, offsets, curv, counts, st);
        case SF_METHOD_EXPLICIT_DISPARITY:
            return launch_pass<DT, SF_METHOD_EXPLICIT_DISPARITY>(c, nfr, depth, normals, offsets, curv, counts, st);
        default:
            return launch_pass<DT, SF_METHOD_EXPLICIT_STANDARD>(c, nfr, depth, normals, offsets, curv, counts, st);
    }
}

// Fixed-point bits of the quadtree's node sums: nodes of up to 64 x 64 pixels
// with offsets |j|, |i| <= 32 from the node's centre keep sum v^2 (disparity)
// and sum v^2 j^2 (standard: 2^12 * 2^10 * 2^40 = 2^62) inside int64.
int quad_bits(int method) { return sf::base_method(method) == SF_METHOD_STANDARD ? 20 : 24; }

template <int DT, int M>
sf_status launch_quadtree(sf_ctx* c, int nfr, int frame_base, const void* depth, const sf_quad_params* p,
                          sf_quad_node* nodes, int capacity, int32_t* n_nodes, size_t roots, cudaStream_t st) {
    constexpr int B = sf::base_method(M);
    const size_t fe = (size_t)c->W * c->H;
    const int raw_z = sf::fixed_quantum<DT, B>() ? 1 : 0;
    const int bits = quad_bits(M);
    SF_CUDA(cudaMemsetAsync(c->vmax, 0, sizeof(unsigned) * nfr, st));
    if (!raw_z) {
        const int blocks = range_blocks(c, fe, nfr);
        sf::range_kernel<DT, B><<<dim3(blocks, nfr), 256, 0, st>>>(depth, fe, codec_of(c), c->vmax);
    }
    SF_CUDA(cudaMemsetAsync(c->quad_cnt, 0, sizeof(int) * 8, st));
    sf::quad_roots_kernel<<<(int)std::min<size_t>((roots + 255) / 256, 1024), 256, 0, st>>>(c->W, c->H, p->tile, nfr,
                                                                                            c->quad_q[0], c->quad_cnt);
    size_t level_max = roots;
    for (int l = 0; l <= p->max_level; ++l) {
        const size_t n = std::min(level_max, c->quad_cap);
        const int blocks = (int)((n + 7) / 8);
        sf::quad_level_kernel<DT, M><<<blocks, 256, 0, st>>>(
            depth, c->W, c->H, codec_of(c), c->vmax, bits, c->rays64, c->quad_q[l & 1], c->quad_cnt + l, l,
            p->max_level, (double)p->tau, c->min_valid, p->min_valid_permille, c->quad_q[(l + 1) & 1],
            c->quad_cnt + l + 1, (int)c->quad_cap, nodes, n_nodes, capacity, frame_base);
        level_max *= 4;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "quadtree launch");
    return SF_OK;
}

template <int DT>
sf_status launch_quadtree_for(sf_ctx* c, int nfr, int frame_base, const void* depth, const sf_quad_params* p,
                              sf_quad_node* nodes, int capacity, int32_t* n_nodes, size_t roots, cudaStream_t st) {
    switch (c->method) {
        case SF_METHOD_DISPARITY:
            return launch_quadtree<DT, SF_METHOD_DISPARITY>(c, nfr, frame_base, depth, p, nodes, capacity, n_nodes,
                                                            roots, st);
        case SF_METHOD_STANDARD:
            return launch_quadtree<DT, SF_METHOD_STANDARD>(c, nfr, frame_base, depth, p, nodes, capacity, n_nodes,
                                                           roots, st);
        case SF_METHOD_EXPLICIT_DISPARITY:
            return launch_quadtree<DT, SF_METHOD_EXPLICIT_DISPARITY>(c, nfr, frame_base, depth, p, nodes, capacity,
                                                                     n_nodes, roots, st);
        default:
            return launch_quadtree<DT, SF_METHOD_EXPLICIT_STANDARD>(c, nfr, frame_base, depth, p, nodes, capacity,
                                                                    n_nodes, roots, st);
    }
}

// The disparity-form pass with a per-pixel table of ray adjustments
// (sf_set_delta_table): range as usual, then the table's row and column passes.
template <int DT, bool U4>
sf_status launch_pass_delta(sf_ctx* c, int nfr, const void* depth, float* normals, float* offsets, float* curv,
                            int32_t* counts, cudaStream_t st) {
    constexpr int M = SF_METHOD_DISPARITY;
    const size_t fe = (size_t)c->W * c->H;
    const int raw_z = sf::fixed_quantum<DT, M>() ? 1 : 0;
    const int bits = quant_bits(M, c->k);
    SF_CUDA(cudaMemsetAsync(c->vmax, 0, sizeof(unsigned) * nfr, st));
    if (!raw_z) {
        StageTimer t(c, 0, st);
        const int blocks = range_blocks(c, fe, nfr);
        sf::range_kernel<DT, M><<<dim3(blocks, nfr), 256, 0, st>>>(depth, fe, codec_of(c), c->vmax);
    }
    {
        StageTimer t(c, 1, st);
        dim3 grid((c->W + 31) / 32, (c->H + sf::kHThreads - 1) / sf::kHThreads, nfr);
        const size_t smem = 3 * sizeof(int) * sf::kHThreads * (size_t)((32 + 2 * c->r) | 1);
        sf::hpass_delta_kernel<DT><<<grid, sf::kHThreads, smem, st>>>(depth, c->dtab, c->W, c->H, c->r, codec_of(c),
                                                                     c->vmax, bits, c->plane_elems, c->planes);
    }
    // precision modes: the column pass queues the windows it cannot vouch for
    // (mode 1) or every window (mode 2), and the direct kernel solves them again
    // in FP64 from the unrounded depth
    const bool fb = c->precision_mode > 0 && c->flags;
    if (fb) SF_CUDA(cudaMemsetAsync(c->flag_count, 0, 3 * sizeof(unsigned), st));
    {
        StageTimer t(c, 2, st);
        const int band = vertical_band(c, nfr);
        dim3 grid((c->W + sf::kVThreads - 1) / sf::kVThreads, (c->H + band - 1) / band, nfr);
        const float tau = c->precision_mode == 2 ? INFINITY : c->tau;
        sf::vpass_delta_kernel<DT, U4><<<grid, sf::kVThreads, 0, st>>>(
            depth, c->W, c->H, c->r, codec_of(c), c->vmax, bits, c->plane_elems, c->planes, calib_of(c),
            c->min_valid, c->require_center, band, normals, offsets, curv, counts, tau, fb ? c->flags : nullptr,
            c->flag_count);
    }
    if (fb) {
        StageTimer t(c, 3, st);
        static const int nb = resident_blocks(c, sf::direct_delta_kernel<DT, U4>, 128);
        sf::direct_delta_kernel<DT, U4><<<nb, 128, 0, st>>>(depth, c->dtab, c->W, c->H, c->r, codec_of(c),
                                                             c->rays64, c->flags, c->flag_count, normals, offsets,
                                                             curv);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return SF_OK;
}

// reuse: the scratch planes and quanta already hold the row pass of these
// frames (the forward fit's), so only the adjoint and the gather run.
template <int DT, int M>
sf_status launch_backward(sf_ctx* c, int nfr, const void* depth, const float* gn, const float* gd, const float* gk,
                          float* g_depth, bool reuse, cudaStream_t st) {
    const size_t fe = (size_t)c->W * c->H;
    const int raw_z = sf::fixed_quantum<DT, M>() ? 1 : 0;
    const int bits = quant_bits(M, c->k);
    if (!reuse) SF_CUDA(cudaMemsetAsync(c->vmax, 0, sizeof(unsigned) * nfr, st));
    if (!reuse && !raw_z) {
        const int blocks = range_blocks(c, fe, nfr);
        sf::range_kernel<DT, M><<<dim3(blocks, nfr), 256, 0, st>>>(depth, fe, codec_of(c), c->vmax);
    }
    if (!reuse) {
        const int seg = horizontal_seg(c, nfr);
        dim3 grid((c->W + seg - 1) / seg, (c->H + sf::kHThreads - 1) / sf::kHThreads, nfr);
        const int IW = seg + 2 * c->r;
        const size_t smem = sizeof(int) * sf::kHThreads * (size_t)(IW | 1);
        launch_hpass<DT, M>(grid, smem, st, depth, c, bits, raw_z, seg);
    }
    const sf::Calib cal = calib_of(c);
    {
        const int band = vertical_band(c, nfr);
        dim3 grid((c->W + sf::kVThreads - 1) / sf::kVThreads, (c->H + band - 1) / band, nfr);
        SF_CUDA(cudaMemsetAsync(c->adj_max, 0, sizeof(float) * 3 * nfr, st));
        sf::vadjoint_kernel<DT, M><<<grid, sf::kVThreads, 0, st>>>(depth, c->W, c->H, c->r, codec_of(c), c->vmax,
                                                                  bits, c->Wp, c->plane_elems, c->planes, cal,
                                                                  c->min_valid, c->require_center, band, gn, gd, gk,
                                                                  c->adj, c->adj_max);
    }
    {
        const size_t smem = sf::gather_smem_bytes(sf::gather_channels_box<M>(), c->r);
        dim3 grid((c->W + sf::kGTile - 1) / sf::kGTile, (c->H + sf::kGTile - 1) / sf::kGTile, nfr);
        sf::gather_kernel<DT, M><<<grid, dim3(32, 8), smem, st>>>(depth, c->W, c->H, c->r, codec_of(c), cal, c->adj,
                                                                   c->adj_max, g_depth);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "backward kernel launch");
    return SF_OK;
}

template <int DT, int M>
sf_status batch_enqueue_t(sf_batch* b, cudaStream_t st) {
    // claim counter and error word, then the per-frame quantum bits and counters
    // (the poll limit in between is kept)
    SF_CUDA(cudaMemsetAsync(b->d_sync, 0, 2 * sizeof(unsigned), st));
    SF_CUDA(cudaMemsetAsync(b->d_sync + 3, 0, 3 * sizeof(unsigned) * b->n, st));
    const sf::Codec cd{b->depth_scale, 0, 0};
    sf::batch_kernel<DT, M><<<b->grid, sf::kVThreads, b->hsmem, st>>>(
        b->d_desc, b->d_items, b->n_r, b->n_h, b->n_v, sf::BatchSync{b->d_sync, b->n}, b->d_planes, b->stride, cd,
        b->min_valid, b->require_center);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
    return SF_OK;
}

template <int DT, int M>
void batch_grids_t(sf_batch* b, int sms) {
    int nb = 0;
    cudaFuncSetAttribute(sf::batch_kernel<DT, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->hsmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sf::batch_kernel<DT, M>, sf::kVThreads, b->hsmem);
    b->grid = std::max(1, nb) * sms;
}

// Opt the kernels that take large dynamic shared memory in to their maximum.
template <int DT>
void set_kernel_smem_t() {
    const int IW = 128 + 2 * sf::kMaxR;
    const int smem = (int)(sizeof(int) * sf::kHThreads * (size_t)(IW | 1));
    set_hpass_smem_one<DT, SF_METHOD_DISPARITY>(smem);
    set_hpass_smem_one<DT, SF_METHOD_STANDARD>(smem);
    const int dsmem = (int)(3 * sizeof(int) * sf::kHThreads * (size_t)((32 + 2 * sf::kMaxR) | 1));
    cudaFuncSetAttribute(sf::hpass_delta_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem);
    if constexpr (DT != SF_DEPTH_DISPARITY_U16) {
        cudaFuncSetAttribute(sf::gather_kernel<DT, SF_METHOD_DISPARITY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sf::gather_smem_bytes(4, sf::kMaxR));
        cudaFuncSetAttribute(sf::gather_kernel<DT, SF_METHOD_STANDARD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sf::gather_smem_bytes(9, sf::kMaxR));
    }
}

}  // namespace
}  // namespace sfh

// Defines the extern launchers of sf_host.h for one depth encoding.
#define SF_DEFINE_LAUNCHERS(dt, DT)                                                                                    \
    namespace sfh {                                                                                                    \
    sf_status fit_pass_##dt(sf_ctx* c, int nfr, const void* depth, float* normals, float* offsets, float* curv,      \
                            int32_t* counts, cudaStream_t st) {                                                        \
        return launch_pass_for<DT>(c, nfr, depth, normals, offsets, curv, counts, st);                                \
    }                                                                                                                  \
    sf_status delta_pass_##dt(sf_ctx* c, int nfr, const void* depth, float* normals, float* offsets, float* curv,    \
                              int32_t* counts, cudaStream_t st) {                                                      \
        return c->constraint == SF_CONSTRAINT_UNIT4                                                                    \
                   ? launch_pass_delta<DT, true>(c, nfr, depth, normals, offsets, curv, counts, st)                    \
                   : launch_pass_delta<DT, false>(c, nfr, depth, normals, offsets, curv, counts, st);                  \
    }                                                                                                                  \
    sf_status backward_##dt(sf_ctx* c, int nfr, const void* depth, const float* gn, const float* gd, const float* gk, \
                            float* g_depth, bool reuse, cudaStream_t st) {                                             \
        if constexpr (DT == SF_DEPTH_DISPARITY_U16) {                                                                  \
            return fail(SF_ERR_UNSUPPORTED, "the backward takes depth input (f32 or u16)");                           \
        } else {                                                                                                       \
            return c->method == SF_METHOD_DISPARITY                                                                    \
                       ? launch_backward<DT, SF_METHOD_DISPARITY>(c, nfr, depth, gn, gd, gk, g_depth, reuse, st)       \
                       : launch_backward<DT, SF_METHOD_STANDARD>(c, nfr, depth, gn, gd, gk, g_depth, reuse, st);       \
        }                                                                                                              \
    }                                                                                                                  \
    sf_status quadtree_##dt(sf_ctx* c, int nfr, int frame_base, const void* depth, const sf_quad_params* p,         \
                            sf_quad_node* nodes, int capacity, int32_t* n_nodes, size_t roots, cudaStream_t st) {     \
        return launch_quadtree_for<DT>(c, nfr, frame_base, depth, p, nodes, capacity, n_nodes, roots, st);            \
    }                                                                                                                  \
    sf_status batch_enqueue_##dt(sf_batch* b, cudaStream_t st) {                                                      \
        if constexpr (DT == SF_DEPTH_DISPARITY_U16) {                                                                  \
            return fail(SF_ERR_UNSUPPORTED, "batches take depth input (f32 or u16)");                                 \
        } else {                                                                                                       \
            return b->method == SF_METHOD_DISPARITY ? batch_enqueue_t<DT, SF_METHOD_DISPARITY>(b, st)                 \
                                                    : batch_enqueue_t<DT, SF_METHOD_STANDARD>(b, st);                 \
        }                                                                                                              \
    }                                                                                                                  \
    void batch_grids_##dt(sf_batch* b, int sms) {                                                                     \
        if constexpr (DT != SF_DEPTH_DISPARITY_U16) {                                                                  \
            if (b->method == SF_METHOD_DISPARITY) batch_grids_t<DT, SF_METHOD_DISPARITY>(b, sms);                      \
            else batch_grids_t<DT, SF_METHOD_STANDARD>(b, sms);                                                        \
        }                                                                                                              \
    }                                                                                                                  \
    void set_kernel_smem_##dt() { set_kernel_smem_t<DT>(); }                                                          \
    unsigned long long bounds_word_##dt() {                                                                            \
        unsigned long long v = 0;                                                                                      \
        if (cudaMemcpyFromSymbol(&v, sf::sf_bounds_word, sizeof(v)) != cudaSuccess) return 0;                          \
        if (v) {                                                                                                       \
            const unsigned long long z = 0;                                                                            \
            cudaMemcpyToSymbol(sf::sf_bounds_word, &z, sizeof(z));                                                     \
        }                                                                                                              \
        return v;                                                                                                      \
    }                                                                                                                  \
    }
