// surffit.cu -- C ABI of the dense RGBD plane-fitting library (host side:
// contexts, argument checks, batches, staging, the allocation-free entry
// point).  Kernel launches live in fit_f32.cu, fit_u16.cu and fit_disp.cu, one
// per depth encoding (sf_launch.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "surffit.h"
#include "sf_host.h"
#include "sf_kernels.cuh"
#include "sf_delta.cuh"

using sfh::cuda_fail;
using sfh::fail;

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace sfh {

sf_status fail(sf_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

sf_status cuda_fail(cudaError_t e, const char* what) {
    // running out of device memory is an allocation failure, whichever call met it
    return fail(e == cudaErrorMemoryAllocation ? SF_ERR_ALLOC : SF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t plane_bytes_per_frame(int method, size_t plane_elems) {
    // disparity: 3 x int32 + 1 x int64 ; standard: 1 x int32 + 5 x int64
    return plane_elems * (sf::base_method(method) == SF_METHOD_STANDARD ? (4 + 5 * 8) : (3 * 4 + 8));
}

// Fixed-point bits for a method and window: the most that keeps every exact
// window sum and every re-centring product below 2^63.
//   disparity: 2 * m * sum w <= 2 k^2 2^(2b)                 -> b < 31 - log2 k
//   standard:  sum z^2 j^2   <= k * sum_{|j|<=r} j^2 * 2^(2b) and 2 k^2 2^(2b)
int quant_bits(int method, int k) {
    const int r = (k - 1) / 2;
    double weight = 2.0 * k * k;
    if (method == SF_METHOD_STANDARD || method == SF_METHOD_EXPLICIT_STANDARD) {
        const double wjj = (double)k * (double)r * (r + 1) * (2 * r + 1) / 3.0;
        weight = std::max(weight, wjj);
    }
    int b = (int)std::floor((63.0 - std::log2(weight)) / 2.0 - 1e-9);
    if (sf::base_method(method) == SF_METHOD_DISPARITY) {
        // the row sums of v are stored as int32: k 2^b < 2^31; those of v j
        // as 32 + 5 bits: r (r + 1) 2^b < 2^36
        b = std::min(b, (int)std::floor(31.0 - std::log2((double)k) - 1e-9));
        b = std::min(b, (int)std::floor(36.0 - std::log2((double)std::max(1, r * (r + 1))) - 1e-9));
    }
    return std::min(28, std::max(16, b));
}

}  // namespace sfh

namespace {

size_t depth_bytes(int depth_type) { return depth_type == SF_DEPTH_F32 ? 4 : 2; }

// Kernel attributes (large dynamic shared memory) of every launcher.
void set_kernel_attributes() {
    sfh::set_kernel_smem_f32();
    sfh::set_kernel_smem_u16();
    sfh::set_kernel_smem_disp();
}

sf_status fit_pass(sf_ctx* c, int nfr, const void* depth, float* normals, float* offsets, float* curv,
                   int32_t* counts, cudaStream_t st) {
    if (c->dtab) {
        switch (c->depth_type) {
            case SF_DEPTH_F32: return sfh::delta_pass_f32(c, nfr, depth, normals, offsets, curv, counts, st);
            case SF_DEPTH_U16: return sfh::delta_pass_u16(c, nfr, depth, normals, offsets, curv, counts, st);
            default: return sfh::delta_pass_disp(c, nfr, depth, normals, offsets, curv, counts, st);
        }
    }
    switch (c->depth_type) {
        case SF_DEPTH_F32: return sfh::fit_pass_f32(c, nfr, depth, normals, offsets, curv, counts, st);
        case SF_DEPTH_U16: return sfh::fit_pass_u16(c, nfr, depth, normals, offsets, curv, counts, st);
        default: return sfh::fit_pass_disp(c, nfr, depth, normals, offsets, curv, counts, st);
    }
}

}  // namespace

namespace sfh {
// Output columns per thread of the horizontal pass: 32, unless the call has
// too few rows x segments to fill the GPU (a single small frame), where
// narrower segments give more threads and shorter serial chains (each thread
// slides seg + 2r columns).
int horizontal_seg(const sf_ctx* c, int nfr) {
    if (c->hseg > 0) return c->hseg;
    int seg = sf::kHSeg;
    while (seg > 8 && (size_t)((c->W + seg - 1) / seg) * c->H * nfr < (size_t)152 * 256) seg /= 2;
    return seg;
}
// Band height of the vertical pass: long bands amortise the 2r-row warm-up,
// short bands give enough threads to fill the GPU.
int vertical_band(const sf_ctx* c, int nfr) {
    if (c->vband > 0) return c->vband;
    const size_t cols = (size_t)((c->W + sf::kVThreads - 1) / sf::kVThreads) * sf::kVThreads * nfr;
    // at least 152 x 2048 threads (about 2.7 waves of 24 resident warps per
    // SM): short bands cost a 2r-row warm-up each, but with fewer waves the
    // tail of the last one costs more.  Small frames with small windows go
    // down to 4-row bands: there the serial chain of solves per thread, not
    // the warm-up, bounds the pass (one 640 x 480 frame at k = 7: 12.8 us at
    // 4 rows, 16.9 at 16); larger windows keep bands of at least r + 1 rows
    const int min_band = std::max(4, std::min(16, c->r + 1));
    int band = 256;
    while (band / 2 >= min_band && cols * (size_t)((c->H + band - 1) / band) < (size_t)152 * 64 * 32) band /= 2;
    return band;
}
}  // namespace sfh

// Every device allocation of the library goes through dev_alloc.  A test can
// make the allocations after the next n fail (sf_debug_fail_allocs) and so run
// each SF_ERR_ALLOC path, and its clean-up, without exhausting the device.
static std::atomic<long long> g_alloc_budget{-1};  // allocations left before failing; < 0: no limit
static std::atomic<long long> g_live_allocs{0};    // device allocations of the library not yet freed

template <class T>
static cudaError_t dev_alloc(T** p, size_t bytes) {
    long long b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
    }
    const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();  // not sticky: clear it so that no later launch check reports it
    } else {
        ++g_live_allocs;
    }
    return e;
}

static void dev_free(void* p) {
    if (!p) return;
    cudaFree(p);
    --g_live_allocs;
}

static sf_status ensure_planes(sf_ctx* c, int frames) {
    const size_t delta_bytes = (sf::kDeltaPlanes32 * 4 + sf::kDeltaPlanes64 * 8) * c->plane_elems;
    const size_t need = std::max(sfh::plane_bytes_per_frame(SF_METHOD_STANDARD, c->plane_elems),
                                 c->dtab ? delta_bytes : (size_t)0) * (size_t)frames;
    if (c->planes && c->planes_bytes >= need && c->planes_frames >= frames) return SF_OK;
    if (c->planes) dev_free(c->planes);
    c->planes = nullptr;
    c->planes_bytes = 0;
    c->planes_frames = 0;
    cudaError_t e = dev_alloc(&c->planes, need);
    if (e != cudaSuccess) return fail(SF_ERR_ALLOC, "scratch allocation of %zu bytes failed: %s", need,
                                      cudaGetErrorString(e));
    c->planes_bytes = need;
    c->planes_frames = frames;
    ++c->gen;
    return SF_OK;
}

// Polls per wait of the merged batch kernel (about a second at its sleep between polls).
static constexpr unsigned kBatchWaitPolls = 1u << 22;

static bool misaligned(const void* p, size_t a) { return ((uintptr_t)p & (a - 1)) != 0; }

extern "C" {

const char* sf_last_error(void) { return g_last_error.c_str(); }

namespace {
__global__ void acos_eval_kernel(const float* __restrict__ x, float* __restrict__ y, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = sf::acos_fast(x[i]);
}
}  // namespace

sf_status sf_eval_acos(const float* x, float* y, int n, void* stream) {
    if (n < 0) return fail(SF_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return SF_OK;
    if (!x || !y) return fail(SF_ERR_INVALID_ARG, "null buffer");
    if (misaligned(x, 4) || misaligned(y, 4)) return fail(SF_ERR_INVALID_ARG, "buffers must be 4-byte aligned");
    acos_eval_kernel<<<(n + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(x, y, n);
    SF_CUDA(cudaGetLastError());
    return SF_OK;
}

sf_status sf_debug_fail_allocs(long long after) {
    g_alloc_budget.store(after < 0 ? -1 : after);
    return SF_OK;
}

sf_status sf_backward_reuses(const sf_ctx* c, long long* n) {
    if (!c || !n) return fail(SF_ERR_INVALID_ARG, "null context or output");
    *n = c->backward_reuses;
    return SF_OK;
}

sf_status sf_graph_replays(const sf_ctx* c, long long* n) {
    if (!c || !n) return fail(SF_ERR_INVALID_ARG, "null context or output");
    *n = c->graph_replays;
    return SF_OK;
}

sf_status sf_debug_live_allocs(long long* n) {
    if (!n) return fail(SF_ERR_INVALID_ARG, "null output");
    *n = g_live_allocs.load();
    return SF_OK;
}

const char* sf_version(void) { return "surffit-gb300 0.1 (sm_103a)"; }

sf_status sf_channel_counts(int method, int* depth_channels, int* mask_channels) {
    if (!depth_channels || !mask_channels) return fail(SF_ERR_INVALID_ARG, "null output pointer");
    switch (method) {
        case SF_METHOD_DISPARITY:  // sum w, sum w j, sum w i, sum w^2 ; mask n, j, i, j^2, ji, i^2
            *depth_channels = 4; *mask_channels = 6; return SF_OK;
        case SF_METHOD_STANDARD:   // z, zj, zi, z^2, z^2 j, z^2 i, z^2 j^2, z^2 ji, z^2 i^2 ; mask n
            *depth_channels = 9; *mask_channels = 1; return SF_OK;
        case SF_METHOD_EXPLICIT_DISPARITY:  // w, w j, w i ; mask n, j, i, j^2, ji, i^2
            *depth_channels = 3; *mask_channels = 6; return SF_OK;
        case SF_METHOD_EXPLICIT_STANDARD:   // X^2, XY, X, Y^2, Y, ZX, ZY, Z in window-relative form
            *depth_channels = 8; *mask_channels = 1; return SF_OK;
        default:
            return fail(SF_ERR_INVALID_ARG, "unknown method %d", method);
    }
}

sf_status sf_create(const sf_intrinsics* K, int W, int H, int window, sf_ctx** out) {
    if (!K || !out) return fail(SF_ERR_INVALID_ARG, "null intrinsics or output pointer");
    *out = nullptr;
    if (W < 1 || H < 1) return fail(SF_ERR_INVALID_ARG, "image size %dx%d must be positive", W, H);
    if ((size_t)W * (size_t)H > ((size_t)1 << 31)) return fail(SF_ERR_INVALID_ARG, "image too large");
    if (window < 1 || (window & 1) == 0 || window > SF_MAX_WINDOW)
        return fail(SF_ERR_INVALID_ARG, "window %d must be odd and in [1, %d]", window, SF_MAX_WINDOW);
    if (!(K->fx != 0.0) || !(K->fy != 0.0) || !std::isfinite(K->fx) || !std::isfinite(K->fy) ||
        !std::isfinite(K->cx) || !std::isfinite(K->cy) || !std::isfinite(K->dx) || !std::isfinite(K->dy))
        return fail(SF_ERR_INVALID_ARG, "intrinsics must be finite with nonzero focal lengths");
    sf_ctx* c = new (std::nothrow) sf_ctx();
    if (!c) return fail(SF_ERR_ALLOC, "context allocation failed");
    c->K = *K;
    c->W = W; c->H = H; c->k = window; c->r = (window - 1) / 2;
    c->Wp = (W + 63) / 64 * 64;
    c->plane_elems = (size_t)c->Wp * H;
    cudaGetDevice(&c->device);
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || c->sms < 1)
        c->sms = 152;
    // Calibration tables (Eq. 10), computed in FP64 on the host, stored as FP32.
    float* htx = (float*)malloc(sizeof(float) * W);
    float* hty = (float*)malloc(sizeof(float) * H);
    if (!htx || !hty) { free(htx); free(hty); delete c; return fail(SF_ERR_ALLOC, "host table allocation failed"); }
    for (int x = 0; x < W; ++x) htx[x] = (float)((x + K->dx - K->cx) / K->fx);
    for (int y = 0; y < H; ++y) hty[y] = (float)((y + K->dy - K->cy) / K->fy);
    cudaError_t e = dev_alloc(&c->tx, sizeof(float) * W);
    if (e == cudaSuccess) e = dev_alloc(&c->ty, sizeof(float) * H);
    if (e == cudaSuccess) e = cudaMemcpy(c->tx, htx, sizeof(float) * W, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->ty, hty, sizeof(float) * H, cudaMemcpyHostToDevice);
    free(htx); free(hty);
    if (e != cudaSuccess) { sf_destroy(c); return cuda_fail(e, "sf_create tables"); }
    // Frames per pass: every frame of a call in one launch (up to 64), so the
    // grid fills the GPU; the scratch moments are sized for them on demand.
    c->max_frames_per_pass = 64;
    e = dev_alloc(&c->vmax, sizeof(unsigned) * 64);
    if (e != cudaSuccess) { sf_destroy(c); return cuda_fail(e, "sf_create vmax"); }
    e = dev_alloc(&c->flag_count, 3 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->flag_count, 0, 3 * sizeof(unsigned));
    if (e != cudaSuccess) { sf_destroy(c); return cuda_fail(e, "sf_create flag counter"); }
    {
        // FP64 ray tables for the precision fallback
        double* h = (double*)malloc(sizeof(double) * (W + H + 2));
        if (!h) { sf_destroy(c); return fail(SF_ERR_ALLOC, "host table allocation failed"); }
        for (int x = 0; x < W; ++x) h[x] = (x + K->dx - K->cx) / K->fx;
        for (int y = 0; y < H; ++y) h[W + y] = (y + K->dy - K->cy) / K->fy;
        h[W + H] = 1.0 / K->fx;
        h[W + H + 1] = 1.0 / K->fy;
        e = dev_alloc(&c->rays64, sizeof(double) * (W + H + 2));
        if (e == cudaSuccess) e = cudaMemcpy(c->rays64, h, sizeof(double) * (W + H + 2), cudaMemcpyHostToDevice);
        free(h);
        if (e != cudaSuccess) { sf_destroy(c); return cuda_fail(e, "sf_create FP64 rays"); }
    }
    sf_status s = ensure_planes(c, 1);
    if (s != SF_OK) { sf_destroy(c); return s; }
    {
        set_kernel_attributes();
        e = cudaGetLastError();
        if (e != cudaSuccess) { sf_destroy(c); return cuda_fail(e, "sf_create kernel attributes"); }
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { sf_destroy(c); return cuda_fail(e, "sf_create synchronise"); }
    *out = c;
    return SF_OK;
}

sf_status sf_set_params(sf_ctx* c, int method, int depth_type, float depth_scale, int min_valid,
                        int require_center_valid) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    ++c->gen;  // a captured fit graph no longer applies
    if (method < SF_METHOD_DISPARITY || method > SF_METHOD_EXPLICIT_STANDARD)
        return fail(SF_ERR_INVALID_ARG, "unknown method %d", method);
    if (depth_type != SF_DEPTH_F32 && depth_type != SF_DEPTH_U16 && depth_type != SF_DEPTH_DISPARITY_U16)
        return fail(SF_ERR_INVALID_ARG, "unknown depth type %d", depth_type);
    if (depth_type == SF_DEPTH_U16 && !(depth_scale > 0.f && std::isfinite(depth_scale)))
        return fail(SF_ERR_INVALID_ARG, "depth_scale must be positive and finite");
    if (min_valid < 1) return fail(SF_ERR_INVALID_ARG, "min_valid must be >= 1");
    c->method = method;
    c->depth_type = depth_type;
    c->depth_scale = depth_scale;
    c->min_valid = min_valid;
    c->require_center = require_center_valid ? 1 : 0;
    return SF_OK;
}

}  // extern "C"

// Capture one single-pass fit into the context's graph (updated in place when
// one exists and has the same shape).  On failure the direct path runs.
static sf_status capture_fit(sf_ctx* c, const sf_ctx::FitKey& key, int n, const void* depth, float* normals,
                             float* offsets, float* curvature, int32_t* counts) {
    if (!c->graph_stream) SF_CUDA(cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking));
    SF_CUDA(cudaStreamBeginCapture(c->graph_stream, cudaStreamCaptureModeThreadLocal));
    const sf_status s = fit_pass(c, n, depth, normals, offsets, curvature, counts, c->graph_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->graph_stream, &g);
    if (s != SF_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return s != SF_OK ? s : cuda_fail(e == cudaSuccess ? cudaErrorUnknown : e, "fit graph capture");
    }
    if (c->graph_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(c->graph_exec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
        }
    }
    if (!c->graph_exec) e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph_exec = nullptr;
        return cuda_fail(e, "fit graph instantiate");
    }
    c->graph_key = key;
    return SF_OK;
}

extern "C" {

static sf_status fit_ex_impl(sf_ctx* c, int n_frames, const void* depth, float* normals, float* offsets, float* curvature,
                    int32_t* counts, void* stream) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    if (n_frames < 0) return fail(SF_ERR_INVALID_ARG, "n_frames must be >= 0");
    if (n_frames == 0) return SF_OK;
    if (!depth || !normals || !offsets || !curvature) return fail(SF_ERR_INVALID_ARG, "null buffer");
    if (misaligned(depth, depth_bytes(c->depth_type)) || misaligned(normals, 4) || misaligned(offsets, 4) ||
        misaligned(curvature, 4) || misaligned(counts, 4))
        return fail(SF_ERR_INVALID_ARG, "buffers must be aligned to their element size");
    if (c->constraint == SF_CONSTRAINT_UNIT4 && c->method != SF_METHOD_DISPARITY && c->method != SF_METHOD_STANDARD)
        return fail(SF_ERR_UNSUPPORTED, "the |(a,b,c,d)| = 1 constraint applies to the implicit fits");
    if (c->dtab && c->method != SF_METHOD_DISPARITY)
        return fail(SF_ERR_UNSUPPORTED, "a per-pixel delta table applies to the disparity-form fit");
    if (c->depth_type == SF_DEPTH_DISPARITY_U16 && sf::base_method(c->method) == SF_METHOD_DISPARITY) {
        // the disparity integers go into the int32 row sums unscaled: k w < 2^31
        const double wmax = 128.0 * 65535.0 + std::fabs((double)c->disp_add) + 1.0;
        if (wmax * c->k >= 2147483648.0)
            return fail(SF_ERR_INVALID_ARG, "disparity model offset too large for a %d x %d window", c->k, c->k);
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t fe = (size_t)c->W * c->H;
    const size_t dbytes = depth_bytes(c->depth_type);
    int per = std::min(c->max_frames_per_pass, 64);
    sf_status s = ensure_planes(c, std::min(per, n_frames));
    if (s != SF_OK) return s;
    if (c->precision_mode > 0) {
        // every pixel may be queued, plus one partly used chunk of slots per warp of the column pass
        const int nfr1 = std::min(per, n_frames);
        const size_t vwarps = (size_t)((c->W + sf::kVThreads - 1) / sf::kVThreads) * (sf::kVThreads / 32) *
                              (size_t)((c->H + sfh::vertical_band(c, nfr1) - 1) / sfh::vertical_band(c, nfr1)) *
                              (size_t)nfr1;
        const size_t cap = fe * (size_t)nfr1 + sf::kQueueChunk * vwarps;
        if (c->flags_cap < cap) {
            if (c->flags) dev_free(c->flags);
            c->flags = nullptr;
            c->flags_cap = 0;
            if (c->queue_c) dev_free(c->queue_c);
            c->queue_c = nullptr;
            cudaError_t e = dev_alloc(&c->flags, cap * sizeof(unsigned long long));
            if (e == cudaSuccess) e = dev_alloc(&c->queue_c, cap * sizeof(unsigned));
            if (e != cudaSuccess) return fail(SF_ERR_ALLOC, "precision-fallback queue of %zu entries failed", cap);
            c->flags_cap = cap;
            ++c->gen;
        }
        // the exact moments of queued windows: every window in mode 2, a quarter of
        // them in mode 1 (windows queued beyond that re-read their moments from
        // the scratch planes)
        // (the delta-table path solves from the depth and keeps no moments)
        const size_t mcap = c->dtab ? 0 : c->precision_mode == 2 ? cap : (cap + 3) / 4;
        if (c->moments_cap < mcap) {
            if (c->moments_q) dev_free(c->moments_q);
            c->moments_q = nullptr;
            c->moments_cap = 0;
            cudaError_t e = dev_alloc(&c->moments_q, mcap * sfh::kMomentEntryBytes);
            if (e != cudaSuccess)
                return fail(SF_ERR_ALLOC, "precision-fallback moments of %zu entries failed", mcap);
            c->moments_cap = mcap;
            ++c->gen;
        }
    }
    if (n_frames <= per && !c->profiling) {
        const sf_ctx::FitKey key{c->gen, n_frames, depth, normals, offsets, curvature, counts};
        if (c->graph_exec && key == c->graph_key) {
            SF_CUDA(cudaGraphLaunch(c->graph_exec, st));
            ++c->graph_replays;
            return SF_OK;
        }
        const bool again = key == c->last_key;
        c->last_key = key;
        if (again && capture_fit(c, key, n_frames, depth, normals, offsets, curvature, counts) == SF_OK) {
            SF_CUDA(cudaGraphLaunch(c->graph_exec, st));
            ++c->graph_replays;
            return SF_OK;
        }
    }
    for (int f0 = 0; f0 < n_frames; f0 += per) {
        const int nfr = std::min(per, n_frames - f0);
        const void* dp = static_cast<const char*>(depth) + dbytes * fe * f0;
        float* np_ = normals + 3 * fe * f0;
        float* op = offsets + fe * f0;
        float* cp = curvature + fe * f0;
        int32_t* kp = counts ? counts + fe * f0 : nullptr;
        s = fit_pass(c, nfr, dp, np_, op, cp, kp, st);
        if (s != SF_OK) return s;
    }
    return SF_OK;
}

sf_status sf_fit(sf_ctx* c, const void* depth, float* normals, float* offsets, float* curvature, void* stream) {
    return sf_fit_ex(c, 1, depth, normals, offsets, curvature, nullptr, stream);
}

static sf_status fit_host_impl(sf_ctx* c, int n_frames, const void* depth, float* normals, float* offsets, float* curvature,
                      int32_t* counts, void* stream) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    if (n_frames < 0) return fail(SF_ERR_INVALID_ARG, "n_frames must be >= 0");
    if (n_frames == 0) return SF_OK;
    if (!depth || !normals || !offsets || !curvature) return fail(SF_ERR_INVALID_ARG, "null buffer");
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    const size_t fe = (size_t)c->W * c->H;
    const size_t dpx = depth_bytes(c->depth_type);
    // Frames go through in chunks on two streams: the copy-out of chunk i-1
    // overlaps the copy-in and fit of chunk i.  Copies read and write the
    // caller's (pageable) buffers directly; the fits share the context's
    // scratch, so each waits for the previous one.
    const int nchunks = std::min(n_frames, 4);
    const int per = (n_frames + nchunks - 1) / nchunks;
    const size_t dbytes = dpx * fe * per;
    const size_t need = dbytes + (20 + (counts ? 4 : 0)) * fe * per;
    if (!c->io_stream[0]) {
        for (int i = 0; i < 2; ++i) {
            SF_CUDA(cudaStreamCreateWithFlags(&c->io_stream[i], cudaStreamNonBlocking));
            SF_CUDA(cudaEventCreateWithFlags(&c->io_fit_done[i], cudaEventDisableTiming));
        }
        SF_CUDA(cudaEventCreateWithFlags(&c->io_entry, cudaEventDisableTiming));
    }
    if (c->d_io_bytes < need) {
        for (int i = 0; i < 2; ++i) {
            if (c->d_io[i]) dev_free(c->d_io[i]);
            c->d_io[i] = nullptr;
        }
        c->d_io_bytes = 0;
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = dev_alloc(&c->d_io[i], need);
            if (e != cudaSuccess) return fail(SF_ERR_ALLOC, "device staging of 2 x %zu bytes failed", need);
        }
        c->d_io_bytes = need;
    }
    // work already queued on the caller's stream (e.g. a fit using the same
    // scratch) comes first
    SF_CUDA(cudaEventRecord(c->io_entry, user));
    for (int i = 0; i < 2; ++i) SF_CUDA(cudaStreamWaitEvent(c->io_stream[i], c->io_entry, 0));
    auto copy_out = [&](int ci) -> sf_status {
        const int f0 = ci * per, nf = std::min(per, n_frames - f0);
        cudaStream_t st = c->io_stream[ci & 1];
        const char* ds = static_cast<const char*>(c->d_io[ci & 1]);
        const float* dn = reinterpret_cast<const float*>(ds + dbytes);
        const float* dof = dn + 3 * fe * per;
        const float* dc = dof + fe * per;
        const int32_t* dk = reinterpret_cast<const int32_t*>(dc + fe * per);
        SF_CUDA(cudaMemcpyAsync(normals + 3 * fe * f0, dn, 12 * fe * nf, cudaMemcpyDeviceToHost, st));
        SF_CUDA(cudaMemcpyAsync(offsets + fe * f0, dof, 4 * fe * nf, cudaMemcpyDeviceToHost, st));
        SF_CUDA(cudaMemcpyAsync(curvature + fe * f0, dc, 4 * fe * nf, cudaMemcpyDeviceToHost, st));
        if (counts) SF_CUDA(cudaMemcpyAsync(counts + fe * f0, dk, 4 * fe * nf, cudaMemcpyDeviceToHost, st));
        return SF_OK;
    };
    for (int ci = 0; ci < nchunks; ++ci) {
        const int f0 = ci * per, nf = std::min(per, n_frames - f0);
        if (nf <= 0) break;
        cudaStream_t st = c->io_stream[ci & 1];
        char* ds = static_cast<char*>(c->d_io[ci & 1]);
        SF_CUDA(cudaMemcpyAsync(ds, static_cast<const char*>(depth) + dpx * fe * f0, dpx * fe * nf,
                                cudaMemcpyHostToDevice, st));
        if (ci > 0) SF_CUDA(cudaStreamWaitEvent(st, c->io_fit_done[(ci - 1) & 1], 0));
        float* dn = reinterpret_cast<float*>(ds + dbytes);
        float* dof = dn + 3 * fe * per;
        float* dc = dof + fe * per;
        int32_t* dk = counts ? reinterpret_cast<int32_t*>(dc + fe * per) : nullptr;
        // each output plane of the staging buffer has room for [per] frames
        sf_status s = sf_fit_ex(c, nf, ds, dn, dof, dc, dk, st);
        if (s != SF_OK) return s;
        SF_CUDA(cudaEventRecord(c->io_fit_done[ci & 1], st));
        if (ci > 0) {
            s = copy_out(ci - 1);
            if (s != SF_OK) return s;
        }
    }
    sf_status s = copy_out((n_frames - 1) / per);
    if (s != SF_OK) return s;
    for (int i = 0; i < 2; ++i) SF_CUDA(cudaStreamSynchronize(c->io_stream[i]));
    return SF_OK;
}

static sf_status quadtree_impl(sf_ctx* c, int n_frames, const void* depth, const sf_quad_params* p, sf_quad_node* nodes,
                      int capacity, int32_t* n_nodes, void* stream) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    if (!p || !n_nodes) return fail(SF_ERR_INVALID_ARG, "null params or n_nodes");
    if (c->dtab) return fail(SF_ERR_UNSUPPORTED, "the segmentation does not take a per-pixel delta table");
    if (c->constraint != SF_CONSTRAINT_UNIT3)
        return fail(SF_ERR_UNSUPPORTED, "the segmentation uses the |(a,b,c)| = 1 constraint only");
    if (n_frames < 0) return fail(SF_ERR_INVALID_ARG, "n_frames must be >= 0");
    if (capacity < 0 || (capacity > 0 && !nodes)) return fail(SF_ERR_INVALID_ARG, "bad node buffer");
    if (p->tile < 2 || p->tile > 64) return fail(SF_ERR_INVALID_ARG, "tile must be in [2, 64]");
    if (p->max_level < 0 || p->max_level > 6) return fail(SF_ERR_INVALID_ARG, "max_level must be in [0, 6]");
    if (!(p->tau > 0.f) || !std::isfinite(p->tau)) return fail(SF_ERR_INVALID_ARG, "tau must be finite and > 0");
    if (p->min_valid_permille < 0 || p->min_valid_permille > 1000)
        return fail(SF_ERR_INVALID_ARG, "min_valid_permille must be in [0, 1000]");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    SF_CUDA(cudaMemsetAsync(n_nodes, 0, sizeof(int32_t), st));
    if (n_frames == 0) return SF_OK;
    if (!depth) return fail(SF_ERR_INVALID_ARG, "null depth");
    if (misaligned(depth, depth_bytes(c->depth_type))) return fail(SF_ERR_INVALID_ARG, "depth must be aligned to its element size");
    // frames go through in groups of at most 64 (the per-frame quantum slots)
    const int per = std::min(n_frames, 64);
    const size_t tiles = (size_t)((c->W + p->tile - 1) / p->tile) * ((c->H + p->tile - 1) / p->tile);
    const size_t roots = tiles * per;
    size_t cap = roots;
    for (int l = 0; l < p->max_level; ++l) cap *= 4;
    cap = std::min(cap, (size_t)c->W * c->H * per);  // a node holds at least one pixel
    if (cap > ((size_t)1 << 28)) return fail(SF_ERR_INVALID_ARG, "quadtree too large: %zu nodes per level", cap);
    if (c->quad_cap < cap) {
        for (int i = 0; i < 2; ++i) {
            if (c->quad_q[i]) dev_free(c->quad_q[i]);
            c->quad_q[i] = nullptr;
        }
        c->quad_cap = 0;
        for (int i = 0; i < 2; ++i) {
            cudaError_t e = dev_alloc(&c->quad_q[i], sizeof(sf::QuadRect) * cap);
            if (e != cudaSuccess) return fail(SF_ERR_ALLOC, "quadtree queue of %zu nodes failed", cap);
        }
        c->quad_cap = cap;
    }
    if (!c->quad_cnt) {
        cudaError_t e = dev_alloc(&c->quad_cnt, sizeof(int) * 8);
        if (e != cudaSuccess) return fail(SF_ERR_ALLOC, "quadtree counters failed");
    }
    const size_t fe = (size_t)c->W * c->H;
    const size_t dbytes = depth_bytes(c->depth_type);
    for (int f0 = 0; f0 < n_frames; f0 += per) {
        const int nfr = std::min(per, n_frames - f0);
        const void* dp = static_cast<const char*>(depth) + dbytes * fe * f0;
        const size_t roots_n = tiles * nfr;
        sf_status s =
            c->depth_type == SF_DEPTH_F32 ? sfh::quadtree_f32(c, nfr, f0, dp, p, nodes, capacity, n_nodes, roots_n, st)
            : c->depth_type == SF_DEPTH_U16
                ? sfh::quadtree_u16(c, nfr, f0, dp, p, nodes, capacity, n_nodes, roots_n, st)
                : sfh::quadtree_disp(c, nfr, f0, dp, p, nodes, capacity, n_nodes, roots_n, st);
        if (s != SF_OK) return s;
    }
    return SF_OK;
}

sf_status sf_set_delta_table(sf_ctx* c, const float* ddx, const float* ddy) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    ++c->gen;  // a captured fit graph no longer applies
    if (!ddx != !ddy) return fail(SF_ERR_INVALID_ARG, "give both tables or neither");
    // fits already queued on the context's device may still read the old table
    {
        int prev = 0;
        SF_CUDA(cudaGetDevice(&prev));
        if (prev != c->device) SF_CUDA(cudaSetDevice(c->device));
        const cudaError_t e = cudaDeviceSynchronize();
        if (prev != c->device) cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(e, "sf_set_delta_table: synchronise");
    }
    if (!ddx) {
        if (c->dtab) dev_free(c->dtab);
        c->dtab = nullptr;
        return SF_OK;
    }
    const size_t n = (size_t)c->W * c->H;
    // the D plane then the E plane, in 1/kDeltaScale pixel
    std::vector<int> planes(2 * n);
    for (size_t i = 0; i < n; ++i) {
        const float a = ddx[i], b = ddy[i];
        if (!std::isfinite(a) || !std::isfinite(b) || std::fabs((double)a) * sf::kDeltaScale > sf::kDeltaMax ||
            std::fabs((double)b) * sf::kDeltaScale > sf::kDeltaMax)
            return fail(SF_ERR_INVALID_ARG, "delta table entry %zu (%g, %g) must be finite and below 16 pixels", i,
                        (double)a, (double)b);
        planes[i] = (int)std::lrint((double)a * sf::kDeltaScale);
        planes[n + i] = (int)std::lrint((double)b * sf::kDeltaScale);
    }
    if (!c->dtab) {
        cudaError_t e = dev_alloc(&c->dtab, 2 * n * sizeof(int));
        if (e != cudaSuccess) { c->dtab = nullptr; return fail(SF_ERR_ALLOC, "delta table of %zu bytes", n * 8); }
    }
    SF_CUDA(cudaMemcpy(c->dtab, planes.data(), 2 * n * sizeof(int), cudaMemcpyHostToDevice));
    SF_CUDA(cudaGetLastError());
    return SF_OK;
}

sf_status sf_set_tiles(sf_ctx* c, int hseg, int vband) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    ++c->gen;  // a captured fit graph no longer applies
    if (hseg != 0 && hseg != 8 && hseg != 16 && hseg != 32 && hseg != 64 && hseg != 128)
        return fail(SF_ERR_INVALID_ARG, "hseg must be 0, 8, 16, 32, 64 or 128");
    if (vband != 0 && (vband < 2 || vband > 1024)) return fail(SF_ERR_INVALID_ARG, "vband must be 0 or in [2, 1024]");
    c->hseg = hseg;
    c->vband = vband;
    return SF_OK;
}

sf_status sf_set_precision(sf_ctx* c, int mode, float tau) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    ++c->gen;  // a captured fit graph no longer applies
    if (mode < 0 || mode > 2) return fail(SF_ERR_INVALID_ARG, "precision mode %d must be 0, 1 or 2", mode);
    if (mode == 1 && !(tau > 0.f && tau <= 1.f)) return fail(SF_ERR_INVALID_ARG, "tau must be in (0, 1]");
    c->precision_mode = mode;
    if (mode == 1) c->tau = tau;
    return SF_OK;
}

sf_status sf_set_constraint(sf_ctx* c, int constraint) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    ++c->gen;  // a captured fit graph no longer applies
    if (constraint != SF_CONSTRAINT_UNIT3 && constraint != SF_CONSTRAINT_UNIT4)
        return fail(SF_ERR_INVALID_ARG, "constraint %d must be SF_CONSTRAINT_UNIT3 or SF_CONSTRAINT_UNIT4", constraint);
    c->constraint = constraint;
    return SF_OK;
}

sf_status sf_set_disparity_model(sf_ctx* c, double alpha, double beta) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    ++c->gen;  // a captured fit graph no longer applies
    if (!(alpha != 0.0) || !std::isfinite(alpha) || !std::isfinite(beta))
        return fail(SF_ERR_INVALID_ARG, "alpha must be finite and nonzero, beta finite");
    const double k = 128.0 * beta / std::fabs(alpha);
    if (!(std::fabs(k) <= 8388608.0)) return fail(SF_ERR_INVALID_ARG, "|128 beta / alpha| must be <= 2^23");
    c->disp_q = (float)(std::fabs(alpha) / 128.0);
    c->disp_mul = alpha > 0.0 ? 128 : -128;
    // 128 beta / |alpha| = integer part + fraction in [0, 1)
    const double fl = std::floor(k);
    c->disp_add = (int)fl;
    c->disp_frac = (float)(k - fl);
    if (c->disp_frac >= 1.f) { c->disp_add += 1; c->disp_frac = 0.f; }
    return SF_OK;
}

static sf_status fit_backward_impl(sf_ctx* c, int n_frames, const void* depth, const float* g_normals, const float* g_offsets,
                          const float* g_curvature, float* g_depth, unsigned flags, void* stream) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    if (n_frames < 0) return fail(SF_ERR_INVALID_ARG, "n_frames must be >= 0");
    if (n_frames == 0) return SF_OK;
    if (!depth || !g_normals || !g_offsets || !g_curvature || !g_depth)
        return fail(SF_ERR_INVALID_ARG, "null buffer");
    if (misaligned(depth, depth_bytes(c->depth_type)) || misaligned(g_normals, 4) || misaligned(g_offsets, 4) ||
        misaligned(g_curvature, 4) || misaligned(g_depth, 4))
        return fail(SF_ERR_INVALID_ARG, "buffers must be aligned to their element size");
    if (c->method != SF_METHOD_DISPARITY && c->method != SF_METHOD_STANDARD)
        return fail(SF_ERR_UNSUPPORTED, "the backward covers the implicit fits only");
    if (c->dtab) return fail(SF_ERR_UNSUPPORTED, "the backward does not take a per-pixel delta table");
    if (c->constraint != SF_CONSTRAINT_UNIT3)
        return fail(SF_ERR_UNSUPPORTED, "the backward covers the |(a,b,c)| = 1 constraint only");
    if (c->depth_type == SF_DEPTH_DISPARITY_U16)
        return fail(SF_ERR_UNSUPPORTED, "the backward takes depth input (f32 or u16)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t fe = (size_t)c->W * c->H;
    const size_t dbytes = depth_bytes(c->depth_type);
    const int per = std::min(c->max_frames_per_pass, 64);
    const int first = std::min(per, n_frames);
    sf_status s = ensure_planes(c, first);
    if (s != SF_OK) return s;
    // 12 adjoint planes per frame, then the per-frame bounds of their terms
    const size_t planes_bytes = sizeof(float) * 12 * fe * (size_t)first;
    const size_t need = planes_bytes + sizeof(float) * 3 * 64;
    if (c->adj_bytes < need) {
        if (c->adj) dev_free(c->adj);
        c->adj = nullptr;
        c->adj_max = nullptr;
        c->adj_bytes = 0;
        cudaError_t e = dev_alloc(&c->adj, need);
        if (e != cudaSuccess) return fail(SF_ERR_ALLOC, "adjoint scratch of %zu bytes failed", need);
        c->adj_bytes = need;
    }
    c->adj_max = reinterpret_cast<float*>(reinterpret_cast<char*>(c->adj) + c->adj_bytes - sizeof(float) * 3 * 64);
    // the caller vouches for the depth being unchanged since the last fit; the
    // rest (settings, buffer, frame count, one pass, no other call since that
    // wrote the scratch) is checked here, else the row pass runs again
    const sf_ctx::PlanesFrom& pf = c->planes_from;
    const bool reuse = (flags & SF_BACKWARD_AFTER_FIT) && n_frames <= per && pf.n == n_frames &&
                       pf.depth == depth && pf.gen == c->gen;
    if (reuse) ++c->backward_reuses;
    for (int f0 = 0; f0 < n_frames; f0 += per) {
        const int nfr = std::min(per, n_frames - f0);
        const void* dp = static_cast<const char*>(depth) + dbytes * fe * f0;
        const float* gn = g_normals + 3 * fe * f0;
        const float* gd = g_offsets + fe * f0;
        const float* gk = g_curvature + fe * f0;
        float* gz = g_depth + fe * f0;
        s = c->depth_type == SF_DEPTH_F32 ? sfh::backward_f32(c, nfr, dp, gn, gd, gk, gz, reuse, st)
                                           : sfh::backward_u16(c, nfr, dp, gn, gd, gk, gz, reuse, st);
        if (s != SF_OK) return s;
    }
    return SF_OK;
}

sf_status sf_precision_stats(sf_ctx* c, unsigned long long* queued, unsigned long long* resummed) {
    if (!c || !queued || !resummed) return fail(SF_ERR_INVALID_ARG, "null argument");
    unsigned h[3] = {0u, 0u, 0u};
    if (c->precision_mode > 0) {
        int prev = 0;
        SF_CUDA(cudaGetDevice(&prev));
        if (prev != c->device) SF_CUDA(cudaSetDevice(c->device));
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(h, c->flag_count, sizeof(h), cudaMemcpyDeviceToHost);
        if (prev != c->device) cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(e, "sf_precision_stats");
    }
    // [0] counts reserved queue slots (holes included) except on the ray-table path, which
    // reserves no chunks; [2] counts the windows queued
    *queued = c->dtab ? h[0] : h[2];
    *resummed = c->precision_mode == 2 ? *queued : h[1];  // mode 2 re-sums every queued window
    return SF_OK;
}

sf_status sf_profile_enable(sf_ctx* c, int on) {
    if (!c) return fail(SF_ERR_INVALID_ARG, "null context");
    for (auto& r : c->recs) { c->event_pool.push_back(r.a); c->event_pool.push_back(r.b); }
    c->recs.clear();
    c->profiling = on != 0;
    return SF_OK;
}

sf_status sf_profile_read(sf_ctx* c, int n_stages, double* ms, int* launches) {
    if (!c || n_stages < 0 || (n_stages > 0 && (!ms || !launches)))
        return fail(SF_ERR_INVALID_ARG, "bad profile_read arguments");
    for (int s = 0; s < n_stages; ++s) { ms[s] = 0.0; launches[s] = 0; }
    for (auto& r : c->recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(e, "profile event");
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        if (r.stage < n_stages) { ms[r.stage] += t; launches[r.stage] += 1; }
        c->event_pool.push_back(r.a);
        c->event_pool.push_back(r.b);
    }
    c->recs.clear();
    return SF_OK;
}

sf_status sf_destroy(sf_ctx* c) {
    if (!c) return SF_OK;
    for (auto& r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->tx) dev_free(c->tx);
    if (c->ty) dev_free(c->ty);
    if (c->vmax) dev_free(c->vmax);
    if (c->planes) dev_free(c->planes);
    for (int i = 0; i < 2; ++i) {
        if (c->d_io[i]) dev_free(c->d_io[i]);
        if (c->io_stream[i]) cudaStreamDestroy(c->io_stream[i]);
        if (c->io_fit_done[i]) cudaEventDestroy(c->io_fit_done[i]);
    }
    if (c->io_entry) cudaEventDestroy(c->io_entry);
    if (c->adj) dev_free(c->adj);
    if (c->dtab) dev_free(c->dtab);
    if (c->flags) dev_free(c->flags);
    if (c->moments_q) dev_free(c->moments_q);
    if (c->queue_c) dev_free(c->queue_c);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph_stream) cudaStreamDestroy(c->graph_stream);
    if (c->flag_count) dev_free(c->flag_count);
    if (c->rays64) dev_free(c->rays64);
    for (int i = 0; i < 2; ++i)
        if (c->quad_q[i]) dev_free(c->quad_q[i]);
    if (c->quad_cnt) dev_free(c->quad_cnt);
    delete c;
    return SF_OK;
}

}  // extern "C"

// ===========================================================================
// Mixed-resolution batches
// ===========================================================================
namespace {

sf_status batch_enqueue(sf_batch* b, cudaStream_t st) {
    return b->depth_type == SF_DEPTH_F32 ? sfh::batch_enqueue_f32(b, st) : sfh::batch_enqueue_u16(b, st);
}

}  // namespace

extern "C" {

sf_status sf_batch_destroy(sf_batch* b) {
    if (!b) return SF_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    dev_free(b->d_desc);
    dev_free(b->d_items);
    dev_free(b->d_sync);
    if (b->done) cudaEventDestroy(b->done);
    dev_free(b->d_rays);
    dev_free(b->d_planes);
    delete b;
    return SF_OK;
}

sf_status sf_batch_create(const sf_batch_frame* frames, int n_frames, int method, int depth_type, float depth_scale,
                          int min_valid, int require_center_valid, int use_graph, sf_batch** out) {
    if (!frames || !out || n_frames < 1) return fail(SF_ERR_INVALID_ARG, "need at least one frame and an output");
    *out = nullptr;
    if (n_frames > 65535) return fail(SF_ERR_INVALID_ARG, "at most 65535 frames per batch");
    if (method != SF_METHOD_DISPARITY && method != SF_METHOD_STANDARD)
        return fail(SF_ERR_UNSUPPORTED, "batches support the disparity and standard implicit fits");
    if (depth_type == SF_DEPTH_DISPARITY_U16)
        return fail(SF_ERR_UNSUPPORTED, "disparity input goes through a context (sf_fit_ex, sf_quadtree)");
    if (depth_type != SF_DEPTH_F32 && depth_type != SF_DEPTH_U16)
        return fail(SF_ERR_INVALID_ARG, "unknown depth type %d", depth_type);
    if (depth_type == SF_DEPTH_U16 && !(depth_scale > 0.f && std::isfinite(depth_scale)))
        return fail(SF_ERR_INVALID_ARG, "depth_scale must be positive and finite");
    if (min_valid < 1) return fail(SF_ERR_INVALID_ARG, "min_valid must be >= 1");
    std::vector<sf::FrameDesc> desc(n_frames);
    std::vector<int> order(n_frames);
    size_t stride = 0, rays = 0;
    int max_r = 0, max_seg = 32;
    long long pixels = 0;
    for (int f = 0; f < n_frames; ++f) {
        const sf_batch_frame& F = frames[f];
        if (F.W < 1 || F.H < 1 || (size_t)F.W * F.H > ((size_t)1 << 31))
            return fail(SF_ERR_INVALID_ARG, "frame %d: bad size %dx%d", f, F.W, F.H);
        if (F.window < 1 || (F.window & 1) == 0 || F.window > SF_MAX_WINDOW)
            return fail(SF_ERR_INVALID_ARG, "frame %d: window %d must be odd and in [1, %d]", f, F.window,
                        SF_MAX_WINDOW);
        if (!F.depth || !F.normals || !F.offsets || !F.curvature)
            return fail(SF_ERR_INVALID_ARG, "frame %d: null buffer", f);
        const sf_intrinsics& K = F.K;
        if (!(K.fx != 0.0) || !(K.fy != 0.0) || !std::isfinite(K.fx) || !std::isfinite(K.fy) ||
            !std::isfinite(K.cx) || !std::isfinite(K.cy) || !std::isfinite(K.dx) || !std::isfinite(K.dy))
            return fail(SF_ERR_INVALID_ARG, "frame %d: intrinsics must be finite with nonzero focal lengths", f);
        int seg = F.hseg ? F.hseg : sf::kHSeg;
        if (seg != 32 && seg != 64 && seg != 128) return fail(SF_ERR_INVALID_ARG, "frame %d: hseg must be 32, 64 or 128", f);
        if (method == SF_METHOD_STANDARD) seg = 32;  // the batch kernel's tiles of the standard form
        const int band = F.vband ? F.vband : 64;
        if (band < 8 || band > 1024) return fail(SF_ERR_INVALID_ARG, "frame %d: vband must be in [8, 1024]", f);
        sf::FrameDesc& d = desc[f];
        d.depth = F.depth; d.normals = F.normals; d.offsets = F.offsets; d.curvature = F.curvature;
        d.W = F.W; d.H = F.H; d.r = (F.window - 1) / 2; d.bits = sfh::quant_bits(method, F.window);
        d.Wp = (F.W + 63) / 64 * 64; d.seg = seg; d.band = band;
        d.a = (float)(1.0 / K.fx); d.b = (float)(1.0 / K.fy);
        d.pofs = stride;
        stride += (size_t)d.Wp * F.H;
        rays += (size_t)F.W + F.H;
        max_r = std::max(max_r, d.r);
        max_seg = std::max(max_seg, seg);
        pixels += (long long)F.W * F.H;
        order[f] = f;
    }
    sf_batch* b = new (std::nothrow) sf_batch();
    if (!b) return fail(SF_ERR_ALLOC, "batch allocation failed");
    b->n = n_frames; b->method = method; b->depth_type = depth_type; b->depth_scale = depth_scale;
    b->min_valid = min_valid; b->require_center = require_center_valid ? 1 : 0;
    b->stride = stride; b->pixels = pixels;
    // ray tables (Eq. 10) in FP64 -> FP32, all frames in one buffer
    std::vector<float> hr(rays);
    size_t ro = 0;
    std::vector<size_t> rofs(n_frames);
    for (int f = 0; f < n_frames; ++f) {
        const sf_batch_frame& F = frames[f];
        rofs[f] = ro;
        for (int x = 0; x < F.W; ++x) hr[ro + x] = (float)((x + F.K.dx - F.K.cx) / F.K.fx);
        for (int y = 0; y < F.H; ++y) hr[ro + F.W + y] = (float)((y + F.K.dy - F.K.cy) / F.K.fy);
        ro += (size_t)F.W + F.H;
    }
    // work items, largest frames first so that the tail holds the small ones
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (long long)desc[a].W * desc[a].H > (long long)desc[c].W * desc[c].H;
    });
    // in claim order: every frame's quantum chunks, then its tiles, then its bands
    const bool fixed_q = depth_type == SF_DEPTH_U16 && method == SF_METHOD_STANDARD;  // raw depth, no quantum
    std::vector<int3> ritems, hitems, vitems;
    for (int f : order) {
        sf::FrameDesc& d = desc[f];
        const size_t fe = (size_t)d.W * d.H;
        d.nr = fixed_q ? 0 : (int)((fe + sf::kRangeChunk - 1) / sf::kRangeChunk);
        for (int c = 0; c < d.nr; ++c) ritems.push_back(make_int3(f, c, 0));
        d.nh = 0;
        for (int y0 = 0; y0 < d.H; y0 += sf::kHThreads)
            for (int x0 = 0; x0 < d.W; x0 += d.seg) { hitems.push_back(make_int3(f, x0, y0)); ++d.nh; }
        for (int y0 = 0; y0 < d.H; y0 += d.band)
            for (int x0 = 0; x0 < d.W; x0 += sf::kVThreads) vitems.push_back(make_int3(f, x0, y0));
    }
    b->n_r = (int)ritems.size();
    b->n_h = (int)hitems.size();
    b->n_v = (int)vitems.size();
    std::vector<int3> items(ritems);
    items.insert(items.end(), hitems.begin(), hitems.end());
    items.insert(items.end(), vitems.begin(), vitems.end());
    cudaError_t e = dev_alloc(&b->d_rays, sizeof(float) * std::max<size_t>(rays, 1));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_rays, hr.data(), sizeof(float) * rays, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        for (int f = 0; f < n_frames; ++f) {
            desc[f].tx = b->d_rays + rofs[f];
            desc[f].ty = b->d_rays + rofs[f] + desc[f].W;
        }
        e = dev_alloc(&b->d_desc, sizeof(sf::FrameDesc) * n_frames);
    }
    if (e == cudaSuccess) e = cudaMemcpy(b->d_desc, desc.data(), sizeof(sf::FrameDesc) * n_frames, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_alloc(&b->d_items, sizeof(int3) * items.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), sizeof(int3) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_alloc(&b->d_sync, sizeof(unsigned) * (3 + 3 * (size_t)n_frames));
    if (e == cudaSuccess) e = cudaMemset(b->d_sync, 0, sizeof(unsigned) * (3 + 3 * (size_t)n_frames));
    if (e == cudaSuccess) {
        const unsigned limit = kBatchWaitPolls;
        e = cudaMemcpy(b->d_sync + 2, &limit, sizeof(unsigned), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = dev_alloc(&b->d_planes, sfh::plane_bytes_per_frame(method, stride));
    if (e != cudaSuccess) { sf_batch_destroy(b); return fail(SF_ERR_ALLOC, "batch buffers: %s", cudaGetErrorString(e)); }
    b->hsmem = sizeof(int) * sf::kHThreads * (size_t)((max_seg + 2 * max_r) | 1);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (depth_type == SF_DEPTH_F32) sfh::batch_grids_f32(b, sms);
    else sfh::batch_grids_u16(b, sms);
    e = cudaGetLastError();
    if (e != cudaSuccess) { sf_batch_destroy(b); return cuda_fail(e, "batch kernel attributes"); }
    if (use_graph) {
        // capture the whole pass once; sf_batch_run then replays it
        e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { sf_batch_destroy(b); return cuda_fail(e, "batch graph capture"); }
        sf_status s = batch_enqueue(b, b->cap);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(b->cap, &g);
        if (s != SF_OK) { if (g) cudaGraphDestroy(g); sf_batch_destroy(b); return s; }
        if (e != cudaSuccess) { sf_batch_destroy(b); return cuda_fail(e, "batch graph capture"); }
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) { sf_batch_destroy(b); return cuda_fail(e, "batch graph instantiate"); }
        b->use_graph = true;
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { sf_batch_destroy(b); return cuda_fail(e, "batch setup"); }
    *out = b;
    return SF_OK;
}

static sf_status batch_run_impl(sf_batch* b, void* stream) {
    if (!b) return fail(SF_ERR_INVALID_ARG, "null batch");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (b->use_graph) {
        cudaError_t e = cudaGraphLaunch(b->exec, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
    } else {
        sf_status s = batch_enqueue(b, st);
        if (s != SF_OK) return s;
    }
    SF_CUDA(cudaEventRecord(b->done, st));
    return SF_OK;
}

sf_status sf_batch_check(sf_batch* b) {
    if (!b) return fail(SF_ERR_INVALID_ARG, "null batch");
    SF_CUDA(cudaEventSynchronize(b->done));
    unsigned err = 0;
    SF_CUDA(cudaMemcpy(&err, b->d_sync + 1, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err)
        return fail(SF_ERR_TIMEOUT, "batch: a %s gave up waiting (error word 0x%x); its outputs are not written",
                    (err & 2) ? "column band" : "horizontal tile", err);
    return SF_OK;
}

sf_status sf_batch_set_wait_limit(sf_batch* b, unsigned polls) {
    if (!b) return fail(SF_ERR_INVALID_ARG, "null batch");
    SF_CUDA(cudaEventSynchronize(b->done));
    SF_CUDA(cudaMemcpy(b->d_sync + 2, &polls, sizeof(unsigned), cudaMemcpyHostToDevice));
    return SF_OK;
}

sf_status sf_batch_info(const sf_batch* b, long long* pixels, int* launches) {
    if (!b || !pixels || !launches) return fail(SF_ERR_INVALID_ARG, "null argument");
    *pixels = b->pixels;
    *launches = 1;
    return SF_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free entry point: sf_fit_static
// ===========================================================================
// Some callers cannot allocate device memory at the point where they need a
// fit: code running while a CUDA graph is being captured, real-time loops that
// forbid allocator calls after start-up, or hosts that hand the GPU's memory
// to their own allocator and leave none to cudaMalloc.  sf_fit_static serves
// them: it takes the same inputs and outputs as sf_fit but keeps every byte
// of its scratch (the fixed-point quantum, the ray tables and the horizontal
// moment planes) in one statically sized device array that exists from module
// load until process exit.
namespace sf {

constexpr size_t kStaticScratchBytes = (size_t)SF_STATIC_SCRATCH_BYTES;  // per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Ray tangents of Eq. 10 computed in FP64 and rounded to FP32, the same
// values sf_create computes on the host.
__global__ void ray_table_kernel(double fx, double fy, double cx, double cy, double dx, double dy, int W, int H,
                                 float* __restrict__ tx, float* __restrict__ ty) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < W) tx[i] = (float)((i + dx - cx) / fx);
    if (i < H) ty[i] = (float)((i + dy - cy) / fy);
}

}  // namespace sf

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_base[kStaticMaxDevices] = {nullptr};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device address of the static scratch for the current device, resolved once.
sf_status static_scratch_base(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "sf_fit_static: cudaGetDevice");
    if (dev < 0 || dev >= kStaticMaxDevices) return fail(SF_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_base[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, sf::g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "sf_fit_static: cudaGetSymbolAddress");
        set_kernel_attributes();
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "sf_fit_static: kernel attributes");
        g_static_base[dev] = p;
    }
    *out = g_static_base[dev];
    return SF_OK;
}

}  // namespace

static sf_status fit_static_impl(const sf_intrinsics* K, int W, int H, int window, int method, int depth_type,
                                 float depth_scale, int min_valid, int require_center_valid, const void* depth,
                                 float* normals, float* offsets, float* curvature, void* stream) {
    if (!K) return fail(SF_ERR_INVALID_ARG, "null intrinsics");
    if (!depth || !normals || !offsets || !curvature) return fail(SF_ERR_INVALID_ARG, "null buffer");
    if (misaligned(depth, depth_type == SF_DEPTH_F32 ? 4 : 2) || misaligned(normals, 4) || misaligned(offsets, 4) ||
        misaligned(curvature, 4))
        return fail(SF_ERR_INVALID_ARG, "buffers must be aligned to their element size");
    if (W < 1 || H < 1) return fail(SF_ERR_INVALID_ARG, "image size %dx%d must be positive", W, H);
    if (window < 1 || (window & 1) == 0 || window > SF_MAX_WINDOW)
        return fail(SF_ERR_INVALID_ARG, "window %d must be odd and in [1, %d]", window, SF_MAX_WINDOW);
    if (!(K->fx != 0.0) || !(K->fy != 0.0) || !std::isfinite(K->fx) || !std::isfinite(K->fy) ||
        !std::isfinite(K->cx) || !std::isfinite(K->cy) || !std::isfinite(K->dx) || !std::isfinite(K->dy))
        return fail(SF_ERR_INVALID_ARG, "intrinsics must be finite with nonzero focal lengths");
    if (method != SF_METHOD_DISPARITY && method != SF_METHOD_STANDARD)
        return fail(SF_ERR_UNSUPPORTED, "sf_fit_static supports the disparity and standard implicit fits");
    if (depth_type == SF_DEPTH_DISPARITY_U16)
        return fail(SF_ERR_UNSUPPORTED, "disparity input goes through a context (sf_fit_ex, sf_quadtree)");
    if (depth_type != SF_DEPTH_F32 && depth_type != SF_DEPTH_U16)
        return fail(SF_ERR_INVALID_ARG, "unknown depth type %d", depth_type);
    if (depth_type == SF_DEPTH_U16 && !(depth_scale > 0.f && std::isfinite(depth_scale)))
        return fail(SF_ERR_INVALID_ARG, "depth_scale must be positive and finite");
    if (min_valid < 1) return fail(SF_ERR_INVALID_ARG, "min_valid must be >= 1");
    // scratch layout inside the static array: quantum word | tx[W] | ty[H] | moment planes
    const int Wp = (W + 63) / 64 * 64;
    const size_t plane_elems = (size_t)Wp * H;
    const size_t off_tx = 256;
    const size_t off_ty = off_tx + align256(sizeof(float) * W);
    const size_t off_planes = off_ty + align256(sizeof(float) * H);
    const size_t need = off_planes + sfh::plane_bytes_per_frame(method, plane_elems);
    if (need > sf::kStaticScratchBytes)
        return fail(SF_ERR_INVALID_ARG,
                    "sf_fit_static: a %dx%d frame needs %zu bytes of scratch, more than the %zu-byte static array "
                    "(use sf_create/sf_fit for larger frames)", W, H, need, sf::kStaticScratchBytes);
    void* base = nullptr;
    sf_status s = static_scratch_base(&base);
    if (s != SF_OK) return s;
    char* b = static_cast<char*>(base);
    // A context on the stack that points into the static array: nothing is allocated.
    sf_ctx c;
    c.K = *K;
    c.W = W; c.H = H; c.k = window; c.r = (window - 1) / 2;
    c.Wp = Wp;
    c.plane_elems = plane_elems;
    c.method = method;
    c.depth_type = depth_type;
    c.depth_scale = depth_scale;
    c.min_valid = min_valid;
    c.require_center = require_center_valid ? 1 : 0;
    c.vmax = reinterpret_cast<unsigned*>(b);
    c.tx = reinterpret_cast<float*>(b + off_tx);
    c.ty = reinterpret_cast<float*>(b + off_ty);
    c.planes = b + off_planes;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    {
        const int n = std::max(W, H);
        sf::ray_table_kernel<<<(n + 255) / 256, 256, 0, st>>>(K->fx, K->fy, K->cx, K->cy, K->dx, K->dy, W, H, c.tx,
                                                            c.ty);
    }
    // the pass clears the quantum word itself (cudaMemsetAsync) before use
    s = depth_type == SF_DEPTH_F32 ? sfh::fit_pass_f32(&c, 1, depth, normals, offsets, curvature, nullptr, st)
                                   : sfh::fit_pass_u16(&c, 1, depth, normals, offsets, curvature, nullptr, st);
    // c points into the static array: nothing to free
    c.tx = nullptr; c.ty = nullptr; c.vmax = nullptr; c.planes = nullptr;
    return s;
}

// Bounds-checked build: after the work, report the first out-of-range moment
// plane access any kernel recorded (SF_ERR_CUDA).  Synchronises the device.
static sf_status check_bounds(sf_status s) {
#if SF_CHECK_BOUNDS
    if (s != SF_OK) return s;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "bounds check synchronise");
    const unsigned long long w[3] = {sfh::bounds_word_f32(), sfh::bounds_word_u16(), sfh::bounds_word_disp()};
    for (unsigned long long v : w)
        if (v)
            return fail(SF_ERR_CUDA, "out-of-range moment plane access (site %d, entry %llu)", (int)((v >> 56) & 127),
                        v & ((1ull << 56) - 1));
#endif
    return s;
}

extern "C" {

// Every call that writes the scratch planes or the per-frame quanta records
// what they hold afterwards (a fit or backward of at most one pass of frames
// without a delta table), or that they hold nothing known.
static void note_planes(sf_ctx* c, int n_frames, const void* depth, sf_status s) {
    if (!c) return;
    const bool one_pass = n_frames > 0 && n_frames <= std::min(c->max_frames_per_pass, 64);
    if (s == SF_OK && one_pass && depth && !c->dtab) c->planes_from = sf_ctx::PlanesFrom{c->gen, depth, n_frames};
    else c->planes_from = sf_ctx::PlanesFrom{};
}

sf_status sf_fit_ex(sf_ctx* c, int n_frames, const void* depth, float* normals, float* offsets, float* curvature,
                    int32_t* counts, void* stream) {
    const sf_status s = check_bounds(fit_ex_impl(c, n_frames, depth, normals, offsets, curvature, counts, stream));
    note_planes(c, n_frames, depth, s);
    return s;
}
sf_status sf_fit_host(sf_ctx* c, int n_frames, const void* depth, float* normals, float* offsets, float* curvature,
                      int32_t* counts, void* stream) {
    return check_bounds(fit_host_impl(c, n_frames, depth, normals, offsets, curvature, counts, stream));
}
sf_status sf_fit_backward_ex(sf_ctx* c, int n_frames, const void* depth, const float* g_normals,
                             const float* g_offsets, const float* g_curvature, float* g_depth, unsigned flags,
                             void* stream) {
    const sf_status s = check_bounds(
        fit_backward_impl(c, n_frames, depth, g_normals, g_offsets, g_curvature, g_depth, flags, stream));
    note_planes(c, n_frames, depth, s);
    return s;
}
sf_status sf_fit_backward(sf_ctx* c, int n_frames, const void* depth, const float* g_normals, const float* g_offsets,
                          const float* g_curvature, float* g_depth, void* stream) {
    return sf_fit_backward_ex(c, n_frames, depth, g_normals, g_offsets, g_curvature, g_depth, 0u, stream);
}
sf_status sf_quadtree(sf_ctx* c, int n_frames, const void* depth, const sf_quad_params* params, sf_quad_node* nodes,
                      int capacity, int32_t* n_nodes, void* stream) {
    if (c) c->planes_from = sf_ctx::PlanesFrom{};  // its range pass overwrites the quanta
    return check_bounds(quadtree_impl(c, n_frames, depth, params, nodes, capacity, n_nodes, stream));
}
sf_status sf_batch_run(sf_batch* b, void* stream) { return check_bounds(batch_run_impl(b, stream)); }

}  // extern "C"

extern "C" sf_status sf_fit_static(const sf_intrinsics* K, int W, int H, int window, int method, int depth_type,
                                   float depth_scale, int min_valid, int require_center_valid, const void* depth,
                                   float* normals, float* offsets, float* curvature, void* stream) {
    return check_bounds(fit_static_impl(K, W, H, window, method, depth_type, depth_scale, min_valid,
                                        require_center_valid, depth, normals, offsets, curvature, stream));
}
