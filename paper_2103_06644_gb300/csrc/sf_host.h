// sf_host.h -- host-side internals shared by the library's translation units:
// the context and batch objects, error reporting, and the per-depth-type
// launchers.  Every launcher for one depth encoding lives in its own .cu file
// (fit_f32.cu, fit_u16.cu, fit_disp.cu) so that the kernels compile in
// parallel; surffit.cu holds the C ABI and dispatches to them.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "surffit.h"

namespace sf {
struct QuadRect;
struct FrameDesc;
}  // namespace sf

struct sf_ctx {
    sf_intrinsics K;
    int W, H, k, r;
    int Wp;
    size_t plane_elems;
    int method = SF_METHOD_DISPARITY;
    int depth_type = SF_DEPTH_F32;
    int hseg = 0;         // horizontal tile width (8, 16, 32, 64 or 128; 0: automatic)
    int vband = 0;        // vertical band height (0: chosen from the grid size)
    float depth_scale = 1e-3f;
    // SF_DEPTH_DISPARITY_U16: 1/Z = disp_q * (disp_mul * D + disp_add + disp_frac)
    float disp_q = 1.f / 128.f;
    int disp_mul = 128, disp_add = 0;
    float disp_frac = 0.f;    // in [0, 1)
    int min_valid = 3;
    int require_center = 1;
    int device = 0;
    int sms = 152;        // streaming multiprocessors of the device (grid sizing)
    float* tx = nullptr;  // [W]
    float* ty = nullptr;  // [H]
    unsigned* vmax = nullptr;  // [max_frames]
    void* planes = nullptr;
    int planes_frames = 0;     // frames the planes buffer holds
    size_t planes_bytes = 0;
    int max_frames_per_pass = 1;
    // sf_fit_host: two device staging buffers and copy streams (one per
    // chunk parity) and the event that orders the fits on the shared scratch
    void* d_io[2] = {nullptr, nullptr};
    size_t d_io_bytes = 0;
    cudaStream_t io_stream[2] = {nullptr, nullptr};
    cudaEvent_t io_fit_done[2] = {nullptr, nullptr};
    cudaEvent_t io_entry = nullptr;
    float* adj = nullptr;      // backward: per-window adjoint planes
    float* adj_max = nullptr;  // backward: per-frame bounds of the adjoint terms [64][3] (inside adj)
    size_t adj_bytes = 0;
    int* dtab = nullptr;       // per-pixel ray adjustments: D plane then E plane [H][W], 1/2^18 pixel, or none
    // precision fallback
    int precision_mode = 0;    // 0 float32 solve, 1 + refinement where gap < tau, 2 refinement everywhere
    int constraint = SF_CONSTRAINT_UNIT3;  // normalisation of the implicit fits (Eq. 4)
    float tau = 1e-3f;
    unsigned long long* flags = nullptr;   // queue of flagged windows (frame, y, x)
    size_t flags_cap = 0;      // entries
    unsigned* flag_count = nullptr;        // [3]: queue slots reserved, windows to re-sum, windows queued
    unsigned* queue_c = nullptr;           // queue indices of the windows to re-sum (flags_cap)
    void* moments_q = nullptr; // exact window moments of the first moments_cap queued windows
    size_t moments_cap = 0;    // entries
    double* rays64 = nullptr;  // [W] tx, [H] ty, 1/fx, 1/fy in FP64
    // sf_quadtree: two node queues (ping-pong between levels) and the per-level counters
    sf::QuadRect* quad_q[2] = {nullptr, nullptr};
    size_t quad_cap = 0;       // entries per queue
    int* quad_cnt = nullptr;   // [8]
    // sf_fit_ex: the last single-pass call captured in a CUDA graph, replayed
    // while the same buffers and configuration recur (a call whose key
    // repeats the previous call's is captured; `gen` changes with every
    // setter and scratch reallocation)
    struct FitKey {
        unsigned long long gen;
        int n;
        const void* depth;
        const float *normals, *offsets, *curvature;
        const int32_t* counts;
        bool operator==(const FitKey& o) const {
            return gen == o.gen && n == o.n && depth == o.depth && normals == o.normals && offsets == o.offsets &&
                   curvature == o.curvature && counts == o.counts;
        }
    };
    unsigned long long gen = 1;
    FitKey last_key{}, graph_key{};
    cudaStream_t graph_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_replays = 0;  // fit calls served by replaying graph_exec
    long long backward_reuses = 0;  // backward calls that reused the last fit's row pass
    // what the scratch planes and per-frame quanta hold: the row pass of the n
    // frames at `depth` under settings generation gen (n == 0: unknown)
    struct PlanesFrom {
        unsigned long long gen = 0;
        const void* depth = nullptr;
        int n = 0;
    } planes_from;
    // profiling: (stage, start event, stop event) per recorded launch
    bool profiling = false;
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
};

struct sf_batch {
    int n = 0;
    int method = SF_METHOD_DISPARITY, depth_type = SF_DEPTH_F32;
    float depth_scale = 1e-3f;
    int min_valid = 3, require_center = 1;
    sf::FrameDesc* d_desc = nullptr;
    int3* d_items = nullptr;         // quantum chunks, horizontal tiles, column bands
    int n_r = 0, n_h = 0, n_v = 0;
    unsigned* d_sync = nullptr;      // claim, error word, poll limit, then per frame [3][n]
    float* d_rays = nullptr;
    void* d_planes = nullptr;
    size_t stride = 0;
    size_t hsmem = 0;
    int grid = 0;
    cudaEvent_t done = nullptr;      // recorded after each run
    long long pixels = 0;
    bool use_graph = false;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace sfh {

// Record a message for sf_last_error (calling thread) and return the status.
sf_status fail(sf_status s, const char* fmt, ...);
sf_status cuda_fail(cudaError_t e, const char* what);

#define SF_CUDA(call)                                              \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::sfh::cuda_fail(_e, #call); \
    } while (0)

// Output columns per thread of the horizontal pass and rows per band of the
// vertical pass for nfr frames (the context's hseg / vband, else chosen from
// the grid size and the window).
int horizontal_seg(const sf_ctx* c, int nfr);
int vertical_band(const sf_ctx* c, int nfr);
// Bytes of horizontal-moment scratch per frame of plane_elems entries.
size_t plane_bytes_per_frame(int method, size_t plane_elems);
// Fixed-point bits of a method and window (the most that keeps every exact
// window sum and re-centring product inside its integer type).
int quant_bits(int method, int k);
// Bytes of one queued window's exact moments (precision mode 1).
constexpr size_t kMomentEntryBytes = 80;

// Per-depth-encoding launchers (one translation unit each).  `nfr` frames of
// the context's size, at most 64, already validated by the caller.
#define SF_DECLARE_LAUNCHERS(dt)                                                                                       \
    sf_status fit_pass_##dt(sf_ctx* c, int nfr, const void* depth, float* normals, float* offsets, float* curv,      \
                            int32_t* counts, cudaStream_t st);                                                         \
    sf_status delta_pass_##dt(sf_ctx* c, int nfr, const void* depth, float* normals, float* offsets, float* curv,    \
                              int32_t* counts, cudaStream_t st);                                                       \
    sf_status backward_##dt(sf_ctx* c, int nfr, const void* depth, const float* gn, const float* gd, const float* gk, \
                            float* g_depth, bool reuse, cudaStream_t st);                                              \
    sf_status quadtree_##dt(sf_ctx* c, int nfr, int frame_base, const void* depth, const sf_quad_params* p,         \
                            sf_quad_node* nodes, int capacity, int32_t* n_nodes, size_t roots, cudaStream_t st);      \
    sf_status batch_enqueue_##dt(sf_batch* b, cudaStream_t st);                                                       \
    void batch_grids_##dt(sf_batch* b, int sms);                                                                      \
    void set_kernel_smem_##dt();                                                                                      \
    unsigned long long bounds_word_##dt();
SF_DECLARE_LAUNCHERS(f32)
SF_DECLARE_LAUNCHERS(u16)
SF_DECLARE_LAUNCHERS(disp)
#undef SF_DECLARE_LAUNCHERS

}  // namespace sfh
