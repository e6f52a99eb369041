// sf_kernels.cuh -- GB300 (sm_103a) device kernels for dense RGBD plane fitting
//
// Pipeline for one frame (all device work, no host synchronisation):
//   1. range     max of the fixed-point variable over the frame's valid pixels
//                (1/Z for the disparity form, Z for the standard form), giving
//                a power-of-two quantum so that every value fits in `bits`
//                bits (26-28 for the disparity form, 23-28 for the standard
//                form: the most that keeps every exact sum inside int64).
//   2. hpass     one thread per image row slides a k-wide window along the row
//                and writes exact integer horizontal window moments
//                (sums of v, v*j, v*j^2 for the mask, w and w^2 ...) to scratch.
//   3. vpass     one thread per image column slides the window down the
//                column over those moments (plus the i-weighted sums), which
//                yields the exact 2D window moments of every pixel, and solves
//                the plane fit in registers (sf_solve.cuh).
//
// The integral-image idea of Section II.C appears here as running sums: every
// window sum costs O(1) per pixel regardless of k.  All sums are integers, so
// they are exact and the result does not depend on the image size or on the
// order of summation (no floating-point summed-area table is ever formed).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "surffit.h"
#include "sf_solve.cuh"

namespace sf {

constexpr int kMaxR = (SF_MAX_WINDOW - 1) / 2;
constexpr int kHThreads = 128;   // rows per hpass block
constexpr int kHSeg = 32;        // default output columns per hpass thread (runtime: 8..128)
constexpr int kVThreads = 128;   // columns per vpass block


// The moments an explicit fit needs are those of its implicit counterpart.
__host__ __device__ constexpr int base_method(int M) {
    return M == SF_METHOD_EXPLICIT_DISPARITY ? SF_METHOD_DISPARITY
                                             : (M == SF_METHOD_EXPLICIT_STANDARD ? SF_METHOD_STANDARD : M);
}

// Register budget of the vertical-pass kernels, as resident blocks per SM:
// 6 blocks (24 warps, 80 registers).  The scratch loads need the warps for
// latency hiding; at 8 blocks (64 registers) the per-column pass spills.
constexpr int kVBlocks = 6;

// The precision modes' window queue: entries (frame << 48 | y << 24 | x).  A
// warp of the column pass reserves kQueueChunk slots at a time (one atomic per
// chunk instead of one per row: a single counter hammered by every warp cost
// the pass a fifth of its time) and marks the slots it leaves unused as holes,
// which the queue's readers skip.
constexpr unsigned long long kQueueHole = ~0ull;
constexpr unsigned kQueueChunk = 32;


// ---------------------------------------------------------------------------
// Depth decoding.  Codec: how a stored value becomes depth.
//   SF_DEPTH_F32             metres (scale unused)
//   SF_DEPTH_U16             raw * scale metres, raw == 0 missing
//   SF_DEPTH_DISPARITY_U16   raw disparity D: 1/Z = scale * (dmul * D + dadd + frac)
//                            (dmul = +-128, dadd an integer and frac in [0, 1):
//                            the sensor model 1/Z = alpha D + beta with
//                            scale = |alpha| / 128 and dadd + frac =
//                            128 beta / |alpha|); D == 0 or 1/Z <= 0 missing.
//                            The integer part w = dmul D + dadd is what the
//                            exact sums hold; frac shifts every value of a
//                            window alike, so it enters the solve only through
//                            the mean disparity.
// ---------------------------------------------------------------------------
struct Codec {
    float scale;
    int dmul, dadd;
    float frac;
};

// A kernel launched with programmatic dependent launch may start while the
// previous kernel of its stream is still finishing; it waits here until that
// kernel has completed and its writes are visible (a no-op for a kernel
// launched without it).
__device__ __forceinline__ void wait_for_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Raw stored value: metres for float32, raw units for uint16 (0 = missing).
template <int DT>
__device__ __forceinline__ float load_raw(const void* base, size_t idx) {
    if (DT == SF_DEPTH_F32) return __ldg(reinterpret_cast<const float*>(base) + idx);
    return (float)__ldg(reinterpret_cast<const unsigned short*>(base) + idx);
}

// Disparity input: the integer part w = dmul * D + dadd (units of scale) of a
// valid pixel (w + frac > 0), or -1.
__device__ __forceinline__ int disparity_units(float d_raw, const Codec& cd) {
    const int D = (int)d_raw;
    const int w = cd.dmul * D + cd.dadd;
    return (D != 0 && (cd.frac > 0.f ? w >= 0 : w > 0)) ? w : -1;
}

// Depth in metres (0 when missing).
template <int DT>
__device__ __forceinline__ float load_depth(const void* base, size_t idx, const Codec& cd) {
    const float raw = load_raw<DT>(base, idx);
    if (DT == SF_DEPTH_F32) return raw;
    if (DT == SF_DEPTH_U16) return raw != 0.f ? raw * cd.scale : 0.f;
    const int w = disparity_units(raw, cd);
    return w >= 0 ? 1.f / (cd.scale * ((float)w + cd.frac)) : 0.f;
}

__device__ __forceinline__ bool depth_valid(float z) { return z > 0.f && z < INFINITY; }

// The variable summed by each method, before fixed-point scaling:
//   disparity 1/Z (float32 depth), 1/raw (uint16 depth; the metric scale is
//   folded into the quantum) or w (disparity input); standard Z (float32 or
//   disparity input) or raw (uint16).
template <int DT, int M>
__device__ __forceinline__ float fit_variable_of(float zin, const Codec& cd = Codec{1.f, 0, 0}) {
    if (DT == SF_DEPTH_DISPARITY_U16) {
        const int w = disparity_units(zin, cd);
        if (base_method(M) == SF_METHOD_DISPARITY) return (float)w;
        return w >= 0 ? 1.f / (cd.scale * ((float)w + cd.frac)) : 0.f;
    }
    if (base_method(M) == SF_METHOD_DISPARITY) return rcp_approx(zin);
    return zin;
}

// round(sc / z) to the nearest integer for sc = 2^e, without the 24-bit limit
// of a float32 reciprocal: y = rcp(z) is refined by the exact FMA residual
// e = 1 - z*y (exact in float32 for |e| <= 2^-22), so 1/z = y + y*e to about
// 2^-44; the integer is assembled from the two parts without re-rounding.
__device__ __forceinline__ int quant_recip(float z, float sc) {
    const float y = rcp_approx(z);
    const float e = fmaf(-z, y, 1.f);
    const float hi = y * sc;           // exact: power-of-two scaling
    const float lo = (y * e) * sc;
    const float hr = rintf(hi);
    return (int)hr + (int)rintf((hi - hr) + lo);
}

// round(K / (w + f)) for an integer 0 <= w < 2^24, f in [0, 1), w + f > 0 and
// any K > 0 with K / (w + f) < 2^30: y = rcp(w + f) refined by its residual
// e = 1 - (w + f) y (exact FMA for w, f y to float32 of a quantity below
// 2^-23 relative), and K y split exactly into p + pe (FMA), so
// K / (w + f) = p + pe + p e to about 2^-44 relative.
__device__ __forceinline__ int quant_div(float K, int w, float f = 0.f) {
    const float wf = (float)w;
    const float y = rcp_approx(wf + f);
    const float e = fmaf(-wf, y, 1.f) - f * y;
    const float p = K * y;
    const float pe = fmaf(K, y, -p);
    const float hr = rintf(p);
    return (int)hr + (int)rintf((p - hr) + fmaf(p, e, pe));
}

// Exponent e such that v * 2^e <= 2^bits for all v <= vmax.
__device__ __forceinline__ int quant_exponent(unsigned vmax_bits, int bits) {
    const float vmax = __uint_as_float(vmax_bits);
    if (!(vmax > 0.f)) return 0;
    int E;
    frexpf(vmax, &E);
    return bits - E;
}

// Fixed-point value of a valid pixel (>= 0), or -1 for a missing one, from
// its raw stored value.  Disparity input needs no reciprocal for the
// disparity form: its integer w is the fixed-point value itself.
template <int DT, int M>
__device__ __forceinline__ int quantize_raw(float zin, float sc, const Codec& cd) {
    if (DT == SF_DEPTH_DISPARITY_U16) {
        const int w = disparity_units(zin, cd);
        if (base_method(M) == SF_METHOD_DISPARITY || w < 0) return w;
        // Z / quantum = (sc / scale) / (w + frac), correctly rounded for the
        // frame's one K = sc / scale (its own rounding scales every depth alike)
        return quant_div(sc / cd.scale, w, cd.frac);
    }
    if (!depth_valid(zin)) return -1;
    if (DT == SF_DEPTH_U16 && base_method(M) == SF_METHOD_STANDARD) return (int)zin;
    if (base_method(M) == SF_METHOD_DISPARITY) return quant_recip(zin, sc);
    return __float2int_rn(zin * sc);
}

template <int DT, int M>
__device__ __forceinline__ int quantize(const void* depth, size_t idx, float sc, const Codec& cd) {
    return quantize_raw<DT, M>(load_raw<DT>(depth, idx), sc, cd);
}

// The quantum is fixed by the input (no range pass) for uint16 depth in the
// standard form and for disparity input in the disparity form.
template <int DT, int M>
__host__ __device__ constexpr bool fixed_quantum() {
    return (DT == SF_DEPTH_U16 && base_method(M) == SF_METHOD_STANDARD) ||
           (DT == SF_DEPTH_DISPARITY_U16 && base_method(M) == SF_METHOD_DISPARITY);
}

// Metric size of one fixed-point unit.
template <int DT, int M>
__device__ __forceinline__ float quantum(unsigned vmax_bits, int bits, const Codec& cd) {
    if (DT == SF_DEPTH_U16 && base_method(M) == SF_METHOD_STANDARD) return cd.scale;
    if (DT == SF_DEPTH_DISPARITY_U16 && base_method(M) == SF_METHOD_DISPARITY) return cd.scale;
    const float q = ldexpf(1.f, -quant_exponent(vmax_bits, bits));
    if (DT == SF_DEPTH_U16 && base_method(M) == SF_METHOD_DISPARITY) return q / cd.scale;
    return q;
}

// ---------------------------------------------------------------------------
// 1. range
// ---------------------------------------------------------------------------
// Raw stored values of one 16-byte vector: 4 float32 or 8 uint16 values.
template <int DT>
struct RawVec {
    static constexpr int kN = DT == SF_DEPTH_F32 ? 4 : 8;
    __device__ static __forceinline__ float get(const uint4& v, int e) {
        const unsigned w = e < kN / 4 ? v.x : e < kN / 2 ? v.y : e < 3 * kN / 4 ? v.z : v.w;
        if (DT == SF_DEPTH_F32) return __uint_as_float(w);
        return (float)((e & 1) ? (w >> 16) : (w & 0xffffu));
    }
};

template <int DT, int M>
__device__ __forceinline__ float range_update(float vmax, float z, const Codec& cd) {
    return depth_valid(z) ? fmaxf(vmax, fit_variable_of<DT, M>(z, cd)) : vmax;
}

// Largest fit variable of each frame (blockIdx.y).  The frame is read as
// 16-byte vectors, two in flight per thread (8 resident 256-thread blocks
// per SM fit in 32 registers) (issue is in order: a load
// consumed right away would expose its whole latency); the elements before
// the first 16-byte boundary and after the last whole vector are read singly.
template <int DT, int M>
__global__ void __launch_bounds__(256, 8) range_kernel(const void* __restrict__ depth, size_t frame_elems, Codec scale,
                                                    unsigned* __restrict__ vmax_bits) {
    constexpr size_t kES = DT == SF_DEPTH_F32 ? 4 : 2;
    constexpr int kN = RawVec<DT>::kN;
    const int f = blockIdx.y;
    const char* fb = static_cast<const char*>(depth) + kES * (size_t)f * frame_elems;
    const size_t head = min(frame_elems, (size_t)((16u - ((uintptr_t)fb & 15u)) & 15u) / kES);
    const size_t nvec = (frame_elems - head) / kN;
    const size_t tail = head + nvec * kN;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    float vmax = 0.f;
    if (tid < head) vmax = range_update<DT, M>(vmax, load_raw<DT>(fb, tid), scale);
    if (tid < frame_elems - tail) vmax = range_update<DT, M>(vmax, load_raw<DT>(fb, tail + tid), scale);
    const uint4* vb = reinterpret_cast<const uint4*>(fb + kES * head);
    for (size_t i0 = tid; i0 < nvec; i0 += 2 * stride) {
        uint4 v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const size_t i = i0 + u * stride;
            v[u] = i < nvec ? __ldg(vb + i) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int e = 0; e < kN; ++e) vmax = range_update<DT, M>(vmax, RawVec<DT>::get(v[u], e), scale);
    }
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    __shared__ float red[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = vmax;
    __syncthreads();
    if (warp == 0) {
        vmax = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        if (lane == 0 && vmax > 0.f) atomicMax(vmax_bits + f, __float_as_uint(vmax));
    }
}

// ---------------------------------------------------------------------------
// Scratch layout of the horizontal moments.  Each frame's block of a plane
// holds Wp x H entries (Wp = W rounded up to 64) interleaved in groups of 8
// columns: entry (x, y) sits at pofs + (x / 8) * 8H + 8y + x % 8.  The
// horizontal pass (one thread per row) then writes 32 rows of a group as one
// contiguous run, and the vertical pass (one thread per column) still reads
// whole 32-byte sectors: consecutive columns of a row are adjacent.
// ---------------------------------------------------------------------------
// Disparity planes, each a block of n_frames * plane_elems entries, in order:
//   hm int32 packed mask moments: count | (sum j + 512) << 6 | sum j^2 << 16
//   g0 int32 sum w,  g1 int32 low 32 bits of sum w j (high part in hm),
//   q0 int64 sum w^2
// Standard planes:
//   hc int32 count, z0 int64 sum z, z1 int64 sum z j,
//   b0 int64 sum z^2, b1 int64 sum z^2 j, b2 int64 sum z^2 j^2
// Frame f of a call occupies elements [pofs_f, pofs_f + Wp_f * H_f) of every
// plane; `stride` is the number of elements in one plane (all frames).
constexpr int kGroup = 8;  // columns per interleaved group; also the row stride inside a group

__device__ __forceinline__ size_t plane_index(size_t pofs, int x, int y, int H) {
    return pofs + (size_t)(x >> 3) * ((size_t)H << 3) + ((size_t)y << 3) + (size_t)(x & 7);
}

// n32 int32 planes (the disparity form: mask, sum w, sum w j -- every row sum
// of these fits 31 bits by the choice of fixed-point bits) then the int64
// planes (the disparity form: sum w^2; the standard form: 1 int32 + 5 int64).
template <int M>
__host__ __device__ constexpr int planes32() { return base_method(M) == SF_METHOD_DISPARITY ? 3 : 1; }

// Bounds-checked build (SF_CHECK_BOUNDS=1): every access of a moment plane
// checks its index against the plane's length; one out of range is skipped
// (a load reads 0) and the first one is recorded in this translation unit's
// bounds word -- bit 63, the access site in bits 56-62, the index below --
// which the library's entry points read after the work and report.
#ifndef SF_CHECK_BOUNDS
#define SF_CHECK_BOUNDS 0
#endif
static __device__ unsigned long long sf_bounds_word;
enum BoundsSite : int { kSiteColumnLoad = 1, kSiteRowStore = 2 };
__device__ __forceinline__ bool plane_index_ok(size_t o, size_t limit, int site) {
    if (!SF_CHECK_BOUNDS || o < limit) return true;
    atomicCAS(&sf_bounds_word, 0ull, (1ull << 63) | ((unsigned long long)site << 56) | (o & ((1ull << 56) - 1)));
    return false;
}

struct Planes {
    int32_t* p32;       // first int32 plane (the packed mask); plane c is p32 + c * stride
    int64_t* p64;       // first int64 plane; plane c is p64 + c * stride
    size_t stride;
    __host__ __device__ Planes(void* base, size_t stride_, int n32)
        : p32(reinterpret_cast<int32_t*>(base)),
          p64(reinterpret_cast<int64_t*>(reinterpret_cast<int32_t*>(base) + (size_t)n32 * stride_)),
          stride(stride_) {}
    __device__ __forceinline__ int32_t* c32(int c) const { return p32 + (size_t)c * stride; }
    __device__ __forceinline__ int64_t* c64(int c) const { return p64 + (size_t)c * stride; }
};

// Packed per-row word: count (bits 0-4, <= 31), sum j + 512 (bits 5-14), sum
// j^2 (bits 15-26, <= 2480 for r <= 15) and, for the disparity form, the high
// part hi (bits 27-31, signed) of the row sum of w j, whose low 32 bits are
// stored in their own plane: sum w j = hi 2^32 + (uint32) lo (|sum w j| <
// 2^34 by the choice of fixed-point bits).  A row without valid pixels has
// the word kEmptyMask, never 0 (0 marks a row outside the image).
__device__ __forceinline__ int32_t pack_mask(int h0, int h1, int h2, int hi = 0) {
    return (int32_t)((uint32_t)h0 | ((uint32_t)(h1 + 512) << 5) | ((uint32_t)h2 << 15) | ((uint32_t)hi << 27));
}
// the packed mask moments of a row without valid pixels (every field zero)
constexpr int32_t kEmptyMask = 512 << 5;
__device__ __forceinline__ void unpack_mask(int32_t v, int& h0, int& h1, int& h2) {
    h0 = v & 31;
    h1 = ((v >> 5) & 1023) - 512;
    h2 = (v >> 15) & 4095;
}
__device__ __forceinline__ int mask_hi(int32_t v) { return v >> 27; }
__device__ __forceinline__ int32_t lo32(int64_t v) { return (int32_t)(uint32_t)((uint64_t)v & 0xffffffffull); }
// the row sum of w j from its high part (in the packed word) and low 32 bits
__device__ __forceinline__ int64_t join_wj(int32_t word, int32_t lo) {
    return ((int64_t)mask_hi(word) << 32) + (int64_t)(uint32_t)lo;
}

// Running sums of c, c*j, c*j^2 over j in [-r, r] slide by one column with
//   S0' = S0 - out + in
//   S1' = S1 + r*out + (r+1)*in - S0'
//   S2' = S2 - r(r+2)*out + (r+1)(r-1)*in - 2*S1 + S0'
// (out leaves at j = -r, in enters at j = r + 1; S1 on the right is the old one).
template <typename T>
__device__ __forceinline__ void slide3(T& S0, T& S1, T& S2, T out, T in, int r) {
    // exact for integers, and for float32 while every value stays below 2^24
    const T n0 = S0 - out + in;
    const T n1 = S1 + (T)r * out + (T)(r + 1) * in - n0;
    const T n2 = S2 - (T)(r * (r + 2)) * out + (T)((r + 1) * (r - 1)) * in - 2 * S1 + n0;
    S0 = n0; S1 = n1; S2 = n2;
}
template <typename T>
__device__ __forceinline__ void slide2(T& S0, T& S1, T out, T in, int r) {
    const T n0 = S0 - out + in;
    S1 = S1 + (T)r * out + (T)(r + 1) * in - n0;
    S0 = n0;
}

// ---------------------------------------------------------------------------
// 2. hpass: block = 128 rows x 64 output columns, tile of fixed-point values
//    staged in shared memory with coalesced loads, one thread per row.
// ---------------------------------------------------------------------------
// Load and quantise the raw depth of a horizontal tile into shared memory:
// rows [y0, y0 + rows), columns [x0 - r, x0 - r + IW), at row pitch `pitch`.
// Warp w takes rows w, w + 4, ...; lanes sweep a row (coalesced).
// kRowsPerBatch rows x CHUNKS 32-column chunks are loaded before any is used,
// so that many loads per thread are in flight at once (issue is in order: a
// load consumed right away would expose its whole latency).
template <int DT, int M, int CHUNKS, int kRowsPerBatch = 8>
__device__ __forceinline__ void load_tile(const void* __restrict__ depth, int W, int r, float sc, const Codec& cd,
                                          int x0, int y0, int rows, int IW, int pitch, int* tile) {
    constexpr int kWarps = kHThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int rb = warp; rb < rows; rb += kWarps * kRowsPerBatch) {
        float raw[kRowsPerBatch][CHUNKS];
#pragma unroll
        for (int k = 0; k < kRowsPerBatch; ++k) {
            const int ry = rb + k * kWarps;
#pragma unroll
            for (int c = 0; c < CHUNKS; ++c) {
                const int cx = lane + 32 * c, x = x0 - r + cx;
                raw[k][c] = (ry < rows && cx < IW && x >= 0 && x < W)
                                ? load_raw<DT>(depth, (size_t)(y0 + ry) * W + x) : 0.f;
            }
        }
#pragma unroll
        for (int k = 0; k < kRowsPerBatch; ++k) {
            const int ry = rb + k * kWarps;
#pragma unroll
            for (int c = 0; c < CHUNKS; ++c) {
                const int cx = lane + 32 * c;
                if (ry < rows && cx < IW) tile[ry * pitch + cx] = quantize_raw<DT, M>(raw[k][c], sc, cd);
            }
        }
    }
}

// load_tile for tiles at most 16 columns wide: the two halves of a warp take
// two rows at once (lanes 0-15 and 16-31), so that each lane loads and
// quantises 16 values instead of 32 with half its lanes idle.  Warp w still
// fills rows w, w + 4, ..., w + 124, with the same values as load_tile.
template <int DT, int M>
__device__ __forceinline__ void load_tile_pairs(const void* __restrict__ depth, int W, int r, float sc,
                                                const Codec& cd, int x0, int y0, int rows, int IW, int pitch,
                                                int* tile) {
    constexpr int kWarps = kHThreads / 32;
    constexpr int kPerLane = kHThreads / (2 * kWarps);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = lane >> 4, cx = lane & 15, x = x0 - r + cx;
    const bool col = cx < IW && x >= 0 && x < W;
    float raw[kPerLane];
#pragma unroll
    for (int k = 0; k < kPerLane; ++k) {
        const int ry = warp + kWarps * (2 * k + half);
        raw[k] = (ry < rows && col) ? load_raw<DT>(depth, (size_t)(y0 + ry) * W + x) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kPerLane; ++k) {
        const int ry = warp + kWarps * (2 * k + half);
        if (ry < rows && cx < IW) tile[ry * pitch + cx] = quantize_raw<DT, M>(raw[k], sc, cd);
    }
}

// Running horizontal sums of one row over one 32-column output segment:
// mask moments (count, sum j, sum j^2) and value moments.  The disparity
// form's row sum of v fits 31 bits (the fixed-point bits are chosen so): it
// slides in 32-bit unsigned arithmetic, exact modulo 2^32, which the stored
// int32 value is; its row sum of v j is exact in 64 bits and stored split
// (low 32 bits in a plane, the high part in the packed mask word).
template <int M>
struct HRowState {
    using Acc = typename std::conditional<base_method(M) == SF_METHOD_DISPARITY, uint32_t, int64_t>::type;
    int h0 = 0, h1 = 0, h2 = 0;
    Acc a0 = 0;                      // sum v
    int64_t a1 = 0;                  // sum v j
    int64_t s0 = 0, s1 = 0, s2 = 0;  // sum v^2, sum v^2 j, sum v^2 j^2 (s1, s2: standard only)
    // window of output column x0: tile columns x0 - xt .. x0 - xt + 2r
    __device__ __forceinline__ void init(const int* row, int c0, int r) {
        for (int j = -r; j <= r; ++j) {
            const int v = row[c0 + j + r];
            if (v >= 0) {
                const int64_t vv = (int64_t)v * v;
                h0 += 1; h1 += j; h2 += j * j;
                a0 += (Acc)v; a1 += (int64_t)v * j;
                s0 += vv;
                if (base_method(M) == SF_METHOD_STANDARD) { s1 += vv * j; s2 += vv * (j * j); }
            }
        }
    }
    // slide from output column c to c + 1 (tile-relative c)
    __device__ __forceinline__ void step(const int* row, int c, int r) {
        const int vo = row[c];              // column x - r leaves
        const int vi = row[c + 2 * r + 1];  // column x + r + 1 enters
        const int mo = vo >= 0, mi = vi >= 0;
        slide3(h0, h1, h2, mo, mi, r);
        const int64_t co = mo ? vo : 0, ci = mi ? vi : 0;
        a0 = a0 - (Acc)co + (Acc)ci;
        a1 = a1 + (int64_t)r * co + (int64_t)(r + 1) * ci - (int64_t)a0;
        const int64_t qo = co * co, qi = ci * ci;
        if (base_method(M) == SF_METHOD_STANDARD) slide3(s0, s1, s2, qo, qi, r);
        else s0 = s0 - qo + qi;
    }
};

// One row of a tile: L independent kSub-column output segments [x0 + kSub l,
// x0 + kSub (l + 1)) clipped to xend, slid in lock step (L independent
// dependency chains per thread), four columns per store.  kSub is 32, or 16
// or 8 for small frames (more threads, shorter serial chains).
template <int M, int L, int kSub = 32>
__device__ __forceinline__ void hpass_row(const int* row, int x0, int xend, int y, int H, int r, const Planes& P,
                                          size_t pofs) {
    static_assert(kSub % 4 == 0 && (L == 1 || kSub == 32), "L segments of 32 columns, or one of kSub");
    HRowState<M> st[L];
#pragma unroll
    for (int l = 0; l < L; ++l)
        if (x0 + l * kSub < xend) st[l].init(row, l * kSub, r);
    for (int xb = 0; xb < kSub; xb += 4) {
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const int xs = x0 + l * kSub + xb;  // first of the four columns
            const int xe = min(x0 + (l + 1) * kSub, xend);
            if (xs >= xe) continue;
            int32_t hmv[4];
            typename HRowState<M>::Acc c0v[4];
            int64_t c1v[4], c2v[4], c3v[4], c4v[4];
            HRowState<M>& S = st[l];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                hmv[u] = pack_mask(S.h0, S.h1, S.h2,
                                   base_method(M) == SF_METHOD_DISPARITY ? (int)(S.a1 >> 32) : 0);
                c0v[u] = S.a0; c1v[u] = S.a1; c2v[u] = S.s0; c3v[u] = S.s1; c4v[u] = S.s2;
                if (xs + u + 1 < xe) S.step(row, xs + u - x0, r);
            }
            const size_t o = plane_index(pofs, xs, y, H);  // xs % 4 == 0: 4 entries in one group
            if (!plane_index_ok(o + 3, P.stride, kSiteRowStore)) continue;
            if (base_method(M) == SF_METHOD_DISPARITY) {
                if (xs + 4 <= xe) {
                    *reinterpret_cast<int4*>(P.p32 + o) = make_int4(hmv[0], hmv[1], hmv[2], hmv[3]);
                    *reinterpret_cast<int4*>(P.c32(1) + o) =
                        make_int4((int)c0v[0], (int)c0v[1], (int)c0v[2], (int)c0v[3]);
                    *reinterpret_cast<int4*>(P.c32(2) + o) = make_int4(lo32(c1v[0]), lo32(c1v[1]), lo32(c1v[2]),
                                                                       lo32(c1v[3]));
                    int64_t* q0 = P.c64(0) + o;
                    *reinterpret_cast<longlong2*>(q0) = make_longlong2(c2v[0], c2v[1]);
                    *reinterpret_cast<longlong2*>(q0 + 2) = make_longlong2(c2v[2], c2v[3]);
                } else {
                    for (int u = 0; u < 4 && xs + u < xe; ++u) {
                        P.p32[o + u] = hmv[u];
                        P.c32(1)[o + u] = (int)c0v[u]; P.c32(2)[o + u] = lo32(c1v[u]);
                        P.c64(0)[o + u] = c2v[u];
                    }
                }
            } else if (xs + 4 <= xe) {
                *reinterpret_cast<int4*>(P.p32 + o) = make_int4(hmv[0], hmv[1], hmv[2], hmv[3]);
                int64_t* c0 = P.c64(0) + o;
                int64_t* c1 = P.c64(1) + o;
                int64_t* c2 = P.c64(2) + o;
                int64_t* c3 = P.c64(3) + o;
                int64_t* c4 = P.c64(4) + o;
                *reinterpret_cast<longlong2*>(c0) = make_longlong2(c0v[0], c0v[1]);
                *reinterpret_cast<longlong2*>(c0 + 2) = make_longlong2(c0v[2], c0v[3]);
                *reinterpret_cast<longlong2*>(c1) = make_longlong2(c1v[0], c1v[1]);
                *reinterpret_cast<longlong2*>(c1 + 2) = make_longlong2(c1v[2], c1v[3]);
                *reinterpret_cast<longlong2*>(c2) = make_longlong2(c2v[0], c2v[1]);
                *reinterpret_cast<longlong2*>(c2 + 2) = make_longlong2(c2v[2], c2v[3]);
                *reinterpret_cast<longlong2*>(c3) = make_longlong2(c3v[0], c3v[1]);
                *reinterpret_cast<longlong2*>(c3 + 2) = make_longlong2(c3v[2], c3v[3]);
                *reinterpret_cast<longlong2*>(c4) = make_longlong2(c4v[0], c4v[1]);
                *reinterpret_cast<longlong2*>(c4 + 2) = make_longlong2(c4v[2], c4v[3]);
            } else {
                for (int u = 0; u < 4 && xs + u < xe; ++u) {
                    P.p32[o + u] = hmv[u];
                    P.c64(0)[o + u] = c0v[u]; P.c64(1)[o + u] = c1v[u]; P.c64(2)[o + u] = c2v[u];
                    P.c64(3)[o + u] = c3v[u]; P.c64(4)[o + u] = c4v[u];
                }
            }
        }
    }
}

// Horizontal moments of one tile: rows [y0, y0 + 128) x output columns
// [x0, x0 + kSub L) of one frame.  `depth` points at the frame, `pofs` is the
// frame's offset in the planes; `tile` is shared memory of
// kHThreads * ((kSub L + 2r) | 1) ints.
template <int DT, int M, int L, int kSub = 32>
__device__ __forceinline__ void hpass_tile(const void* __restrict__ depth, int W, int H, int r, float sc,
                                           const Codec& cd, const Planes& P, size_t pofs, int x0, int y0,
                                           int* tile) {
    constexpr int seg = kSub * L;
    const int IW = seg + 2 * r;
    const int pitch = IW | 1;  // odd pitch: the 32 rows of a warp hit 32 banks
    const int rows = min(kHThreads, H - y0);
    // the tile's raw depth, quantised; ceil(IW / 32) column chunks per row
    // (IW <= seg + 2 kMaxR): 2 for seg 8 to 32, 3 for 48 and 64, 5 for 128.
    // The narrow segments of small calls with small windows (IW <= 32) take
    // each warp's 32 rows in one batch: one memory round trip instead of four;
    // tiles at most 16 wide take two rows per warp instruction
    if constexpr (kSub <= 16) {
        if (IW <= 16) load_tile_pairs<DT, M>(depth, W, r, sc, cd, x0, y0, rows, IW, pitch, tile);
        else if (IW <= 32) load_tile<DT, M, 1, 32>(depth, W, r, sc, cd, x0, y0, rows, IW, pitch, tile);
        else load_tile<DT, M, 2>(depth, W, r, sc, cd, x0, y0, rows, IW, pitch, tile);
    } else {
        load_tile<DT, M, (seg + 2 * kMaxR + 31) / 32>(depth, W, r, sc, cd, x0, y0, rows, IW, pitch, tile);
    }
    __syncthreads();
    if ((int)threadIdx.x < rows)
        hpass_row<M, L, kSub>(tile + threadIdx.x * pitch, x0, min(x0 + seg, W), y0 + threadIdx.x, H, r, P, pofs);
}

// Resident blocks per SM of the horizontal pass for 32 L-column tiles (shared
// memory: 32 KB, 48 KB, 80 KB per block at r = 15), which caps the registers
// (6 for the standard form's 32-column tiles: its int64 sums need more).
template <int M, int L>
__host__ __device__ constexpr int hpass_blocks() {
    return L == 1 ? (base_method(M) == SF_METHOD_STANDARD ? 6 : 7) : (L == 2 ? 4 : 2);
}

template <int DT, int M, int L, int kSub = 32>
__global__ void __launch_bounds__(kHThreads, hpass_blocks<M, L>()) hpass_kernel(
    const void* __restrict__ depth, int W, int H, int r, Codec scale, const unsigned* __restrict__ vmax_bits, int bits,
    int raw_z, int Wp, size_t plane_elems, void* planes_base) {
    extern __shared__ int tile[];
    wait_for_prior_grid();  // the range pass's maximum
    const int f = blockIdx.z;
    const float sc = ldexpf(1.f, quant_exponent(vmax_bits[f], bits));  // 2^e, exact
    const size_t dbytes = (DT == SF_DEPTH_F32) ? 4 : 2;
    const void* dframe = static_cast<const char*>(depth) + dbytes * (size_t)f * W * H;
    const Planes P(planes_base, (size_t)gridDim.z * plane_elems, planes32<M>());
    hpass_tile<DT, M, L, kSub>(dframe, W, H, r, sc, scale, P, (size_t)f * plane_elems, blockIdx.x * kSub * L,
                               blockIdx.y * kHThreads, tile);
}

// ---------------------------------------------------------------------------
// 3. vpass + solve: one thread per column, band of `band` output rows.
// ---------------------------------------------------------------------------
struct Calib {
    const float* tx;  // [W] ray tangent per column
    const float* ty;  // [H] ray tangent per row
    float a, b;       // 1/fx, 1/fy
};

// Load of a horizontal-moment plane entry (entry o of a plane of `limit`
// entries): through the read-only cache, or (kCoh) coherently from L2, for a
// kernel that also writes the planes (the merged batch kernel, whose column
// items read what its tile items wrote).
template <bool kCoh, typename T>
__device__ __forceinline__ T load_plane(const T* base, size_t o, size_t limit) {
    if (!plane_index_ok(o, limit, kSiteColumnLoad)) return T(0);
    if constexpr (kCoh) return __ldcg(base + o);
    else return __ldg(base + o);
}

// Vertical running sums of the disparity form's moments for one column.
template <bool kCoh = false>
struct DispStateT {
    const int32_t* hm; const int32_t* g0; const int32_t* g1; const int64_t* q0;
    // mask moments: exact small integers, kept in float32 (all < 2^24)
    float n = 0.f, Sj = 0.f, Sjj = 0.f, Si = 0.f, Sji = 0.f, Sii = 0.f;
    int64_t Sw = 0, Swj = 0, Swi = 0, Sww = 0;
    size_t lim;  // entries per plane
    __device__ DispStateT(const Planes& P)
        : hm(P.p32), g0(P.c32(1)), g1(P.c32(2)), q0(P.c64(0)), lim(P.stride) {}
    // window of output row y0 from rows y0 - r .. y0 + r (clipped to the
    // image), in batches of kInitRows rows whose loads are all issued before
    // any is used; rows past the end of a batch read as empty
    static constexpr int kInitRows = 8;
    __device__ __forceinline__ void init(size_t pb, int rs, int H, int y0, int r) {
        const int ylo = max(y0 - r, 0), yhi = min(y0 + r, H - 1);
        for (int yb = ylo; yb <= yhi; yb += kInitRows) {
            int32_t hv[kInitRows], av[kInitRows], bv[kInitRows];
            int64_t qv[kInitRows];
#pragma unroll
            for (int u = 0; u < kInitRows; ++u) {
                hv[u] = kEmptyMask; av[u] = 0; bv[u] = 0; qv[u] = 0;
                if (yb + u <= yhi) {
                    const size_t o = pb + (size_t)(yb + u) * rs;
                    hv[u] = load_plane<kCoh>(hm, o, lim); av[u] = load_plane<kCoh>(g0, o, lim);
                    bv[u] = load_plane<kCoh>(g1, o, lim); qv[u] = load_plane<kCoh>(q0, o, lim);
                }
            }
#pragma unroll
            for (int u = 0; u < kInitRows; ++u) {
                const int i = yb + u - y0;
                int c0, c1, c2;
                unpack_mask(hv[u], c0, c1, c2);
                const float f0 = (float)c0, f1 = (float)c1, fi = (float)i;
                n += f0; Sj += f1; Sjj += (float)c2; Si += fi * f0; Sji += fi * f1; Sii += fi * fi * f0;
                Sw += av[u]; Swj += join_wj(hv[u], bv[u]); Swi += (int64_t)i * av[u]; Sww += qv[u];
            }
        }
    }
    // The two horizontal-moment rows of the slide from output row y to y + 1
    // (leaving row y - r, entering row y + r + 1; zero outside the image).
    // fetch() only issues the loads, so a caller can overlap them with the
    // solve of row y and apply() them afterwards; fetch_rows / apply_rows do
    // the same with a caller-held buffer (several slides in flight).
    struct Rows {
        int32_t m_o = 0, m_i = 0, w_o = 0, w_i = 0, wj_o = 0, wj_i = 0;
        int64_t ww_o = 0, ww_i = 0;
    };
    Rows pend;
    __device__ __forceinline__ void fetch_rows(Rows& R, size_t pb, int rs, int H, int y, int r) const {
        const int yo = y - r, yi = y + r + 1;
        R = Rows();
        if (yo >= 0) {
            const size_t o = pb + (size_t)yo * rs;
            R.m_o = load_plane<kCoh>(hm, o, lim); R.w_o = load_plane<kCoh>(g0, o, lim);
            R.wj_o = load_plane<kCoh>(g1, o, lim); R.ww_o = load_plane<kCoh>(q0, o, lim);
        }
        if (yi < H) {
            const size_t o = pb + (size_t)yi * rs;
            R.m_i = load_plane<kCoh>(hm, o, lim); R.w_i = load_plane<kCoh>(g0, o, lim);
            R.wj_i = load_plane<kCoh>(g1, o, lim); R.ww_i = load_plane<kCoh>(q0, o, lim);
        }
    }
    __device__ __forceinline__ void apply_rows(const Rows& R, int r) {
        int o0 = 0, o1 = 0, o2 = 0, i0 = 0, i1 = 0, i2 = 0;
        if (R.m_o) unpack_mask(R.m_o, o0, o1, o2);
        if (R.m_i) unpack_mask(R.m_i, i0, i1, i2);
        // vertical moments: (n, Si, Sii) from the counts, (Sj, Sji) from sum j, Sjj plain
        slide3(n, Si, Sii, (float)o0, (float)i0, r);
        slide2(Sj, Sji, (float)o1, (float)i1, r);
        Sjj += (float)(i2 - o2);
        slide2(Sw, Swi, (int64_t)R.w_o, (int64_t)R.w_i, r);
        Swj += join_wj(R.m_i, R.wj_i) - join_wj(R.m_o, R.wj_o);
        Sww += R.ww_i - R.ww_o;
    }
    __device__ __forceinline__ void fetch(size_t pb, int rs, int H, int y, int r) { fetch_rows(pend, pb, rs, H, y, r); }
    __device__ __forceinline__ void apply(int r) { apply_rows(pend, r); }
    // slide from output row y to y + 1
    __device__ __forceinline__ void slide(size_t pb, int rs, int H, int y, int r) {
        fetch(pb, rs, H, y, r);
        apply(r);
    }
    __device__ __forceinline__ int count() const { return (int)n; }
};
using DispState = DispStateT<false>;

// Vertical running sums of the standard form's moments for one column.  With
// kMask the image moments of the valid pixels (sum j, j^2, i, ji, i^2) are
// kept too: the explicit standard fit needs them for its rank test.
template <bool kMask = false, bool kCoh = false>
struct StdStateT {
    const int32_t* hc; const int64_t* z0; const int64_t* z1; const int64_t* b0; const int64_t* b1; const int64_t* b2;
    int n = 0;
    float fn = 0.f, Sj = 0.f, Sjj = 0.f, Si = 0.f, Sji = 0.f, Sii = 0.f;  // kMask only
    int64_t Sz = 0, Szi = 0, Szj = 0, Szz = 0, Szzi = 0, Szzii = 0, Szzj = 0, Szzji = 0, Szzjj = 0;
    size_t lim;  // entries per plane
    __device__ StdStateT(const Planes& P)
        : hc(P.p32), z0(P.c64(0)), z1(P.c64(1)), b0(P.c64(2)), b1(P.c64(3)), b2(P.c64(4)), lim(P.stride) {}
    // as DispState::init, in batches of kInitRows rows
    static constexpr int kInitRows = 4;
    __device__ __forceinline__ void init(size_t pb, int rs, int H, int y0, int r) {
        const int ylo = max(y0 - r, 0), yhi = min(y0 + r, H - 1);
        for (int yb = ylo; yb <= yhi; yb += kInitRows) {
            int32_t hv[kInitRows];
            int64_t zv[kInitRows], zjv[kInitRows], q0v[kInitRows], q1v[kInitRows], q2v[kInitRows];
#pragma unroll
            for (int u = 0; u < kInitRows; ++u) {
                hv[u] = kEmptyMask; zv[u] = zjv[u] = q0v[u] = q1v[u] = q2v[u] = 0;
                if (yb + u <= yhi) {
                    const size_t o = pb + (size_t)(yb + u) * rs;
                    hv[u] = load_plane<kCoh>(hc, o, lim); zv[u] = load_plane<kCoh>(z0, o, lim); zjv[u] = load_plane<kCoh>(z1, o, lim);
                    q0v[u] = load_plane<kCoh>(b0, o, lim); q1v[u] = load_plane<kCoh>(b1, o, lim); q2v[u] = load_plane<kCoh>(b2, o, lim);
                }
            }
#pragma unroll
            for (int u = 0; u < kInitRows; ++u) {
                const int64_t i = yb + u - y0;
                int c0, c1, c2;
                unpack_mask(hv[u], c0, c1, c2);
                n += c0;
                if constexpr (kMask) {
                    const float fi = (float)i, f0 = (float)c0, f1 = (float)c1;
                    fn += f0; Sj += f1; Sjj += (float)c2; Si += fi * f0; Sji += fi * f1; Sii += fi * fi * f0;
                }
                Sz += zv[u]; Szi += i * zv[u]; Szj += zjv[u];
                Szz += q0v[u]; Szzi += i * q0v[u]; Szzii += i * i * q0v[u];
                Szzj += q1v[u]; Szzji += i * q1v[u]; Szzjj += q2v[u];
            }
        }
    }
    // fetch() / apply(): the slide from output row y to y + 1 split into its
    // loads and its arithmetic (as for DispState); fetch_rows / apply_rows
    // with a caller-held buffer.
    struct Rows {
        int32_t m_o = 0, m_i = 0;
        int64_t zo = 0, zjo = 0, qo0 = 0, qo1 = 0, qo2 = 0, zi = 0, zji = 0, qi0 = 0, qi1 = 0, qi2 = 0;
    };
    Rows pend;
    __device__ __forceinline__ void fetch_rows(Rows& R, size_t pb, int rs, int H, int y, int r) const {
        const int yo = y - r, yi = y + r + 1;
        R = Rows();
        if (yo >= 0) {
            const size_t o = pb + (size_t)yo * rs;
            R.m_o = load_plane<kCoh>(hc, o, lim); R.zo = load_plane<kCoh>(z0, o, lim); R.zjo = load_plane<kCoh>(z1, o, lim);
            R.qo0 = load_plane<kCoh>(b0, o, lim); R.qo1 = load_plane<kCoh>(b1, o, lim); R.qo2 = load_plane<kCoh>(b2, o, lim);
        }
        if (yi < H) {
            const size_t o = pb + (size_t)yi * rs;
            R.m_i = load_plane<kCoh>(hc, o, lim); R.zi = load_plane<kCoh>(z0, o, lim); R.zji = load_plane<kCoh>(z1, o, lim);
            R.qi0 = load_plane<kCoh>(b0, o, lim); R.qi1 = load_plane<kCoh>(b1, o, lim); R.qi2 = load_plane<kCoh>(b2, o, lim);
        }
    }
    __device__ __forceinline__ void apply_rows(const Rows& R, int r) {
        int o0 = 0, o1 = 0, o2 = 0, i0 = 0, i1 = 0, i2 = 0;
        if (R.m_o) unpack_mask(R.m_o, o0, o1, o2);
        if (R.m_i) unpack_mask(R.m_i, i0, i1, i2);
        n += i0 - o0;
        if constexpr (kMask) {
            slide3(fn, Si, Sii, (float)o0, (float)i0, r);
            slide2(Sj, Sji, (float)o1, (float)i1, r);
            Sjj += (float)(i2 - o2);
        }
        slide2(Sz, Szi, R.zo, R.zi, r);
        Szj += R.zji - R.zjo;
        slide3(Szz, Szzi, Szzii, R.qo0, R.qi0, r);
        slide2(Szzj, Szzji, R.qo1, R.qi1, r);
        Szzjj += R.qi2 - R.qo2;
    }
    __device__ __forceinline__ void fetch(size_t pb, int rs, int H, int y, int r) { fetch_rows(pend, pb, rs, H, y, r); }
    __device__ __forceinline__ void apply(int r) { apply_rows(pend, r); }
    __device__ __forceinline__ void slide(size_t pb, int rs, int H, int y, int r) {
        fetch(pb, rs, H, y, r);
        apply(r);
    }
    __device__ __forceinline__ int count() const { return n; }
};
using StdState = StdStateT<false>;

// Vertical moments + solve for one column x of one frame, output rows
// [y0, y0 + band).  `depth` and the output pointers point at the frame.
// Not inlined: the single-context and the batch kernels then run the same
// machine code, so their results agree bit for bit (inlined copies may be
// contracted into FMAs differently); one call covers a whole band.
template <int DT, int M, bool U4 = false, bool kGuard = false>
__device__ __noinline__ void vpass_column(const void* __restrict__ depth, int W, int H, int r, Codec scale, float q,
                                             const Planes P, size_t pofs, int x, int y0, int band,
                                             const float* __restrict__ txt, const float* __restrict__ tyt, float a,
                                             float b, int min_valid, int require_center, float* __restrict__ normals,
                                             float* __restrict__ offsets, float* __restrict__ curvature,
                                             int32_t* __restrict__ counts, float tau,
                                             unsigned long long* __restrict__ flags, unsigned* __restrict__ flag_count,
                                             int frame_tag, void* __restrict__ mq, unsigned mcap) {
    const int y1 = min(y0 + band, H);
    const size_t pb = plane_index(pofs, x, 0, H);
    const float tx = txt[x];
    constexpr int B = base_method(M);
    const float wfrac = DT == SF_DEPTH_DISPARITY_U16 ? scale.frac : 0.f;  // disparity input offset
    // the scratch is read coherently from L2 in every kernel that runs this
    // function (the batch kernel writes it in the same launch), so that all of
    // them run one compiled copy: the compiler may fuse a float32 multiply and
    // add differently in each copy of a function
    typename std::conditional<B == SF_METHOD_DISPARITY, DispStateT<true>,
                              StdStateT<M == SF_METHOD_EXPLICIT_STANDARD, true>>::type S(P);
    S.init(pb, kGroup, H, y0, r);
    // row pointers, advanced by one image row per output row
    size_t oi = (size_t)y0 * W + x;
    float* pn = normals + 3 * oi;
    float* po = offsets + oi;
    float* pc = curvature + oi;
    int32_t* pk = counts ? counts + oi : nullptr;
    float zc = load_depth<DT>(depth, oi, scale);
    float tyn = tyt[y0];
    unsigned q_next = 0, q_end = 0, q_count = 0;  // this warp's reserved queue slots, windows queued
    const unsigned act = __activemask();           // the lanes running this column loop
    for (int y = y0; y < y1; ++y) {
        const bool cvalid = depth_valid(zc);
        const float ty = tyn;
        // issue the loads of the next slide (and the next centre depth and
        // ray) now: the solve below hides their latency
        const bool more = y + 1 < y1;
        oi += W;
        if (more) {
            S.fetch(pb, kGroup, H, y, r);
            zc = load_depth<DT>(depth, oi, scale);
            tyn = tyt[y + 1];
        }
        const int n = S.count();
        bool ok = n >= min_valid && n > 0 && (cvalid || !require_center);
        float nx = NAN, ny = NAN, nz = NAN, d = NAN, cu = NAN;
        FitOut fo_;
        if (ok) {
            if constexpr (M == SF_METHOD_DISPARITY)
                fo_ = solve_disparity<float, U4, kGuard>(S.n, S.Sj, S.Si, S.Sjj, S.Sji, S.Sii, S.Sw, S.Swj, S.Swi,
                                                         S.Sww, q, tx, ty, a, b, wfrac);
            else if constexpr (M == SF_METHOD_STANDARD)
                fo_ = solve_standard<float, U4, kGuard>((float)S.n, S.Sz, S.Szj, S.Szi, S.Szz, S.Szzj, S.Szzi, S.Szzjj,
                                                        S.Szzji, S.Szzii, q, tx, ty, a, b);
            else if constexpr (M == SF_METHOD_EXPLICIT_DISPARITY)
                fo_ = solve_explicit_disparity(S.n, S.Sj, S.Si, S.Sjj, S.Sji, S.Sii, S.Sw, S.Swj, S.Swi, S.Sww, q,
                                               tx, ty, a, b, ok, wfrac);
            else
                fo_ = solve_explicit_standard((float)S.n, S.Sj, S.Si, S.Sjj, S.Sji, S.Sii, S.Sz, S.Szj, S.Szi,
                                              S.Szz, S.Szzj, S.Szzi, S.Szzjj, S.Szzji, S.Szzii, q, tx, ty, a, b,
                                              ok);
        }
        bool queue = false;
        if (ok) {
            nx = fo_.nx; ny = fo_.ny; nz = fo_.nz; d = fo_.d; cu = fo_.curv;
            // queue a near-degenerate window, and (kGuard) one whose fixed-point
            // rounding could move its normal by more than the refinement's threshold
            queue = flags && !(fo_.gap >= tau);
            if constexpr (kGuard) queue = queue || (flags && fo_.qerr2 > kRefineRounding * kRefineRounding);
        }
        if (flags) {
            // all the loop's lanes take part (the chunk state stays the same in every lane)
            const unsigned qm = __ballot_sync(act, queue);
            if (qm) {
                const unsigned k = __popc(qm), rem = q_end - q_next;
                const int leader = __ffs(act) - 1;
                unsigned s = 0;
                if (k > rem) {
                    if ((int)(threadIdx.x & 31) == leader) s = atomicAdd(flag_count, kQueueChunk);
                    s = __shfl_sync(act, s, leader);
                }
                if (queue) {
                    const int lane = threadIdx.x & 31;
                    const unsigned rank = __popc(qm & ((1u << lane) - 1u));
                    const unsigned slot = rank < rem ? q_next + rank : s + (rank - rem);
                    flags[slot] = ((unsigned long long)frame_tag << 48) | ((unsigned long long)y << 24) |
                                  (unsigned long long)x;
                    if (slot < mcap) {
                        // the window's exact moments travel with it (80 B, five 16-byte stores)
                        longlong2* e = reinterpret_cast<longlong2*>(static_cast<char*>(mq) + (size_t)slot * 80);
                        if constexpr (B == SF_METHOD_DISPARITY) {
                            e[0] = make_longlong2((long long)S.n, (long long)S.Sj);
                            e[1] = make_longlong2((long long)S.Si, (long long)S.Sjj);
                            e[2] = make_longlong2((long long)S.Sji, (long long)S.Sii);
                            e[3] = make_longlong2(S.Sw, S.Swj);
                            e[4] = make_longlong2(S.Swi, S.Sww);
                        } else {
                            e[0] = make_longlong2((long long)S.n, S.Sz);
                            e[1] = make_longlong2(S.Szj, S.Szi);
                            e[2] = make_longlong2(S.Szz, S.Szzj);
                            e[3] = make_longlong2(S.Szzi, S.Szzjj);
                            e[4] = make_longlong2(S.Szzji, S.Szzii);
                        }
                    }
                }
                if (k > rem) {
                    q_next = s + (k - rem);
                    q_end = s + kQueueChunk;
                } else {
                    q_next += k;
                }
                q_count += k;
            }
        }
        pn[0] = nx; pn[1] = ny; pn[2] = nz;
        *po = d; *pc = cu;
        if (pk) { *pk = n; pk += W; }
        pn += 3 * (size_t)W; po += W; pc += W;
        if (more) S.apply(r);
    }
    if (flags) {
        __syncwarp(act);
        if ((int)(threadIdx.x & 31) == __ffs(act) - 1) {
            for (unsigned i = q_next; i < q_end; ++i) flags[i] = kQueueHole;
            if (q_count) atomicAdd(flag_count + 2, q_count);
        }
    }
}

// kGuard: the instantiation of precision modes 1 and 2 (implicit |(a,b,c)| = 1
// fits), which also queues windows by their estimated rounding error.
// Resident blocks per SM of the column pass: 6 (80 registers), except the
// standard forms' implicit and explicit fits, whose int64 running sums spill
// there: 5 (96 registers; on the benchmark batch 3-10 % faster than 6).  The
// |(a,b,c,d)| = 1 fits, which spill at 6 as well, measured no faster at 5.
template <int M, bool U4>
__host__ __device__ constexpr int vpass_blocks() {
    return (base_method(M) == SF_METHOD_STANDARD && !U4) ? kVBlocks - 1 : kVBlocks;
}

template <int DT, int M, bool U4 = false, bool kGuard = false>
__global__ void __launch_bounds__(kVThreads, vpass_blocks<M, U4>()) vpass_kernel(const void* __restrict__ depth, int W, int H, int r,
                                                          Codec scale, const unsigned* __restrict__ vmax_bits,
                                                          int bits, int raw_z, int Wp, size_t plane_elems,
                                                          void* __restrict__ planes_base, Calib cal,
                                                          int min_valid, int require_center, int band,
                                                          float* __restrict__ normals, float* __restrict__ offsets,
                                                          float* __restrict__ curvature, int32_t* __restrict__ counts,
                                                          float tau, unsigned long long* __restrict__ flags,
                                                          unsigned* __restrict__ flag_count, void* __restrict__ mq,
                                                          unsigned mcap) {
    wait_for_prior_grid();  // the horizontal pass's scratch
    const int f = blockIdx.z;
    const int x = blockIdx.x * kVThreads + threadIdx.x;
    if (x >= W) return;
    const size_t fe = (size_t)W * H;
    const size_t dbytes = (DT == SF_DEPTH_F32) ? 4 : 2;
    const void* dframe = static_cast<const char*>(depth) + dbytes * (size_t)f * fe;
    const float q = quantum<DT, M>(vmax_bits[f], bits, scale);  // metric value of one fixed-point unit
    const Planes P(planes_base, (size_t)gridDim.z * plane_elems, planes32<M>());
    vpass_column<DT, M, U4, kGuard>(dframe, W, H, r, scale, q, P, (size_t)f * plane_elems, x, blockIdx.y * band, band, cal.tx,
                        cal.ty, cal.a, cal.b, min_valid, require_center, normals + 3 * fe * f, offsets + fe * f,
                        curvature + fe * f, counts ? counts + fe * f : nullptr, tau, flags, flag_count, f, mq,
                        mcap);
}

// ---------------------------------------------------------------------------
// Mixed-resolution batches: one persistent kernel over a table of work items.
// Each frame has its own size, window, intrinsics and tile shape.  The items
// are, in claim order, the quantum chunks of every frame, then its horizontal
// tiles, then its column bands; a CTA claims the next item with one atomicAdd.
// A tile waits until every quantum chunk of its frame is done, a band until
// every tile of its frame is: each wait is for items claimed earlier, which
// CTAs that are running hold, so the kernel cannot deadlock.  Every wait is
// bounded (a number of polls read from device memory); one that gives up sets
// the batch's error word and skips its item, so that the kernel still ends
// and the host reports SF_ERR_TIMEOUT.
// ---------------------------------------------------------------------------
struct FrameDesc {
    const void* depth;
    float* normals;
    float* offsets;
    float* curvature;
    const float* tx;   // [W] ray tangents
    const float* ty;   // [H]
    float a, b;        // 1/fx, 1/fy
    int W, H, r, bits, Wp, seg, band;
    int nr, nh;        // quantum chunks and horizontal tiles of the frame
    size_t pofs;       // offset of the frame in every moment plane
};

// Elements of a frame per quantum chunk.
constexpr int kRangeChunk = 16384;

// The batch's synchronisation words: [0] claim counter, [1] error word (bit 0:
// a tile gave up waiting for its frame's quantum, bit 1: a band gave up
// waiting for its frame's tiles), [2] polls per wait, then per frame the
// quantum bits, the finished quantum chunks and the finished tiles.
struct BatchSync {
    unsigned* w;
    int n;
    __device__ __forceinline__ unsigned* claim() const { return w; }
    __device__ __forceinline__ unsigned* error() const { return w + 1; }
    __device__ __forceinline__ unsigned limit() const { return __ldcg(w + 2); }
    __device__ __forceinline__ unsigned* vmax(int f) const { return w + 3 + f; }
    __device__ __forceinline__ unsigned* done_range(int f) const { return w + 3 + n + f; }
    __device__ __forceinline__ unsigned* done_tiles(int f) const { return w + 3 + 2 * n + f; }
};

__device__ __forceinline__ unsigned load_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Claim the next work item for the whole CTA (one atomicAdd).
__device__ __forceinline__ int claim_item(unsigned* counter, int* slot) {
    __syncthreads();
    if (threadIdx.x == 0) *slot = (int)atomicAdd(counter, 1u);
    __syncthreads();
    return *slot;
}

// CTA-wide wait until *ctr >= target, polled by thread 0 at most `limit`
// times (none needed for target 0; a limit of 0 gives up at once otherwise);
// false when it gave up.  Acquire: what the counted items wrote is visible
// to the whole CTA afterwards.
__device__ __forceinline__ bool cta_wait(const unsigned* ctr, unsigned target, unsigned limit, int* flag) {
    if (threadIdx.x == 0) {
        bool ok = target == 0;
        for (unsigned i = 0; !ok && i < limit; ++i) {
            ok = load_acquire(ctr) >= target;
            if (!ok) __nanosleep(256);
        }
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// Count a finished item (release: the CTA's writes become visible first).
__device__ __forceinline__ void cta_signal(unsigned* ctr) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
    }
}

template <int DT, int M>
__device__ __forceinline__ void range_chunk(const FrameDesc& d, int chunk, unsigned* vmax_bits, float* red) {
    const size_t fe = (size_t)d.W * d.H;
    const size_t i0 = (size_t)chunk * kRangeChunk, i1 = min(fe, i0 + kRangeChunk);
    // kFly loads per thread in flight before any is used (issue is in order:
    // a load consumed right away would expose its whole latency, 128 times
    // per chunk); the maximum does not depend on the order
    constexpr int kFly = 16;
    float vmax = 0.f;
    for (size_t ib = i0 + threadIdx.x; ib < i1; ib += (size_t)kFly * blockDim.x) {
        float z[kFly];
#pragma unroll
        for (int u = 0; u < kFly; ++u) {
            const size_t i = ib + (size_t)u * blockDim.x;
            z[u] = i < i1 ? load_raw<DT>(d.depth, i) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kFly; ++u)
            if (depth_valid(z[u])) vmax = fmaxf(vmax, fit_variable_of<DT, M>(z[u]));
    }
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = vmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) vmax = fmaxf(vmax, red[k]);
        if (vmax > 0.f) atomicMax(vmax_bits, __float_as_uint(vmax));
    }
}

// Two blocks fewer per SM than vpass_kernel: the claim loop's state stays
// live across the column calls, which spill at 5 blocks (96 registers) and
// not at 4 (128); 4 blocks run the mixed batches fastest (3 lose latency
// hiding).
template <int DT, int M>
__global__ void __launch_bounds__(kVThreads, kVBlocks - 2) batch_kernel(const FrameDesc* __restrict__ descs,
                                                                        const int3* __restrict__ items, int n_r,
                                                                        int n_h, int n_v, BatchSync sync,
                                                                        void* planes_base, size_t stride,
                                                                        Codec scale, int min_valid,
                                                                        int require_center) {
    static_assert(kHThreads == kVThreads, "one block shape for every item");
    extern __shared__ int tile[];
    __shared__ int slot, ok;
    __shared__ float red[kVThreads / 32];
    const Planes P(planes_base, stride, planes32<M>());
    const unsigned limit = sync.limit();
    for (;;) {
        const int it = claim_item(sync.claim(), &slot);
        if (it >= n_r + n_h + n_v) break;
        const int3 w = items[it];
        const FrameDesc& d = descs[w.x];
        if (it < n_r) {
            range_chunk<DT, M>(d, w.y, sync.vmax(w.x), red);
            cta_signal(sync.done_range(w.x));
        } else if (it < n_r + n_h) {
            if (!cta_wait(sync.done_range(w.x), (unsigned)d.nr, limit, &ok)) {
                if (threadIdx.x == 0) atomicOr(sync.error(), 1u);
                continue;
            }
            const float sc = ldexpf(1.f, quant_exponent(__ldcg(sync.vmax(w.x)), d.bits));
            // the standard form's wider tiles (several int64 running states per
            // thread) would spill under this kernel's register budget: its frames
            // are tiled 32 columns wide (tiling never changes the exact sums)
            if (base_method(M) == SF_METHOD_STANDARD || d.seg <= 32)
                hpass_tile<DT, M, 1>(d.depth, d.W, d.H, d.r, sc, scale, P, d.pofs, w.y, w.z, tile);
            else if (d.seg <= 64) hpass_tile<DT, M, 2>(d.depth, d.W, d.H, d.r, sc, scale, P, d.pofs, w.y, w.z, tile);
            else hpass_tile<DT, M, 4>(d.depth, d.W, d.H, d.r, sc, scale, P, d.pofs, w.y, w.z, tile);
            cta_signal(sync.done_tiles(w.x));
        } else {
            if (!cta_wait(sync.done_tiles(w.x), (unsigned)d.nh, limit, &ok)) {
                if (threadIdx.x == 0) atomicOr(sync.error(), 2u);
                continue;
            }
            const int x = w.y + threadIdx.x;
            if (x < d.W) {
                const float q = quantum<DT, M>(__ldcg(sync.vmax(w.x)), d.bits, scale);
                vpass_column<DT, M>(d.depth, d.W, d.H, d.r, scale, q, P, d.pofs, x, w.z, d.band,
                                                        d.tx, d.ty, d.a, d.b, min_valid, require_center, d.normals,
                                                        d.offsets, d.curvature, nullptr, INFINITY, nullptr, nullptr,
                                                        w.x, nullptr, 0u);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 re-solve of the queued windows: the exact window moments are
// recomputed from the scratch planes (the 2r + 1 rows of the pixel's column),
// then the whole solve runs in double precision and overwrites the outputs.
// The moments are exact integers, so this removes every float32 rounding of
// the solve; only the fixed-point quantisation of the depth remains.
// ---------------------------------------------------------------------------
template <int DT, int M, bool U4 = false>
__global__ void __launch_bounds__(128) resolve_kernel(int W, int H, int r, Codec scale,
                                                      const unsigned* __restrict__ vmax_bits, int bits, int Wp,
                                                      size_t plane_elems, int nframes, void* __restrict__ planes_base,
                                                      Calib cal, const double* __restrict__ rays,
                                                      const unsigned long long* __restrict__ flags,
                                                      const unsigned* __restrict__ flag_count,
                                                      float* __restrict__ normals, float* __restrict__ offsets,
                                                      float* __restrict__ curvature) {
    const unsigned count = *flag_count;
    const Planes P(planes_base, (size_t)nframes * plane_elems, planes32<M>());
    for (unsigned idx = blockIdx.x * blockDim.x + threadIdx.x; idx < count; idx += gridDim.x * blockDim.x) {
        const unsigned long long e = flags[idx];
        if (e == kQueueHole) continue;
        const int f = (int)(e >> 48), y = (int)((e >> 24) & 0xffffff), x = (int)(e & 0xffffff);
        const size_t pb = plane_index((size_t)f * plane_elems, x, 0, H);
        const double q = (double)quantum<DT, M>(vmax_bits[f], bits, scale);
        const double tx = rays[x], ty = rays[W + y];  // FP64 ray tangents
        const double a = rays[W + H], b = rays[W + H + 1];
        const double wfrac = DT == SF_DEPTH_DISPARITY_U16 ? (double)scale.frac : 0.0;
        FitOutT<double> o;
        bool ok = true;
        if constexpr (M == SF_METHOD_DISPARITY) {
            DispState S(P);
            S.init(pb, kGroup, H, y, r);
            o = solve_disparity<double, U4>((double)S.n, (double)S.Sj, (double)S.Si, (double)S.Sjj, (double)S.Sji,
                                        (double)S.Sii, S.Sw, S.Swj, S.Swi, S.Sww, q, tx, ty, a, b, wfrac);
        } else if constexpr (M == SF_METHOD_STANDARD) {
            StdState S(P);
            S.init(pb, kGroup, H, y, r);
            o = solve_standard<double, U4>((double)S.n, S.Sz, S.Szj, S.Szi, S.Szz, S.Szzj, S.Szzi, S.Szzjj, S.Szzji,
                                       S.Szzii, q, tx, ty, a, b);
        } else if constexpr (M == SF_METHOD_EXPLICIT_DISPARITY) {
            DispState S(P);
            S.init(pb, kGroup, H, y, r);
            o = solve_explicit_disparity<double>((double)S.n, (double)S.Sj, (double)S.Si, (double)S.Sjj,
                                                 (double)S.Sji, (double)S.Sii, S.Sw, S.Swj, S.Swi, S.Sww, q, tx, ty,
                                                 a, b, ok, wfrac);
        } else {
            StdStateT<true> S(P);
            S.init(pb, kGroup, H, y, r);
            o = solve_explicit_standard<double>((double)S.n, (double)S.Sj, (double)S.Si, (double)S.Sjj,
                                                (double)S.Sji, (double)S.Sii, S.Sz, S.Szj, S.Szi, S.Szz, S.Szzj,
                                                S.Szzi, S.Szzjj, S.Szzji, S.Szzii, q, tx, ty, a, b, ok);
        }
        if (!ok) o.nx = o.ny = o.nz = o.d = o.curv = NAN;
        const size_t oi = (size_t)f * W * H + (size_t)y * W + x;
        normals[3 * oi] = (float)o.nx; normals[3 * oi + 1] = (float)o.ny; normals[3 * oi + 2] = (float)o.nz;
        offsets[oi] = (float)o.d;
        curvature[oi] = (float)o.curv;
    }
}

// ---------------------------------------------------------------------------
// Backward, step 1: per-window adjoint.  For every valid window p, from the
// same exact moments as the forward pass and the upstream gradients
// (gn, gd, gk) of (normal, offset, curvature), write the quantities that
// carry the window's contribution to each of its pixels q:
//   disparity: dL_p/dw_q = w_q [(P_q - mu_p) . gbar_p - c_p]   (7 floats: gbar, mu, c)
//   standard:  dL_p/dP_q = 2 Rbar_p (P_q - mu_p) - e_p         (12 floats: 2Rbar, mu, e)
// with mu_p the window's (weighted) centroid.  The disparity form follows
// from R = A - g g^T / s, g = sum w m, s = sum w^2: gbar = -2 Rbar mu - gd n/s,
// sbar = g^T Rbar g / s^2 + gd n.g / s^2, and mu.gbar + 2 sbar = -gd d / s,
// so the contribution gbar.m_q + 2 w_q sbar is centred on the window and
// never subtracts two large numbers.  Invalid windows write zeros.
// Adjoint planes: channel c of frame f at adj + (c * nf + f) * fe.
// ---------------------------------------------------------------------------
template <int DT, int M>
__global__ void __launch_bounds__(kVThreads) vadjoint_kernel(const void* __restrict__ depth, int W, int H, int r,
                                                             Codec scale, const unsigned* __restrict__ vmax_bits,
                                                             int bits, int Wp, size_t plane_elems,
                                                             void* __restrict__ planes_base, Calib cal, int min_valid,
                                                             int require_center, int band,
                                                             const float* __restrict__ g_normals,
                                                             const float* __restrict__ g_offsets,
                                                             const float* __restrict__ g_curv,
                                                             float* __restrict__ adj, float* __restrict__ adj_max) {
    const int f = blockIdx.z;
    const int x = blockIdx.x * kVThreads + threadIdx.x;
    if (x >= W) return;
    const int y0 = blockIdx.y * band;
    const int y1 = min(y0 + band, H);
    const size_t nf = gridDim.z;
    const size_t fe = (size_t)W * H;
    const size_t pb = plane_index((size_t)f * plane_elems, x, 0, H);
    const float q = quantum<DT, M>(vmax_bits[f], bits, scale);
    const float tx = cal.tx[x];
    const size_t fo = (size_t)f * fe;
    const Planes P(planes_base, nf * plane_elems, planes32<M>());
    constexpr int NC = (M == SF_METHOD_DISPARITY) ? 7 : 12;
    typename std::conditional<M == SF_METHOD_DISPARITY, DispState, StdState>::type S(P);
    S.init(pb, kGroup, H, y0, r);
    float tmax[3] = {0.f, 0.f, 0.f};
    // the row's centre depth, upstream gradients and ray; those of the next
    // row and the loads of the slide are issued before this row's solve (issue
    // is in order: loads consumed right away would expose their latency on
    // every row)
    size_t oin = fo + (size_t)y0 * W + x;
    float zn = load_depth<DT>(depth, oin, scale);
    float gnxn = g_normals[3 * oin], gnyn = g_normals[3 * oin + 1], gnzn = g_normals[3 * oin + 2];
    float gdn = g_offsets[oin], gkn = g_curv[oin], tyn = cal.ty[y0];
    for (int y = y0; y < y1; ++y) {
        const size_t oi = oin;
        const bool cvalid = depth_valid(zn);
        const float gnx = gnxn, gny = gnyn, gnz = gnzn, gd = gdn, gk = gkn, ty = tyn;
        const bool more = y + 1 < y1;
        if (more) {
            S.fetch(pb, kGroup, H, y, r);
            oin += W;
            zn = load_depth<DT>(depth, oin, scale);
            gnxn = g_normals[3 * oin]; gnyn = g_normals[3 * oin + 1]; gnzn = g_normals[3 * oin + 2];
            gdn = g_offsets[oin]; gkn = g_curv[oin]; tyn = cal.ty[y + 1];
        }
        const int n = S.count();
        const bool ok = n >= min_valid && n > 0 && (cvalid || !require_center);
        float out[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) out[c] = 0.f;
        if (ok) {
            float R11, R12, R13, R22, R23, R33, mux, muy, muz, s_or_n;
            if constexpr (M == SF_METHOD_DISPARITY) {
                const DispWindow w = build_disparity(S.n, S.Sj, S.Si, S.Sjj, S.Sji, S.Sii, S.Sw, S.Swj, S.Swi,
                                                     S.Sww, tx, ty, cal.a, cal.b);
                R11 = w.R11; R12 = w.R12; R13 = w.R13; R22 = w.R22; R23 = w.R23; R33 = w.R33;
                const float iwm = 1.f / (w.what * q);  // 1 / what_metric
                mux = w.mx * iwm; muy = w.my * iwm; muz = iwm;
                s_or_n = S.n * (w.wbar * q) * (w.what * q);  // sum w^2 = n wbar what
            } else {
                // covariance of the points in metric units (see solve_standard)
                const float nf = (float)S.n, inv_n = 1.f / nf;
                const int m = __float2int_rn(Fn<float>::from_i64(S.Sz) * inv_n);
                const int64_t T0 = S.Sz - (int64_t)S.n * m;
                const int64_t Tzz = S.Szz - (int64_t)m * (S.Sz + T0);
                const int64_t Tzj = S.Szzj - (int64_t)m * S.Szj;
                const int64_t Tzi = S.Szzi - (int64_t)m * S.Szi;
                const float t0 = (float)(int)T0 * inv_n;
                const float fSzj = Fn<float>::from_i64(S.Szj), fSzi = Fn<float>::from_i64(S.Szi);
                const float q2 = q * q;
                const float Czz = (Fn<float>::from_i64(Tzz) - (float)(int)T0 * t0) * q2;
                const float Cjz = (Fn<float>::from_i64(Tzj) - fSzj * t0) * q2;
                const float Ciz = (Fn<float>::from_i64(Tzi) - fSzi * t0) * q2;
                const float qj = fSzj * inv_n, qi = fSzi * inv_n;
                const float Cjj = (Fn<float>::from_i64(S.Szzjj) - fSzj * qj) * q2;
                const float Cji = (Fn<float>::from_i64(S.Szzji) - fSzj * qi) * q2;
                const float Cii = (Fn<float>::from_i64(S.Szzii) - fSzi * qi) * q2;
                const float a = cal.a, b = cal.b;
                R11 = a * a * Cjj + 2.f * a * tx * Cjz + tx * tx * Czz;
                R12 = a * b * Cji + a * ty * Cjz + b * tx * Ciz + tx * ty * Czz;
                R13 = a * Cjz + tx * Czz;
                R22 = b * b * Cii + 2.f * b * ty * Ciz + ty * ty * Czz;
                R23 = b * Ciz + ty * Czz;
                R33 = Czz;
                const float zb = ((float)m + t0) * q;
                mux = a * qj * q + tx * zb; muy = b * qi * q + ty * zb; muz = zb;
                s_or_n = nf;
            }
            float v0, v1, v2, l0n, gap;
            smallest_eigpair(R11, R12, R13, R22, R23, R33, v0, v1, v2, l0n, gap);
            const float tr = R11 + R22 + R33;
            const float d0 = -(v0 * mux + v1 * muy + v2 * muz);
            float nx = v0, ny = v1, nz = v2, d = d0;
            orient(nx, ny, nz, d);
            const float sg = (nx * v0 + ny * v1 + nz * v2) >= 0.f ? 1.f : -1.f;
            // d = -n . mu: gradient wrt the oriented normal, then wrt v0
            const float bx = sg * (gnx - gd * mux), by = sg * (gny - gd * muy), bz = sg * (gnz - gd * muz);
            const Sym3 Rb = eig_adjoint(R11, R12, R13, R22, R23, R33, v0, v1, v2, l0n * tr, tr, bx, by, bz, gk);
            if constexpr (M == SF_METHOD_DISPARITY) {
                const float is = 1.f / s_or_n;
                out[0] = -2.f * (Rb.a11 * mux + Rb.a12 * muy + Rb.a13 * muz) - gd * nx * is;
                out[1] = -2.f * (Rb.a12 * mux + Rb.a22 * muy + Rb.a23 * muz) - gd * ny * is;
                out[2] = -2.f * (Rb.a13 * mux + Rb.a23 * muy + Rb.a33 * muz) - gd * nz * is;
                out[3] = mux; out[4] = muy; out[5] = muz;
                out[6] = gd * d * is;
            } else {
                const float in = 1.f / s_or_n;
                out[0] = 2.f * Rb.a11; out[1] = 2.f * Rb.a12; out[2] = 2.f * Rb.a13;
                out[3] = 2.f * Rb.a22; out[4] = 2.f * Rb.a23; out[5] = 2.f * Rb.a33;
                out[6] = mux; out[7] = muy; out[8] = muz;
                out[9] = gd * nx * in; out[10] = gd * ny * in; out[11] = gd * nz * in;
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            adj[((size_t)c * nf + f) * fe + (size_t)y * W + x] = out[c];
            // the frame's bounds of the box-summed terms (gather_kernel's fixed-point scales)
            const int grp = M == SF_METHOD_DISPARITY ? (c < 3 ? 0 : (c < 6 ? 1 : 2)) : (c < 6 ? 0 : (c < 9 ? 1 : 2));
            tmax[grp] = fmaxf(tmax[grp], fabsf(out[c]));
        }
        if (more) S.apply(r);
    }
    // non-negative floats order as their bit patterns
    const unsigned mask = __activemask();
    const bool leader = (threadIdx.x & 31) == __ffs(mask) - 1;
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        const unsigned m = __reduce_max_sync(mask, __float_as_uint(tmax[g]));
        if (leader && m) atomicMax(reinterpret_cast<unsigned*>(adj_max) + 3 * f + g, m);
    }
}

// ---------------------------------------------------------------------------
// Backward, step 2: every pixel q sums the contributions of the windows p that
// contain it (p in the k x k window around q, by symmetry) and applies the
// chain rule
//   disparity: dL/dZ_q = -w_q^3 sum_p [(P_q - mu_p) . gbar_p - c_p]
//   standard:  dL/dZ_q = m_q . sum_p [2 Rbar_p (P_q - mu_p) - e_p]
// With a reference point P0 the sums factor into k x k box sums of per-window
// quantities, O(1) per pixel like the forward's window sums (Section II.C):
//   disparity: (P_q - P0) . G_q - E_q,      G = box(gbar), E = box((mu - P0) . gbar + c)
//   standard:  A_q (P_q - P0) - V_q,        A = box(2 Rbar), V = box(2 Rbar (mu - P0) + e)
// P0 is the centroid of the output tile's centre window.  The two terms
// cancel by the ratio of |P_q - P0| to the window's extent (large where a
// tile straddles a depth edge), so the box sums are exact: the per-window
// terms are quantised to int64 fixed point with a power of two per channel
// group that puts the frame's bound on them (from the maxima the adjoint
// kernel records) below 2^39, so that sums of up to 961 terms stay below
// 2^49, and the final difference is formed in float-float arithmetic.
// Block: 32 x 8 threads, one 32 x 32 output tile.  Each warp takes whole rows
// of the tile and its r-pixel halo (two staged columns per lane, every
// channel loaded at once), quantises them and forms the horizontal window
// sums with a warp scan; the 32 sums of each row go to shared memory, where
// the columns are box-summed in place (running sums).  Missing pixels get 0.
// ---------------------------------------------------------------------------
constexpr int kGTile = 32;
template <int M>
__host__ __device__ constexpr int gather_channels_box() { return M == SF_METHOD_DISPARITY ? 4 : 9; }
// boxed channels in the first group (gbar; 2 Rbar), the rest in the second
template <int M>
__host__ __device__ constexpr int gather_group0() { return M == SF_METHOD_DISPARITY ? 3 : 6; }
__host__ __device__ constexpr size_t gather_smem_bytes(int nb, int r) {
    return sizeof(long long) * (size_t)nb * (size_t)(kGTile + 2 * r) * kGTile;
}

// round(t) for |t| < 2^41 as int64 without a 64-bit conversion instruction:
// |t| < 2^31 rounds through int32; larger t are integers already (24-bit
// significand) and split exactly into 2^32 hi + lo with lo in [0, 2^32).
__device__ __forceinline__ long long round_i64(float t) {
    if (fabsf(t) < 2147483648.f) return (long long)__float2int_rn(t);
    const float hi = floorf(t * 2.3283064365386963e-10f);  // t / 2^32
    const float lo = fmaf(hi, -4294967296.f, t);            // exact
    return ((long long)(int)hi << 32) + (long long)__float2uint_rn(lo);
}

// Adjoint channels of one window read by the gather (all that the adjoint
// kernel writes: 7 for the disparity form, 12 for the standard form).
template <int M>
__host__ __device__ constexpr int gather_channels_read() { return M == SF_METHOD_DISPARITY ? 7 : 12; }

// The adjoint channels of the two staged columns lane and lane + 32 of staged
// row ty_ (ok: inside the staged tile and the frame; 0 elsewhere).
template <int M>
__device__ __forceinline__ void gather_fetch(const float* __restrict__ src, size_t cstride, int W, int H, int x0,
                                             int y0, int r, int T, int lane, int ty_,
                                             float (&a)[2][gather_channels_read<M>()], bool (&ok)[2]) {
    const int yy = y0 - r + ty_;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int xx = x0 - r + lane + 32 * h;
        ok[h] = ty_ < T && lane + 32 * h < T && xx >= 0 && xx < W && yy >= 0 && yy < H;
        const size_t o = ok[h] ? (size_t)yy * W + xx : 0;
#pragma unroll
        for (int c = 0; c < gather_channels_read<M>(); ++c) a[h][c] = ok[h] ? src[c * cstride + o] : 0.f;
    }
}

// The boxed terms of one window from its adjoint channels a.
template <int M>
__device__ __forceinline__ void gather_terms(const float* a, float p0x, float p0y, float p0z, float* v) {
    if constexpr (M == SF_METHOD_DISPARITY) {
        const float ux = a[3] - p0x, uy = a[4] - p0y, uz = a[5] - p0z;
        v[0] = a[0]; v[1] = a[1]; v[2] = a[2];
        v[3] = fmaf(ux, a[0], fmaf(uy, a[1], fmaf(uz, a[2], a[6])));
    } else {
        const float ux = a[6] - p0x, uy = a[7] - p0y, uz = a[8] - p0z;
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = a[c];
        v[6] = fmaf(a[0], ux, fmaf(a[1], uy, fmaf(a[2], uz, a[9])));
        v[7] = fmaf(a[1], ux, fmaf(a[3], uy, fmaf(a[4], uz, a[10])));
        v[8] = fmaf(a[2], ux, fmaf(a[4], uy, fmaf(a[5], uz, a[11])));
    }
}

// Float-float arithmetic for the final difference (FP64 runs at a small
// fraction of the float32 rate): x = hi + lo with |lo| <= ulp(hi) / 2.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return FF{s, (a - (s - bb)) + (b - bb)};
}
// an exact integer sum (|v| < 2^49) times a power of two, to float-float:
// v = h 2^32 + m 2^16 + l with h < 2^17 and m, l < 2^16 (each exact in
// float32); the two error-free sums leave only the low word's rounding
// (2^-48 relative)
__device__ __forceinline__ FF ff_from_i64(long long v, float sc) {
    const float h = (float)(int)(v >> 32) * 4294967296.f * sc;
    const float m = (float)(int)((v >> 16) & 0xffff) * 65536.f * sc;
    const float l = (float)(int)(v & 0xffff) * sc;
    const FF a = ff_two_sum(h, m);
    const FF b = ff_two_sum(a.hi, l);
    return FF{b.hi, b.lo + a.lo};
}
// acc += u * x (u float), error-free up to the low-order products
__device__ __forceinline__ void ff_fma(FF& acc, float u, FF x) {
    const float p = u * x.hi, pe = fmaf(u, x.hi, -p);
    const FF s = ff_two_sum(acc.hi, p);
    acc.hi = s.hi;
    acc.lo += s.lo + pe + u * x.lo;
}
__device__ __forceinline__ void ff_sub(FF& acc, FF x) {
    const FF s = ff_two_sum(acc.hi, -x.hi);
    acc.hi = s.hi;
    acc.lo += s.lo - x.lo;
}

// Power-of-two scale putting values up to `bound` below 2^39 (0 for a zero or
// non-finite bound: the channel group contributes nothing).
__device__ __forceinline__ float gather_scale(float bound) {
    if (!(bound > 0.f && bound < INFINITY)) return 0.f;
    int e = 0;
    frexpf(bound, &e);
    return ldexpf(1.f, 39 - e);
}

template <int DT, int M>
__global__ void __launch_bounds__(256) gather_kernel(const void* __restrict__ depth, int W, int H, int r, Codec scale,
                                                     Calib cal, const float* __restrict__ adj,
                                                     const float* __restrict__ adj_max, float* __restrict__ g_depth) {
    extern __shared__ long long hs[];  // [channel][staged row][output column]
    constexpr int NB = gather_channels_box<M>(), NG = gather_group0<M>();
    constexpr int MU = (M == SF_METHOD_DISPARITY) ? 3 : 6;  // first centroid channel
    const int f = blockIdx.z;
    const size_t fe = (size_t)W * H;
    const size_t cstride = (size_t)gridDim.z * fe;
    const float* src = adj + (size_t)f * fe;
    const int x0 = blockIdx.x * kGTile, y0 = blockIdx.y * kGTile;
    const int K = 2 * r + 1, T = kGTile + 2 * r;
    const int lane = threadIdx.x, warp = threadIdx.y, tid = warp * 32 + lane;
    // reference point: the centroid of the window at the tile centre (0 where that window is invalid)
    const size_t oc = (size_t)min(y0 + kGTile / 2, H - 1) * W + min(x0 + kGTile / 2, W - 1);
    const float p0x = src[MU * cstride + oc], p0y = src[(MU + 1) * cstride + oc], p0z = src[(MU + 2) * cstride + oc];
    // |group 0| <= gm; |group 1| <= |mu - P0|_max |gbar|_1 + |c| <= 2 mm 3 gm + cm (likewise 2 Rbar, e)
    const float gm = adj_max[3 * f], mm = adj_max[3 * f + 1], cm = adj_max[3 * f + 2];
    const float s0 = gather_scale(gm), s1 = gather_scale(6.f * mm * gm + cm);
    // the loads of the warp's next staged row are issued before this row's
    // arithmetic (issue is in order: a load consumed right away would expose
    // its whole latency on every row)
    constexpr int NR = gather_channels_read<M>();
    float cur[2][NR], nxt[2][NR];
    bool cok[2], nok[2];
    gather_fetch<M>(src, cstride, W, H, x0, y0, r, T, lane, warp, cur, cok);
    for (int ty_ = warp; ty_ < T; ty_ += 8) {
        gather_fetch<M>(src, cstride, W, H, x0, y0, r, T, lane, ty_ + 8, nxt, nok);
        float v[2][NB];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int c = 0; c < NB; ++c) v[h][c] = 0.f;
            if (cok[h]) gather_terms<M>(cur[h], p0x, p0y, p0z, v[h]);
        }
        const int hi = lane + 2 * r;  // last staged column of output column `lane`'s window (< 64)
#pragma unroll
        for (int c = 0; c < NB; ++c) {
            const float sc = c < NG ? s0 : s1;
            long long a = round_i64(v[0][c] * sc), b = round_i64(v[1][c] * sc);
            // inclusive prefix sums over staged columns 0..31 (a) and 32..63 (b)
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long ta = __shfl_up_sync(0xffffffffu, a, o), tb = __shfl_up_sync(0xffffffffu, b, o);
                if (lane >= o) { a += ta; b += tb; }
            }
            b += __shfl_sync(0xffffffffu, a, 31);
            const long long pa = __shfl_sync(0xffffffffu, a, hi & 31), pb = __shfl_sync(0xffffffffu, b, hi & 31);
            const long long pl = __shfl_sync(0xffffffffu, a, (lane + 31) & 31);
            hs[((size_t)c * T + ty_) * kGTile + lane] = (hi < 32 ? pa : pb) - (lane > 0 ? pl : 0ll);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            cok[h] = nok[h];
#pragma unroll
            for (int c = 0; c < NR; ++c) cur[h][c] = nxt[h][c];
        }
    }
    __syncthreads();
    // vertical box sums of every output column, in place
    for (int item = tid; item < NB * kGTile; item += 256) {
        long long* a = hs + (size_t)(item / kGTile) * T * kGTile + (item % kGTile);
        long long S = 0;
        for (int i = 0; i < K; ++i) S += a[(size_t)i * kGTile];
        for (int i = 0; i < kGTile; ++i) {
            const long long out = S;
            if (i + 1 < kGTile) S += a[(size_t)(i + K) * kGTile] - a[(size_t)i * kGTile];
            a[(size_t)i * kGTile] = out;
        }
    }
    __syncthreads();
    // 1 / scale: powers of two, so scaling is exact
    const float i0 = s0 > 0.f ? 1.f / s0 : 0.f, i1 = s1 > 0.f ? 1.f / s1 : 0.f;
    const size_t cs = (size_t)T * kGTile;
    const int x = x0 + lane;
    if (x >= W) return;
    const float tx = cal.tx[x];
    for (int yr = warp; yr < kGTile; yr += 8) {
        const int y = y0 + yr;
        if (y >= H) break;
        const size_t oi = (size_t)f * fe + (size_t)y * W + x;
        const float z = load_depth<DT>(depth, oi, scale);
        float g = 0.f;
        if (depth_valid(z)) {
            const float ty = cal.ty[y];
            const float ux = z * tx - p0x, uy = z * ty - p0y, uz = z - p0z;
            const size_t p = (size_t)yr * kGTile + lane;
            if constexpr (M == SF_METHOD_DISPARITY) {
                FF acc{0.f, 0.f};
                ff_fma(acc, ux, ff_from_i64(hs[p], i0));
                ff_fma(acc, uy, ff_from_i64(hs[cs + p], i0));
                ff_fma(acc, uz, ff_from_i64(hs[2 * cs + p], i0));
                ff_sub(acc, ff_from_i64(hs[3 * cs + p], i1));
                const float w = 1.f / z;
                g = -w * w * w * (acc.hi + acc.lo);
            } else {
                const FF a11 = ff_from_i64(hs[p], i0), a12 = ff_from_i64(hs[cs + p], i0);
                const FF a13 = ff_from_i64(hs[2 * cs + p], i0), a22 = ff_from_i64(hs[3 * cs + p], i0);
                const FF a23 = ff_from_i64(hs[4 * cs + p], i0), a33 = ff_from_i64(hs[5 * cs + p], i0);
                FF ax{0.f, 0.f}, ay{0.f, 0.f}, az{0.f, 0.f};
                ff_fma(ax, ux, a11); ff_fma(ax, uy, a12); ff_fma(ax, uz, a13);
                ff_fma(ay, ux, a12); ff_fma(ay, uy, a22); ff_fma(ay, uz, a23);
                ff_fma(az, ux, a13); ff_fma(az, uy, a23); ff_fma(az, uz, a33);
                ff_sub(ax, ff_from_i64(hs[6 * cs + p], i1));
                ff_sub(ay, ff_from_i64(hs[7 * cs + p], i1));
                ff_sub(az, ff_from_i64(hs[8 * cs + p], i1));
                g = tx * (ax.hi + ax.lo) + ty * (ay.hi + ay.lo) + (az.hi + az.lo);
            }
        }
        g_depth[oi] = g;
    }
}

// ---------------------------------------------------------------------------
// Planar segmentation by tile subdivision (Section III): one warp per node.
// The lanes sum the node's exact integer moments over its rectangle (offsets
// j, i from the rectangle's centre pixel (x0 + w/2, y0 + h/2), |j|, |i| <= 32),
// reduce them across the warp, and
// lane 0 solves the fit in FP64, decides the node's status and, for a split,
// appends its four children to the next level's queue.
// ---------------------------------------------------------------------------
struct QuadRect {
    int frame, x0, y0, w, h;
};

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int DT, int M>
__global__ void __launch_bounds__(256) quad_level_kernel(const void* __restrict__ depth, int W, int H, Codec scale,
                                                         const unsigned* __restrict__ vmax_bits, int bits,
                                                         const double* __restrict__ rays, const QuadRect* __restrict__ in,
                                                         const int* __restrict__ in_count, int level, int max_level,
                                                         double tau, int min_valid, int permille,
                                                         QuadRect* __restrict__ next, int* __restrict__ next_count,
                                                         int next_cap, sf_quad_node* __restrict__ nodes,
                                                         int* __restrict__ node_count, int node_cap,
                                                         int frame_base) {
    constexpr int B = base_method(M);
    const int lane = threadIdx.x & 31;
    const int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (idx >= *in_count) return;
    const QuadRect q = in[idx];
    const size_t fe = (size_t)W * H;
    const size_t dbytes = (DT == SF_DEPTH_F32) ? 4 : 2;
    const void* dframe = static_cast<const char*>(depth) + dbytes * (size_t)q.frame * fe;
    const float sc = ldexpf(1.f, quant_exponent(vmax_bits[q.frame], bits));
    // exact sums: mask moments in int32 (< 2^31 for sides <= 64), values in int64
    int n = 0, Sj = 0, Si = 0, Sjj = 0, Sji = 0, Sii = 0;
    int64_t c0 = 0, cj = 0, ci = 0, c2 = 0, c2j = 0, c2i = 0, c2jj = 0, c2ji = 0, c2ii = 0;
    const int area = q.w * q.h;
    const int xc = q.x0 + (q.w >> 1), yc = q.y0 + (q.h >> 1);
    // kFly pixels per lane loaded before any is used (issue is in order: a
    // load consumed right away would expose its whole latency, up to 128
    // times per lane for a 64 x 64 node); the sums are exact, in any order
    constexpr int kFly = 8;
    for (int p0 = lane; p0 < area; p0 += 32 * kFly) {
        float raw[kFly];
        int pi[kFly], pj[kFly];
#pragma unroll
        for (int u = 0; u < kFly; ++u) {
            const int p = p0 + 32 * u;
            pi[u] = p / q.w;
            pj[u] = p - pi[u] * q.w;
            raw[u] = p < area ? load_raw<DT>(dframe, (size_t)(q.y0 + pi[u]) * W + q.x0 + pj[u]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kFly; ++u) {
            if (p0 + 32 * u >= area) break;
            const int i = q.y0 + pi[u] - yc, j = q.x0 + pj[u] - xc;
            const int v = quantize_raw<DT, M>(raw[u], sc, scale);
            if (v < 0) continue;
            n += 1; Sj += j; Si += i; Sjj += j * j; Sji += j * i; Sii += i * i;
            const int64_t vv = (int64_t)v * v;
            c0 += v; cj += (int64_t)v * j; ci += (int64_t)v * i; c2 += vv;
            if (B == SF_METHOD_STANDARD) { c2j += vv * j; c2i += vv * i; c2jj += vv * (j * j); c2ji += vv * (j * i); c2ii += vv * (i * i); }
        }
    }
    n = warp_sum(n); Sj = warp_sum(Sj); Si = warp_sum(Si); Sjj = warp_sum(Sjj); Sji = warp_sum(Sji); Sii = warp_sum(Sii);
    c0 = warp_sum(c0); cj = warp_sum(cj); ci = warp_sum(ci); c2 = warp_sum(c2);
    if (B == SF_METHOD_STANDARD) {
        c2j = warp_sum(c2j); c2i = warp_sum(c2i); c2jj = warp_sum(c2jj); c2ji = warp_sum(c2ji); c2ii = warp_sum(c2ii);
    }
    if (lane != 0) return;
    sf_quad_node o;
    o.frame = frame_base + q.frame; o.x0 = q.x0; o.y0 = q.y0; o.w = q.w; o.h = q.h; o.level = level; o.count = n;
    o.normal[0] = o.normal[1] = o.normal[2] = NAN;
    o.offset = o.curvature = o.rms = NAN;
    const int need = max(min_valid, (int)(((int64_t)permille * area + 999) / 1000));
    // collinear pixels have no surface fit with any method (the implicit one
    // would be the plane of their camera rays, d = 0): exact integer test
    bool ok = n >= need && n > 0 && pixels_span_plane<double>(n, Sj, Si, Sjj, Sji, Sii);
    double rms = 0.0;
    if (ok) {
        const double qv = (double)quantum<DT, M>(vmax_bits[q.frame], bits, scale);
        const double tx = rays[xc], ty = rays[W + yc], a = rays[W + H], b = rays[W + H + 1];
        const double nf = (double)n;
        const double wfrac = DT == SF_DEPTH_DISPARITY_U16 ? (double)scale.frac : 0.0;
        FitOutT<double> f;
        if constexpr (M == SF_METHOD_DISPARITY)
            f = solve_disparity<double>(nf, (double)Sj, (double)Si, (double)Sjj, (double)Sji, (double)Sii, c0, cj,
                                        ci, c2, qv, tx, ty, a, b, wfrac);
        else if constexpr (M == SF_METHOD_STANDARD)
            f = solve_standard<double>(nf, c0, cj, ci, c2, c2j, c2i, c2jj, c2ji, c2ii, qv, tx, ty, a, b);
        else if constexpr (M == SF_METHOD_EXPLICIT_DISPARITY)
            f = solve_explicit_disparity<double>(nf, (double)Sj, (double)Si, (double)Sjj, (double)Sji, (double)Sii,
                                                 c0, cj, ci, c2, qv, tx, ty, a, b, ok, wfrac);
        else
            f = solve_explicit_standard<double>(nf, (double)Sj, (double)Si, (double)Sjj, (double)Sji, (double)Sii,
                                                c0, cj, ci, c2, c2j, c2i, c2jj, c2ji, c2ii, qv, tx, ty, a, b, ok);
        if (ok) {
            // mean squared residual: lambda0 / n (implicit), the regression's own (explicit)
            const double ms = (M == SF_METHOD_DISPARITY || M == SF_METHOD_STANDARD) ? f.curv * f.tr / nf : f.curv;
            rms = sqrt(ms > 0.0 ? ms : 0.0);
            o.normal[0] = (float)f.nx; o.normal[1] = (float)f.ny; o.normal[2] = (float)f.nz;
            o.offset = (float)f.d; o.curvature = (float)f.curv; o.rms = (float)rms;
        }
    }
    if (!ok) {
        o.status = SF_QUAD_INVALID;
    } else if (rms > tau && level < max_level && q.w >= 2 && q.h >= 2) {
        o.status = SF_QUAD_SPLIT;
        const int base = atomicAdd(next_count, 4);
        if (base + 4 <= next_cap) {
            const int w1 = q.w >> 1, h1 = q.h >> 1;
            next[base + 0] = QuadRect{q.frame, q.x0, q.y0, w1, h1};
            next[base + 1] = QuadRect{q.frame, q.x0 + w1, q.y0, q.w - w1, h1};
            next[base + 2] = QuadRect{q.frame, q.x0, q.y0 + h1, w1, q.h - h1};
            next[base + 3] = QuadRect{q.frame, q.x0 + w1, q.y0 + h1, q.w - w1, q.h - h1};
        }
    } else {
        o.status = rms <= tau ? SF_QUAD_FIT : SF_QUAD_HIGH_ERROR;
    }
    const int slot = atomicAdd(node_count, 1);
    if (slot < node_cap) nodes[slot] = o;
}

// The root tiles of every frame, in frame-major, row-major order.
static __global__ void quad_roots_kernel(int W, int H, int tile, int nfr, QuadRect* __restrict__ out, int* __restrict__ count) {
    const int tw = (W + tile - 1) / tile, th = (H + tile - 1) / tile;
    const int total = tw * th * nfr;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int f = t / (tw * th), rem = t - f * tw * th, ty = rem / tw, tx = rem - ty * tw;
        const int x0 = tx * tile, y0 = ty * tile;
        out[t] = QuadRect{f, x0, y0, min(tile, W - x0), min(tile, H - y0)};
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = total;
}

}  // namespace sf
