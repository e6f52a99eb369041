// sf_delta.cuh -- per-pixel ray adjustments (a delta table) for the disparity
// form (device code, included after sf_kernels.cuh).
//
// Eq. 1 and Eq. 10 add an adjustment (dx, dy) to a pixel's coordinates before
// its ray is formed.  With one adjustment per pixel the ray of pixel q in the
// window of p is
//   tx_q = tx_p + a (j + D_q / S),   ty_q = ty_p + b (i + E_q / S)
// (a = 1/fx, b = 1/fy, tx_p, ty_p the rays without the table, D, E the table
// in units of 1/S pixel, S = 2^18), so every sum over the window's pixel
// offsets j, i becomes a sum over the shifted offsets jh = j + D/S,
// ih = i + E/S.  With integer D, E these sums stay exact integers, in units of
// 1/S (first moments) and 1/S^2 (second moments): the row pass adds the sums
// of D, D j, E, E j, D^2, E^2, D E, v D and v E (valid pixels) to its usual
// ones, the column pass slides them (with i weights where a moment needs
// them), and the build forms the shifted moments exactly (128-bit products)
// before the usual centring and solve.
//
// The resolution: the table's rounding to 1/S pixel moves each pixel's ray
// like a pixel-position error of up to 1/(2S); at S = 2^18 that keeps the
// normal within ~1e-5 rad of the unrounded rays on 5 x 5 windows (the error
// scales with 1/S and falls with the window size).
#pragma once

namespace sf {

constexpr int kDeltaScale = 1 << 18;  // table units per pixel
constexpr int kDeltaMax = 16 * kDeltaScale - 1;
// scratch planes of the table path: int32 mask, sum v, sum v j (low word),
// sum D, sum E; int64 sum v^2, sum D j, sum E j, sum D^2, sum E^2, sum D E,
// sum v D, sum v E (20 + 64 = 84 B per pixel)
constexpr int kDeltaPlanes32 = 5;
constexpr int kDeltaPlanes64 = 8;

// Row sums of one row over one 32-column output segment, with the table's sums.
// drow / erow: the row's table entries D and E (tile-relative like row).
__device__ __forceinline__ void hpass_row_delta(const int* row, const int* drow, const int* erow, int x0, int xend,
                                                int y, int H, int r, const Planes& P, size_t pofs) {
    HRowState<SF_METHOD_DISPARITY> S;
    int64_t d0 = 0, d1 = 0, e0 = 0, e1 = 0, dd = 0, ee = 0, de = 0, vd = 0, ve = 0;
    S.init(row, 0, r);
    for (int j = -r; j <= r; ++j) {
        const int v = row[j + r];
        if (v >= 0) {
            const int64_t D = drow[j + r], E = erow[j + r];
            d0 += D; d1 += D * j; e0 += E; e1 += E * j;
            dd += D * D; ee += E * E; de += D * E;
            vd += (int64_t)v * D; ve += (int64_t)v * E;
        }
    }
    for (int xb = x0; xb < xend; xb += 4) {
        int32_t hmv[4], c0v[4], c1v[4], t32[2][4];
        int64_t t64[8][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = xb + u;
            hmv[u] = pack_mask(S.h0, S.h1, S.h2, (int)(S.a1 >> 32));
            c0v[u] = (int)S.a0; c1v[u] = lo32(S.a1);
            t32[0][u] = (int32_t)d0; t32[1][u] = (int32_t)e0;
            t64[0][u] = S.s0; t64[1][u] = d1; t64[2][u] = e1; t64[3][u] = dd; t64[4][u] = ee; t64[5][u] = de;
            t64[6][u] = vd; t64[7][u] = ve;
            if (x + 1 < xend) {
                const int c = x - x0;
                const int vo = row[c], vi = row[c + 2 * r + 1];
                const int64_t Do = vo >= 0 ? drow[c] : 0, Eo = vo >= 0 ? erow[c] : 0;
                const int64_t Di = vi >= 0 ? drow[c + 2 * r + 1] : 0, Ei = vi >= 0 ? erow[c + 2 * r + 1] : 0;
                slide2(d0, d1, Do, Di, r);
                slide2(e0, e1, Eo, Ei, r);
                dd += Di * Di - Do * Do; ee += Ei * Ei - Eo * Eo; de += Di * Ei - Do * Eo;
                const int64_t co = vo >= 0 ? vo : 0, ci = vi >= 0 ? vi : 0;
                vd += ci * Di - co * Do; ve += ci * Ei - co * Eo;
                S.step(row, c, r);
            }
        }
        const size_t o = plane_index(pofs, xb, y, H);  // xb % 4 == 0: 4 entries in one group
        if (xb + 4 <= xend) {
            *reinterpret_cast<int4*>(P.p32 + o) = make_int4(hmv[0], hmv[1], hmv[2], hmv[3]);
            *reinterpret_cast<int4*>(P.c32(1) + o) = make_int4(c0v[0], c0v[1], c0v[2], c0v[3]);
            *reinterpret_cast<int4*>(P.c32(2) + o) = make_int4(c1v[0], c1v[1], c1v[2], c1v[3]);
#pragma unroll
            for (int q = 0; q < 2; ++q)
                *reinterpret_cast<int4*>(P.c32(3 + q) + o) = make_int4(t32[q][0], t32[q][1], t32[q][2], t32[q][3]);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int64_t* a = P.c64(q) + o;
                *reinterpret_cast<longlong2*>(a) = make_longlong2(t64[q][0], t64[q][1]);
                *reinterpret_cast<longlong2*>(a + 2) = make_longlong2(t64[q][2], t64[q][3]);
            }
        } else {
            for (int u = 0; u < 4 && xb + u < xend; ++u) {
                P.p32[o + u] = hmv[u]; P.c32(1)[o + u] = c0v[u]; P.c32(2)[o + u] = c1v[u];
                for (int q = 0; q < 2; ++q) P.c32(3 + q)[o + u] = t32[q][u];
                for (int q = 0; q < 8; ++q) P.c64(q)[o + u] = t64[q][u];
            }
        }
    }
}

// Row pass with the table: tiles of 128 rows x 32 columns; shared memory holds
// the quantised depth tile and the table's two tiles, each kHThreads x
// ((32 + 2r) | 1).  dtab holds the table's D plane then its E plane ([H][W] each).
template <int DT>
__global__ void __launch_bounds__(kHThreads) hpass_delta_kernel(const void* __restrict__ depth,
                                                                const int* __restrict__ dtab, int W, int H, int r,
                                                                Codec scale, const unsigned* __restrict__ vmax_bits,
                                                                int bits, size_t plane_elems, void* planes_base) {
    extern __shared__ int tile[];
    constexpr int seg = 32;
    const int f = blockIdx.z;
    const float sc = ldexpf(1.f, quant_exponent(vmax_bits[f], bits));  // 2^e, exact
    const size_t dbytes = (DT == SF_DEPTH_F32) ? 4 : 2;
    const void* dframe = static_cast<const char*>(depth) + dbytes * (size_t)f * W * H;
    const Planes P(planes_base, (size_t)gridDim.z * plane_elems, kDeltaPlanes32);
    const int x0 = blockIdx.x * seg, y0 = blockIdx.y * kHThreads;
    const int IW = seg + 2 * r, pitch = IW | 1, rows = min(kHThreads, H - y0);
    int* dt = tile + kHThreads * pitch;
    int* et = dt + kHThreads * pitch;
    const size_t fe = (size_t)W * H;
    load_tile<DT, SF_METHOD_DISPARITY, 2>(dframe, W, r, sc, scale, x0, y0, rows, IW, pitch, tile);
    for (int idx = threadIdx.x; idx < rows * IW; idx += kHThreads) {
        const int ry = idx / IW, cx = idx - ry * IW, x = x0 - r + cx;
        const bool in = x >= 0 && x < W;
        const size_t g = (size_t)(y0 + ry) * W + x;
        dt[ry * pitch + cx] = in ? __ldg(dtab + g) : 0;
        et[ry * pitch + cx] = in ? __ldg(dtab + fe + g) : 0;
    }
    __syncthreads();
    if ((int)threadIdx.x < rows)
        hpass_row_delta(tile + threadIdx.x * pitch, dt + threadIdx.x * pitch, et + threadIdx.x * pitch, x0,
                        min(x0 + seg, W), y0 + threadIdx.x, H, r, P, (size_t)f * plane_elems);
}

// Column sums of the table path: the usual disparity sums (DispState on the
// same first planes) plus the table's, i-weighted where the shifted moments
// need it: sum D, sum i D (and E) slide as a pair; sum D j, D^2, E^2, D E,
// v D, v E are plain sums of the row sums.
struct DispDeltaState {
    DispState B;
    const int32_t* pd[2];  // row sum D, row sum E
    const int64_t* pq[7];  // row sums D j, E j, D^2, E^2, D E, v D, v E
    int64_t TD = 0, TDi = 0, TE = 0, TEi = 0;
    int64_t T[7] = {0, 0, 0, 0, 0, 0, 0};  // window sums D j, E j, D^2, E^2, D E, v D, v E
    int32_t qo[2] = {0, 0}, qi[2] = {0, 0};
    int64_t wo[7] = {0, 0, 0, 0, 0, 0, 0}, wi[7] = {0, 0, 0, 0, 0, 0, 0};
    __device__ DispDeltaState(const Planes& P) : B(P) {
        pd[0] = P.c32(3); pd[1] = P.c32(4);
        for (int q = 0; q < 7; ++q) pq[q] = P.c64(1 + q);
    }
    __device__ __forceinline__ void init(size_t pb, int rs, int H, int y0, int r) {
        B.init(pb, rs, H, y0, r);
        const int ylo = max(y0 - r, 0), yhi = min(y0 + r, H - 1);
        for (int yy = ylo; yy <= yhi; ++yy) {
            const size_t o = pb + (size_t)yy * rs;
            const int64_t i = yy - y0;
            const int64_t d0 = __ldg(pd[0] + o), e0 = __ldg(pd[1] + o);
            TD += d0; TDi += i * d0;
            TE += e0; TEi += i * e0;
            for (int q = 0; q < 7; ++q) T[q] += __ldg(pq[q] + o);
        }
    }
    __device__ __forceinline__ void fetch(size_t pb, int rs, int H, int y, int r) {
        B.fetch(pb, rs, H, y, r);
        const int yo = y - r, yi = y + r + 1;
        qo[0] = qo[1] = qi[0] = qi[1] = 0;
        for (int q = 0; q < 7; ++q) { wo[q] = 0; wi[q] = 0; }
        if (yo >= 0) {
            const size_t o = pb + (size_t)yo * rs;
            qo[0] = __ldg(pd[0] + o); qo[1] = __ldg(pd[1] + o);
            for (int q = 0; q < 7; ++q) wo[q] = __ldg(pq[q] + o);
        }
        if (yi < H) {
            const size_t o = pb + (size_t)yi * rs;
            qi[0] = __ldg(pd[0] + o); qi[1] = __ldg(pd[1] + o);
            for (int q = 0; q < 7; ++q) wi[q] = __ldg(pq[q] + o);
        }
    }
    __device__ __forceinline__ void apply(int r) {
        B.apply(r);
        slide2(TD, TDi, (int64_t)qo[0], (int64_t)qi[0], r);
        slide2(TE, TEi, (int64_t)qo[1], (int64_t)qi[1], r);
        for (int q = 0; q < 7; ++q) T[q] += wi[q] - wo[q];
    }
    __device__ __forceinline__ int count() const { return B.count(); }
};

// float32 value of a 128-bit integer (to float32 rounding): the magnitude's
// 32-bit words scaled and summed from the top, then the sign
__device__ __forceinline__ float from_i128(__int128 v) {
    const bool neg = v < 0;
    const unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
    float f = __uint2float_rn((uint32_t)(hi >> 32)) * 4294967296.f + __uint2float_rn((uint32_t)hi);
    f = f * 4294967296.f + __uint2float_rn((uint32_t)(lo >> 32));
    f = f * 4294967296.f + __uint2float_rn((uint32_t)lo);
    return neg ? -f : f;
}

// The disparity window (as build_disparity) from the shifted offsets
// jh = j + D/S, ih = i + E/S.  Every shifted moment is an exact integer:
// J = S sum jh, JJ = S^2 sum jh^2, JI = S^2 sum jh ih, WJ = S sum w jh (w in
// units of qw), and the centred moments n JJ - J^2 etc. are formed in
// 128-bit integers before the conversion to float.  wfrac: the fractional
// offset of disparity input (added to the mean disparity).
__device__ __forceinline__ DispWindowT<float> build_disparity_delta(const DispDeltaState& st, float tx, float ty,
                                                                    float a, float b, float wfrac) {
    using T = float;
    const DispState& s = st.B;
    const int64_t S = kDeltaScale;
    const int n = (int)s.n;
    const int64_t Sj = (int)s.Sj, Si = (int)s.Si, Sjj = (int)s.Sjj, Sji = (int)s.Sji, Sii = (int)s.Sii;
    const int64_t TDj = st.T[0], TEj = st.T[1], TDD = st.T[2], TEE = st.T[3], TDE = st.T[4], TwD = st.T[5],
                  TwE = st.T[6];
    const int64_t J = S * Sj + st.TD, I = S * Si + st.TE;
    const int64_t JJ = S * S * Sjj + 2 * S * TDj + TDD;
    const int64_t JI = S * S * Sji + S * TEj + S * st.TDi + TDE;
    const int64_t II = S * S * Sii + 2 * S * st.TEi + TEE;
    const int64_t WJ = S * s.Swj + TwD, WI = S * s.Swi + TwE;
    const T nf = (T)n;
    const T inv_n = Fn<T>::rcp(nf);
    // exact re-centring of w on an integer m near its mean (as build_disparity)
    const int m = __float2int_rn(Fn<T>::from_i64(s.Sw) * inv_n);
    const int64_t T0 = s.Sw - (int64_t)n * m;
    const int64_t Tww = s.Sww - (int64_t)m * (s.Sw + T0);
    const int64_t TWJ = WJ - (int64_t)m * J;  // S sum (w - m) jh
    const int64_t TWI = WI - (int64_t)m * I;
    const T fT0 = (T)(int)T0;
    const T t0 = fT0 * inv_n;
    const T iS = T(1) / T(kDeltaScale);
    const T fJ = Fn<T>::from_i64(J), fI = Fn<T>::from_i64(I);
    const T jb = fJ * iS * inv_n, ib = fI * iS * inv_n;
    const T inS2 = iS * iS * inv_n;
    const T Cjj = from_i128((__int128)n * JJ - (__int128)J * J) * inS2;
    const T Cji = from_i128((__int128)n * JI - (__int128)J * I) * inS2;
    const T Cii = from_i128((__int128)n * II - (__int128)I * I) * inS2;
    const T Cjw = (Fn<T>::from_i64(TWJ) - fJ * t0) * iS;
    const T Ciw = (Fn<T>::from_i64(TWI) - fI * t0) * iS;
    const T Cww = Fn<T>::from_i64(Tww) - fT0 * t0;
    const T wbar = (T)m + t0 + wfrac;
    const T inv_nw = Fn<T>::rcp(nf * wbar);
    const T dj = Cjw * inv_nw, di = Ciw * inv_nw, e = Cww * inv_nw;
    const T what = wbar + e;
    const T Yjj = Cjj + nf * dj * dj, Yji = Cji + nf * dj * di, Yii = Cii + nf * di * di;
    const T Yjr = -nf * dj, Yir = -nf * di;
    const T iw = Fn<T>::rcp(what);
    const T Yrr = (Cww + nf * e * e) * iw * iw;
    DispWindowT<T> w;
    w.mx = tx + a * (jb + dj);
    w.my = ty + b * (ib + di);
    w.R11 = a * a * Yjj + T(2) * a * w.mx * Yjr + w.mx * w.mx * Yrr;
    w.R12 = a * b * Yji + a * w.my * Yjr + b * w.mx * Yir + w.mx * w.my * Yrr;
    w.R13 = a * Yjr + w.mx * Yrr;
    w.R22 = b * b * Yii + T(2) * b * w.my * Yir + w.my * w.my * Yrr;
    w.R23 = b * Yir + w.my * Yrr;
    w.R33 = Yrr;
    w.what = what;
    w.wbar = wbar;
    return w;
}

// Column pass + solve with the table (disparity form; U4 the literal
// |(a,b,c,d)| = 1 constraint), one thread per column over a band of rows.
// With flags (precision modes 1 and 2) windows whose float32 eigen-gap is
// below tau, or whose fixed-point rounding could move the normal by more than
// kRefineRounding, are queued for direct_delta_kernel.
template <int DT, bool U4>
__global__ void __launch_bounds__(kVThreads) vpass_delta_kernel(const void* __restrict__ depth, int W, int H, int r,
                                                                Codec scale, const unsigned* __restrict__ vmax_bits,
                                                                int bits, size_t plane_elems, void* planes_base,
                                                                Calib cal, int min_valid, int require_center,
                                                                int band, float* __restrict__ normals,
                                                                float* __restrict__ offsets,
                                                                float* __restrict__ curvature,
                                                                int32_t* __restrict__ counts, float tau,
                                                                unsigned long long* __restrict__ flags,
                                                                unsigned* __restrict__ flag_count) {
    const int f = blockIdx.z;
    const int x = blockIdx.x * kVThreads + threadIdx.x;
    if (x >= W) return;
    const size_t fe = (size_t)W * H;
    const size_t dbytes = (DT == SF_DEPTH_F32) ? 4 : 2;
    const void* dframe = static_cast<const char*>(depth) + dbytes * (size_t)f * fe;
    const float q = quantum<DT, SF_METHOD_DISPARITY>(vmax_bits[f], bits, scale);
    const float wfrac = DT == SF_DEPTH_DISPARITY_U16 ? scale.frac : 0.f;
    const int lane = threadIdx.x & 31;
    const Planes P(planes_base, (size_t)gridDim.z * plane_elems, kDeltaPlanes32);
    const size_t pb = plane_index((size_t)f * plane_elems, x, 0, H);
    const int y0 = blockIdx.y * band, y1 = min(y0 + band, H);
    const float tx = cal.tx[x];
    DispDeltaState S(P);
    S.init(pb, kGroup, H, y0, r);
    float zc = load_depth<DT>(dframe, (size_t)y0 * W + x, scale);
    for (int y = y0; y < y1; ++y) {
        const size_t oi = (size_t)f * fe + (size_t)y * W + x;
        const bool cvalid = depth_valid(zc);
        // the next slide's rows (and the next centre depth) load while this row solves
        const bool more = y + 1 < y1;
        if (more) {
            S.fetch(pb, kGroup, H, y, r);
            zc = load_depth<DT>(dframe, (size_t)(y + 1) * W + x, scale);
        }
        const int n = S.count();
        const bool ok = n >= min_valid && n > 0 && (cvalid || !require_center);
        float nx = NAN, ny = NAN, nz = NAN, d = NAN, cu = NAN;
        if (ok) {
            const DispWindowT<float> w = build_disparity_delta(S, tx, cal.ty[y], cal.a, cal.b, wfrac);
            FitOut fo;
            bool queue = false;
            if constexpr (U4) {
                const float sw = q * (float)n * w.wbar;
                fo = solve_unit4<float>(w.R11, w.R12, w.R13, w.R22, w.R23, w.R33, sw * w.mx, sw * w.my, sw,
                                        sw * q * w.what);
                queue = flags && !(fo.gap >= tau);
            } else {
                float l0, l2n;
                smallest_eigpair<float>(w.R11, w.R12, w.R13, w.R22, w.R23, w.R33, fo.nx, fo.ny, fo.nz, l0, fo.gap,
                                        &l2n);
                fo.curv = l0;
                if (flags) {
                    queue = !(fo.gap >= tau);
                    if (!queue && !fixed_quantum<DT, SF_METHOD_DISPARITY>()) {
                        const float tr = w.R11 + w.R22 + w.R33, iw = 1.f / w.what;
                        const float thr2 = kRefineRounding * kRefineRounding;
                        queue = rounding_error2_screened<float>(w.R11, w.R12, w.R13, w.R22, w.R23, w.R33, fo.nx,
                                                                fo.ny, fo.nz, w.mx * iw, w.my * iw, iw, l0 * tr,
                                                                (l0 + fo.gap * l2n) * tr, l2n * tr, thr2) > thr2;
                    }
                }
                fo.d = -(fo.nx * w.mx + fo.ny * w.my + fo.nz) * Fn<float>::rcp(w.what * q);
                orient<float>(fo.nx, fo.ny, fo.nz, fo.d);
            }
            nx = fo.nx; ny = fo.ny; nz = fo.nz; d = fo.d; cu = fo.curv;
            if (queue) {
                const unsigned mask = __activemask();
                const int leader = __ffs(mask) - 1;
                unsigned base = 0;
                if (lane == leader) base = atomicAdd(flag_count, (unsigned)__popc(mask));
                base = __shfl_sync(mask, base, leader);
                flags[base + __popc(mask & ((1u << lane) - 1u))] =
                    ((unsigned long long)f << 48) | ((unsigned long long)y << 24) | (unsigned long long)x;
            }
        }
        normals[3 * oi] = nx; normals[3 * oi + 1] = ny; normals[3 * oi + 2] = nz;
        offsets[oi] = d; curvature[oi] = cu;
        if (counts) counts[oi] = n;
        if (more) S.apply(r);
    }
}

// ---------------------------------------------------------------------------
// Precision modes with a table: the queued windows solved again in FP64 from
// sums of the unrounded depth and the table's rays, as the paper defines the
// fit (Eq. 14 with the rays of Eq. 1 / Eq. 10), with no fixed point.  Each
// warp takes up to 32 windows; for each in turn its lanes sum the window's columns
// (lane l: column offset j = l - r), first the count and the disparity to
// centre on, then the moments of the shifted offsets jh = j + D/S,
// ih = i + E/S and of w' = w - wc; every lane then solves its own window.
// ---------------------------------------------------------------------------
// Disparity (1/m) of a stored value in FP64, or -1 for a missing pixel,
// under the same validity rule as the fixed-point path.
template <int DT>
__device__ __forceinline__ double disparity_f64(float zin, const Codec& cd) {
    if (DT == SF_DEPTH_DISPARITY_U16) {
        const int w = disparity_units(zin, cd);
        return w < 0 ? -1.0 : (double)cd.scale * ((double)w + (double)cd.frac);
    }
    if (DT == SF_DEPTH_U16) return zin != 0.f ? 1.0 / ((double)zin * (double)cd.scale) : -1.0;
    return depth_valid(zin) ? 1.0 / (double)zin : -1.0;
}

constexpr int kDirectSums = 10;  // n, sum jh, ih, jh^2, jh ih, ih^2, w', w' jh, w' ih, w'^2

template <int DT>
__device__ __forceinline__ void direct_sums(const void* __restrict__ dframe, const int* __restrict__ dtab, int W,
                                            int H, int r, const Codec& cd, int px, int py, double* out) {
    const int lane = threadIdx.x & 31;
    const int j = lane - r;
    const int x = px + j;
    const bool col = lane <= 2 * r && x >= 0 && x < W;
    const size_t fe = (size_t)W * H;
    // pass 1: the mean disparity, to centre the second moments on
    double n = 0.0, sw = 0.0;
#pragma unroll 1
    for (int i = -r; i <= r; ++i) {
        const int y = py + i;
        if (!(col && y >= 0 && y < H)) continue;
        const double w = disparity_f64<DT>(load_raw<DT>(dframe, (size_t)y * W + x), cd);
        if (w < 0.0) continue;
        n += 1.0; sw += w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, o);
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
    }
    const double wc = n > 0.0 ? sw / n : 0.0;
    double v[kDirectSums];
#pragma unroll
    for (int c = 0; c < kDirectSums; ++c) v[c] = 0.0;
    const double iS = 1.0 / (double)kDeltaScale;
#pragma unroll 1
    for (int i = -r; i <= r; ++i) {
        const int y = py + i;
        if (!(col && y >= 0 && y < H)) continue;
        const size_t g = (size_t)y * W + x;
        double w = disparity_f64<DT>(load_raw<DT>(dframe, g), cd);
        if (w < 0.0) continue;
        w -= wc;
        const double jh = (double)j + (double)__ldg(dtab + g) * iS;
        const double ih = (double)i + (double)__ldg(dtab + fe + g) * iS;
        v[0] += 1.0; v[1] += jh; v[2] += ih; v[3] += jh * jh; v[4] += jh * ih; v[5] += ih * ih;
        v[6] += w; v[7] += w * jh; v[8] += w * ih; v[9] += w * w;
    }
#pragma unroll
    for (int c = 0; c < kDirectSums; ++c) {
        double a = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        out[c] = a;
    }
    out[kDirectSums] = wc;
}

// The disparity window (as build_disparity: R = K Y K^T) from FP64 sums of the
// shifted offsets and of w' = w - wc (w in 1/m).
__device__ __forceinline__ DispWindowT<double> disparity_window_f64(const double* m, double tx, double ty, double a,
                                                                    double b) {
    using T = double;
    const T n = m[0], wc = m[kDirectSums];
    const T jb = m[1] / n, ib = m[2] / n;
    const T Cjj = m[3] - m[1] * jb, Cji = m[4] - m[1] * ib, Cii = m[5] - m[2] * ib;
    const T t0 = m[6] / n;
    const T Cjw = m[7] - m[1] * t0, Ciw = m[8] - m[2] * t0, Cww = m[9] - m[6] * t0;
    const T wbar = wc + t0;
    const T inv_nw = T(1) / (n * wbar);
    const T dj = Cjw * inv_nw, di = Ciw * inv_nw, e = Cww * inv_nw;
    const T what = wbar + e;
    const T Yjj = Cjj + n * dj * dj, Yji = Cji + n * dj * di, Yii = Cii + n * di * di;
    const T Yjr = -n * dj, Yir = -n * di;
    const T iw = T(1) / what;
    const T Yrr = (Cww + n * e * e) * iw * iw;
    DispWindowT<T> w;
    w.mx = tx + a * (jb + dj);
    w.my = ty + b * (ib + di);
    w.R11 = a * a * Yjj + T(2) * a * w.mx * Yjr + w.mx * w.mx * Yrr;
    w.R12 = a * b * Yji + a * w.my * Yjr + b * w.mx * Yir + w.mx * w.my * Yrr;
    w.R13 = a * Yjr + w.mx * Yrr;
    w.R22 = b * b * Yii + T(2) * b * w.my * Yir + w.my * w.my * Yrr;
    w.R23 = b * Yir + w.my * Yrr;
    w.R33 = Yrr;
    w.what = what;
    w.wbar = wbar;
    return w;
}

template <int DT, bool U4>
__global__ void __launch_bounds__(128) direct_delta_kernel(const void* __restrict__ depth,
                                                           const int* __restrict__ dtab, int W, int H, int r,
                                                           Codec cd, const double* __restrict__ rays,
                                                           const unsigned long long* __restrict__ flags,
                                                           const unsigned* __restrict__ flag_count,
                                                           float* __restrict__ normals, float* __restrict__ offsets,
                                                           float* __restrict__ curvature) {
    const unsigned count = *flag_count;
    const int lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    const size_t fe = (size_t)W * H;
    const size_t dbytes = (DT == SF_DEPTH_F32) ? 4 : 2;
    // lane l of warp w: window w + l W (W warps), so that a short queue spreads over every warp
    for (unsigned base = warp; base < count; base += nwarps * 32u) {
        const unsigned mine_idx = base + (unsigned)lane * nwarps;
        const bool active = mine_idx < count && flags[mine_idx] != kQueueHole;
        int f = 0, x = 0, y = 0;
        if (active) {
            const unsigned long long e = flags[mine_idx];
            f = (int)(e >> 48); y = (int)((e >> 24) & 0xffffff); x = (int)(e & 0xffffff);
        }
        double mine[kDirectSums + 1];
        unsigned todo = __ballot_sync(0xffffffffu, active);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int sf_ = __shfl_sync(0xffffffffu, f, src);
            const int sx = __shfl_sync(0xffffffffu, x, src);
            const int sy = __shfl_sync(0xffffffffu, y, src);
            const void* dframe = static_cast<const char*>(depth) + dbytes * (size_t)sf_ * fe;
            double sums[kDirectSums + 1];
            direct_sums<DT>(dframe, dtab, W, H, r, cd, sx, sy, sums);
            if (lane == src) {
#pragma unroll
                for (int c = 0; c <= kDirectSums; ++c) mine[c] = sums[c];
            }
        }
        if (!active) continue;
        const DispWindowT<double> w = disparity_window_f64(mine, rays[x], rays[W + y], rays[W + H], rays[W + H + 1]);
        FitOutT<double> o;
        if constexpr (U4) {
            const double sw = mine[0] * w.wbar;  // sum w (1/m); sum w^2 = sw what
            o = solve_unit4<double>(w.R11, w.R12, w.R13, w.R22, w.R23, w.R33, sw * w.mx, sw * w.my, sw, sw * w.what);
        } else {
            double l0;
            smallest_eigpair_iso<double>(w.R11, w.R12, w.R13, w.R22, w.R23, w.R33, o.nx, o.ny, o.nz, l0, o.gap);
            o.curv = l0;
            o.d = -(o.nx * w.mx + o.ny * w.my + o.nz) / w.what;
            orient<double>(o.nx, o.ny, o.nz, o.d);
        }
        const size_t oi = (size_t)f * fe + (size_t)y * W + x;
        normals[3 * oi] = (float)o.nx; normals[3 * oi + 1] = (float)o.ny; normals[3 * oi + 2] = (float)o.nz;
        offsets[oi] = (float)o.d;
        curvature[oi] = (float)o.curv;
    }
}

}  // namespace sf
