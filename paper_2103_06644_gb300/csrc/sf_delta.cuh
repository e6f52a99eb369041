// sf_delta.cuh -- per-pixel ray adjustments (a delta table) for the disparity
// form (device code, included by surffit.cu after sf_kernels.cuh).
//
// Eq. 1 and Eq. 10 add an adjustment (dx, dy) to a pixel's coordinates before
// its ray is formed.  With one adjustment per pixel the ray of pixel q in the
// window of p is
//   tx_q = tx_p + a (j + D_q / 256),   ty_q = ty_p + b (i + E_q / 256)
// (a = 1/fx, b = 1/fy, tx_p, ty_p the rays without the table, D, E the table
// in 1/256 pixel), so every sum over the window's pixel offsets j, i becomes a
// sum over the shifted offsets jh = j + D/256, ih = i + E/256.  With integer
// D, E these sums stay exact integers, in units of 1/256 (first moments) and
// 1/65536 (second moments): the row pass adds the sums of D, D j, E, E j, D^2,
// E^2, D E, v D and v E (valid pixels) to its usual ones, the column pass
// slides them (with i weights where a moment needs them), and the build forms
// the shifted moments exactly before the usual centring and solve.
#pragma once

namespace sf {

constexpr int kDeltaScale = 256;  // table units per pixel
constexpr int kDeltaMax = 16 * kDeltaScale - 1;
// scratch planes of the table path: int32 mask, sum v, sum v j (low word),
// sum D, sum D j, sum E, sum E j, sum D^2, sum E^2, sum D E; int64 sum v^2,
// sum v D, sum v E (20 + 44 = 64 B per pixel)
constexpr int kDeltaPlanes32 = 10;
constexpr int kDeltaPlanes64 = 3;

// a table entry packs D (low 16 bits) and E (high 16 bits), both signed
__device__ __forceinline__ int delta_x(int p) { return (int)(int16_t)(p & 0xffff); }
__device__ __forceinline__ int delta_y(int p) { return p >> 16; }

// Row sums of one row over one 32-column output segment, with the table's sums.
__device__ __forceinline__ void hpass_row_delta(const int* row, const int* drow, int x0, int xend, int y, int H,
                                                int r, const Planes& P, size_t pofs) {
    HRowState<SF_METHOD_DISPARITY> S;
    int d0 = 0, d1 = 0, e0 = 0, e1 = 0, dd = 0, ee = 0, de = 0;
    int64_t vd = 0, ve = 0;
    S.init(row, 0, r);
    for (int j = -r; j <= r; ++j) {
        const int v = row[j + r];
        if (v >= 0) {
            const int p = drow[j + r], D = delta_x(p), E = delta_y(p);
            d0 += D; d1 += D * j; e0 += E; e1 += E * j;
            dd += D * D; ee += E * E; de += D * E;
            vd += (int64_t)v * D; ve += (int64_t)v * E;
        }
    }
    for (int xb = x0; xb < xend; xb += 4) {
        int32_t hmv[4], c0v[4], c1v[4], t[7][4];
        int64_t c2v[4], vdv[4], vev[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = xb + u;
            hmv[u] = pack_mask(S.h0, S.h1, S.h2, (int)(S.a1 >> 32));
            c0v[u] = (int)S.a0; c1v[u] = lo32(S.a1); c2v[u] = S.s0;
            t[0][u] = d0; t[1][u] = d1; t[2][u] = e0; t[3][u] = e1; t[4][u] = dd; t[5][u] = ee; t[6][u] = de;
            vdv[u] = vd; vev[u] = ve;
            if (x + 1 < xend) {
                const int c = x - x0;
                const int vo = row[c], vi = row[c + 2 * r + 1];
                const int po = vo >= 0 ? drow[c] : 0, pi = vi >= 0 ? drow[c + 2 * r + 1] : 0;
                const int Do = delta_x(po), Eo = delta_y(po), Di = delta_x(pi), Ei = delta_y(pi);
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
            for (int q = 0; q < 7; ++q)
                *reinterpret_cast<int4*>(P.c32(3 + q) + o) = make_int4(t[q][0], t[q][1], t[q][2], t[q][3]);
            int64_t* a = P.c64(0) + o;
            int64_t* b = P.c64(1) + o;
            int64_t* c = P.c64(2) + o;
            *reinterpret_cast<longlong2*>(a) = make_longlong2(c2v[0], c2v[1]);
            *reinterpret_cast<longlong2*>(a + 2) = make_longlong2(c2v[2], c2v[3]);
            *reinterpret_cast<longlong2*>(b) = make_longlong2(vdv[0], vdv[1]);
            *reinterpret_cast<longlong2*>(b + 2) = make_longlong2(vdv[2], vdv[3]);
            *reinterpret_cast<longlong2*>(c) = make_longlong2(vev[0], vev[1]);
            *reinterpret_cast<longlong2*>(c + 2) = make_longlong2(vev[2], vev[3]);
        } else {
            for (int u = 0; u < 4 && xb + u < xend; ++u) {
                P.p32[o + u] = hmv[u]; P.c32(1)[o + u] = c0v[u]; P.c32(2)[o + u] = c1v[u];
                for (int q = 0; q < 7; ++q) P.c32(3 + q)[o + u] = t[q][u];
                P.c64(0)[o + u] = c2v[u]; P.c64(1)[o + u] = vdv[u]; P.c64(2)[o + u] = vev[u];
            }
        }
    }
}

// Row pass with the table: tiles of 128 rows x 32 columns; shared memory holds
// the quantised depth tile and the table's tile, each kHThreads x ((32 + 2r) | 1).
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
    load_tile<DT, SF_METHOD_DISPARITY, 2>(dframe, W, r, sc, scale, x0, y0, rows, IW, pitch, tile);
    for (int idx = threadIdx.x; idx < rows * IW; idx += kHThreads) {
        const int ry = idx / IW, cx = idx - ry * IW, x = x0 - r + cx;
        dt[ry * pitch + cx] = (x >= 0 && x < W) ? __ldg(dtab + (size_t)(y0 + ry) * W + x) : 0;
    }
    __syncthreads();
    if ((int)threadIdx.x < rows)
        hpass_row_delta(tile + threadIdx.x * pitch, dt + threadIdx.x * pitch, x0, min(x0 + seg, W), y0 + threadIdx.x,
                        H, r, P, (size_t)f * plane_elems);
}

// Column sums of the table path: the usual disparity sums (DispState on the
// same first planes) plus the table's, i-weighted where the shifted moments
// need it: sum D, sum i D (and E) slide as a pair; sum D j, D^2, E^2, D E,
// v D, v E are plain sums of the row sums.
struct DispDeltaState {
    DispState B;
    const int32_t* pd[7];  // sum D, sum D j, sum E, sum E j, sum D^2, sum E^2, sum D E
    const int64_t* pv[2];  // sum v D, sum v E
    int TD = 0, TDi = 0, TDj = 0, TE = 0, TEi = 0, TEj = 0;
    int64_t TDD = 0, TEE = 0, TDE = 0, TwD = 0, TwE = 0;
    int32_t qo[7] = {0, 0, 0, 0, 0, 0, 0}, qi[7] = {0, 0, 0, 0, 0, 0, 0};
    int64_t wo[2] = {0, 0}, wi[2] = {0, 0};
    __device__ DispDeltaState(const Planes& P) : B(P) {
        for (int q = 0; q < 7; ++q) pd[q] = P.c32(3 + q);
        pv[0] = P.c64(1); pv[1] = P.c64(2);
    }
    __device__ __forceinline__ void init(size_t pb, int rs, int H, int y0, int r) {
        B.init(pb, rs, H, y0, r);
        const int ylo = max(y0 - r, 0), yhi = min(y0 + r, H - 1);
        for (int yy = ylo; yy <= yhi; ++yy) {
            const size_t o = pb + (size_t)yy * rs;
            const int i = yy - y0;
            const int d0 = __ldg(pd[0] + o), e0 = __ldg(pd[2] + o);
            TD += d0; TDi += i * d0; TDj += __ldg(pd[1] + o);
            TE += e0; TEi += i * e0; TEj += __ldg(pd[3] + o);
            TDD += __ldg(pd[4] + o); TEE += __ldg(pd[5] + o); TDE += __ldg(pd[6] + o);
            TwD += __ldg(pv[0] + o); TwE += __ldg(pv[1] + o);
        }
    }
    __device__ __forceinline__ void fetch(size_t pb, int rs, int H, int y, int r) {
        B.fetch(pb, rs, H, y, r);
        const int yo = y - r, yi = y + r + 1;
        for (int q = 0; q < 7; ++q) { qo[q] = 0; qi[q] = 0; }
        wo[0] = wo[1] = wi[0] = wi[1] = 0;
        if (yo >= 0) {
            const size_t o = pb + (size_t)yo * rs;
            for (int q = 0; q < 7; ++q) qo[q] = __ldg(pd[q] + o);
            wo[0] = __ldg(pv[0] + o); wo[1] = __ldg(pv[1] + o);
        }
        if (yi < H) {
            const size_t o = pb + (size_t)yi * rs;
            for (int q = 0; q < 7; ++q) qi[q] = __ldg(pd[q] + o);
            wi[0] = __ldg(pv[0] + o); wi[1] = __ldg(pv[1] + o);
        }
    }
    __device__ __forceinline__ void apply(int r) {
        B.apply(r);
        slide2(TD, TDi, qo[0], qi[0], r);
        TDj += qi[1] - qo[1];
        slide2(TE, TEi, qo[2], qi[2], r);
        TEj += qi[3] - qo[3];
        TDD += (int64_t)qi[4] - qo[4]; TEE += (int64_t)qi[5] - qo[5]; TDE += (int64_t)qi[6] - qo[6];
        TwD += wi[0] - wo[0]; TwE += wi[1] - wo[1];
    }
    __device__ __forceinline__ int count() const { return B.count(); }
};

// The disparity window (as build_disparity) from the shifted offsets
// jh = j + D/256, ih = i + E/256.  With S = 256, every shifted moment is an
// exact integer: J = S sum jh, JJ = S^2 sum jh^2, JI = S^2 sum jh ih,
// WJ = S sum w jh (w in units of qw), and the centred moments
// n JJ - J^2 etc. are formed in int64 before the conversion to float.
__device__ __forceinline__ DispWindowT<float> build_disparity_delta(const DispDeltaState& st, float tx, float ty,
                                                                    float a, float b) {
    using T = float;
    const DispState& s = st.B;
    const int64_t S = kDeltaScale;
    const int n = (int)s.n;
    const int64_t Sj = (int)s.Sj, Si = (int)s.Si, Sjj = (int)s.Sjj, Sji = (int)s.Sji, Sii = (int)s.Sii;
    const int64_t J = S * Sj + st.TD, I = S * Si + st.TE;
    const int64_t JJ = S * S * Sjj + 2 * S * st.TDj + st.TDD;
    const int64_t JI = S * S * Sji + S * (int64_t)st.TEj + S * (int64_t)st.TDi + st.TDE;
    const int64_t II = S * S * Sii + 2 * S * st.TEi + st.TEE;
    const int64_t WJ = S * s.Swj + st.TwD, WI = S * s.Swi + st.TwE;
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
    const T Cjj = Fn<T>::from_i64((int64_t)n * JJ - J * J) * inS2;
    const T Cji = Fn<T>::from_i64((int64_t)n * JI - J * I) * inS2;
    const T Cii = Fn<T>::from_i64((int64_t)n * II - I * I) * inS2;
    const T Cjw = (Fn<T>::from_i64(TWJ) - fJ * t0) * iS;
    const T Ciw = (Fn<T>::from_i64(TWI) - fI * t0) * iS;
    const T Cww = Fn<T>::from_i64(Tww) - fT0 * t0;
    const T wbar = (T)m + t0;
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
template <int DT, bool U4>
__global__ void __launch_bounds__(kVThreads) vpass_delta_kernel(const void* __restrict__ depth, int W, int H, int r,
                                                                Codec scale, const unsigned* __restrict__ vmax_bits,
                                                                int bits, size_t plane_elems, void* planes_base,
                                                                Calib cal, int min_valid, int require_center,
                                                                int band, float* __restrict__ normals,
                                                                float* __restrict__ offsets,
                                                                float* __restrict__ curvature,
                                                                int32_t* __restrict__ counts) {
    const int f = blockIdx.z;
    const int x = blockIdx.x * kVThreads + threadIdx.x;
    if (x >= W) return;
    const size_t fe = (size_t)W * H;
    const size_t dbytes = (DT == SF_DEPTH_F32) ? 4 : 2;
    const void* dframe = static_cast<const char*>(depth) + dbytes * (size_t)f * fe;
    const float q = quantum<DT, SF_METHOD_DISPARITY>(vmax_bits[f], bits, scale);
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
            const DispWindowT<float> w = build_disparity_delta(S, tx, cal.ty[y], cal.a, cal.b);
            FitOut fo;
            if constexpr (U4) {
                const float sw = q * (float)n * w.wbar;
                fo = solve_unit4<float>(w.R11, w.R12, w.R13, w.R22, w.R23, w.R33, sw * w.mx, sw * w.my, sw,
                                        sw * q * w.what);
            } else {
                float l0;
                smallest_eigpair<float>(w.R11, w.R12, w.R13, w.R22, w.R23, w.R33, fo.nx, fo.ny, fo.nz, l0, fo.gap);
                fo.curv = l0;
                fo.d = -(fo.nx * w.mx + fo.ny * w.my + fo.nz) * Fn<float>::rcp(w.what * q);
                orient<float>(fo.nx, fo.ny, fo.nz, fo.d);
            }
            nx = fo.nx; ny = fo.ny; nz = fo.nz; d = fo.d; cu = fo.curv;
        }
        normals[3 * oi] = nx; normals[3 * oi + 1] = ny; normals[3 * oi + 2] = nz;
        offsets[oi] = d; curvature[oi] = cu;
        if (counts) counts[oi] = n;
        if (more) S.apply(r);
    }
}

}  // namespace sf
