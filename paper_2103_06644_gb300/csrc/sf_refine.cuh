// sf_refine.cuh -- precision fallback of the implicit fits (precision modes 1
// and 2): the smallest eigenvector of a window's Schur complement R refined
// to double-float accuracy, and the window's sums corrected for the
// fixed-point rounding of the depth where that rounding could move the normal.
//
// Why: the float32 solve carries an error of about 1e-7 / gamma rad
// (gamma = (lambda1 - lambda0) / lambda2, the eigenvector's sensitivity to
// a perturbation of R, Eq. 4-5), and the fixed-point depth of the exact window
// sums perturbs R like extra sensor noise of half a quantum per pixel.  Near
// degenerate windows (small gamma) therefore need both a more precise solve
// and, for a few of them, sums of the unrounded depth.
//
// How, per queued window (tiers B and C; tier A is the float32 solve):
//   B1. R is built in double-float (pairs of float32, ~48-bit significands)
//       from the exact integer moments, centred exactly as in the float32
//       build (sf_solve.cuh).  The rays come from the FP64 ray table.
//   B2. The float32 eigen-solve of R rounded to float32 gives v0 and v1.
//   B3. One Newton step of the Rayleigh quotient in the basis (v0, u1, u2),
//       u1 = v1 orthogonalised, u2 = v0 x u1: with r_ab = u_a^T R u_b and the
//       Gram matrix g_ab = u_a^T u_b both in double-float (the basis is
//       orthonormal only to float32 rounding, so g enters at first order),
//       sigma = r00 / g00 and
//         [M11 M12; M12 M22] [alpha; beta] = -[r01 - sigma g01; r02 - sigma g02],
//       M_ab = r_ab - sigma g_ab; the normal is v0 + alpha u1 + beta u2.  The
//       residuals and M are formed in double-float before rounding, so the
//       step is accurate to float32 relative to its own size; the error left
//       is of third order in the starting error.  A second step runs when the
//       first moved the vector by more than 1e-2.
//   C.  The first-order effect of the fixed-point rounding on the normal is
//       estimated from the refined eigen-decomposition: rounding errors of
//       +-q/2 per pixel perturb u1^T R v0 by a sum whose standard deviation is
//       q sqrt(d^2 lambda1 + (u1 . c)^2 lambda0) / sqrt(12) (disparity form; c
//       the weighted centroid, d the offset), which divided by lambda1 -
//       lambda0 is the normal's error.  Where 5.5 times that estimate exceeds
//       kTierC rad, the warp re-reads the window's depth, sums the residuals
//       w/q - round(w/q) of its pixels (float32 sums of values below one
//       quantum, added to the exact integers in double-float) and refines
//       again from the corrected moments.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "sf_kernels.cuh"

namespace sf {

// Threshold of tier C: re-sum from the depth where the estimated normal error
// due to the fixed-point rounding (5.5 standard deviations) exceeds this.  It
// sits well below the 1e-3 rad normal tolerance because a normal error dn
// moves the offset d = -n . c by up to |dn| |c|, against a 1e-4 |c| offset
// tolerance.
constexpr float kTierC = kRefineRounding;

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2.  The
// error-free transforms are Knuth's two-sum, Dekker's fast-two-sum (|a| >=
// |b|) and the FMA two-product; every step uses the _rn intrinsics so that the
// compiler cannot contract or reorder them.
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return df{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df dfv(float a) { return df{a, 0.f}; }
__device__ __forceinline__ df operator-(df a) { return df{-a.hi, -a.lo}; }
__device__ __forceinline__ df operator+(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator+(df a, float b) {
    const df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df operator-(df a, float b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
    const df p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ df operator*(df a, float b) {
    const df p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
// a / b: a float32 quotient corrected once by the double-float remainder
__device__ __forceinline__ df operator/(df a, df b) {
    const float ib = __frcp_rn(b.hi);
    const float q1 = __fmul_rn(a.hi, ib);
    const df r = a - b * q1;
    return fast_two_sum(q1, __fmul_rn(r.hi, ib));
}
__device__ __forceinline__ float to_f(df a) { return __fadd_rn(a.hi, a.lo); }

// Exact conversions of integers: 16-bit halves are exact in float32.
__device__ __forceinline__ df df_u32(uint32_t v) {
    return two_sum(__uint2float_rn(v >> 16) * 65536.f, __uint2float_rn(v & 0xffffu));
}
__device__ __forceinline__ df df_i32(int v) {
    return two_sum(__int2float_rn(v >> 16) * 65536.f, __int2float_rn(v & 0xffff));
}
// int64 (to ~48 bits): high word scaled by 2^32 plus the unsigned low word
__device__ __forceinline__ df df_i64(int64_t v) {
    const df h = df_i32((int)(v >> 32));
    return df{h.hi * 4294967296.f, h.lo * 4294967296.f} + df_u32((uint32_t)(uint64_t)v);
}
__device__ __forceinline__ df df_d(double v) {
    const float h = __double2float_rn(v);
    return df{h, __double2float_rn(v - (double)h)};
}

// ---------------------------------------------------------------------------
// Queued windows: the exact moments a flagged window carries from the
// vertical pass to the refinement (10 int64; disparity n, Sj, Si, Sjj, Sji,
// Sii, Sw, Swj, Swi, Sww; standard n, Sz, Szj, Szi, Szz, Szzj, Szzi, Szzjj,
// Szzji, Szzii).
// ---------------------------------------------------------------------------
constexpr int kMomentEntryBytes = 80;

// Symmetric 3x3 in double-float.
struct Sym3df {
    df a11, a12, a13, a22, a23, a33;
};

// The window quantities a refinement produces and consumes.
struct WinGeo {
    float cx, cy, cz;  // centroid direction: d = -n . c (metres)
    float qscale;      // metric per unit of R's eigenvalues (for the curvature scale only)
};

// Centred moments of a disparity-form window in double-float: the integer
// mean m of the fixed-point disparity v, T0 = sum (v - m), Twj = sum (v - m) j,
// Twi = sum (v - m) i, Tww = sum (v - m)^2 (exact integers, or corrected by
// tier C), with the exact mask moments.
struct DispCentred {
    int n, Sj, Si, Sjj, Sji, Sii, m;
    df T0, Twj, Twi, Tww;
    float frac;  // fractional offset of disparity input, added to every value
};

__device__ __forceinline__ DispCentred centre_disparity(const int64_t* v) {
    DispCentred c;
    c.n = (int)v[0]; c.Sj = (int)v[1]; c.Si = (int)v[2]; c.Sjj = (int)v[3]; c.Sji = (int)v[4]; c.Sii = (int)v[5];
    const int64_t Sw = v[6], Swj = v[7], Swi = v[8], Sww = v[9];
    const float inv_n = 1.f / (float)c.n;
    c.m = __float2int_rn(Fn<float>::from_i64(Sw) * inv_n);
    const int64_t T0 = Sw - (int64_t)c.n * c.m;
    c.T0 = df_i64(T0);
    c.Twj = df_i64(Swj - (int64_t)c.m * c.Sj);
    c.Twi = df_i64(Swi - (int64_t)c.m * c.Si);
    c.Tww = df_i64(Sww - (int64_t)c.m * (Sw + T0));
    c.frac = 0.f;
    return c;
}

// The Schur complement R = K Y K^T of the disparity form (see build_disparity
// in sf_solve.cuh for the derivation) in double-float, and the centroid.
__device__ __forceinline__ Sym3df build_disparity_df(const DispCentred& w, df tx, df ty, df a, df b, float qw,
                                                     WinGeo& geo) {
    const float nf = (float)w.n;
    const df inv_n = dfv(1.f) / dfv(nf);
    const df Cjj = df_i32(w.n * w.Sjj - w.Sj * w.Sj) * inv_n;
    const df Cji = df_i32(w.n * w.Sji - w.Sj * w.Si) * inv_n;
    const df Cii = df_i32(w.n * w.Sii - w.Si * w.Si) * inv_n;
    const df Cjw = (w.Twj * nf - w.T0 * (float)w.Sj) * inv_n;
    const df Ciw = (w.Twi * nf - w.T0 * (float)w.Si) * inv_n;
    const df Cww = (w.Tww * nf - w.T0 * w.T0) * inv_n;
    // n wbar (the fractional offset moves the mean only: the centred sums are shift-invariant)
    const df Sw = w.T0 + df_i64((int64_t)w.n * w.m) + two_prod(nf, w.frac);
    const df inv_nw = dfv(1.f) / Sw;
    const df dj = Cjw * inv_nw, di = Ciw * inv_nw, e = Cww * inv_nw;
    const df wbar = Sw * inv_n;
    const df what = wbar + e;
    const df Yjj = Cjj + dj * dj * nf, Yji = Cji + dj * di * nf, Yii = Cii + di * di * nf;
    const df Yjr = -(dj * nf), Yir = -(di * nf);
    const df iw = dfv(1.f) / what;
    const df Yrr = (Cww + e * e * nf) * iw * iw;
    const df jb = df_i32(w.Sj) * inv_n, ib = df_i32(w.Si) * inv_n;
    const df mx = tx + a * (jb + dj), my = ty + b * (ib + di);
    // R = K Y K^T, K = [[a, 0, mx], [0, b, my], [0, 0, 1]]
    const df u1 = a * Yjj + mx * Yjr, u3 = a * Yjr + mx * Yrr;
    const df v1 = b * Yji + my * Yjr, v3 = b * Yir + my * Yrr;
    const df w2 = b * Yii + my * Yir;
    Sym3df R;
    R.a11 = a * u1 + mx * u3;
    R.a12 = a * v1 + mx * v3;
    R.a13 = u3;
    R.a22 = b * w2 + my * v3;
    R.a23 = v3;
    R.a33 = Yrr;
    // weighted centroid c = mhat / (what q) (metres): d = -n . c
    const float iwq = 1.f / (to_f(what) * qw);
    geo.cx = to_f(mx) * iwq; geo.cy = to_f(my) * iwq; geo.cz = iwq;
    geo.qscale = 1.f;
    return R;
}

// Centred moments of a standard-form window: integer mean m of the fixed-point
// depth z, T0 = sum (z - m), Tzz = sum (z - m)^2, Tzj = sum z j (z - m),
// Tzi = sum z i (z - m), and the uncentred Szj, Szi, Szzjj, Szzji, Szzii.
struct StdCentred {
    int n, m;
    df T0, Tzz, Tzj, Tzi, Szj, Szi, Szzjj, Szzji, Szzii;
};

__device__ __forceinline__ StdCentred centre_standard(const int64_t* v) {
    StdCentred c;
    c.n = (int)v[0];
    const int64_t Sz = v[1], Szj = v[2], Szi = v[3], Szz = v[4], Szzj = v[5], Szzi = v[6];
    const float inv_n = 1.f / (float)c.n;
    c.m = __float2int_rn(Fn<float>::from_i64(Sz) * inv_n);
    const int64_t T0 = Sz - (int64_t)c.n * c.m;
    c.T0 = df_i64(T0);
    c.Tzz = df_i64(Szz - (int64_t)c.m * (Sz + T0));
    c.Tzj = df_i64(Szzj - (int64_t)c.m * Szj);
    c.Tzi = df_i64(Szzi - (int64_t)c.m * Szi);
    c.Szj = df_i64(Szj); c.Szi = df_i64(Szi);
    c.Szzjj = df_i64(v[7]); c.Szzji = df_i64(v[8]); c.Szzii = df_i64(v[9]);
    return c;
}

// R = T C T^T of the standard form (solve_standard in sf_solve.cuh) in
// double-float, in units of the fixed-point depth squared, and the centroid.
__device__ __forceinline__ Sym3df build_standard_df(const StdCentred& w, df tx, df ty, df a, df b, float qz,
                                                    WinGeo& geo) {
    const float nf = (float)w.n;
    const df inv_n = dfv(1.f) / dfv(nf);
    const df Czz = (w.Tzz * nf - w.T0 * w.T0) * inv_n;
    const df Cjz = (w.Tzj * nf - w.Szj * w.T0) * inv_n;
    const df Ciz = (w.Tzi * nf - w.Szi * w.T0) * inv_n;
    const df qj = w.Szj * inv_n, qi = w.Szi * inv_n;
    const df Cjj = w.Szzjj - w.Szj * qj, Cji = w.Szzji - w.Szj * qi, Cii = w.Szzii - w.Szi * qi;
    // R = T C T^T, T = [[a, 0, tx], [0, b, ty], [0, 0, 1]]
    const df u1 = a * Cjj + tx * Cjz, u3 = a * Cjz + tx * Czz;
    const df v1 = b * Cji + ty * Cjz, v3 = b * Ciz + ty * Czz;
    const df w2 = b * Cii + ty * Ciz;
    Sym3df R;
    R.a11 = a * u1 + tx * u3;
    R.a12 = a * v1 + tx * v3;
    R.a13 = u3;
    R.a22 = b * w2 + ty * v3;
    R.a23 = v3;
    R.a33 = Czz;
    // centroid (metres): (a qj + tx zb, b qi + ty zb, zb) q
    const df zb = dfv((float)w.m) + w.T0 * inv_n;
    geo.cx = to_f(a * qj + tx * zb) * qz;
    geo.cy = to_f(b * qi + ty * zb) * qz;
    geo.cz = to_f(zb) * qz;
    geo.qscale = qz * qz;
    return R;
}

// ---------------------------------------------------------------------------
// Eigenvectors of the rounded matrix (tier B2).  The trigonometric estimate
// cannot tell two clustered eigenvalues apart: its cos(phi) argument q is
// within float32 rounding of +-1 there, which for a line-like window (lambda0
// ~ lambda1 << lambda2, q -> 1) leaves lambda0 and lambda1 unresolved below
// ~1e-4 of the trace.  So the eigenvector of the isolated eigenvalue (lambda2
// when q >= 0, lambda0 otherwise) is taken first, by a cofactor column and one
// inverse-iteration step, and the other two come from the closed-form 2x2
// eigen-problem of R restricted to its orthogonal complement, whose
// difference of eigenvalues 2 sqrt(h^2 + b^2) involves no cancellation.
// ---------------------------------------------------------------------------
struct Eig3 {
    float v0[3], u1[3], u2[3];
};

__device__ __forceinline__ void normalize3(float* v) {
    const float s = rsqrtf(fmaxf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2], 1e-30f));
    v[0] *= s; v[1] *= s; v[2] *= s;
}
__device__ __forceinline__ void cross3(const float* a, const float* b, float* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ float quad3(float r11, float r12, float r13, float r22, float r23, float r33,
                                       const float* a, const float* b) {
    return a[0] * (r11 * b[0] + r12 * b[1] + r13 * b[2]) + a[1] * (r12 * b[0] + r22 * b[1] + r23 * b[2]) +
           a[2] * (r13 * b[0] + r23 * b[1] + r33 * b[2]);
}

__device__ __forceinline__ Eig3 start_basis(const Sym3df& R) {
    const float tr = to_f(R.a11 + R.a22 + R.a33);
    const float s = tr > 0.f ? 1.f / tr : 1.f;
    const float r11 = to_f(R.a11) * s, r12 = to_f(R.a12) * s, r13 = to_f(R.a13) * s;
    const float r22 = to_f(R.a22) * s, r23 = to_f(R.a23) * s, r33 = to_f(R.a33) * s;
    const float t = 1.f / 3.f;
    const float b11 = r11 - t, b22 = r22 - t, b33 = r33 - t;
    const float p2 = (b11 * b11 + b22 * b22 + b33 * b33 + 2.f * (r12 * r12 + r13 * r13 + r23 * r23)) / 6.f;
    const float p = sqrtf(fmaxf(p2, 1e-30f));
    const float detB = b11 * (b22 * b33 - r23 * r23) - r12 * (r12 * b33 - r23 * r13) + r13 * (r12 * r23 - b22 * r13);
    const float q = fminf(fmaxf(0.5f * detB / (p2 * p + 1e-30f), -1.f), 1.f);
    const float phi = acos_fast(q) * t;
    float sn, cs;
    __sincosf(phi, &sn, &cs);
    const bool top = q >= 0.f;  // lambda2 is the isolated eigenvalue
    const float liso = top ? t + 2.f * p * cs : t - p * (cs + 1.7320508f * sn);
    float e[3];
    null_vector<float>(r11, r12, r13, r22, r23, r33, liso, e[0], e[1], e[2]);
    {
        // one inverse-iteration step with the Rayleigh quotient as shift
        const float lr = quad3(r11, r12, r13, r22, r23, r33, e, e);
        const float a11 = r11 - lr, a22 = r22 - lr, a33 = r33 - lr;
        const float c11 = a22 * a33 - r23 * r23, c22 = a11 * a33 - r13 * r13, c33 = a11 * a22 - r12 * r12;
        const float c12 = r13 * r23 - r12 * a33, c13 = r12 * r23 - r13 * a22, c23 = r12 * r13 - a11 * r23;
        float w[3] = {c11 * e[0] + c12 * e[1] + c13 * e[2], c12 * e[0] + c22 * e[1] + c23 * e[2],
                      c13 * e[0] + c23 * e[1] + c33 * e[2]};
        if (w[0] * w[0] + w[1] * w[1] + w[2] * w[2] > 1e-36f) {
            normalize3(w);
            e[0] = w[0]; e[1] = w[1]; e[2] = w[2];
        }
    }
    // orthonormal basis (pa, pb) of the complement of e
    float ax[3] = {0.f, 0.f, 0.f};
    const float x0 = fabsf(e[0]), x1 = fabsf(e[1]), x2 = fabsf(e[2]);
    ax[(x0 <= x1 && x0 <= x2) ? 0 : (x1 <= x2 ? 1 : 2)] = 1.f;
    float pa[3], pb[3];
    cross3(e, ax, pa);
    normalize3(pa);
    cross3(e, pa, pb);
    normalize3(pb);
    // 2x2 eigen-problem in the complement: [[c11, c12], [c12, c22]]
    const float c11 = quad3(r11, r12, r13, r22, r23, r33, pa, pa);
    const float c12 = quad3(r11, r12, r13, r22, r23, r33, pa, pb);
    const float c22 = quad3(r11, r12, r13, r22, r23, r33, pb, pb);
    const float h = 0.5f * (c11 - c22);
    const float rt = sqrtf(h * h + c12 * c12);
    // eigenvector of the smaller eigenvalue, from the better-conditioned row
    float sx = h >= 0.f ? c12 : rt - h, sy = h >= 0.f ? -(h + rt) : -c12;
    const float ns = sx * sx + sy * sy;
    if (!(ns > 1e-36f)) { sx = 1.f; sy = 0.f; }
    const float is = rsqrtf(fmaxf(sx * sx + sy * sy, 1e-36f));
    sx *= is; sy *= is;
    float vs[3], vl[3];  // smaller and larger eigenvectors of the complement
    for (int c = 0; c < 3; ++c) {
        vs[c] = sx * pa[c] + sy * pb[c];
        vl[c] = -sy * pa[c] + sx * pb[c];
    }
    Eig3 E;
    for (int c = 0; c < 3; ++c) {
        E.v0[c] = top ? vs[c] : e[c];
        E.u1[c] = top ? vl[c] : vs[c];
    }
    normalize3(E.v0);
    float d = E.u1[0] * E.v0[0] + E.u1[1] * E.v0[1] + E.u1[2] * E.v0[2];
    for (int c = 0; c < 3; ++c) E.u1[c] -= d * E.v0[c];
    normalize3(E.u1);
    cross3(E.v0, E.u1, E.u2);
    normalize3(E.u2);
    return E;
}

// R u in double-float for a float32 vector u
__device__ __forceinline__ void mat_vec(const Sym3df& R, const float* u, df* out) {
    out[0] = R.a11 * u[0] + R.a12 * u[1] + R.a13 * u[2];
    out[1] = R.a12 * u[0] + R.a22 * u[1] + R.a23 * u[2];
    out[2] = R.a13 * u[0] + R.a23 * u[1] + R.a33 * u[2];
}
__device__ __forceinline__ df dot_df(const float* u, const df* v) { return v[0] * u[0] + v[1] * u[1] + v[2] * u[2]; }
// exact dot product of two float32 vectors (to double-float rounding)
__device__ __forceinline__ df dot_ff(const float* u, const float* v) {
    return two_prod(u[0], v[0]) + two_prod(u[1], v[1]) + two_prod(u[2], v[2]);
}

struct Refined {
    float n[3];     // unit normal (not yet oriented)
    float l0, l1, l2;  // eigenvalues of R in its own units
    float step;     // |alpha| + |beta| of the last Newton step
    float u1[3];    // second basis vector after the step (for the error estimate)
};

// One Newton step (tier B3) from the basis E; returns the refined vector in E.v0
// and the new basis.  Only the quantities of the (v0, u1) plane need double-
// float: there lambda1 - lambda0 can be 1e-6 of the trace.  The coupling to u2
// (lambda2 - lambda0 of the order of the trace) is a correction of the size of
// the float32 eigenvector error, so its residual, M12 and M22 are float32.
__device__ __forceinline__ Refined newton_step(const Sym3df& R, Eig3& E) {
    df Rv0[3], Ru1[3];
    mat_vec(R, E.v0, Rv0);
    mat_vec(R, E.u1, Ru1);
    const df r00 = dot_df(E.v0, Rv0), r01 = dot_df(E.u1, Rv0), r11 = dot_df(E.u1, Ru1);
    const df g00 = dot_ff(E.v0, E.v0), g01 = dot_ff(E.v0, E.u1), g11 = dot_ff(E.u1, E.u1);
    const float f11 = R.a11.hi, f12 = R.a12.hi, f13 = R.a13.hi, f22 = R.a22.hi, f23 = R.a23.hi, f33 = R.a33.hi;
    const float r02 = quad3(f11, f12, f13, f22, f23, f33, E.u2, E.v0);
    const float r12 = quad3(f11, f12, f13, f22, f23, f33, E.u2, E.u1);
    const float r22 = quad3(f11, f12, f13, f22, f23, f33, E.u2, E.u2);
    const float g02 = E.u2[0] * E.v0[0] + E.u2[1] * E.v0[1] + E.u2[2] * E.v0[2];
    const float g12 = E.u2[0] * E.u1[0] + E.u2[1] * E.u1[1] + E.u2[2] * E.u1[2];
    const float g22 = E.u2[0] * E.u2[0] + E.u2[1] * E.u2[1] + E.u2[2] * E.u2[2];
    const df sigma = r00 / g00;
    const float sg = to_f(sigma);
    const float b1 = -to_f(r01 - sigma * g01), b2 = -(r02 - sg * g02);
    const float M11 = to_f(r11 - sigma * g11), M12 = r12 - sg * g12, M22 = r22 - sg * g22;
    const float det = M11 * M22 - M12 * M12;
    Refined o;
    float al = 0.f, be = 0.f;
    if (M11 > 0.f && M22 > 0.f && det > 0.f) {
        const float id = 1.f / det;
        al = (b1 * M22 - b2 * M12) * id;
        be = (M11 * b2 - M12 * b1) * id;
    } else {
        // the start is not near the minimum: a basis vector with a smaller
        // Rayleigh quotient becomes the start of the next step
        const bool first = M11 <= M22;
        al = first ? 1e3f : 0.f;
        be = first ? 0.f : 1e3f;
    }
    o.n[0] = E.v0[0] + al * E.u1[0] + be * E.u2[0];
    o.n[1] = E.v0[1] + al * E.u1[1] + be * E.u2[1];
    o.n[2] = E.v0[2] + al * E.u1[2] + be * E.u2[2];
    normalize3(o.n);
    o.step = fabsf(al) + fabsf(be);
    // Rayleigh quotient at the new vector: sigma - (alpha b1 + beta b2) / (its squared norm)
    const float nn = 1.f + al * al + be * be;
    o.l0 = sg - (al * b1 + be * b2) / nn;
    const float hm = 0.5f * (M11 + M22), dm = 0.5f * (M11 - M22);
    const float rt = sqrtf(dm * dm + M12 * M12);
    o.l1 = sg + hm - rt;
    o.l2 = sg + hm + rt;
    // next basis: u1 re-orthogonalised against the new vector
    float u[3] = {E.u1[0], E.u1[1], E.u1[2]};
    const float d = u[0] * o.n[0] + u[1] * o.n[1] + u[2] * o.n[2];
    u[0] -= d * o.n[0]; u[1] -= d * o.n[1]; u[2] -= d * o.n[2];
    normalize3(u);
    E.v0[0] = o.n[0]; E.v0[1] = o.n[1]; E.v0[2] = o.n[2];
    E.u1[0] = u[0]; E.u1[1] = u[1]; E.u1[2] = u[2];
    cross3(o.n, u, E.u2);
    normalize3(E.u2);
    o.u1[0] = u[0]; o.u1[1] = u[1]; o.u1[2] = u[2];
    return o;
}

// Tier B: refine until the step is below 1e-2 (at most three steps).
__device__ __forceinline__ Refined refine(const Sym3df& R, Eig3& E) {
    Refined o = newton_step(R, E);
#pragma unroll 1
    for (int it = 0; it < 2 && o.step > 1e-2f; ++it) o = newton_step(R, E);
    return o;
}

// 5.5 standard deviations of the normal's error due to rounding every
// pixel's fixed-point value by up to half a quantum (tier C test).
//   disparity: R is unitless, the perturbation of w (1/m) is q_metric / 2:
//              q sqrt(d^2 l1 + (u1 . c)^2 l0) / (sqrt(12) (l1 - l0))
//   standard:  R in quanta^2, the perturbation of Z is q / 2 (P = Z m):
//              sqrt(d^2 l1 + (u1 . c)^2 l0) / (sqrt(12) |c_z| (l1 - l0))
template <int B>
__device__ __forceinline__ float rounding_error_estimate(const Refined& o, const WinGeo& g, float q, float d) {
    const float uc = o.u1[0] * g.cx + o.u1[1] * g.cy + o.u1[2] * g.cz;
    const float gapl = o.l1 - o.l0;
    if (!(gapl > 0.f)) return INFINITY;
    const float s = sqrtf(fmaxf(d * d * fmaxf(o.l1, 0.f) + uc * uc * fmaxf(o.l0, 0.f), 0.f));
    const float scale = B == SF_METHOD_DISPARITY ? q : 1.f / fmaxf(fabsf(g.cz), 1e-30f);
    return 5.5f * 0.28867513f * scale * s / gapl;
}

// ---------------------------------------------------------------------------
// Tier C: the fixed-point residuals of one window's depth, summed by a warp.
// Lane l covers the window column j = l - r; rows i = -r..r in turn.  For
// every valid pixel with fixed-point value V = round(v / q) and residual
// delta = v / q - V (|delta| <= 1/2):
//   disparity sums: delta, delta j, delta i, (V - m) delta, delta^2
//   standard sums:  delta, delta j, delta i, (V - m) delta, delta^2,
//                   (delta (2V - m) + delta^2) j, .. i,
//                   (2V delta + delta^2) j^2, .. j i, .. i^2
// The residual comes from the same double-float reciprocal and rounding as
// the fixed-point value itself (quant_recip), so V is the value the exact
// sums hold.
// ---------------------------------------------------------------------------
constexpr int kResidSums = 10;

template <int DT, int B>
__device__ __forceinline__ void residual_of(float zin, float sc, const Codec& cd, int& V, float& delta, bool& valid) {
    valid = false; V = 0; delta = 0.f;
    if (DT == SF_DEPTH_DISPARITY_U16) {
        // the disparity form sums the input integers themselves (no residual);
        // the standard form rounds K / w like quant_div
        const int w = disparity_units(zin, cd);
        if (w <= 0) return;
        valid = true;
        if (B == SF_METHOD_DISPARITY) { V = w; return; }
        const float K = sc / cd.scale;
        const float wf = (float)w;
        const float y = rcp_approx(wf + cd.frac);
        const float e = fmaf(-wf, y, 1.f) - cd.frac * y;
        const float p = K * y;
        const float pe = fmaf(K, y, -p);
        const float hr = rintf(p);
        const float f = (p - hr) + fmaf(p, e, pe);
        const float fr = rintf(f);
        V = (int)hr + (int)fr;
        delta = f - fr;
        return;
    }
    if (!depth_valid(zin)) return;
    valid = true;
    if (B == SF_METHOD_DISPARITY) {
        const float y = rcp_approx(zin);
        const float e = fmaf(-zin, y, 1.f);
        const float hi = y * sc;
        const float lo = (y * e) * sc;
        const float hr = rintf(hi);
        const float f = (hi - hr) + lo;
        const float fr = rintf(f);
        V = (int)hr + (int)fr;
        delta = f - fr;
    } else {
        if (DT == SF_DEPTH_U16) { V = (int)zin; return; }  // raw units: exact
        const float t = zin * sc;  // exact: power-of-two scaling
        const float tr = rintf(t);
        V = __float2int_rn(t);
        delta = t - tr;
    }
}

// Every lane returns the warp's totals.  (fx, fy) the window centre, dframe
// the frame's depth, m the integer mean of the window's fixed-point values.
template <int DT, int B>
__device__ __forceinline__ void residual_sums(const void* __restrict__ dframe, int W, int H, int r, float sc,
                                              const Codec& cd, int px, int py, int m, float* out) {
    const int lane = threadIdx.x & 31;
    const int j = lane - r;
    const int x = px + j;
    const bool col = lane <= 2 * r && x >= 0 && x < W;
    float s0 = 0.f, si = 0.f, sv = 0.f, s2 = 0.f, t0 = 0.f, ti = 0.f, u0 = 0.f, ui = 0.f, uii = 0.f, s2i = 0.f;
    // rows in batches of kRows, every load of a batch issued before any is used
    constexpr int kRows = 8;
#pragma unroll 1
    for (int i0 = -r; i0 <= r; i0 += kRows) {
        float zin[kRows];
        bool in[kRows];
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            const int y = py + i0 + u;
            in[u] = col && i0 + u <= r && y >= 0 && y < H;
            zin[u] = in[u] ? load_raw<DT>(dframe, (size_t)y * W + x) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kRows; ++u) {
            int V;
            float dl;
            bool ok;
            residual_of<DT, B>(zin[u], sc, cd, V, dl, ok);
            if (!(in[u] && ok)) continue;
            const float fi = (float)(i0 + u);
            s0 += dl; si += dl * fi; sv += (float)(V - m) * dl; s2 += dl * dl; s2i += dl * dl * fi;
            if (B == SF_METHOD_STANDARD) {
                const float g = (float)(2 * V - m) * dl;  // delta (2V - m)
                const float h = fmaf(2.f * (float)V, dl, dl * dl);  // 2 V delta + delta^2
                t0 += g; ti += g * fi;
                u0 += h; ui += h * fi; uii += h * fi * fi;
            }
        }
    }
    const float fj = (float)j;
    float v[kResidSums];
    v[0] = s0; v[1] = s0 * fj; v[2] = si; v[3] = sv; v[4] = s2;
    v[5] = (t0 + s2) * fj; v[6] = ti + s2i; v[7] = u0 * fj * fj; v[8] = ui * fj; v[9] = uii;
#pragma unroll
    for (int c = 0; c < kResidSums; ++c) {
        float a = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        out[c] = a;
    }
}

__device__ __forceinline__ void correct_disparity(DispCentred& w, const float* s) {
    w.T0 = w.T0 + s[0];
    w.Twj = w.Twj + s[1];
    w.Twi = w.Twi + s[2];
    w.Tww = w.Tww + (two_prod(2.f, s[3]) + s[4]);
}

// z = V + delta: sum z = sum V + sum delta; sum z j (z - m) = Tzj +
// sum (delta (2V - m) + delta^2) j; sum z^2 j^2 = Szzjj + sum (2 V delta + delta^2) j^2 ...
__device__ __forceinline__ void correct_standard(StdCentred& w, const float* s) {
    w.T0 = w.T0 + s[0];
    w.Szj = w.Szj + s[1];
    w.Szi = w.Szi + s[2];
    w.Tzz = w.Tzz + (two_prod(2.f, s[3]) + s[4]);
    w.Tzj = w.Tzj + s[5];
    w.Tzi = w.Tzi + s[6];
    w.Szzjj = w.Szzjj + s[7];
    w.Szzji = w.Szzji + s[8];
    w.Szzii = w.Szzii + s[9];
}

// ---------------------------------------------------------------------------
// A queued window: its position and exact moments, from the moment queue
// (entries below moments_cap) or re-read from the scratch planes.
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void load_window(unsigned idx, const unsigned long long* __restrict__ flags,
                                           const void* __restrict__ moments, unsigned moments_cap, const Planes& P,
                                           size_t plane_elems, int H, int r, int& f, int& x, int& y, int64_t* mo) {
    constexpr int B = base_method(M);
    const unsigned long long e = flags[idx];
    f = (int)(e >> 48); y = (int)((e >> 24) & 0xffffff); x = (int)(e & 0xffffff);
    if (idx < moments_cap) {
        const longlong2* src =
            reinterpret_cast<const longlong2*>(static_cast<const char*>(moments) + (size_t)idx * kMomentEntryBytes);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const longlong2 t = src[c];
            mo[2 * c] = t.x; mo[2 * c + 1] = t.y;
        }
        return;
    }
    const size_t pb = plane_index((size_t)f * plane_elems, x, 0, H);
    if constexpr (B == SF_METHOD_DISPARITY) {
        DispState S(P);
        S.init(pb, kGroup, H, y, r);
        mo[0] = (int64_t)S.n; mo[1] = (int64_t)S.Sj; mo[2] = (int64_t)S.Si; mo[3] = (int64_t)S.Sjj;
        mo[4] = (int64_t)S.Sji; mo[5] = (int64_t)S.Sii; mo[6] = S.Sw; mo[7] = S.Swj; mo[8] = S.Swi; mo[9] = S.Sww;
    } else {
        StdState S(P);
        S.init(pb, kGroup, H, y, r);
        mo[0] = S.n; mo[1] = S.Sz; mo[2] = S.Szj; mo[3] = S.Szi; mo[4] = S.Szz; mo[5] = S.Szzj; mo[6] = S.Szzi;
        mo[7] = S.Szzjj; mo[8] = S.Szzji; mo[9] = S.Szzii;
    }
}

// Refined normal, offset and curvature of one window to its outputs.
__device__ __forceinline__ void write_refined(const Refined& o, const Sym3df& R, float d, size_t oi,
                                              float* __restrict__ normals, float* __restrict__ offsets,
                                              float* __restrict__ curvature) {
    float nx = o.n[0], ny = o.n[1], nz = o.n[2];
    orient<float>(nx, ny, nz, d);
    const float tr = to_f(R.a11 + R.a22 + R.a33);
    normals[3 * oi] = nx; normals[3 * oi + 1] = ny; normals[3 * oi + 2] = nz;
    offsets[oi] = d;
    curvature[oi] = tr > 0.f ? fmaxf(o.l0, 0.f) / tr : 0.f;
}

// ---------------------------------------------------------------------------
// The refinement kernel of precision mode 1: one thread per queued window.
// flag_count[0] is the queue length; windows that need tier C are appended to
// queue_c (length flag_count[1]) for resum_kernel, which writes them.  A
// queued window whose moments were not stored (queue entry beyond the moment
// capacity) recomputes them from the scratch planes.
// ---------------------------------------------------------------------------
template <int DT, int M>
__global__ void __launch_bounds__(128) refine_kernel(const void* __restrict__ depth, int W, int H, int r, Codec cd,
                                                     const unsigned* __restrict__ vmax_bits, int bits,
                                                     size_t plane_elems, int nframes, void* __restrict__ planes_base,
                                                     const double* __restrict__ rays,
                                                     const unsigned long long* __restrict__ flags,
                                                     unsigned* __restrict__ flag_count,
                                                     unsigned* __restrict__ queue_c,
                                                     const void* __restrict__ moments, unsigned moments_cap,
                                                     float* __restrict__ normals,
                                                     float* __restrict__ offsets,
                                                     float* __restrict__ curvature) {
    constexpr int B = base_method(M);
    const unsigned count = *flag_count;
    const int lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    const Planes P(planes_base, (size_t)nframes * plane_elems, planes32<M>());
    const size_t fe = (size_t)W * H;
    const df a = df_d(rays[W + H]), b = df_d(rays[W + H + 1]);
    for (unsigned base = warp * 32u; base < count; base += nwarps * 32u) {
        const unsigned idx = base + lane;
        const bool active = idx < count && flags[idx] != kQueueHole;
        int f = 0, x = 0, y = 0;
        int64_t mo[10];
        if (active) load_window<M>(idx, flags, moments, moments_cap, P, plane_elems, H, r, f, x, y, mo);
        const unsigned vb = active ? vmax_bits[f] : 0u;
        const float q = quantum<DT, B>(vb, bits, cd);
        df tx = dfv(0.f), ty = dfv(0.f);
        typename std::conditional<B == SF_METHOD_DISPARITY, DispCentred, StdCentred>::type wc{};
        WinGeo geo{};
        Sym3df R{};
        Eig3 E{};
        Refined o{};
        float d = 0.f;
        bool needC = false;
        if (active) {
            tx = df_d(rays[x]); ty = df_d(rays[W + y]);
            if constexpr (B == SF_METHOD_DISPARITY) {
                wc = centre_disparity(mo);
                if (DT == SF_DEPTH_DISPARITY_U16) wc.frac = cd.frac;
                R = build_disparity_df(wc, tx, ty, a, b, q, geo);
            } else {
                wc = centre_standard(mo);
                R = build_standard_df(wc, tx, ty, a, b, q, geo);
            }
            E = start_basis(R);
            o = refine(R, E);
            d = -(o.n[0] * geo.cx + o.n[1] * geo.cy + o.n[2] * geo.cz);
            constexpr bool kExactInput = fixed_quantum<DT, B>();
            const float est = rounding_error_estimate<B>(o, geo, q, d);
            needC = !kExactInput && est > kTierC && est < INFINITY;
        }
        // windows to re-sum go to the second queue (the re-sum kernel writes them)
        const unsigned want = __ballot_sync(0xffffffffu, needC);
        unsigned cbase = 0;
        if (lane == 0 && want) cbase = atomicAdd(flag_count + 1, (unsigned)__popc(want));
        cbase = __shfl_sync(0xffffffffu, cbase, 0);
        if (needC) queue_c[cbase + __popc(want & ((1u << lane) - 1u))] = idx;
        if (active && !needC)
            write_refined(o, R, d, (size_t)f * fe + (size_t)y * W + x, normals, offsets, curvature);
    }
}

// ---------------------------------------------------------------------------
// Tier C for the windows of the second queue: each warp takes up to 32
// windows (lane l of warp w: window w + l W for W warps, so that a short
// queue spreads over every warp of the grid), sums the fixed-point residuals
// of each in turn with all its lanes, then every lane corrects its window's
// moments and refines it again.
// ---------------------------------------------------------------------------
template <int DT, int M>
__global__ void __launch_bounds__(128) resum_kernel(const void* __restrict__ depth, int W, int H, int r, Codec cd,
                                                    const unsigned* __restrict__ vmax_bits, int bits,
                                                    size_t plane_elems, int nframes, void* __restrict__ planes_base,
                                                    const double* __restrict__ rays,
                                                    const unsigned long long* __restrict__ flags,
                                                    const unsigned* __restrict__ flag_count,
                                                    const unsigned* __restrict__ queue_c,
                                                    const void* __restrict__ moments, unsigned moments_cap,
                                                    float* __restrict__ normals, float* __restrict__ offsets,
                                                    float* __restrict__ curvature) {
    constexpr int B = base_method(M);
    // queue_c NULL: every window of the first queue (precision mode 2)
    const unsigned count = queue_c ? flag_count[1] : flag_count[0];
    const int lane = threadIdx.x & 31;
    const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nwarps = (gridDim.x * blockDim.x) >> 5;
    const Planes P(planes_base, (size_t)nframes * plane_elems, planes32<M>());
    const size_t fe = (size_t)W * H;
    const size_t dbytes = (DT == SF_DEPTH_F32) ? 4 : 2;
    const df a = df_d(rays[W + H]), b = df_d(rays[W + H + 1]);
    for (unsigned base = warp; base < count; base += nwarps * 32u) {
        const unsigned mine_idx = base + (unsigned)lane * nwarps;
        // (the second queue holds windows; the first may hold holes)
        const bool active = mine_idx < count && (queue_c || flags[mine_idx] != kQueueHole);
        int f = 0, x = 0, y = 0;
        int64_t mo[10];
        if (active) {
            const unsigned idx = queue_c ? queue_c[mine_idx] : mine_idx;
            load_window<M>(idx, flags, moments, moments_cap, P, plane_elems, H, r, f, x, y, mo);
        }
        typename std::conditional<B == SF_METHOD_DISPARITY, DispCentred, StdCentred>::type wc{};
        if (active) {
            if constexpr (B == SF_METHOD_DISPARITY) {
                wc = centre_disparity(mo);
                if (DT == SF_DEPTH_DISPARITY_U16) wc.frac = cd.frac;
            } else {
                wc = centre_standard(mo);
            }
        }
        const unsigned vb = active ? vmax_bits[f] : 0u;
        float mine[kResidSums];
        unsigned todo = __ballot_sync(0xffffffffu, active);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1u;
            const int sf_ = __shfl_sync(0xffffffffu, f, src);
            const int sx = __shfl_sync(0xffffffffu, x, src);
            const int sy = __shfl_sync(0xffffffffu, y, src);
            const int sm = __shfl_sync(0xffffffffu, wc.m, src);
            const unsigned svb = __shfl_sync(0xffffffffu, vb, src);
            const float sc = ldexpf(1.f, quant_exponent(svb, bits));
            const void* dframe = static_cast<const char*>(depth) + dbytes * (size_t)sf_ * fe;
            float s[kResidSums];
            residual_sums<DT, B>(dframe, W, H, r, sc, cd, sx, sy, sm, s);
            if (lane == src) {
#pragma unroll
                for (int c = 0; c < kResidSums; ++c) mine[c] = s[c];
            }
        }
        if (!active) continue;
        const float q = quantum<DT, B>(vb, bits, cd);
        const df tx = df_d(rays[x]), ty = df_d(rays[W + y]);
        WinGeo geo;
        Sym3df R;
        if constexpr (B == SF_METHOD_DISPARITY) {
            correct_disparity(wc, mine);
            R = build_disparity_df(wc, tx, ty, a, b, q, geo);
        } else {
            correct_standard(wc, mine);
            R = build_standard_df(wc, tx, ty, a, b, q, geo);
        }
        Eig3 E = start_basis(R);
        const Refined o = refine(R, E);
        const float d = -(o.n[0] * geo.cx + o.n[1] * geo.cy + o.n[2] * geo.cz);
        write_refined(o, R, d, (size_t)f * fe + (size_t)y * W + x, normals, offsets, curvature);
    }
}

}  // namespace sf
