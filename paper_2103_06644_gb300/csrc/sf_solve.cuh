// sf_solve.cuh -- per-pixel solve of the window plane fit from exact integer
// window moments (device code, included by the kernels).
//
// The window sums reaching this file are exact integers (fixed-point depth or
// disparity, window-relative pixel offsets j = x_q - x_p, i = y_q - y_p), so
// they can be re-centred on the window's own mean without rounding.  Every
// floating-point step below works on centred, well-scaled quantities; no raw
// second moment is ever subtracted in floating point.
#pragma once
#include <cstdint>

namespace sf {

template <typename T>
struct FitOutT {
    T nx, ny, nz, d, curv;
    T gap;  // (lambda1 - lambda0) / lambda2 of the normalised 3x3 matrix
    T tr;   // trace of R in metric units (implicit fits): lambda0 = curv * tr
    // squared estimate of the normal's error due to the fixed-point rounding
    // of the depth (rounding_error2; computed by the solves only on request)
    T qerr2;
};

using FitOut = FitOutT<float>;

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// arccos on [-1, 1] in the form of Abramowitz & Stegun 4.4.45,
// acos(x) = sqrt(1 - x) P(x) for x in [0, 1] and pi - acos(-x) below 0, with
// P a degree-6 polynomial fitted here by iterated weighted least squares
// (max error 9e-8 in exact arithmetic, ~1.5e-6 evaluated in float32).  The
// eigenvalue estimate it feeds is refined afterwards, so this accuracy is
// ample.
__device__ __forceinline__ float acos_fast(float x) {
    const float a = fabsf(x);
    float p = 2.611499099e-03f;
    p = fmaf(p, a, -1.200276181e-02f);
    p = fmaf(p, a, 2.776222800e-02f);
    p = fmaf(p, a, -4.919708793e-02f);
    p = fmaf(p, a, 8.883580176e-02f);
    p = fmaf(p, a, -2.145910804e-01f);
    p = fmaf(p, a, 1.570796239e+00f);
    const float u = 1.f - a;
    const float r = (u > 0.f) ? u * rsqrt_approx(u) * p : 0.f;
    return (x >= 0.f) ? r : 3.14159265f - r;
}

// Elementary functions for the two solve precisions: fast approximations in
// float32 (the refinement steps absorb their error), IEEE operations in FP64.
template <typename T> struct Fn;
template <> struct Fn<float> {
    static __device__ __forceinline__ float rcp(float x) { return rcp_approx(x); }
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrt_approx(x); }
    static __device__ __forceinline__ float sqrt(float x) { return x > 0.f ? x * rsqrt_approx(x) : 0.f; }
    static __device__ __forceinline__ float acos(float x) { return acos_fast(x); }
    static __device__ __forceinline__ void sincos(float x, float* s, float* c) { __sincosf(x, s, c); }
    static __device__ __forceinline__ float tiny() { return 1e-36f; }
    static __device__ __forceinline__ float p2min() { return 1e-20f; }
    // int64 -> float32 from two signed 32-bit parts, v = hi 2^32 + lo with
    // lo in [-2^31, 2^31) (within 1 ulp): a direct 64-bit conversion executes
    // on the FP64 unit, a few per SM and clock.
    static __device__ __forceinline__ float from_i64(int64_t v) {
        const int lo = (int)(uint32_t)v;
        const int hi = (int)((v - (int64_t)lo) >> 32);
        return fmaf((float)hi, 4294967296.f, (float)lo);
    }
};
template <> struct Fn<double> {
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / ::sqrt(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double acos(double x) { return ::acos(x); }
    static __device__ __forceinline__ void sincos(double x, double* s, double* c) { ::sincos(x, s, c); }
    static __device__ __forceinline__ double tiny() { return 1e-280; }
    static __device__ __forceinline__ double p2min() { return 1e-40; }
    static __device__ __forceinline__ double from_i64(int64_t v) { return (double)v; }
};

// Squared estimate, 5.5 standard deviations, of the normal's error (rad) due to
// rounding every pixel's fixed-point value by up to half a unit, for a window
// whose R (upper triangle r..) has eigenvalues l0 <= l1 <= l2, n the unit
// eigenvector of l0 and c the centroid in units where the rounding is half a
// unit (d = -n . c).  A rounding error e_q of pixel q moves n1^T R n0 by
// e_q (d f_q - (n1 . c) r_q) to first order (r_q, f_q the pixel's residuals
// along n0 and n1), so its standard deviation is
// sqrt((d^2 l1 + (n1 . c)^2 l0) / 12) and the normal moves by that over
// l1 - l0.  n1 is not formed: with cp = c + d n = (n1 . c) n1 + (n2 . c) n2,
// (n1 . c)^2 = (l2 |cp|^2 - cp^T R cp) / (l2 - l1), padded by the rounding of
// that difference and bounded by |cp|^2.  The estimate assumes the rounding
// errors of the pixels independent, as they are for depths that do not repeat.
template <typename T>
__device__ __forceinline__ T rounding_error2(T r11, T r12, T r13, T r22, T r23, T r33, T nx, T ny, T nz, T cx, T cy,
                                             T cz, T l0, T l1, T l2) {
    const T d = -(nx * cx + ny * cy + nz * cz);
    const T px = cx + d * nx, py = cy + d * ny, pz = cz + d * nz;
    const T p2 = px * px + py * py + pz * pz;
    const T pRp = px * (r11 * px + r12 * py + r13 * pz) + py * (r12 * px + r22 * py + r23 * pz) +
                  pz * (r13 * px + r23 * py + r33 * pz);
    const T dl = l1 - l0, d21 = l2 - l1;
    T n1c2 = p2;
    if (d21 > T(0)) {
        const T t = (l2 * p2 - pRp + T(5e-7) * l2 * p2) * Fn<T>::rcp(d21);
        n1c2 = t < p2 ? (t > T(0) ? t : T(0)) : p2;
    }
    if (!(dl > T(0))) return T(INFINITY);
    const T num = d * d * (l1 > T(0) ? l1 : T(0)) + n1c2 * (l0 > T(0) ? l0 : T(0));
    return T(2.5208333) * num * Fn<T>::rcp(dl * dl);
}

// Normal error (rad) above which a window's fixed-point rounding sends it to
// the refinement of precision modes 1 and 2 (the tier-C threshold there).
constexpr float kRefineRounding = 3e-5f;

// rounding_error2 where it can exceed thr2, else 0: a cheap upper bound (|cp|^2
// in place of (n1 . c)^2, no reciprocal) screens out the windows it clears,
// and only the others pay for the full estimate.
template <typename T>
__device__ __forceinline__ T rounding_error2_screened(T r11, T r12, T r13, T r22, T r23, T r33, T nx, T ny, T nz,
                                                      T cx, T cy, T cz, T l0, T l1, T l2, T thr2) {
    const T d = -(nx * cx + ny * cy + nz * cz);
    const T px = cx + d * nx, py = cy + d * ny, pz = cz + d * nz;
    const T p2 = px * px + py * py + pz * pz;
    const T dl = l1 - l0;
    const T loose = T(2.5208333) * (d * d * (l1 > T(0) ? l1 : T(0)) + p2 * (l0 > T(0) ? l0 : T(0)));
    if (dl > T(0) && loose <= thr2 * dl * dl) return T(0);
    return rounding_error2<T>(r11, r12, r13, r22, r23, r33, nx, ny, nz, cx, cy, cz, l0, l1, l2);
}

// Null vector of the symmetric matrix M = R - l I: the column of the
// cofactor matrix adj(M) with the largest diagonal entry (each column is a
// cross product of two rows of M; adj(M) = det(M) M^{-1} is dominated by
// (l1 - l)(l2 - l) v0 v0^T, whose diagonal is largest where |v0_i| is, so
// that column is v0 scaled by at least 1/sqrt(3) of its largest value).
template <typename T>
__device__ __forceinline__ void null_vector(T r11, T r12, T r13, T r22, T r23, T r33, T l, T& v0, T& v1, T& v2) {
    const T a11 = r11 - l, a22 = r22 - l, a33 = r33 - l;
    const T c11 = a22 * a33 - r23 * r23, c22 = a11 * a33 - r13 * r13, c33 = a11 * a22 - r12 * r12;
    const T c12 = r13 * r23 - r12 * a33, c13 = r12 * r23 - r13 * a22, c23 = r12 * r13 - a11 * r23;
    const T d1 = c11 < T(0) ? -c11 : c11, d2 = c22 < T(0) ? -c22 : c22, d3 = c33 < T(0) ? -c33 : c33;
    T b0 = c11, b1 = c12, b2 = c13, db = d1;
    if (d2 > db) { b0 = c12; b1 = c22; b2 = c23; db = d2; }
    if (d3 > db) { b0 = c13; b1 = c23; b2 = c33; }
    const T nb = b0 * b0 + b1 * b1 + b2 * b2;
    // l is (numerically) a double root where every cofactor vanishes: any unit
    // vector of the null space (selects rather than a branch)
    const bool deg = !(nb > Fn<T>::tiny());
    const bool e0 = a11 <= a22 && a11 <= a33, e1 = !e0 && a22 <= a33;
    const T s = Fn<T>::rsqrt(deg ? T(1) : nb);
    v0 = deg ? (e0 ? T(1) : T(0)) : b0 * s;
    v1 = deg ? (e1 ? T(1) : T(0)) : b1 * s;
    v2 = deg ? (e0 || e1 ? T(0) : T(1)) : b2 * s;
}

// Smallest eigenpair of a symmetric positive semi-definite 3x3 matrix R
// (upper triangle r11..r33), scaled to unit trace.
//  1. lambda estimate: trigonometric solution of the characteristic cubic
//     (Smith, CACM 4(4):168, 1961).  It stays accurate (~1e-6 absolute) when
//     lambda0 and lambda1 cluster, where Newton's method on the cubic crawls.
//  2. v = null vector of R - lambda I (cofactor column, above).
//  3. Rayleigh quotient lr = v^T R v (insensitive to the cancellation in det R).
//  4. one step of inverse iteration with shift lr: v <- adj(R - lr I) v.
// The eigenvector error left is ~|dR| / (lambda1 - lambda0).
template <typename T>
__device__ __forceinline__ void smallest_eigpair(T r11, T r12, T r13, T r22, T r23, T r33, T& v0, T& v1, T& v2, T& l0,
                                                 T& gap, T* l2 = nullptr) {
    const T tr = r11 + r22 + r33;
    const T s = Fn<T>::rcp(tr);
    r11 *= s; r12 *= s; r13 *= s; r22 *= s; r23 *= s; r33 *= s;
    const T third = T(1) / T(3);
    const T b11 = r11 - third, b22 = r22 - third, b33 = r33 - third;
    const T p2 = (b11 * b11 + b22 * b22 + b33 * b33 + T(2) * (r12 * r12 + r13 * r13 + r23 * r23)) * (T(1) / T(6));
    // p2 <= p2min: three equal eigenvalues (computed with a stand-in p2, then discarded)
    const bool spread = p2 > Fn<T>::p2min();
    const T p2s = spread ? p2 : T(1);
    const T p = Fn<T>::sqrt(p2s);
    const T detB = b11 * (b22 * b33 - r23 * r23) - r12 * (r12 * b33 - r23 * r13) + r13 * (r12 * r23 - b22 * r13);
    T q = T(0.5) * detB * Fn<T>::rcp(p2s * p);
    q = q > T(1) ? T(1) : (q < T(-1) ? T(-1) : q);
    const T phi = Fn<T>::acos(q) * third;  // in [0, pi/3]
    T sn, cs;
    Fn<T>::sincos(phi, &sn, &cs);
    const T lmax = spread ? third + T(2) * p * cs : third;
    const T lmin = spread ? third - p * (cs + T(1.7320508075688772) * sn) : third;
    const T lmid = spread ? T(1) - lmax - lmin : third;
    T a0, a1, a2;
    null_vector<T>(r11, r12, r13, r22, r23, r33, lmin, a0, a1, a2);
    const T t0 = r11 * a0 + r12 * a1 + r13 * a2;
    const T t1 = r12 * a0 + r22 * a1 + r23 * a2;
    const T t2 = r13 * a0 + r23 * a1 + r33 * a2;
    const T lr = a0 * t0 + a1 * t1 + a2 * t2;
    // inverse iteration: w = adj(R - lr I) a
    {
        const T c11 = (r22 - lr) * (r33 - lr) - r23 * r23, c22 = (r11 - lr) * (r33 - lr) - r13 * r13;
        const T c33 = (r11 - lr) * (r22 - lr) - r12 * r12;
        const T c12 = r13 * r23 - r12 * (r33 - lr), c13 = r12 * r23 - r13 * (r22 - lr);
        const T c23 = r12 * r13 - (r11 - lr) * r23;
        const T w0 = c11 * a0 + c12 * a1 + c13 * a2;
        const T w1 = c12 * a0 + c22 * a1 + c23 * a2;
        const T w2 = c13 * a0 + c23 * a1 + c33 * a2;
        const T nw = w0 * w0 + w1 * w1 + w2 * w2;
        const bool okw = nw > Fn<T>::tiny();  // else keep a (an exact eigenvector already)
        const T q = Fn<T>::rsqrt(okw ? nw : T(1));
        a0 = okw ? w0 * q : a0; a1 = okw ? w1 * q : a1; a2 = okw ? w2 * q : a2;
    }
    v0 = a0; v1 = a1; v2 = a2;
    l0 = lr > T(0) ? lr : T(0);
    gap = (lmax > T(0)) ? (lmid - lmin) * Fn<T>::rcp(lmax > T(0) ? lmax : T(1)) : T(0);
    if (l2) *l2 = lmax;
}

// Orientation: d > 0 (the camera centre lies on the positive side); d == 0
// is broken toward n_z < 0, then toward a negative first nonzero component.
template <typename T>
__device__ __forceinline__ void orient(T& nx, T& ny, T& nz, T& d) {
    const bool tie = (nz > T(0)) || (nz == T(0) && (nx > T(0) || (nx == T(0) && ny > T(0))));
    const bool flip = d < T(0) || (d == T(0) && tie);
    nx = flip ? -nx : nx; ny = flip ? -ny : ny; nz = flip ? -nz : nz; d = flip ? -d : d;
}

// Smallest eigenpair as smallest_eigpair, robust to a cluster of the two
// smallest eigenvalues: the trigonometric estimate cannot separate a pair of
// eigenvalues much closer than sqrt(eps) of the trace (its cos argument q is
// within rounding of +-1 there), so the eigenvector of the isolated eigenvalue
// (lambda2 when q >= 0, lambda0 otherwise) is found first (cofactor column and
// one inverse-iteration step), and the other two from the closed-form 2x2
// problem of R on its orthogonal complement, whose eigenvalue difference
// 2 sqrt(h^2 + b^2) involves no cancellation.  l0 and gap as smallest_eigpair.
template <typename T>
__device__ __forceinline__ void smallest_eigpair_iso(T r11, T r12, T r13, T r22, T r23, T r33, T& v0, T& v1, T& v2,
                                                     T& l0, T& gap) {
    const T tr = r11 + r22 + r33;
    const T s = tr > T(0) ? T(1) / tr : T(1);
    r11 *= s; r12 *= s; r13 *= s; r22 *= s; r23 *= s; r33 *= s;
    const T third = T(1) / T(3);
    const T b11 = r11 - third, b22 = r22 - third, b33 = r33 - third;
    const T p2 = (b11 * b11 + b22 * b22 + b33 * b33 + T(2) * (r12 * r12 + r13 * r13 + r23 * r23)) / T(6);
    const T p = Fn<T>::sqrt(p2 > Fn<T>::p2min() ? p2 : Fn<T>::p2min());
    const T detB = b11 * (b22 * b33 - r23 * r23) - r12 * (r12 * b33 - r23 * r13) + r13 * (r12 * r23 - b22 * r13);
    T q = T(0.5) * detB / (p * p * p);
    q = q > T(1) ? T(1) : (q < T(-1) ? T(-1) : q);
    const T phi = Fn<T>::acos(q) * third;
    T sn, cs;
    Fn<T>::sincos(phi, &sn, &cs);
    const bool top = q >= T(0);  // lambda2 is the isolated eigenvalue
    const T liso = top ? third + T(2) * p * cs : third - p * (cs + T(1.7320508075688772) * sn);
    T e0, e1, e2;
    null_vector<T>(r11, r12, r13, r22, r23, r33, liso, e0, e1, e2);
    T le = e0 * (r11 * e0 + r12 * e1 + r13 * e2) + e1 * (r12 * e0 + r22 * e1 + r23 * e2) +
           e2 * (r13 * e0 + r23 * e1 + r33 * e2);
    {
        // one inverse-iteration step, shift = the Rayleigh quotient
        const T a11 = r11 - le, a22 = r22 - le, a33 = r33 - le;
        const T c11 = a22 * a33 - r23 * r23, c22 = a11 * a33 - r13 * r13, c33 = a11 * a22 - r12 * r12;
        const T c12 = r13 * r23 - r12 * a33, c13 = r12 * r23 - r13 * a22, c23 = r12 * r13 - a11 * r23;
        const T w0 = c11 * e0 + c12 * e1 + c13 * e2, w1 = c12 * e0 + c22 * e1 + c23 * e2;
        const T w2 = c13 * e0 + c23 * e1 + c33 * e2;
        const T nw = w0 * w0 + w1 * w1 + w2 * w2;
        if (nw > Fn<T>::tiny()) {
            const T iw = Fn<T>::rsqrt(nw);
            e0 = w0 * iw; e1 = w1 * iw; e2 = w2 * iw;
            le = e0 * (r11 * e0 + r12 * e1 + r13 * e2) + e1 * (r12 * e0 + r22 * e1 + r23 * e2) +
                 e2 * (r13 * e0 + r23 * e1 + r33 * e2);
        }
    }
    // orthonormal basis (pa, pb) of e's complement, from the axis least aligned with e
    const T x0 = e0 < T(0) ? -e0 : e0, x1 = e1 < T(0) ? -e1 : e1, x2 = e2 < T(0) ? -e2 : e2;
    const int ax = (x0 <= x1 && x0 <= x2) ? 0 : (x1 <= x2 ? 1 : 2);
    T pa0 = ax == 0 ? T(0) : (ax == 1 ? -e2 : e1);
    T pa1 = ax == 0 ? e2 : (ax == 1 ? T(0) : -e0);
    T pa2 = ax == 0 ? -e1 : (ax == 1 ? e0 : T(0));
    const T ia = Fn<T>::rsqrt(pa0 * pa0 + pa1 * pa1 + pa2 * pa2);
    pa0 *= ia; pa1 *= ia; pa2 *= ia;
    const T pb0 = e1 * pa2 - e2 * pa1, pb1 = e2 * pa0 - e0 * pa2, pb2 = e0 * pa1 - e1 * pa0;
    // R on the complement: [[c11, c12], [c12, c22]]
    const T ra0 = r11 * pa0 + r12 * pa1 + r13 * pa2, ra1 = r12 * pa0 + r22 * pa1 + r23 * pa2;
    const T ra2 = r13 * pa0 + r23 * pa1 + r33 * pa2;
    const T c11 = pa0 * ra0 + pa1 * ra1 + pa2 * ra2, c12 = pb0 * ra0 + pb1 * ra1 + pb2 * ra2;
    const T c22 = pb0 * (r11 * pb0 + r12 * pb1 + r13 * pb2) + pb1 * (r12 * pb0 + r22 * pb1 + r23 * pb2) +
                  pb2 * (r13 * pb0 + r23 * pb1 + r33 * pb2);
    const T h = T(0.5) * (c11 - c22), m = T(0.5) * (c11 + c22);
    const T rt = Fn<T>::sqrt(h * h + c12 * c12);
    // eigenvector of the smaller eigenvalue of the 2x2, from its better-conditioned row
    T sx = h >= T(0) ? c12 : rt - h, sy = h >= T(0) ? -(h + rt) : -c12;
    const T ns = sx * sx + sy * sy;
    if (!(ns > Fn<T>::tiny())) { sx = T(1); sy = T(0); }
    const T is = Fn<T>::rsqrt(sx * sx + sy * sy);
    sx *= is; sy *= is;
    const T lsm = m - rt, lbg = m + rt;
    if (top) {
        v0 = sx * pa0 + sy * pb0; v1 = sx * pa1 + sy * pb1; v2 = sx * pa2 + sy * pb2;
        l0 = lsm;
        gap = le > T(0) ? (lbg - lsm) / le : T(0);
    } else {
        v0 = e0; v1 = e1; v2 = e2;
        l0 = le;
        gap = lbg > T(0) ? (lsm - le) / lbg : T(0);
    }
    l0 = l0 > T(0) ? l0 : T(0);
}

// The literal constraint of Eq. 4, |(a, b, c, d)| = 1: the smallest eigenpair
// of the 4x4 scatter M = [[A, g], [g^T, s]] (metric units).  With
// alpha = (u, t), the eigen-equations give t = g.u / (lambda - s) and
// (A - g g^T / (s - lambda)) u = lambda u, i.e. u is an eigenvector of
// R_lambda = R - lambda / (s (s - lambda)) g g^T (R the Schur complement) for
// the eigenvalue lambda itself.  Iteration: u = smallest eigenvector of
// R_lambda (a 3x3 solve on the centred R), then lambda = the Rayleigh
// quotient of M at (u, t(u)),
//   rho = [u^T R u + (g.u)^2 lambda^2 / (s (s - lambda)^2)] / [1 + (g.u)^2 / (s - lambda)^2],
// a sum of non-negative terms (no cancellation, where lambda0(R) - c (g.u)^2
// would lose a factor ~d^2 for distant planes).  Rayleigh quotients stay
// >= lambda_min(M) and converge quadratically: 4-5 steps to 1e-6 typically,
// at most kU4Steps.  Outputs: n = u, d = t (|u| = 1), curvature
// lambda / trace(M).  R_lambda can be line-like (two small eigenvalues close
// together), so its 3x3 solves take the isolated eigenvalue first
// (smallest_eigpair_iso), and the iteration divides exactly (IEEE).  Working on R rather than on M keeps the raw second
// moments of M, whose smallest eigenvalue is ~1e-6 of its largest, out of
// the floating-point arithmetic.
constexpr int kU4Steps = 10;

template <typename T>
__device__ __forceinline__ FitOutT<T> solve_unit4(T R11, T R12, T R13, T R22, T R23, T R33, T g0, T g1, T g2, T s) {
    FitOutT<T> o;
    const T g2sum = g0 * g0 + g1 * g1 + g2 * g2;
    T lam = T(0), u0 = T(0), u1 = T(0), u2 = T(1), l0n = T(0), gap = T(0), l0R = T(0), gu = T(0);
#pragma unroll 1
    for (int it = 0;; ++it) {
        const T c = lam / (s * (s - lam));
        const T a11 = R11 - c * g0 * g0, a12 = R12 - c * g0 * g1, a13 = R13 - c * g0 * g2;
        const T a22 = R22 - c * g1 * g1, a23 = R23 - c * g1 * g2, a33 = R33 - c * g2 * g2;
        // R_lambda may be indefinite: its eigenvalues are >= lambda0(R) - c|g|^2, so a shift by
        // the excess keeps it semi-definite with the same eigenvectors (0 near the root)
        const T ex = c * g2sum - l0R;
        const T sh = ex > T(0) ? ex : T(0);
        smallest_eigpair_iso<T>(a11 + sh, a12, a13, a22 + sh, a23, a33 + sh, u0, u1, u2, l0n, gap);
        const T uRu = u0 * (R11 * u0 + R12 * u1 + R13 * u2) + u1 * (R12 * u0 + R22 * u1 + R23 * u2) +
                      u2 * (R13 * u0 + R23 * u1 + R33 * u2);
        if (it == 0) l0R = uRu > T(0) ? uRu : T(0);
        gu = g0 * u0 + g1 * u1 + g2 * u2;
        const T sl = s - lam;
        const T isl2 = T(1) / (sl * sl);
        T rho = (uRu + gu * gu * lam * lam / s * isl2) / (T(1) + gu * gu * isl2);
        const T top = s * T(0.999999);
        rho = rho < T(0) ? T(0) : (rho > top ? top : rho);
        const T step = rho > lam ? rho - lam : lam - rho;
        const bool done = step <= T(1e-6) * rho || it == kU4Steps;
        lam = rho;
        if (done) break;
    }
    o.nx = u0; o.ny = u1; o.nz = u2;
    o.d = gu / (lam - s);
    orient<T>(o.nx, o.ny, o.nz, o.d);
    const T trM = R11 + R22 + R33 + g2sum * Fn<T>::rcp(s) + s;
    o.curv = lam * Fn<T>::rcp(trM);
    o.gap = gap;
    o.tr = trM;
    return o;
}

// Disparity (RGBD-space) implicit fit of one window, Eq. 12 / Eq. 14.
//
// Inputs are exact window sums over the valid pixels q of the window:
//   n, Sj = sum j, Si = sum i, Sjj = sum j^2, Sji = sum j i, Sii = sum i^2
//   Sw = sum w, Swj = sum w j, Swi = sum w i, Sww = sum w^2
// where w = 1/Z is stored as an integer in units of qw (w_metric = qw * w).
// tx, ty are the ray tangents of the window centre, a = 1/fx, b = 1/fy.
//
// With m_q = [tx + a j, ty + b i, 1] the Schur complement of the 4x4 scatter
// [[sum m m^T, sum w m], [., sum w^2]] is the 1/Z^2-weighted covariance of
// the window's 3D points.  Writing the weighted centroid ray
// mhat = [tx + a jhat, ty + b ihat, 1] with jhat = sum w j / sum w and
// what = sum w^2 / sum w, that complement equals K Y K^T with
//   K = [[a, 0, mhat_x], [0, b, mhat_y], [0, 0, 1]],
//   Y = sum y y^T over y = [j - jhat, i - ihat, (what - w)/what],
// and every entry of Y follows from the centred integer moments below.
// The offset is d = -(n . mhat) / what.
template <typename T>
struct DispWindowT {
    T R11, R12, R13, R22, R23, R33;  // Schur complement in ray units (K Y K^T)
    T mx, my;                        // weighted centroid ray mhat = [mx, my, 1]
    T what;                          // sum w^2 / sum w, in units of qw
    T wbar;                          // mean w, in units of qw
};
using DispWindow = DispWindowT<float>;

template <typename T>
__device__ __forceinline__ DispWindowT<T> build_disparity(T nf, T fSj, T fSi, T fSjj, T fSji, T fSii, int64_t Sw,
                                                          int64_t Swj, int64_t Swi, int64_t Sww, T tx, T ty, T a,
                                                          T b, T wfrac = T(0)) {
    // the mask moments are exact integers held in T (all < 2^24)
    const T inv_n = Fn<T>::rcp(nf);
    const int n = (int)nf, Sj = (int)fSj, Si = (int)fSi;
    // exact re-centring on an integer m near the mean disparity (m < 2^31)
    const int m = __float2int_rn((float)(Fn<T>::from_i64(Sw) * inv_n));
    const int64_t T0 = Sw - (int64_t)n * m;
    const int64_t Tww = Sww - (int64_t)m * (Sw + T0);            // sum (w - m)^2
    const int64_t Twj = Swj - (int64_t)m * Sj;                   // sum (w - m) j
    const int64_t Twi = Swi - (int64_t)m * Si;                   // sum (w - m) i
    const T fT0 = (T)(int)T0;                                    // |T0| < 2^31
    const T t0 = fT0 * inv_n;
    const T jb = fSj * inv_n, ib = fSi * inv_n;
    const T Cjj = fSjj - fSj * jb;
    const T Cji = fSji - fSj * ib;
    const T Cii = fSii - fSi * ib;
    const T Cjw = Fn<T>::from_i64(Twj) - fSj * t0;
    const T Ciw = Fn<T>::from_i64(Twi) - fSi * t0;
    const T Cww = Fn<T>::from_i64(Tww) - fT0 * t0;
    // mean disparity (units of qw); wfrac shifts every value alike (disparity
    // input with a fractional offset) and so leaves the covariances unchanged
    const T wbar = (T)m + t0 + wfrac;
    const T inv_nw = Fn<T>::rcp(nf * wbar);
    const T dj = Cjw * inv_nw;     // jhat - jbar
    const T di = Ciw * inv_nw;     // ihat - ibar
    const T e = Cww * inv_nw;      // what - wbar
    const T what = wbar + e;
    const T Yjj = Cjj + nf * dj * dj;
    const T Yji = Cji + nf * dj * di;
    const T Yii = Cii + nf * di * di;
    const T Yjr = -nf * dj;
    const T Yir = -nf * di;
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

template <typename T = float, bool U4 = false, bool kEst = false>
__device__ __forceinline__ FitOutT<T> solve_disparity(T nf, T fSj, T fSi, T fSjj, T fSji, T fSii, int64_t Sw,
                                                      int64_t Swj, int64_t Swi, int64_t Sww, T qw, T tx, T ty, T a,
                                                      T b, T wfrac = T(0)) {
    const DispWindowT<T> w = build_disparity<T>(nf, fSj, fSi, fSjj, fSji, fSii, Sw, Swj, Swi, Sww, tx, ty, a, b,
                                                wfrac);
    if constexpr (U4) {
        // g = sum w m = (sum w) mhat, s = sum w^2 = n wbar what (metric)
        const T sw = qw * nf * w.wbar;
        return solve_unit4<T>(w.R11, w.R12, w.R13, w.R22, w.R23, w.R33, sw * w.mx, sw * w.my, sw,
                              sw * qw * w.what);
    }
    FitOutT<T> o;
    T l0, l2n;
    smallest_eigpair<T>(w.R11, w.R12, w.R13, w.R22, w.R23, w.R33, o.nx, o.ny, o.nz, l0, o.gap, &l2n);
    o.curv = l0;
    o.tr = w.R11 + w.R22 + w.R33;  // R = K Y K^T is the Schur complement itself (no unit)
    o.qerr2 = T(0);
    if constexpr (kEst) {
        // the weighted centroid mhat / (what qw) in units of 1 / qw
        const T iw = Fn<T>::rcp(w.what);
        o.qerr2 = rounding_error2_screened<T>(w.R11, w.R12, w.R13, w.R22, w.R23, w.R33, o.nx, o.ny, o.nz,
                                              w.mx * iw, w.my * iw, iw, l0 * o.tr, (l0 + o.gap * l2n) * o.tr,
                                              l2n * o.tr, T(kRefineRounding) * T(kRefineRounding));
    }
    o.d = -(o.nx * w.mx + o.ny * w.my + o.nz) * Fn<T>::rcp(w.what * qw);
    orient<T>(o.nx, o.ny, o.nz, o.d);
    return o;
}

// Standard implicit fit of one window, Eq. 3-6, from exact integer sums of
// z = Z / qz (fixed point) with window-relative offsets j, i:
//   n, Sz, Szj, Szi, Szz, Szzj, Szzi, Szzjj, Szzji, Szzii.
// P_q = Z_q m_q = T [Z j, Z i, Z] with T = [[a, 0, tx], [0, b, ty], [0, 0, 1]],
// so the covariance of the points is T C T^T, C the covariance of
// [z j, z i, z] (re-centred on an integer near the mean depth first).
template <typename T>
struct StdWindowT {
    T R11, R12, R13, R22, R23, R33;  // covariance of the window's points (units of qz^2)
    T px, py, zb;                    // their centroid (units of qz)
};

template <typename T = float>
__device__ __forceinline__ StdWindowT<T> build_standard(T nf, int64_t Sz, int64_t Szj, int64_t Szi, int64_t Szz,
                                                        int64_t Szzj, int64_t Szzi, int64_t Szzjj, int64_t Szzji,
                                                        int64_t Szzii, T tx, T ty, T a, T b) {
    const T inv_n = Fn<T>::rcp(nf);
    const int n = (int)nf;
    const int m = __float2int_rn((float)(Fn<T>::from_i64(Sz) * inv_n));       // m < 2^31
    const int64_t T0 = Sz - (int64_t)n * m;
    const int64_t Tzz = Szz - (int64_t)m * (Sz + T0);           // sum (z - m)^2
    const int64_t Tzj = Szzj - (int64_t)m * Szj;                // sum z j (z - m)
    const int64_t Tzi = Szzi - (int64_t)m * Szi;                // sum z i (z - m)
    const T t0 = (T)(int)T0 * inv_n;                            // zbar - m
    const T fSzj = Fn<T>::from_i64(Szj), fSzi = Fn<T>::from_i64(Szi);
    const T Czz = Fn<T>::from_i64(Tzz) - (T)(int)T0 * t0;
    const T Cjz = Fn<T>::from_i64(Tzj) - fSzj * t0;
    const T Ciz = Fn<T>::from_i64(Tzi) - fSzi * t0;
    const T qj = fSzj * inv_n, qi = fSzi * inv_n;               // means of z j, z i
    const T Cjj = Fn<T>::from_i64(Szzjj) - fSzj * qj;
    const T Cji = Fn<T>::from_i64(Szzji) - fSzj * qi;
    const T Cii = Fn<T>::from_i64(Szzii) - fSzi * qi;
    StdWindowT<T> w;
    w.R11 = a * a * Cjj + T(2) * a * tx * Cjz + tx * tx * Czz;
    w.R12 = a * b * Cji + a * ty * Cjz + b * tx * Ciz + tx * ty * Czz;
    w.R13 = a * Cjz + tx * Czz;
    w.R22 = b * b * Cii + T(2) * b * ty * Ciz + ty * ty * Czz;
    w.R23 = b * Ciz + ty * Czz;
    w.R33 = Czz;
    w.zb = (T)m + t0;
    w.px = a * qj + tx * w.zb;
    w.py = b * qi + ty * w.zb;
    return w;
}

template <typename T = float, bool U4 = false, bool kEst = false>
__device__ __forceinline__ FitOutT<T> solve_standard(T nf, int64_t Sz, int64_t Szj, int64_t Szi, int64_t Szz,
                                                     int64_t Szzj, int64_t Szzi, int64_t Szzjj, int64_t Szzji,
                                                     int64_t Szzii, T qz, T tx, T ty, T a, T b) {
    const StdWindowT<T> w = build_standard<T>(nf, Sz, Szj, Szi, Szz, Szzj, Szzi, Szzjj, Szzji, Szzii, tx, ty, a, b);
    const T R11 = w.R11, R12 = w.R12, R13 = w.R13, R22 = w.R22, R23 = w.R23, R33 = w.R33;
    const T px = w.px, py = w.py, zb = w.zb;
    if constexpr (U4) {
        // metric: R qz^2, g = sum P = n qz (px, py, zb), s = n
        const T q2 = qz * qz, gn = nf * qz;
        return solve_unit4<T>(R11 * q2, R12 * q2, R13 * q2, R22 * q2, R23 * q2, R33 * q2, gn * px, gn * py,
                              gn * zb, nf);
    }
    FitOutT<T> o;
    T l0, l2n;
    smallest_eigpair<T>(R11, R12, R13, R22, R23, R33, o.nx, o.ny, o.nz, l0, o.gap, &l2n);
    o.curv = l0;
    const T trR = R11 + R22 + R33;
    o.tr = trR * qz * qz;  // R is in units of the fixed-point depth squared
    o.qerr2 = T(0);
    if constexpr (kEst) {
        // the centroid (px, py, zb) qz over its depth zb qz: a rounding of half a
        // unit of z perturbs P by m / 2, m = P / Z the pixel's ray
        const T iz = Fn<T>::rcp(zb);
        o.qerr2 = rounding_error2_screened<T>(R11, R12, R13, R22, R23, R33, o.nx, o.ny, o.nz, px * iz, py * iz,
                                              T(1), l0 * trR, (l0 + o.gap * l2n) * trR, l2n * trR,
                                              T(kRefineRounding) * T(kRefineRounding));
    }
    o.d = -(o.nx * px + o.ny * py + o.nz * zb) * qz;
    orient<T>(o.nx, o.ny, o.nz, o.d);
    return o;
}

// ---------------------------------------------------------------------------
// Explicit fits (Section I.D, Section II.B).  Both are linear least squares
// on the same exact window moments; the regression is done on centred
// quantities (a 2x2 system for the two slopes, the intercept from the means).
// A window without a unique fit (collinear pixels) returns ok = false.
// Third output: mean squared residual in the fit's own units.
// ---------------------------------------------------------------------------

// Eq. 15-16: 1/Z = ax tx + ay ty + ac.  With w = qw * omega and
// tx = tx_p + a j, the regression of omega on (j, i) gives the slopes per
// pixel; the plane ax tx + ay ty + ac - 1/Z = 0 is n.P + d = 0 with
// n = -(ax, ay, ac)/|.|, d = 1/|(ax, ay, ac)|.
// Exact rank test of the image coordinates of a window's valid pixels:
// n^2 det cov(j, i) == 0 iff they are collinear (every moment is an integer).
template <typename T>
__device__ __forceinline__ bool pixels_span_plane(T nf, T fSj, T fSi, T fSjj, T fSji, T fSii) {
    const int n = (int)nf, Sj = (int)fSj, Si = (int)fSi;
    const int64_t cjj = (int64_t)n * (int)fSjj - (int64_t)Sj * Sj;
    const int64_t cii = (int64_t)n * (int)fSii - (int64_t)Si * Si;
    const int64_t cji = (int64_t)n * (int)fSji - (int64_t)Sj * Si;
    return cjj * cii - cji * cji != 0;
}

template <typename T = float>
__device__ __forceinline__ FitOutT<T> solve_explicit_disparity(T nf, T fSj, T fSi, T fSjj, T fSji, T fSii,
                                                               int64_t Sw, int64_t Swj, int64_t Swi, int64_t Sww,
                                                               T qw, T tx, T ty, T a, T b, bool& ok,
                                                               T wfrac = T(0)) {
    FitOutT<T> o;
    const int n = (int)nf, Sj = (int)fSj, Si = (int)fSi;
    ok = pixels_span_plane<T>(nf, fSj, fSi, fSjj, fSji, fSii);
    const T inv_n = Fn<T>::rcp(nf);
    const int m = __float2int_rn((float)(Fn<T>::from_i64(Sw) * inv_n));
    const int64_t T0 = Sw - (int64_t)n * m;
    const int64_t Tww = Sww - (int64_t)m * (Sw + T0);
    const int64_t Twj = Swj - (int64_t)m * Sj;
    const int64_t Twi = Swi - (int64_t)m * Si;
    const T fT0 = (T)(int)T0;
    const T t0 = fT0 * inv_n;
    const T jb = fSj * inv_n, ib = fSi * inv_n;
    const T Cjj = fSjj - fSj * jb, Cji = fSji - fSj * ib, Cii = fSii - fSi * ib;
    const T Cjw = Fn<T>::from_i64(Twj) - fSj * t0, Ciw = Fn<T>::from_i64(Twi) - fSi * t0, Cww = Fn<T>::from_i64(Tww) - fT0 * t0;
    const T idet = Fn<T>::rcp(Cjj * Cii - Cji * Cji);
    const T bj = (Cii * Cjw - Cji * Ciw) * idet;   // d omega / d j
    const T bi = (Cjj * Ciw - Cji * Cjw) * idet;   // d omega / d i
    const T bc = ((T)m + t0 + wfrac) - bj * jb - bi * ib;  // omega at the window centre pixel
    const T ax = qw * bj * Fn<T>::rcp(a), ay = qw * bi * Fn<T>::rcp(b);
    const T ac = qw * bc - ax * tx - ay * ty;
    const T s = Fn<T>::rsqrt(ax * ax + ay * ay + ac * ac);
    o.nx = -ax * s; o.ny = -ay * s; o.nz = -ac * s;
    o.d = s;
    orient<T>(o.nx, o.ny, o.nz, o.d);
    const T res = Cww - bj * Cjw - bi * Ciw;
    o.curv = (res > T(0) ? res : T(0)) * qw * qw * inv_n;
    o.gap = T(1);
    o.tr = T(0);
    return o;
}

// Eq. 7-9: Z = ae X + be Y + ce, regression of Z on (X, Y) from the
// covariance of the window's points (as in solve_standard).  The plane
// ae X + be Y - Z + ce = 0 is normalised and oriented.  fSj .. fSii are the
// image moments of the valid pixels (rank test).
template <typename T = float>
__device__ __forceinline__ FitOutT<T> solve_explicit_standard(T nf, T fSj, T fSi, T fSjj, T fSji, T fSii,
                                                              int64_t Sz, int64_t Szj, int64_t Szi, int64_t Szz,
                                                              int64_t Szzj, int64_t Szzi, int64_t Szzjj,
                                                              int64_t Szzji, int64_t Szzii, T qz, T tx, T ty, T a,
                                                              T b, bool& ok) {
    FitOutT<T> o;
    const T inv_n = Fn<T>::rcp(nf);
    const int n = (int)nf;
    const int m = __float2int_rn((float)(Fn<T>::from_i64(Sz) * inv_n));
    const int64_t T0 = Sz - (int64_t)n * m;
    const int64_t Tzz = Szz - (int64_t)m * (Sz + T0);
    const int64_t Tzj = Szzj - (int64_t)m * Szj;
    const int64_t Tzi = Szzi - (int64_t)m * Szi;
    const T t0 = (T)(int)T0 * inv_n;
    const T fSzj = Fn<T>::from_i64(Szj), fSzi = Fn<T>::from_i64(Szi);
    const T Czz = Fn<T>::from_i64(Tzz) - (T)(int)T0 * t0;
    const T Cjz = Fn<T>::from_i64(Tzj) - fSzj * t0;
    const T Ciz = Fn<T>::from_i64(Tzi) - fSzi * t0;
    const T qj = fSzj * inv_n, qi = fSzi * inv_n;
    const T Cjj = Fn<T>::from_i64(Szzjj) - fSzj * qj, Cji = Fn<T>::from_i64(Szzji) - fSzj * qi, Cii = Fn<T>::from_i64(Szzii) - fSzi * qi;
    const T Cxx = a * a * Cjj + T(2) * a * tx * Cjz + tx * tx * Czz;
    const T Cxy = a * b * Cji + a * ty * Cjz + b * tx * Ciz + tx * ty * Czz;
    const T Cxz = a * Cjz + tx * Czz;
    const T Cyy = b * b * Cii + T(2) * b * ty * Ciz + ty * ty * Czz;
    const T Cyz = b * Ciz + ty * Czz;
    const T det = Cxx * Cyy - Cxy * Cxy;
    ok = pixels_span_plane<T>(nf, fSj, fSi, fSjj, fSji, fSii);
    const T idet = Fn<T>::rcp(det);
    const T ae = (Cyy * Cxz - Cxy * Cyz) * idet;
    const T be = (Cxx * Cyz - Cxy * Cxz) * idet;
    const T zb = (T)m + t0;
    const T px = a * qj + tx * zb, py = b * qi + ty * zb;
    const T ce = (zb - ae * px - be * py) * qz;
    const T s = Fn<T>::rsqrt(ae * ae + be * be + T(1));
    o.nx = ae * s; o.ny = be * s; o.nz = -s;
    o.d = ce * s;
    orient<T>(o.nx, o.ny, o.nz, o.d);
    const T res = Czz - ae * Cxz - be * Cyz;
    o.curv = (res > T(0) ? res : T(0)) * qz * qz * inv_n;
    o.gap = T(1);
    o.tr = T(0);
    return o;
}

// ---------------------------------------------------------------------------
// Backward: adjoint of the implicit fit of one window with respect to its
// Schur complement R (any units), for upstream gradients gn (normal), gk
// (curvature).  n = sigma v0 with the orientation sign sigma locally constant.
//   eigenvector:  dv0 = -(R - l0 I)^+ dR v0, so Rbar = -sym(x v0^T) with
//                 x = (R - l0 I + c v0 v0^T)^{-1} vbar_perp (c > 0 any: the
//                 v0 direction is projected out of vbar);
//   curvature:    kappa = l0 / tr R: Rbar += gk (v0 v0^T / tr - l0 / tr^2 I).
// Returns Rbar (symmetric, upper triangle).  vbar must already hold the
// gradient with respect to the oriented normal, including the offset term.
// ---------------------------------------------------------------------------
struct Sym3 { float a11, a12, a13, a22, a23, a33; };

__device__ __forceinline__ Sym3 eig_adjoint(float r11, float r12, float r13, float r22, float r23, float r33,
                                            float v0, float v1, float v2, float l0, float tr, float b0, float b1,
                                            float b2, float gk) {
    // project vbar onto the complement of v0
    const float pv = b0 * v0 + b1 * v1 + b2 * v2;
    b0 -= pv * v0; b1 -= pv * v1; b2 -= pv * v2;
    // M = R - l0 I + tr v0 v0^T (symmetric, positive on the complement)
    const float m11 = r11 - l0 + tr * v0 * v0, m12 = r12 + tr * v0 * v1, m13 = r13 + tr * v0 * v2;
    const float m22 = r22 - l0 + tr * v1 * v1, m23 = r23 + tr * v1 * v2, m33 = r33 - l0 + tr * v2 * v2;
    const float c11 = m22 * m33 - m23 * m23, c12 = m13 * m23 - m12 * m33, c13 = m12 * m23 - m13 * m22;
    const float c22 = m11 * m33 - m13 * m13, c23 = m12 * m13 - m11 * m23, c33 = m11 * m22 - m12 * m12;
    const float det = m11 * c11 + m12 * c12 + m13 * c13;
    Sym3 o;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (det != 0.f) {
        const float id = 1.f / det;
        x0 = (c11 * b0 + c12 * b1 + c13 * b2) * id;
        x1 = (c12 * b0 + c22 * b1 + c23 * b2) * id;
        x2 = (c13 * b0 + c23 * b1 + c33 * b2) * id;
    }
    o.a11 = -x0 * v0; o.a22 = -x1 * v1; o.a33 = -x2 * v2;
    o.a12 = -0.5f * (x0 * v1 + x1 * v0);
    o.a13 = -0.5f * (x0 * v2 + x2 * v0);
    o.a23 = -0.5f * (x1 * v2 + x2 * v1);
    if (tr > 0.f) {
        const float it = 1.f / tr, li = l0 * it * it;
        o.a11 += gk * (v0 * v0 * it - li); o.a22 += gk * (v1 * v1 * it - li); o.a33 += gk * (v2 * v2 * it - li);
        o.a12 += gk * v0 * v1 * it; o.a13 += gk * v0 * v2 * it; o.a23 += gk * v1 * v2 * it;
    }
    return o;
}

}  // namespace sf
