// elbm_device.cuh -- device-side building blocks of the essentially entropic
// lattice Boltzmann step (arXiv:2203.12946) for sm_103a.
//
// Contents
//   * lattice constants of D2Q9 / D3Q27 as compile-time functions of the
//     velocity index (tensor products of D1Q3, Sec. I);
//   * storage traits (FP64, FP32, FP16/BF16 deviation storage);
//   * node_collide: moments, product-form entropic equilibrium, departures x,
//     the closed-form path length of Sec. III / Appendix C with the cutoff and
//     positivity clamp of Appendix D, evaluated on registers;
//   * FP64 helpers for the diagnostics (Eq. hdef, Eq. deltaH3).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace eelbm {

// ---------------------------------------------------------------------------
// Lattice: velocity i enumerates (c_x, c_y[, c_z]) in {-1,0,1}^D with the last
// axis fastest.  Weights are products of the D1Q3 weights {1/6, 4/6, 1/6}.
// ---------------------------------------------------------------------------
template <int D>
struct Lattice {
    static constexpr int Q = D == 2 ? 9 : 27;
};

__host__ __device__ constexpr int vel(int D, int i, int a)
{
    return (a == D - 1 ? i : (a == D - 2 ? i / 3 : i / 9)) % 3 - 1;
}

__host__ __device__ constexpr double weight(int D, int i)
{
    double w = 1.0;
    for (int a = 0; a < D; ++a) w *= (vel(D, i, a) == 0 ? 4.0 / 6.0 : 1.0 / 6.0);
    return w;
}

// Every weight is a power of two times W = 6^-D: w_i = k_i W, k_i in {1, 4, 16, 64}
// (Sec. I, products of the D1Q3 weights 1/6, 4/6, 1/6).  In floating point
// k_i T(W) is then exactly T(w_i), and with r = rho W formed once per node,
// k_i r = w_i rho up to one rounding of r shared by every population.
__host__ __device__ constexpr double weight_unit(int D) { return D == 2 ? 1.0 / 36.0 : 1.0 / 216.0; }
__host__ __device__ constexpr double weight_k(int D, int i)
{
    double k = 1.0;
    for (int a = 0; a < D; ++a) k *= (vel(D, i, a) == 0 ? 4.0 : 1.0);
    return k;
}
template <int D, class T>
__host__ __device__ constexpr T weight_unit_lo()
{
    return T(weight_unit(D) - double(T(weight_unit(D))));
}

// Sum of the weights after rounding to T, minus one (zero in exact arithmetic).
template <int D, class T>
__host__ __device__ constexpr double weight_sum_error()
{
    double s = 0.0;
    for (int i = 0; i < (D == 2 ? 9 : 27); ++i) s += double(T(weight(D, i)));
    return s - 1.0;
}

struct Geometry {
    int nx, ny, nz;
    int64_t N;
};

// Near-equilibrium cutoff of Appendix D (strict test |x|max < 1e-3).
constexpr double kCutoff = 1e-3;

enum { kModeHigher = 0, kModeLower = 1, kModeLBGK = 2, kModeIterate1 = 3 };
enum { kBranchCutoff = 0, kBranchSolved = 1, kBranchClamped = 2 };

struct CollideParams {
    double beta;
    int mode;      // kMode*
    int cutoff;    // 1 = Appendix D shortcut on
    int b_variant; // 0 = derived denominators (alpha_L beta x), 1 = printed (alpha_L x)
    double rho0;   // reference density of deviation storage
    double force[3] = {0.0, 0.0, 0.0}; // uniform body force (not from the paper), used by the forced kernels
    float beta_f = 0.0f;  // beta rounded to FP32 once on the host (no FP64 conversion per thread)
    float dunit_f = 0.0f; // R = W rho0 rounded to FP32: the unit of the deviation references c_i = k_i R
    int pop_stream = 0;   // host side: the D3Q27 step loads with the evict-first policy (ld_pop)
};

// beta in the compute type.
template <class T>
__device__ __forceinline__ T beta_of(const CollideParams &p)
{
    if constexpr (sizeof(T) == 4) return p.beta_f;
    else return p.beta;
}

// Deviation storage keeps d_i = f_i - c_i with the reference c_i = k_i R,
// R = W rho0 rounded to FP32 (W = 6^-D; w_i = k_i W with k_i a power of two, so
// c_i is w_i rho0 rounded to FP32, and the same value in every precision).  With
// the reference exact in FP32, sum_i c_i = 6^D R and rho = 6^D R + sum_i d_i.
template <int D>
__host__ __device__ inline float dev_unit(double rho0)
{
    return float(weight_unit(D) * rho0);
}
// c_i in the compute type T, from R in FP32.
template <int D, class T>
__device__ __forceinline__ T dev_ref(int i, float R)
{
    return T(weight_k(D, i)) * T(R);
}

// ---------------------------------------------------------------------------
// Arithmetic helpers.  FP32 divisions on the hot path multiply by the
// approximate reciprocal (rcp.approx.ftz: one MUFU operation, ~1 ulp); every
// divisor on the path is a normal number of moderate size (populations,
// 1 + O(x) polynomials), so flushing subnormals changes nothing.  FP64 uses
// IEEE division.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_(float b)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
    return r;
}
__device__ __forceinline__ float div_(float a, float b) { return a * rcp_(b); }
// 1/rho for the velocity u = j/rho: the approximate reciprocal followed by one
// Newton-Raphson step for 1/b (r + r (1 - b r)), which brings it to within about
// half an ulp; u carries every other quantity of the node, so it gets the
// accurate reciprocal for two extra fused multiply-adds per node.
__device__ __forceinline__ float rcp_nr(float b)
{
    const float r = rcp_(b);
    return fmaf(r, fmaf(-b, r, 1.0f), r);
}
__device__ __forceinline__ double rcp_nr(double b) { return 1.0 / b; }
__device__ __forceinline__ double div_(double a, double b) { return a / b; }
// FP32 square roots on the path act on 1 + O(u^2) and 1 - 4pq >= 1: the
// approximate instruction (relative error ~2^-23) loses nothing there.
__device__ __forceinline__ float sqrt_(float a)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
// correctly rounded division, for the few divisions whose rounding reaches f^eq
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return a / b; }
__device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }

// ---------------------------------------------------------------------------
// Storage traits.  raw/pack convert between the stored element and the compute
// type as they are (populations, or deviations d_i = f_i - c_i where kDev);
// load/store (and load64/store64 for FP64 companions) take the reference c_i of
// population i and convert to and from populations f_i.  The step kernels load
// with step_in and store with step_out, which give the values the collision
// works on: the deviations themselves where kDevCollide (FP32 deviations, so that
// no rounding happens at the scale of w_i), populations otherwise (the 16-bit
// storages, whose quantisation to 11 or 8 significant bits dwarfs the FP32
// rounding of f).
// ---------------------------------------------------------------------------
struct StoreF64 {
    using S = double;
    using T = double;
    static constexpr bool kDev = false, kDevCollide = false;
    static constexpr int kRows = 0; // row-staged kernel not instantiated (FP64 is the parity path)
    __device__ static __forceinline__ T raw(S s) { return s; }
    __device__ static __forceinline__ S pack(T v) { return v; }
    __device__ static __forceinline__ T load(S s, T) { return s; }
    __device__ static __forceinline__ S store(T f, T) { return f; }
    __device__ static __forceinline__ double load64(S s, double) { return s; }
    __device__ static __forceinline__ S store64(double f, double) { return f; }
};
struct StoreF32 {
    using S = float;
    using T = float;
    static constexpr bool kDev = false, kDevCollide = false;
    static constexpr int kRows = 1;
    __device__ static __forceinline__ T raw(S s) { return s; }
    __device__ static __forceinline__ S pack(T v) { return v; }
    __device__ static __forceinline__ T load(S s, T) { return s; }
    __device__ static __forceinline__ S store(T f, T) { return f; }
    __device__ static __forceinline__ double load64(S s, double) { return double(s); }
    __device__ static __forceinline__ S store64(double f, double) { return float(f); }
};
struct StoreF32Dev {
    using S = float;
    using T = float;
    static constexpr bool kDev = true, kDevCollide = true;
    static constexpr int kRows = 1;
    __device__ static __forceinline__ T raw(S s) { return s; }
    __device__ static __forceinline__ S pack(T v) { return v; }
    __device__ static __forceinline__ T load(S s, T c) { return c + s; }
    __device__ static __forceinline__ S store(T f, T c) { return f - c; }
    __device__ static __forceinline__ double load64(S s, double c) { return c + double(s); }
    __device__ static __forceinline__ S store64(double f, double c) { return float(f - c); }
};
struct StoreF16Dev {
    using S = __half;
    using T = float;
    static constexpr bool kDev = true, kDevCollide = false;
    static constexpr int kRows = 1;
    __device__ static __forceinline__ T raw(S s) { return __half2float(s); }
    __device__ static __forceinline__ S pack(T v) { return __float2half_rn(v); }
    __device__ static __forceinline__ T load(S s, T c) { return c + raw(s); }
    __device__ static __forceinline__ S store(T f, T c) { return pack(f - c); }
    __device__ static __forceinline__ double load64(S s, double c) { return c + double(__half2float(s)); }
    __device__ static __forceinline__ S store64(double f, double c) { return __double2half(f - c); }
};
struct StoreBF16Dev {
    using S = __nv_bfloat16;
    using T = float;
    static constexpr bool kDev = true, kDevCollide = false;
    static constexpr int kRows = 1;
    __device__ static __forceinline__ T raw(S s) { return __bfloat162float(s); }
    __device__ static __forceinline__ S pack(T v) { return __float2bfloat16_rn(v); }
    __device__ static __forceinline__ T load(S s, T c) { return c + raw(s); }
    __device__ static __forceinline__ S store(T f, T c) { return pack(f - c); }
    __device__ static __forceinline__ double load64(S s, double c) { return c + double(__bfloat162float(s)); }
    __device__ static __forceinline__ S store64(double f, double c) { return __double2bfloat16(f - c); }
};

// The values a step kernel collides on (see kDevCollide), from the stored element s of
// population i with reference c, and back.
template <class ST>
__device__ __forceinline__ typename ST::T step_in(typename ST::S s, typename ST::T c)
{
    if constexpr (ST::kDevCollide || !ST::kDev) return ST::raw(s);
    else return ST::load(s, c);
}
template <class ST>
__device__ __forceinline__ typename ST::S step_out(typename ST::T v, typename ST::T c)
{
    if constexpr (ST::kDevCollide || !ST::kDev) return ST::pack(v);
    else return ST::store(v, c);
}

template <class T>
__device__ __forceinline__ T g_entropy(T y);

// ---------------------------------------------------------------------------
// Positive root of -alpha^2 a + alpha b - c in the conjugate form of Eq.
// alphaLowerSoln, 2c / (b + sqrt(b^2 - 4ac)), evaluated with b factored out,
// 2q / (1 + sqrt(1 - 4 p q)) with q = c/b, p = a/b, so that no power of the
// O(x^2) coefficients can underflow in FP32.  Requires b > 0; a <= 0 <= c.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T quad_root(T a, T b, T c)
{
    const T q = div_(c, b);
    const T p = div_(a, b);
    return div_(T(2) * q, T(1) + sqrt_(T(1) - T(4) * p * q));
}

// ---------------------------------------------------------------------------
// Per-node collision on registers.
//   in : f[Q]  pre-collision populations
//   out: f[Q]  post-collision populations f* = f + alpha beta (f^eq - f)
//              (only when kRelax)
//        x[Q]  departures x_i = f^eq_i / f_i - 1 (Eq. xdef)
//        returns alpha; *branch receives kBranch*
//
// Evaluation order (the arithmetic is the paper's; only the grouping differs):
//  * f^eq - f is formed in deviation form.  With d_i = f_i - w_i,
//    rho = 1 + drho, and per axis eps(c) = Upsilon z^c - 1 (c = -1, 0, 1),
//    f^eq_i - f_i = w_i (drho + rho E_i) - d_i,  E_i = prod_a (1 + eps_a(c_ia)) - 1,
//    so no rounding happens at the scale of w_i (FP32 keeps ~u times more
//    digits of f^eq - f than the product form evaluated directly).  The
//    difference itself is formed as (k_i r) E_i + (k_i r - f_i) with
//    w_i = k_i W, r = rho W (see below), rounded once.  With
//    s = sqrt(1 + 3u^2) and t = s - 1 = 3u^2/(1+s), the axis factors reduce
//    exactly to Upsilon - 1 = -t and Upsilon z^{+-1} - 1 = 2t +- 3u (since
//    (2-s)(2u+s) = (1-u)(2s-1+3u) and 1/z(u) = z(-u)): one reciprocal per axis,
//    and the first moment (eps(+1) - eps(-1))/6 = u carries no bias from it.
//  * The Gauss-Legendre denominator factors: 60 + 90x + 36x^2 + 3x^3 =
//    (2 + x)(30 + 30x + 3x^2), so the c1 and c terms share one reciprocal,
//    and as 60 + 60x + 11x^2 = 2(30 + 30x + 3x^2) + 5x^2, c = c1 + 5 <f, A x^2>
//    with A = x^2 / ((2 + x)(30 + 30x + 3x^2)).
//  * The Omega+ bracket 2/(4+t) + 1/(4+2t) + 2/(4+3t) is the single rational
//    (80 + 80t + 19t^2) / (64 + 96t + 44t^2 + 6t^3).
//  * a is assembled from the Omega- power sums S_k = <f, x^k>_- (k = 3..6);
//    a1 = S3/2 and a2 = beta^2 S3/6.
//  * The relaxation uses f^eq - f = x f, so only f and x stay live.
// ---------------------------------------------------------------------------
template <int D, class T, bool kRelax = true>
__device__ __forceinline__ T node_collide(T (&f)[Lattice<D>::Q], T (&x)[Lattice<D>::Q],
                                          const CollideParams &p, int *branch)
{
    constexpr int Q = Lattice<D>::Q;
    const T beta = beta_of<T>(p);

    // Deviations from the weights and the moments (Sec. I): rho = <f,1>,
    // rho u = <f,c> = <d,c> (the weights carry no momentum).  Sums are taken
    // along the last axis first, then the middle, then the first.
    T dev[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) dev[i] = f[i] - T(weight_k(D, i)) * T(weight_unit(D)); // exact
    constexpr int P = Q / 3; // columns along the last axis
    T s0[P], s1[P];          // per column: sum over c_last, and (c_last=+1) - (c_last=-1)
#pragma unroll
    for (int k = 0; k < P; ++k) {
        s0[k] = dev[3 * k] + dev[3 * k + 1] + dev[3 * k + 2];
        s1[k] = dev[3 * k + 2] - dev[3 * k];
    }
    T drho, j[D];
    if (D == 2) {
        drho = s0[0] + s0[1] + s0[2];
        j[0] = s0[2] - s0[0];
        j[D - 1] = s1[0] + s1[1] + s1[2];
    } else {
        T t0[3], ty[3], tz[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            t0[a] = s0[3 * a] + s0[3 * a + 1] + s0[3 * a + 2];
            ty[a] = s0[3 * a + 2] - s0[3 * a];
            tz[a] = s1[3 * a] + s1[3 * a + 1] + s1[3 * a + 2];
        }
        drho = t0[0] + t0[1] + t0[2];
        j[0] = t0[2] - t0[0];
        j[1] = ty[0] + ty[1] + ty[2];
        j[D - 1] = tz[0] + tz[1] + tz[2];
    }
    // The deviations were taken from k_i T(W); the rest of W (sum k_i = 6^D) is
    // taken off drho, so rho = sum f to rounding.  r = rho W in two parts.
    drho -= T(double(Q == 9 ? 36 : 216) * double(weight_unit_lo<D, T>()));
    const T rho = T(1) + drho;
    const T r = fma(rho, T(weight_unit(D)), rho * weight_unit_lo<D, T>());
    const T irho = rcp_nr(rho);

    // Per axis eps(c) = Upsilon z^c - 1 for c = -1, 0, +1 (Sec. I equilibrium),
    // in the reduced form -t, 2t +- 3u.
    T eps[D][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const T u = j[a] * irho;
        const T s = sqrt_(T(1) + T(3) * u * u);
        const T t = div_(T(3) * u * u, T(1) + s); // s - 1, without cancellation
        eps[a][0] = T(2) * t - T(3) * u;          // Upsilon / z - 1
        eps[a][1] = -t;                           // Upsilon - 1
        eps[a][2] = T(2) * t + T(3) * u;          // Upsilon z - 1
    }

    // x_i = (f^eq_i - f_i) / f_i with f^eq_i - f_i = (k_i r) E_i + (k_i r - f_i): k_i r
    // is exact (a power of two times r) and so is k_i r - f_i wherever f_i is within
    // a factor two of f^eq_i (Sterbenz), leaving one rounding, at the scale of
    // f^eq - f.  Forming w_i (drho + rho E_i) - d_i instead rounds at the scale of
    // w_i u and with the rounded w_i, which in FP32 biased the momentum of f^eq by
    // ~3e-8 of itself per step (the kinetic energy of a decaying D2Q9 vortex,
    // beta = 0.9, 8e-5 above FP64 after 2000 steps).
    T xabs = T(0), xmin = T(0);
    T fx[Q];
#pragma unroll
    for (int k = 0; k < P; ++k) {
        // E for the column: first D-1 axes fixed, last axis varies
        T A;
        if (D == 2) {
            A = eps[0][k];
        } else {
            const T ex = eps[0][k / 3], ey = eps[1][k % 3];
            A = ex + ey + ex * ey;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int i = 3 * k + c;
            const T el = eps[D - 1][c];
            const T E = A + el + A * el;
            const T kr = T(weight_k(D, i)) * r;
            const T delta = fma(kr, E, kr - f[i]);
            x[i] = div_(delta, f[i]);
            fx[i] = delta; // f_i x_i, reused by the sums below
            xabs = fmax(xabs, fabs(x[i]));
            xmin = fmin(xmin, x[i]);
        }
    }

    T alpha = T(2);
    int br = kBranchCutoff;
    if (p.mode != kModeLBGK && !(p.cutoff && xabs < T(kCutoff))) {
        // Eq. alphaLowerCoeffs and the x-only parts of Eq. qaud_tight_coeff:
        //   b1 = <f, x^2/2>, c1 = <f, 2x^2/(2+x)>,
        //   c  = <f, x^2 (60 + 60x + 11x^2)/((2+x)(30 + 30x + 3x^2))>,
        //   S_k = <f, x^k>_{Omega-} (k = 3..6), a1 = S3/2, a2 = beta^2 S3/6.
        T b1 = T(0), c1 = T(0), c = T(0), S3 = T(0), S4 = T(0), S5 = T(0), S6 = T(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T xi = x[i];
            const T fx2 = fx[i] * xi;
            const T K = T(30) + xi * (T(30) + T(3) * xi);
            const T A = div_(fx2, (T(2) + xi) * K);
            b1 += fx2;
            c1 += A * K;
            c += A * (xi * xi); // c = c1 + 5 <f, A x^2> below
            if (xi < T(0)) {
                const T fx3 = fx2 * xi;
                S3 += fx3;
                S4 += fx3 * xi;
                S5 += fx3 * xi * xi;
                S6 += fx3 * xi * xi * xi;
            }
        }
        b1 *= T(0.5);
        c1 *= T(2);
        c = c1 + T(5) * c;
        if (b1 > T(0)) {
            // alpha_Lower (Eq. alphaLowerSoln).
            const T aL = quad_root(T(0.5) * S3, b1, c1);
            if (p.mode == kModeLower) {
                alpha = aL;
            } else if (p.mode == kModeIterate1) {
                // alpha_Iterate1 (Sec. IV): one Newton step of the mirror-state equation
                // H[f + alpha (f^eq - f)] = H[f] (Eq. deltaH_) from alpha_Lower:
                // F(a) = <f, g(a x)> - a <f, x log(1+x)> with g(y) = (1+y) log(1+y) - y
                // (using <f,x> = 0), F'(a) = <f, x (log(1+a x) - log(1+x))>.  Where the
                // step is undefined (some 1 + aL x_i <= 0) or F'(aL) <= 0, aL is kept.
                T Fv = T(0), dF = T(0);
                bool ok = true;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const T xi = x[i];
                    ok = ok && (T(1) + aL * xi > T(0));
                    const T l1 = log1p(xi), la = log1p(aL * xi);
                    Fv += f[i] * (g_entropy<T>(aL * xi) - aL * xi * l1);
                    dF += f[i] * xi * (la - l1);
                }
                alpha = (ok && dF > T(0)) ? aL - Fv / dF : aL;
            } else {
                // b of Eq. qaud_tight_coeff, k = alpha_L beta (derived) or alpha_L (printed).
                const T k = p.b_variant ? aL : aL * beta;
                T bp = T(0);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const T xi = x[i];
                    if (xi >= T(0)) {
                        const T t = k * xi;
                        bp += div_(f[i] * xi * xi * xi * (T(80) + t * (T(80) + T(19) * t)),
                                   T(64) + t * (T(96) + t * (T(44) + T(6) * t)));
                    }
                }
                const T b = b1 - T(2.0 / 15.0) * aL * beta * beta * bp;
                // Upper bound h: positive root of Eq. gaplhah0, a2 = beta^2 <f,x^3/6>_-.
                const T h = quad_root(beta * beta * S3 * T(1.0 / 6.0), b, c);
                // a of Eq. qaud_tight_coeff from the power sums.
                const T hb = h * beta;
                const T a = beta * beta *
                            (S3 * T(1.0 / 6.0) - hb * S4 * T(1.0 / 12.0) + hb * hb * S5 * T(1.0 / 20.0) -
                             hb * hb * hb * S6 * T(1.0 / 5.0));
                alpha = quad_root(a, b, c); // alpha_Higher
            }
            br = kBranchSolved;
        }
    }
    if (p.mode != kModeLBGK && xmin < T(0) && alpha * beta * (-xmin) > T(1)) {
        // Positivity (Appendix D): alpha_max = -1/(beta x_min); alpha > alpha_max
        // becomes (1 + alpha_max)/2, and alpha_max/2 when that still exceeds it.
        const T amax = div_(T(-1), beta * xmin);
        alpha = T(0.5) * (T(1) + amax);
        if (alpha > amax) alpha = T(0.5) * amax;
        br = kBranchClamped;
    }
    if (kRelax) {
        const T ab = alpha * beta;
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = fma(ab * x[i], f[i], f[i]);
    }
    *branch = br;
    return alpha;
}

// ---------------------------------------------------------------------------
// FP32 collision on packed population pairs.
//
// The same arithmetic as node_collide<D, float>, evaluated on float2 pairs of
// populations with the sm_100-family paired FP32 instructions (__ffma2_rn,
// __fmul2_rn, __fadd2_rn: two IEEE FP32 operations per instruction).  The two
// populations of a pair have velocities that mirror each other along one axis m
// (lane 0: c_m = -1, lane 1: c_m = +1) and agree on the other axes, so both lanes
// share the weight and the other axes' equilibrium factors: first the Q/3 pairs
// mirrored along the last axis, then, among the populations at rest along it, those
// mirrored along the axis before, and so on; the rest population comes last with a
// padding lane (f = 1, x = 0) that contributes nothing to any sum.  The
// Omega-/Omega+ restricted sums are taken branch-free with min(x,0) / max(x,0): a
// term of the other set is exactly zero, so the sums equal the restricted ones.
// The populations are reached through an accessor pa (pa.get(k): pair k; pa.put(k, v):
// the post-collision pair k); the kernels pass PairRegs, the pairs held in registers.
// Deviation form (kDev): the pairs hold d_i throughout; the departures are formed at
// the scale of d_i, the sums use f_i = k_i R + d_i (needed only to FP32 relative
// accuracy) and the relaxation is d*_i = d_i + alpha beta x_i f_i.
//   in : pa.get  pre-collision populations (deviations d_i = f_i - k_i R when kDev),
//                pair layout
//   out: pa.put  post-collision values of the same kind (when kRelax)
//        xp[NP]  departures x_i (Eq. xdef), pair layout
//        returns alpha; *branch receives kBranch*
// ---------------------------------------------------------------------------
template <int D>
struct Pairs {
    static constexpr int Q = Lattice<D>::Q;
    static constexpr int NP = (Q + 1) / 2;
};

// Population held by lane `lane` of pair k (-1: the padding lane), lexicographic
// population order i = sum_a 3^(D-1-a) (c_a + 1).
__host__ __device__ constexpr int pair_pop(int D, int k, int lane)
{
    if (D == 3) {
        if (k < 9) return 3 * k + 2 * lane;            // (c_x, c_y) from k; c_z = -1, +1
        if (k < 12) return 9 * (k - 9) + 1 + 6 * lane; // c_x = k - 10; c_y = -1, +1; c_z = 0
        if (k == 12) return 4 + 18 * lane;             // c_x = -1, +1; c_y = c_z = 0
        return lane ? -1 : 13;                         // rest
    }
    if (k < 3) return 3 * k + 2 * lane; // c_x = k - 1; c_y = -1, +1
    if (k == 3) return 1 + 6 * lane;    // c_x = -1, +1; c_y = 0
    return lane ? -1 : 4;               // rest
}
// Mirrored axis of pair k (-1 for the rest pair).
__host__ __device__ constexpr int pair_axis(int D, int k)
{
    return D == 3 ? (k < 9 ? 2 : k < 12 ? 1 : k == 12 ? 0 : -1) : (k < 3 ? 1 : k == 3 ? 0 : -1);
}
// Slot 2 k + lane that holds population i.
__host__ __device__ constexpr int pair_slot(int D, int i)
{
    for (int k = 0; k < (Lattice<3>::Q + 1) / 2; ++k)
        for (int lane = 0; lane < 2; ++lane)
            if (pair_pop(D, k, lane) == i) return 2 * k + lane;
    return -1;
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 prcp(float2 a) { return f2(rcp_(a.x), rcp_(a.y)); }

// Weight of pair k's lane, as k_i T(W) (0 in the padding lane), and its k_i.
template <int D>
__host__ __device__ constexpr float wpair(int k, int lane)
{
    return pair_pop(D, k, lane) >= 0 ? float(weight_k(D, pair_pop(D, k, lane))) * float(weight_unit(D)) : 0.0f;
}
template <int D>
__host__ __device__ constexpr float kpair(int k, int lane)
{
    return pair_pop(D, k, lane) >= 0 ? float(weight_k(D, pair_pop(D, k, lane))) : 0.0f;
}

// Populations of the pair layout held in registers.
template <int NP>
struct PairRegs {
    float2 (&a)[NP];
    __device__ __forceinline__ float2 get(int k) const { return a[k]; }
    __device__ __forceinline__ void put(int k, float2 v) { a[k] = v; }
};

// The same value, opaque to the compiler: k_i R + d_i formed again after the departures
// instead of being kept from there (which would hold both f and d in registers).
__device__ __forceinline__ float2 opaque(float2 v)
{
    asm volatile("" : "+f"(v.x), "+f"(v.y));
    return v;
}

template <int D, bool kRelax = true, bool kDev = false, class PA>
__device__ __forceinline__ float node_collide_pairs(PA &pa, float2 (&xp)[Pairs<D>::NP], const CollideParams &p,
                                                    int *branch)
{
    constexpr int Q = Lattice<D>::Q;
    constexpr int NP = Pairs<D>::NP;
    constexpr bool kPad = (Q % 2) == 1;
    const float beta = p.beta_f;
    const float R = p.dunit_f; // deviation form: f_i = k_i R + d_i

    // Deviations and the moments (Sec. I): d_i = f_i - w_i, or the stored d_i = f_i - k_i R.
    // Sums along the last axis first: per column (the first D-1 components fixed) s0 =
    // sum of d, s1 = (c_last = +1) - (c_last = -1).  The first Q/3 pairs are mirrored
    // along the last axis, one per column, and start each column's sums; the rest add
    // the columns' c_last = 0 populations.
    constexpr int P = Q / 3;
    float s0[P], s1[P];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float2 v = pa.get(k);
        const float2 d = kDev ? v : psub(v, f2(wpair<D>(k, 0), wpair<D>(k, 1)));
        if (k < P) {
            s0[k] = d.x + d.y;
            s1[k] = d.y - d.x;
        } else {
#pragma unroll
            for (int lane = 0; lane < 2; ++lane) {
                const int i = pair_pop(D, k, lane);
                if (i >= 0) s0[i / 3] += lane ? d.y : d.x;
            }
        }
    }
    float drho, j[D];
    if (D == 2) {
        drho = s0[0] + s0[1] + s0[2];
        j[0] = s0[2] - s0[0];
        j[D - 1] = s1[0] + s1[1] + s1[2];
    } else {
        float t0[3], ty[3], tz[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            t0[a] = s0[3 * a] + s0[3 * a + 1] + s0[3 * a + 2];
            ty[a] = s0[3 * a + 2] - s0[3 * a];
            tz[a] = s1[3 * a] + s1[3 * a + 1] + s1[3 * a + 2];
        }
        drho = t0[0] + t0[1] + t0[2];
        j[0] = t0[2] - t0[0];
        j[1] = ty[0] + ty[1] + ty[2];
        j[D - 1] = tz[0] + tz[1] + tz[2];
    }
    float rho, r, dr;
    if constexpr (kDev) {
        // rho = 6^D R + drho and, as 6^D W = 1, r - R = rho W - R = W drho exactly: the
        // equilibrium's scale r = R + dr is kept in two parts (dr below)
        rho = fmaf(float(Q == 9 ? 36 : 216), R, drho);
        dr = fmaf(drho, float(weight_unit(D)), drho * weight_unit_lo<D, float>());
        r = R;
    } else {
        drho -= float(double(Q == 9 ? 36 : 216) * double(weight_unit_lo<D, float>())); // as in node_collide
        rho = 1.0f + drho;
        r = fmaf(rho, float(weight_unit(D)), rho * weight_unit_lo<D, float>());
        dr = 0.0f;
    }
    const float irho = rcp_nr(rho);
    // f of pair k: the populations themselves, or k_i R + d_i (the padding lane has k = 0
    // and holds 1); fagain(k) forms it anew past the departures
    auto fval = [&](int k) -> float2 {
        if constexpr (kDev) return pfma(f2(kpair<D>(k, 0), kpair<D>(k, 1)), f2(R), pa.get(k));
        else return pa.get(k);
    };
    auto fagain = [&](int k) -> float2 {
        if constexpr (kDev) return pfma(f2(kpair<D>(k, 0), kpair<D>(k, 1)), f2(R), opaque(pa.get(k)));
        else return pa.get(k);
    };

    // Per axis eps(c) = Upsilon z^c - 1 (as in node_collide).
    float eps[D][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float u = j[a] * irho;
        const float s = sqrt_(1.0f + 3.0f * u * u);
        const float t = div_(3.0f * u * u, 1.0f + s);
        eps[a][0] = 2.0f * t - 3.0f * u;
        eps[a][1] = -t;
        eps[a][2] = 2.0f * t + 3.0f * u;
    }
    // E_i = prod_a (1 + eps_a(c_ia)) - 1 per pair: G = prod over the axes other than the
    // mirrored one m, minus 1 (shared by both lanes), then E = G + e + G e with
    // e = (eps_m(-1), eps_m(+1)).
    auto E_pair = [&](int k) -> float2 {
        const int m = pair_axis(D, k), i0 = pair_pop(D, k, 0);
        float G = 0.0f;
        bool first = true;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            if (a == m) continue;
            const float e = eps[a][vel(D, i0, a) + 1];
            G = first ? e : G + e + G * e;
            first = false;
        }
        if (m < 0) return f2(G, 0.0f);
        const float2 em = f2(eps[m][0], eps[m][2]);
        return pfma(f2(G), em, padd(f2(G), em));
    };

    // x_i = (f^eq_i - f_i) / f_i and its extremes; the sums of the path length are
    // taken only past the cutoff test, so warps whose nodes all take the shortcut skip them.
    float xabs = 0.0f, xmin = 0.0f;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float2 E = E_pair(k);
        const float2 K = f2(kpair<D>(k, 0), kpair<D>(k, 1));
        float2 delta;
        if constexpr (kDev) {
            // f^eq - f = k_i (R + dr)(1 + E_i) - k_i R - d_i = k_i [R E_i + dr (1 + E_i)] - d_i:
            // the bracket is rounded at the scale of R E_i, k_i (a power of two) scales it
            // exactly, and the difference with d_i is rounded once
            const float2 t = pfma(f2(R), E, pfma(f2(dr), E, f2(dr)));
            delta = pfma(K, t, psub(f2(0.0f), pa.get(k)));
        } else {
            // f^eq - f = (k_i r) E_i + (k_i r - f_i), one rounding (as in node_collide)
            const float2 kr = pmul(K, f2(r));
            delta = pfma(kr, E, psub(kr, pa.get(k)));
        }
        if (kPad && k == NP - 1) delta.y = 0.0f; // padding lane: f = 1, x = 0
        const float2 xi = pmul(delta, prcp(fval(k)));
        xp[k] = xi;
        xabs = fmaxf(xabs, fmaxf(fabsf(xi.x), fabsf(xi.y))); // three-input max
        xmin = fminf(xmin, fminf(xi.x, xi.y));
    }

    float alpha = 2.0f;
    int br = kBranchCutoff;
    if (p.mode != kModeLBGK && !(p.cutoff && xabs < float(kCutoff))) {
        // Eq. alphaLowerCoeffs and the x-only parts of Eq. qaud_tight_coeff, and the
        // Omega- power sums S3..S6 (as in node_collide).  Where |x|max < kSeriesX the
        // three rational terms are summed from power sums M_k = <f, x^k> (all i) and
        // S_k (Omega-), their series truncated below FP32 rounding:
        //   2/(2 + x) = sum_k (-x/2)^k                     (c1 = <f, x^2 2/(2+x)>)
        //   (60 + 60x + 11x^2)/(60 + 90x + 36x^2 + 3x^3)
        //       = 1 - x/2 + x^2/3 - x^3/4 + x^4/5 - ...      (c; log(1+x)/x to x^5)
        //   2/(4+t) + 1/(4+2t) + 2/(4+3t) = 5/4 - 5t/8 + 3t^2/8 - t^3/4 + ...   (b, t = k x)
        // with the Omega+ sums P_m = M_m - S_m.  Kept to M6: below |x|max = 0.04 the
        // dropped terms move c1 by ~2e-9, c by ~1e-8 and b by ~4e-8 of themselves, and
        // the path length by less than 7e-8 (half an FP32 ulp of 2).  Where |x|max < kShortX the
        // series stop at x^4 (M2..M4, S3, S4): the dropped terms are bounded by
        // |x|max^3 = 1.25e-7 of M2 times their coefficients (1/8 in c1, 1/4 in c), and
        // alpha moves by at most ~3e-8 relative, below FP32 rounding.  The series forms
        // need no reciprocal per population and no second pass for b.
        // The form is chosen once per warp, from its largest |x|max among the lanes
        // solving here: a warp whose lanes straddle a threshold runs the longer form
        // on all of them instead of each form in turn (the forms agree below FP32
        // rounding, so which one a lane gets moves its path length by less than that).
        constexpr float kSeriesX = 0.04f, kShortX = 0.005f;
        const int form = __reduce_max_sync(__activemask(), xabs < kShortX ? 0 : (xabs < kSeriesX ? 1 : 2));
        const bool series = form < 2;
        float sb1, sc1, sc, s3, s4, s5 = 0.0f, s6 = 0.0f, m3 = 0.0f, m4 = 0.0f, m5 = 0.0f, m6 = 0.0f;
        if (form == 0) {
            float2 M2 = f2(0.0f), M3 = f2(0.0f), M4 = f2(0.0f), S3 = f2(0.0f), S4 = f2(0.0f);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float2 xi = xp[k];
                const float2 fx2 = pmul(fagain(k), pmul(xi, xi)); // f x^2
                const float2 q3 = pmul(fx2, xi);
                M2 = padd(M2, fx2);
                M3 = padd(M3, q3);
                M4 = pfma(q3, xi, M4);
                const float2 xm = f2(fminf(xi.x, 0.0f), fminf(xi.y, 0.0f));
                const float2 q = pmul(fx2, xm); // f x^3 on Omega-, 0 elsewhere
                S3 = padd(S3, q);
                S4 = pfma(q, xm, S4);
            }
            const float m2 = M2.x + M2.y;
            m3 = M3.x + M3.y, m4 = M4.x + M4.y;
            sb1 = 0.5f * m2;
            sc1 = m2 + (m3 * -0.5f + m4 * 0.25f);
            sc = m2 + (m3 * -0.5f + m4 * (1.0f / 3.0f));
            s3 = S3.x + S3.y, s4 = S4.x + S4.y;
        } else if (series) {
            float2 M2 = f2(0.0f), M3 = f2(0.0f), M4 = f2(0.0f), M5 = f2(0.0f), M6 = f2(0.0f);
            float2 S3 = f2(0.0f), S4 = f2(0.0f), S5 = f2(0.0f), S6 = f2(0.0f);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float2 xi = xp[k];
                const float2 x2 = pmul(xi, xi);
                const float2 fx2 = pmul(fagain(k), x2); // f x^2
                const float2 q3 = pmul(fx2, xi);
                const float2 q5 = pmul(q3, x2);
                M2 = padd(M2, fx2);
                M3 = padd(M3, q3);
                M4 = pfma(q3, xi, M4);
                M5 = padd(M5, q5);
                M6 = pfma(q5, xi, M6);
                const float2 xm = f2(fminf(xi.x, 0.0f), fminf(xi.y, 0.0f));
                const float2 q = pmul(fx2, xm); // f x^3 on Omega-, 0 elsewhere
                const float2 xm2 = pmul(xm, xm);
                S3 = padd(S3, q);
                S4 = pfma(q, xm, S4);
                S5 = pfma(q, xm2, S5);
                S6 = pfma(pmul(q, xm), xm2, S6);
            }
            const float m2 = M2.x + M2.y;
            m3 = M3.x + M3.y, m4 = M4.x + M4.y, m5 = M5.x + M5.y, m6 = M6.x + M6.y;
            sb1 = 0.5f * m2;
            sc1 = m2 + (m3 * -0.5f + (m4 * 0.25f + (m5 * -0.125f + m6 * 0.0625f))); // <f, 2x^2/(2+x)>
            sc = m2 + (m3 * -0.5f + (m4 * (1.0f / 3.0f) + (m5 * -0.25f + m6 * 0.2f)));
            s3 = S3.x + S3.y, s4 = S4.x + S4.y, s5 = S5.x + S5.y, s6 = S6.x + S6.y;
        } else {
            float2 b1 = f2(0.0f), c1 = f2(0.0f), c = f2(0.0f);
            float2 S3 = f2(0.0f), S4 = f2(0.0f), S5 = f2(0.0f), S6 = f2(0.0f);
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                const float2 xi = xp[k];
                const float2 fx2 = pmul(pmul(fagain(k), xi), xi); // f x^2
                const float2 K = pfma(pfma(f2(3.0f), xi, f2(30.0f)), xi, f2(30.0f));
                const float2 A = pmul(fx2, prcp(pmul(padd(f2(2.0f), xi), K)));
                b1 = padd(b1, fx2);
                c1 = pfma(A, K, c1);
                c = pfma(pmul(A, xi), xi, c); // c = c1 + 5 <f, A x^2> below
                const float2 xm = f2(fminf(xi.x, 0.0f), fminf(xi.y, 0.0f));
                const float2 q = pmul(fx2, xm); // f x^3 on Omega-, 0 elsewhere
                const float2 xm2 = pmul(xm, xm);
                S3 = padd(S3, q);
                S4 = pfma(q, xm, S4);
                S5 = pfma(q, xm2, S5);
                S6 = pfma(pmul(q, xm), xm2, S6);
            }
            sb1 = 0.5f * (b1.x + b1.y), sc1 = 2.0f * (c1.x + c1.y), sc = sc1 + 5.0f * (c.x + c.y);
            s3 = S3.x + S3.y, s4 = S4.x + S4.y, s5 = S5.x + S5.y, s6 = S6.x + S6.y;
        }
        if (sb1 > 0.0f) {
            const float aL = quad_root(0.5f * s3, sb1, sc1); // alpha_Lower
            if (p.mode == kModeLower) {
                alpha = aL;
            } else {
                // b: Omega+ Boole term with k = alpha_L beta (derived) or alpha_L (printed).
                const float kk = p.b_variant ? aL : aL * beta;
                float bsum;
                if (series) {
                    const float p3 = m3 - s3, p4 = m4 - s4, p5 = m5 - s5, p6 = m6 - s6;
                    bsum = 1.25f * p3 + kk * (-0.625f * p4 + kk * (0.375f * p5 + kk * (-0.25f * p6)));
                } else {
                    float2 bp = f2(0.0f);
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const float2 xi = xp[k];
                        const float2 xq = f2(fmaxf(xi.x, 0.0f), fmaxf(xi.y, 0.0f));
                        const float2 t = pmul(f2(kk), xq);
                        const float2 nu = pfma(pfma(f2(19.0f), t, f2(80.0f)), t, f2(80.0f));
                        const float2 de = pfma(pfma(pfma(f2(6.0f), t, f2(44.0f)), t, f2(96.0f)), t, f2(64.0f));
                        // f x^3 on Omega+ (0 elsewhere) times the bracket
                        bp = pfma(pmul(pmul(fagain(k), pmul(pmul(xi, xi), xq)), nu), prcp(de), bp);
                    }
                    bsum = bp.x + bp.y;
                }
                const float b = sb1 - (2.0f / 15.0f) * aL * beta * beta * bsum;
                const float h = quad_root(beta * beta * s3 * (1.0f / 6.0f), b, sc);
                const float hb = h * beta;
                const float a = beta * beta *
                                (s3 * (1.0f / 6.0f) - hb * s4 * (1.0f / 12.0f) + hb * hb * s5 * (1.0f / 20.0f) -
                                 hb * hb * hb * s6 * (1.0f / 5.0f));
                alpha = quad_root(a, b, sc); // alpha_Higher
            }
            br = kBranchSolved;
        }
    }
    if (p.mode != kModeLBGK && xmin < 0.0f && alpha * beta * (-xmin) > 1.0f) {
        const float amax = div_(-1.0f, beta * xmin);
        alpha = 0.5f * (1.0f + amax);
        if (alpha > amax) alpha = 0.5f * amax;
        br = kBranchClamped;
    }
    if (kRelax) {
        // f* = f + alpha beta (f^eq - f) with f^eq - f = x f (deviation form:
        // d* = d + alpha beta x f, rounded at the scale of d)
        const float2 ab = f2(alpha * beta);
#pragma unroll
        for (int k = 0; k < NP; ++k) pa.put(k, pfma(pmul(ab, xp[k]), fagain(k), pa.get(k)));
    }
    *branch = br;
    return alpha;
}

// ---------------------------------------------------------------------------
// One node's collision on scalar arrays, whatever the compute type: FP32 goes
// through the packed-pair routine (on deviations d_i = f_i - k_i R when kDev),
// FP64 through node_collide.  f holds populations (or deviations when kDev) and
// receives the post-collision values of the same kind.
// ---------------------------------------------------------------------------
template <int D, class T, bool kRelax = true, bool kDev = false>
__device__ __forceinline__ T collide(T (&f)[Lattice<D>::Q], T (&x)[Lattice<D>::Q], const CollideParams &p,
                                     int *branch)
{
    constexpr int Q = Lattice<D>::Q;
    if constexpr (sizeof(T) == 4) {
        if (p.mode == kModeIterate1) {
            // alpha_Iterate1 (a comparison variant with logarithms) stays on the scalar
            // path, which takes populations
            if constexpr (kDev) {
#pragma unroll
                for (int i = 0; i < Q; ++i) f[i] += dev_ref<D, T>(i, p.dunit_f);
            }
            const T alpha = node_collide<D, T, kRelax>(f, x, p, branch);
            if constexpr (kDev) {
#pragma unroll
                for (int i = 0; i < Q; ++i) f[i] -= dev_ref<D, T>(i, p.dunit_f);
            }
            return alpha;
        }
        constexpr int NP = Pairs<D>::NP;
        float2 fp[NP], xp[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const int i1 = pair_pop(D, k, 1);
            fp[k] = make_float2(f[pair_pop(D, k, 0)], i1 >= 0 ? f[i1] : 1.0f);
        }
        PairRegs<NP> pr{fp};
        const float alpha = node_collide_pairs<D, kRelax, kDev>(pr, xp, p, branch);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int sl = pair_slot(D, i);
            x[i] = (sl & 1) ? xp[sl >> 1].y : xp[sl >> 1].x;
            if (kRelax) f[i] = (sl & 1) ? fp[sl >> 1].y : fp[sl >> 1].x;
        }
        return alpha;
    } else {
        static_assert(!kDev, "deviation storage computes in FP32");
        return node_collide<D, T, kRelax>(f, x, p, branch);
    }
}

// The collision of a step kernel on the values it loaded with step_in: deviations for
// the FP32 deviation storage, populations otherwise; they are stored back with step_out.
template <int D, class ST, bool kRelax = true>
__device__ __forceinline__ typename ST::T collide_stored(typename ST::T (&v)[Lattice<D>::Q],
                                                         typename ST::T (&x)[Lattice<D>::Q],
                                                         const CollideParams &p, int *branch)
{
    return collide<D, typename ST::T, kRelax, ST::kDevCollide>(v, x, p, branch);
}

// ---------------------------------------------------------------------------
// D2Q9 collision of two nodes at once, FP32.
//
// The arithmetic of node_collide_pairs, with the two lanes of every float2 holding
// two different nodes (A in .x, B in .y) and population i in slot i.  All per-node
// work -- moments, axis factors, the three quadratic roots of Eq. alphaLowerSoln and
// Eq. qaud_tight, the clamp of Appendix D -- is one paired instruction for both nodes,
// where the population-pair form spends one per node: a D2Q9 node has only nine
// populations, so that scalar work is a large share of its collision.  The lanes never
// mix; a node's result depends on its partner only through the coefficient form, chosen
// once per warp over every lane that solves (as in node_collide_pairs; the forms agree
// below FP32 rounding).  Where one node takes the cutoff (or has b1 <= 0) and the other
// solves, both lanes are evaluated and the first keeps alpha = 2.
//   in : f[9]  pre-collision values of both nodes (deviations d_i = f_i - k_i R when kDev)
//   out: f[9]  post-collision values of the same kind (when kRelax)
//        x[9]  departures x_i (Eq. xdef)
//        returns alpha of both nodes; br[0], br[1] receive kBranch*
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 psqrt(float2 a) { return f2(sqrt_(a.x), sqrt_(a.y)); }
__device__ __forceinline__ float2 pneg(float2 a) { return pmul(a, f2(-1.0f)); }
// quad_root on both lanes
__device__ __forceinline__ float2 pquad_root(float2 a, float2 b, float2 c)
{
    const float2 rb = prcp(b);
    const float2 q = pmul(c, rb), pq = pmul(a, rb);
    const float2 disc = pfma(pmul(f2(-4.0f), pq), q, f2(1.0f));
    return pmul(padd(q, q), prcp(padd(f2(1.0f), psqrt(disc))));
}

template <bool kRelax = true, bool kDev = false>
__device__ __forceinline__ float2 node_collide_x2(float2 (&f)[9], float2 (&x)[9], const CollideParams &p,
                                                  int (&br)[2])
{
    constexpr int D = 2, Q = 9;
    const float beta = p.beta_f;
    const float R = p.dunit_f; // deviation form: f_i = k_i R + d_i
    auto K = [](int i) { return f2(float(weight_k(D, i))); };
    auto fval = [&](int i) -> float2 {
        if constexpr (kDev) return pfma(K(i), f2(R), f[i]);
        else return f[i];
    };
    auto fagain = [&](int i) -> float2 {
        if constexpr (kDev) return pfma(K(i), f2(R), opaque(f[i]));
        else return f[i];
    };

    // Moments (Sec. I) from d_i, along y first: per column (c_x fixed) s0 = sum of d,
    // s1 = (c_y = +1) - (c_y = -1).
    float2 s0[3], s1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float2 d[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            d[c] = kDev ? f[3 * k + c] : psub(f[3 * k + c], f2(float(weight_k(D, 3 * k + c)) * float(weight_unit(D))));
        s0[k] = padd(padd(d[0], d[2]), d[1]);
        s1[k] = psub(d[2], d[0]);
    }
    float2 drho = padd(padd(s0[0], s0[1]), s0[2]);
    const float2 j[2] = {psub(s0[2], s0[0]), padd(padd(s1[0], s1[1]), s1[2])};
    float2 rho, r, dr;
    if constexpr (kDev) {
        // rho = 36 R + drho; r - R = W drho exactly (36 W = 1), kept apart as dr
        rho = pfma(f2(36.0f), f2(R), drho);
        dr = pfma(drho, f2(float(weight_unit(D))), pmul(drho, f2(weight_unit_lo<D, float>())));
        r = f2(R);
    } else {
        drho = psub(drho, f2(float(36.0 * double(weight_unit_lo<D, float>()))));
        rho = padd(f2(1.0f), drho);
        r = pfma(rho, f2(float(weight_unit(D))), pmul(rho, f2(weight_unit_lo<D, float>())));
        dr = f2(0.0f);
    }
    // 1/rho: approximate reciprocal and one Newton-Raphson step (as rcp_nr)
    const float2 r0 = prcp(rho);
    const float2 irho = pfma(r0, pfma(pneg(rho), r0, f2(1.0f)), r0);

    // Per axis eps(c) = Upsilon z^c - 1 = (2t - 3u, -t, 2t + 3u), t = 3u^2/(1 + s).
    float2 eps[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float2 u = pmul(j[a], irho);
        const float2 uu3 = pmul(f2(3.0f), pmul(u, u));
        const float2 t = pmul(uu3, prcp(padd(f2(1.0f), psqrt(padd(f2(1.0f), uu3)))));
        const float2 t2 = padd(t, t), u3 = pmul(f2(3.0f), u);
        eps[a][0] = psub(t2, u3);
        eps[a][1] = pneg(t);
        eps[a][2] = padd(t2, u3);
    }

    // x_i = (f^eq_i - f_i) / f_i with E_i = (1 + eps_x)(1 + eps_y) - 1, as in node_collide_pairs.
    float xabs[2] = {0.0f, 0.0f}, xmin[2] = {0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float2 A = eps[0][vel(D, i, 0) + 1], el = eps[1][vel(D, i, 1) + 1];
        const float2 E = pfma(A, el, padd(A, el));
        float2 delta;
        if constexpr (kDev) {
            const float2 t = pfma(f2(R), E, pfma(dr, E, dr));
            delta = pfma(K(i), t, pneg(f[i]));
        } else {
            const float2 kr = pmul(K(i), r);
            delta = pfma(kr, E, psub(kr, f[i]));
        }
        const float2 xi = pmul(delta, prcp(fval(i)));
        x[i] = xi;
        xabs[0] = fmaxf(xabs[0], fabsf(xi.x));
        xabs[1] = fmaxf(xabs[1], fabsf(xi.y));
        xmin[0] = fminf(xmin[0], xi.x);
        xmin[1] = fminf(xmin[1], xi.y);
    }

    float2 alpha = f2(2.0f);
    br[0] = br[1] = kBranchCutoff;
    const bool lbgk = p.mode == kModeLBGK;
    const bool need[2] = {!lbgk && !(p.cutoff && xabs[0] < float(kCutoff)),
                          !lbgk && !(p.cutoff && xabs[1] < float(kCutoff))};
    if (need[0] || need[1]) {
        // Coefficient forms of node_collide_pairs: x^4 series below kShortX, x^6 series
        // below kSeriesX, per-population rational terms above; one form per warp.
        constexpr float kSeriesX = 0.04f, kShortX = 0.005f;
        auto form_of = [&](int l) { return !need[l] ? 0 : (xabs[l] < kShortX ? 0 : (xabs[l] < kSeriesX ? 1 : 2)); };
        const int form = __reduce_max_sync(__activemask(), max(form_of(0), form_of(1)));
        const bool series = form < 2;
        float2 sb1, sc1, sc, s3, s4, s5 = f2(0.0f), s6 = f2(0.0f), m3 = f2(0.0f), m4 = f2(0.0f), m5 = f2(0.0f),
                                     m6 = f2(0.0f);
        if (form == 0) {
            float2 M2 = f2(0.0f), S3 = f2(0.0f), S4 = f2(0.0f);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float2 xi = x[i];
                const float2 fx2 = pmul(fagain(i), pmul(xi, xi));
                const float2 q3 = pmul(fx2, xi);
                M2 = padd(M2, fx2);
                m3 = padd(m3, q3);
                m4 = pfma(q3, xi, m4);
                const float2 xm = f2(fminf(xi.x, 0.0f), fminf(xi.y, 0.0f));
                const float2 q = pmul(fx2, xm);
                S3 = padd(S3, q);
                S4 = pfma(q, xm, S4);
            }
            sb1 = pmul(f2(0.5f), M2);
            sc1 = padd(M2, pfma(m3, f2(-0.5f), pmul(m4, f2(0.25f))));
            sc = padd(M2, pfma(m3, f2(-0.5f), pmul(m4, f2(1.0f / 3.0f))));
            s3 = S3, s4 = S4;
        } else if (series) {
            float2 M2 = f2(0.0f), S3 = f2(0.0f), S4 = f2(0.0f), S5 = f2(0.0f), S6 = f2(0.0f);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float2 xi = x[i];
                const float2 x2 = pmul(xi, xi);
                const float2 fx2 = pmul(fagain(i), x2);
                const float2 q3 = pmul(fx2, xi);
                const float2 q5 = pmul(q3, x2);
                M2 = padd(M2, fx2);
                m3 = padd(m3, q3);
                m4 = pfma(q3, xi, m4);
                m5 = padd(m5, q5);
                m6 = pfma(q5, xi, m6);
                const float2 xm = f2(fminf(xi.x, 0.0f), fminf(xi.y, 0.0f));
                const float2 q = pmul(fx2, xm);
                const float2 xm2 = pmul(xm, xm);
                S3 = padd(S3, q);
                S4 = pfma(q, xm, S4);
                S5 = pfma(q, xm2, S5);
                S6 = pfma(pmul(q, xm), xm2, S6);
            }
            sb1 = pmul(f2(0.5f), M2);
            // <f, 2x^2/(2+x)> and c, Horner in the power sums
            sc1 = padd(M2, pfma(m3, f2(-0.5f), pfma(m4, f2(0.25f), pfma(m5, f2(-0.125f), pmul(m6, f2(0.0625f))))));
            sc = padd(M2, pfma(m3, f2(-0.5f), pfma(m4, f2(1.0f / 3.0f), pfma(m5, f2(-0.25f), pmul(m6, f2(0.2f))))));
            s3 = S3, s4 = S4, s5 = S5, s6 = S6;
        } else {
            float2 b1 = f2(0.0f), c1 = f2(0.0f), c = f2(0.0f), S3 = f2(0.0f), S4 = f2(0.0f), S5 = f2(0.0f),
                   S6 = f2(0.0f);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float2 xi = x[i];
                const float2 fx2 = pmul(pmul(fagain(i), xi), xi);
                const float2 Kq = pfma(pfma(f2(3.0f), xi, f2(30.0f)), xi, f2(30.0f));
                const float2 A = pmul(fx2, prcp(pmul(padd(f2(2.0f), xi), Kq)));
                b1 = padd(b1, fx2);
                c1 = pfma(A, Kq, c1);
                c = pfma(pmul(A, xi), xi, c);
                const float2 xm = f2(fminf(xi.x, 0.0f), fminf(xi.y, 0.0f));
                const float2 q = pmul(fx2, xm);
                const float2 xm2 = pmul(xm, xm);
                S3 = padd(S3, q);
                S4 = pfma(q, xm, S4);
                S5 = pfma(q, xm2, S5);
                S6 = pfma(pmul(q, xm), xm2, S6);
            }
            sb1 = pmul(f2(0.5f), b1);
            sc1 = padd(c1, c1);
            sc = pfma(f2(5.0f), c, sc1);
            s3 = S3, s4 = S4, s5 = S5, s6 = S6;
        }
        const bool ok[2] = {need[0] && sb1.x > 0.0f, need[1] && sb1.y > 0.0f};
        if (ok[0] || ok[1]) {
            const float2 aL = pquad_root(pmul(f2(0.5f), s3), sb1, sc1); // alpha_Lower
            float2 asol;
            if (p.mode == kModeLower) {
                asol = aL;
            } else {
                const float2 kk = p.b_variant ? aL : pmul(aL, f2(beta));
                float2 bsum;
                if (series) {
                    const float2 p3 = psub(m3, s3), p4 = psub(m4, s4), p5 = psub(m5, s5), p6 = psub(m6, s6);
                    bsum = pfma(f2(1.25f), p3,
                                pmul(kk, pfma(f2(-0.625f), p4,
                                              pmul(kk, pfma(f2(0.375f), p5, pmul(kk, pmul(f2(-0.25f), p6)))))));
                } else {
                    bsum = f2(0.0f);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const float2 xi = x[i];
                        const float2 xq = f2(fmaxf(xi.x, 0.0f), fmaxf(xi.y, 0.0f));
                        const float2 t = pmul(kk, xq);
                        const float2 nu = pfma(pfma(f2(19.0f), t, f2(80.0f)), t, f2(80.0f));
                        const float2 de = pfma(pfma(pfma(f2(6.0f), t, f2(44.0f)), t, f2(96.0f)), t, f2(64.0f));
                        bsum = pfma(pmul(pmul(fagain(i), pmul(pmul(xi, xi), xq)), nu), prcp(de), bsum);
                    }
                }
                const float bb = beta * beta;
                const float2 b = pfma(pmul(f2(-(2.0f / 15.0f) * bb), aL), bsum, sb1);
                const float2 h = pquad_root(pmul(f2(bb * (1.0f / 6.0f)), s3), b, sc);
                const float2 hb = pmul(h, f2(beta));
                // a = beta^2 (S3/6 - hb S4/12 + hb^2 S5/20 - hb^3 S6/5), Horner in hb
                const float2 a = pmul(f2(bb), pfma(hb, pfma(hb, pfma(hb, pmul(f2(-0.2f), s6), pmul(f2(0.05f), s5)),
                                                            pmul(f2(-1.0f / 12.0f), s4)),
                                                   pmul(f2(1.0f / 6.0f), s3)));
                asol = pquad_root(a, b, sc); // alpha_Higher
            }
            alpha = f2(ok[0] ? asol.x : 2.0f, ok[1] ? asol.y : 2.0f);
            if (ok[0]) br[0] = kBranchSolved;
            if (ok[1]) br[1] = kBranchSolved;
        }
    }
    if (!lbgk) {
        // positivity (Appendix D), per node: alpha beta (-x_min) > 1
        const float2 lim = pmul(pmul(alpha, f2(beta)), f2(xmin[0], xmin[1]));
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            if ((l ? lim.y : lim.x) < -1.0f) {
                const float amax = div_(-1.0f, beta * xmin[l]);
                float al = 0.5f * (1.0f + amax);
                if (al > amax) al = 0.5f * amax;
                if (l) alpha.y = al;
                else alpha.x = al;
                br[l] = kBranchClamped;
            }
        }
    }
    if (kRelax) {
        const float2 ab = pmul(alpha, f2(beta));
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = pfma(pmul(ab, x[i]), fagain(i), f[i]);
    }
    return alpha;
}

// Nodes per thread of the step kernels: two for D2Q9 with FP32 arithmetic (the
// two-node collision), one otherwise.
template <int D, class ST>
__host__ __device__ constexpr int nodes_per_thread()
{
    return (D == 2 && sizeof(typename ST::T) == 4) ? 2 : 1;
}

// Two nodes' collision in a step kernel, on the values loaded with step_in (as
// collide_stored): node_collide_x2 where nodes_per_thread is 2 (alpha_Iterate1, a
// comparison variant with logarithms, stays on the one-node path), else node by node.
template <int D, class ST, bool kRelax = true>
__device__ __forceinline__ void collide2_stored(typename ST::T (&fa)[Lattice<D>::Q],
                                                typename ST::T (&fb)[Lattice<D>::Q], const CollideParams &p)
{
    using T = typename ST::T;
    constexpr int Q = Lattice<D>::Q;
    if constexpr (nodes_per_thread<D, ST>() == 2) {
        if (p.mode != kModeIterate1) {
            float2 v[9], x[9];
            int br[2];
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i] = make_float2(fa[i], fb[i]);
            node_collide_x2<kRelax, ST::kDevCollide>(v, x, p, br);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                fa[i] = v[i].x;
                fb[i] = v[i].y;
            }
            return;
        }
    }
    T x[Q];
    int br;
    collide_stored<D, ST, kRelax>(fa, x, p, &br);
    collide_stored<D, ST, kRelax>(fb, x, p, &br);
}

// Population loads of the step kernels: through the read-only path (ld.global.nc), or,
// with kStream, with the evict-first (streaming) policy (ld.global.cs): each line is read
// once from DRAM and again, within a few warps, by the neighbours' shifted loads.  The
// D3Q27 step takes the second where most nodes need the longer coefficient forms: there it
// spills through L1, and population lines that leave L1 first keep room for the spills
// (D3Q27 256^3 FP32, same box: 0.6807 against 0.6867 ms late in the benchmark flow, but
// 0.5787 against 0.5727 early, where the step is bound by DRAM).
template <bool kStream, class S>
__device__ __forceinline__ S ld_pop(const S *p)
{
    if constexpr (kStream) return __ldcs(p);
    else return __ldg(p);
}

// ---------------------------------------------------------------------------
// Pull streaming (Eq. advection): population i at node (x, y, z) comes from
// (x - c_ix, y - c_iy, z - c_iz) with periodic wrap.
// ---------------------------------------------------------------------------
// f receives populations (ST::load); with kStep, the values a step kernel collides on (step_in).
template <int D, class ST, bool kStep = false>
__device__ __forceinline__ void pull_load(const typename ST::S *__restrict__ fin, const Geometry &g,
                                          int x, int y, int z, float R,
                                          typename ST::T (&f)[Lattice<D>::Q])
{
    using T = typename ST::T;
    constexpr int Q = Lattice<D>::Q;
    const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = vel(D, i, 0), cy = vel(D, i, 1);
        const int cz = D == 3 ? vel(D, i, 2) : 0;
        const int sx = cx == 1 ? xm : (cx == -1 ? xp : x);
        const int sy = cy == 1 ? ym : (cy == -1 ? yp : y);
        const int sz = cz == 1 ? zm : (cz == -1 ? zp : z);
        const int64_t src = ((int64_t)sz * g.ny + sy) * g.nx + sx;
        const typename ST::S sv = __ldg(fin + (int64_t)i * g.N + src);
        f[i] = kStep ? step_in<ST>(sv, dev_ref<D, T>(i, R)) : ST::load(sv, dev_ref<D, T>(i, R));
    }
}

// ---------------------------------------------------------------------------
// Uniform body force F (the paper has none; it serves gradient studies): after
// the collision, the exact-difference term
//   f_i += f^eq_i(rho, u + F/rho) - f^eq_i(rho, u)
// with rho, u the node's moments (the collision conserves them).  It keeps the
// mass and adds exactly F to the momentum.  Evaluated without rounding at the
// scale of w_i u: per axis the factor difference
//   eps(c; v) - eps(c; u) = 2 (t_v - t_u) + 3 c (v - u),
//   t_v - t_u = s_v - s_u = 3 (v - u)(v + u) / (s_v + s_u),
// and f^eq(v) - f^eq(u) = k_i r sum_a d_a prod_{b<a} (1 + eps_b(v)) prod_{b>a} (1 + eps_b(u))
// with the products kept as 1 + (small).
// ---------------------------------------------------------------------------
// f holds populations, or deviations d_i = f_i - k_i R when kDev (the added term is
// the same for both).
template <int D, class T, bool kDev = false>
__device__ __forceinline__ void add_force(T (&f)[Lattice<D>::Q], const CollideParams &p)
{
    constexpr int Q = Lattice<D>::Q;
    T drho = T(0), j[D];
#pragma unroll
    for (int a = 0; a < D; ++a) j[a] = T(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const T di = kDev ? f[i] : f[i] - T(weight_k(D, i)) * T(weight_unit(D)); // exact
        drho += di;
#pragma unroll
        for (int a = 0; a < D; ++a) j[a] += T(vel(D, i, a)) * di;
    }
    T rho;
    if constexpr (kDev) {
        rho = fma(T(Q == 9 ? 36 : 216), T(p.dunit_f), drho);
    } else {
        drho -= T(double(Q == 9 ? 36 : 216) * double(weight_unit_lo<D, T>()));
        rho = T(1) + drho;
    }
    const T irho = T(1) / rho;
    const T r = fma(rho, T(weight_unit(D)), rho * weight_unit_lo<D, T>());
    T eu[D][3], ev[D][3], de[D][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const T u = j[a] * irho, dv = T(p.force[a]) * irho, v = u + dv;
        const T su = sqrt(T(1) + T(3) * u * u), sv = sqrt(T(1) + T(3) * v * v);
        const T tu = T(3) * u * u / (T(1) + su), tv = T(3) * v * v / (T(1) + sv);
        const T dt = T(3) * dv * (u + v) / (su + sv);
        eu[a][0] = T(2) * tu - T(3) * u;
        eu[a][1] = -tu;
        eu[a][2] = T(2) * tu + T(3) * u;
        ev[a][0] = T(2) * tv - T(3) * v;
        ev[a][1] = -tv;
        ev[a][2] = T(2) * tv + T(3) * v;
        de[a][0] = T(2) * dt - T(3) * dv;
        de[a][1] = -dt;
        de[a][2] = T(2) * dt + T(3) * dv;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T dE = T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            T q = T(0); // prod_{b<a} (1 + eps_b(v)) prod_{b>a} (1 + eps_b(u)) - 1
#pragma unroll
            for (int b = 0; b < D; ++b)
                if (b != a) {
                    const T e = b < a ? ev[b][vel(D, i, b) + 1] : eu[b][vel(D, i, b) + 1];
                    q = q + e + q * e;
                }
            const T d = de[a][vel(D, i, a) + 1];
            dE += fma(d, q, d);
        }
        f[i] += (T(weight_k(D, i)) * r) * dE;
    }
}

// ---------------------------------------------------------------------------
// Diagnostics helpers.
// g(y) = (1+y) log(1+y) - y; near 0 the Taylor series
// sum_{k>=2} (-1)^k y^k / (k(k-1)) avoids the cancellation of the direct form.
// The series is summed to k = 20 in FP64 and k = 9 in FP32 (for |y| < 0.1 the
// dropped terms are below the type's rounding).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T g_entropy(T y)
{
    constexpr int kTerms = sizeof(T) == 8 ? 20 : 9;
    if (y <= T(-1)) return T(1);
    if (fabs(y) < T(0.1)) {
        T s = T(0);
#pragma unroll
        for (int k = kTerms; k >= 2; --k) s = s * y + T(((k % 2 == 0) ? 1.0 : -1.0) / double(k * (k - 1)));
        return s * y * y;
    }
    return (T(1) + y) * log1p(y) - y;
}

} // namespace eelbm
