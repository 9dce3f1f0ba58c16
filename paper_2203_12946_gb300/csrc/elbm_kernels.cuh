// elbm_kernels.cuh -- kernels of the essentially entropic lattice Boltzmann
// step and its companions, instantiated once per lattice by elbm_d2q9.cu and
// elbm_d3q27.cu (include this file after defining ELBM_DIM and ELBM_SUFFIX).
//
//   k_step     fused pull-stream + collide + store (Eq. advection, Eq.
//              fstar_def, path length of Sec. III / Appendix C-D), one node per
//              thread, ping-pong buffers
//   k_init     f = f^eq(rho, u) (Sec. I equilibrium, FP64, rounded to storage)
//   k_moments  rho and u of the stored state (FP64; exact fixed-point sums of FP32 values)
//   k_alpha    path length of the next collision (no write-back)
//   k_diag     domain reductions: mass, momentum, H (Eq. hdef), alpha statistics
//              and per-node H[f*] - H[f] (Eq. deltaH3) in FP64; warp shuffles,
//              then shared memory, then one atomic per block and quantity
#pragma once

#include "elbm_device.cuh"
#include "elbm_launch.h"
#include "elbm_tma.cuh"
#include "elbm_adjoint.cuh"

namespace eelbm {
namespace ELBM_SUFFIX {

constexpr int D = ELBM_DIM;
constexpr int Q = Lattice<D>::Q;
// Threads per block of the direct step kernel (a tuning knob: block sizes that are
// not a multiple of the register allocation unit leave resident warps unused).
#ifndef ELBM_STEP_BLOCK_D3
#define ELBM_STEP_BLOCK_D3 128
#endif
constexpr int kStepBlock = D == 2 ? 256 : ELBM_STEP_BLOCK_D3;
constexpr int kAuxBlock = 256;


__device__ __forceinline__ void node_coords(int64_t n, const Geometry &g, int &x, int &y, int &z)
{
    if (g.N <= 0xffffffffll) { // 32-bit division where the indices fit (the common case)
        const uint32_t m = uint32_t(n), nx = uint32_t(g.nx), ny = uint32_t(g.ny);
        const uint32_t t = m / nx;
        x = int(m - t * nx);
        z = int(t / ny);
        y = int(t - uint32_t(z) * ny);
        return;
    }
    const int64_t t = n / g.nx;
    x = int(n - t * g.nx);
    z = int(t / g.ny);
    y = int(t - (int64_t)z * g.ny);
}

// One node per thread.  Launched either on a 3D grid (x from blockIdx.x,
// y = blockIdx.y, z = blockIdx.z: no index arithmetic, 32-bit offsets) or, when
// ny or nz exceed the grid limits or Q N reaches 2^32, on a 1D grid over all nodes.
// Minimum resident blocks per SM requested from the register allocator for the
// direct step kernel.  D3Q27 with FP32 storage: 7 blocks of 128 (72 registers).
// Near equilibrium the step is bound by load latency, and the extra resident warps
// outweigh the spills, which fall in the per-population form of the coefficients
// (large |x| only): 0.640 -> 0.627 ms per 256^3 step on GB300.  The 16-bit storages
// lose with that cap (their loads and stores need more live values): 5 blocks, the
// allocation they had unbounded.  FP32 deviations (d_i kept, f_i formed again at each
// use): 6 blocks of 128 (80 registers; 0.6375 against 0.6574 ms early at 7).  FP64 (the
// parity path): no bound.
// ELBM_STEP_MIN_BLOCKS overrides.
#ifndef ELBM_STEP_MIN_BLOCKS
#define ELBM_STEP_MIN_BLOCKS 0
#endif
// D2Q9 with FP32 arithmetic runs two nodes per thread (node_collide_x2), in blocks of
// kStepBlock / 2 threads: 8 of them per SM (at most 64 registers) for FP32 and 16-bit
// storage, 6 (80 registers) for FP32 deviations, whose collision keeps d_i and spills at 64
// (4096^2 shear layer: 0.190 against 0.193 ms; FP32 storage loses with 80: 0.188 against
// 0.179).
#ifndef ELBM_PAIR_MIN_BLOCKS
#define ELBM_PAIR_MIN_BLOCKS 8
#endif
#ifndef ELBM_PAIR_MIN_BLOCKS_DEV
#define ELBM_PAIR_MIN_BLOCKS_DEV 6
#endif
template <class ST>
constexpr int step_min_blocks()
{
    return ELBM_STEP_MIN_BLOCKS > 0 ? ELBM_STEP_MIN_BLOCKS
                                    : (sizeof(typename ST::T) != 4 ? 1
                                       : D == 2 ? (ST::kDevCollide ? ELBM_PAIR_MIN_BLOCKS_DEV : ELBM_PAIR_MIN_BLOCKS)
                                       : ST::kDevCollide          ? 6
                                       : sizeof(typename ST::S) == 4 ? 7 : 5);
}
// Two-node kernels: warp w of a block takes the aligned run of kPairSpan nodes
// [kPairSpan w, kPairSpan (w + 1)) of the block's nodes, lane l nodes l and l + 32 of
// it.  A warp's nodes (and so its coefficient form) are then the same whatever the
// block width, and each of its loads covers 32 consecutive nodes.
constexpr uint32_t kPairSpan = 64;
__device__ __forceinline__ uint32_t pair_node(uint32_t t) { return (t >> 5) * kPairSpan + (t & 31u); }
// threads per block of the direct step kernel
template <class ST>
constexpr int step_threads()
{
    return kStepBlock / nodes_per_thread<D, ST>();
}
#define ELBM_STEP_BOUNDS __launch_bounds__(step_threads<ST>(), step_min_blocks<ST>())

template <class ST, bool kGrid3D, bool kForce = false, bool kStream = false>
__global__ void ELBM_STEP_BOUNDS k_step(const typename ST::S *__restrict__ fin,
                                                    typename ST::S *__restrict__ fout, Geometry g,
                                                    CollideParams p)
{
    using T = typename ST::T;
    if constexpr (nodes_per_thread<D, ST>() == 2) {
        // Two nodes per thread (pair_node); a second node past the end of the row (or of
        // the domain) is a copy of the first, collided and not stored.
        constexpr uint32_t H = kPairSpan / 2;
        T fa[Q], fb[Q];
        if constexpr (kGrid3D) {
            const uint32_t nx = uint32_t(g.nx), ny = uint32_t(g.ny), N = uint32_t(g.N);
            const uint32_t xa = blockIdx.x * kStepBlock + pair_node(threadIdx.x);
            if (xa >= nx) return;
            const bool hasb = xa + H < nx;
            const uint32_t xb = hasb ? xa + H : xa;
            const uint32_t y = blockIdx.y;
            const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            auto src = [&](uint32_t x, int i) -> uint32_t {
                const int cx = vel(D, i, 0), cy = vel(D, i, 1);
                const uint32_t sx = cx == 1 ? (x == 0 ? nx - 1 : x - 1) : (cx == -1 ? (x == nx - 1 ? 0 : x + 1) : x);
                const uint32_t sy = cy == 1 ? ym : (cy == -1 ? yp : y);
                return uint32_t(i) * N + sy * nx + sx;
            };
#pragma unroll
            for (int i = 0; i < Q; ++i) fa[i] = step_in<ST>(ld_pop<false>(fin + src(xa, i)), dev_ref<D, T>(i, p.dunit_f));
#pragma unroll
            for (int i = 0; i < Q; ++i) fb[i] = step_in<ST>(ld_pop<false>(fin + src(xb, i)), dev_ref<D, T>(i, p.dunit_f));
            collide2_stored<D, ST, true>(fa, fb, p);
            if constexpr (kForce) {
                add_force<D, T, ST::kDevCollide>(fa, p);
                add_force<D, T, ST::kDevCollide>(fb, p);
            }
            const uint32_t na = y * nx + xa, nb = y * nx + xb;
#pragma unroll
            for (int i = 0; i < Q; ++i)
                __stcs(fout + (uint32_t(i) * N + na), step_out<ST>(fa[i], dev_ref<D, T>(i, p.dunit_f)));
            if (hasb) {
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    __stcs(fout + (uint32_t(i) * N + nb), step_out<ST>(fb[i], dev_ref<D, T>(i, p.dunit_f)));
            }
        } else {
            const int64_t na = (int64_t)blockIdx.x * kStepBlock + pair_node(threadIdx.x);
            if (na >= g.N) return;
            const bool hasb = na + H < g.N;
            const int64_t nb = hasb ? na + H : na;
            int x, y, z;
            node_coords(na, g, x, y, z);
            pull_load<D, ST, true>(fin, g, x, y, z, p.dunit_f, fa);
            node_coords(nb, g, x, y, z);
            pull_load<D, ST, true>(fin, g, x, y, z, p.dunit_f, fb);
            collide2_stored<D, ST, true>(fa, fb, p);
            if constexpr (kForce) {
                add_force<D, T, ST::kDevCollide>(fa, p);
                add_force<D, T, ST::kDevCollide>(fb, p);
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) __stcs(fout + (int64_t)i * g.N + na, step_out<ST>(fa[i], dev_ref<D, T>(i, p.dunit_f)));
            if (hasb) {
#pragma unroll
                for (int i = 0; i < Q; ++i)
                    __stcs(fout + (int64_t)i * g.N + nb, step_out<ST>(fb[i], dev_ref<D, T>(i, p.dunit_f)));
            }
        }
        return;
    }
    T f[Q], xd[Q]; // the stored values (deviations for deviation storage)
    int br;
    if constexpr (kGrid3D) {
        // 3D grid with Q N < 2^32: element offsets in 32 bits (the source rows of
        // (y - c_y, z - c_z) depend on the block only).  Measured faster on GB300 than
        // per-thread base pointers with block-uniform row offsets.
        const uint32_t x = blockIdx.x * kStepBlock + threadIdx.x;
        const uint32_t nx = uint32_t(g.nx), ny = uint32_t(g.ny), nz = uint32_t(g.nz), N = uint32_t(g.N);
        if (x >= nx) return;
        const uint32_t y = blockIdx.y, z = blockIdx.z;
        const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const uint32_t zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        // element offset of population i pulled into this node
        auto src = [&](int i) -> uint32_t {
            const int cx = vel(D, i, 0), cy = vel(D, i, 1), cz = D == 3 ? vel(D, i, 2) : 0;
            const uint32_t sx = cx == 1 ? xm : (cx == -1 ? xp : x);
            const uint32_t sy = cy == 1 ? ym : (cy == -1 ? yp : y);
            const uint32_t sz = cz == 1 ? zm : (cz == -1 ? zp : z);
            return uint32_t(i) * N + (sz * ny + sy) * nx + sx;
        };
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = step_in<ST>(ld_pop<kStream>(fin + src(i)), dev_ref<D, T>(i, p.dunit_f));
        collide_stored<D, ST, true>(f, xd, p, &br);
        if constexpr (kForce) add_force<D, T, ST::kDevCollide>(f, p);
        const uint32_t n = (z * ny + y) * nx + x;
#pragma unroll
        for (int i = 0; i < Q; ++i) __stcs(fout + (uint32_t(i) * N + n), step_out<ST>(f[i], dev_ref<D, T>(i, p.dunit_f)));
    } else {
        const int64_t n = (int64_t)blockIdx.x * kStepBlock + threadIdx.x;
        if (n >= g.N) return;
        int x, y, z;
        node_coords(n, g, x, y, z);
        pull_load<D, ST, true>(fin, g, x, y, z, p.dunit_f, f);
        collide_stored<D, ST, true>(f, xd, p, &br);
        if constexpr (kForce) add_force<D, T, ST::kDevCollide>(f, p);
#pragma unroll
        for (int i = 0; i < Q; ++i) __stcs(fout + (int64_t)i * g.N + n, step_out<ST>(f[i], dev_ref<D, T>(i, p.dunit_f)));
    }
}

// FP64 equilibrium from rho and u (same product form as node_collide).  Per axis
// phi(-1) = Y den / (6 num) and phi(+1) = Y num / (6 den); with kOneDiv they share one
// division, r = Y / (6 num den), phi(-1) = r den^2, phi(+1) = r num^2 (a few FP64 ulp
// apart: used where the result is rounded to FP32 or below).
template <bool kOneDiv>
__device__ __forceinline__ void equilibrium64(double rho, const double (&u)[3], double (&feq)[Q])
{
    double phi[3][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const double s = sqrt(1.0 + 3.0 * u[a] * u[a]);
        const double Y = 2.0 - s;
        const double num = 2.0 * u[a] + s, den = 1.0 - u[a];
        if (kOneDiv) {
            const double r = Y / (6.0 * num * den);
            phi[a][0] = r * den * den;
            phi[a][2] = r * num * num;
        } else {
            phi[a][0] = Y * den / (6.0 * num);
            phi[a][2] = Y * num / (6.0 * den);
        }
        phi[a][1] = Y * (4.0 / 6.0);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        double v = rho;
#pragma unroll
        for (int a = 0; a < D; ++a) v *= phi[a][vel(D, i, a) + 1];
        feq[i] = v;
    }
}

// Double-length FP32 arithmetic ("double-float": a value hi + lo with |lo| <= ulp(hi)/2):
// Dekker's product with a fused multiply-add for the exact error of hi * hi, Knuth's
// two-sum and Dekker's fast two-sum for additions, and one Newton correction on the FP32
// square root and quotient.  About 44 significant bits, at FP32 instruction rates.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ DF df_from_double(double x)
{
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - double(h))};
}
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const float s = a.hi + b.hi, bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb); // two-sum error
    return df_fast_two_sum(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_mulf(DF a, float b)
{
    const float p = a.hi * b;
    return df_fast_two_sum(p, fmaf(a.lo, b, fmaf(a.hi, b, -p)));
}
__device__ __forceinline__ DF df_div(DF a, DF b)
{
    const float q = a.hi / b.hi;
    const DF qb = df_mulf(b, q);
    const float r = ((a.hi - qb.hi) - qb.lo) + a.lo; // a - q b, to the first order
    return df_fast_two_sum(q, r / b.hi);
}
__device__ __forceinline__ DF df_sqrt(DF a)
{
    const float r = sqrtf(a.hi);
    const float e = fmaf(-r, r, a.hi) + a.lo; // a - r^2
    return df_fast_two_sum(r, e / (2.0f * r));
}

// The equilibrium of equilibrium64<true> in double-float: f^eq rounded once to FP32
// (|stored - f^eq| <= half an FP32 ulp + 2^-43 f^eq), without the FP64 pipe.
__device__ __forceinline__ void equilibrium_df(double rho, const double (&u)[3], float (&feq)[Q])
{
    constexpr double kTwoThirds = 2.0 / 3.0;
    const DF two3 = {float(kTwoThirds), float(kTwoThirds - double(float(kTwoThirds)))};
    DF phi[3][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const DF U = df_from_double(u[a]);
        const DF S = df_sqrt(df_add({1.0f, 0.0f}, df_mulf(df_mul(U, U), 3.0f)));
        const DF Y = df_add({2.0f, 0.0f}, {-S.hi, -S.lo});
        const DF num = df_add({2.0f * U.hi, 2.0f * U.lo}, S), den = df_add({1.0f, 0.0f}, {-U.hi, -U.lo});
        const DF r = df_div(Y, df_mulf(df_mul(num, den), 6.0f));
        phi[a][0] = df_mul(r, df_mul(den, den));
        phi[a][1] = df_mul(Y, two3);
        phi[a][2] = df_mul(r, df_mul(num, num));
    }
    const DF R = df_from_double(rho);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        DF v = R;
#pragma unroll
        for (int a = 0; a < D; ++a) v = df_mul(v, phi[a][vel(D, i, a) + 1]);
        feq[i] = v.hi;
    }
}

// f = f^eq(rho, u) for the nodes n0 .. n0 + count - 1 (SoA with stride g.N).
template <class ST>
__global__ void __launch_bounds__(kAuxBlock) k_init(const double *__restrict__ rho,
                                                   const double *__restrict__ u,
                                                   typename ST::S *__restrict__ f, Geometry g,
                                                   double rho_uniform, double rho0, int64_t n0, int64_t count)
{
    const int64_t k = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
    if (k >= count) return;
    const int64_t n = n0 + k;
    double un[3] = {0.0, 0.0, 0.0}, feq[Q];
#pragma unroll
    for (int a = 0; a < D; ++a) un[a] = u[(int64_t)a * g.N + n];
    if constexpr (!ST::kDev && sizeof(typename ST::S) == 4) {
        // FP32 populations: the equilibrium in double-float, rounded once
        float fe[Q];
        equilibrium_df(rho ? rho[n] : rho_uniform, un, fe);
#pragma unroll
        for (int i = 0; i < Q; ++i) f[(int64_t)i * g.N + n] = fe[i];
        return;
    }
    equilibrium64<sizeof(typename ST::S) < 8>(rho ? rho[n] : rho_uniform, un, feq);
    const double R = double(dev_unit<D>(rho0));
#pragma unroll
    for (int i = 0; i < Q; ++i) f[(int64_t)i * g.N + n] = ST::store64(feq[i], weight_k(D, i) * R);
}

// Exact sums of FP32 values in 64-bit fixed point.  A finite FP32 value is m 2^(e - 150),
// e its biased exponent (taken as 1 for subnormals) and m its significand (with the hidden
// bit for normal numbers).  Scaled to a common exponent E0 = e_max - 33 of the values summed,
// each becomes an integer below 2^57 (a value more than 2^33 below the largest loses its low
// bits), 32 of them add without overflow, and the integer sum converts to FP64 with one
// rounding (none while it stays below 2^53).
__device__ __forceinline__ int f32_expo(float v)
{
    const int e = int((__float_as_uint(v) >> 23) & 0xffu);
    return e ? e : 1;
}
__device__ __forceinline__ long long f32_fixed(float v, int E0)
{
    const uint32_t b = __float_as_uint(v);
    const int e = int((b >> 23) & 0xffu);
    const uint32_t m = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
    const int sh = (e ? e : 1) - E0;
    const unsigned long long mag =
        sh >= 0 ? (unsigned long long)m << sh : (sh > -24 ? (unsigned long long)(m >> -sh) : 0ull);
    return (b >> 31) ? -(long long)mag : (long long)mag;
}
__device__ __forceinline__ double fixed_to_f64(long long q, int E0)
{
    return double(q) * __longlong_as_double((long long)(E0 - 150 + 1023) << 52);
}

// rho and u of the stored state (FP64) for the nodes n0 .. n0 + count - 1.  FP64 storage
// sums in FP64.  The FP32-arithmetic storages hold FP32 values (populations, or deviations
// d_i of the reference c_i = k_i R with sum_i c_i = 6^D R and sum_i c_i c_i = 0): their sums
// are taken exactly in fixed point (f32_fixed) and rounded once to FP64, the result the FP64
// sums of the same values give whenever those are exact, without the FP64 pipe's rate; a
// node holding a value that is not finite is summed in FP64.
template <class ST>
__global__ void __launch_bounds__(kAuxBlock) k_moments(const typename ST::S *__restrict__ f,
                                                      Geometry g, double rho0,
                                                      double *__restrict__ rho_out,
                                                      double *__restrict__ u_out, int64_t n0, int64_t count)
{
    const int64_t k = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
    if (k >= count) return;
    const int64_t n = n0 + k;
    const double R = double(dev_unit<D>(rho0));
    if constexpr (sizeof(typename ST::T) == 4) {
        float v[Q];
        int emax = 1;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            v[i] = ST::raw(f[(int64_t)i * g.N + n]);
            emax = max(emax, f32_expo(v[i]));
        }
        const float Rf = dev_unit<D>(rho0);
        if (ST::kDev) emax = max(emax, f32_expo(Rf) + 8); // 6^D R < 2^8 R
        if (emax < 255) {
            const int E0 = emax - 33;
            long long r = 0, j[3] = {0, 0, 0};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const long long q = f32_fixed(v[i], E0);
                r += q;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    if (vel(D, i, a) == 1) j[a] += q;
                    if (vel(D, i, a) == -1) j[a] -= q;
                }
            }
            if (ST::kDev) r += f32_fixed(Rf, E0) * (Q == 9 ? 36 : 216);
            const double rho = fixed_to_f64(r, E0);
            if (rho_out) rho_out[n] = rho;
            if (u_out) {
                const double ir = 1.0 / rho;
#pragma unroll
                for (int a = 0; a < D; ++a) u_out[(int64_t)a * g.N + n] = fixed_to_f64(j[a], E0) * ir;
            }
            return;
        }
    }
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const double v = ST::load64(f[(int64_t)i * g.N + n], weight_k(D, i) * R);
        r += v;
#pragma unroll
        for (int a = 0; a < D; ++a) j[a] += vel(D, i, a) * v;
    }
    if (rho_out) rho_out[n] = r;
    if (u_out) {
#pragma unroll
        for (int a = 0; a < D; ++a) u_out[(int64_t)a * g.N + n] = j[a] / r;
    }
}

// Path length of the next collision; optionally the subgrid viscosity of Sec. VI,
// nu_T = theta dt (2 - alpha) / (2 alpha beta) (Eq. nuT, theta = 1/3, dt = 1).
template <class ST>
__global__ void __launch_bounds__(kStepBlock) k_alpha(const typename ST::S *__restrict__ fin,
                                                     Geometry g, CollideParams p,
                                                     double *__restrict__ alpha_out,
                                                     uint8_t *__restrict__ flags,
                                                     double *__restrict__ nut_out)
{
    using T = typename ST::T;
    const int64_t n = (int64_t)blockIdx.x * kStepBlock + threadIdx.x;
    if (n >= g.N) return;
    int x, y, z;
    node_coords(n, g, x, y, z);
    T f[Q], xd[Q];
    pull_load<D, ST, true>(fin, g, x, y, z, p.dunit_f, f); // stored values, as the step collides them
    int br;
    const T alpha = collide_stored<D, ST, false>(f, xd, p, &br);
    if (alpha_out) alpha_out[n] = double(alpha);
    if (flags) flags[n] = uint8_t(br);
    if (nut_out) nut_out[n] = (1.0 / 3.0) * (2.0 - double(alpha)) / (2.0 * double(alpha) * p.beta);
}

// --------------------------------------------------------------------------
// Diagnostics reduction.
// --------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_max(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ unsigned long long warp_min(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Per-thread accumulation of the domain diagnostics of a node and of the collision
// it undergoes (used by k_diag and by the step fused with diagnostics).  Partial sums
// in the compute type of the small parts (deviations, H + 1, alpha - 2) over the
// thread's nodes; the exact parts (one per node, 2 per alpha) and the conversion to
// FP64 are added once per thread in diag_finish (FP64 arithmetic is slow on this GPU,
// and per node it was a third of the pass).
template <class T>
struct DiagThread {
    double sum[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long cnt[kDiagCounts] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long dmax = 0ULL, amin = ~0ULL, amax = 0ULL;
    T p_dr = T(0), p_j[3] = {T(0), T(0), T(0)}, p_h = T(0), p_al = T(0);
    T p_dmax = -INFINITY, p_amin = INFINITY, p_amax = -INFINITY;
    unsigned long long p_nodes = 0, p_hnodes = 0;

    // fc: the node's pre-collision populations; xd, alpha_t, br: departures, path length
    // and branch of its collision; s_hist: the block's histogram in shared memory.
    __device__ __forceinline__ void node(const T (&fc)[Q], const T (&xd)[Q], const T alpha_t, const int br,
                                         const CollideParams &p, unsigned int *s_hist)
    {
        bool bad = false;
#pragma unroll
        for (int i = 0; i < Q; ++i) bad |= !(fc[i] > T(0)) || !isfinite(fc[i]);

        // Mass and momentum through the deviations d_i = f_i - w_i (small numbers).
        T dr = T(0), jt[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T di = fc[i] - T(weight(D, i));
            dr += di;
#pragma unroll
            for (int a = 0; a < D; ++a) jt[a] += T(vel(D, i, a)) * di;
        }
        p_nodes += 1;
        p_dr += dr;
        for (int a = 0; a < D; ++a) p_j[a] += jt[a];
        if (bad) {
            cnt[3] += 1;
        } else {
            // H[f] = <f, log(f/w)> - rho (Eq. hdef), with log(f/w) = log1p(d/w), and
            // the entropy change of this node's collision (Eq. deltaH3, with <f,x> = 0
            // removing alpha beta <f,x> from both sums):
            // H[f*] - H[f] = <f, g(ab x)> - ab <f, x log(1+x)>, g(y) = (1+y) log(1+y) - y.
            // Per-node sums in the path's compute type, domain sums in FP64.
            const T ab = alpha_t * beta_of<T>(p);
            T hl = T(0), s3 = T(0), xa = T(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const T fi = fc[i], xi = xd[i];
                hl += fi * log1p((fi - T(weight(D, i))) * T(1.0 / weight(D, i)));
                s3 += fi * xi * xi;
                xa = fmax(xa, fabs(xi));
            }
            T dH;
            if (xa < T(0.1) && ab <= T(2.2)) {
                // g(ab x) - ab x log(1+x) = sum_{k>=2} c_k x^k,
                // c_k = (-1)^k ab/(k-1) (ab^(k-1)/k - 1), summed to k = kTop (for |x| < 0.1
                // and ab <= 2.2 the rest is below 5e-10 x^2).  c_2 = ab (ab - 2)/2 takes
                // ab - 2 from one rounding of alpha beta - 2; the two sums of the direct
                // form cancel to that small leading coefficient instead.
                constexpr int kTop = 13;
                T ck[kTop + 1];
                ck[2] = T(0.5) * ab * fma(alpha_t, beta_of<T>(p), T(-2));
                T abk = ab * ab; // ab^(k-1) at k = 3
#pragma unroll
                for (int k = 3; k <= kTop; ++k) {
                    const T v = ab * T(1.0 / (k - 1)) * (abk * T(1.0 / k) - T(1));
                    ck[k] = (k & 1) ? -v : v;
                    abk *= ab;
                }
                T sd = T(0);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const T xi = xd[i];
                    T poly = ck[kTop];
#pragma unroll
                    for (int k = kTop - 1; k >= 2; --k) poly = fma(poly, xi, ck[k]);
                    sd += fc[i] * (poly * xi * xi);
                }
                dH = sd;
            } else {
                T s1 = T(0), s2 = T(0);
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const T fi = fc[i], xi = xd[i];
                    s1 += fi * g_entropy<T>(ab * xi);
                    s2 += fi * xi * log1p(xi);
                }
                dH = s1 - ab * s2;
            }
            // H of the node + (1 + e_w) (the node's -rho without its exact part)
            p_h += hl - dr;
            p_hnodes += 1;
            p_dmax = fmax(p_dmax, dH);
            if (dH > T(1e-6) * s3 && s3 > T(0)) cnt[4] += 1;
            // |x|max band: the cutoff of Appendix D, then the FP32 coefficient forms
            cnt[xa < T(1e-3) ? 5 : (xa < T(5e-3) ? 6 : (xa < T(4e-2) ? 7 : 8))] += 1;
        }
        p_al += alpha_t - T(2);
        cnt[br == kBranchCutoff ? 0 : (br == kBranchSolved ? 1 : 2)] += 1;
        p_amin = fmin(p_amin, alpha_t);
        p_amax = fmax(p_amax, alpha_t);
        // bin of alpha on [1.9, 2.1): alpha - 1.9 with 1.9 in two parts of T
        constexpr T kLo = T(1.9), kLo2 = T(1.9 - double(T(1.9)));
        const T off = (alpha_t - kLo) - kLo2;
        int bin;
        if (!(off >= T(0))) bin = 0;
        else if (off >= T(0.2)) bin = ELBM_HIST_BINS + 1;
        else bin = 1 + min(ELBM_HIST_BINS - 1, int(off * T(ELBM_HIST_BINS / 0.2)));
        atomicAdd(&s_hist[bin], 1u);
    }
};

// Block reduction of the per-thread diagnostics into the FP64 accumulator (warp
// shuffles, then shared memory, then one atomic per block and quantity).  NT >= 65.
template <int NT, class T>
__device__ __forceinline__ void diag_finish(DiagThread<T> &dt, DiagAcc *__restrict__ acc, unsigned int *s_hist)
{
    constexpr int kWarps = NT / 32;
    __shared__ double s_sum[kWarps][6];
    __shared__ unsigned long long s_cnt[kWarps][kDiagCounts];
    __shared__ unsigned long long s_ext[kWarps][3];
    double (&sum)[6] = dt.sum;
    unsigned long long (&cnt)[kDiagCounts] = dt.cnt;
    unsigned long long &dmax = dt.dmax, &amin = dt.amin, &amax = dt.amax;
    const T &p_dr = dt.p_dr, &p_h = dt.p_h, &p_al = dt.p_al;
    const T(&p_j)[3] = dt.p_j;
    const T &p_dmax = dt.p_dmax, &p_amin = dt.p_amin, &p_amax = dt.p_amax;
    const unsigned long long p_nodes = dt.p_nodes, p_hnodes = dt.p_hnodes;
    // this thread's nodes into the FP64 sums: mass = sum (1 + e_w + dr), H = sum hl - rho
    {
        const double nn = double(p_nodes), one = 1.0 + weight_sum_error<D, T>();
        sum[0] = nn * one + double(p_dr);
        for (int a = 0; a < D; ++a) sum[1 + a] = double(p_j[a]);
        sum[4] = double(p_h) - double(p_hnodes) * one;
        sum[5] = 2.0 * nn + double(p_al);
        if (p_nodes) {
            dmax = p_hnodes ? ordered_bits(double(p_dmax)) : 0ULL;
            amin = ordered_bits(double(p_amin));
            amax = ordered_bits(double(p_amax));
        }
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) sum[k] = warp_sum(sum[k]);
#pragma unroll
    for (int k = 0; k < kDiagCounts; ++k) cnt[k] = warp_sum(cnt[k]);
    dmax = warp_max(dmax);
    amin = warp_min(amin);
    amax = warp_max(amax);
    if (lane == 0) {
        for (int k = 0; k < 6; ++k) s_sum[warp][k] = sum[k];
        for (int k = 0; k < kDiagCounts; ++k) s_cnt[warp][k] = cnt[k];
        s_ext[warp][0] = dmax;
        s_ext[warp][1] = amin;
        s_ext[warp][2] = amax;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0.0;
        for (int w = 0; w < kWarps; ++w) v += s_sum[w][threadIdx.x];
        atomicAdd(&acc->sum[threadIdx.x], v);
    } else if (threadIdx.x >= 32 && threadIdx.x < 32 + kDiagCounts) {
        const int k = threadIdx.x - 32;
        unsigned long long v = 0;
        for (int w = 0; w < kWarps; ++w) v += s_cnt[w][k];
        atomicAdd(&acc->cnt[k], v);
    } else if (threadIdx.x == 64) {
        unsigned long long a = 0, b = ~0ULL, c = 0;
        for (int w = 0; w < kWarps; ++w) {
            a = max(a, s_ext[w][0]);
            b = min(b, s_ext[w][1]);
            c = max(c, s_ext[w][2]);
        }
        atomicMax(&acc->dH_max_ord, a);
        atomicMin(&acc->amin_ord, b);
        atomicMax(&acc->amax_ord, c);
    }
    for (int b = threadIdx.x; b < ELBM_HIST_BINS + 2; b += NT)
        if (s_hist[b]) atomicAdd(&acc->hist[b], (unsigned long long)s_hist[b]);
}

template <class ST>
__global__ void __launch_bounds__(kAuxBlock) k_diag(const typename ST::S *__restrict__ fin,
                                                   Geometry g, CollideParams p,
                                                   DiagAcc *__restrict__ acc)
{
    using T = typename ST::T;
    __shared__ unsigned int s_hist[ELBM_HIST_BINS + 2];
    for (int b = threadIdx.x; b < ELBM_HIST_BINS + 2; b += kAuxBlock) s_hist[b] = 0u;
    __syncthreads();
    DiagThread<T> dt;
    for (int64_t n = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x; n < g.N;
         n += (int64_t)gridDim.x * kAuxBlock) {
        int x, y, z;
        node_coords(n, g, x, y, z);
        T f[Q], xd[Q], fc[Q];
        pull_load<D, ST, true>(fin, g, x, y, z, p.dunit_f, f); // stored values, as the step collides them
#pragma unroll
        for (int i = 0; i < Q; ++i) fc[i] = ST::kDevCollide ? f[i] + dev_ref<D, T>(i, p.dunit_f) : f[i]; // populations
        int br;
        const T alpha_t = collide_stored<D, ST, false>(f, xd, p, &br);
        dt.node(fc, xd, alpha_t, br, p, s_hist);
    }
    diag_finish<kAuxBlock>(dt, acc, s_hist);
}

// The step fused with the diagnostics of the state it advances (the quantities of
// k_diag, taken from the collision the step performs): 3D-grid addressing with 32-bit
// offsets, one node per thread, a grid of a few blocks per SM looping over the
// (x-block, y, z) items so that each block reduces and posts its sums once.
// Its own register budget: the diagnostics' extra live values spilled heavily under
// the step's 72-register cap (3 blocks of 128 for D3Q27, 2 of 256 for D2Q9; FP64 unbounded).
template <class ST>
constexpr int step_diag_min_blocks()
{
    return sizeof(typename ST::T) != 4 ? 1 : (D == 3 ? 3 : 2);
}
template <class ST>
__global__ void __launch_bounds__(kStepBlock, step_diag_min_blocks<ST>()) k_step_diag(const typename ST::S *__restrict__ fin,
                                             typename ST::S *__restrict__ fout, Geometry g, CollideParams p,
                                             DiagAcc *__restrict__ acc)
{
    using T = typename ST::T;
    __shared__ unsigned int s_hist[ELBM_HIST_BINS + 2];
    for (int b = threadIdx.x; b < ELBM_HIST_BINS + 2; b += kStepBlock) s_hist[b] = 0u;
    __syncthreads();
    DiagThread<T> dt;
    const uint32_t nx = uint32_t(g.nx), ny = uint32_t(g.ny), nz = uint32_t(g.nz), N = uint32_t(g.N);
    const uint32_t xblocks = (nx + kStepBlock - 1) / kStepBlock;
    const uint32_t items = xblocks * ny * nz;
    for (uint32_t it = blockIdx.x; it < items; it += gridDim.x) {
        const uint32_t xb = it % xblocks, yz = it / xblocks;
        const uint32_t y = yz % ny, z = yz / ny;
        const uint32_t x = xb * kStepBlock + threadIdx.x;
        if (x >= nx) continue;
        const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const uint32_t zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        T f[Q], xd[Q], fc[Q];
        auto src = [&](int i) -> uint32_t {
            const int cx = vel(D, i, 0), cy = vel(D, i, 1), cz = D == 3 ? vel(D, i, 2) : 0;
            const uint32_t sx = cx == 1 ? xm : (cx == -1 ? xp : x);
            const uint32_t sy = cy == 1 ? ym : (cy == -1 ? yp : y);
            const uint32_t sz = cz == 1 ? zm : (cz == -1 ? zp : z);
            return uint32_t(i) * N + (sz * ny + sy) * nx + sx;
        };
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[i] = step_in<ST>(ld_pop<false>(fin + src(i)), dev_ref<D, T>(i, p.dunit_f));
            fc[i] = ST::kDevCollide ? f[i] + dev_ref<D, T>(i, p.dunit_f) : f[i]; // populations
        }
        int br;
        const T alpha_t = collide_stored<D, ST, true>(f, xd, p, &br);
        dt.node(fc, xd, alpha_t, br, p, s_hist);
        const uint32_t n = (z * ny + y) * nx + x;
#pragma unroll
        for (int i = 0; i < Q; ++i) __stcs(fout + (uint32_t(i) * N + n), step_out<ST>(f[i], dev_ref<D, T>(i, p.dunit_f)));
    }
    diag_finish<kStepBlock>(dt, acc, s_hist);
}

// Two nodes x and x + 32 of row y of a D2Q9 domain (nx by ny, N nodes, populations
// at in / out): pull, collide (node_collide_x2), store; a second node past the end of
// the row is a copy of the first, collided and not stored.  Plain loads when kCoherent
// (buffers written during the launch), else ld_pop.
template <class ST, bool kCoherent = false>
__device__ __forceinline__ void step2_row(const typename ST::S *in, typename ST::S *out, uint32_t nx, uint32_t ny,
                                          uint32_t N, uint32_t xa, uint32_t y, const CollideParams &p)
{
    using T = typename ST::T;
    constexpr uint32_t H = kPairSpan / 2;
    const bool hasb = xa + H < nx;
    const uint32_t xb = hasb ? xa + H : xa;
    const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    auto src = [&](uint32_t x, int i) -> uint32_t {
        const int cx = vel(D, i, 0), cy = vel(D, i, 1);
        const uint32_t sx = cx == 1 ? (x == 0 ? nx - 1 : x - 1) : (cx == -1 ? (x == nx - 1 ? 0 : x + 1) : x);
        const uint32_t sy = cy == 1 ? ym : (cy == -1 ? yp : y);
        return uint32_t(i) * N + sy * nx + sx;
    };
    auto ld = [&](uint32_t o) { return kCoherent ? in[o] : ld_pop<false>(in + o); };
    T fa[Q], fb[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fa[i] = step_in<ST>(ld(src(xa, i)), dev_ref<D, T>(i, p.dunit_f));
#pragma unroll
    for (int i = 0; i < Q; ++i) fb[i] = step_in<ST>(ld(src(xb, i)), dev_ref<D, T>(i, p.dunit_f));
    collide2_stored<D, ST, true>(fa, fb, p);
    const uint32_t na = y * nx + xa, nb = y * nx + xb;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const typename ST::S v = step_out<ST>(fa[i], dev_ref<D, T>(i, p.dunit_f));
        if (kCoherent) out[uint32_t(i) * N + na] = v;
        else __stcs(out + (uint32_t(i) * N + na), v);
    }
    if (hasb) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const typename ST::S v = step_out<ST>(fb[i], dev_ref<D, T>(i, p.dunit_f));
            if (kCoherent) out[uint32_t(i) * N + nb] = v;
            else __stcs(out + (uint32_t(i) * N + nb), v);
        }
    }
}

// --------------------------------------------------------------------------
// --------------------------------------------------------------------------
// Batched ensemble: one launch advances up to kBatchTableDomains domains.  Block
// b is one work item, nodes x0 .. x0 + BX - 1 of one x-row of one domain; the
// block finds its domain in the launch's parameter table (a coarse index, then a
// forward scan over the item counts) and its row by division, both uniform over the
// block, so each thread then addresses its populations as k_step does (32-bit
// offsets inside the domain).  Each domain has its own beta; everything else is the
// single-domain step.
// --------------------------------------------------------------------------
// Resident threads per SM requested from the register allocator for the batched ensemble
// kernel (0: no bound).  Two-node D2Q9 kernels: 1024 (at most 64 registers; 74.7 against
// 65.7 GLUPS on the 64-domain ensemble with the 80 the compiler picks unbounded), 768 for
// FP32 deviations (80 registers); one node per thread: no bound.  The persistent kernel
// keeps the compiler's choice (bounded to 64 registers it spills: 60.2 against 62.6 GLUPS).
#ifndef ELBM_BATCH_THREADS_PER_SM
#define ELBM_BATCH_THREADS_PER_SM 0
#endif
template <class ST>
constexpr int batch_threads_per_sm()
{
    return ELBM_BATCH_THREADS_PER_SM > 0 ? ELBM_BATCH_THREADS_PER_SM
           : nodes_per_thread<D, ST>() == 2 ? (ST::kDevCollide ? 768 : 1024)
                                            : 0;
}
template <class ST, int BX>
constexpr int batch_min_blocks()
{
    return batch_threads_per_sm<ST>() / (BX / nodes_per_thread<D, ST>());
}
template <class ST, int BX>
__global__ void __launch_bounds__(BX / nodes_per_thread<D, ST>(), batch_min_blocks<ST, BX>()) k_step_batch(const typename ST::S *__restrict__ fin,
                                                  typename ST::S *__restrict__ fout,
                                                  const __grid_constant__ BatchTable tab, CollideParams p)
{
    using T = typename ST::T;
    const int bid = int(blockIdx.x);
    int lo = tab.coarse[bid >> tab.shift]; // item0[lo] <= bid
    while (tab.item0[lo + 1] <= bid) ++lo;
    const BatchTableDom &dm = tab.dom[lo];
    const uint32_t nx = uint32_t(dm.nx), ny = uint32_t(dm.ny), nz = uint32_t(dm.nz), xb = uint32_t(dm.xblocks);
    const uint32_t it = uint32_t(bid - tab.item0[lo]);
    const uint32_t row = it / xb;
    const uint32_t x = (it - row * xb) * BX + (nodes_per_thread<D, ST>() == 2 ? pair_node(threadIdx.x) : threadIdx.x);
    if (x >= nx) return;
    const uint32_t z = row / ny, y = row - z * ny, N = nx * ny * nz;
    p.beta = dm.beta;
    p.beta_f = dm.beta_f;
    const typename ST::S *in = fin + dm.off;
    typename ST::S *out = fout + dm.off;
    if constexpr (nodes_per_thread<D, ST>() == 2) {
        // two nodes per thread (D2Q9: z = 0), as in k_step
        step2_row<ST>(in, out, nx, ny, N, x, y, p);
        return;
    }
    const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const uint32_t zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    T f[Q], xd[Q];
    auto src = [&](int i) -> uint32_t {
        const int cx = vel(D, i, 0), cy = vel(D, i, 1), cz = D == 3 ? vel(D, i, 2) : 0;
        const uint32_t sx = cx == 1 ? xm : (cx == -1 ? xp : x);
        const uint32_t sy = cy == 1 ? ym : (cy == -1 ? yp : y);
        const uint32_t sz = cz == 1 ? zm : (cz == -1 ? zp : z);
        return uint32_t(i) * N + (sz * ny + sy) * nx + sx;
    };
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = step_in<ST>(ld_pop<false>(in + src(i)), dev_ref<D, T>(i, p.dunit_f));
    int br;
    collide_stored<D, ST, true>(f, xd, p, &br);
    const uint32_t n = (z * ny + y) * nx + x;
#pragma unroll
    for (int i = 0; i < Q; ++i) __stcs(out + (uint32_t(i) * N + n), step_out<ST>(f[i], dev_ref<D, T>(i, p.dunit_f)));
}

// --------------------------------------------------------------------------
// Persistent ensemble: one cooperative launch advances every domain by nsteps.
// Blocks draw tickets in order from one counter; ticket k is chunk k mod M of step
// k / M (plan.chunks: runs of work items inside one domain, numbered within it and
// located by division as in k_step_batch).  Domains are independent, so before step
// t on domain d a block waits only until cnt[d] has counted every chunk of d at step
// t - 1 (release: stores, barrier, fence, atomic add; acquire: bounded spin, fence,
// barrier).  The chunks it waits for hold smaller tickets, so the smallest unfinished
// ticket never waits and the launch cannot deadlock; idle blocks take the next chunk
// at once, which balances the domains as the hardware scheduler does for separate
// launches.  Populations are read with plain coherent loads, not through the read-only
// path, since the buffers change during the launch; offsets inside a domain are 32-bit
// (Q N < 2^32 per domain, checked when the batch is created).  Every wait is bounded
// (kWaitLimitNs of %globaltimer, also abandoned once another block has flagged an
// error): on expiry the block records ELBM_ERR_TIMEOUT in *err and returns.
// --------------------------------------------------------------------------
__device__ __forceinline__ bool wait_count(const unsigned *cnt, unsigned target, const int *err)
{
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
        if (v >= target) return true;
        if (*(volatile const int *)err != 0 || global_ns() - t0 > kWaitLimitNs) return false;
        __nanosleep(64);
    }
}

template <class ST, int BX>
__global__ void __launch_bounds__(BX / nodes_per_thread<D, ST>()) k_step_persist(typename ST::S *pop0, typename ST::S *pop1, int cur,
                                                    int nsteps, const BatchTableDom *__restrict__ doms,
                                                    PersistPlan plan, CollideParams p, int *err)
{
    using T = typename ST::T;
    using S = typename ST::S;
    __shared__ unsigned s_ticket;
    __shared__ int s_ok;
    const unsigned M = plan.nchunks, total = unsigned(nsteps) * M; // below 2^32 (host)
    const uint32_t tx = nodes_per_thread<D, ST>() == 2 ? pair_node(threadIdx.x) : threadIdx.x;
    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(plan.ticket, 1u);
        __syncthreads();
        const unsigned tk = s_ticket;
        if (tk >= total) return;
        const unsigned t = tk / M;
        const int4 seg = plan.chunks[tk - t * M];
        if (t > 0) {
            if (threadIdx.x == 0) {
                s_ok = wait_count(plan.cnt + seg.x, t * plan.owners[seg.x], err);
                if (!s_ok) atomicExch(err, ELBM_ERR_TIMEOUT);
                __threadfence();
            }
            __syncthreads();
            if (!s_ok) return;
        }
        const bool odd = ((unsigned(cur) + t) & 1u) != 0;
        const S *fin = odd ? pop1 : pop0;
        S *fout = odd ? pop0 : pop1;
        const BatchTableDom dm = doms[seg.x];
        p.beta = dm.beta;
        p.beta_f = dm.beta_f;
        const uint32_t nx = uint32_t(dm.nx), ny = uint32_t(dm.ny), nz = uint32_t(dm.nz), N = nx * ny * nz;
        const uint32_t xb = uint32_t(dm.xblocks);
        const S *in = fin + dm.off;
        S *out = fout + dm.off;
        // the chunk's work items: row-major (z, y), then the x-chunk c; one division for
        // the first item, then counters
        uint32_t row = uint32_t(seg.y) / xb, c = uint32_t(seg.y) - row * xb;
        uint32_t z = row / ny, y = row - z * ny;
        for (uint32_t w = uint32_t(seg.y); w < uint32_t(seg.z); ++w) {
            const uint32_t x = c * BX + tx;
            const uint32_t yc = y, zc = z;
            if (++c == xb) { // next row
                c = 0;
                if (++y == ny) {
                    y = 0;
                    ++z;
                }
            }
            if (x >= nx) continue;
            if constexpr (nodes_per_thread<D, ST>() == 2) {
                step2_row<ST, true>(in, out, nx, ny, N, x, yc, p);
                continue;
            }
            const uint32_t y = yc, z = zc;
            const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
            const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
            const uint32_t zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
            T f[Q], xd[Q];
            auto src = [&](int i) -> uint32_t {
                const int cx = vel(D, i, 0), cy = vel(D, i, 1), cz = D == 3 ? vel(D, i, 2) : 0;
                const uint32_t sx = cx == 1 ? xm : (cx == -1 ? xp : x);
                const uint32_t sy = cy == 1 ? ym : (cy == -1 ? yp : y);
                const uint32_t sz = cz == 1 ? zm : (cz == -1 ? zp : z);
                return uint32_t(i) * N + (sz * ny + sy) * nx + sx;
            };
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = step_in<ST>(in[src(i)], dev_ref<D, T>(i, p.dunit_f));
            int br;
            collide_stored<D, ST, true>(f, xd, p, &br);
            const uint32_t n = (z * ny + y) * nx + x;
#pragma unroll
            for (int i = 0; i < Q; ++i) out[uint32_t(i) * N + n] = step_out<ST>(f[i], dev_ref<D, T>(i, p.dunit_f));
        }
        __syncthreads(); // every store of this chunk issued; s_ticket and s_ok read by all
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(plan.cnt + seg.x, 1u);
        }
    }
}

// --------------------------------------------------------------------------
// Adjoint of one step (f^{t+1} = collide(stream(f^t))): given gnext = dL/df^{t+1},
// write gout = dL/df^t.  Per node x: the pre-collision populations F(x) are
// pulled from f^t as in the step, h = J^T gnext(x) is the collision's VJP, and
// the transpose of pull streaming sends h_i(x) to node x - c_i (a push).
// Gradient arrays are SoA [Q][N] in the compute type.
// --------------------------------------------------------------------------
template <class ST, bool kForce = false>
__global__ void __launch_bounds__(kAuxBlock) k_step_adjoint(const typename ST::S *__restrict__ fin,
                                                           const typename ST::T *__restrict__ gnext,
                                                           typename ST::T *__restrict__ gout, Geometry g,
                                                           CollideParams p, double *__restrict__ dforce)
{
    using T = typename ST::T;
    const int64_t n = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
    T dfl[3] = {T(0), T(0), T(0)};
    if (n < g.N) {
        int x, y, z;
        node_coords(n, g, x, y, z);
        T F[Q], gl[Q], h[Q];
        pull_load<D, ST>(fin, g, x, y, z, p.dunit_f, F);
#pragma unroll
        for (int i = 0; i < Q; ++i) gl[i] = gnext[(int64_t)i * g.N + n];
        node_vjp<D, T, kForce>(F, gl, p, h, dfl);
        const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int cx = vel(D, i, 0), cy = vel(D, i, 1), cz = D == 3 ? vel(D, i, 2) : 0;
            const int dx = cx == 1 ? xm : (cx == -1 ? xp : x);
            const int dy = cy == 1 ? ym : (cy == -1 ? yp : y);
            const int dz = cz == 1 ? zm : (cz == -1 ? zp : z);
            gout[(int64_t)i * g.N + ((int64_t)dz * g.ny + dy) * g.nx + dx] = h[i];
        }
    }
    if constexpr (kForce) {
        // d/dF_b summed over the block (FP64), one atomic per block and component
        __shared__ double s_df[kAuxBlock / 32][3];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const double v = warp_sum(double(dfl[a]));
            if (lane == 0) s_df[warp][a] = v;
        }
        __syncthreads();
        if (dforce && threadIdx.x < D) {
            double v = 0.0;
            for (int w = 0; w < kAuxBlock / 32; ++w) v += s_df[w][threadIdx.x];
            atomicAdd(&dforce[threadIdx.x], v);
        }
    }
}

// Kinetic energy L = 1/2 sum rho |u|^2 of a stored field (FP64 sum into acc[0])
// and, optionally, its gradient dL/df_i = c_i . u - |u|^2 / 2.
template <class ST>
__global__ void __launch_bounds__(kAuxBlock) k_kinetic_energy(const typename ST::S *__restrict__ f,
                                                             Geometry g, double rho0, double *__restrict__ acc,
                                                             typename ST::T *__restrict__ grad)
{
    using T = typename ST::T;
    double e = 0.0;
    const double R = double(dev_unit<D>(rho0));
    for (int64_t n = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x; n < g.N; n += (int64_t)gridDim.x * kAuxBlock) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        double fv[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            fv[i] = ST::load64(f[(int64_t)i * g.N + n], weight_k(D, i) * R);
            r += fv[i];
#pragma unroll
            for (int a = 0; a < D; ++a) j[a] += vel(D, i, a) * fv[i];
        }
        double uu = 0.0, u[3];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            u[a] = j[a] / r;
            uu += u[a] * u[a];
        }
        e += 0.5 * r * uu;
        if (grad) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                double cu = 0.0;
#pragma unroll
                for (int a = 0; a < D; ++a) cu += vel(D, i, a) * u[a];
                grad[(int64_t)i * g.N + n] = T(cu - 0.5 * uu);
            }
        }
    }
    e = warp_sum(e);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, e);
}

// Derivatives of f = f^eq(rho, u) (the initial state) with respect to rho and u:
// drho = sum_i g_i feq_i / rho, du_a = sum_i g_i feq_i d log phi_a(c_ia) / du_a.
template <class T>
__global__ void __launch_bounds__(kAuxBlock) k_equilibrium_vjp(const double *__restrict__ rho,
                                                              const double *__restrict__ u,
                                                              const T *__restrict__ gf, Geometry g, double rho_uniform,
                                                              double *__restrict__ drho, double *__restrict__ du)
{
    const int64_t n = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
    if (n >= g.N) return;
    const double r = rho ? rho[n] : rho_uniform;
    double phi[3][3], dlp[3][3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const double ua = u[(int64_t)a * g.N + n];
        const double s = sqrt(1.0 + 3.0 * ua * ua), Y = 2.0 - s, num = 2.0 * ua + s, den = 1.0 - ua;
        const double zz = num / den, dY = -3.0 * ua / s, dlz = (2.0 + 3.0 * ua / s) / num + 1.0 / den;
        phi[a][0] = Y / (6.0 * zz);
        phi[a][1] = Y * (4.0 / 6.0);
        phi[a][2] = Y * zz / 6.0;
        dlp[a][0] = dY / Y - dlz;
        dlp[a][1] = dY / Y;
        dlp[a][2] = dY / Y + dlz;
    }
    double sr = 0.0, su[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        double v = r;
#pragma unroll
        for (int a = 0; a < D; ++a) v *= phi[a][vel(D, i, a) + 1];
        const double gv = double(gf[(int64_t)i * g.N + n]) * v;
        sr += gv;
#pragma unroll
        for (int a = 0; a < D; ++a) su[a] += gv * dlp[a][vel(D, i, a) + 1];
    }
    if (drho) drho[n] = sr / r;
    if (du) {
#pragma unroll
        for (int a = 0; a < D; ++a) du[(int64_t)a * g.N + n] = su[a];
    }
}

// --------------------------------------------------------------------------
// Launchers (storage dispatch).
// --------------------------------------------------------------------------
#define ELBM_STORAGE_SWITCH(storage, CALL)                                                     \
    switch (storage) {                                                                         \
    case ELBM_STORE_F64: { using ST = StoreF64; CALL; break; }                                 \
    case ELBM_STORE_F32: { using ST = StoreF32; CALL; break; }                                 \
    case ELBM_STORE_F32DEV: { using ST = StoreF32Dev; CALL; break; }                           \
    case ELBM_STORE_F16DEV: { using ST = StoreF16Dev; CALL; break; }                           \
    case ELBM_STORE_BF16DEV: { using ST = StoreBF16Dev; CALL; break; }                         \
    default: return cudaErrorInvalidValue;                                                     \
    }

static inline unsigned blocks_for(int64_t N, int block) { return unsigned((N + block - 1) / block); }

} // namespace ELBM_SUFFIX

#define ELBM_CAT2(a, b) a##_##b
#define ELBM_CAT(a, b) ELBM_CAT2(a, b)

// A lattice may be compiled in two units: ELBM_PART 1 holds the step launcher (and the
// row pipeline), ELBM_PART 2 every other launcher; without ELBM_PART one unit holds all.
#if !defined(ELBM_PART) || ELBM_PART == 1
namespace ELBM_SUFFIX {

// Row-staged instantiations: (NXMAX, stages) per storage element size.
constexpr int kRowThreads = 256;
template <class S>
constexpr int row_stages()
{
    return sizeof(S) >= 4 ? (D == 3 ? 3 : 3) : 5;
}

template <class ST, int NXMAX>
cudaError_t launch_rows(const void *fin, void *fout, const Geometry &g, const CollideParams &p, int num_sms,
                        int *err, cudaStream_t s)
{
    using S = typename ST::S;
    constexpr int STAGES = (D == 3 && NXMAX > 256) ? 2 : row_stages<S>();
    constexpr size_t smem = rows_smem_bytes<Q, S, NXMAX, STAGES>();
    auto kern = k_step_rows<D, ST, NXMAX, kRowThreads, STAGES>;
    // one-time set-up per instantiation (single-device library use)
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kRowThreads, smem);
        if (e != cudaSuccess) return e;
        per_sm = n < 1 ? 1 : n;
    }
    const int rows = g.ny * g.nz;
    int grid = per_sm * (num_sms > 0 ? num_sms : 1);
    if (grid > rows) grid = rows;
    kern<<<grid, kRowThreads, smem, s>>>(static_cast<const S *>(fin), static_cast<S *>(fout), g, p, err);
    return cudaGetLastError();
}

template <class ST>
int rows_nxmax(const Geometry &g)
{
    using S = typename ST::S;
    if (ST::kRows == 0) return 0;
    if ((size_t(g.nx) * sizeof(S)) % 16 != 0) return 0;
    const int cands[3] = {D == 3 ? 128 : 256, D == 3 ? 256 : 1024, D == 3 ? 512 : 0};
    for (int c : cands)
        if (c && g.nx <= c) return c;
    return 0;
}

} // namespace ELBM_SUFFIX

bool ELBM_CAT(rows_kernel_applies, ELBM_SUFFIX)(int storage, const Geometry &g)
{
    using namespace ELBM_SUFFIX;
    switch (storage) {
    case ELBM_STORE_F32: return rows_nxmax<StoreF32>(g) > 0;
    case ELBM_STORE_F32DEV: return rows_nxmax<StoreF32Dev>(g) > 0;
    case ELBM_STORE_F16DEV: return rows_nxmax<StoreF16Dev>(g) > 0;
    case ELBM_STORE_BF16DEV: return rows_nxmax<StoreBF16Dev>(g) > 0;
    default: return false;
    }
}

cudaError_t ELBM_CAT(launch_step, ELBM_SUFFIX)(int storage, const void *fin, void *fout,
                                               const Geometry &g, const CollideParams &p, int kernel,
                                               int num_sms, int *err, cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    if (g.N == 0) return cudaSuccess;
    const bool forced = p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0;
    // AUTO takes DIRECT: on GB300 it is the faster of the two at every size measured
    // (D3Q27 256^3 FP32: 0.63 ms against 0.70 ms for ROWS).  The body force runs on DIRECT only.
    if (kernel == ELBM_KERNEL_ROWS && forced) return cudaErrorNotSupported;
    if (kernel == ELBM_KERNEL_ROWS && ELBM_CAT(rows_kernel_applies, ELBM_SUFFIX)(storage, g)) {
        // the row pipeline is only instantiated for the FP32 and 16-bit storages
#define ELBM_ROWS_FOR(STT)                                                                        \
    {                                                                                             \
        const int nm = rows_nxmax<STT>(g);                                                        \
        if (nm == (D == 3 ? 128 : 256))                                                           \
            return launch_rows<STT, (D == 3 ? 128 : 256)>(fin, fout, g, p, num_sms, err, s);      \
        if (nm == (D == 3 ? 256 : 1024))                                                          \
            return launch_rows<STT, (D == 3 ? 256 : 1024)>(fin, fout, g, p, num_sms, err, s);     \
        if (D == 3 && nm == 512) return launch_rows<STT, 512>(fin, fout, g, p, num_sms, err, s);  \
    }
        switch (storage) {
        case ELBM_STORE_F32: ELBM_ROWS_FOR(StoreF32) break;
        case ELBM_STORE_F32DEV: ELBM_ROWS_FOR(StoreF32Dev) break;
        case ELBM_STORE_F16DEV: ELBM_ROWS_FOR(StoreF16Dev) break;
        case ELBM_STORE_BF16DEV: ELBM_ROWS_FOR(StoreBF16Dev) break;
        default: break;
        }
#undef ELBM_ROWS_FOR
    }
    if (kernel == ELBM_KERNEL_ROWS) return cudaErrorNotSupported;
    if (g.ny <= 65535 && g.nz <= 65535 && uint64_t(Q) * uint64_t(g.N) <= 0xffffffffull) {
        const dim3 grid(unsigned((g.nx + kStepBlock - 1) / kStepBlock), unsigned(g.ny), unsigned(g.nz));
        if constexpr (D == 3) {
            // the evict-first variant for the FP32-arithmetic storages (FP64, the parity
            // path, keeps the read-only path)
            if (!forced && p.pop_stream && storage != ELBM_STORE_F64) {
#define ELBM_STREAM_STEP(STT)                                                                     \
    k_step<STT, true, false, true><<<grid, step_threads<STT>(), 0, s>>>(                          \
        static_cast<const typename STT::S *>(fin), static_cast<typename STT::S *>(fout), g, p)
                switch (storage) {
                case ELBM_STORE_F32: ELBM_STREAM_STEP(StoreF32); break;
                case ELBM_STORE_F32DEV: ELBM_STREAM_STEP(StoreF32Dev); break;
                case ELBM_STORE_F16DEV: ELBM_STREAM_STEP(StoreF16Dev); break;
                case ELBM_STORE_BF16DEV: ELBM_STREAM_STEP(StoreBF16Dev); break;
                default: return cudaErrorInvalidValue;
                }
#undef ELBM_STREAM_STEP
                return cudaGetLastError();
            }
        }
        if (forced) {
            ELBM_STORAGE_SWITCH(storage, (k_step<ST, true, true><<<grid, step_threads<ST>(), 0, s>>>(
                                             static_cast<const typename ST::S *>(fin),
                                             static_cast<typename ST::S *>(fout), g, p)));
        } else {
            ELBM_STORAGE_SWITCH(storage, (k_step<ST, true><<<grid, step_threads<ST>(), 0, s>>>(
                                             static_cast<const typename ST::S *>(fin),
                                             static_cast<typename ST::S *>(fout), g, p)));
        }
    } else {
        if (forced) {
            ELBM_STORAGE_SWITCH(storage,
                                (k_step<ST, false, true><<<blocks_for(g.N, kStepBlock), step_threads<ST>(), 0, s>>>(
                                    static_cast<const typename ST::S *>(fin),
                                    static_cast<typename ST::S *>(fout), g, p)));
        } else {
            ELBM_STORAGE_SWITCH(storage, (k_step<ST, false><<<blocks_for(g.N, kStepBlock), step_threads<ST>(), 0, s>>>(
                                             static_cast<const typename ST::S *>(fin),
                                             static_cast<typename ST::S *>(fout), g, p)));
        }
    }
    return cudaGetLastError();
}

#endif

#if !defined(ELBM_PART) || ELBM_PART == 2
cudaError_t ELBM_CAT(launch_step_diag, ELBM_SUFFIX)(int storage, const void *fin, void *fout, const Geometry &g,
                                                    const CollideParams &p, DiagAcc *acc, int num_sms,
                                                    cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    if (g.N == 0) return cudaSuccess;
    const bool forced = p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0;
    if (forced || uint64_t(Q) * uint64_t(g.N) > 0xffffffffull) return cudaErrorNotSupported;
    const uint64_t items = uint64_t((g.nx + kStepBlock - 1) / kStepBlock) * uint64_t(g.ny) * uint64_t(g.nz);
    const uint64_t cap = uint64_t(num_sms > 0 ? num_sms : 1) * 8u;
    const unsigned grid = unsigned(items < cap ? items : cap);
    ELBM_STORAGE_SWITCH(storage, (k_step_diag<ST><<<grid, kStepBlock, 0, s>>>(
                                     static_cast<const typename ST::S *>(fin), static_cast<typename ST::S *>(fout),
                                     g, p, acc)));
    return cudaGetLastError();
}

cudaError_t ELBM_CAT(launch_step_batch, ELBM_SUFFIX)(int storage, const void *fin, void *fout,
                                                     const BatchTable &tab, int bx, const CollideParams &p,
                                                     cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    const int nitems = tab.item0[tab.n];
    if (tab.n <= 0 || nitems <= 0) return cudaSuccess;
#define ELBM_BATCH_BX(BXV)                                                                             \
    ELBM_STORAGE_SWITCH(storage, (k_step_batch<ST, BXV><<<unsigned(nitems), BXV / nodes_per_thread<D, ST>(), 0, s>>>( \
                                     static_cast<const typename ST::S *>(fin),                          \
                                     static_cast<typename ST::S *>(fout), tab, p)))
    switch (bx) {
    case 64: ELBM_BATCH_BX(64); break;
    case 128: ELBM_BATCH_BX(128); break;
    case 256: ELBM_BATCH_BX(256); break;
    default: return cudaErrorInvalidValue;
    }
#undef ELBM_BATCH_BX
    return cudaGetLastError();
}

cudaError_t ELBM_CAT(persist_blocks_per_sm, ELBM_SUFFIX)(int storage, int bx, int *blocks)
{
    using namespace ELBM_SUFFIX;
    *blocks = 0;
#define ELBM_PERSIST_OCC(BXV)                                                                          \
    ELBM_STORAGE_SWITCH(storage, return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks,           \
                                                                             k_step_persist<ST, BXV>, BXV / nodes_per_thread<D, ST>(), 0))
    switch (bx) {
    case 64: ELBM_PERSIST_OCC(64); break;
    case 128: ELBM_PERSIST_OCC(128); break;
    case 256: ELBM_PERSIST_OCC(256); break;
    default: return cudaErrorInvalidValue;
    }
#undef ELBM_PERSIST_OCC
    return cudaErrorInvalidValue;
}

cudaError_t ELBM_CAT(launch_step_persist, ELBM_SUFFIX)(int storage, void *pop0, void *pop1, int cur, int nsteps,
                                                       const BatchTableDom *doms, const PersistPlan &plan, int bx,
                                                       const CollideParams &p, int *err, cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    if (nsteps <= 0 || plan.grid <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative; // all blocks resident: they wait on one another
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(unsigned(plan.grid));
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define ELBM_PERSIST_BX(BXV)                                                                           \
    ELBM_STORAGE_SWITCH(storage, cfg.blockDim = dim3(BXV / nodes_per_thread<D, ST>());                 \
                                 return cudaLaunchKernelEx(&cfg, k_step_persist<ST, BXV>,               \
                                                           static_cast<typename ST::S *>(pop0),        \
                                                           static_cast<typename ST::S *>(pop1), cur,   \
                                                           nsteps, doms, plan, p, err))
    switch (bx) {
    case 64: ELBM_PERSIST_BX(64); break;
    case 128: ELBM_PERSIST_BX(128); break;
    case 256: ELBM_PERSIST_BX(256); break;
    default: return cudaErrorInvalidValue;
    }
#undef ELBM_PERSIST_BX
    return cudaErrorInvalidValue;
}

cudaError_t ELBM_CAT(launch_step_adjoint, ELBM_SUFFIX)(int storage, const void *fin, const void *gnext,
                                                       void *gout, const Geometry &g, const CollideParams &p,
                                                       double *dforce, cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    if (g.N == 0) return cudaSuccess;
    const bool forced = dforce || p.force[0] != 0.0 || p.force[1] != 0.0 || p.force[2] != 0.0;
    if (forced) {
        ELBM_STORAGE_SWITCH(storage, (k_step_adjoint<ST, true><<<blocks_for(g.N, kAuxBlock), kAuxBlock, 0, s>>>(
                                         static_cast<const typename ST::S *>(fin),
                                         static_cast<const typename ST::T *>(gnext),
                                         static_cast<typename ST::T *>(gout), g, p, dforce)));
    } else {
        ELBM_STORAGE_SWITCH(storage, (k_step_adjoint<ST><<<blocks_for(g.N, kAuxBlock), kAuxBlock, 0, s>>>(
                                         static_cast<const typename ST::S *>(fin),
                                         static_cast<const typename ST::T *>(gnext),
                                         static_cast<typename ST::T *>(gout), g, p, nullptr)));
    }
    return cudaGetLastError();
}

cudaError_t ELBM_CAT(launch_kinetic_energy, ELBM_SUFFIX)(int storage, const void *f, const Geometry &g, double rho0,
                                                         double *acc, void *grad, int num_sms, cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    if (g.N == 0) return cudaSuccess;
    unsigned blocks = blocks_for(g.N, kAuxBlock);
    const unsigned cap = unsigned(num_sms > 0 ? num_sms : 1) * 8u;
    if (blocks > cap) blocks = cap;
    ELBM_STORAGE_SWITCH(storage, (k_kinetic_energy<ST><<<blocks, kAuxBlock, 0, s>>>(
                                     static_cast<const typename ST::S *>(f), g, rho0, acc,
                                     static_cast<typename ST::T *>(grad))));
    return cudaGetLastError();
}

cudaError_t ELBM_CAT(launch_equilibrium_vjp, ELBM_SUFFIX)(int storage, const double *rho, const double *u,
                                                          const void *gf, const Geometry &g, double rho_uniform,
                                                          double *drho, double *du, cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    if (g.N == 0) return cudaSuccess;
    if (storage == ELBM_STORE_F64)
        k_equilibrium_vjp<double><<<blocks_for(g.N, kAuxBlock), kAuxBlock, 0, s>>>(
            rho, u, static_cast<const double *>(gf), g, rho_uniform, drho, du);
    else
        k_equilibrium_vjp<float><<<blocks_for(g.N, kAuxBlock), kAuxBlock, 0, s>>>(
            rho, u, static_cast<const float *>(gf), g, rho_uniform, drho, du);
    return cudaGetLastError();
}

cudaError_t ELBM_CAT(launch_init, ELBM_SUFFIX)(int storage, const double *rho, const double *u,
                                               void *f, const Geometry &g, double rho_uniform,
                                               double rho0, int64_t n0, int64_t count, cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    if (count <= 0) return cudaSuccess;
    ELBM_STORAGE_SWITCH(storage, (k_init<ST><<<blocks_for(count, kAuxBlock), kAuxBlock, 0, s>>>(
                                     rho, u, static_cast<typename ST::S *>(f), g, rho_uniform, rho0, n0, count)));
    return cudaGetLastError();
}

cudaError_t ELBM_CAT(launch_moments, ELBM_SUFFIX)(int storage, const void *f, const Geometry &g,
                                                  double rho0, double *rho_out, double *u_out,
                                                  int64_t n0, int64_t count, cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    if (count <= 0) return cudaSuccess;
    ELBM_STORAGE_SWITCH(storage, (k_moments<ST><<<blocks_for(count, kAuxBlock), kAuxBlock, 0, s>>>(
                                     static_cast<const typename ST::S *>(f), g, rho0, rho_out, u_out, n0, count)));
    return cudaGetLastError();
}

cudaError_t ELBM_CAT(launch_alpha, ELBM_SUFFIX)(int storage, const void *f, const Geometry &g,
                                                const CollideParams &p, double *alpha_out,
                                                uint8_t *flags, double *nut_out, cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    if (g.N == 0) return cudaSuccess;
    ELBM_STORAGE_SWITCH(storage, (k_alpha<ST><<<blocks_for(g.N, kStepBlock), kStepBlock, 0, s>>>(
                                     static_cast<const typename ST::S *>(f), g, p, alpha_out, flags, nut_out)));
    return cudaGetLastError();
}

cudaError_t ELBM_CAT(launch_diag, ELBM_SUFFIX)(int storage, const void *f, const Geometry &g,
                                               const CollideParams &p, DiagAcc *acc, int num_sms,
                                               cudaStream_t s)
{
    using namespace ELBM_SUFFIX;
    if (g.N == 0) return cudaSuccess;
    unsigned blocks = blocks_for(g.N, kAuxBlock);
    const unsigned cap = unsigned(num_sms > 0 ? num_sms : 1) * 8u;
    if (blocks > cap) blocks = cap;
    ELBM_STORAGE_SWITCH(storage, (k_diag<ST><<<blocks, kAuxBlock, 0, s>>>(
                                     static_cast<const typename ST::S *>(f), g, p, acc)));
    return cudaGetLastError();
}

#endif

} // namespace eelbm
