// elbm_tma.cuh -- bulk-async (TMA engine) row staging for the fused step.
//
// A persistent CTA walks over x-rows (fixed y, z) of the lattice.  For a row,
// pull streaming (Eq. advection) needs, for every velocity i, the source row
// (y - c_iy, z - c_iz) shifted by c_ix along x.  Because a row spans the whole
// periodic x extent, the shift is a wrap-around index into the staged row, so
// each velocity needs exactly one contiguous row of nx elements: one
// cp.async.bulk copy of nx * sizeof(S) bytes into shared memory, completed on an
// mbarrier.  STAGES rows are in flight while one is being collided.
//
// Waits on the mbarriers are bounded: after kWaitLimitNs (1 s) the CTA records
// ELBM_ERR_TIMEOUT in *err, waits (again bounded) for the copies it issued, and
// leaves.  The decision to leave is taken by the whole CTA (__syncthreads_or) so
// no thread is left at a barrier.
#pragma once

#include "elbm.h"
#include "elbm_device.cuh"

namespace eelbm {

// Wall-clock limit of a device-side wait (nanoseconds of %globaltimer).
constexpr unsigned long long kWaitLimitNs = 1000000000ULL;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait; returns false once kWaitLimitNs have passed without completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int n = 0; n < 256; ++n)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
}

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16),
// completion counted in bytes on *bar.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                              uint64_t policy)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
                 " [%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
                 : "memory");
}

// Shared-memory bytes of the row pipeline.
template <int Q, class S, int NXMAX, int STAGES>
constexpr size_t rows_smem_bytes()
{
    return size_t(STAGES) * Q * NXMAX * sizeof(S);
}

// ---------------------------------------------------------------------------
// The fused step over staged rows.  Requirements (checked by the launcher):
// nx <= NXMAX, nx * sizeof(S) % 16 == 0, 16-byte aligned buffers.
//
// Stage hand-off without CTA barriers: every warp waits for the stage's
// mbarrier, collides its nodes of the row, and then increments the stage's
// release counter; the warp that brings the counter to the number of warps is
// the last reader of that stage, so it resets the counter and issues the bulk
// copies of the row STAGES iterations ahead into it.  A warp whose bounded wait
// expires raises the CTA's abort flag (the other warps see it in their own
// waits) and the error word; the CTA then lets its issued copies land and exits.
// ---------------------------------------------------------------------------
template <int D, class ST, int NXMAX, int NT, int STAGES>
__global__ void __launch_bounds__(NT) k_step_rows(const typename ST::S *__restrict__ fin,
                                                  typename ST::S *__restrict__ fout, Geometry g,
                                                  CollideParams p, int *__restrict__ err)
{
    using S = typename ST::S;
    using T = typename ST::T;
    constexpr int Q = Lattice<D>::Q;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S *tiles = reinterpret_cast<S *>(smem_raw); // [STAGES][Q][NXMAX]
    __shared__ uint64_t bar[STAGES];
    __shared__ int released[STAGES];
    __shared__ int armed[STAGES]; // iteration index last issued into each stage
    __shared__ volatile int abort_flag;

    const int rows = g.ny * g.nz;
    const int G = gridDim.x;
    if (int(blockIdx.x) >= rows) return; // uniform over the CTA
    const uint32_t row_bytes = uint32_t(g.nx) * uint32_t(sizeof(S));
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&bar[s], 1);
            released[s] = 0;
            armed[s] = -1;
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();

    const uint64_t policy = l2_policy_evict_first();

    // Issue the Q source rows of iteration k (destination row blockIdx.x + k G) into
    // stage k % STAGES; called by one whole warp: lane 0 posts the byte count, lane
    // i < Q copies velocity i's source row.
    auto issue = [&](int k) {
        const int row = int(blockIdx.x) + k * G;
        const int st = k % STAGES;
        if (lane == 0) {
            armed[st] = k;
            mbar_arrive_expect_tx(&bar[st], uint32_t(Q) * row_bytes);
        }
        __syncwarp();
        const int y = row % g.ny, z = row / g.ny;
        for (int i = lane; i < Q; i += 32) {
            const int cy = (D == 2 ? i : i / 3) % 3 - 1; // velocity component along y
            const int cz = D == 3 ? i % 3 - 1 : 0;       // along z (D3Q27)
            int sy = y - cy, sz = z - cz;                 // pull: source row of velocity i
            sy = sy < 0 ? sy + g.ny : (sy >= g.ny ? sy - g.ny : sy);
            sz = sz < 0 ? sz + g.nz : (sz >= g.nz ? sz - g.nz : sz);
            const S *src = fin + (int64_t)i * g.N + ((int64_t)sz * g.ny + sy) * g.nx;
            bulk_copy_g2s(tiles + ((size_t)st * Q + i) * NXMAX, src, row_bytes, &bar[st], policy);
        }
    };

    const int iters = (rows - int(blockIdx.x) + G - 1) / G;
    if (threadIdx.x < 32) {
        for (int k = 0; k < STAGES && k < iters; ++k) issue(k);
    }
    __syncthreads(); // the first stages are armed before anyone waits on them

    bool aborted = false;
    for (int k = 0; k < iters; ++k) {
        const int row = int(blockIdx.x) + k * G;
        const int st = k % STAGES;
        const uint32_t parity = uint32_t(k / STAGES) & 1u;
        // bounded wait, abandoned as soon as another warp has aborted
        bool ok = mbar_try_wait(&bar[st], parity);
        if (!ok) {
            const unsigned long long t0 = global_ns();
            while (!ok) {
                for (int n = 0; n < 256 && !ok; ++n) ok = mbar_try_wait(&bar[st], parity);
                if (ok) break;
                if (abort_flag || global_ns() - t0 > kWaitLimitNs) break;
            }
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                abort_flag = 1;
                atomicExch(err, ELBM_ERR_TIMEOUT);
            }
            aborted = true;
            break;
        }
        const S *tile = tiles + (size_t)st * Q * NXMAX;
        const int64_t rowbase = (int64_t)row * g.nx;
        for (int x = threadIdx.x; x < g.nx; x += NT) {
            const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
            T f[Q], xd[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int cx = vel(D, i, 0);
                const int sx = cx == 1 ? xm : (cx == -1 ? xp : x);
                f[i] = step_in<ST>(tile[i * NXMAX + sx], dev_ref<D, T>(i, p.dunit_f));
            }
            int br;
            collide_stored<D, ST, true>(f, xd, p, &br);
#pragma unroll
            for (int i = 0; i < Q; ++i) __stcs(fout + (int64_t)i * g.N + rowbase + x, step_out<ST>(f[i], dev_ref<D, T>(i, p.dunit_f)));
        }
        // release the stage; the last warp out refills it
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&released[st], 1) == NW - 1;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            if (lane == 0) {
                released[st] = 0;
                __threadfence_block();
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (k + STAGES < iters) issue(k + STAGES);
        }
    }

    __syncthreads();
    if (aborted || abort_flag) {
        if (threadIdx.x == 0) {
            atomicExch(err, ELBM_ERR_TIMEOUT);
            // let the copies already issued land before the CTA's shared memory goes away
            for (int s = 0; s < STAGES; ++s)
                if (armed[s] >= 0) mbar_wait_bounded(&bar[s], uint32_t(armed[s] / STAGES) & 1u);
        }
        __syncthreads();
    }
}

} // namespace eelbm
