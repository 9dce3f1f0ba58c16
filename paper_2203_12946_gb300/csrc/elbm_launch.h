// elbm_launch.h -- internal (C++) interface between the C-ABI layer and the
// per-lattice kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "elbm.h"

namespace eelbm {

struct Geometry;
struct CollideParams;

// One domain of a batched ensemble: its own periodic box, populations at
// element offset `off` of the shared buffers (SoA [Q][N] inside), and beta.
struct BatchDomain {
    int nx, ny, nz;
    float beta_f; // beta rounded to FP32 on the host
    int64_t N;
    int64_t off;
    double beta;
};

// The domains one batched launch advances, passed by value in the kernel's parameter
// space (a __grid_constant__ argument): domain d's work items -- x-row chunks of the
// launch's width, row-major over (z, y), then x -- are blocks item0[d] .. item0[d+1]-1.
// coarse[b >> shift] is the domain of block (b >> shift) << shift, so a block finds its
// domain with one table read and a short forward scan.  Every thread of a block finds
// the same domain, so the lookup and the row arithmetic are uniform; offsets inside a
// domain are 32-bit (Q N_d < 2^32, checked on creation).
constexpr int kBatchTableDomains = 64;
constexpr int kBatchCoarse = 1024;
struct BatchTableDom {
    int nx, ny, nz, xblocks; // sides, and x-chunks per row
    long long off;           // element offset of the domain's SoA block
    double beta;
    float beta_f;
    int pad;
};
struct BatchTable {
    int n;     // domains in the table
    int shift; // blocks per coarse entry = 2^shift
    int item0[kBatchTableDomains + 1];
    BatchTableDom dom[kBatchTableDomains];
    unsigned char coarse[kBatchCoarse];
};

// Work of one persistent ensemble launch (device arrays): one step is cut into
// nchunks chunks {domain, first item, end item, 0} (items numbered within the
// domain), chunks[k] in domain order; owners[d] chunks belong to domain d, and cnt[d]
// counts its finished (chunk, step) pairs.  Blocks draw tickets from *ticket in
// order: ticket k is chunk k mod nchunks of step k / nchunks.
struct PersistPlan {
    int grid = 0;
    unsigned nchunks = 0;
    const int4 *chunks = nullptr;
    const unsigned *owners = nullptr;
    unsigned *cnt = nullptr;
    unsigned *ticket = nullptr;
};

// Device-side accumulator of the diagnostics reduction (library scratch).
constexpr int kDiagCounts = 9;
struct DiagAcc {
    double sum[6]; // mass, momentum x/y/z, H, sum of alpha
    // cutoff, solved, clamped, nonpositive, dH-positive, then |x|max in
    // [0, 1e-3), [1e-3, 5e-3), [5e-3, 4e-2), [4e-2, inf)
    unsigned long long cnt[kDiagCounts];
    unsigned long long dH_max_ord; // order-preserving encodings of doubles
    unsigned long long amin_ord;
    unsigned long long amax_ord;
    unsigned long long hist[ELBM_HIST_BINS + 2];
};

// Order-preserving map double -> uint64 (unsigned comparison == double
// comparison for non-NaN values) and its inverse.
__host__ __device__ inline unsigned long long ordered_bits(double d)
{
    unsigned long long b;
    memcpy(&b, &d, sizeof b);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
__host__ __device__ inline double from_ordered_bits(unsigned long long o)
{
    unsigned long long b = (o >> 63) ? (o & 0x7FFFFFFFFFFFFFFFULL) : ~o;
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
}

#define ELBM_DECLARE_LAUNCHERS(SUFFIX)                                                               \
    cudaError_t launch_step_##SUFFIX(int storage, const void *fin, void *fout, const Geometry &g,   \
                                     const CollideParams &p, int kernel, int num_sms, int *err,      \
                                     cudaStream_t s);                                                \
    bool rows_kernel_applies_##SUFFIX(int storage, const Geometry &g);                               \
    cudaError_t launch_init_##SUFFIX(int storage, const double *rho, const double *u, void *f,      \
                                     const Geometry &g, double rho_uniform, double rho0,             \
                                     int64_t n0, int64_t count, cudaStream_t s);                     \
    cudaError_t launch_moments_##SUFFIX(int storage, const void *f, const Geometry &g, double rho0, \
                                        double *rho_out, double *u_out, int64_t n0, int64_t count,  \
                                        cudaStream_t s);                                            \
    cudaError_t launch_alpha_##SUFFIX(int storage, const void *f, const Geometry &g,                \
                                      const CollideParams &p, double *alpha_out, uint8_t *flags,    \
                                      double *nut_out, cudaStream_t s);                              \
    cudaError_t launch_diag_##SUFFIX(int storage, const void *f, const Geometry &g,                 \
                                     const CollideParams &p, DiagAcc *acc, int num_sms,             \
                                     cudaStream_t s);                                                \
    cudaError_t launch_step_diag_##SUFFIX(int storage, const void *fin, void *fout, const Geometry &g,    \
                                          const CollideParams &p, DiagAcc *acc, int num_sms,            \
                                          cudaStream_t s);                                              \
    cudaError_t launch_step_batch_##SUFFIX(int storage, const void *fin, void *fout,                \
                                           const BatchTable &tab, int bx, const CollideParams &p,    \
                                           cudaStream_t s);                                          \
    cudaError_t launch_step_persist_##SUFFIX(int storage, void *pop0, void *pop1, int cur, int nsteps,  \
                                             const BatchTableDom *doms, const PersistPlan &plan,     \
                                             int bx, const CollideParams &p, int *err,               \
                                             cudaStream_t s);                                        \
    cudaError_t persist_blocks_per_sm_##SUFFIX(int storage, int bx, int *blocks);                   \
    cudaError_t launch_step_adjoint_##SUFFIX(int storage, const void *fin, const void *gnext,       \
                                             void *gout, const Geometry &g, const CollideParams &p,  \
                                             double *dforce, cudaStream_t s);                        \
    cudaError_t launch_kinetic_energy_##SUFFIX(int storage, const void *f, const Geometry &g,       \
                                               double rho0, double *acc, void *grad, int num_sms,    \
                                               cudaStream_t s);                                      \
    cudaError_t launch_equilibrium_vjp_##SUFFIX(int storage, const double *rho, const double *u,    \
                                                const void *gf, const Geometry &g,                   \
                                                double rho_uniform, double *drho, double *du,        \
                                                cudaStream_t s);

// Sets the message returned by elbm_last_error(NULL) (calls without a handle).
void set_handle_free_error(const char *msg);

ELBM_DECLARE_LAUNCHERS(d2q9)
ELBM_DECLARE_LAUNCHERS(d3q27)

} // namespace eelbm
