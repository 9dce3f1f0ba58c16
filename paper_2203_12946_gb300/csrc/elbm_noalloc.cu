// elbm_noalloc.cu -- elbm_diagnostics_noalloc: the domain diagnostics of a
// caller-owned population buffer without any device allocation.
//
// Why it exists: elbm_diagnostics needs a handle, and elbm_create allocates
// device memory (the reduction accumulator, an error word).  Some callers can
// not allocate at all: an application whose device memory is owned by another
// allocator or a fixed pool, code that must not grow its footprint after
// start-up, or a monitoring hook running inside someone else's time step.
// This entry point takes the populations directly and keeps its reduction
// accumulator in a file-scope __device__ array that is part of the library
// image, so nothing is allocated per call.
//
// The array is allocated on every GPU that loads the library and lives until
// the process exits.  All calls share it; each call clears it first, and
// calls that overlap on the GPU (different streams, or host threads issuing
// concurrently) race on it and must be serialised by the caller.  The array's
// device address is looked up once per device and kept; a cudaDeviceReset
// destroys the context it belongs to, so the call is not valid after one in the
// same process.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "elbm.h"
#include "elbm_device.cuh"
#include "elbm_launch.h"

namespace {

using eelbm::DiagAcc;

// The scratch: one diagnostics accumulator record, rounded up to the stated
// maximum of ELBM_NOALLOC_SCRATCH_BYTES.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ELBM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool ready = false;
    void *scratch = nullptr; // device address of g_noalloc_scratch on this device
    int num_sms = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// Failures are reported through elbm_last_error(NULL).
int noalloc_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    eelbm::set_handle_free_error(buf);
    return code;
}

} // namespace

extern "C" int elbm_diagnostics_noalloc(int lattice, const int64_t dims[3], double beta, const elbm_opts *opts,
                                        const void *populations, elbm_diag *out, int64_t *alpha_hist)
{
    if (!dims || !populations || !out)
        return noalloc_fail(ELBM_ERR_ARG, "elbm_diagnostics_noalloc: null argument");
    if (lattice != ELBM_D2Q9 && lattice != ELBM_D3Q27)
        return noalloc_fail(ELBM_ERR_ARG, "elbm_diagnostics_noalloc: lattice must be 9 or 27, got %d", lattice);
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (int64_t(1) << 30))
            return noalloc_fail(ELBM_ERR_ARG, "elbm_diagnostics_noalloc: dims[%d] = %lld out of range", a,
                                (long long)dims[a]);
    if (lattice == ELBM_D2Q9 && dims[2] != 1)
        return noalloc_fail(ELBM_ERR_ARG, "elbm_diagnostics_noalloc: D2Q9 needs dims[2] == 1");
    // the node count in 128 bits: each side may reach 2^30, and their product must not
    // wrap around in 64 bits before it is compared
    const unsigned __int128 nodes = (unsigned __int128)dims[0] * (unsigned __int128)dims[1] * (unsigned __int128)dims[2];
    if (nodes > ((unsigned __int128)1 << 31))
        return noalloc_fail(ELBM_ERR_ARG, "elbm_diagnostics_noalloc: more than 2^31 nodes");
    if (!(beta > 0.0 && beta < 1.0))
        return noalloc_fail(ELBM_ERR_ARG, "elbm_diagnostics_noalloc: beta must lie in (0, 1), got %g", beta);
    elbm_opts o;
    elbm_default_opts(&o);
    if (opts) o = *opts;
    size_t elem = 0;
    switch (o.storage) {
    case ELBM_STORE_F64: elem = 8; break;
    case ELBM_STORE_F32:
    case ELBM_STORE_F32DEV: elem = 4; break;
    case ELBM_STORE_F16DEV:
    case ELBM_STORE_BF16DEV: elem = 2; break;
    default: return noalloc_fail(ELBM_ERR_ARG, "elbm_diagnostics_noalloc: unknown storage %d", o.storage);
    }
    // the buffer does not come from the library: a pointer that is not aligned to its
    // element would make the kernel's loads fault
    if (reinterpret_cast<uintptr_t>(populations) % elem != 0)
        return noalloc_fail(ELBM_ERR_ARG,
                            "elbm_diagnostics_noalloc: populations is not aligned to its %zu-byte element", elem);
    if (o.alpha_mode < ELBM_ALPHA_HIGHER || o.alpha_mode > ELBM_ALPHA_ITERATE1 || (o.cutoff != 0 && o.cutoff != 1) ||
        (o.b_variant != ELBM_B_DERIVED && o.b_variant != ELBM_B_PRINTED) || !(o.rho0 > 0.0))
        return noalloc_fail(ELBM_ERR_ARG, "elbm_diagnostics_noalloc: invalid options");
    // The scratch this call needs must fit the fixed array.
    const size_t need = sizeof(DiagAcc);
    if (need > size_t(ELBM_NOALLOC_SCRATCH_BYTES))
        return noalloc_fail(ELBM_ERR_ARG,
                            "elbm_diagnostics_noalloc: needs %zu bytes of scratch, the fixed maximum is %d",
                            need, ELBM_NOALLOC_SCRATCH_BYTES);

    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(ELBM_ERR_CUDA, "elbm_diagnostics_noalloc: cudaGetDevice: %s",
                                              cudaGetErrorString(e));
    if (!opts) o.device = dev; // no options: the current device
    if (dev != o.device) {
        return noalloc_fail(ELBM_ERR_ARG,
                            "elbm_diagnostics_noalloc: opts->device = %d but device %d is current; make the "
                            "populations' device current before the call",
                            o.device, dev);
    }
    if (dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(ELBM_ERR_ARG, "elbm_diagnostics_noalloc: device ordinal %d not supported", dev);
    // the buffer must be device (or managed) memory of the current device; the query
    // allocates nothing
    cudaPointerAttributes attr;
    e = cudaPointerGetAttributes(&attr, populations);
    if (e != cudaSuccess) {
        cudaGetLastError(); // the failed query leaves no error behind for later calls
        return noalloc_fail(ELBM_ERR_ARG, "elbm_diagnostics_noalloc: populations is not a CUDA pointer (%s)",
                            cudaGetErrorString(e));
    }
    if ((attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) || attr.device != dev)
        return noalloc_fail(ELBM_ERR_ARG,
                            "elbm_diagnostics_noalloc: populations is not device memory of the current device %d",
                            dev);

    // Set-up once per device, with that device current: the device address of
    // the scratch array (its host-side name is only a stand-in) and the SM count.
    DeviceSetup setup;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        DeviceSetup &s = g_setup[dev];
        if (!s.ready) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return noalloc_fail(ELBM_ERR_CUDA, "elbm_diagnostics_noalloc: cudaGetSymbolAddress: %s",
                                    cudaGetErrorString(e));
            int sms = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess)
                return noalloc_fail(ELBM_ERR_CUDA, "elbm_diagnostics_noalloc: cudaDeviceGetAttribute: %s",
                                    cudaGetErrorString(e));
            s.scratch = ptr;
            s.num_sms = sms;
            s.ready = true;
        }
        setup = s;
    }

    cudaStream_t stream = static_cast<cudaStream_t>(o.stream);
    DiagAcc *acc = static_cast<DiagAcc *>(setup.scratch);
    // The array keeps the previous call's sums: clear it (min-encoded alpha starts at all ones).
    e = cudaMemsetAsync(acc, 0, sizeof(DiagAcc), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&acc->amin_ord, 0xFF, sizeof(unsigned long long), stream);
    if (e != cudaSuccess)
        return noalloc_fail(ELBM_ERR_CUDA, "elbm_diagnostics_noalloc: clear scratch: %s", cudaGetErrorString(e));

    eelbm::Geometry g;
    g.nx = int(dims[0]);
    g.ny = int(dims[1]);
    g.nz = int(dims[2]);
    g.N = dims[0] * dims[1] * dims[2];
    eelbm::CollideParams p;
    p.beta = beta;
    p.mode = o.alpha_mode;
    p.cutoff = o.cutoff;
    p.b_variant = o.b_variant;
    p.rho0 = o.rho0;
    p.beta_f = float(p.beta);
    p.dunit_f = lattice == ELBM_D2Q9 ? eelbm::dev_unit<2>(p.rho0) : eelbm::dev_unit<3>(p.rho0);
    e = lattice == ELBM_D2Q9 ? eelbm::launch_diag_d2q9(o.storage, populations, g, p, acc, setup.num_sms, stream)
                             : eelbm::launch_diag_d3q27(o.storage, populations, g, p, acc, setup.num_sms, stream);
    if (e != cudaSuccess)
        return noalloc_fail(ELBM_ERR_CUDA, "elbm_diagnostics_noalloc: kernel launch: %s", cudaGetErrorString(e));
    DiagAcc host;
    e = cudaMemcpyAsync(&host, acc, sizeof host, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess)
        return noalloc_fail(ELBM_ERR_CUDA, "elbm_diagnostics_noalloc: read back: %s", cudaGetErrorString(e));

    const int64_t N = g.N;
    out->mass = host.sum[0];
    out->momentum[0] = host.sum[1];
    out->momentum[1] = host.sum[2];
    out->momentum[2] = lattice == ELBM_D3Q27 ? host.sum[3] : 0.0;
    out->H = host.sum[4];
    out->dH_max = eelbm::from_ordered_bits(host.dH_max_ord);
    out->alpha_min = eelbm::from_ordered_bits(host.amin_ord);
    out->alpha_max = eelbm::from_ordered_bits(host.amax_ord);
    out->alpha_mean = host.sum[5] / double(N);
    out->n_nodes = N;
    out->n_cutoff = int64_t(host.cnt[0]);
    out->n_solved = int64_t(host.cnt[1]);
    out->n_clamped = int64_t(host.cnt[2]);
    out->n_nonpositive = int64_t(host.cnt[3]);
    out->n_dH_positive = int64_t(host.cnt[4]);
    for (int b = 0; b < 4; ++b) out->n_xmax_band[b] = int64_t(host.cnt[5 + b]);
    if (alpha_hist)
        for (int b = 0; b < ELBM_HIST_BINS + 2; ++b) alpha_hist[b] = int64_t(host.hist[b]);
    if (out->n_nonpositive > 0)
        return noalloc_fail(ELBM_ERR_NONPHYSICAL,
                            "elbm_diagnostics_noalloc: %lld nodes with a population <= 0 or not finite",
                            (long long)out->n_nonpositive);
    return ELBM_OK;
}
