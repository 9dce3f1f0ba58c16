// elbm_api.cu -- the C ABI declared in include/elbm.h: argument validation,
// buffer ownership, stream handling and kernel dispatch.  All arithmetic of the
// step lives in the kernels (elbm_kernels.cuh); this file only marshals.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "elbm.h"
#include "elbm_device.cuh"
#include "elbm_launch.h"

using eelbm::CollideParams;
using eelbm::DiagAcc;
using eelbm::Geometry;

struct elbm {
    int lattice = 0, D = 0, Q = 0;
    Geometry g{};
    double beta = 0.0;
    elbm_opts opts{};
    cudaStream_t stream = nullptr;
    void *pop[2] = {nullptr, nullptr};
    bool owned = false; // library allocated pop[]
    size_t pop_bytes = 0;
    int cur = 0; // buffer holding the current state
    double *stage = nullptr;
    size_t stage_bytes = 0;
    // host transfers of FP64 fields: a copy stream and events, so that the copies of one
    // node range overlap the kernel of another (created with the staging buffer)
    cudaStream_t copy = nullptr;
    cudaEvent_t ev[1 + 8] = {};
    DiagAcc *acc = nullptr;
    int *err_word = nullptr; // device: ELBM_ERR_TIMEOUT when a bounded device wait expired
    int num_sms = 0;
    int64_t steps = 0;
    double force[3] = {0.0, 0.0, 0.0}; // uniform body force (elbm_set_force)
    // load policy of the D3Q27 step (ld_pop): evict-first once the last diagnostics saw
    // more than half of the nodes at |x|max >= 0.005 (the x^6 and per-population forms)
    bool pop_stream = false;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

int fail(elbm_t *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_create_error = buf;
    return code;
}

int cuda_fail(elbm_t *h, cudaError_t e, const char *what)
{
    return fail(h, ELBM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

size_t storage_size(int storage)
{
    switch (storage) {
    case ELBM_STORE_F64: return 8;
    case ELBM_STORE_F32:
    case ELBM_STORE_F32DEV: return 4;
    case ELBM_STORE_F16DEV:
    case ELBM_STORE_BF16DEV: return 2;
    default: return 0;
    }
}

CollideParams params_of(const elbm_t *h)
{
    CollideParams p;
    p.beta = h->beta;
    p.mode = h->opts.alpha_mode;
    p.cutoff = h->opts.cutoff;
    p.b_variant = h->opts.b_variant;
    p.rho0 = h->opts.rho0;
    p.beta_f = float(p.beta);
    p.dunit_f = h->D == 2 ? eelbm::dev_unit<2>(p.rho0) : eelbm::dev_unit<3>(p.rho0);
    for (int a = 0; a < 3; ++a) p.force[a] = h->force[a];
    p.pop_stream = h->pop_stream ? 1 : 0;
    return p;
}

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    cudaError_t status = cudaSuccess;
    explicit DeviceGuard(int dev)
    {
        status = cudaGetDevice(&prev);
        if (status == cudaSuccess && prev != dev) status = cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

int ensure_populations(elbm_t *h)
{
    if (h->pop[0]) return ELBM_OK;
    void *a = nullptr, *b = nullptr;
    cudaError_t e = cudaMalloc(&a, h->pop_bytes);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(populations)");
    e = cudaMalloc(&b, h->pop_bytes);
    if (e != cudaSuccess) {
        cudaFree(a);
        return cuda_fail(h, e, "cudaMalloc(populations)");
    }
    h->pop[0] = a;
    h->pop[1] = b;
    h->owned = true;
    h->cur = 0;
    return ELBM_OK;
}

// The host transfers of elbm_init_equilibrium and elbm_moments are cut into
// kStageChunks node ranges (of at least 2^20 nodes), pipelined on two streams.
constexpr int kStageChunks = 8;
int stage_chunks(int64_t N) { return N >= (int64_t(kStageChunks) << 20) ? kStageChunks : 1; }

int ensure_stage(elbm_t *h, size_t bytes)
{
    if (!h->copy) {
        cudaError_t e = cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking);
        for (int k = 0; k < 1 + kStageChunks && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&h->ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreate/cudaEventCreate(staging)");
    }
    if (h->stage_bytes >= bytes) return ELBM_OK;
    if (h->stage) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
        cudaFree(h->stage);
        h->stage = nullptr;
        h->stage_bytes = 0;
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&h->stage), bytes);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc(staging)");
    h->stage_bytes = bytes;
    return ELBM_OK;
}

// Reads (and clears) the device error word after the stream has been
// synchronised; returns ELBM_ERR_TIMEOUT when a bounded device wait expired.
int check_device_flag(elbm_t *h, const char *what)
{
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, h->err_word, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    if (flag != 0) {
        cudaMemset(h->err_word, 0, sizeof(int));
        return fail(h, ELBM_ERR_TIMEOUT, "%s: a bounded device-side wait expired (the step was not completed)", what);
    }
    return ELBM_OK;
}

#define ELBM_BY_LATTICE(h, FN, ...)                                                               \
    ((h)->D == 2 ? eelbm::FN##_d2q9(__VA_ARGS__) : eelbm::FN##_d3q27(__VA_ARGS__))

} // namespace

void eelbm::set_handle_free_error(const char *msg) { g_create_error = msg; }

extern "C" {

void elbm_default_opts(elbm_opts *o)
{
    if (!o) return;
    o->storage = ELBM_STORE_F32;
    o->alpha_mode = ELBM_ALPHA_HIGHER;
    o->cutoff = 1;
    o->b_variant = ELBM_B_DERIVED;
    o->device = 0;
    o->rho0 = 1.0;
    o->stream = nullptr;
    o->kernel = ELBM_KERNEL_AUTO;
}

int elbm_population_bytes(int lattice, const int64_t dims[3], int storage, size_t *bytes)
{
    if (!dims || !bytes) return fail(nullptr, ELBM_ERR_ARG, "elbm_population_bytes: null argument");
    if (lattice != ELBM_D2Q9 && lattice != ELBM_D3Q27)
        return fail(nullptr, ELBM_ERR_ARG, "elbm_population_bytes: lattice must be 9 or 27");
    const size_t es = storage_size(storage);
    if (!es) return fail(nullptr, ELBM_ERR_ARG, "elbm_population_bytes: unknown storage %d", storage);
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (int64_t(1) << 30))
            return fail(nullptr, ELBM_ERR_ARG, "elbm_population_bytes: dims[%d] = %lld out of range", a,
                        (long long)dims[a]);
    const unsigned __int128 n = (unsigned __int128)dims[0] * dims[1] * dims[2] * lattice * es;
    if (n > (unsigned __int128)SIZE_MAX / 4)
        return fail(nullptr, ELBM_ERR_ARG, "elbm_population_bytes: domain too large");
    *bytes = size_t(n);
    return ELBM_OK;
}

int elbm_create(elbm_t **out, int lattice, const int64_t dims[3], double beta, int bc,
                const elbm_opts *opts)
{
    if (!out) return fail(nullptr, ELBM_ERR_ARG, "elbm_create: out is NULL");
    *out = nullptr;
    if (!dims) return fail(nullptr, ELBM_ERR_ARG, "elbm_create: dims is NULL");
    if (lattice != ELBM_D2Q9 && lattice != ELBM_D3Q27)
        return fail(nullptr, ELBM_ERR_ARG, "elbm_create: lattice must be ELBM_D2Q9 (9) or ELBM_D3Q27 (27), got %d",
                    lattice);
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (int64_t(1) << 30))
            return fail(nullptr, ELBM_ERR_ARG, "elbm_create: dims[%d] = %lld out of range", a, (long long)dims[a]);
    if (lattice == ELBM_D2Q9 && dims[2] != 1)
        return fail(nullptr, ELBM_ERR_ARG, "elbm_create: D2Q9 needs dims[2] == 1");
    if (!(beta > 0.0 && beta < 1.0))
        return fail(nullptr, ELBM_ERR_ARG, "elbm_create: beta must lie in (0, 1), got %g", beta);
    if (bc != ELBM_BC_PERIODIC)
        return fail(nullptr, ELBM_ERR_UNSUPPORTED, "elbm_create: only periodic boundaries are supported");
    elbm_opts o;
    elbm_default_opts(&o);
    if (opts) o = *opts;
    if (!storage_size(o.storage)) return fail(nullptr, ELBM_ERR_ARG, "elbm_create: unknown storage %d", o.storage);
    if (o.alpha_mode < ELBM_ALPHA_HIGHER || o.alpha_mode > ELBM_ALPHA_ITERATE1)
        return fail(nullptr, ELBM_ERR_ARG, "elbm_create: unknown alpha_mode %d", o.alpha_mode);
    if (o.b_variant != ELBM_B_DERIVED && o.b_variant != ELBM_B_PRINTED)
        return fail(nullptr, ELBM_ERR_ARG, "elbm_create: unknown b_variant %d", o.b_variant);
    if (o.cutoff != 0 && o.cutoff != 1) return fail(nullptr, ELBM_ERR_ARG, "elbm_create: cutoff must be 0 or 1");
    if (!(o.rho0 > 0.0)) return fail(nullptr, ELBM_ERR_ARG, "elbm_create: rho0 must be positive");
    if (o.kernel < ELBM_KERNEL_AUTO || o.kernel > ELBM_KERNEL_ROWS)
        return fail(nullptr, ELBM_ERR_ARG, "elbm_create: unknown kernel %d", o.kernel);
    size_t bytes = 0;
    int st = elbm_population_bytes(lattice, dims, o.storage, &bytes);
    if (st != ELBM_OK) return st;
    if (dims[0] * dims[1] * dims[2] > (int64_t(1) << 31))
        return fail(nullptr, ELBM_ERR_ARG, "elbm_create: more than 2^31 nodes");

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "elbm_create: cudaGetDeviceCount");
    if (o.device < 0 || o.device >= ndev)
        return fail(nullptr, ELBM_ERR_ARG, "elbm_create: device %d not present (%d devices)", o.device, ndev);
    DeviceGuard guard(o.device);
    if (guard.status != cudaSuccess) return cuda_fail(nullptr, guard.status, "elbm_create: cudaSetDevice");

    elbm_t *h = new (std::nothrow) elbm_t();
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_create: out of host memory");
    h->lattice = lattice;
    h->D = lattice == ELBM_D2Q9 ? 2 : 3;
    h->Q = lattice;
    h->g.nx = int(dims[0]);
    h->g.ny = int(dims[1]);
    h->g.nz = int(dims[2]);
    h->g.N = dims[0] * dims[1] * dims[2];
    h->beta = beta;
    h->opts = o;
    h->stream = static_cast<cudaStream_t>(o.stream);
    h->pop_bytes = bytes;
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, o.device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(nullptr, e, "elbm_create: cudaDeviceGetAttribute");
    }
    e = cudaMalloc(reinterpret_cast<void **>(&h->acc), sizeof(DiagAcc));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&h->err_word), sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->err_word, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(h->acc);
        cudaFree(h->err_word);
        delete h;
        return cuda_fail(nullptr, e, "elbm_create: cudaMalloc(scratch)");
    }
    if (o.kernel == ELBM_KERNEL_ROWS) {
        const bool ok = lattice == ELBM_D2Q9 ? eelbm::rows_kernel_applies_d2q9(o.storage, h->g)
                                             : eelbm::rows_kernel_applies_d3q27(o.storage, h->g);
        if (!ok) {
            cudaFree(h->acc);
            cudaFree(h->err_word);
            delete h;
            return fail(nullptr, ELBM_ERR_UNSUPPORTED,
                        "elbm_create: the ROWS kernel needs FP32/16-bit storage, nx * element size a multiple "
                        "of 16 bytes and nx <= %d",
                        lattice == ELBM_D2Q9 ? 1024 : 512);
        }
    }
    *out = h;
    return ELBM_OK;
}

void elbm_destroy(elbm_t *h)
{
    if (!h) return;
    DeviceGuard guard(h->opts.device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    if (h->owned) {
        cudaFree(h->pop[0]);
        cudaFree(h->pop[1]);
    }
    cudaFree(h->stage);
    cudaFree(h->acc);
    cudaFree(h->err_word);
    for (cudaEvent_t ev : h->ev)
        if (ev) cudaEventDestroy(ev);
    if (h->copy) cudaStreamDestroy(h->copy);
    delete h;
}

const char *elbm_last_error(const elbm_t *h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

int elbm_bind_buffers(elbm_t *h, void *pop_a, void *pop_b, size_t bytes)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_bind_buffers: handle is NULL");
    if (!pop_a || !pop_b) return fail(h, ELBM_ERR_ARG, "elbm_bind_buffers: buffer is NULL");
    if (pop_a == pop_b) return fail(h, ELBM_ERR_ARG, "elbm_bind_buffers: the two buffers alias");
    if (bytes < h->pop_bytes)
        return fail(h, ELBM_ERR_ARG, "elbm_bind_buffers: %zu bytes given, %zu needed", bytes, h->pop_bytes);
    if ((reinterpret_cast<uintptr_t>(pop_a) | reinterpret_cast<uintptr_t>(pop_b)) & 255u)
        return fail(h, ELBM_ERR_ARG, "elbm_bind_buffers: buffers must be 256-byte aligned");
    const char *a = static_cast<const char *>(pop_a), *b = static_cast<const char *>(pop_b);
    if (a < b + h->pop_bytes && b < a + h->pop_bytes)
        return fail(h, ELBM_ERR_ARG, "elbm_bind_buffers: the two buffers overlap");
    DeviceGuard guard(h->opts.device);
    if (h->owned) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "elbm_bind_buffers: cudaStreamSynchronize");
        cudaFree(h->pop[0]);
        cudaFree(h->pop[1]);
    }
    h->pop[0] = pop_a;
    h->pop[1] = pop_b;
    h->owned = false;
    h->cur = 0;
    h->steps = 0;
    h->pop_stream = false; // a new state: the load policy waits for its diagnostics
    return ELBM_OK;
}

int elbm_set_stream(elbm_t *h, void *stream)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_set_stream: handle is NULL");
    h->stream = static_cast<cudaStream_t>(stream);
    h->opts.stream = stream;
    return ELBM_OK;
}

int elbm_init_equilibrium(elbm_t *h, const double *rho, const double *u, int where)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_init_equilibrium: handle is NULL");
    if (!u) return fail(h, ELBM_ERR_ARG, "elbm_init_equilibrium: u is NULL");
    if (where != ELBM_MEM_DEVICE && where != ELBM_MEM_HOST)
        return fail(h, ELBM_ERR_ARG, "elbm_init_equilibrium: bad memory location %d", where);
    DeviceGuard guard(h->opts.device);
    int st = ensure_populations(h);
    if (st != ELBM_OK) return st;
    const int64_t N = h->g.N;
    cudaError_t e;
    if (where == ELBM_MEM_HOST) {
        const size_t need = size_t(N) * (1 + h->D) * sizeof(double);
        if ((st = ensure_stage(h, need)) != ELBM_OK) return st;
        double *srho = rho ? h->stage : nullptr, *su = h->stage + N;
        // the copies start after the work already queued on the handle's stream; the
        // kernel of each node range waits for that range's copies
        e = cudaEventRecord(h->ev[0], h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy, h->ev[0], 0);
        const int C = stage_chunks(N);
        for (int c = 0; c < C && e == cudaSuccess; ++c) {
            const int64_t n0 = N * c / C, cnt = N * (c + 1) / C - n0;
            if (rho) e = cudaMemcpyAsync(srho + n0, rho + n0, size_t(cnt) * sizeof(double), cudaMemcpyHostToDevice,
                                         h->copy);
            for (int a = 0; a < h->D && e == cudaSuccess; ++a)
                e = cudaMemcpyAsync(su + a * N + n0, u + a * N + n0, size_t(cnt) * sizeof(double),
                                    cudaMemcpyHostToDevice, h->copy);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev[1 + c], h->copy);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev[1 + c], 0);
            if (e == cudaSuccess)
                e = ELBM_BY_LATTICE(h, launch_init, h->opts.storage, srho, su, h->pop[0], h->g, h->opts.rho0,
                                    h->opts.rho0, n0, cnt, h->stream);
        }
        // the caller may reuse its host arrays as soon as we return
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "elbm_init_equilibrium: copy, kernel or synchronize");
    } else {
        e = ELBM_BY_LATTICE(h, launch_init, h->opts.storage, rho, u, h->pop[0], h->g, h->opts.rho0, h->opts.rho0,
                            0, N, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "elbm_init_equilibrium: kernel launch");
    }
    h->cur = 0;
    h->steps = 0;
    h->pop_stream = false; // a new state: the load policy waits for its diagnostics
    return ELBM_OK;
}

int elbm_step(elbm_t *h, int64_t n)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_step: handle is NULL");
    if (n < 0) return fail(h, ELBM_ERR_ARG, "elbm_step: n = %lld < 0", (long long)n);
    if (!h->pop[0]) return fail(h, ELBM_ERR_ARG, "elbm_step: no state (call elbm_init_equilibrium first)");
    DeviceGuard guard(h->opts.device);
    const CollideParams p = params_of(h);
    for (int64_t k = 0; k < n; ++k) {
        cudaError_t e = ELBM_BY_LATTICE(h, launch_step, h->opts.storage, h->pop[h->cur], h->pop[h->cur ^ 1], h->g, p,
                                        h->opts.kernel, h->num_sms, h->err_word, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "elbm_step: kernel launch");
        h->cur ^= 1;
        h->steps += 1;
    }
    return ELBM_OK;
}

int elbm_moments(elbm_t *h, double *rho_out, double *u_out, int where)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_moments: handle is NULL");
    if (where != ELBM_MEM_DEVICE && where != ELBM_MEM_HOST)
        return fail(h, ELBM_ERR_ARG, "elbm_moments: bad memory location %d", where);
    if (!h->pop[0]) return fail(h, ELBM_ERR_ARG, "elbm_moments: no state");
    if (!rho_out && !u_out) return ELBM_OK;
    DeviceGuard guard(h->opts.device);
    const int64_t N = h->g.N;
    int st;
    if (where == ELBM_MEM_HOST) {
        if ((st = ensure_stage(h, size_t(N) * (1 + h->D) * sizeof(double))) != ELBM_OK) return st;
        double *drho = rho_out ? h->stage : nullptr, *du = u_out ? h->stage + N : nullptr;
        // the copies of each node range wait for that range's kernel
        const int C = stage_chunks(N);
        cudaError_t e = cudaSuccess;
        for (int c = 0; c < C && e == cudaSuccess; ++c) {
            const int64_t n0 = N * c / C, cnt = N * (c + 1) / C - n0;
            e = ELBM_BY_LATTICE(h, launch_moments, h->opts.storage, h->pop[h->cur], h->g, h->opts.rho0, drho, du,
                                n0, cnt, h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev[1 + c], h->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy, h->ev[1 + c], 0);
            if (rho_out && e == cudaSuccess)
                e = cudaMemcpyAsync(rho_out + n0, drho + n0, size_t(cnt) * sizeof(double), cudaMemcpyDeviceToHost,
                                    h->copy);
            for (int a = 0; u_out && a < h->D && e == cudaSuccess; ++a)
                e = cudaMemcpyAsync(u_out + a * N + n0, du + a * N + n0, size_t(cnt) * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->copy);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->copy);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "elbm_moments: kernel, copy or synchronize");
        return check_device_flag(h, "elbm_moments");
    }
    cudaError_t e = ELBM_BY_LATTICE(h, launch_moments, h->opts.storage, h->pop[h->cur], h->g, h->opts.rho0, rho_out,
                                    u_out, 0, N, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_moments: kernel launch");
    return ELBM_OK;
}

int elbm_alpha_field(elbm_t *h, double *alpha_out, uint8_t *flags_out, int where)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_alpha_field: handle is NULL");
    if (!alpha_out) return fail(h, ELBM_ERR_ARG, "elbm_alpha_field: alpha_out is NULL");
    if (where != ELBM_MEM_DEVICE && where != ELBM_MEM_HOST)
        return fail(h, ELBM_ERR_ARG, "elbm_alpha_field: bad memory location %d", where);
    if (!h->pop[0]) return fail(h, ELBM_ERR_ARG, "elbm_alpha_field: no state");
    DeviceGuard guard(h->opts.device);
    const int64_t N = h->g.N;
    double *da = alpha_out;
    uint8_t *df = flags_out;
    int st;
    if (where == ELBM_MEM_HOST) {
        if ((st = ensure_stage(h, size_t(N) * (sizeof(double) + 1) + 256)) != ELBM_OK) return st;
        da = h->stage;
        df = flags_out ? reinterpret_cast<uint8_t *>(h->stage + N) : nullptr;
    }
    cudaError_t e = ELBM_BY_LATTICE(h, launch_alpha, h->opts.storage, h->pop[h->cur], h->g, params_of(h), da, df,
                                    nullptr, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_alpha_field: kernel launch");
    if (where == ELBM_MEM_HOST) {
        e = cudaMemcpyAsync(alpha_out, da, size_t(N) * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "elbm_alpha_field: copy alpha");
        if (flags_out) {
            e = cudaMemcpyAsync(flags_out, df, size_t(N), cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "elbm_alpha_field: copy flags");
        }
        e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "elbm_alpha_field: synchronize");
    }
    return ELBM_OK;
}

int elbm_subgrid_viscosity(elbm_t *h, double *nut_out, int where)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_subgrid_viscosity: handle is NULL");
    if (!nut_out) return fail(h, ELBM_ERR_ARG, "elbm_subgrid_viscosity: nut_out is NULL");
    if (where != ELBM_MEM_DEVICE && where != ELBM_MEM_HOST)
        return fail(h, ELBM_ERR_ARG, "elbm_subgrid_viscosity: bad memory location %d", where);
    if (!h->pop[0]) return fail(h, ELBM_ERR_ARG, "elbm_subgrid_viscosity: no state");
    DeviceGuard guard(h->opts.device);
    const int64_t N = h->g.N;
    double *dn = nut_out;
    int st;
    if (where == ELBM_MEM_HOST) {
        if ((st = ensure_stage(h, size_t(N) * sizeof(double))) != ELBM_OK) return st;
        dn = h->stage;
    }
    cudaError_t e = ELBM_BY_LATTICE(h, launch_alpha, h->opts.storage, h->pop[h->cur], h->g, params_of(h), nullptr,
                                    nullptr, dn, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_subgrid_viscosity: kernel launch");
    if (where == ELBM_MEM_HOST) {
        e = cudaMemcpyAsync(nut_out, dn, size_t(N) * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "elbm_subgrid_viscosity: read back");
    }
    return ELBM_OK;
}

namespace {

// Clears the handle's diagnostics accumulator (on its stream).
cudaError_t clear_diag_acc(elbm_t *h)
{
    cudaError_t e = cudaMemsetAsync(h->acc, 0, sizeof(DiagAcc), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&h->acc->amin_ord, 0xFF, sizeof(unsigned long long), h->stream);
    return e;
}

// Reads the accumulator back (synchronising the stream) and fills *out / alpha_hist.
int read_diag_acc(elbm_t *h, elbm_diag *out, int64_t *alpha_hist, const char *what)
{
    DiagAcc acc;
    cudaError_t e = cudaMemcpyAsync(&acc, h->acc, sizeof acc, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    int st = check_device_flag(h, what);
    if (st != ELBM_OK) return st;
    const int64_t N = h->g.N;
    out->mass = acc.sum[0];
    out->momentum[0] = acc.sum[1];
    out->momentum[1] = acc.sum[2];
    out->momentum[2] = h->D == 3 ? acc.sum[3] : 0.0;
    out->H = acc.sum[4];
    out->dH_max = eelbm::from_ordered_bits(acc.dH_max_ord);
    out->alpha_min = eelbm::from_ordered_bits(acc.amin_ord);
    out->alpha_max = eelbm::from_ordered_bits(acc.amax_ord);
    out->alpha_mean = N ? acc.sum[5] / double(N) : 0.0;
    out->n_nodes = N;
    out->n_cutoff = int64_t(acc.cnt[0]);
    out->n_solved = int64_t(acc.cnt[1]);
    out->n_clamped = int64_t(acc.cnt[2]);
    out->n_nonpositive = int64_t(acc.cnt[3]);
    out->n_dH_positive = int64_t(acc.cnt[4]);
    for (int b = 0; b < 4; ++b) out->n_xmax_band[b] = int64_t(acc.cnt[5 + b]);
    h->pop_stream = 2 * (acc.cnt[7] + acc.cnt[8]) > uint64_t(N);
    if (alpha_hist)
        for (int b = 0; b < ELBM_HIST_BINS + 2; ++b) alpha_hist[b] = int64_t(acc.hist[b]);
    if (out->n_nonpositive > 0)
        return fail(h, ELBM_ERR_NONPHYSICAL, "%s: %lld nodes with a population <= 0 or not finite", what,
                    (long long)out->n_nonpositive);
    return ELBM_OK;
}

} // namespace

int elbm_diagnostics(elbm_t *h, elbm_diag *out, int64_t *alpha_hist)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_diagnostics: handle is NULL");
    if (!out) return fail(h, ELBM_ERR_ARG, "elbm_diagnostics: out is NULL");
    if (!h->pop[0]) return fail(h, ELBM_ERR_ARG, "elbm_diagnostics: no state");
    DeviceGuard guard(h->opts.device);
    cudaError_t e = clear_diag_acc(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_diagnostics: clear scratch");
    e = ELBM_BY_LATTICE(h, launch_diag, h->opts.storage, h->pop[h->cur], h->g, params_of(h), h->acc, h->num_sms,
                        h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_diagnostics: kernel launch");
    return read_diag_acc(h, out, alpha_hist, "elbm_diagnostics");
}

int elbm_step_diag(elbm_t *h, int64_t n, elbm_diag *out, int64_t *alpha_hist)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_step_diag: handle is NULL");
    if (!out) return fail(h, ELBM_ERR_ARG, "elbm_step_diag: out is NULL");
    if (n < 1) return fail(h, ELBM_ERR_ARG, "elbm_step_diag: n = %lld < 1", (long long)n);
    if (!h->pop[0]) return fail(h, ELBM_ERR_ARG, "elbm_step_diag: no state");
    DeviceGuard guard(h->opts.device);
    cudaError_t e = clear_diag_acc(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_step_diag: clear scratch");
    const CollideParams p = params_of(h);
    int64_t done = 0;
    if (h->opts.kernel != ELBM_KERNEL_ROWS) {
        e = ELBM_BY_LATTICE(h, launch_step_diag, h->opts.storage, h->pop[h->cur], h->pop[h->cur ^ 1], h->g, p,
                            h->acc, h->num_sms, h->stream);
        if (e == cudaSuccess) {
            h->cur ^= 1;
            ++h->steps;
            done = 1;
        } else if (e != cudaErrorNotSupported) {
            return cuda_fail(h, e, "elbm_step_diag: kernel launch");
        }
    }
    if (!done) { // diagnostics pass, then the step (rows kernel, body force, very large domains)
        e = ELBM_BY_LATTICE(h, launch_diag, h->opts.storage, h->pop[h->cur], h->g, p, h->acc, h->num_sms,
                            h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "elbm_step_diag: kernel launch");
    }
    const int st = elbm_step(h, n - done);
    if (st != ELBM_OK) return st;
    return read_diag_acc(h, out, alpha_hist, "elbm_step_diag");
}

int elbm_get_populations(elbm_t *h, void *dst, int where)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_get_populations: handle is NULL");
    if (!dst) return fail(h, ELBM_ERR_ARG, "elbm_get_populations: dst is NULL");
    if (where != ELBM_MEM_DEVICE && where != ELBM_MEM_HOST)
        return fail(h, ELBM_ERR_ARG, "elbm_get_populations: bad memory location %d", where);
    if (!h->pop[0]) return fail(h, ELBM_ERR_ARG, "elbm_get_populations: no state");
    DeviceGuard guard(h->opts.device);
    cudaError_t e = cudaMemcpyAsync(dst, h->pop[h->cur], h->pop_bytes,
                                    where == ELBM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e == cudaSuccess && where == ELBM_MEM_HOST) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_get_populations");
    if (where == ELBM_MEM_HOST) return check_device_flag(h, "elbm_get_populations");
    return ELBM_OK;
}

int elbm_set_populations(elbm_t *h, const void *src, int where)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_set_populations: handle is NULL");
    if (!src) return fail(h, ELBM_ERR_ARG, "elbm_set_populations: src is NULL");
    if (where != ELBM_MEM_DEVICE && where != ELBM_MEM_HOST)
        return fail(h, ELBM_ERR_ARG, "elbm_set_populations: bad memory location %d", where);
    DeviceGuard guard(h->opts.device);
    int st = ensure_populations(h);
    if (st != ELBM_OK) return st;
    cudaError_t e = cudaMemcpyAsync(h->pop[0], src, h->pop_bytes,
                                    where == ELBM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e == cudaSuccess && where == ELBM_MEM_HOST) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_set_populations");
    h->cur = 0;
    h->steps = 0;
    h->pop_stream = false; // a new state: the load policy waits for its diagnostics
    return ELBM_OK;
}

int elbm_adjoint_step(elbm_t *h, const void *f_t, const void *g_next, void *g_t)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_adjoint_step: handle is NULL");
    if (!f_t || !g_next || !g_t) return fail(h, ELBM_ERR_ARG, "elbm_adjoint_step: null pointer");
    if (g_next == g_t) return fail(h, ELBM_ERR_ARG, "elbm_adjoint_step: g_t must not alias g_next");
    DeviceGuard guard(h->opts.device);
    cudaError_t e = ELBM_BY_LATTICE(h, launch_step_adjoint, h->opts.storage, f_t, g_next, g_t, h->g, params_of(h),
                                    nullptr, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_adjoint_step: kernel launch");
    return ELBM_OK;
}

int elbm_adjoint_step_force(elbm_t *h, const void *f_t, const void *g_next, void *g_t, double *dforce)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_adjoint_step_force: handle is NULL");
    if (!f_t || !g_next || !g_t || !dforce) return fail(h, ELBM_ERR_ARG, "elbm_adjoint_step_force: null pointer");
    if (g_next == g_t) return fail(h, ELBM_ERR_ARG, "elbm_adjoint_step_force: g_t must not alias g_next");
    DeviceGuard guard(h->opts.device);
    cudaError_t e = ELBM_BY_LATTICE(h, launch_step_adjoint, h->opts.storage, f_t, g_next, g_t, h->g, params_of(h),
                                    dforce, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_adjoint_step_force: kernel launch");
    return ELBM_OK;
}

int elbm_set_force(elbm_t *h, const double *force)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_set_force: handle is NULL");
    double F[3] = {0.0, 0.0, 0.0};
    if (force)
        for (int a = 0; a < h->D; ++a) {
            if (!std::isfinite(force[a])) return fail(h, ELBM_ERR_ARG, "elbm_set_force: component %d is not finite", a);
            F[a] = force[a];
        }
    if (h->opts.kernel == ELBM_KERNEL_ROWS && (F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0))
        return fail(h, ELBM_ERR_UNSUPPORTED, "elbm_set_force: the body force runs on the DIRECT kernel only");
    for (int a = 0; a < 3; ++a) h->force[a] = F[a];
    return ELBM_OK;
}

int elbm_kinetic_energy(elbm_t *h, const void *f, double *L, void *grad)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_kinetic_energy: handle is NULL");
    if (!L) return fail(h, ELBM_ERR_ARG, "elbm_kinetic_energy: L is NULL");
    if (!f && !h->pop[0]) return fail(h, ELBM_ERR_ARG, "elbm_kinetic_energy: no state");
    DeviceGuard guard(h->opts.device);
    const void *src = f ? f : h->pop[h->cur];
    double *acc = &h->acc->sum[0];
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double), h->stream);
    if (e == cudaSuccess)
        e = ELBM_BY_LATTICE(h, launch_kinetic_energy, h->opts.storage, src, h->g, h->opts.rho0, acc, grad, h->num_sms,
                            h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L, acc, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_kinetic_energy");
    return ELBM_OK;
}

int elbm_equilibrium_vjp(elbm_t *h, const double *rho, const double *u, const void *g, double *drho, double *du)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_equilibrium_vjp: handle is NULL");
    if (!u || !g) return fail(h, ELBM_ERR_ARG, "elbm_equilibrium_vjp: u or g is NULL");
    DeviceGuard guard(h->opts.device);
    cudaError_t e = ELBM_BY_LATTICE(h, launch_equilibrium_vjp, h->opts.storage, rho, u, g, h->g, h->opts.rho0, drho,
                                    du, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_equilibrium_vjp: kernel launch");
    return ELBM_OK;
}

int elbm_step_count(const elbm_t *h, int64_t *steps)
{
    if (!h || !steps) return fail(nullptr, ELBM_ERR_ARG, "elbm_step_count: null argument");
    *steps = h->steps;
    return ELBM_OK;
}

int elbm_synchronize(elbm_t *h)
{
    if (!h) return fail(nullptr, ELBM_ERR_ARG, "elbm_synchronize: handle is NULL");
    DeviceGuard guard(h->opts.device);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "elbm_synchronize");
    return check_device_flag(h, "elbm_synchronize");
}

} // extern "C"
