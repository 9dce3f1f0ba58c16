// elbm_batch.cu -- C ABI of batched ensembles (include/elbm.h, "Batched
// ensembles"): many independent periodic domains of one lattice, each with its
// own size and beta, advanced together.
//
// Layout: every domain's populations are one SoA block [Q][N_d] inside a shared
// pair of buffers, at an element offset rounded up to 256 bytes, so all
// single-domain kernels (init, moments, diagnostics) run on a domain's block
// unchanged.  A step is one launch of k_step_batch per run of up to 64 domains,
// whose sides, offsets, betas and work-item counts travel in the launch's
// parameter table (one block per x-row chunk); elbm_batch_step can also replay the n launches
// as one CUDA graph, advance all n steps in one cooperative launch of
// k_step_persist (blocks own fixed runs of work items and wait, with bounded
// spins, only for the other owners of their domains), or launch the
// single-domain kernel once per domain (the comparison the batched forms are
// measured against).  elbm_batch_tune times the candidate block widths on the
// current state without changing it; elbm_batch_tune_persistent times the
// persistent launch against the batched launches on a copy of the state and
// sets which one ELBM_BATCH_AUTO issues.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "elbm.h"
#include "elbm_device.cuh"
#include "elbm_launch.h"

using eelbm::BatchDomain;
using eelbm::CollideParams;
using eelbm::DiagAcc;
using eelbm::Geometry;

struct elbm_batch {
    int lattice = 0, D = 0, Q = 0;
    elbm_opts opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<BatchDomain> doms;
    size_t elem = 0;          // bytes per stored element
    size_t total_elems = 0;   // elements per buffer
    void *pop[2] = {nullptr, nullptr};
    int cur = 0;
    int bx = 128;                          // work-item width (autotuned)
    std::map<int, std::vector<eelbm::BatchTable>> tables; // per width: the launches of one batched step
    double *stage = nullptr;
    size_t stage_bytes = 0;
    DiagAcc *acc = nullptr;
    int num_sms = 0;
    int64_t steps = 0;
    std::map<std::pair<int64_t, int>, cudaGraphExec_t> graphs; // (n, starting buffer) -> graph
    struct Persist {                                            // persistent launch plan per width
        eelbm::PersistPlan plan;
        int4 *chunks = nullptr;
        unsigned *owners = nullptr;
        unsigned *cnt = nullptr; // one counter per domain, then the ticket counter
        eelbm::BatchTableDom *doms = nullptr; // every domain's entry at this width (device)
        std::vector<unsigned> h_owners; // host copy
        int max_steps = 1;              // steps per launch that keep steps x chunks below 2^32
    };
    std::map<int, Persist> persist;
    int *err_word = nullptr; // device: ELBM_ERR_TIMEOUT when a bounded device wait expired
    int pbx = 64;                             // work-item width of the persistent mode (tuned)
    int auto_mode = ELBM_BATCH_GRAPH;         // what ELBM_BATCH_AUTO issues (tuned)
    double graph_ms = 0.0;                    // per-step time of the width trials (0: not run)
    std::string err;
};

namespace {

thread_local std::string g_batch_create_error;

int bfail(elbm_batch_t *b, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_batch_create_error = buf;
    return code;
}

int bcuda(elbm_batch_t *b, cudaError_t e, const char *what)
{
    return bfail(b, ELBM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

size_t elem_size(int storage)
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

CollideParams params_of(const elbm_batch_t *b, double beta)
{
    CollideParams p;
    p.beta = beta;
    p.mode = b->opts.alpha_mode;
    p.cutoff = b->opts.cutoff;
    p.b_variant = b->opts.b_variant;
    p.rho0 = b->opts.rho0;
    p.beta_f = float(p.beta);
    p.dunit_f = b->D == 2 ? eelbm::dev_unit<2>(p.rho0) : eelbm::dev_unit<3>(p.rho0);
    return p;
}

Geometry geom_of(const BatchDomain &d)
{
    Geometry g;
    g.nx = d.nx;
    g.ny = d.ny;
    g.nz = d.nz;
    g.N = d.N;
    return g;
}

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

int check_domain(elbm_batch_t *b, int d, const char *what)
{
    if (!b) return bfail(nullptr, ELBM_ERR_ARG, "%s: batch is NULL", what);
    if (d < 0 || d >= int(b->doms.size()))
        return bfail(b, ELBM_ERR_ARG, "%s: domain %d out of range [0, %d)", what, d, int(b->doms.size()));
    return ELBM_OK;
}

// Parameter tables of the batched launches of width bx: consecutive runs of up to
// kBatchTableDomains domains, one launch each.
int build_tables(elbm_batch_t *b, int bx)
{
    if (b->tables.count(bx)) return ELBM_OK;
    std::vector<eelbm::BatchTable> tabs;
    const int nd = int(b->doms.size());
    for (int d0 = 0; d0 < nd; d0 += eelbm::kBatchTableDomains) {
        eelbm::BatchTable t;
        memset(&t, 0, sizeof t);
        t.n = std::min(nd - d0, eelbm::kBatchTableDomains);
        int64_t items = 0;
        for (int k = 0; k < t.n; ++k) {
            const BatchDomain &dm = b->doms[size_t(d0 + k)];
            eelbm::BatchTableDom &td = t.dom[k];
            td.nx = dm.nx;
            td.ny = dm.ny;
            td.nz = dm.nz;
            td.xblocks = (dm.nx + bx - 1) / bx;
            td.off = dm.off;
            td.beta = dm.beta;
            td.beta_f = dm.beta_f;
            t.item0[k] = int(items);
            items += int64_t(td.xblocks) * dm.ny * dm.nz;
            if (items > int64_t(0x7fffffff))
                return bfail(b, ELBM_ERR_ARG, "elbm_batch: too many work items in one launch");
        }
        t.item0[t.n] = int(items);
        t.shift = 0;
        while (((items - 1) >> t.shift) >= eelbm::kBatchCoarse) ++t.shift;
        for (int c = 0, d = 0; c < eelbm::kBatchCoarse; ++c) {
            const int64_t b0 = int64_t(c) << t.shift;
            while (d + 1 < t.n && t.item0[d + 1] <= b0) ++d;
            t.coarse[c] = (unsigned char)d;
        }
        tabs.push_back(t);
    }
    b->tables[bx] = std::move(tabs);
    return ELBM_OK;
}

cudaError_t launch_batch(elbm_batch_t *b, const void *fin, void *fout, int bx)
{
    const CollideParams p = params_of(b, 0.0); // beta comes from the domain table
    if (build_tables(b, bx) != ELBM_OK) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    for (const eelbm::BatchTable &t : b->tables[bx]) {
        e = b->D == 2 ? eelbm::launch_step_batch_d2q9(b->opts.storage, fin, fout, t, bx, p, b->stream)
                      : eelbm::launch_step_batch_d3q27(b->opts.storage, fin, fout, t, bx, p, b->stream);
        if (e != cudaSuccess) break;
    }
    return e;
}

int ensure_stage(elbm_batch_t *b, size_t bytes)
{
    if (b->stage_bytes >= bytes) return ELBM_OK;
    if (b->stage) {
        cudaStreamSynchronize(b->stream);
        cudaFree(b->stage);
        b->stage = nullptr;
        b->stage_bytes = 0;
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&b->stage), bytes);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch: cudaMalloc(staging)");
    b->stage_bytes = bytes;
    return ELBM_OK;
}

void drop_graphs(elbm_batch_t *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

void drop_persist(elbm_batch_t *b)
{
    for (auto &kv : b->persist) {
        cudaFree(kv.second.chunks);
        cudaFree(kv.second.owners);
        cudaFree(kv.second.cnt);
        cudaFree(kv.second.doms);
    }
    b->persist.clear();
}

// Work chunks of the persistent launch at width bx: every domain's work items cut into
// runs of kPersistChunkItems (the last run of a domain shorter), in domain order; the
// grid is every resident block (blocks per SM from the occupancy calculator, times
// the SM count).  On the 64-domain D2Q9 ensemble: 71.5 GLUPS with runs of 16 items,
// 69.0 with 8, 54.1 with 32 (longer waits at each domain's step boundary).
#ifndef ELBM_PERSIST_CHUNK
#define ELBM_PERSIST_CHUNK 16
#endif
constexpr int kPersistChunkItems = ELBM_PERSIST_CHUNK;
int build_persist(elbm_batch_t *b, int bx)
{
    if (b->persist.count(bx)) return ELBM_OK;
    int st = build_tables(b, bx);
    if (st != ELBM_OK) return st;
    std::vector<eelbm::BatchTableDom> tdoms;
    for (const eelbm::BatchTable &t : b->tables[bx])
        for (int k = 0; k < t.n; ++k) tdoms.push_back(t.dom[k]);
    std::vector<int4> chunks;
    std::vector<unsigned> owners(tdoms.size(), 0u);
    for (size_t d = 0; d < tdoms.size(); ++d) {
        const int64_t items = int64_t(tdoms[d].xblocks) * tdoms[d].ny * tdoms[d].nz;
        for (int64_t w = 0; w < items; w += kPersistChunkItems) {
            chunks.push_back(make_int4(int(d), int(w), int(std::min<int64_t>(items, w + kPersistChunkItems)), 0));
            owners[d] += 1u;
        }
    }
    if (chunks.size() >= (size_t(1) << 31)) return bfail(b, ELBM_ERR_ARG, "elbm_batch: too many work chunks");
    int per_sm = 0;
    cudaError_t e = b->D == 2 ? eelbm::persist_blocks_per_sm_d2q9(b->opts.storage, bx, &per_sm)
                              : eelbm::persist_blocks_per_sm_d3q27(b->opts.storage, bx, &per_sm);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch: occupancy of the persistent kernel");
    if (per_sm < 1) return bfail(b, ELBM_ERR_UNSUPPORTED, "elbm_batch: persistent kernel cannot be resident");
    const int G = int(std::min<int64_t>(int64_t(b->num_sms) * per_sm, int64_t(chunks.size())));
    elbm_batch_t::Persist ps;
    e = cudaMalloc(reinterpret_cast<void **>(&ps.chunks), chunks.size() * sizeof(int4));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&ps.owners), owners.size() * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&ps.cnt), (owners.size() + 1) * sizeof(unsigned));
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&ps.doms), tdoms.size() * sizeof(eelbm::BatchTableDom));
    if (e == cudaSuccess)
        e = cudaMemcpy(ps.doms, tdoms.data(), tdoms.size() * sizeof(eelbm::BatchTableDom), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ps.chunks, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ps.owners, owners.data(), owners.size() * sizeof(unsigned), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(ps.chunks);
        cudaFree(ps.owners);
        cudaFree(ps.cnt);
        cudaFree(ps.doms);
        return bcuda(b, e, "elbm_batch: persistent plan");
    }
    ps.plan.grid = G;
    ps.plan.nchunks = unsigned(chunks.size());
    ps.plan.chunks = ps.chunks;
    ps.plan.owners = ps.owners;
    ps.plan.cnt = ps.cnt;
    ps.plan.ticket = ps.cnt + owners.size();
    ps.h_owners = owners;
    // tickets (steps x chunks) and counters (steps x chunks of a domain) stay below 2^32
    ps.max_steps = int(std::min<uint64_t>(uint64_t(1) << 20, 0xffffffffull / (uint64_t(chunks.size()) + 1u)));
    b->persist[bx] = ps;
    return ELBM_OK;
}

// Enqueues n steps as persistent launches (counters cleared before each).
cudaError_t launch_persist(elbm_batch_t *b, int64_t n, int cur)
{
    const elbm_batch_t::Persist &ps = b->persist[b->pbx];
    const CollideParams p = params_of(b, 0.0); // beta comes from the domain table
    cudaError_t e = cudaSuccess;
    for (int64_t done = 0; done < n && e == cudaSuccess;) {
        const int k = int(std::min<int64_t>(n - done, ps.max_steps)); // counters stay below 2^32
        e = cudaMemsetAsync(ps.cnt, 0, (b->doms.size() + 1) * sizeof(unsigned), b->stream);
        if (e == cudaSuccess)
            e = b->D == 2 ? eelbm::launch_step_persist_d2q9(b->opts.storage, b->pop[0], b->pop[1], cur, k, ps.doms,
                                                            ps.plan, b->pbx, p, b->err_word, b->stream)
                          : eelbm::launch_step_persist_d3q27(b->opts.storage, b->pop[0], b->pop[1], cur, k, ps.doms,
                                                             ps.plan, b->pbx, p, b->err_word, b->stream);
        cur ^= k & 1;
        done += k;
    }
    return e;
}

// Reads (and clears) the device error word after the stream has been synchronised.
int check_flag(elbm_batch_t *b, const char *what)
{
    int flag = 0;
    cudaError_t e = cudaMemcpy(&flag, b->err_word, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, what);
    if (flag != 0) {
        cudaMemset(b->err_word, 0, sizeof(int));
        return bfail(b, ELBM_ERR_TIMEOUT, "%s: a bounded device-side wait expired (the steps were not completed)",
                     what);
    }
    return ELBM_OK;
}

} // namespace

extern "C" {

int elbm_batch_create(elbm_batch_t **out, int lattice, int ndomains, const int64_t *dims, const double *beta,
                      const elbm_opts *opts)
{
    if (!out) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: out is NULL");
    *out = nullptr;
    if (lattice != ELBM_D2Q9 && lattice != ELBM_D3Q27)
        return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: lattice must be 9 or 27, got %d", lattice);
    if (ndomains < 1) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: ndomains = %d < 1", ndomains);
    if (!dims || !beta) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: dims or beta is NULL");
    elbm_opts o;
    elbm_default_opts(&o);
    if (opts) o = *opts;
    const size_t es = elem_size(o.storage);
    if (!es) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: unknown storage %d", o.storage);
    if (o.alpha_mode < ELBM_ALPHA_HIGHER || o.alpha_mode > ELBM_ALPHA_ITERATE1 || (o.cutoff != 0 && o.cutoff != 1) ||
        (o.b_variant != ELBM_B_DERIVED && o.b_variant != ELBM_B_PRINTED) || !(o.rho0 > 0.0))
        return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: invalid options");
    const int Q = lattice;
    std::vector<BatchDomain> doms(ndomains);
    size_t total = 0;
    const size_t align = 256 / es; // elements per 256 bytes
    for (int d = 0; d < ndomains; ++d) {
        const int64_t *dd = dims + 3 * d;
        for (int a = 0; a < 3; ++a)
            if (dd[a] < 1 || dd[a] > 65535)
                return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: domain %d dims[%d] = %lld out of [1, 65535]",
                             d, a, (long long)dd[a]);
        if (lattice == ELBM_D2Q9 && dd[2] != 1)
            return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: domain %d: D2Q9 needs dims[2] == 1", d);
        if (!(beta[d] > 0.0 && beta[d] < 1.0))
            return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: domain %d: beta = %g outside (0, 1)", d,
                         beta[d]);
        if (uint64_t(Q) * uint64_t(dd[0] * dd[1] * dd[2]) > 0xffffffffull)
            return bfail(nullptr, ELBM_ERR_UNSUPPORTED,
                         "elbm_batch_create: domain %d: Q N = %lld populations exceed the 32-bit offsets of the "
                         "batched kernels (at most 2^32 - 1)",
                         d, (long long)(Q * dd[0] * dd[1] * dd[2]));
        BatchDomain &m = doms[d];
        m.nx = int(dd[0]);
        m.ny = int(dd[1]);
        m.nz = int(dd[2]);
        m.N = dd[0] * dd[1] * dd[2];
        m.off = int64_t(total);
        m.beta = beta[d];
        m.beta_f = float(beta[d]);
        total += (size_t(Q) * size_t(m.N) + align - 1) / align * align;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return bcuda(nullptr, e, "elbm_batch_create: cudaGetDeviceCount");
    if (o.device < 0 || o.device >= ndev)
        return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: device %d not present", o.device);
    DeviceGuard guard(o.device);
    elbm_batch_t *b = new (std::nothrow) elbm_batch_t();
    if (!b) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_create: out of host memory");
    b->lattice = lattice;
    b->D = lattice == ELBM_D2Q9 ? 2 : 3;
    b->Q = Q;
    b->opts = o;
    b->doms = doms;
    b->elem = es;
    b->total_elems = total;
    if (o.stream) {
        b->stream = static_cast<cudaStream_t>(o.stream);
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return bcuda(nullptr, e, "elbm_batch_create: cudaStreamCreate");
        }
        b->own_stream = true;
    }
    e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, o.device);
    if (e == cudaSuccess) e = cudaMalloc(&b->pop[0], total * es);
    if (e == cudaSuccess) e = cudaMalloc(&b->pop[1], total * es);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->acc), sizeof(DiagAcc));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->err_word), sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->err_word, 0, sizeof(int));
    if (e != cudaSuccess) {
        elbm_batch_destroy(b);
        return bcuda(nullptr, e, "elbm_batch_create: device allocation");
    }
    int st = build_tables(b, b->bx);
    if (st != ELBM_OK) {
        std::string msg = b->err;
        elbm_batch_destroy(b);
        return bfail(nullptr, st, "%s", msg.c_str());
    }
    *out = b;
    return ELBM_OK;
}

void elbm_batch_destroy(elbm_batch_t *b)
{
    if (!b) return;
    DeviceGuard guard(b->opts.device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    cudaFree(b->pop[0]);
    cudaFree(b->pop[1]);
    cudaFree(b->stage);
    cudaFree(b->acc);
    cudaFree(b->err_word);
    drop_persist(b);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *elbm_batch_last_error(const elbm_batch_t *b)
{
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

int elbm_batch_init_equilibrium(elbm_batch_t *b, int domain, const double *rho, const double *u, int where)
{
    int st = check_domain(b, domain, "elbm_batch_init_equilibrium");
    if (st != ELBM_OK) return st;
    if (!u) return bfail(b, ELBM_ERR_ARG, "elbm_batch_init_equilibrium: u is NULL");
    if (where != ELBM_MEM_DEVICE && where != ELBM_MEM_HOST)
        return bfail(b, ELBM_ERR_ARG, "elbm_batch_init_equilibrium: bad memory location %d", where);
    DeviceGuard guard(b->opts.device);
    const BatchDomain &dm = b->doms[domain];
    const double *drho = rho, *du = u;
    cudaError_t e;
    if (where == ELBM_MEM_HOST) {
        if ((st = ensure_stage(b, size_t(dm.N) * (1 + b->D) * sizeof(double))) != ELBM_OK) return st;
        if (rho) {
            e = cudaMemcpyAsync(b->stage, rho, size_t(dm.N) * sizeof(double), cudaMemcpyHostToDevice, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_init_equilibrium: copy rho");
            drho = b->stage;
        }
        e = cudaMemcpyAsync(b->stage + dm.N, u, size_t(dm.N) * b->D * sizeof(double), cudaMemcpyHostToDevice,
                            b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_init_equilibrium: copy u");
        du = b->stage + dm.N;
    }
    // both buffers hold the domain's state, so the step parity does not matter
    for (int k = 0; k < 2; ++k) {
        void *f = static_cast<char *>(b->pop[k]) + size_t(dm.off) * b->elem;
        e = b->D == 2 ? eelbm::launch_init_d2q9(b->opts.storage, drho, du, f, geom_of(dm), b->opts.rho0, b->opts.rho0,
                                                0, dm.N, b->stream)
                      : eelbm::launch_init_d3q27(b->opts.storage, drho, du, f, geom_of(dm), b->opts.rho0,
                                                 b->opts.rho0, 0, dm.N, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_init_equilibrium: kernel launch");
    }
    if (where == ELBM_MEM_HOST) {
        e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_init_equilibrium: synchronize");
    }
    return ELBM_OK;
}

int elbm_batch_step(elbm_batch_t *b, int64_t n, int mode)
{
    if (!b) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_step: batch is NULL");
    if (n < 0) return bfail(b, ELBM_ERR_ARG, "elbm_batch_step: n = %lld < 0", (long long)n);
    if (mode != ELBM_BATCH_GRAPH && mode != ELBM_BATCH_LAUNCHES && mode != ELBM_BATCH_PER_DOMAIN &&
        mode != ELBM_BATCH_PERSISTENT && mode != ELBM_BATCH_AUTO)
        return bfail(b, ELBM_ERR_ARG, "elbm_batch_step: unknown mode %d", mode);
    if (mode == ELBM_BATCH_AUTO) mode = b->auto_mode;
    if (n == 0) return ELBM_OK;
    DeviceGuard guard(b->opts.device);
    cudaError_t e;
    if (mode == ELBM_BATCH_PER_DOMAIN) {
        for (int64_t k = 0; k < n; ++k) {
            for (const BatchDomain &dm : b->doms) {
                const void *fin = static_cast<const char *>(b->pop[b->cur]) + size_t(dm.off) * b->elem;
                void *fout = static_cast<char *>(b->pop[b->cur ^ 1]) + size_t(dm.off) * b->elem;
                e = b->D == 2 ? eelbm::launch_step_d2q9(b->opts.storage, fin, fout, geom_of(dm), params_of(b, dm.beta),
                                                        ELBM_KERNEL_DIRECT, b->num_sms, nullptr, b->stream)
                              : eelbm::launch_step_d3q27(b->opts.storage, fin, fout, geom_of(dm),
                                                         params_of(b, dm.beta), ELBM_KERNEL_DIRECT, b->num_sms,
                                                         nullptr, b->stream);
                if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_step: per-domain launch");
            }
            b->cur ^= 1;
            b->steps += 1;
        }
        return ELBM_OK;
    }
    if (mode == ELBM_BATCH_LAUNCHES) {
        for (int64_t k = 0; k < n; ++k) {
            e = launch_batch(b, b->pop[b->cur], b->pop[b->cur ^ 1], b->bx);
            if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_step: launch");
            b->cur ^= 1;
            b->steps += 1;
        }
        return ELBM_OK;
    }
    if (mode == ELBM_BATCH_PERSISTENT) {
        int st = build_persist(b, b->pbx);
        if (st != ELBM_OK) return st;
    }
    // ELBM_BATCH_GRAPH: the n launches captured once per (n, starting buffer, width);
    // ELBM_BATCH_PERSISTENT: the persistent launch(es) of n steps, captured likewise
    const std::pair<int64_t, int> key(n, mode == ELBM_BATCH_PERSISTENT ? 4096 + b->cur + 2 * b->pbx
                                                                      : b->cur + 2 * b->bx);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_step: cudaStreamBeginCapture");
        int c = b->cur;
        cudaError_t le = cudaSuccess;
        if (mode == ELBM_BATCH_PERSISTENT) {
            le = launch_persist(b, n, c);
        } else {
            for (int64_t k = 0; k < n && le == cudaSuccess; ++k) {
                le = launch_batch(b, b->pop[c], b->pop[c ^ 1], b->bx);
                c ^= 1;
            }
        }
        e = cudaStreamEndCapture(b->stream, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return bcuda(b, le, "elbm_batch_step: captured launch");
        }
        if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_step: cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_step: cudaGraphInstantiate");
        it = b->graphs.emplace(key, exec).first;
    }
    e = cudaGraphLaunch(it->second, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_step: cudaGraphLaunch");
    b->cur ^= int(n & 1);
    b->steps += n;
    return ELBM_OK;
}

int elbm_batch_tune(elbm_batch_t *b, int *chosen, double *ms_per_step)
{
    if (!b) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_tune: batch is NULL");
    DeviceGuard guard(b->opts.device);
    static const int cands[3] = {64, 128, 256};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_tune: cudaEventCreate");
    double best = 1e300;
    int best_bx = b->bx;
    for (int c = 0; c < 3; ++c) {
        const int bx = cands[c];
        int st = build_tables(b, bx);
        if (st != ELBM_OK) return st;
        // trial steps read the current buffer and write the other one: the state is kept
        const void *fin = b->pop[b->cur];
        void *fout = b->pop[b->cur ^ 1];
        e = launch_batch(b, fin, fout, bx);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = launch_batch(b, fin, fout, bx);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return bcuda(b, e, "elbm_batch_tune: trial");
        }
        if (ms_per_step) ms_per_step[c] = ms / 5.0;
        if (ms < best) {
            best = ms;
            best_bx = bx;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_bx != b->bx) drop_graphs(b);
    b->bx = best_bx;
    b->graph_ms = best / 5.0; // marks the width trials as done
    if (chosen) *chosen = best_bx;
    return ELBM_OK;
}

int elbm_batch_tune_persistent(elbm_batch_t *b, int *chosen_mode, double *ms_per_step)
{
    if (!b) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_tune_persistent: batch is NULL");
    DeviceGuard guard(b->opts.device);
    static const int cands[3] = {64, 128, 256};
    constexpr int kTrial = 50; // timed steps per trial, after 2 untimed ones
    if (b->graph_ms <= 0.0) {  // the graph's width, from its own trials
        int st = elbm_batch_tune(b, nullptr, nullptr);
        if (st != ELBM_OK) return st;
    }
    // the trials advance a copy of the state: save the current buffer, restore it after
    const size_t bytes = b->total_elems * b->elem;
    void *save = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&save, bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(save, b->pop[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // every trial starts from the saved state (steps near equilibrium are cheaper)
    auto restore = [&]() {
        return cudaMemcpyAsync(b->pop[b->cur], save, bytes, cudaMemcpyDeviceToDevice, b->stream);
    };
    // the batched launches at the graph's width, kTrial steps as one CUDA graph (the form
    // ELBM_BATCH_GRAPH replays): captured, replayed once untimed, then timed from the
    // saved state
    float graph_ms = 0.0f;
    cudaGraphExec_t trial = nullptr;
    if (e == cudaSuccess) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        cudaError_t le = cudaSuccess;
        int c = b->cur;
        for (int k = 0; k < kTrial && e == cudaSuccess && le == cudaSuccess; ++k) {
            le = launch_batch(b, b->pop[c], b->pop[c ^ 1], b->bx);
            c ^= 1;
        }
        if (e == cudaSuccess) e = cudaStreamEndCapture(b->stream, &graph);
        if (e == cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&trial, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess) e = cudaGraphLaunch(trial, b->stream);
        if (e == cudaSuccess) e = restore();
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(trial, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&graph_ms, e0, e1);
    }
    if (trial) cudaGraphExecDestroy(trial);
    double best = 1e300;
    int best_bx = b->pbx, st = ELBM_OK;
    for (int c = 0; c < 3 && e == cudaSuccess && st == ELBM_OK; ++c) {
        const int keep = b->pbx;
        b->pbx = cands[c];
        st = build_persist(b, b->pbx);
        if (st == ELBM_OK) {
            e = restore();
            if (e == cudaSuccess) e = launch_persist(b, 2, b->cur);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess) e = launch_persist(b, kTrial, b->cur);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess) {
                if (ms_per_step) ms_per_step[c] = ms / kTrial;
                if (ms < best) {
                    best = ms;
                    best_bx = cands[c];
                }
            }
        }
        b->pbx = keep;
    }
    cudaError_t er = cudaSuccess;
    if (save) {
        er = restore();
        if (er == cudaSuccess) er = cudaStreamSynchronize(b->stream);
        cudaFree(save);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != ELBM_OK) return st;
    if (e == cudaSuccess) e = er;
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_tune_persistent");
    if ((st = check_flag(b, "elbm_batch_tune_persistent")) != ELBM_OK) return st;
    b->pbx = best_bx;
    b->auto_mode = best < graph_ms ? ELBM_BATCH_PERSISTENT : ELBM_BATCH_GRAPH;
    if (chosen_mode) *chosen_mode = b->auto_mode;
    return ELBM_OK;
}

int elbm_batch_moments(elbm_batch_t *b, int domain, double *rho_out, double *u_out, int where)
{
    int st = check_domain(b, domain, "elbm_batch_moments");
    if (st != ELBM_OK) return st;
    if (where != ELBM_MEM_DEVICE && where != ELBM_MEM_HOST)
        return bfail(b, ELBM_ERR_ARG, "elbm_batch_moments: bad memory location %d", where);
    if (!rho_out && !u_out) return ELBM_OK;
    DeviceGuard guard(b->opts.device);
    const BatchDomain &dm = b->doms[domain];
    double *drho = rho_out, *du = u_out;
    if (where == ELBM_MEM_HOST) {
        if ((st = ensure_stage(b, size_t(dm.N) * (1 + b->D) * sizeof(double))) != ELBM_OK) return st;
        drho = rho_out ? b->stage : nullptr;
        du = u_out ? b->stage + dm.N : nullptr;
    }
    const void *f = static_cast<const char *>(b->pop[b->cur]) + size_t(dm.off) * b->elem;
    cudaError_t e = b->D == 2 ? eelbm::launch_moments_d2q9(b->opts.storage, f, geom_of(dm), b->opts.rho0, drho, du,
                                                           0, dm.N, b->stream)
                              : eelbm::launch_moments_d3q27(b->opts.storage, f, geom_of(dm), b->opts.rho0, drho,
                                                            du, 0, dm.N, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_moments: kernel launch");
    if (where == ELBM_MEM_HOST) {
        if (rho_out) e = cudaMemcpyAsync(rho_out, drho, size_t(dm.N) * sizeof(double), cudaMemcpyDeviceToHost,
                                         b->stream);
        if (e == cudaSuccess && u_out)
            e = cudaMemcpyAsync(u_out, du, size_t(dm.N) * b->D * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_moments: read back");
    }
    return ELBM_OK;
}

int elbm_batch_diagnostics(elbm_batch_t *b, int domain, elbm_diag *out, int64_t *alpha_hist)
{
    int st = check_domain(b, domain, "elbm_batch_diagnostics");
    if (st != ELBM_OK) return st;
    if (!out) return bfail(b, ELBM_ERR_ARG, "elbm_batch_diagnostics: out is NULL");
    DeviceGuard guard(b->opts.device);
    const BatchDomain &dm = b->doms[domain];
    cudaError_t e = cudaMemsetAsync(b->acc, 0, sizeof(DiagAcc), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&b->acc->amin_ord, 0xFF, sizeof(unsigned long long), b->stream);
    const void *f = static_cast<const char *>(b->pop[b->cur]) + size_t(dm.off) * b->elem;
    if (e == cudaSuccess)
        e = b->D == 2 ? eelbm::launch_diag_d2q9(b->opts.storage, f, geom_of(dm), params_of(b, dm.beta), b->acc,
                                                b->num_sms, b->stream)
                      : eelbm::launch_diag_d3q27(b->opts.storage, f, geom_of(dm), params_of(b, dm.beta), b->acc,
                                                 b->num_sms, b->stream);
    DiagAcc acc;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&acc, b->acc, sizeof acc, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_diagnostics");
    out->mass = acc.sum[0];
    out->momentum[0] = acc.sum[1];
    out->momentum[1] = acc.sum[2];
    out->momentum[2] = b->D == 3 ? acc.sum[3] : 0.0;
    out->H = acc.sum[4];
    out->dH_max = eelbm::from_ordered_bits(acc.dH_max_ord);
    out->alpha_min = eelbm::from_ordered_bits(acc.amin_ord);
    out->alpha_max = eelbm::from_ordered_bits(acc.amax_ord);
    out->alpha_mean = acc.sum[5] / double(dm.N);
    out->n_nodes = dm.N;
    out->n_cutoff = int64_t(acc.cnt[0]);
    out->n_solved = int64_t(acc.cnt[1]);
    out->n_clamped = int64_t(acc.cnt[2]);
    out->n_nonpositive = int64_t(acc.cnt[3]);
    out->n_dH_positive = int64_t(acc.cnt[4]);
    for (int b = 0; b < 4; ++b) out->n_xmax_band[b] = int64_t(acc.cnt[5 + b]);
    if (alpha_hist)
        for (int k = 0; k < ELBM_HIST_BINS + 2; ++k) alpha_hist[k] = int64_t(acc.hist[k]);
    if (out->n_nonpositive > 0)
        return bfail(b, ELBM_ERR_NONPHYSICAL, "elbm_batch_diagnostics: %lld nodes with a population <= 0",
                     (long long)out->n_nonpositive);
    return ELBM_OK;
}

int elbm_batch_get_populations(elbm_batch_t *b, int domain, void *dst, int where)
{
    int st = check_domain(b, domain, "elbm_batch_get_populations");
    if (st != ELBM_OK) return st;
    if (!dst || (where != ELBM_MEM_DEVICE && where != ELBM_MEM_HOST))
        return bfail(b, ELBM_ERR_ARG, "elbm_batch_get_populations: bad destination");
    DeviceGuard guard(b->opts.device);
    const BatchDomain &dm = b->doms[domain];
    const void *src = static_cast<const char *>(b->pop[b->cur]) + size_t(dm.off) * b->elem;
    cudaError_t e = cudaMemcpyAsync(dst, src, size_t(b->Q) * size_t(dm.N) * b->elem,
                                    where == ELBM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                    b->stream);
    if (e == cudaSuccess && where == ELBM_MEM_HOST) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_get_populations");
    return ELBM_OK;
}

int elbm_batch_set_populations(elbm_batch_t *b, int domain, const void *src, int where)
{
    int st = check_domain(b, domain, "elbm_batch_set_populations");
    if (st != ELBM_OK) return st;
    if (!src || (where != ELBM_MEM_DEVICE && where != ELBM_MEM_HOST))
        return bfail(b, ELBM_ERR_ARG, "elbm_batch_set_populations: bad source");
    DeviceGuard guard(b->opts.device);
    const BatchDomain &dm = b->doms[domain];
    const size_t bytes = size_t(b->Q) * size_t(dm.N) * b->elem;
    cudaError_t e = cudaSuccess;
    // write both buffers so that the step parity does not matter
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(static_cast<char *>(b->pop[k]) + size_t(dm.off) * b->elem, src, bytes,
                            where == ELBM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess && where == ELBM_MEM_HOST) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_set_populations");
    return ELBM_OK;
}

int elbm_batch_synchronize(elbm_batch_t *b)
{
    if (!b) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_synchronize: batch is NULL");
    DeviceGuard guard(b->opts.device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_synchronize");
    return check_flag(b, "elbm_batch_synchronize");
}

int elbm_batch_check_wait_timeout(elbm_batch_t *b)
{
    if (!b) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_check_wait_timeout: batch is NULL");
    DeviceGuard guard(b->opts.device);
    int st = build_persist(b, b->pbx);
    if (st != ELBM_OK) return st;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_check_wait_timeout: synchronize");
    if ((st = check_flag(b, "elbm_batch_check_wait_timeout")) != ELBM_OK) return st;
    // every domain gets one chunk more than it has: that chunk never arrives
    const elbm_batch_t::Persist &ps = b->persist[b->pbx];
    std::vector<unsigned> ghost(ps.h_owners);
    for (unsigned &o : ghost) o += 1u;
    unsigned *d_ghost = nullptr;
    e = cudaMalloc(reinterpret_cast<void **>(&d_ghost), ghost.size() * sizeof(unsigned));
    if (e == cudaSuccess)
        e = cudaMemcpy(d_ghost, ghost.data(), ghost.size() * sizeof(unsigned), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(ps.cnt, 0, (ghost.size() + 1) * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) {
        eelbm::PersistPlan plan = ps.plan;
        plan.owners = d_ghost;
        const CollideParams p = params_of(b, 0.0);
        // two steps: step 0 writes the spare buffer, every wait before step 1 expires,
        // so the current buffer (the state) is never written
        e = b->D == 2 ? eelbm::launch_step_persist_d2q9(b->opts.storage, b->pop[0], b->pop[1], b->cur, 2, ps.doms,
                                                        plan, b->pbx, p, b->err_word, b->stream)
                      : eelbm::launch_step_persist_d3q27(b->opts.storage, b->pop[0], b->pop[1], b->cur, 2, ps.doms,
                                                         plan, b->pbx, p, b->err_word, b->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d_ghost);
    if (e != cudaSuccess) return bcuda(b, e, "elbm_batch_check_wait_timeout: launch");
    st = check_flag(b, "elbm_batch_check_wait_timeout");
    if (st == ELBM_ERR_TIMEOUT) return ELBM_OK; // detected, flag cleared
    if (st != ELBM_OK) return st;
    return bfail(b, ELBM_ERR_CUDA, "elbm_batch_check_wait_timeout: the expired wait was not reported");
}

int elbm_batch_info(const elbm_batch_t *b, int *ndomains, int64_t *nodes, int *block_width)
{
    if (!b) return bfail(nullptr, ELBM_ERR_ARG, "elbm_batch_info: batch is NULL");
    if (ndomains) *ndomains = int(b->doms.size());
    if (nodes) {
        int64_t s = 0;
        for (const BatchDomain &d : b->doms) s += d.N;
        *nodes = s;
    }
    if (block_width) *block_width = b->bx;
    return ELBM_OK;
}

} // extern "C"
