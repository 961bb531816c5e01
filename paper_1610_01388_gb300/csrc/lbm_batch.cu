// Batched stepping of many resident domains (lbm_batch_*) and the serving
// loop with continuous batching built on it (lbm_server_*).
//
// A batch keeps one solver per domain (device memory from the stream-ordered
// pool, admitted against a byte budget) and, per (lattice, model, storage)
// group, a device table of BatchDesc plus a block -> domain map.  One launch
// of k_step_batch per group advances every domain of the group by one step;
// the A/B buffer of a domain is phase ^ parity0, so graphs that alternate the
// phase stay valid.  Check steps reduce per-block partials into one stats row
// per domain (its "slot"), copied to pinned host memory.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "kernels.cuh"
#include "solver.h"

using namespace blbm;

namespace {

constexpr int kMaxSlots = 8192;     // domains resident at once
constexpr int kFlowChangeSlot = kStatFlowChange;
static_assert(kFlowChangeSlot == kNumStats - 1 && kStatNonFinite < kFlowChangeSlot,
              "the flow change takes the stats row's last entry, which check steps leave at 0");
constexpr int kGraphLen = 16;       // steps per captured graph (even)

// Per domain: the fixed-order sum of its tiles' partials into its stats row,
// and in the row's last entry the relative change of the flow-rate vector
// against the row's previous contents, |S - S_prev| / |S| with S the sums of
// u_real over fluid cells (the change of the mean velocity vector); -1 when
// the row held no previous check (lbm_batch_add clears it).
__global__ void k_finalize_domains(const BatchDesc* __restrict__ descs,
                                   const double* __restrict__ partials, double* __restrict__ slots) {
    const BatchDesc& D = descs[blockIdx.x];
    double* row = slots + (int64_t)D.slot * kNumStats;
    double prev[3] = {0.0, 0.0, 0.0};
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) prev[a] = row[kStatUx + a];   // read before the row is rewritten
    double v[kNumStats];
#pragma unroll
    for (int k = 0; k < kNumStats; ++k) v[k] = 0.0;
    for (int b = threadIdx.x; b < D.nblocks; b += kBlock) {
        const double* p = partials + (int64_t)(D.block_begin + b) * kNumStats;
#pragma unroll
        for (int k = 0; k < kNumStats; ++k) v[k] += p[k];
    }
    __shared__ double sm[kBlock][kNumStats];
#pragma unroll
    for (int k = 0; k < kNumStats; ++k) sm[threadIdx.x][k] = v[k];
    __syncthreads();
    for (int o = kBlock / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < kNumStats; ++k) sm[threadIdx.x][k] += sm[threadIdx.x + o][k];
        __syncthreads();
    }
    if (threadIdx.x < kFlowChangeSlot) row[threadIdx.x] = sm[0][threadIdx.x];
    if (threadIdx.x == 0) {
        double d2 = 0.0, s2 = 0.0, p2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double cur = sm[0][kStatUx + a];
            d2 += (cur - prev[a]) * (cur - prev[a]);
            s2 += cur * cur;
            p2 += prev[a] * prev[a];
        }
        row[kFlowChangeSlot] = (p2 > 0.0 && s2 > 0.0) ? sqrt(d2 / s2) : -1.0;
    }
}

cudaError_t launch_batch(int lat, int model, int storage, bool check, const BatchDesc* d,
                         const int* bd, int nblocks, int grid, int phase, double* partials,
                         int threads, int cpt, cudaStream_t st) {
    switch (lat) {
    case LBM_D2Q9: return launch_step_batch_D2Q9(model, storage, check, d, bd, nblocks, grid, phase, partials, threads, cpt, st);
    case LBM_D3Q15: return launch_step_batch_D3Q15(model, storage, check, d, bd, nblocks, grid, phase, partials, threads, cpt, st);
    case LBM_D3Q19: return launch_step_batch_D3Q19(model, storage, check, d, bd, nblocks, grid, phase, partials, threads, cpt, st);
    default: return launch_step_batch_D3Q27(model, storage, check, d, bd, nblocks, grid, phase, partials, threads, cpt, st);
    }
}

struct Group {
    int lat = 0, model = 0, storage = 0;   // model: kernel-side model code
    int user_model = 0;                    // lbm_model, the schedule key
    std::vector<int64_t> ids;
    int nblocks = 0;                       // check steps: tiles of kBlock cells
    int grid = 0;                          // check steps: CTAs per launch
    int tile_threads = kBlock;             // plain steps: tile shape of the schedule
    int tile_cpt = 1;
    int pnblocks = 0;                      // plain steps: tiles of tile_threads x tile_cpt cells
    int pgrid = 0;                         // plain steps: CTAs per launch
    BatchDesc* d_desc = nullptr;
    int* d_block_dom = nullptr;
    int* d_pblock_dom = nullptr;
    double* d_partials = nullptr;
    int cap_desc = 0, cap_blocks = 0, cap_pblocks = 0;
};

struct Dom {
    lbm_solver* s = nullptr;
    void* ws = nullptr;
    size_t bytes = 0;
    int parity0 = 0;
    int slot = -1;
    int64_t checks = 0;
};

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Process-wide batch schedule: CTAs per SM of each (lattice, model, storage)
// group's launch (0 = one CTA per tile) and whether captured graphs run the
// groups as concurrent branches.  Batches adopt a change at their next step.
std::mutex g_sched_mu;
std::map<int, int> g_sched_ctas;
std::map<int, std::map<int, std::pair<int, int>>> g_sched_tile;   // key -> size class -> shape
std::atomic<int> g_sched_concurrent{0};
std::atomic<uint64_t> g_sched_version{1};

int sched_key(int lat, int model, int storage) { return (lat * 4 + model) * 8 + storage; }

int sched_ctas(int lat, int model, int storage) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    auto it = g_sched_ctas.find(sched_key(lat, model, storage));
    return it == g_sched_ctas.end() ? 0 : it->second;
}

// size class of a group: floor(log2) of its domains' mean cell count
int batch_size_class(int64_t cells) {
    int c = 0;
    while (c < 62 && ((int64_t)1 << (c + 1)) <= cells) ++c;
    return c;
}

// Plain-step tile shape for a group of this class: the entry of the class,
// else the entry of the nearest class set for (lattice, model, storage),
// else 256 x 1.
std::pair<int, int> sched_tile(int lat, int model, int storage, int cls) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    auto it = g_sched_tile.find(sched_key(lat, model, storage));
    if (it == g_sched_tile.end() || it->second.empty()) return {kBlock, 1};
    int best = -1, dist = 1 << 30;
    for (const auto& kv : it->second) {
        const int d = std::abs(kv.first - cls);
        if (d < dist) {
            dist = d;
            best = kv.first;
        }
    }
    return it->second.at(best);
}

bool valid_tile(int threads, int cpt) {
    return (threads == 128 || threads == 256 || threads == 512) && (cpt == 1 || cpt == 2) &&
           !(threads == 512 && cpt == 2);
}

}  // namespace

void blbm::clear_batch_schedule() {
    {
        std::lock_guard<std::mutex> lk(g_sched_mu);
        g_sched_ctas.clear();
        g_sched_tile.clear();
    }
    g_sched_concurrent.store(0);
    g_sched_version.fetch_add(1);
}

struct lbm_batch {
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    int device = 0;
    size_t budget = 0, used = 0;
    int k = 0;
    int64_t gstep = 0;
    int phase = 0;
    int64_t next_id = 1;
    std::map<int64_t, Dom> doms;
    std::vector<Group> groups;
    std::vector<int> free_slots;
    double* d_slots = nullptr;      // [kMaxSlots][kNumStats]
    double* h_slots = nullptr;      // pinned mirror
    bool dirty = true;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool poisoned = false;
    int sms = 1;                          // multiprocessors of the device
    uint64_t sched_version = 0;           // schedule the groups were built with
    bool concurrent = false;              // graphs run groups as parallel branches
    std::vector<cudaStream_t> branch;     // capture branches, one per group
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
};

namespace {

lbm_status bfail(lbm_batch* b, cudaError_t e, const char* what) {
    if (b) b->poisoned = true;
    cudaGetLastError();
    return fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BCK(b, expr, what)                                     \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return bfail(b, e_, what);      \
    } while (0)

#define BWAIT(b, what)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = bounded_sync((b)->stream);                                         \
        if (e_ == cudaErrorNotReady)                                                        \
            return fail(LBM_ETIMEOUT, "%s: queued work still running after the %g s wait limit", \
                        what, wait_limit());                                                \
        if (e_ != cudaSuccess) return bfail(b, e_, what);                                   \
    } while (0)

lbm_status benter(const lbm_batch* b) {
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (b->poisoned) return fail(LBM_ECUDA, "batch is in an error state after a CUDA failure");
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev != b->device) cudaSetDevice(b->device);
    return LBM_OK;
}

void drop_graphs(lbm_batch* b) {
    for (int p = 0; p < 2; ++p)
        if (b->graph[p]) {
            cudaGraphExecDestroy(b->graph[p]);
            b->graph[p] = nullptr;
        }
}

// (Re)build the per-group device tables after the set of domains or the
// schedule changed.
lbm_status rebuild(lbm_batch* b) {
    drop_graphs(b);
    b->sched_version = g_sched_version.load();
    b->concurrent = g_sched_concurrent.load() != 0;
    std::vector<Group> old;
    old.swap(b->groups);
    for (auto& kv : b->doms) {
        const lbm_solver* s = kv.second.s;
        const int km = kernel_model(s->p.model, s->kp.newton);   // kernel-side model code
        Group* g = nullptr;
        for (auto& x : b->groups)
            if (x.lat == s->lat && x.model == km && x.storage == s->p.storage) g = &x;
        if (!g) {
            b->groups.emplace_back();
            g = &b->groups.back();
            g->lat = s->lat;
            g->model = km;
            g->user_model = s->p.model;
            g->storage = s->p.storage;
            for (auto& o : old)     // reuse device tables of a group that persists
                if (o.lat == g->lat && o.model == g->model && o.storage == g->storage && o.d_desc) {
                    g->d_desc = o.d_desc;
                    g->d_block_dom = o.d_block_dom;
                    g->d_pblock_dom = o.d_pblock_dom;
                    g->d_partials = o.d_partials;
                    g->cap_desc = o.cap_desc;
                    g->cap_blocks = o.cap_blocks;
                    g->cap_pblocks = o.cap_pblocks;
                    o.d_desc = nullptr;
                }
        }
        g->ids.push_back(kv.first);
    }
    for (auto& o : old)
        if (o.d_desc) {
            cudaFreeAsync(o.d_desc, b->stream);
            cudaFreeAsync(o.d_block_dom, b->stream);
            if (o.d_pblock_dom) cudaFreeAsync(o.d_pblock_dom, b->stream);
            cudaFreeAsync(o.d_partials, b->stream);
        }
    for (auto& g : b->groups) {
        std::vector<BatchDesc> desc(g.ids.size());
        std::vector<int> bd, pbd;
        int blocks = 0, pblocks = 0;
        // plain-step tile shape of the group's size class (FP64 and the
        // Newton-implicit PR step: 256 x 1)
        int64_t cells = 0;
        for (int64_t id : g.ids) cells += b->doms[id].s->ncells;
        const int cls = batch_size_class(cells / (int64_t)g.ids.size());
        std::pair<int, int> shape = sched_tile(g.lat, g.user_model, g.storage, cls);
        if (g.storage == LBM_F64 || g.model == kModelPRImplicit) shape = {kBlock, 1};
        g.tile_threads = shape.first;
        g.tile_cpt = shape.second;
        const int tile_cells = g.tile_threads * g.tile_cpt;
        for (size_t j = 0; j < g.ids.size(); ++j) {
            Dom& d = b->doms[g.ids[j]];
            const lbm_solver* s = d.s;
            BatchDesc& D = desc[j];
            std::memset(&D, 0, sizeof(D));
            D.kp = s->kp;
            D.cf = make_coef_lat<float>(s->kp, s->lat);
            D.cd = make_coef_lat<double>(s->kp, s->lat);
            D.f[0] = s->f[0];
            D.f[1] = s->f[1];
            D.links = s->links;
            D.tau = s->tau;
            D.usnap = s->usnap;
            D.rng = (uint32_t*)(s->stats + 2 * kNumStats);
            D.parity0 = d.parity0;
            D.block_begin = blocks;
            D.nblocks = step_grid(s->ncells);
            D.slot = d.slot;
            D.pblock_begin = pblocks;
            for (int q = 0; q < D.nblocks; ++q) bd.push_back((int)j);
            blocks += D.nblocks;
            const int ptiles = (s->ncells + tile_cells - 1) / tile_cells;
            for (int q = 0; q < ptiles; ++q) pbd.push_back((int)j);
            pblocks += ptiles;
        }
        g.nblocks = blocks;
        g.pnblocks = pblocks;
        const int ctas = sched_ctas(g.lat, g.user_model, g.storage);
        g.grid = ctas > 0 ? std::min(blocks, ctas * b->sms) : blocks;
        g.pgrid = ctas > 0 ? std::min(pblocks, ctas * b->sms) : pblocks;
        if ((int)desc.size() > g.cap_desc) {
            if (g.d_desc) cudaFreeAsync(g.d_desc, b->stream);
            g.cap_desc = (int)desc.size() * 2;
            BCK(b, cudaMallocAsync((void**)&g.d_desc, sizeof(BatchDesc) * g.cap_desc, b->stream), "batch table");
        }
        if (blocks > g.cap_blocks) {
            if (g.d_block_dom) cudaFreeAsync(g.d_block_dom, b->stream);
            if (g.d_partials) cudaFreeAsync(g.d_partials, b->stream);
            g.cap_blocks = blocks * 2;
            BCK(b, cudaMallocAsync((void**)&g.d_block_dom, sizeof(int) * g.cap_blocks, b->stream), "batch block map");
            BCK(b, cudaMallocAsync((void**)&g.d_partials, sizeof(double) * kNumStats * g.cap_blocks, b->stream), "batch partials");
        }
        if (pblocks > g.cap_pblocks) {
            if (g.d_pblock_dom) cudaFreeAsync(g.d_pblock_dom, b->stream);
            g.cap_pblocks = pblocks * 2;
            BCK(b, cudaMallocAsync((void**)&g.d_pblock_dom, sizeof(int) * g.cap_pblocks, b->stream), "batch tile map");
        }
        BCK(b, cudaMemcpyAsync(g.d_desc, desc.data(), sizeof(BatchDesc) * desc.size(), cudaMemcpyHostToDevice, b->stream), "batch table upload");
        BCK(b, cudaMemcpyAsync(g.d_block_dom, bd.data(), sizeof(int) * bd.size(), cudaMemcpyHostToDevice, b->stream), "batch block map upload");
        BCK(b, cudaMemcpyAsync(g.d_pblock_dom, pbd.data(), sizeof(int) * pbd.size(), cudaMemcpyHostToDevice, b->stream), "batch tile map upload");
        // pageable sources: make sure the copies are done before the vectors go
        BCK(b, cudaStreamSynchronize(b->stream), "batch table sync");
    }
    b->dirty = false;
    return LBM_OK;
}

cudaError_t launch_group(lbm_batch* b, const Group& g, bool check, int phase, cudaStream_t st) {
    cudaError_t e = check ? launch_batch(g.lat, g.model, g.storage, true, g.d_desc, g.d_block_dom,
                                         g.nblocks, g.grid, phase, g.d_partials, kBlock, 1, st)
                          : launch_batch(g.lat, g.model, g.storage, false, g.d_desc,
                                         g.d_pblock_dom, g.pnblocks, g.pgrid, phase, nullptr,
                                         g.tile_threads, g.tile_cpt, st);
    if (e != cudaSuccess || !check) return e;
    k_finalize_domains<<<(int)g.ids.size(), kBlock, 0, st>>>(g.d_desc, g.d_partials, b->d_slots);
    return cudaGetLastError();
}

cudaError_t launch_all(lbm_batch* b, bool check, cudaStream_t st) {
    for (auto& g : b->groups) {
        if (g.ids.empty()) continue;
        cudaError_t e = launch_group(b, g, check, b->phase, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Graph body with one branch per group: the groups touch disjoint memory, so
// their step chains need no order between them.  Every forked branch is
// joined back into the origin stream, also after an error, so the capture
// can always be ended.
cudaError_t capture_branches(lbm_batch* b, int par, int active) {
    cudaError_t e = cudaSuccess;
    if (!b->fork) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    while (e == cudaSuccess && (int)b->branch.size() < active) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->branch.push_back(st);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->join.push_back(ev);
    }
    if (e != cudaSuccess) return e;     // nothing forked yet
    e = cudaEventRecord(b->fork, b->cap);
    if (e != cudaSuccess) return e;
    int k = 0;
    for (const auto& g : b->groups) {
        if (g.ids.empty()) continue;
        cudaStream_t st = b->branch[k];
        cudaError_t eb = cudaStreamWaitEvent(st, b->fork, 0);
        for (int t = 0; t < kGraphLen && eb == cudaSuccess; ++t)
            eb = launch_group(b, g, false, par ^ (t & 1), st);
        cudaError_t ej = cudaEventRecord(b->join[k], st);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(b->cap, b->join[k], 0);
        if (e == cudaSuccess) e = eb != cudaSuccess ? eb : ej;
        ++k;
    }
    return e;
}

cudaError_t capture(lbm_batch* b, int par) {
    if (!b->cap) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    const int saved = b->phase;
    b->phase = par;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        b->phase = saved;
        return e;
    }
    int active = 0;
    for (const auto& g : b->groups) active += !g.ids.empty();
    if (b->concurrent && active > 1) {
        e = capture_branches(b, par, active);
    } else {
        for (int t = 0; t < kGraphLen && e == cudaSuccess; ++t) {
            e = launch_all(b, false, b->cap);
            b->phase ^= 1;
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    b->phase = saved;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    if (e2 != cudaSuccess) return e2;
    e = cudaGraphInstantiate(&b->graph[par], g, 0);
    cudaGraphDestroy(g);
    return e;
}

void sync_solvers(lbm_batch* b, int64_t nsteps) {
    for (auto& kv : b->doms) {
        lbm_solver* s = kv.second.s;
        s->cur = b->phase ^ kv.second.parity0;
        s->steps += nsteps;
    }
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(lbm_batch** out, size_t budget, int32_t check_every, void* stream) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (check_every < 1) return fail(LBM_EINVAL, "check_every must be >= 1");
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return fail(LBM_ENOMEM, "host allocation failed");
    b->budget = budget;
    b->k = check_every;
    b->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_slots, sizeof(double) * kNumStats * kMaxSlots);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_slots, sizeof(double) * kNumStats * kMaxSlots);
    if (e == cudaSuccess) e = cudaMemset(b->d_slots, 0, sizeof(double) * kNumStats * kMaxSlots);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lbm_batch_destroy(b);
        return fail(LBM_ECUDA, "batch creation: %s", cudaGetErrorString(e));
    }
    std::memset(b->h_slots, 0, sizeof(double) * kNumStats * kMaxSlots);
    for (int i = kMaxSlots - 1; i >= 0; --i) b->free_slots.push_back(i);
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_add(lbm_batch* b, lbm_lattice lat, int nx, int ny, int nz,
                         const uint8_t* mask, const lbm_params* p, int64_t* id) {
    lbm_status v = benter(b);
    if (v != LBM_OK) return v;
    if (!p || !id) return fail(LBM_EINVAL, "NULL argument");
    if (p->flags & LBM_FLAG_COMPACT)
        return fail(LBM_EINVAL, "batch domains use the dense layout (LBM_FLAG_COMPACT set)");
    if (b->free_slots.empty()) return fail(LBM_EBUSY, "the batch holds %d domains already", kMaxSlots);
    lbm_params q = *p;
    q.check_every = b->k;
    size_t bytes = 0;
    if ((v = lbm_workspace_bytes(lat, nx, ny, nz, &q, &bytes)) != LBM_OK) return v;
    const int Q = lattice_q(lat);
    const int64_t plane = ((int64_t)nx * ny * nz + 63) / 64 * 64;
    if ((int64_t)Q * plane >= (int64_t)0x7fffffff)
        return fail(LBM_EINVAL, "domain too large for a batch (Q * cells >= 2^31)");
    if (b->used + bytes > b->budget)
        return fail(LBM_EBUSY, "budget: %zu bytes in use, %zu more requested, budget %zu", b->used, bytes, b->budget);
    void* ws = nullptr;
    BCK(b, cudaMallocAsync(&ws, bytes, b->stream), "domain allocation");
    lbm_solver* s = nullptr;
    v = lbm_create_with_workspace(&s, lat, nx, ny, nz, mask, &q, b->stream, ws, bytes);
    if (v != LBM_OK) {
        cudaFreeAsync(ws, b->stream);
        return v;
    }
    Dom d;
    d.s = s;
    d.ws = ws;
    d.bytes = bytes;
    d.parity0 = b->phase ^ s->cur;
    d.slot = b->free_slots.back();
    // a reused row holds its last occupant's stats: the first check step of
    // this domain must find it empty
    if (cudaMemsetAsync(b->d_slots + (int64_t)d.slot * kNumStats, 0, kNumStats * sizeof(double),
                        b->stream) != cudaSuccess) {
        lbm_destroy(s);
        cudaFreeAsync(ws, b->stream);
        return bfail(b, cudaGetLastError(), "stats row reset");
    }
    std::memset(b->h_slots + (int64_t)d.slot * kNumStats, 0, kNumStats * sizeof(double));
    b->free_slots.pop_back();
    *id = b->next_id++;
    b->doms[*id] = d;
    b->used += bytes;
    b->dirty = true;
    return LBM_OK;
}

lbm_status lbm_batch_remove(lbm_batch* b, int64_t id) {
    lbm_status v = benter(b);
    if (v != LBM_OK) return v;
    auto it = b->doms.find(id);
    if (it == b->doms.end()) return fail(LBM_EINVAL, "unknown domain %lld", (long long)id);
    BWAIT(b, "lbm_batch_remove");
    lbm_destroy(it->second.s);
    BCK(b, cudaFreeAsync(it->second.ws, b->stream), "domain release");
    b->used -= it->second.bytes;
    b->free_slots.push_back(it->second.slot);
    b->doms.erase(it);
    b->dirty = true;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps) {
    lbm_status v = benter(b);
    if (v != LBM_OK) return v;
    if (nsteps < 0) return fail(LBM_EINVAL, "nsteps must be >= 0");
    if (b->doms.empty() || nsteps == 0) {
        b->gstep += nsteps;
        return LBM_OK;
    }
    if (b->sched_version != g_sched_version.load()) b->dirty = true;
    if (b->dirty && (v = rebuild(b)) != LBM_OK) return v;
    int64_t left = nsteps;
    while (left > 0) {
        const int64_t to_check = b->k - (b->gstep % b->k);
        int64_t plain = std::min(to_check - 1, left);
        while (plain >= kGraphLen) {
            if (!b->graph[b->phase]) BCK(b, capture(b, b->phase), "batch graph capture");
            BCK(b, cudaGraphLaunch(b->graph[b->phase], b->stream), "batch graph launch");
            b->gstep += kGraphLen;          // even: the phase is unchanged
            plain -= kGraphLen;
            left -= kGraphLen;
        }
        while (plain > 0) {
            BCK(b, launch_all(b, false, b->stream), "batch step");
            b->phase ^= 1;
            b->gstep += 1;
            --plain;
            --left;
        }
        if (left > 0) {
            BCK(b, launch_all(b, true, b->stream), "batch check step");
            b->phase ^= 1;
            b->gstep += 1;
            --left;
            BCK(b, cudaMemcpyAsync(b->h_slots, b->d_slots, sizeof(double) * kNumStats * kMaxSlots,
                                   cudaMemcpyDeviceToHost, b->stream), "batch stats copy");
            for (auto& kv : b->doms) kv.second.checks += 1;
        }
    }
    sync_solvers(b, nsteps);
    return LBM_OK;
}

lbm_status lbm_batch_domain_status(lbm_batch* b, int64_t id, lbm_domain_status* st) {
    lbm_status v = benter(b);
    if (v != LBM_OK) return v;
    auto it = b->doms.find(id);
    if (it == b->doms.end() || !st) return fail(LBM_EINVAL, "unknown domain %lld", (long long)id);
    BWAIT(b, "lbm_batch_domain_status");
    const Dom& d = it->second;
    const double* r = b->h_slots + (int64_t)d.slot * kNumStats;
    std::memset(st, 0, sizeof(*st));
    st->steps = d.s->steps;
    st->checks = d.checks;
    const int len[3] = {d.s->nx, d.s->ny, d.s->nz};
    for (int a = 0; a < 3; ++a) st->flow[a] = d.checks > 0 ? r[kStatUx + a] / len[a] : 0.0;
    st->residual = (d.checks >= 2 && r[kStatU2] > 0.0) ? std::sqrt(r[kStatDu2] / r[kStatU2]) : -1.0;
    st->nonfinite = (d.checks > 0 && r[kStatNonFinite] != 0.0) ? 1 : 0;
    st->flow_change = d.checks >= 2 ? r[kStatFlowChange] : -1.0;
    return LBM_OK;
}

lbm_status lbm_batch_solver(lbm_batch* b, int64_t id, lbm_solver** s) {
    if (!b || !s) return fail(LBM_EINVAL, "NULL argument");
    auto it = b->doms.find(id);
    if (it == b->doms.end()) return fail(LBM_EINVAL, "unknown domain %lld", (long long)id);
    *s = it->second.s;
    return LBM_OK;
}

lbm_status lbm_batch_usage(const lbm_batch* b, size_t* bytes, int64_t* domains, int64_t* cells) {
    if (!b) return fail(LBM_EINVAL, "batch is NULL");
    if (bytes) *bytes = b->used;
    if (domains) *domains = (int64_t)b->doms.size();
    if (cells) {
        int64_t c = 0;
        for (auto& kv : b->doms) c += kv.second.s->nfluid;
        *cells = c;
    }
    return LBM_OK;
}

lbm_status lbm_tuning_set_batch(lbm_lattice lat, int32_t model, int32_t storage,
                                 int32_t ctas_per_sm) {
    if (lattice_q(lat) == 0) return fail(LBM_EINVAL, "unknown lattice %d", lat);
    if (model != LBM_MODEL_PR && model != LBM_MODEL_IR) return fail(LBM_EINVAL, "unknown model %d", model);
    if (storage_bytes(storage) == 0) return fail(LBM_EINVAL, "unknown storage %d", storage);
    if (ctas_per_sm < 0 || ctas_per_sm > 32) return fail(LBM_EINVAL, "ctas_per_sm must be in 0..32");
    {
        std::lock_guard<std::mutex> lk(g_sched_mu);
        g_sched_ctas[sched_key(lat, model, storage)] = ctas_per_sm;
    }
    g_sched_version.fetch_add(1);
    return LBM_OK;
}

lbm_status lbm_tuning_get_batch(lbm_lattice lat, int32_t model, int32_t storage,
                                 int32_t* ctas_per_sm) {
    if (!ctas_per_sm) return fail(LBM_EINVAL, "ctas_per_sm is NULL");
    if (lattice_q(lat) == 0) return fail(LBM_EINVAL, "unknown lattice %d", lat);
    if (model != LBM_MODEL_PR && model != LBM_MODEL_IR) return fail(LBM_EINVAL, "unknown model %d", model);
    if (storage_bytes(storage) == 0) return fail(LBM_EINVAL, "unknown storage %d", storage);
    *ctas_per_sm = sched_ctas(lat, model, storage);
    return LBM_OK;
}

lbm_status lbm_tuning_set_batch_tile(lbm_lattice lat, int32_t model, int32_t storage,
                                     int32_t size_class, int32_t threads, int32_t cells_per_thread) {
    if (lattice_q(lat) == 0) return fail(LBM_EINVAL, "unknown lattice %d", lat);
    if (model != LBM_MODEL_PR && model != LBM_MODEL_IR) return fail(LBM_EINVAL, "unknown model %d", model);
    if (storage_bytes(storage) == 0) return fail(LBM_EINVAL, "unknown storage %d", storage);
    if (size_class < 0 || size_class > 62) return fail(LBM_EINVAL, "size_class must be in 0..62");
    if (!valid_tile(threads, cells_per_thread))
        return fail(LBM_EINVAL, "tile shape %d x %d is not one of 128/256/512 x 1, 128/256 x 2",
                    threads, cells_per_thread);
    if (storage == LBM_F64 && !(threads == kBlock && cells_per_thread == 1))
        return fail(LBM_EINVAL, "FP64 storage runs 256 x 1 tiles only");
    {
        std::lock_guard<std::mutex> lk(g_sched_mu);
        g_sched_tile[sched_key(lat, model, storage)][size_class] = {threads, cells_per_thread};
    }
    g_sched_version.fetch_add(1);
    return LBM_OK;
}

lbm_status lbm_tuning_get_batch_tile(lbm_lattice lat, int32_t model, int32_t storage,
                                     int64_t mean_cells, int32_t* threads,
                                     int32_t* cells_per_thread, int32_t* size_class) {
    if (lattice_q(lat) == 0) return fail(LBM_EINVAL, "unknown lattice %d", lat);
    if (model != LBM_MODEL_PR && model != LBM_MODEL_IR) return fail(LBM_EINVAL, "unknown model %d", model);
    if (storage_bytes(storage) == 0) return fail(LBM_EINVAL, "unknown storage %d", storage);
    if (mean_cells < 1) return fail(LBM_EINVAL, "mean_cells must be >= 1");
    const int cls = batch_size_class(mean_cells);
    const std::pair<int, int> t = sched_tile(lat, model, storage, cls);
    if (threads) *threads = t.first;
    if (cells_per_thread) *cells_per_thread = t.second;
    if (size_class) *size_class = cls;
    return LBM_OK;
}

lbm_status lbm_tuning_set_batch_concurrency(int32_t concurrent) {
    if (concurrent != 0 && concurrent != 1) return fail(LBM_EINVAL, "concurrent must be 0 or 1");
    g_sched_concurrent.store(concurrent);
    g_sched_version.fetch_add(1);
    return LBM_OK;
}

lbm_status lbm_tuning_get_batch_concurrency(int32_t* concurrent) {
    if (!concurrent) return fail(LBM_EINVAL, "concurrent is NULL");
    *concurrent = g_sched_concurrent.load();
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev != b->device) cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (auto& kv : b->doms) {
        lbm_destroy(kv.second.s);
        cudaFreeAsync(kv.second.ws, b->stream);
    }
    for (auto& g : b->groups) {
        if (g.d_desc) cudaFreeAsync(g.d_desc, b->stream);
        if (g.d_block_dom) cudaFreeAsync(g.d_block_dom, b->stream);
        if (g.d_pblock_dom) cudaFreeAsync(g.d_pblock_dom, b->stream);
        if (g.d_partials) cudaFreeAsync(g.d_partials, b->stream);
    }
    cudaStreamSynchronize(b->stream);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t st : b->branch) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->d_slots) cudaFree(b->d_slots);
    if (b->h_slots) cudaFreeHost(b->h_slots);
    cudaGetLastError();
    delete b;
}

}  // extern "C"

// ===========================================================================
// serving

namespace {

struct Req {
    lbm_request r{};
    std::vector<uint8_t> mask;
    lbm_result res{};
    int64_t dom = 0;
    size_t bytes = 0;
    std::vector<double> fields;   // rho, ux, uy, uz of the final state (keep_fields)
};

}  // namespace

struct lbm_server {
    lbm_batch* batch = nullptr;
    size_t budget = 0;
    int k = 0;
    double t0 = 0.0;
    int64_t next_id = 1;
    std::map<int64_t, Req> reqs;
    std::deque<int64_t> queue;
    std::vector<int64_t> running;
};

extern "C" {

lbm_status lbm_server_create(lbm_server** out, size_t budget, int32_t check_every, void* stream) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_server* s = new (std::nothrow) lbm_server();
    if (!s) return fail(LBM_ENOMEM, "host allocation failed");
    lbm_status v = lbm_batch_create(&s->batch, budget, check_every, stream);
    if (v != LBM_OK) {
        delete s;
        return v;
    }
    s->budget = budget;
    s->k = check_every;
    s->t0 = now_s();
    *out = s;
    return LBM_OK;
}

lbm_status lbm_server_now(const lbm_server* s, double* t) {
    if (!s || !t) return fail(LBM_EINVAL, "NULL argument");
    *t = now_s() - s->t0;
    return LBM_OK;
}

lbm_status lbm_server_submit(lbm_server* s, const lbm_request* req, int64_t* id) {
    if (!s || !req || !id) return fail(LBM_EINVAL, "NULL argument");
    if (req->max_steps < 1) return fail(LBM_EINVAL, "max_steps must be >= 1");
    if (!(req->tolerance > 0.0)) return fail(LBM_EINVAL, "tolerance must be > 0");
    if (req->criterion != LBM_STEADY_FLOW && req->criterion != LBM_STEADY_RESIDUAL)
        return fail(LBM_EINVAL, "unknown steady-state criterion %d", req->criterion);
    if (req->nx < 1 || req->ny < 1 || req->nz < 1 || !req->solid_mask)
        return fail(LBM_EINVAL, "bad extents or mask");
    if (req->params.flags & (LBM_FLAG_COMPACT | LBM_FLAG_Z_GHOSTS))
        return fail(LBM_EINVAL, "served domains are whole domains in the dense layout (flags 0x%x)",
                    req->params.flags);
    lbm_params q = req->params;
    q.check_every = s->k;
    size_t bytes = 0;
    lbm_status v = lbm_workspace_bytes((lbm_lattice)req->lattice, req->nx, req->ny, req->nz, &q, &bytes);
    if (v != LBM_OK) return v;
    if (bytes > s->budget) return fail(LBM_EINVAL, "request needs %zu bytes, budget is %zu", bytes, s->budget);
    Req r;
    r.r = *req;
    const size_t n = (size_t)req->nx * req->ny * req->nz;
    r.mask.assign(req->solid_mask, req->solid_mask + n);
    r.r.solid_mask = nullptr;
    r.bytes = bytes;
    r.res.state = LBM_REQ_QUEUED;
    r.res.t_submit = now_s() - s->t0;
    *id = s->next_id++;
    s->reqs[*id] = std::move(r);
    s->queue.push_back(*id);
    return LBM_OK;
}

static lbm_status retire(lbm_server* s, int64_t rid, int state) {
    Req& r = s->reqs[rid];
    lbm_solver* sol = nullptr;
    lbm_status v = lbm_batch_solver(s->batch, r.dom, &sol);
    if (v != LBM_OK) return v;
    lbm_domain_status ds;
    if ((v = lbm_batch_domain_status(s->batch, r.dom, &ds)) != LBM_OK) return v;
    r.res.steps = ds.steps;
    r.res.residual = ds.residual;
    if ((v = lbm_flowrate(sol, 0, &r.res.flow_x)) != LBM_OK) return v;
    if (r.r.keep_fields) {
        const size_t n = (size_t)sol->ncells;
        r.fields.resize(4 * n);
        if ((v = lbm_fields(sol, r.fields.data(), r.fields.data() + n, r.fields.data() + 2 * n,
                            r.fields.data() + 3 * n)) != LBM_OK)
            return v;
    }
    if ((v = lbm_batch_remove(s->batch, r.dom)) != LBM_OK) return v;
    r.res.state = state;
    r.res.t_done = now_s() - s->t0;
    return LBM_OK;
}

lbm_status lbm_server_advance(lbm_server* s, int64_t nsteps, int32_t* completed) {
    if (!s) return fail(LBM_EINVAL, "server is NULL");
    if (nsteps < 1 || nsteps % s->k != 0) return fail(LBM_EINVAL, "nsteps must be a positive multiple of check_every");
    int32_t done = 0;
    // admission: submission order, smaller later requests may pass a blocked one
    size_t used = 0;
    lbm_batch_usage(s->batch, &used, nullptr, nullptr);
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Req& r = s->reqs[*it];
        if (used + r.bytes > s->budget) {
            ++it;
            continue;
        }
        int64_t dom = 0;
        lbm_status v = lbm_batch_add(s->batch, (lbm_lattice)r.r.lattice, r.r.nx, r.r.ny, r.r.nz,
                                     r.mask.data(), &r.r.params, &dom);
        if (v == LBM_EBUSY) {
            ++it;
            continue;
        }
        if (v != LBM_OK) {   // malformed parameters: fail this request only
            r.res.state = LBM_REQ_FAILED;
            r.res.t_done = now_s() - s->t0;
            it = s->queue.erase(it);
            ++done;
            continue;
        }
        lbm_solver* sol = nullptr;
        lbm_batch_solver(s->batch, dom, &sol);
        r.dom = dom;
        r.res.fluid_cells = sol->nfluid;
        r.res.state = LBM_REQ_RUNNING;
        r.res.t_admit = now_s() - s->t0;
        used += r.bytes;
        s->running.push_back(*it);
        it = s->queue.erase(it);
    }
    if (s->running.empty()) {
        if (completed) *completed = done;
        return LBM_OK;
    }
    lbm_status v = lbm_batch_step(s->batch, nsteps);
    if (v != LBM_OK) return v;
    std::vector<int64_t> still;
    for (int64_t rid : s->running) {
        Req& r = s->reqs[rid];
        lbm_domain_status ds;
        if ((v = lbm_batch_domain_status(s->batch, r.dom, &ds)) != LBM_OK) return v;
        int state = -1;
        // the change between the last two check steps (check_every apart)
        const double change = r.r.criterion == LBM_STEADY_RESIDUAL ? ds.residual : ds.flow_change;
        const bool steady = change >= 0.0 && change < r.r.tolerance;
        if (ds.nonfinite) state = LBM_REQ_FAILED;
        else if (steady) state = LBM_REQ_CONVERGED;
        else if (ds.steps >= r.r.max_steps) state = LBM_REQ_CAPPED;
        if (state >= 0) {
            if ((v = retire(s, rid, state)) != LBM_OK) return v;
            ++done;
        } else {
            still.push_back(rid);
        }
    }
    s->running.swap(still);
    if (completed) *completed = done;
    return LBM_OK;
}

lbm_status lbm_server_result(const lbm_server* s, int64_t id, lbm_result* res) {
    if (!s || !res) return fail(LBM_EINVAL, "NULL argument");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(LBM_EINVAL, "unknown request %lld", (long long)id);
    *res = it->second.res;
    return LBM_OK;
}

lbm_status lbm_server_fields(const lbm_server* s, int64_t id, double* rho, double* ux, double* uy,
                             double* uz) {
    if (!s) return fail(LBM_EINVAL, "server is NULL");
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(LBM_EINVAL, "unknown request %lld", (long long)id);
    const Req& r = it->second;
    if (r.fields.empty()) return fail(LBM_EINVAL, "request %lld has no kept fields", (long long)id);
    const size_t n = r.fields.size() / 4;
    double* out[4] = {rho, ux, uy, uz};
    for (int k = 0; k < 4; ++k)
        if (out[k]) std::memcpy(out[k], r.fields.data() + k * n, n * sizeof(double));
    return LBM_OK;
}

lbm_status lbm_server_pending(const lbm_server* s, int64_t* queued, int64_t* running, size_t* used) {
    if (!s) return fail(LBM_EINVAL, "server is NULL");
    if (queued) *queued = (int64_t)s->queue.size();
    if (running) *running = (int64_t)s->running.size();
    if (used) lbm_batch_usage(s->batch, used, nullptr, nullptr);
    return LBM_OK;
}

void lbm_server_destroy(lbm_server* s) {
    if (!s) return;
    lbm_batch_destroy(s->batch);
    delete s;
}

}  // extern "C"
