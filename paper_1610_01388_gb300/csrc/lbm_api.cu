// Host implementation of the C ABI declared in include/bingham_lbm.h.
//
// Device memory of one solver (one allocation or one caller workspace, each
// region 256-byte aligned):
//   f[2]      population offsets f_i - w_i, SoA [Q][plane], A/B buffers
//   links     per-cell bounce-back bits (bit i: cell at x - c_i is solid;
//             bit 31: the cell itself is solid)
// With LBM_FLAG_COMPACT, f, links, tau and usnap hold the fluid cells only
// (one slot each, in cell-index order; plane >= the fluid count), and two
// more regions map between slots and cells:
//   cellidx   cell index of each slot
//   rank      slot of each cell, -1 for a solid cell
//   tau       PR relaxation time per cell, updated in place
//   usnap     check-step velocity snapshot [3][plane]
//   partials  per-block FP64 reduction partials
//   stats     finalised reduction results, then two u32 launch counters
//             (stochastic rounding of the 16-bit storage forms)
//   mask      the uploaded solid mask (bytes)
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/bingham_lbm.h"
#include "lbm_internal.h"
#include "solver.h"

using namespace blbm;

namespace blbm {

thread_local std::string g_err;

lbm_status fail(lbm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

int lattice_q(int lat) {
    switch (lat) {
    case LBM_D2Q9: return 9;
    case LBM_D3Q15: return 15;
    case LBM_D3Q19: return 19;
    case LBM_D3Q27: return 27;
    default: return 0;
    }
}

size_t storage_bytes(int storage) {
    switch (storage) {
    case LBM_F64: return 8;
    case LBM_F32: return 4;
    case LBM_F16_OFS:
    case LBM_BF16_OFS: return 2;
    default: return 0;
    }
}

size_t arith_bytes(int storage) { return storage == LBM_F64 ? 8 : 4; }

bool storage_built(int storage) { return storage_bytes(storage) != 0; }

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// held: the cells the planes hold (every cell; the fluid cells in the
// compact layout)
Layout make_layout(int lat, int nx, int ny, int nz, const lbm_params& p, int64_t held) {
    Layout L{};
    const int64_t ncells = (int64_t)nx * ny * nz;
    const bool compact = (p.flags & LBM_FLAG_COMPACT) != 0;
    if (!compact) held = ncells;
    L.plane = (held + 63) / 64 * 64;
    const int Q = lattice_q(lat);
    const size_t fb = align256((size_t)Q * L.plane * storage_bytes(p.storage));
    const size_t rs = arith_bytes(p.storage);
    size_t o = 0;
    L.off_f[0] = o; o += fb;
    L.off_f[1] = o; o += fb;
    L.off_links = o; o += align256((size_t)L.plane * 4);
    L.off_tau = o; o += (p.model == LBM_MODEL_PR) ? align256((size_t)L.plane * rs) : 0;
    L.off_usnap = o; o += (p.check_every > 0) ? align256((size_t)3 * L.plane * rs) : 0;
    const int g1 = step_grid((int)held), g2 = reduce_grid((int)held);
    L.nparts = g1 > g2 ? g1 : g2;
    L.off_partials = o; o += align256((size_t)L.nparts * kNumStats * sizeof(double));
    L.off_stats = o; o += align256(2 * kNumStats * sizeof(double));
    L.off_mask = o; o += align256((size_t)ncells);
    L.off_cellidx = o; o += compact ? align256((size_t)L.plane * 4) : 0;
    L.off_rank = o; o += compact ? align256((size_t)ncells * 4) : 0;
    L.total = o;
    return L;
}

// cells the step kernels update: all of them (dense) or the slots (compact)
int held_cells(const lbm_solver* s) { return s->rank ? s->kp.nslots : s->ncells; }

lbm_status validate(int lat, int nx, int ny, int nz, const uint8_t* mask, const lbm_params* p) {
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    if (lattice_q(lat) == 0) return fail(LBM_EINVAL, "unknown lattice %d", lat);
    if (nx < 1 || ny < 1 || nz < 1) return fail(LBM_EINVAL, "extents must be >= 1 (got %d,%d,%d)", nx, ny, nz);
    if (lat == LBM_D2Q9 && nz != 1) return fail(LBM_EINVAL, "D2Q9 needs nz == 1 (got %d)", nz);
    const int64_t n = (int64_t)nx * ny * nz;
    if (n > (int64_t)0x7fffffff - 64) return fail(LBM_EINVAL, "too many cells (%lld)", (long long)n);
    if (p->model != LBM_MODEL_PR && p->model != LBM_MODEL_IR) return fail(LBM_EINVAL, "unknown model %d", p->model);
    if (storage_bytes(p->storage) == 0) return fail(LBM_EINVAL, "unknown storage %d", p->storage);
    if (!storage_built(p->storage)) return fail(LBM_EUNSUPPORTED, "storage %d is not built into this library", p->storage);
    if (!(p->mu_p > 0.0) || !std::isfinite(p->mu_p)) return fail(LBM_EINVAL, "mu_p must be > 0");
    if (!(p->sigma_y >= 0.0) || !std::isfinite(p->sigma_y)) return fail(LBM_EINVAL, "sigma_y must be >= 0");
    if (p->model == LBM_MODEL_PR) {
        if (!(p->m >= 0.0) || !std::isfinite(p->m)) return fail(LBM_EINVAL, "m must be >= 0");
        if (!(p->gammadot_c > 0.0) || !std::isfinite(p->gammadot_c)) return fail(LBM_EINVAL, "gammadot_c must be > 0");
        if (!(p->magic > 0.0) || !std::isfinite(p->magic)) return fail(LBM_EINVAL, "magic must be > 0");
    }
    for (int d = 0; d < 3; ++d)
        if (!std::isfinite(p->g[d])) return fail(LBM_EINVAL, "g must be finite");
    if (lat == LBM_D2Q9 && p->g[2] != 0.0) return fail(LBM_EINVAL, "D2Q9 needs g[2] == 0");
    if (p->check_every < 0) return fail(LBM_EINVAL, "check_every must be >= 0");
    if (p->flags & ~(LBM_FLAG_BURNETT_X | LBM_FLAG_Z_GHOSTS | LBM_FLAG_COMPACT))
        return fail(LBM_EINVAL, "unknown flags 0x%x", p->flags);
    if ((p->flags & LBM_FLAG_Z_GHOSTS) && (lat == LBM_D2Q9 || nz < 3))
        return fail(LBM_EINVAL, "ghost planes need a 3D lattice and nz >= 3 (got nz = %d)", nz);
    if ((p->flags & LBM_FLAG_Z_GHOSTS) && (p->flags & LBM_FLAG_COMPACT))
        return fail(LBM_EINVAL, "ghost planes need the dense layout (LBM_FLAG_COMPACT set)");
    if (p->newton_iters < 0 || p->newton_iters > 64)
        return fail(LBM_EINVAL, "newton_iters must be in 0..64 (got %d)", p->newton_iters);
    if (p->reserved != 0) return fail(LBM_EINVAL, "reserved must be 0");
    if (!mask) return fail(LBM_EINVAL, "solid_mask is NULL");
    int64_t fluid = 0;
    const int64_t plane = (int64_t)nx * ny;
    const bool ghosts = (p->flags & LBM_FLAG_Z_GHOSTS) != 0;
    for (int64_t i = ghosts ? plane : 0; i < (ghosts ? n - plane : n); ++i) fluid += mask[i] == 0;
    if (fluid == 0) return fail(LBM_EINVAL, "the mask has no fluid cell");
    return LBM_OK;
}

}  // namespace blbm

namespace {

lbm_status cuda_fail(lbm_solver* s, cudaError_t e, const char* what) {
    if (s) s->poisoned = true;
    cudaGetLastError();
    return fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(s, expr, what)                                  \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, what); \
    } while (0)

// Bounded wait for the solver's queued work: LBM_ETIMEOUT (handle still
// usable, nothing written) when the wait limit runs out.
#define WAIT(s, what)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = bounded_sync((s)->stream);                                         \
        if (e_ == cudaErrorNotReady)                                                        \
            return fail(LBM_ETIMEOUT, "%s: queued work still running after the %g s wait limit", \
                        what, wait_limit());                                                \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, what);                               \
    } while (0)

lbm_status enter(const lbm_solver* s) {
    if (!s) return fail(LBM_EINVAL, "solver is NULL");
    if (s->poisoned) return fail(LBM_ECUDA, "solver is in an error state after a CUDA failure");
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev != s->device) cudaSetDevice(s->device);
    return LBM_OK;
}

cudaError_t launch_step(lbm_solver* s, bool check, cudaStream_t st) {
    StepArgs a;
    a.fsrc = s->f[s->cur];
    a.fdst = s->f[s->cur ^ 1];
    a.links = s->links;
    a.tau = s->tau;
    a.usnap = s->usnap;
    a.partials = s->partials;
    a.rng_ctr = (uint32_t*)(s->stats + 2 * kNumStats);
    a.parity = s->cur;
    a.block = s->block;
    a.cpt = s->cpt;
    a.copy = s->copy;
    a.cellidx = s->cellidx;
    a.rank = s->rank;
    const int km = kernel_model(s->p.model, s->kp.newton);
    switch (s->lat) {
    case LBM_D2Q9: return launch_step_D2Q9(km, s->p.storage, check, s->kp, a, st);
    case LBM_D3Q15: return launch_step_D3Q15(km, s->p.storage, check, s->kp, a, st);
    case LBM_D3Q19: return launch_step_D3Q19(km, s->p.storage, check, s->kp, a, st);
    default: return launch_step_D3Q27(km, s->p.storage, check, s->kp, a, st);
    }
}

cudaError_t launch_links(lbm_solver* s, const uint8_t* mask) {
    switch (s->lat) {
    case LBM_D2Q9: return launch_links_D2Q9(s->kp, mask, s->links, s->cellidx, s->stream);
    case LBM_D3Q15: return launch_links_D3Q15(s->kp, mask, s->links, s->cellidx, s->stream);
    case LBM_D3Q19: return launch_links_D3Q19(s->kp, mask, s->links, s->cellidx, s->stream);
    default: return launch_links_D3Q27(s->kp, mask, s->links, s->cellidx, s->stream);
    }
}

cudaError_t launch_fields(lbm_solver* s, double* rho, double* ux, double* uy, double* uz) {
    const void* f = s->f[s->cur];
    switch (s->lat) {
    case LBM_D2Q9: return launch_fields_D2Q9(s->p.storage, s->kp, f, s->links, s->rank, rho, ux, uy, uz, s->stream);
    case LBM_D3Q15: return launch_fields_D3Q15(s->p.storage, s->kp, f, s->links, s->rank, rho, ux, uy, uz, s->stream);
    case LBM_D3Q19: return launch_fields_D3Q19(s->p.storage, s->kp, f, s->links, s->rank, rho, ux, uy, uz, s->stream);
    default: return launch_fields_D3Q27(s->p.storage, s->kp, f, s->links, s->rank, rho, ux, uy, uz, s->stream);
    }
}

cudaError_t launch_reduce(lbm_solver* s, int mode, int nblocks) {
    const void* f = s->f[s->cur];
    switch (s->lat) {
    case LBM_D2Q9: return launch_reduce_D2Q9(s->p.storage, mode, s->kp, f, s->links, s->cellidx, s->rank, s->partials, nblocks, s->stream);
    case LBM_D3Q15: return launch_reduce_D3Q15(s->p.storage, mode, s->kp, f, s->links, s->cellidx, s->rank, s->partials, nblocks, s->stream);
    case LBM_D3Q19: return launch_reduce_D3Q19(s->p.storage, mode, s->kp, f, s->links, s->cellidx, s->rank, s->partials, nblocks, s->stream);
    default: return launch_reduce_D3Q27(s->p.storage, mode, s->kp, f, s->links, s->cellidx, s->rank, s->partials, nblocks, s->stream);
    }
}

cudaError_t launch_convert(lbm_solver* s, bool to_device, int q, double* buf, int which) {
    void* f = s->f[which];
    switch (s->lat) {
    case LBM_D2Q9: return launch_convert_D2Q9(s->p.storage, to_device, s->kp, q, f, buf, s->rank, s->stream);
    case LBM_D3Q15: return launch_convert_D3Q15(s->p.storage, to_device, s->kp, q, f, buf, s->rank, s->stream);
    case LBM_D3Q19: return launch_convert_D3Q19(s->p.storage, to_device, s->kp, q, f, buf, s->rank, s->stream);
    default: return launch_convert_D3Q27(s->p.storage, to_device, s->kp, q, f, buf, s->rank, s->stream);
    }
}

lbm_status ensure_scratch(lbm_solver* s) {
    if (s->scratch) return LBM_OK;
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)4 * s->ncells * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail(LBM_ENOMEM, "cannot allocate %zu bytes of field scratch",
                    (size_t)4 * s->ncells * sizeof(double));
    }
    s->scratch = (double*)p;
    return LBM_OK;
}

// one ordinary step or check step on stream st
cudaError_t do_step(lbm_solver* s, bool check, cudaStream_t st) {
    cudaError_t e = launch_step(s, check, st);
    if (e != cudaSuccess) return e;
    s->cur ^= 1;
    s->steps += 1;
    if (check) {
        e = launch_finalize(s->partials, step_grid(held_cells(s)), s->stats, st);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(s->host_stats, s->stats, kNumStats * sizeof(double),
                            cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return e;
        s->checks += 1;
        s->last_check = s->steps;
    }
    return cudaSuccess;
}

// graph of graph_len plain steps starting from buffer parity `par`
cudaError_t build_graph(lbm_solver* s, int par) {
    if (!s->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    const int saved_cur = s->cur;
    const int64_t saved_steps = s->steps;
    s->cur = par;
    cudaError_t e = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < s->graph_len && e == cudaSuccess; ++k) e = do_step(s, false, s->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &g);
    s->cur = saved_cur;
    s->steps = saved_steps;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e;
    }
    if (e2 != cudaSuccess) return e2;
    e = cudaGraphInstantiate(&s->graph[par], g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace

namespace blbm {

// Grid stage of the FP64 sums: one block of kFinThreads threads adds the
// per-block partials in a fixed order (thread t takes partials t, t + kFinThreads,
// ...; then a fixed shuffle tree).  1024 threads keep each thread's chain of
// FP64 adds short, which matters at GB300's FP64 rate.
constexpr int kFinThreads = 1024;

__global__ void __launch_bounds__(kFinThreads)
k_finalize(const double* __restrict__ partials, int nparts, double* __restrict__ out) {
    double v[kNumStats];
#pragma unroll
    for (int k = 0; k < kNumStats; ++k) v[k] = 0.0;
    // unrolled so several partials are in flight; the order of the adds is unchanged
#pragma unroll 4
    for (int b = threadIdx.x; b < nparts; b += kFinThreads) {
#pragma unroll
        for (int k = 0; k < kNumStats; ++k) v[k] += partials[(int64_t)b * kNumStats + k];
    }
    __shared__ double sm[kFinThreads / 32][kNumStats];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kNumStats; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < kNumStats; ++k) sm[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < kNumStats; ++k) {
            double t = (lane < kFinThreads / 32) ? sm[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) out[k] = t;
        }
    }
}

cudaError_t launch_finalize(const double* partials, int nparts, double* out, cudaStream_t st) {
    k_finalize<<<1, kFinThreads, 0, st>>>(partials, nparts, out);
    return cudaGetLastError();
}

template <class T>
__global__ void k_fill(T* __restrict__ p, int64_t n, T v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

cudaError_t launch_fill(void* p, int64_t n, int rsize, double value, cudaStream_t st) {
    const int grid = (int)((n + kBlock - 1) / kBlock < 4096 ? (n + kBlock - 1) / kBlock : 4096);
    if (rsize == 8)
        k_fill<double><<<grid, kBlock, 0, st>>>((double*)p, n, value);
    else
        k_fill<float><<<grid, kBlock, 0, st>>>((float*)p, n, (float)value);
    return cudaGetLastError();
}

static std::atomic<double> g_wait_limit{0.0};

double wait_limit() { return g_wait_limit.load(); }

cudaError_t bounded_sync(cudaStream_t st) {
    const double limit = g_wait_limit.load();
    if (!(limit > 0.0)) return cudaStreamSynchronize(st);
    const auto t0 = std::chrono::steady_clock::now();
    for (int polls = 0;; ++polls) {
        const cudaError_t e = cudaStreamQuery(st);
        if (e != cudaErrorNotReady) return e;
        const std::chrono::duration<double> dt = std::chrono::steady_clock::now() - t0;
        if (dt.count() > limit) return cudaErrorNotReady;
        if (polls < 64)
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace blbm

// ===========================================================================
extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

const char* lbm_status_string(lbm_status st) {
    switch (st) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_ENONFINITE: return "non-finite density";
    case LBM_ETIMEOUT: return "timeout";
    case LBM_EBUSY: return "busy";
    case LBM_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
    }
}

lbm_status lbm_set_wait_limit(double seconds) {
    if (!(seconds >= 0.0) || !std::isfinite(seconds))
        return fail(LBM_EINVAL, "wait limit must be finite and >= 0 (got %g)", seconds);
    g_wait_limit.store(seconds);
    return LBM_OK;
}

lbm_status lbm_get_wait_limit(double* seconds) {
    if (!seconds) return fail(LBM_EINVAL, "seconds is NULL");
    *seconds = g_wait_limit.load();
    return LBM_OK;
}

lbm_status lbm_params_default(lbm_params* p) {
    if (!p) return fail(LBM_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->model = LBM_MODEL_IR;
    p->storage = LBM_F32;
    p->mu_p = 0.1;
    p->gammadot_c = 1e-8;
    p->magic = 0.25;
    return LBM_OK;
}

lbm_status lbm_lattice_info(lbm_lattice lat, int* Q, int* D, int* c, double* w) {
    switch (lat) {
    case LBM_D2Q9: lattice_table_D2Q9(c, w); break;
    case LBM_D3Q15: lattice_table_D3Q15(c, w); break;
    case LBM_D3Q19: lattice_table_D3Q19(c, w); break;
    case LBM_D3Q27: lattice_table_D3Q27(c, w); break;
    default: return fail(LBM_EINVAL, "unknown lattice %d", (int)lat);
    }
    if (Q) *Q = lattice_q(lat);
    if (D) *D = lat == LBM_D2Q9 ? 2 : 3;
    return LBM_OK;
}

lbm_status lbm_workspace_bytes(lbm_lattice lat, int nx, int ny, int nz, const lbm_params* p,
                               size_t* bytes) {
    if (!p || !bytes) return fail(LBM_EINVAL, "NULL argument");
    if (lattice_q(lat) == 0) return fail(LBM_EINVAL, "unknown lattice %d", (int)lat);
    if (nx < 1 || ny < 1 || nz < 1) return fail(LBM_EINVAL, "extents must be >= 1");
    if ((int64_t)nx * ny * nz > (int64_t)0x7fffffff - 64) return fail(LBM_EINVAL, "too many cells");
    if (storage_bytes(p->storage) == 0) return fail(LBM_EINVAL, "unknown storage %d", p->storage);
    // compact layout: sized as if every cell were fluid (an upper bound)
    *bytes = make_layout(lat, nx, ny, nz, *p, (int64_t)nx * ny * nz).total;
    return LBM_OK;
}

// fluid cells the step updates (ghost planes are not)
static int64_t stepped_fluid(int nx, int ny, int nz, const uint8_t* mask, uint32_t flags) {
    const int64_t nxy = (int64_t)nx * ny, n = nxy * nz;
    const bool ghosts = (flags & LBM_FLAG_Z_GHOSTS) != 0;
    int64_t nf = 0;
    for (int64_t i = ghosts ? nxy : 0; i < (ghosts ? n - nxy : n); ++i) nf += mask[i] == 0;
    return nf;
}

lbm_status lbm_workspace_bytes_for_mask(lbm_lattice lat, int nx, int ny, int nz,
                                        const uint8_t* solid_mask, const lbm_params* p,
                                        size_t* bytes) {
    if (!bytes) return fail(LBM_EINVAL, "bytes is NULL");
    lbm_status v = validate(lat, nx, ny, nz, solid_mask, p);
    if (v != LBM_OK) return v;
    *bytes = make_layout(lat, nx, ny, nz, *p, stepped_fluid(nx, ny, nz, solid_mask, p->flags)).total;
    return LBM_OK;
}

static lbm_status create_impl(lbm_solver** out, lbm_lattice lat, int nx, int ny, int nz,
                              const uint8_t* mask, const lbm_params* p, void* stream,
                              void* workspace, size_t ws_bytes) {
    if (!out) return fail(LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_status v = validate(lat, nx, ny, nz, mask, p);
    if (v != LBM_OK) return v;
    lbm_solver* s = new (std::nothrow) lbm_solver();
    if (!s) return fail(LBM_ENOMEM, "host allocation failed");
    s->lat = lat;
    s->Q = lattice_q(lat);
    s->D = lat == LBM_D2Q9 ? 2 : 3;
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->ncells = nx * ny * nz;
    s->p = *p;
    s->stream = (cudaStream_t)stream;
    // fluid cells: the stepped ones (ghost planes are not)
    const int nxy = nx * ny;
    const bool ghosts = (p->flags & LBM_FLAG_Z_GHOSTS) != 0;
    const bool compact = (p->flags & LBM_FLAG_COMPACT) != 0;
    auto stepped = [&](int i) { return mask[i] == 0 && !(ghosts && (i < nxy || i >= s->ncells - nxy)); };
    s->nfluid = stepped_fluid(nx, ny, nz, mask, p->flags);
    {
        // warps (32 consecutive cells) holding fluid cells, and those of them
        // that also hold solid cells: the copy-through choice of the 16-bit PR
        // step (taken when at least 1 % of the warps with fluid are mixed)
        int64_t with_fluid = 0, mixed = 0;
        for (int w0 = 0; w0 < s->ncells; w0 += 32) {
            const int w1 = std::min(w0 + 32, s->ncells);
            int nf = 0;
            for (int i = w0; i < w1; ++i) nf += stepped(i);
            with_fluid += nf > 0;
            mixed += nf > 0 && nf < w1 - w0;
        }
        s->copy = 100 * mixed >= with_fluid ? 1 : 0;
    }
    s->lay = make_layout(lat, nx, ny, nz, *p, s->nfluid);
    KParams& kp = s->kp;
    kp.nx = nx;
    kp.ny = ny;
    kp.nz = nz;
    kp.ncells = s->ncells;
    kp.cell_begin = 0;
    kp.cell_end = s->ncells;
    kp.nslots = compact ? (int)s->nfluid : 0;
    kp.plane = s->lay.plane;
    kp.nu_p = p->mu_p;   // rho_0 = 1
    kp.sigma_y = p->sigma_y;
    kp.m = p->m;
    kp.gdot_c = p->gammadot_c > 0.0 ? p->gammadot_c : 1e-8;
    kp.magic = p->magic > 0.0 ? p->magic : 0.25;
    for (int d = 0; d < 3; ++d) kp.g[d] = p->g[d];
    kp.flags = p->flags;
    kp.newton = p->model == LBM_MODEL_PR ? p->newton_iters : 0;
    kp.div_nx = FastDiv::make((uint32_t)nx);
    kp.div_ny = FastDiv::make((uint32_t)ny);

    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        cudaGetLastError();
        return fail(LBM_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    if (workspace) {
        if (ws_bytes < s->lay.total) {
            delete s;
            return fail(LBM_EINVAL, "workspace too small: %zu < %zu", ws_bytes, s->lay.total);
        }
        if (((uintptr_t)workspace & 255u) != 0) {
            delete s;
            return fail(LBM_EINVAL, "workspace must be 256-byte aligned");
        }
        s->base = (char*)workspace;
        s->owns = false;
    } else {
        void* b = nullptr;
        e = cudaMalloc(&b, s->lay.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return fail(LBM_ENOMEM, "cudaMalloc of %zu bytes failed", s->lay.total);
        }
        s->base = (char*)b;
        s->owns = true;
    }
    s->f[0] = s->base + s->lay.off_f[0];
    s->f[1] = s->base + s->lay.off_f[1];
    s->links = (uint32_t*)(s->base + s->lay.off_links);
    s->tau = p->model == LBM_MODEL_PR ? (void*)(s->base + s->lay.off_tau) : nullptr;
    s->usnap = p->check_every > 0 ? (void*)(s->base + s->lay.off_usnap) : nullptr;
    s->partials = (double*)(s->base + s->lay.off_partials);
    s->stats = (double*)(s->base + s->lay.off_stats);
    uint8_t* dmask = (uint8_t*)(s->base + s->lay.off_mask);
    std::vector<int> h_cellidx, h_rank;
    if (compact) {
        s->cellidx = (int*)(s->base + s->lay.off_cellidx);
        s->rank = (int*)(s->base + s->lay.off_rank);
        h_cellidx.reserve((size_t)s->nfluid);
        h_rank.assign((size_t)s->ncells, -1);
        for (int i = 0; i < s->ncells; ++i)
            if (stepped(i)) {
                h_rank[i] = (int)h_cellidx.size();
                h_cellidx.push_back(i);
            }
    }

    lbm_status rc = LBM_OK;
    do {
        e = cudaMallocHost(&s->host_stats, kNumStats * sizeof(double));
        if (e != cudaSuccess) { rc = fail(LBM_ENOMEM, "pinned allocation failed"); cudaGetLastError(); s->host_stats = nullptr; break; }
        std::memset(s->host_stats, 0, kNumStats * sizeof(double));
        const size_t fb = (size_t)s->Q * s->lay.plane * storage_bytes(p->storage);
        if ((e = cudaMemcpyAsync(dmask, mask, (size_t)s->ncells, cudaMemcpyHostToDevice, s->stream)) != cudaSuccess) break;
        if (compact) {
            if ((e = cudaMemcpyAsync(s->cellidx, h_cellidx.data(), h_cellidx.size() * sizeof(int), cudaMemcpyHostToDevice, s->stream)) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(s->rank, h_rank.data(), h_rank.size() * sizeof(int), cudaMemcpyHostToDevice, s->stream)) != cudaSuccess) break;
        }
        if ((e = launch_links(s, dmask)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(s->f[0], 0, fb, s->stream)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(s->f[1], 0, fb, s->stream)) != cudaSuccess) break;
        if (s->tau) {
            const double nu0 = p->mu_p + p->m * p->sigma_y;
            if ((e = launch_fill(s->tau, s->lay.plane, (int)arith_bytes(p->storage), 0.5 + 3.0 * nu0, s->stream)) != cudaSuccess) break;
        }
        if (s->usnap) {
            if ((e = cudaMemsetAsync(s->usnap, 0, (size_t)3 * s->lay.plane * arith_bytes(p->storage), s->stream)) != cudaSuccess) break;
        }
        // stats (2 x kNumStats doubles) and the two rounding counters behind them
        if ((e = cudaMemsetAsync(s->stats, 0, 256, s->stream)) != cudaSuccess) break;
        e = cudaStreamSynchronize(s->stream);
    } while (0);
    if (rc == LBM_OK && e != cudaSuccess) rc = cuda_fail(nullptr, e, "solver initialisation");
    if (rc != LBM_OK) {
        lbm_destroy(s);
        return rc;
    }
    *out = s;
    return LBM_OK;
}

lbm_status lbm_create(lbm_solver** out, lbm_lattice lat, int nx, int ny, int nz,
                      const uint8_t* solid_mask, const lbm_params* p, void* cuda_stream) {
    return create_impl(out, lat, nx, ny, nz, solid_mask, p, cuda_stream, nullptr, 0);
}

lbm_status lbm_create_with_workspace(lbm_solver** out, lbm_lattice lat, int nx, int ny, int nz,
                                     const uint8_t* solid_mask, const lbm_params* p,
                                     void* cuda_stream, void* workspace, size_t workspace_bytes) {
    if (!workspace) return fail(LBM_EINVAL, "workspace is NULL");
    return create_impl(out, lat, nx, ny, nz, solid_mask, p, cuda_stream, workspace, workspace_bytes);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Tuning table: launch shape of the plain step kernel (threads per block,
// cells per thread) per (lattice, model, storage, size class =
// floor(log2 cells)); filled by the autotuner through lbm_tuning_set(_shape),
// read by every solver before it steps.
namespace {

struct Shape {
    int block = kBlock, cpt = 1;
};

std::mutex g_tune_mu;
std::map<uint64_t, Shape> g_tune;
std::atomic<uint64_t> g_tune_version{0};

int size_class(int64_t cells) {
    int c = 0;
    while ((int64_t(1) << (c + 1)) <= cells && c < 62) ++c;
    return c;
}

uint64_t tune_key(int lat, int model, int storage, int cls) {
    return ((uint64_t)lat << 24) | ((uint64_t)model << 16) | ((uint64_t)storage << 8) | (uint64_t)cls;
}

Shape tune_lookup(int lat, int model, int storage, int64_t cells) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(lat, model, storage, size_class(cells)));
    return it == g_tune.end() ? Shape{} : it->second;
}

// Adopt the current table; a changed launch shape invalidates captured graphs.
void apply_tuning(lbm_solver* s) {
    const uint64_t ver = g_tune_version.load();
    if (s->tune_version == ver) return;
    const Shape sh = tune_lookup(s->lat, s->p.model, s->p.storage, s->ncells);
    if (sh.block != s->block || sh.cpt != s->cpt) {
        for (int k = 0; k < 2; ++k)
            if (s->graph[k]) {
                cudaGraphExecDestroy(s->graph[k]);
                s->graph[k] = nullptr;
            }
        s->block = sh.block;
        s->cpt = sh.cpt;
    }
    s->tune_version = ver;
}

lbm_status set_shape(int lat, int32_t model, int32_t storage, int32_t cls, int32_t block,
                     int32_t cpt) {
    if (lattice_q(lat) == 0) return fail(LBM_EINVAL, "unknown lattice %d", lat);
    if (model != LBM_MODEL_PR && model != LBM_MODEL_IR) return fail(LBM_EINVAL, "unknown model %d", model);
    if (storage_bytes(storage) == 0) return fail(LBM_EINVAL, "unknown storage %d", storage);
    if (cls < 0 || cls > 62) return fail(LBM_EINVAL, "size class must be in 0..62");
    if (block != 128 && block != 256 && block != 512) return fail(LBM_EINVAL, "block must be 128, 256 or 512");
    if (cpt != 1 && cpt != 2) return fail(LBM_EINVAL, "cells per thread must be 1 or 2");
    if (cpt == 2 && block == 512) return fail(LBM_EINVAL, "two cells per thread need block 128 or 256");
    if (cpt == 2 && storage == LBM_F64) return fail(LBM_EINVAL, "two cells per thread need FP32 arithmetic (not LBM_F64)");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tune_key(lat, model, storage, cls)] = Shape{block, cpt};
    }
    g_tune_version.fetch_add(1);
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_tuning_set(lbm_lattice lat, int32_t model, int32_t storage, int32_t size_class_,
                          int32_t block) {
    return set_shape(lat, model, storage, size_class_, block, 1);
}

lbm_status lbm_tuning_set_shape(lbm_lattice lat, int32_t model, int32_t storage,
                                int32_t size_class_, int32_t block, int32_t cells_per_thread) {
    return set_shape(lat, model, storage, size_class_, block, cells_per_thread);
}

lbm_status lbm_tuning_get(lbm_lattice lat, int32_t model, int32_t storage, int64_t cells,
                          int32_t* block, int32_t* size_class_) {
    return lbm_tuning_get_shape(lat, model, storage, cells, block, nullptr, size_class_);
}

lbm_status lbm_tuning_get_shape(lbm_lattice lat, int32_t model, int32_t storage, int64_t cells,
                                int32_t* block, int32_t* cells_per_thread, int32_t* size_class_) {
    if (lattice_q(lat) == 0 || cells < 1) return fail(LBM_EINVAL, "bad lattice or cell count");
    const Shape sh = tune_lookup(lat, model, storage, cells);
    if (block) *block = sh.block;
    if (cells_per_thread) *cells_per_thread = sh.cpt;
    if (size_class_) *size_class_ = size_class(cells);
    return LBM_OK;
}

lbm_status lbm_tuning_clear(void) {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune.clear();
    }
    g_tune_version.fetch_add(1);
    clear_batch_schedule();
    return LBM_OK;
}

lbm_status lbm_step(lbm_solver* s, int64_t nsteps) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (nsteps < 0) return fail(LBM_EINVAL, "nsteps must be >= 0");
    apply_tuning(s);
    const int64_t k = s->p.check_every;
    int64_t left = nsteps;
    while (left > 0) {
        // plain steps before the next check step
        int64_t plain = left;
        if (k > 0) {
            const int64_t to_check = k - (s->steps % k);   // the to_check-th step from now is a check step
            plain = (to_check - 1 < left) ? to_check - 1 : left;
        }
        while (plain >= s->graph_len) {
            if (!s->graph[s->cur]) CK(s, build_graph(s, s->cur), "CUDA graph capture");
            CK(s, cudaGraphLaunch(s->graph[s->cur], s->stream), "cudaGraphLaunch");
            s->steps += s->graph_len;   // graph_len is even: the parity is unchanged
            plain -= s->graph_len;
            left -= s->graph_len;
        }
        while (plain > 0) {
            CK(s, do_step(s, false, s->stream), "step launch");
            --plain;
            --left;
        }
        if (left > 0 && k > 0) {
            CK(s, do_step(s, true, s->stream), "check-step launch");
            --left;
        }
    }
    return LBM_OK;
}

lbm_status lbm_step_cells(lbm_solver* s, int64_t cell_begin, int64_t cell_end) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (s->rank) return fail(LBM_EINVAL, "the compact layout takes whole steps only (lbm_step)");
    if (cell_begin < 0 || cell_end < cell_begin || cell_end > s->ncells)
        return fail(LBM_EINVAL, "cell range [%lld, %lld) is not within 0..%d", (long long)cell_begin,
                    (long long)cell_end, s->ncells);
    const int64_t k = s->p.check_every;
    if (k > 0 && (s->steps + 1) % k == 0)
        return fail(LBM_EINVAL, "the next step is a check step: take it whole with lbm_step");
    if (cell_end == cell_begin) return LBM_OK;
    KParams kp = s->kp;
    kp.cell_begin = (int)cell_begin;
    kp.cell_end = (int)cell_end;
    StepArgs a;
    a.fsrc = s->f[s->cur];
    a.fdst = s->f[s->cur ^ 1];
    a.links = s->links;
    a.tau = s->tau;
    a.usnap = s->usnap;
    a.partials = s->partials;
    a.rng_ctr = (uint32_t*)(s->stats + 2 * kNumStats);
    a.parity = s->cur;
    a.block = kBlock;
    a.cpt = 1;
    a.copy = s->copy;
    a.cellidx = nullptr;
    a.rank = nullptr;
    const int km = kernel_model(s->p.model, s->kp.newton);
    cudaError_t e;
    switch (s->lat) {
    case LBM_D2Q9: e = launch_step_D2Q9(km, s->p.storage, false, kp, a, s->stream); break;
    case LBM_D3Q15: e = launch_step_D3Q15(km, s->p.storage, false, kp, a, s->stream); break;
    case LBM_D3Q19: e = launch_step_D3Q19(km, s->p.storage, false, kp, a, s->stream); break;
    default: e = launch_step_D3Q27(km, s->p.storage, false, kp, a, s->stream); break;
    }
    CK(s, e, "partial step launch");
    return LBM_OK;
}

lbm_status lbm_step_commit(lbm_solver* s) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (s->rank) return fail(LBM_EINVAL, "the compact layout takes whole steps only (lbm_step)");
    const int64_t k = s->p.check_every;
    if (k > 0 && (s->steps + 1) % k == 0)
        return fail(LBM_EINVAL, "the next step is a check step: take it whole with lbm_step");
    s->cur ^= 1;
    s->steps += 1;
    return LBM_OK;
}

lbm_status lbm_sync(lbm_solver* s) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    WAIT(s, "lbm_sync");
    return LBM_OK;
}

lbm_status lbm_fields_device(lbm_solver* s, double* rho, double* ux, double* uy, double* uz) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    CK(s, launch_fields(s, rho, ux, uy, uz), "fields kernel");
    return LBM_OK;
}

lbm_status lbm_fields(lbm_solver* s, double* rho, double* ux, double* uy, double* uz) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if ((v = ensure_scratch(s)) != LBM_OK) return v;
    WAIT(s, "lbm_fields");
    const size_t n = (size_t)s->ncells;
    double* d[4] = {s->scratch, s->scratch + n, s->scratch + 2 * n, s->scratch + 3 * n};
    CK(s, launch_fields(s, d[0], d[1], d[2], d[3]), "fields kernel");
    double* h[4] = {rho, ux, uy, uz};
    for (int k = 0; k < 4; ++k)
        if (h[k]) CK(s, cudaMemcpyAsync(h[k], d[k], n * sizeof(double), cudaMemcpyDeviceToHost, s->stream), "fields copy");
    CK(s, cudaStreamSynchronize(s->stream), "fields sync");
    return LBM_OK;
}

static lbm_status reduce_to_host(lbm_solver* s, int mode, double* out) {
    WAIT(s, "reduction");
    const int nb = reduce_grid(held_cells(s));
    CK(s, launch_reduce(s, mode, nb), "reduction kernel");
    CK(s, launch_finalize(s->partials, nb, s->stats + kNumStats, s->stream), "finalize kernel");
    CK(s, cudaMemcpyAsync(out, s->stats + kNumStats, kNumStats * sizeof(double), cudaMemcpyDeviceToHost, s->stream), "reduction copy");
    CK(s, cudaStreamSynchronize(s->stream), "reduction sync");
    return LBM_OK;
}

lbm_status lbm_flowrate(lbm_solver* s, int axis, double* q) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (!q || axis < 0 || axis > 2) return fail(LBM_EINVAL, "axis must be 0, 1 or 2 and q non-NULL");
    double r[kNumStats];
    if ((v = reduce_to_host(s, kReduceFlow, r)) != LBM_OK) return v;
    const int L = axis == 0 ? s->nx : (axis == 1 ? s->ny : s->nz);
    *q = r[kStatUx + axis] / L;
    return LBM_OK;
}

lbm_status lbm_totals(lbm_solver* s, double* mass, double momentum[3]) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    double r[kNumStats];
    if ((v = reduce_to_host(s, kReduceTotals, r)) != LBM_OK) return v;
    if (mass) *mass = (double)s->nfluid + r[kTotMass];
    if (momentum) {
        momentum[0] = r[kTotJx];
        momentum[1] = r[kTotJy];
        momentum[2] = r[kTotJz];
    }
    return LBM_OK;
}

lbm_status lbm_residual(lbm_solver* s, double* residual, int64_t* at_step, double* flow_x) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    WAIT(s, "lbm_residual");
    const double* r = s->host_stats;
    if (at_step) *at_step = s->last_check;
    if (flow_x) *flow_x = s->checks > 0 ? r[kStatUx] / s->nx : 0.0;
    if (residual) *residual = (s->checks >= 2 && r[kStatU2] > 0.0) ? std::sqrt(r[kStatDu2] / r[kStatU2]) : -1.0;
    if (s->checks > 0 && r[kStatNonFinite] != 0.0)
        return fail(LBM_ENONFINITE, "check step %lld saw %g non-finite densities", (long long)s->last_check, r[kStatNonFinite]);
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_solver* s, const double* f) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (!f) return fail(LBM_EINVAL, "f is NULL");
    if ((v = ensure_scratch(s)) != LBM_OK) return v;
    WAIT(s, "lbm_set_populations");
    // both buffers: a step writes every fluid cell of the other buffer, but
    // not every solid cell, so solid-cell populations read back later are the
    // uploaded ones whichever buffer is current then
    for (int q = 0; q < s->Q; ++q) {
        CK(s, cudaMemcpyAsync(s->scratch, f + (size_t)q * s->ncells, (size_t)s->ncells * sizeof(double), cudaMemcpyHostToDevice, s->stream), "population upload");
        CK(s, launch_convert(s, true, q, s->scratch, s->cur), "population convert");
        CK(s, launch_convert(s, true, q, s->scratch, s->cur ^ 1), "population convert");
    }
    CK(s, cudaStreamSynchronize(s->stream), "population sync");
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_solver* s, double* f) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (!f) return fail(LBM_EINVAL, "f is NULL");
    if ((v = ensure_scratch(s)) != LBM_OK) return v;
    WAIT(s, "lbm_get_populations");
    for (int q = 0; q < s->Q; ++q) {
        CK(s, launch_convert(s, false, q, s->scratch, s->cur), "population convert");
        CK(s, cudaMemcpyAsync(f + (size_t)q * s->ncells, s->scratch, (size_t)s->ncells * sizeof(double), cudaMemcpyDeviceToHost, s->stream), "population download");
    }
    CK(s, cudaStreamSynchronize(s->stream), "population sync");
    return LBM_OK;
}

lbm_status lbm_get_populations_cells(lbm_solver* s, const int64_t* cells, int64_t n, double* f) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (n < 0 || n > (int64_t)1 << 24) return fail(LBM_EINVAL, "n must be in 0..2^24");
    if (n == 0) return LBM_OK;
    if (!cells || !f) return fail(LBM_EINVAL, "cells and f must be non-NULL");
    for (int64_t k = 0; k < n; ++k)
        if (cells[k] < 0 || cells[k] >= s->ncells)
            return fail(LBM_EINVAL, "cells[%lld] = %lld is outside 0..%d", (long long)k,
                        (long long)cells[k], s->ncells - 1);
    WAIT(s, "lbm_get_populations_cells");
    int64_t* d_cells = nullptr;
    double* d_out = nullptr;
    const size_t out_bytes = (size_t)n * s->Q * sizeof(double);
    cudaError_t e = cudaMallocAsync((void**)&d_cells, (size_t)n * sizeof(int64_t), s->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_out, out_bytes, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_cells, cells, (size_t)n * sizeof(int64_t), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) {
        const void* fcur = s->f[s->cur];
        switch (s->lat) {
        case LBM_D2Q9: e = launch_gather_D2Q9(s->p.storage, s->kp, fcur, d_cells, (int)n, d_out, s->rank, s->stream); break;
        case LBM_D3Q15: e = launch_gather_D3Q15(s->p.storage, s->kp, fcur, d_cells, (int)n, d_out, s->rank, s->stream); break;
        case LBM_D3Q19: e = launch_gather_D3Q19(s->p.storage, s->kp, fcur, d_cells, (int)n, d_out, s->rank, s->stream); break;
        default: e = launch_gather_D3Q27(s->p.storage, s->kp, fcur, d_cells, (int)n, d_out, s->rank, s->stream); break;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d_out, out_bytes, cudaMemcpyDeviceToHost, s->stream);
    if (d_cells) cudaFreeAsync(d_cells, s->stream);
    if (d_out) cudaFreeAsync(d_out, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "population gather");
    return LBM_OK;
}

// The slots' cell indices (compact layout), for the tau transfers.
static lbm_status slot_cells(lbm_solver* s, std::vector<int>& cell) {
    cell.resize((size_t)held_cells(s));
    CK(s, cudaMemcpy(cell.data(), s->cellidx, cell.size() * sizeof(int), cudaMemcpyDeviceToHost), "slot map download");
    return LBM_OK;
}

lbm_status lbm_set_tau(lbm_solver* s, const double* tau) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (!s->tau) return fail(LBM_EINVAL, "the IR model has no relaxation-time field");
    if (!tau) return fail(LBM_EINVAL, "tau is NULL");
    WAIT(s, "tau transfer");
    const int n = held_cells(s);
    std::vector<int> cell;
    if (s->rank && (v = slot_cells(s, cell)) != LBM_OK) return v;
    auto at = [&](int k) { return tau[s->rank ? cell[k] : k]; };
    if (arith_bytes(s->p.storage) == 8) {
        std::vector<double> t(n);
        for (int k = 0; k < n; ++k) t[k] = at(k);
        CK(s, cudaMemcpy(s->tau, t.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice), "tau upload");
    } else {
        std::vector<float> t(n);
        for (int k = 0; k < n; ++k) t[k] = (float)at(k);
        CK(s, cudaMemcpy(s->tau, t.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice), "tau upload");
    }
    return LBM_OK;
}

lbm_status lbm_get_tau(lbm_solver* s, double* tau) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (!s->tau) return fail(LBM_EINVAL, "the IR model has no relaxation-time field");
    if (!tau) return fail(LBM_EINVAL, "tau is NULL");
    WAIT(s, "tau transfer");
    const int n = held_cells(s);
    std::vector<int> cell;
    if (s->rank) {
        if ((v = slot_cells(s, cell)) != LBM_OK) return v;
        // solid cells hold no tau in the compact layout: the initial value
        const double nu0 = s->p.mu_p + s->p.m * s->p.sigma_y;
        const double t0 = arith_bytes(s->p.storage) == 8 ? 0.5 + 3.0 * nu0 : (double)(float)(0.5 + 3.0 * nu0);
        for (int i = 0; i < s->ncells; ++i) tau[i] = t0;
    }
    auto put = [&](int k, double t) { tau[s->rank ? cell[k] : k] = t; };
    if (arith_bytes(s->p.storage) == 8) {
        std::vector<double> t(n);
        CK(s, cudaMemcpy(t.data(), s->tau, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost), "tau download");
        for (int k = 0; k < n; ++k) put(k, t[k]);
    } else {
        std::vector<float> t(n);
        CK(s, cudaMemcpy(t.data(), s->tau, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost), "tau download");
        for (int k = 0; k < n; ++k) put(k, t[k]);
    }
    return LBM_OK;
}

lbm_status lbm_check_sums(lbm_solver* s, double usum[3], double* du2, double* u2) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    WAIT(s, "lbm_check_sums");
    const double* r = s->host_stats;
    if (usum)
        for (int a = 0; a < 3; ++a) usum[a] = s->checks > 0 ? r[kStatUx + a] : 0.0;
    if (du2) *du2 = s->checks > 0 ? r[kStatDu2] : 0.0;
    if (u2) *u2 = s->checks > 0 ? r[kStatU2] : 0.0;
    return LBM_OK;
}

lbm_status lbm_set_hash_offset(lbm_solver* s, int64_t offset) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    // the hash input is the cell index plus the offset modulo 2^32
    s->kp.hash_offset = (uint32_t)(uint64_t)offset;
    for (int k = 0; k < 2; ++k)   // captured graphs hold the old kernel parameters
        if (s->graph[k]) {
            cudaGraphExecDestroy(s->graph[k]);
            s->graph[k] = nullptr;
        }
    return LBM_OK;
}

static int face_count(int lat) {
    switch (lat) {
    case LBM_D3Q15: return face_count_D3Q15();
    case LBM_D3Q19: return face_count_D3Q19();
    case LBM_D3Q27: return face_count_D3Q27();
    default: return face_count_D2Q9();
    }
}

lbm_status lbm_halo_bytes(const lbm_solver* s, size_t* bytes) {
    if (!s || !bytes) return fail(LBM_EINVAL, "NULL argument");
    if (!(s->p.flags & LBM_FLAG_Z_GHOSTS)) return fail(LBM_EINVAL, "the solver has no ghost planes");
    *bytes = (size_t)face_count(s->lat) * s->nx * s->ny * storage_bytes(s->p.storage);
    return LBM_OK;
}

static lbm_status halo(lbm_solver* s, int side, void* buf, bool pack) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (!(s->p.flags & LBM_FLAG_Z_GHOSTS)) return fail(LBM_EINVAL, "the solver has no ghost planes");
    if (side != 0 && side != 1) return fail(LBM_EINVAL, "side must be 0 (lower face) or 1 (upper face)");
    if (!buf) return fail(LBM_EINVAL, "buffer is NULL");
    if (((uintptr_t)buf % storage_bytes(s->p.storage)) != 0)
        return fail(LBM_EINVAL, "buffer must be aligned to the storage element");
    void* f = s->f[s->cur];
    cudaError_t e;
    switch (s->lat) {
    case LBM_D3Q15: e = launch_halo_D3Q15(s->p.storage, s->kp, f, buf, side, pack, s->stream); break;
    case LBM_D3Q19: e = launch_halo_D3Q19(s->p.storage, s->kp, f, buf, side, pack, s->stream); break;
    default: e = launch_halo_D3Q27(s->p.storage, s->kp, f, buf, side, pack, s->stream); break;
    }
    CK(s, e, pack ? "halo pack kernel" : "halo unpack kernel");
    return LBM_OK;
}

lbm_status lbm_halo_pack(lbm_solver* s, int side, void* buf) { return halo(s, side, buf, true); }

lbm_status lbm_halo_unpack(lbm_solver* s, int side, const void* buf) {
    return halo(s, side, const_cast<void*>(buf), false);
}

lbm_status lbm_get_info(const lbm_solver* s, lbm_info* info) {
    if (!s || !info) return fail(LBM_EINVAL, "NULL argument");
    info->lattice = s->lat;
    info->Q = s->Q;
    info->D = s->D;
    info->nx = s->nx;
    info->ny = s->ny;
    info->nz = s->nz;
    info->cells = s->ncells;
    info->fluid_cells = s->nfluid;
    info->steps_done = s->steps;
    info->model = s->p.model;
    info->storage = s->p.storage;
    // read Q + write Q populations + own mask byte (+ tau read and write for PR)
    const double b = 2.0 * s->Q * storage_bytes(s->p.storage) + 1.0 +
                     (s->p.model == LBM_MODEL_PR ? 2.0 * arith_bytes(s->p.storage) : 0.0);
    info->bytes_per_fluid_update = b;
    info->device_bytes = s->lay.total;
    return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free flow rate (lbm_flowrate_noalloc): the same grid-stride
// reduction kernel as lbm_flowrate, with its block partials in a file-scope
// device array instead of the solver's workspace.
namespace {

constexpr int kStaticParts = kReduceGridCap;   // reduce_grid() never launches more blocks
static __device__ __align__(256) double g_static_partials[kStaticParts * kNumStats];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_addr[kMaxDevices] = {nullptr};

// Device address of g_static_partials on the current device, looked up once
// per device (host code may not use the symbol itself as a device pointer).
lbm_status static_partials(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_EUNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LBM_ECUDA, "cudaGetSymbolAddress of the static reduction scratch: %s",
                        cudaGetErrorString(e));
        }
        g_static_addr[dev] = (double*)p;
    }
    *out = g_static_addr[dev];
    return LBM_OK;
}

// Fixed-order sum of the partials (one block) and Q_a = sum / L_a.
__global__ void k_finalize_axis(int nparts, int slot, double inv_len, double* __restrict__ q) {
    __shared__ double sm[kBlock];
    double v = 0.0;
    for (int b = threadIdx.x; b < nparts; b += kBlock) v += g_static_partials[b * kNumStats + slot];
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = kBlock / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *q = sm[0] * inv_len;
}

}  // namespace

extern "C" {

lbm_status lbm_flowrate_noalloc(lbm_solver* s, int axis, double* q_device) {
    lbm_status v = enter(s);
    if (v != LBM_OK) return v;
    if (axis < 0 || axis > 2) return fail(LBM_EINVAL, "axis must be 0, 1 or 2");
    if (!q_device) return fail(LBM_EINVAL, "q_device is NULL");
    if (((uintptr_t)q_device & 7u) != 0) return fail(LBM_EINVAL, "q_device must be 8-byte aligned");
    const int nb = reduce_grid(held_cells(s));
    if (nb > kStaticParts)
        return fail(LBM_EINVAL, "reduction needs %d partial blocks, the static scratch holds %d",
                    nb, kStaticParts);
    double* parts = nullptr;
    if ((v = static_partials(s->device, &parts)) != LBM_OK) return v;
    const void* f = s->f[s->cur];
    cudaError_t e;
    switch (s->lat) {
    case LBM_D2Q9: e = launch_reduce_D2Q9(s->p.storage, kReduceFlow, s->kp, f, s->links, s->cellidx, s->rank, parts, nb, s->stream); break;
    case LBM_D3Q15: e = launch_reduce_D3Q15(s->p.storage, kReduceFlow, s->kp, f, s->links, s->cellidx, s->rank, parts, nb, s->stream); break;
    case LBM_D3Q19: e = launch_reduce_D3Q19(s->p.storage, kReduceFlow, s->kp, f, s->links, s->cellidx, s->rank, parts, nb, s->stream); break;
    default: e = launch_reduce_D3Q27(s->p.storage, kReduceFlow, s->kp, f, s->links, s->cellidx, s->rank, parts, nb, s->stream); break;
    }
    CK(s, e, "static-scratch reduction kernel");
    const int L = axis == 0 ? s->nx : (axis == 1 ? s->ny : s->nz);
    k_finalize_axis<<<1, kBlock, 0, s->stream>>>(nb, kStatUx + axis, 1.0 / L, q_device);
    CK(s, cudaGetLastError(), "static-scratch finalize kernel");
    return LBM_OK;
}

void lbm_destroy(lbm_solver* s) {
    if (!s) return;
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev != s->device) cudaSetDevice(s->device);
    if (s->stream || s->base) cudaStreamSynchronize(s->stream);
    for (int k = 0; k < 2; ++k)
        if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->scratch) cudaFree(s->scratch);
    if (s->host_stats) cudaFreeHost(s->host_stats);
    if (s->owns && s->base) cudaFree(s->base);
    cudaGetLastError();
    delete s;
}

}  // extern "C"
