// Internal definition of a solver handle, shared by the single-domain C ABI
// (lbm_api.cu) and the batched runtime (lbm_batch.cu).  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/bingham_lbm.h"
#include "lbm_internal.h"

namespace blbm {

// Device memory layout of one solver (offsets into one allocation).
struct Layout {
    int64_t plane;
    size_t off_f[2], off_links, off_tau, off_usnap, off_partials, off_stats, off_mask, total;
    size_t off_cellidx, off_rank;   // compact layout only
    int nparts;
};

lbm_status fail(lbm_status st, const char* fmt, ...);

// Waits for the work queued on `st` for at most the process-wide limit set by
// lbm_set_wait_limit (0 = no limit).  Returns cudaErrorNotReady when the limit
// ran out; the queued work is untouched and keeps running.
cudaError_t bounded_sync(cudaStream_t st);
double wait_limit();
int lattice_q(int lat);
void clear_batch_schedule();   // lbm_tuning_clear's part for batches
size_t storage_bytes(int storage);
size_t arith_bytes(int storage);

}  // namespace blbm

struct lbm_solver {
    int lat = 0, Q = 0, D = 0, nx = 0, ny = 0, nz = 0;
    int ncells = 0;
    int64_t nfluid = 0;
    lbm_params p{};
    blbm::KParams kp{};
    blbm::Layout lay{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0;
    bool owns = false;
    char* base = nullptr;
    void* f[2] = {nullptr, nullptr};   // population buffers; f[cur] is the state
    uint32_t* links = nullptr;         // per cell, or per slot in the compact layout
    int* cellidx = nullptr;            // compact layout: cell index of each slot
    int* rank = nullptr;               // compact layout: slot of each cell (-1: solid)
    void* tau = nullptr;
    void* usnap = nullptr;
    double* partials = nullptr;
    double* stats = nullptr;           // then two u32 rounding counters
    double* host_stats = nullptr;      // pinned, kNumStats doubles of the last check step
    double* scratch = nullptr;         // lazily allocated: 4 x ncells doubles
    int cur = 0;
    int64_t steps = 0;
    int64_t checks = 0;
    int64_t last_check = -1;
    bool poisoned = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_len = 64;
    int block = 256;                   // threads per block of plain steps (tuning table)
    int cpt = 1;                       // cells per thread of plain steps (tuning table)
    int copy = 1;                      // copy-through choice of the 16-bit PR step (geometry)
    uint64_t tune_version = ~uint64_t(0);
};
