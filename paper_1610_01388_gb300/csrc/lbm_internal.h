// Internal interface between the C ABI host code (lbm_api.cu) and the
// per-lattice kernel translation units.  Plain C++ types only.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "fastdiv.h"

namespace blbm {

constexpr int kBlock = 256;          // threads per block of the cell kernels
constexpr int kNumStats = 8;         // doubles per reduction partial
constexpr uint32_t kSolidBit = 1u << 31;
// Kernel-side model code: PR with the Newton-implicit tau update is its own
// instantiation, so the explicit kernels carry none of its code.
constexpr int kModelPRImplicit = 2;
inline int kernel_model(int model, int newton) {
    return (model == LBM_MODEL_PR && newton > 0) ? kModelPRImplicit : model;
}

// Scalars every cell kernel needs.  Rheology is given in double; each kernel
// rounds it to its arithmetic type.
struct KParams {
    int nx, ny, nz;
    int ncells;
    int64_t plane;        // elements between population planes (>= ncells, padded)
    double nu_p, sigma_y, m, gdot_c, magic;
    double g[3];
    uint32_t flags;
    int newton;           // PR: Newton iterations of the implicit tau update (0 = explicit)
    uint32_t hash_offset; // added to the cell index in the stochastic-rounding hash
    int cell_begin, cell_end; // cells the single-domain step kernel covers (0, ncells)
    int nslots;           // compact layout: fluid cells held (0: dense layout)
    FastDiv div_nx, div_ny;   // idx -> (x, y, z) without integer division
};

// Reduction slots.  Check step: flow sums of u_real (x,y,z), sum |u-u_prev|^2,
// sum |u|^2, sum of density offsets, count of non-finite densities.
enum { kStatUx = 0, kStatUy, kStatUz, kStatDu2, kStatU2, kStatDrho, kStatNonFinite };
// Batch stats rows only: relative change of the mean velocity vector since the
// domain's previous check step (-1 before its second one).
enum { kStatFlowChange = 7 };
// Totals mode: mass offset, momentum x,y,z.
enum { kTotMass = 0, kTotJx, kTotJy, kTotJz };

struct StepArgs {
    const void* fsrc;
    void* fdst;
    const uint32_t* links;
    void* tau;           // PR relaxation-time field, updated in place (R per cell)
    void* usnap;         // check step: u snapshot [3][plane] (R)
    double* partials;    // check step: [gridDim][kNumStats]
    uint32_t* rng_ctr;   // 16-bit storage: launch counters for stochastic rounding [2]
    int parity;          // which of the two counters this launch reads
    int block;           // threads per block of plain steps (128, 256 or 512)
    int cpt;             // cells per thread of plain steps (1, or 2 with block 128 / 256)
    int copy;            // 16-bit PR: solid cells of mixed groups copy through (geometry choice)
    const int* cellidx;  // compact layout: cell index of each slot (nullptr: dense layout)
    const int* rank;     // compact layout: slot of each cell, -1 for solid cells
};

enum ReduceMode { kReduceFlow = 0, kReduceTotals = 1 };

struct BatchDesc;   // per-domain descriptor of a batched launch (kernels.cuh)

// Per-lattice launchers (defined in kern_<lattice>.cu).
#define BLBM_DECLARE_LAUNCHERS(L)                                                              \
    cudaError_t launch_step_##L(int model, int storage, bool check, const KParams& kp,          \
                                const StepArgs& a, cudaStream_t st);                            \
    cudaError_t launch_links_##L(const KParams& kp, const uint8_t* mask, uint32_t* links,       \
                                 const int* cellidx, cudaStream_t st);                          \
    cudaError_t launch_fields_##L(int storage, const KParams& kp, const void* f,                \
                                  const uint32_t* links, const int* rank, double* rho,          \
                                  double* ux, double* uy, double* uz, cudaStream_t st);         \
    cudaError_t launch_reduce_##L(int storage, int mode, const KParams& kp, const void* f,      \
                                  const uint32_t* links, const int* cellidx, const int* rank,   \
                                  double* partials, int nblocks, cudaStream_t st);              \
    cudaError_t launch_convert_##L(int storage, bool to_device, const KParams& kp, int q,       \
                                   void* f, double* plane_buf, const int* rank, cudaStream_t st);\
    void lattice_table_##L(int* c, double* w);                                                  \
    cudaError_t launch_gather_##L(int storage, const KParams& kp, const void* f,               \
                                  const int64_t* cells, int n, double* out, const int* rank,    \
                                  cudaStream_t st);                                             \
    cudaError_t launch_halo_##L(int storage, const KParams& kp, void* f, void* buf, int side,   \
                                bool pack, cudaStream_t st);                                    \
    int face_count_##L();                                                                       \
    cudaError_t launch_step_batch_##L(int model, int storage, bool check,                       \
                                      const struct BatchDesc* descs, const int* block_dom,      \
                                      int nblocks, int grid, int phase, double* partials,       \
                                      int threads, int cpt, cudaStream_t st);

BLBM_DECLARE_LAUNCHERS(D2Q9)
BLBM_DECLARE_LAUNCHERS(D3Q15)
BLBM_DECLARE_LAUNCHERS(D3Q19)
BLBM_DECLARE_LAUNCHERS(D3Q27)

cudaError_t launch_finalize(const double* partials, int nparts, double* out, cudaStream_t st);
cudaError_t launch_fill(void* p, int64_t n, int rsize, double value, cudaStream_t st);

// Most blocks a grid-stride reduction (k_reduce) launches: 152 SMs x 8
// blocks.  Every buffer of per-block reduction partials is sized by it.
constexpr int kReduceGridCap = 1216;

inline int step_grid(int ncells) { return (ncells + kBlock - 1) / kBlock; }
inline int reduce_grid(int ncells) {
    int g = (ncells + kBlock - 1) / kBlock;
    return g < kReduceGridCap ? g : kReduceGridCap;
}

}  // namespace blbm
