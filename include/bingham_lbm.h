/*
 * bingham_lbm.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann solver for
 * Bingham fluids.
 *
 * The method is the one of Regulski, Leonardi & Szumbarski, "On the spatial
 * convergence and transient behaviour of lattice Boltzmann methods for
 * modelling fluids with yield stress" (arXiv:1610.01388):
 *
 *   PR  Papanastasiou-regularised model (Sec. 3.1): strain rate from the
 *       non-equilibrium second moment with the previous step's relaxation
 *       time (eq. LBM_strain_rate), apparent viscosity eq. (Pap_reg_1) with the
 *       zero-strain cut-off eq. (PR_interpolation), relaxation time eq.
 *       (tau_visc), TRT collision with magic number Lambda (Sec. 2.1) and
 *       exact-difference forcing eq. (14);
 *   IR  locally implicit model (Secs. 2.3, 3.2): T = sum c c (f - f_eq), the
 *       closed-form Bingham solution of eq. (Vikh_main_short) given by eqs.
 *       (Vikh_sigmaS_formula)/(Vikh_sigmaS_tensor), post-collision populations
 *       eq. (Vikh_postCol) with f^sigma of eq. (Vikh_f_stress) and the force
 *       term of eq. (Vikh_force).
 *
 * Both run on D2Q9, D3Q15, D3Q19 and D3Q27 (Sec. 4.1), with streaming eq. (8)
 * in pull form, halfway bounce-back on solid cells (Sec. 4.3) and periodic
 * wrap at the domain faces.  Where the printed paper is garbled the library
 * takes these readings: the cut-off interpolation divides by gdot^C; IR yields
 * where |T| >= sqrt(2) sigma_y; f^sigma_i = w_i/(2 c_s^4)(c_i c_i - c_s^2 I):A
 * with A = -sigma_bar + s/2 and sigma_bar = sigma - (tr sigma / d) I; the IR
 * force term is Phi_i = w_i (c_i . F)/c_s^2 with F = rho g and the velocity
 * u = (j + F/2)/rho.
 *
 * Conventions for every call:
 *   - Grid: nx * ny * nz cells, x fastest: cell = x + nx * (y + ny * z).
 *     D2Q9 requires nz == 1.  At most 2^31 - 1 cells.
 *   - Populations at the ABI are FULL distribution values f_i (not offsets),
 *     FP64, laid out f[i * N + cell], in the library's velocity order, which
 *     lbm_lattice_info() reports.  This is the post-collision state after the
 *     last completed step (what the next step streams from).
 *   - Macroscopic fields are the moments of the streamed (pre-collision)
 *     populations of the next step: rho and u_real = (j + F/2)/rho (Sec. 2.4).
 *     Solid cells report rho = 0, u = 0.
 *   - Ownership: the library owns the solver handle and, for lbm_create, all
 *     device memory it allocates.  Every host pointer argument is owned by the
 *     caller and only read/written during the call.  The solid mask is copied.
 *   - Streams: work is enqueued on the CUDA stream given at creation (NULL =
 *     the legacy default stream).  lbm_step is asynchronous; calls that return
 *     host data synchronise that stream.
 *   - Errors: every call returns an lbm_status; on failure lbm_last_error()
 *     returns a thread-local message.  After a CUDA error the handle is
 *     poisoned: every later call on it returns LBM_ECUDA until lbm_destroy.
 *     No call throws, aborts or exits.
 */
#ifndef BINGHAM_LBM_H
#define BINGHAM_LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_API_VERSION 1

typedef struct lbm_solver lbm_solver; /* opaque, library-owned */

typedef enum { LBM_D2Q9 = 0, LBM_D3Q15 = 1, LBM_D3Q19 = 2, LBM_D3Q27 = 3 } lbm_lattice;

typedef enum { LBM_MODEL_PR = 0, LBM_MODEL_IR = 1 } lbm_model;

/* Population storage in device memory.  Every form stores the offset
 * f_i - w_i from the rest state; the collision arithmetic is FP64 for
 * LBM_F64 and FP32 for the others.  The 16-bit forms round stochastically on
 * every store.  LBM_F16_OFS is the reduced-precision form: its velocity
 * error against FP64 at equal step count measured 1.7-2.2e-4 relative L2
 * (within 1e-3).  LBM_BF16_OFS keeps 8 significant bits and measured
 * 1.4-1.7e-3: it does NOT meet that 1e-3 tolerance and is an option only. */
typedef enum {
    LBM_F64 = 0,      /* double offsets */
    LBM_F32 = 1,      /* float offsets */
    LBM_F16_OFS = 2,  /* half offsets, scaled by 2^14 / w_i */
    LBM_BF16_OFS = 3  /* bfloat16 offsets, scaled by 1 / w_i (fails the 1e-3 tolerance) */
} lbm_storage;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,       /* invalid argument; nothing was changed */
    LBM_ENOMEM = 2,       /* device or host allocation failed */
    LBM_ECUDA = 3,        /* CUDA runtime error; the handle is poisoned */
    LBM_ENONFINITE = 4,   /* a check step found a non-finite density */
    LBM_ETIMEOUT = 5,     /* a bounded device wait ran out */
    LBM_EBUSY = 6,        /* resource in use */
    LBM_EUNSUPPORTED = 7  /* combination not built into this library */
} lbm_status;

/* Flags (lbm_params.flags). */
#define LBM_FLAG_BURNETT_X 0x1u /* zero the xx components of D (PR) and of T (IR),
                                   the Burnett-suppressed variant of Secs. 4.2.1-4.2.2
                                   for flow along x */
#define LBM_FLAG_Z_GHOSTS 0x2u  /* the solver is one z-slab of a larger domain: its
                                   first and last z-planes are ghost planes that hold
                                   the neighbouring slabs' boundary populations (see
                                   lbm_halo_pack); they are never stepped and never
                                   counted, and their mask rows are the neighbours'
                                   own rows, so bounce-back across the slab faces is
                                   that of the whole domain.  3D lattices, nz >= 3 */
#define LBM_FLAG_COMPACT 0x4u   /* compact layout (no counterpart in the paper; for
                                   domains with many solid cells, e.g. porous media):
                                   the populations, link words, PR tau and check-step
                                   snapshot are held for the fluid cells only, one
                                   slot each in cell-index order, and one thread steps
                                   one slot.  The step's per-cell arithmetic is that
                                   of the dense layout (its own kernel, so the same to
                                   round-off of the arithmetic type: the compiler may
                                   contract multiply-adds differently).  On a porous
                                   medium it moves the fluid cells' bytes only.  Solid
                                   cells hold nothing:
                                   they read back as the rest state (populations w_i,
                                   tau at its initial value) and uploads to them are
                                   dropped.  Not with LBM_FLAG_Z_GHOSTS, not in
                                   batches (LBM_EINVAL); lbm_step_cells and
                                   lbm_step_commit return LBM_EINVAL */

/* Rheology, forcing and run-control parameters (lattice units, rho_0 = 1). */
typedef struct {
    int32_t model;       /* lbm_model */
    int32_t storage;     /* lbm_storage */
    double mu_p;         /* plastic viscosity; nu_p = mu_p / rho_0; > 0 */
    double sigma_y;      /* yield stress; >= 0 */
    double m;            /* Papanastasiou parameter (PR); >= 0 */
    double gammadot_c;   /* PR zero-strain cut-off gdot^C (Sec. 3.1); > 0; default 1e-8 */
    double g[3];         /* body acceleration; force density F = rho g; g[2] = 0 for D2Q9 */
    double magic;        /* TRT magic number Lambda (PR), > 0; default 0.25 (Sec. 2.1) */
    int32_t check_every; /* every k-th step also computes the flow rate and the
                            residual (0 = never) */
    uint32_t flags;      /* LBM_FLAG_* */
    int32_t newton_iters; /* PR: Newton iterations of the implicit relaxation-time
                            update (Sec. 3): each cell solves for the strain rate
                            whose apparent viscosity gives back the tau used in
                            eq. (LBM_strain_rate), starting from the explicit
                            estimate (previous step's tau); iterates are clamped at
                            gdot >= 0, the derivative is floored at 1/2.
                            0 = explicit update (default); 0..64; IR ignores it */
    int32_t reserved;    /* must be 0 */
} lbm_params;

/* Fills *p with defaults: IR, F32, mu_p 0.1, sigma_y 0, m 0, gammadot_c 1e-8,
 * g 0, magic 0.25, check_every 0, flags 0. */
lbm_status lbm_params_default(lbm_params *p);

/* Velocity set of a lattice in the library's order: Q, D, c[Q][3] (int),
 * w[Q] (double).  Any output pointer may be NULL.  Host only. */
lbm_status lbm_lattice_info(lbm_lattice lat, int *Q, int *D, int *c, double *w);

/* Device bytes lbm_create_with_workspace needs for this problem (populations
 * A/B, link masks, the PR relaxation-time field (one, updated in place),
 * residual snapshot, reduction partials).  With LBM_FLAG_COMPACT the size
 * depends on the fluid cells: this is then an upper bound (every cell fluid);
 * lbm_workspace_bytes_for_mask gives the exact size. */
lbm_status lbm_workspace_bytes(lbm_lattice lat, int nx, int ny, int nz,
                               const lbm_params *p, size_t *bytes);

/* The same for a given solid mask (validated as by lbm_create): exact for
 * both layouts.  Host only. */
lbm_status lbm_workspace_bytes_for_mask(lbm_lattice lat, int nx, int ny, int nz,
                                        const uint8_t *solid_mask, const lbm_params *p,
                                        size_t *bytes);

/* Creates a solver at rest (f_i = w_i, rho = 1, u = 0; PR tau = 1/2 + 3 nu_0,
 * nu_0 = nu_p + m sigma_y).  solid_mask: host, nx*ny*nz bytes, nonzero =
 * solid, copied.  At least one cell must be fluid.  cuda_stream: a
 * cudaStream_t or NULL.  The library allocates its device memory. */
lbm_status lbm_create(lbm_solver **out, lbm_lattice lat, int nx, int ny, int nz,
                      const uint8_t *solid_mask, const lbm_params *p, void *cuda_stream);

/* As lbm_create, but the caller provides the device memory: workspace must be
 * a device pointer, 256-byte aligned, of at least lbm_workspace_bytes() bytes,
 * and stay valid until lbm_destroy (e.g. a torch tensor kept alive). */
lbm_status lbm_create_with_workspace(lbm_solver **out, lbm_lattice lat, int nx, int ny,
                                     int nz, const uint8_t *solid_mask, const lbm_params *p,
                                     void *cuda_stream, void *workspace, size_t workspace_bytes);

/* Advances nsteps >= 0 time steps (one fused stream+collide launch each;
 * long runs are replayed through captured CUDA graphs).  Asynchronous. */
lbm_status lbm_step(lbm_solver *s, int64_t nsteps);

/* One plain step taken in parts (no counterpart in the paper; it lets a
 * z-slab update the planes that need no ghost values while its faces are in
 * transit).  lbm_step_cells steps the cells cell_begin <= n < cell_end
 * (0 <= cell_begin <= cell_end <= cells) from the current population buffer
 * into the other one, with exactly the per-cell arithmetic of lbm_step;
 * lbm_step_commit then makes the other buffer current and counts the step.
 * The ranges given between two commits must cover every fluid cell once
 * (a cell stepped twice would update the PR relaxation time twice).  Check
 * steps are taken whole: both calls return LBM_EINVAL when the next step is
 * a check step.  Asynchronous, on the solver's stream. */
lbm_status lbm_step_cells(lbm_solver *s, int64_t cell_begin, int64_t cell_end);
lbm_status lbm_step_commit(lbm_solver *s);

/* Waits for all work enqueued on the solver's stream. */
lbm_status lbm_sync(lbm_solver *s);

/* Wait limit (no counterpart in the paper; a serving safeguard).  Every call
 * that waits for a solver's or a batch's queued work -- lbm_sync, lbm_fields,
 * lbm_flowrate, lbm_totals, lbm_residual, lbm_set/get_populations,
 * lbm_set/get_tau, lbm_batch_domain_status, lbm_batch_remove, and through
 * them lbm_server_advance -- gives up after `seconds` and returns
 * LBM_ETIMEOUT.  It writes no output then; the queued work keeps running; the
 * handle stays usable, and a later call waits again.  lbm_server_advance
 * returning LBM_ETIMEOUT has queued its steps but judged no request; the next
 * advance continues from there.  Destroy calls always wait to completion.
 * 0 (the default) = no limit.  Process-wide; finite and >= 0, else
 * LBM_EINVAL. */
lbm_status lbm_set_wait_limit(double seconds);
lbm_status lbm_get_wait_limit(double *seconds);

/* Copies rho and u_real of every cell to host arrays of N doubles each; any
 * pointer may be NULL.  Synchronises. */
lbm_status lbm_fields(lbm_solver *s, double *rho, double *ux, double *uy, double *uz);

/* Same fields into device arrays (N doubles each, may be NULL); asynchronous. */
lbm_status lbm_fields_device(lbm_solver *s, double *rho, double *ux, double *uy, double *uz);

/* Flow rate along axis a (0 = x, 1 = y, 2 = z): Q_a = (1/L_a) sum over fluid
 * cells of u_real,a, the volumetric flow through one cross-section
 * (Sec. 4.5: U_avg = Q / L^2).  FP64 accumulation in a fixed order.
 * Synchronises. */
lbm_status lbm_flowrate(lbm_solver *s, int axis, double *q);

/* Totals of the current state over fluid cells: mass sum f_i and momentum
 * sum c_i f_i (FP64 accumulation, fixed order).  Synchronises. */
lbm_status lbm_totals(lbm_solver *s, double *mass, double momentum[3]);

/* Result of the last check step (check_every > 0): residual
 * sqrt(sum |u - u_prev|^2 / sum |u|^2) over fluid cells against the previous
 * check step (-1 before two check steps), its step index, and the flow rate
 * along x at that step.  The paper judges convergence by the relative change
 * of U_max between steps (Sec. 4.4) and of the velocity field (Sec. 4.5.2);
 * this residual is the L2 form of the latter.  Returns LBM_ENONFINITE if that check step saw a non-finite
 * density.  Synchronises. */
lbm_status lbm_residual(lbm_solver *s, double *residual, int64_t *at_step, double *flow_x);

/* Replace / read the population state (host, FP64 full f, Q*N, library
 * order).  lbm_set_populations writes both A/B buffers, so a solid cell
 * keeps the uploaded populations through every later step (a step defines
 * nothing for solid cells) and lbm_get_populations returns them (compact
 * layout: solid cells are not held and read back as w_i).  Synchronises. */
lbm_status lbm_set_populations(lbm_solver *s, const double *f);
lbm_status lbm_get_populations(lbm_solver *s, double *f);

/* Full FP64 populations of n listed cells (host array of cell indices
 * x + nx (y + ny z), each in 0..cells-1; n <= 2^24), in the library's velocity
 * order: f[i * n + k] = f_i(cells[k]), a host array of Q n doubles.  A probe of
 * a few cells of a large domain without reading the whole state back (no
 * counterpart in the paper).  Allocates 8 (Q + 1) n bytes of device memory
 * for the call; synchronises. */
lbm_status lbm_get_populations_cells(lbm_solver *s, const int64_t *cells, int64_t n, double *f);

/* PR relaxation-time field tau = 1/2 + 3 nu_app (eq. tau_visc), one value per
 * cell (host, N doubles), the value the next step's strain rate uses
 * (eq. LBM_strain_rate).  Compact layout: solid cells' values are dropped on
 * upload and read back as the initial 1/2 + 3 nu_0.  LBM_EINVAL for IR.
 * Synchronises. */
lbm_status lbm_set_tau(lbm_solver *s, const double *tau);
lbm_status lbm_get_tau(lbm_solver *s, double *tau);

/* ------------------------------------------------------------------------
 * One domain split into z-slabs (no counterpart in the paper: the method is
 * local per cell plus streaming to the nearest neighbours, eq. (8), so a
 * domain decomposes into slabs that exchange one plane of populations per
 * face and step).  Each slab is a solver created with LBM_FLAG_Z_GHOSTS over
 * its own planes plus one ghost plane on each side, whose mask rows are the
 * neighbouring slabs' boundary rows (periodic domain: slab 0's lower
 * neighbour is the last slab).  Before every step, for each face:
 *   lbm_halo_pack(lower slab, 1, buf)   -- its last interior plane's c_z = +1
 *                                          populations
 *   lbm_halo_unpack(upper slab, 0, buf) -- into the upper slab's lower ghost
 *   lbm_halo_pack(upper slab, 0, buf2)  -- its first interior plane's c_z = -1
 *                                          populations
 *   lbm_halo_unpack(lower slab, 1, buf2)-- into the lower slab's upper ghost
 * then every slab takes one step (lbm_step(s, 1)).  The slabs then hold
 * exactly the populations of the undivided domain (same per-cell
 * arithmetic).  buf: a device buffer of lbm_halo_bytes() bytes, stored values
 * in the solver's storage form (no conversion), aligned to the storage
 * element; between processes it can travel by any transport (NCCL
 * send/recv, peer copy), since both slabs use the same lattice and storage.
 * Pack and unpack are asynchronous on the solver's stream and act on its
 * current population buffer; order them against the other slab's stream.
 * LBM_EINVAL if the solver has no ghost planes or side is not 0 or 1.
 * ------------------------------------------------------------------------ */
lbm_status lbm_halo_bytes(const lbm_solver *s, size_t *bytes);
lbm_status lbm_halo_pack(lbm_solver *s, int side, void *buf_device);
lbm_status lbm_halo_unpack(lbm_solver *s, int side, const void *buf_device);

/* Offset added (modulo 2^32) to the cell index in the stochastic-rounding
 * hash of the 16-bit storage forms, so a slab whose local cell n is cell
 * n + offset of the whole domain draws the same random bits as the
 * undivided domain (offset = (z0 - 1) nx ny for a slab whose first interior
 * plane is global plane z0).  Default 0; no effect on FP32 / FP64. */
lbm_status lbm_set_hash_offset(lbm_solver *s, int64_t offset);

/* Raw sums of the last check step over the solver's fluid cells, for
 * combining slabs: usum[a] = sum of u_real,a; du2 = sum |u - u_prev|^2;
 * u2 = sum |u|^2 (the residual of lbm_residual is sqrt(du2 / u2), the flow
 * rate usum[a] / L_a).  Zeros before the first check step.  Synchronises. */
lbm_status lbm_check_sums(lbm_solver *s, double usum[3], double *du2, double *u2);

/* Problem description of a live solver. */
typedef struct {
    int32_t lattice, Q, D, nx, ny, nz;
    int64_t cells, fluid_cells, steps_done;
    int32_t model, storage;
    double bytes_per_fluid_update; /* algorithmic HBM bytes of one fluid-cell update */
    size_t device_bytes;
} lbm_info;
lbm_status lbm_get_info(const lbm_solver *s, lbm_info *info);

/* Flow rate along `axis`, like lbm_flowrate, for callers that must not
 * allocate memory at this point: code that runs under a fixed device-memory
 * budget with every byte handed out up front (a serving loop admitting solves
 * against a budget), code that shares the device through its own memory pool,
 * or code in a latency-critical loop where cudaMalloc (which can synchronise
 * the device and can fail under memory pressure) is not acceptable.
 * The paper has no counterpart; this is an interface convenience.
 *
 * It allocates nothing: no cudaMalloc, cudaFree, host or pinned allocation.
 * Inputs are the solver's resident populations; the output is one double
 * written to q_device, a caller-owned DEVICE pointer (8-byte aligned), as
 * Q_a = (1/L_a) sum over fluid cells of u_real,a.  The work is enqueued on
 * the solver's stream and the call returns without synchronising.
 *
 * Scratch: the per-block FP64 partial sums live in one file-scope device
 * array of the library, 1216 blocks x 8 doubles (76 KiB), which every GPU
 * that loads the library holds until the process exits.  The reduction is a
 * grid-stride loop with at most 1216 blocks, so every domain lbm_create
 * accepts fits; a launch that would need more partials is rejected with
 * LBM_EINVAL.  Each call writes every partial it reads, so nothing has to be
 * cleared between calls, but the array keeps the last call's contents and
 * is shared by all solvers and threads: calls whose work overlaps on the GPU
 * (different streams, or different host threads, without ordering) race on
 * it.  Order such calls on one stream or synchronise between them.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture on that device.  Axis outside 0..2, a NULL
 * q_device or a poisoned handle are rejected before any GPU work. */
lbm_status lbm_flowrate_noalloc(lbm_solver *s, int axis, double *q_device);

/* Releases the handle and the device memory the library allocated. */
void lbm_destroy(lbm_solver *s);

/* ------------------------------------------------------------------------
 * Tuning table (no counterpart in the paper): threads per block (128, 256 or
 * 512) of the plain step kernel for a (lattice, model, storage, size class),
 * size class = floor(log2(cells)).  Process-wide; entries default to 256.
 * Solvers adopt a changed entry at their next lbm_step (re-capturing their
 * graphs).  Check steps always use 256 threads, so flow rates and residuals
 * do not depend on the tuning.  The project's autotuner
 * (paper_1610_01388_gb300.autotune) measures the candidates and fills it.
 * It applies to the dense layout; the compact layout's step has fixed
 * shapes per lattice and model, chosen by measurement on porous boxes. 
 * ------------------------------------------------------------------------ */
lbm_status lbm_tuning_set(lbm_lattice lat, int32_t model, int32_t storage, int32_t size_class,
                          int32_t block);
/* Block used for a problem of `cells` cells, and its size class. */
lbm_status lbm_tuning_get(lbm_lattice lat, int32_t model, int32_t storage, int64_t cells,
                          int32_t *block, int32_t *size_class);
/* Launch shape with the cells each thread steps: 1, or 2 (block 128 or 256;
 * FP32, FP16 or BF16 storage).  With 2, thread t of a block steps cells
 * base + t and base + t + block and runs the collision of both at once in
 * packed two-wide FP32 instructions (fewer issued instructions for the same
 * arithmetic); results agree with one cell per thread to FP32 round-off.
 * lbm_tuning_set is lbm_tuning_set_shape with cells_per_thread = 1. */
lbm_status lbm_tuning_set_shape(lbm_lattice lat, int32_t model, int32_t storage,
                                int32_t size_class, int32_t block, int32_t cells_per_thread);
lbm_status lbm_tuning_get_shape(lbm_lattice lat, int32_t model, int32_t storage, int64_t cells,
                                int32_t *block, int32_t *cells_per_thread, int32_t *size_class);
lbm_status lbm_tuning_clear(void);   /* also resets the batch schedule below */

/* Batch schedule (no counterpart in the paper), read by every batch (and so
 * every server) at its next lbm_batch_step:
 *   ctas_per_sm -- per (lattice, model, storage) group: 0 (default) launches
 *     one CTA per tile; n > 0 launches a persistent grid of min(tiles,
 *     n x SMs) CTAs that walk the tiles.  0..32.
 *   concurrency -- 1: the captured 16-step graphs run the groups as parallel
 *     branches (they touch disjoint memory); 0 (default): one after another.
 * Results do not depend on either: the per-cell arithmetic and the order of
 * every reduction are the same (check-step partials are kept per tile).
 * The project's autotuner (paper_1610_01388_gb300.autotune.tune_batch) times
 * the candidates on a mix of domains and sets the fastest. */
lbm_status lbm_tuning_set_batch(lbm_lattice lat, int32_t model, int32_t storage,
                                int32_t ctas_per_sm);
lbm_status lbm_tuning_get_batch(lbm_lattice lat, int32_t model, int32_t storage,
                                int32_t *ctas_per_sm);
lbm_status lbm_tuning_set_batch_concurrency(int32_t concurrent);
lbm_status lbm_tuning_get_batch_concurrency(int32_t *concurrent);
/* Plain-step tile shape of the batch kernel for a (lattice, model, storage,
 * size class) group, size class = floor(log2(mean cells of the group's
 * domains)): threads per CTA (128, 256, 512) x cells each thread steps one
 * after the other (1, or 2 with 128 or 256 threads); a tile is that many
 * consecutive cells of one domain.  A group with no entry for its class
 * takes the entry of the nearest class set for its (lattice, model,
 * storage), else 256 x 1.  FP64 storage and the Newton-implicit PR step
 * always run 256 x 1 (FP64 entries other than 256 x 1 are LBM_EINVAL).
 * Check steps always run 256-cell tiles, so results do not depend on it.
 * lbm_tuning_get_batch_tile reports the shape a group of mean_cells cells
 * would run and its size class. */
lbm_status lbm_tuning_set_batch_tile(lbm_lattice lat, int32_t model, int32_t storage,
                                     int32_t size_class, int32_t threads, int32_t cells_per_thread);
lbm_status lbm_tuning_get_batch_tile(lbm_lattice lat, int32_t model, int32_t storage,
                                     int64_t mean_cells, int32_t *threads,
                                     int32_t *cells_per_thread, int32_t *size_class);

/* ------------------------------------------------------------------------
 * Batched stepping of many resident domains (no counterpart in the paper: a
 * throughput form for many small, independent solves).
 *
 * A batch owns any number of domains, each a full solver (any lattice, model,
 * storage, extents, rheology).  lbm_batch_step advances ALL of them: one
 * launch per (lattice, model, storage) combination present covers every
 * domain of that combination, long runs are replayed as CUDA graphs, and
 * every check_every-th step also computes each domain's residual and flow
 * rate.  Each domain's arithmetic is identical to lbm_step's (same device
 * code), so a domain's result does not depend on the other domains in the
 * batch (for the 16-bit storage forms up to the stochastic-rounding draw).
 * Device memory of each domain is taken from the CUDA stream-ordered memory
 * pool; the batch admits a domain only if the sum of all domains' bytes stays
 * within device_budget_bytes (LBM_EBUSY otherwise).  All work runs on the
 * batch's stream.  Domains need Q * cells < 2^31.
 * ------------------------------------------------------------------------ */
typedef struct lbm_batch lbm_batch;

typedef struct {
    int64_t steps;      /* time steps this domain has taken */
    int64_t checks;     /* check steps it has seen */
    double residual;    /* last check step; -1 before two check steps */
    double flow[3];     /* flow rate along x, y, z at the last check step */
    int32_t nonfinite;  /* 1 if the last check step saw a non-finite density */
    int32_t pad;
    double flow_change; /* |S - S_prev| / |S|, S the sums of u_real over fluid
                           cells at the last check step and S_prev at the one
                           before (the relative change of the mean velocity
                           vector over check_every steps); -1 before two */
} lbm_domain_status;

lbm_status lbm_batch_create(lbm_batch **out, size_t device_budget_bytes, int32_t check_every,
                            void *cuda_stream);
/* Adds a domain at rest (as lbm_create; p->check_every is replaced by the
 * batch's).  *domain_id receives its handle. */
lbm_status lbm_batch_add(lbm_batch *b, lbm_lattice lat, int nx, int ny, int nz,
                         const uint8_t *solid_mask, const lbm_params *p, int64_t *domain_id);
lbm_status lbm_batch_remove(lbm_batch *b, int64_t domain_id);
lbm_status lbm_batch_step(lbm_batch *b, int64_t nsteps);
/* Synchronises and reports the domain's last check step. */
lbm_status lbm_batch_domain_status(lbm_batch *b, int64_t domain_id, lbm_domain_status *st);
/* Borrows the domain's solver handle for lbm_fields / lbm_flowrate /
 * lbm_get_populations / ...; valid until the domain is removed; must not be
 * destroyed or stepped directly (use lbm_batch_step). */
lbm_status lbm_batch_solver(lbm_batch *b, int64_t domain_id, lbm_solver **s);
lbm_status lbm_batch_usage(const lbm_batch *b, size_t *bytes_used, int64_t *domains,
                           int64_t *fluid_cells);
void lbm_batch_destroy(lbm_batch *b);

/* ------------------------------------------------------------------------
 * Serving with continuous batching (no counterpart in the paper).
 *
 * Requests (independent solves) are submitted at any time and queued on the
 * host.  Each lbm_server_advance call admits queued requests while the
 * device-memory budget allows (in submission order, letting a smaller later
 * request in when an earlier one does not fit), advances every running
 * solve together by nsteps (a multiple of check_every) through one batch,
 * and retires the solves that reached steady state or their step cap,
 * freeing their memory for the next admissions.  Steady state is judged at
 * the last check step of each advance, between it and the check step
 * check_every steps before (the paper judges convergence by the change of
 * U_max between steps, Sec. 4.4, and of the velocity field, Sec. 4.5.2):
 *   LBM_STEADY_FLOW      the mean velocity vector changed by less than
 *                        tolerance (relative; lbm_domain_status.flow_change),
 *                        insensitive to per-cell rounding noise of the
 *                        16-bit storage forms;
 *   LBM_STEADY_RESIDUAL  the field residual sqrt(sum |u - u_prev|^2 /
 *                        sum |u|^2) is below tolerance.
 * Times are seconds on the server's monotonic clock (lbm_server_now).
 * ------------------------------------------------------------------------ */
typedef struct lbm_server lbm_server;

enum { LBM_STEADY_FLOW = 0, LBM_STEADY_RESIDUAL = 1 };

typedef struct {
    int32_t lattice, nx, ny, nz;
    const uint8_t *solid_mask;  /* host, nx*ny*nz, copied at submit */
    lbm_params params;          /* flags: not LBM_FLAG_COMPACT or LBM_FLAG_Z_GHOSTS
                                   (LBM_EINVAL at submit) */
    double tolerance;           /* steady state: change per check interval < tolerance */
    int64_t max_steps;          /* step cap (> 0) */
    int32_t keep_fields;        /* keep rho and u_real of the final state on the host */
    int32_t criterion;          /* LBM_STEADY_FLOW (0) or LBM_STEADY_RESIDUAL */
} lbm_request;

enum { LBM_REQ_QUEUED = 0, LBM_REQ_RUNNING = 1, LBM_REQ_CONVERGED = 2, LBM_REQ_CAPPED = 3,
       LBM_REQ_FAILED = 4 };

typedef struct {
    int32_t state;              /* LBM_REQ_* */
    int32_t pad;
    int64_t steps;
    int64_t fluid_cells;
    double residual;            /* field residual of the last check step */
    double flow_x;              /* flow rate along x at completion (lbm_flowrate) */
    double t_submit, t_admit, t_done;
} lbm_result;

lbm_status lbm_server_create(lbm_server **out, size_t device_budget_bytes, int32_t check_every,
                             void *cuda_stream);
/* Queues a request; LBM_EINVAL if it is malformed or could never fit the
 * budget.  *request_id receives its handle. */
lbm_status lbm_server_submit(lbm_server *s, const lbm_request *req, int64_t *request_id);
lbm_status lbm_server_advance(lbm_server *s, int64_t nsteps, int32_t *completed);
lbm_status lbm_server_result(const lbm_server *s, int64_t request_id, lbm_result *res);
/* rho / u_real (N doubles each, host, any may be NULL) of a completed
 * request submitted with keep_fields. */
lbm_status lbm_server_fields(const lbm_server *s, int64_t request_id, double *rho, double *ux,
                             double *uy, double *uz);
lbm_status lbm_server_pending(const lbm_server *s, int64_t *queued, int64_t *running,
                              size_t *bytes_used);
lbm_status lbm_server_now(const lbm_server *s, double *t);
void lbm_server_destroy(lbm_server *s);

/* Thread-local message of the last failing call on this thread. */
const char *lbm_last_error(void);
const char *lbm_status_string(lbm_status st);

#ifdef __cplusplus
}
#endif
#endif /* BINGHAM_LBM_H */
