/*
 * camp.h -- C ABI of libcamp.so: batched integration of CAMP's coupled stiff
 * multiphase chemistry ODE system for many independent grid cells on one GPU.
 *
 * Paper: M. Dawson et al., "Chemistry Across Multiple Phases (CAMP) version
 * 1.0", arXiv 2111.07436.  The calls follow the paper's statement of the
 * interface (Sect. 2.1 and 2.4.2): a core object is created once per
 * mechanism from its JSON description; the host then passes, per time step,
 * the state (species concentrations), the environment (temperature,
 * pressure, externally computed rates such as photolysis, aerosol state) and
 * the step length, and gets the new state back.
 *
 * Conventions
 *   - Return values: CAMP_OK (0) or a negative CAMP_E_* code; a message for
 *     the calling thread is available from camp_last_error().
 *   - Pointers documented as "device" must be CUDA device (or managed)
 *     memory on the device the mechanism was loaded on; "host" pointers are
 *     ordinary host memory.  The caller owns every array it passes.  The
 *     library owns camp_mech and camp_server handles until the matching
 *     free/destroy call.
 *   - Arrays are row-major with the cell index outermost:
 *       state  [n_cells][n_species]  ppb-equivalent of air, declaration order
 *                                   (gas species, then section b = 0.. of
 *                                   every aerosol-phase species);
 *       env    [n_cells][n_env]      T (K), P (Pa), one entry per
 *                                   PHOTOLYSIS (s^-1) / EMISSION (ppb s^-1)
 *                                   / FIRST_ORDER_LOSS (s^-1) process in
 *                                   declaration order, the relative
 *                                   humidity (0..1; only with a
 *                                   ZSR_AEROSOL_WATER parameter), then per
 *                                   section: radius (m), number (m^-3),
 *                                   water volume fraction (m^3 m^-3; with
 *                                   a water parameter the part not held by
 *                                   its electrolytes);
 *       status [n_cells]             per-cell status (CAMP_CELL_*).
 *   - Calls taking a `stream` are asynchronous on that cudaStream_t (NULL =
 *     legacy default stream); they validate arguments on the host and return
 *     CAMP_E_CUDA if a launch fails.
 */
#ifndef CAMP_H
#define CAMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define CAMP_OK 0
#define CAMP_E_INVAL (-1)       /* bad argument */
#define CAMP_E_PARSE (-2)       /* malformed mechanism description */
#define CAMP_E_NOMEM (-3)       /* device or host allocation failed */
#define CAMP_E_CUDA (-4)        /* CUDA runtime error */
#define CAMP_E_UNSUPPORTED (-5) /* mechanism too large for the device kernels */
#define CAMP_E_BUDGET (-6)      /* request larger than the server's memory budget */
#define CAMP_E_TIMEOUT (-7)     /* bounded wait expired */
#define CAMP_E_CANCELLED (-8)   /* request cancelled before it reached the GPU */

/* ---- per-cell status ---------------------------------------------------- */
#define CAMP_CELL_OK 0          /* integrated to dt */
#define CAMP_CELL_MAXSTEPS 1    /* max_steps internal steps taken before dt */
#define CAMP_CELL_ERRTEST 2     /* repeated error-test failures or h < h_min */
#define CAMP_CELL_NEWTON 3      /* repeated Newton failures */
#define CAMP_CELL_SINGULAR 4    /* tiny or non-finite LU pivot, repeatedly */
#define CAMP_CELL_NONFINITE 5   /* non-finite input or result */
/* A cell with status != 0 keeps its input state. */

typedef struct camp_mech camp_mech;

/* Sizes of a compiled mechanism. */
typedef struct {
    int32_t n_species;      /* state entries per cell */
    int32_t n_rxn;          /* process instances (section processes once per section) */
    int32_t n_env;          /* env entries per cell */
    int32_t n_sections;     /* aerosol sections (instances of the aerosol phase) */
    int32_t nnz_jac;        /* structural non-zeros of df/dy, diagonal included */
    int32_t nnz_lu;         /* non-zeros of L+U after fill */
    int32_t rxn_map_len;    /* entries of the process -> Jacobian map */
    int32_t dense_block;    /* order of the dense trailing block of the LU (0: none) */
    int32_t lu_storage;     /* LU values stored per cell on the device */
    int32_t smem_per_cell_mixed; /* shared-memory bytes per cell, FP32 J/LU */
    int32_t smem_per_cell_fp64;  /* shared-memory bytes per cell, FP64 J/LU */
    int64_t factor_updates; /* multiply-adds one device LU factorisation executes
                               (sparse part plus the dense block) */
    /* algorithmic floating-point operations of the method's steps, from
       the symbolic structure (independent of how the device stores it) */
    int64_t flops_forcing;  /* one f(y) */
    int64_t flops_jacobian; /* one assembly of I - gamma J */
    int64_t flops_factor;   /* one sparse LU factorisation */
    int64_t flops_solve;    /* one forward + backward substitution */
    int32_t env_rh;         /* env index of the relative humidity, -1 without
                               a ZSR_AEROSOL_WATER parameter */
    int32_t n_electrolytes; /* electrolytes of the water parameter (0: none) */
    int64_t model_forcing;  /* sum over process instances of 2 |reactants| +
                               |products| (distinct species): the flops of one
                               f(y) in a per-process cost model that counts
                               one multiply per reactant factor and one add
                               per stoichiometric term */
    int32_t block_arrow;    /* 1: the block-arrow form (particle-resolved; one
                               cell per thread-block cluster, every particle's
                               block eliminated into the gas block), 0: the
                               cell kernels */
    int32_t lanes_per_cell; /* threads that integrate one cell: 32 (one warp),
                               64, 128 or 256; camp_autotune may change it for
                               129-256 species (0 for the block-arrow form) */
} camp_mech_info;

/*
 * Compile a mechanism (paper Sect. 2.3: JSON configuration, no recompilation
 * of the library; Sect. 2.2: processes, aerosol phases and their instances;
 * Table 1: get_used_jacobian_elements / update_ids are done here, once).
 * json/len: UTF-8 text, not necessarily NUL-terminated.  On success *out is
 * a new handle whose tables live on the current CUDA device.  On failure
 * *out is NULL, a message is copied to err (if errlen > 0) and
 * CAMP_E_PARSE / CAMP_E_UNSUPPORTED / CAMP_E_CUDA is returned.
 * Schema: see paper_2111_07436_gb300/workloads.py (module docstring).
 * Process types (Table 2): ARRHENIUS, TROE, PHOTOLYSIS, EMISSION,
 * FIRST_ORDER_LOSS, CUSTOM_H2O2, CUSTOM_OH_HNO3 (gas phase);
 * HL_PHASE_TRANSFER, SIMPOL_PHASE_TRANSFER, AQUEOUS_REVERSIBLE,
 * CONDENSED_ARRHENIUS (one instance per aerosol section, or per
 * computational particle in the particle-resolved representation,
 * SingleParticle of Sect. 2.2.3, Table 6).
 * Parameters (Sect. 2.2.2, Table 4): ZSR_AEROSOL_WATER, the water of each
 * section from its electrolytes by the ZSR mixing rule
 * W = sum_i 1000 M_i / (MW_i m_i(a_w)) with Jacobson-form molality fits
 * sqrt(m_i) = sum_j Y_j a_w^j at a_w = RH.  The section's liquid volume is
 * then L_b(y) = L_env,b + W_b(y) / (1000 kg m^-3), a function of the state:
 * the section processes' constants carry powers of 1/L_b(y), and df/dy
 * includes the chain-rule term (df/dL_b)(dL_b/dy).
 * Limits: at most 2048 species (by default up to 192 a cell runs on one
 * warp, beyond that on a block of 64, 128 or 256 threads; camp_autotune and
 * camp_mech_set_lanes may choose another shape), 32767 stored LU values, and a
 * per-cell working set that fits one SM's shared memory; larger mechanisms
 * return CAMP_E_UNSUPPORTED or CAMP_E_PARSE with the reason.
 */
int camp_mech_load(const char *json, size_t len, camp_mech **out, char *err, size_t errlen);

/* Compile only, on the host: the handle serves camp_mech_info_get,
 * camp_mech_species_index and camp_mech_structure (no GPU needed); solving
 * with it returns CAMP_E_INVAL.  Same arguments and errors as
 * camp_mech_load. */
int camp_mech_compile(const char *json, size_t len, camp_mech **out, char *err, size_t errlen);

/* Release a mechanism and its device tables.  NULL is ignored. */
void camp_mech_free(camp_mech *m);

/* Fill *out with the mechanism's sizes (host struct). */
int camp_mech_info_get(const camp_mech *m, camp_mech_info *out);

/* State index of a species ("O3", or "bin3.a7" for section 3's instance of
 * phase species a7); -1 if unknown. */
int camp_mech_species_index(const camp_mech *m, const char *name);

/*
 * Integer structure of the mechanism, for bit-exact checks (host arrays the
 * caller allocates with the sizes from camp_mech_info; any may be NULL):
 *   rowptr [n+1], colidx [nnz_jac]: CSR pattern of df/dy in declaration
 *       order, columns sorted: the diagonal plus, for every process k, the
 *       rows R_k u P_k times the species D_k its rate depends on
 *       (D_k = R_k, or R_k u P_k for reversible processes); with a water
 *       parameter also, for every section process whose constants carry a
 *       power of 1/L_b, the rows R_k u P_k times the electrolytes of b;
 *   rxn_map [rxn_map_len]: for every process k, every j in D_k, every i in
 *       R_k u P_k (declaration order, reactants first, each species once):
 *       the CSR position of (i, j);
 *   perm [n]: elimination order (position p holds species perm[p]): exact
 *       minimum degree on pattern u pattern^T, ties to the smallest index;
 *   lu_rowptr [n+1], lu_colidx [nnz_lu]: fill pattern of the permuted matrix
 *       under elimination without pivoting;
 *   level_fwd [n], level_bwd [n]: dependency levels of the LU rows.
 */
int camp_mech_structure(const camp_mech *m, int32_t *rowptr, int32_t *colidx, int32_t *rxn_map,
                        int32_t *perm, int32_t *lu_rowptr, int32_t *lu_colidx,
                        int32_t *level_fwd, int32_t *level_bwd);

/* ---- the solve ---------------------------------------------------------- */
#define CAMP_VARIANT_MIXED 0   /* FP32 Jacobian assembly and LU; FP64 state,
                                  residual, Nordsieck history, error test */
#define CAMP_VARIANT_FP64 1    /* everything FP64 */
#define CAMP_NSTATS 5

typedef struct {
    int32_t variant;         /* CAMP_VARIANT_* (default MIXED) */
    int32_t persistent;      /* 1: one resident grid takes cells from a work
                                counter; 0: one group of lanes per cell, static
                                grid; -1: the autotuned choice (default) */
    int32_t max_steps;       /* internal steps per cell (default 10000) */
    int32_t cells_per_block; /* 0: the autotuned choice if any, else the
                                count (1..4) with the most resident cells.
                                Block-arrow (particle-resolved) mechanisms:
                                CTAs per cluster, 1, 2, 4, 8 or 16 (0: 8) */
    double hmin_frac;        /* minimum step = hmin_frac * dt (default 1e-10) */
    int32_t *stats;          /* optional device [n_cells][CAMP_NSTATS]: steps,
                                Newton iterations, Jacobian/LU setups,
                                error-test failures, sum of the BDF order
                                over accepted steps */
    void *workspace;         /* optional device scratch of
                                camp_workspace_bytes() bytes; NULL: the
                                mechanism's own (then calls on one mechanism
                                must not overlap on the GPU) */
    double *step;            /* optional device [n_cells], in/out: warm start
                                across consecutive calls for the same cells
                                (an opt-in; NULL = every call a cold start,
                                the paper's behaviour, Sect. 2.4.2).  In: a
                                value > 0 replaces the initial-step estimate
                                (the cell still starts at order 1, with
                                h = min(value, dt)).  Out: the step size the
                                controller held before its final step was cut
                                to land on dt; 0 for a cell whose status is
                                not 0.  camp_solve_host and
                                camp_solve_host_static take a host array. */
} camp_solve_opts;

/* Fill *o with the defaults for `variant`. */
void camp_solve_opts_default(camp_solve_opts *o, int variant);

/* Scratch bytes one concurrent camp_solve needs (the work counter). */
size_t camp_workspace_bytes(void);

/*
 * Integrate every cell over [0, dt] with the variable-order BDF + Newton +
 * sparse LU method (paper Sect. 2.4.1, CVODE's method class; Sect. 2.4.2:
 * f and its Jacobian assembled from per-process contributions), each cell an
 * independent cold start.
 *   state  device [n_cells][n_species], in/out;
 *   env    device [n_cells][n_env];
 *   dt > 0 (s), rtol > 0;
 *   atol   device [atol_len], atol_len = 1 (all species) or n_species, > 0;
 *   status device [n_cells], out;
 *   opts   may be NULL (defaults for CAMP_VARIANT_MIXED).
 * n_cells = 0 is a no-op.  Asynchronous on `stream` (a cudaStream_t).
 */
int camp_solve(const camp_mech *m, int64_t n_cells, double *state, const double *env, double dt,
               double rtol, const double *atol, int32_t atol_len, int32_t *status,
               const camp_solve_opts *opts, void *stream);

/*
 * n_steps consecutive outer steps of dt for every cell in ONE launch: the
 * host model's box run of Sect. 4.1 (a fixed environment, the state carried
 * from one step to the next), each step integrated as camp_solve would (a
 * cold start unless opts->step carries the step sizes).  trajectory (device
 * [n_steps][n_cells][n_species], or NULL) receives the state after each
 * step; state holds the state after the last step (or after the last step
 * that succeeded: a failing cell stops there, its status says why, and its
 * later trajectory rows are not written).  opts->stats, if set, sums the
 * counters over the steps.  Otherwise as camp_solve; n_steps >= 1.
 */
int camp_solve_sequence(const camp_mech *m, int64_t n_cells, double *state, const double *env, double dt,
                        int32_t n_steps, double *trajectory, double rtol, const double *atol,
                        int32_t atol_len, int32_t *status, const camp_solve_opts *opts, void *stream);

/*
 * Same as camp_solve with HOST arrays: copies state/env/atol to the device,
 * solves and copies state/status back, synchronously, on `stream`.  Device
 * staging buffers are kept per mechanism between calls (grown as needed);
 * concurrent camp_solve_host calls on one mechanism are serialised.  Pinned
 * host memory gives asynchronous DMA copies; pageable memory works too.
 */
int camp_solve_host(const camp_mech *m, int64_t n_cells, double *state, const double *env,
                    double dt, double rtol, const double *atol, int32_t atol_len, int32_t *status,
                    const camp_solve_opts *opts, void *stream);

/* ---- solving without allocating device memory ---------------------------- */
/* camp_solve_host stages the chunk through device buffers it obtains with
 * cudaMalloc (and, for the persistent grid, a work counter).  Some callers
 * cannot let a library allocate: host models that hand all device memory to
 * their own pool allocator, or run under a hard device-memory cap, where a
 * hidden cudaMalloc fails or eats into the pool; time-stepping loops that
 * must not stall on the device-wide synchronisation that cudaMalloc and
 * cudaFree can cause while other streams are busy; and codes that must never
 * see an out-of-memory error in the middle of a run.  This variant allocates
 * nothing: it stages through one array of CAMP_STATIC_SCRATCH_BYTES that is
 * part of the library's device image (every GPU that loads the library
 * holds it until the process exits).
 *   Same arguments and results as camp_solve_host (host arrays in and out,
 *   synchronous on `stream`; opts->stats, if set, is a host array).
 *   The chunk must fit: n_cells * (8 n_species + 8 n_env + 4 [+ 20 with
 *   opts->stats] [+ 8 with opts->step]) + 8 atol_len, each array rounded
 *   up to 256 bytes, plus 256 bytes for the work counter, must not exceed
 *   the array; larger calls return CAMP_E_INVAL and touch nothing -- split
 *   the chunk.
 *   The first call on a device looks up the array's device address (with
 *   that device current) and caches it; make that first call before any
 *   stream capture.
 *   All calls share the array and leave their data in it; the work counter
 *   is reset by every call.  Calls hold a process-wide lock and synchronise
 *   their stream before returning, on error paths too once a copy has been
 *   enqueued; calls that still overlap on the GPU (for example replays of a
 *   captured call on two streams) race on the array.
 * The paper has no counterpart to this entry point. */
#define CAMP_STATIC_SCRATCH_BYTES (16u << 20)
int camp_solve_host_static(const camp_mech *m, int64_t n_cells, double *state, const double *env,
                           double dt, double rtol, const double *atol, int32_t atol_len,
                           int32_t *status, const camp_solve_opts *opts, void *stream);

/* ---- several mechanisms in one call --------------------------------------- */
/* One group of cells per mechanism (e.g. gas-only cells and cells carrying
 * aqueous phases).  Each group runs as its own persistent grid on a stream
 * forked from `stream` (joined back before the call's work completes), the
 * group whose cells cost the most first, so that as one grid drains its
 * counter the next one's blocks take the freed SMs and the batch ends on the
 * cheapest cells.  Capturable in a CUDA
 * graph (the fork/join uses events).  Arrays are device arrays as for
 * camp_solve; groups must not alias.  At most CAMP_MAX_GROUPS groups. */
#define CAMP_MAX_GROUPS 8
typedef struct {
    const camp_mech *mech;
    int64_t n_cells;
    double *state;
    const double *env;
    const double *atol;
    int32_t atol_len;
    int32_t *status;
    int32_t *stats;      /* optional, as camp_solve_opts.stats */
    void *workspace;     /* optional, as camp_solve_opts.workspace */
    double *step;        /* optional, as camp_solve_opts.step */
} camp_group;

int camp_solve_batch(const camp_group *groups, int32_t n_groups, double dt, double rtol,
                     const camp_solve_opts *opts, void *stream);

/* camp_solve_batch on HOST arrays (paper Sect. 2.4.2: the host passes the
 * state of each air mass and reads it back): every group's state, env,
 * atol, status and the optional stats / step are host arrays (workspace is
 * ignored).  Copies all groups in, solves them in one camp_solve_batch,
 * copies states, statuses (and stats / steps) back and synchronises
 * `stream` before returning.  The device staging buffer is kept by the
 * library per device between calls (grown as needed, freed at exit); calls
 * are serialised.  Pinned host memory gives asynchronous copies.  Errors as
 * camp_solve_batch; on an error nothing is copied back. */
int camp_solve_batch_host(const camp_group *groups, int32_t n_groups, double dt, double rtol,
                          const camp_solve_opts *opts, void *stream);

/* ---- launch autotuning ------------------------------------------------------ */
/* Time camp_solve on the given cells (device arrays, left unchanged) for
 * cells-per-block 1 to 4 and both grid mappings -- for a block-arrow
 * (particle-resolved) mechanism, clusters of 2, 4, 8 and 16 CTAs -- and make
 * the fastest the mechanism's default for `variant` (used when
 * opts.cells_per_block is 0 and opts.persistent is -1).  For 129-256 species
 * it also times both cell shapes (one warp a cell, or 64 threads with 4
 * species a lane), rebuilding the per-lane tables, and keeps the faster: the
 * shape is the mechanism's, for both variants (camp_mech_info.lanes_per_cell).
 * Replaced device tables stay allocated until camp_mech_free, so launches
 * queued before, or captured in a graph, stay valid; no other call may use
 * the mechanism while camp_autotune runs.  One untimed solve
 * comes first, then two sweeps over the candidates; each candidate is judged
 * by the faster of its two times.  Synchronous; allocates scratch for one
 * copy of the state.  *best_cpb / *best_persistent (may be NULL) receive the
 * choice; *ms_best the time of one solve with it. */
int camp_autotune(camp_mech *m, int64_t n_cells, const double *state, const double *env, double dt,
                  double rtol, const double *atol, int32_t atol_len, int32_t variant,
                  int32_t *best_cpb, int32_t *best_persistent, double *ms_best, void *stream);

/* Rebuild the mechanism's per-lane tables for `lanes` threads a cell (32, 64,
 * 128 or 256, at most 8 species a lane) -- the cell shape camp_autotune
 * otherwise chooses for 129-256 species -- and make it the mechanism's for
 * both variants.  The integer structure is unchanged; results change only by
 * the order of roundoff-level sums.  Replaced device tables stay allocated
 * until camp_mech_free; no other call may use the mechanism meanwhile.
 * Synchronous.  CAMP_E_INVAL for a lane count outside that set, more than 8
 * species a lane, or a mechanism compiled without a device;
 * CAMP_E_UNSUPPORTED for the block-arrow form or a cell that no longer fits
 * shared memory (the mechanism keeps its shape). */
int camp_mech_set_lanes(camp_mech *m, int32_t lanes);

/* ---- single steps of the method, for testing ----------------------------- */
/* Rate constants (paper Table 2) in ppb units: device env [n_cells][n_env]
 * -> kf, kr device [n_cells][n_rxn] (process order).  The rate of process k
 * is kf_k prod_{reactants} y^s - kr_k prod_{products} y^nu.  With a water
 * parameter the section processes' constants are per unit liquid volume
 * (the powers of 1/L_b(y) are applied at each state). */
int camp_rate_constants(const camp_mech *m, int64_t n_cells, const double *env, double *kf,
                        double *kr, void *stream);

/* Forcing f(y) = sum_k (dy/dt)_k (paper Sect. 2.4.2): device state, env ->
 * device f [n_cells][n_species], FP64. */
int camp_forcing(const camp_mech *m, int64_t n_cells, const double *state, const double *env,
                 double *f, void *stream);

/* Jacobian df_i/dy_j = sum_k (df_i/dy_j)_k (paper Sect. 2.4.2) at the CSR
 * non-zeros of camp_mech_structure: device jac [n_cells][nnz_jac], values
 * computed in the variant's assembly precision (the chain-rule term of a
 * water parameter, Sect. 2.2.2, in FP64). */
int camp_jacobian(const camp_mech *m, int64_t n_cells, const double *state, const double *env,
                  double *jac, int32_t variant, void *stream);

/* Solve (I - gamma J(y)) x = b per cell with the device's static-pivot LU in
 * the variant's precision: device b, x [n_cells][n_species]; device status
 * [n_cells] = CAMP_CELL_SINGULAR on a tiny pivot (x unwritten), else 0. */
int camp_lu_solve(const camp_mech *m, int64_t n_cells, const double *state, const double *env,
                  double gamma, const double *b, double *x, int32_t *status, int32_t variant,
                  void *stream);

/* ---- continuous-batching request loop ----------------------------------- */
/* The host model of the paper hands the solver one air mass (or chunk of
 * grid cells) at a time, every time step (Sect. 2.4.2).  A camp_server takes
 * such chunks -- any size, any loaded mechanism -- while earlier ones are
 * still on the GPU: a worker thread admits them in arrival order as soon as
 * a stream slot and enough of the device-memory budget are free, runs each
 * on its own stream (copy in, camp_solve, copy out), and retires them as they
 * complete; admitted chunks overlap on the device.  Results are the same as
 * a lone camp_solve of the chunk (each cell is an independent cold start). */
typedef struct camp_server camp_server;

typedef struct {
    size_t hbm_budget_bytes; /* device bytes in-flight chunks may hold (> 0) */
    int32_t max_inflight;    /* concurrent chunks (streams); 0 = 8 */
} camp_server_opts;

typedef struct {
    double t_submit, t_admit, t_done; /* seconds on the server's monotonic clock */
    int64_t n_cells;
    int32_t rc;                       /* CAMP_OK, CAMP_E_BUDGET (chunk larger than
                                         the whole budget), or another error */
} camp_request_info;

/* Create a server on the current device. */
int camp_server_create(const camp_server_opts *opts, camp_server **out);

/* Queue a chunk.  state (in/out), env and status are HOST arrays laid out as
 * for camp_solve; they must stay valid and untouched until the request is
 * finished (poll/wait).  Pinned host memory lets the copies overlap.  atol is
 * a scalar.  opts may be NULL (mixed form, persistent grid).  *req_id
 * receives the request's id. */
int camp_server_submit(camp_server *s, const camp_mech *m, int64_t n_cells, double *state,
                       const double *env, double dt, double rtol, double atol, int32_t *status,
                       const camp_solve_opts *opts, uint64_t *req_id);

/* Non-blocking: *done = 1 once the request finished (then *info is filled
 * and the id is released). */
int camp_server_poll(camp_server *s, uint64_t req_id, int32_t *done, camp_request_info *info);

/* Block until the request finishes or timeout_ms passes (CAMP_E_TIMEOUT;
 * the request stays queued and can be waited for again). */
int camp_server_wait(camp_server *s, uint64_t req_id, int32_t timeout_ms, camp_request_info *info);

/* Queue depth, chunks on the device and budget bytes in use. */
int camp_server_stats(camp_server *s, int32_t *pending, int32_t *inflight, size_t *bytes_in_use);

/* Withdraw a request that is still waiting for admission (a host model
 * that has moved on, or is shutting down, no longer needs it): it finishes
 * at once with rc CAMP_E_CANCELLED, its state and status arrays untouched,
 * and is collected by poll/wait like any other.  Returns CAMP_OK; a request
 * already on the GPU or finished cannot be withdrawn (CAMP_E_UNSUPPORTED; it
 * completes normally); an unknown id gives CAMP_E_INVAL.  Not in the paper:
 * part of the serving loop this library adds. */
int camp_server_cancel(camp_server *s, uint64_t req_id);

/* Finish every queued and in-flight chunk, then release the server (and
 * every resident cell set still alive). */
int camp_server_destroy(camp_server *s);

/* ---- resident cell sets ---------------------------------------------------
 * The host model hands the SAME air masses to the solver every time step
 * (Sect. 2.4.2).  A resident set keeps one chunk's state (and status, and
 * with warm_start each cell's step size) in device memory across the host's
 * consecutive steps: create it once from the initial state, then submit one
 * step at a time with that step's env and dt -- only env (8 n_env bytes a
 * cell) crosses the bus -- and read or overwrite the state on demand.  The
 * set's memory counts against the server's budget from create to destroy.
 * Steps of one set run in submission order (each waits for the previous);
 * steps of different sets and ordinary chunks overlap as usual.  With
 * warm_start = 0 every step is a cold start and gives the result of a lone
 * camp_solve of the set's current state; with warm_start = 1 each cell
 * carries its step size from one step to the next (camp_solve_opts.step,
 * starting cold). */
typedef struct camp_resident camp_resident;

/* Allocate the set on the server's device and copy the initial state (HOST
 * [n_cells][n_species]) in; synchronous.  CAMP_E_BUDGET if the set does not
 * fit in what the budget has left. */
int camp_server_resident_create(camp_server *s, const camp_mech *m, int64_t n_cells,
                                const double *state, int32_t warm_start, camp_resident **out);

/* Queue one step of the set: env (HOST [n_cells][n_env]) is copied in when
 * the step is admitted and must stay valid until the request finishes;
 * status (HOST [n_cells], or NULL to leave it on the device) receives the
 * per-cell status.  opts as for camp_server_submit (its stats, step and
 * workspace are ignored).  Completion as for any request (poll / wait). */
int camp_server_resident_step(camp_server *s, camp_resident *r, const double *env, double dt, double rtol,
                              double atol, int32_t *status, const camp_solve_opts *opts, uint64_t *req_id);

/* Wait (up to timeout_ms; CAMP_E_TIMEOUT) until every step submitted to the
 * set has finished, then copy its state (and, if not NULL, the last step's
 * status and the carried step sizes) to HOST arrays. */
int camp_server_resident_read(camp_server *s, camp_resident *r, double *state, int32_t *status,
                              double *step, int32_t timeout_ms);

/* Wait as for read, then overwrite the set's state from a HOST array (the
 * host model's other processes -- transport, emissions -- changed it).
 * Carried step sizes are kept. */
int camp_server_resident_write(camp_server *s, camp_resident *r, const double *state, int32_t timeout_ms);

/* Wait for the set's steps, then release its device memory and budget. */
int camp_server_resident_destroy(camp_server *s, camp_resident *r);

/* ---- measurement --------------------------------------------------------- */
/* Sustained fused multiply-add throughput of the current device in GFLOP/s
 * (2 flops per FMA), FP64 (fp64 = 1) or FP32: 8 independent chains per
 * thread, 8 blocks of 256 threads per SM.  Synchronous on `stream`.  The
 * denominator of the solve's arithmetic roofline (the paper has no
 * counterpart: it is a property of the machine). */
int camp_probe_fma_rate(int32_t fp64, double *gflops, void *stream);

/* Message for the last error on the calling thread ("" if none). */
const char *camp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CAMP_H */
