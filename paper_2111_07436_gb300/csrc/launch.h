// Host-side launch interface between the C ABI (capi.cu) and the kernels,
// which are compiled in one translation unit per LU precision.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "devmech.h"

#include <nvtx3/nvToolsExt.h>

#include "camp.h"

// A named range on the profiler timeline for the life of a scope (NVTX;
// free when no profiler is attached)
struct CampRange {
    explicit CampRange(const char *name) { nvtxRangePushA(name); }
    ~CampRange() { nvtxRangePop(); }
    CampRange(const CampRange &) = delete;
    CampRange &operator=(const CampRange &) = delete;
};

struct SolveArgs {
    long long n_cells;
    double *state;
    const double *env;
    double dt, rtol;
    const double *atol;
    int atol_len;
    int32_t *status;
    int32_t *stats;
    double *step;                   // warm-start step sizes [n_cells] or null
    int max_steps;
    double hmin_frac;
    int cpb;                        // cells per block
    unsigned long long *queue;      // work counter (persistent form) or null
    int n_outer;                    // consecutive outer steps of dt per cell (>= 1)
    double *traj;                   // [n_outer][n_cells][n] states after each outer step, or null
};

// Cell shapes instantiated: one warp per cell (G = 32 lanes) with NPL
// register slots per lane, NPL in {1, 2, 3, 4, 6, 8} (n <= 256; the water
// builds take NPL = 8 for all of them); one block of 64 threads with 4 slots
// (n <= 256), coded CAMP_SHAPE_64X4; or one block of G = 64, 128 or 256
// threads per cell with 8 slots per lane (n <= 8 G), coded as
// CAMP_SHAPE_BLOCK + G / 32.  camp_pick_shape returns the shape for n
// species on `lanes` lanes a cell (the count the mechanism's per-lane tables
// were built for), or -1 (n > 2048 or more than 8 species a lane).
#define CAMP_SHAPE_BLOCK 100
#define CAMP_SHAPE_64X4 (CAMP_SHAPE_BLOCK + 1)
int camp_pick_shape(int n, int lanes);

// Shared-memory bytes per cell for LU element size 4 or 8.
int camp_cell_smem_bytes(const DevMech &m, int lu_elem);

// Launchers (return a cudaError_t).  `lu_elem` 4 = FP32 J/LU, 8 = FP64.
cudaError_t camp_launch_solve_f32(const DevMech &m, const SolveArgs &a, int grid, cudaStream_t s);
cudaError_t camp_launch_solve_f64(const DevMech &m, const SolveArgs &a, int grid, cudaStream_t s);
cudaError_t camp_occupancy_f32(const DevMech &m, int cpb, int *blocks_per_sm);
cudaError_t camp_occupancy_f64(const DevMech &m, int cpb, int *blocks_per_sm);
// the same for mechanisms with a water parameter (DevMech::n_wsec > 0)
cudaError_t camp_launch_solve_f32w(const DevMech &m, const SolveArgs &a, int grid, cudaStream_t s);
cudaError_t camp_launch_solve_f64w(const DevMech &m, const SolveArgs &a, int grid, cudaStream_t s);
cudaError_t camp_occupancy_f32w(const DevMech &m, int cpb, int *blocks_per_sm);
cudaError_t camp_occupancy_f64w(const DevMech &m, int cpb, int *blocks_per_sm);
cudaError_t camp_launch_jacobian_f32w(const DevMech &m, long long n_cells, const double *state,
                                      const double *env, double *jac, cudaStream_t s);
cudaError_t camp_launch_jacobian_f64w(const DevMech &m, long long n_cells, const double *state,
                                      const double *env, double *jac, cudaStream_t s);
cudaError_t camp_launch_lu_solve_f32w(const DevMech &m, long long n_cells, const double *state,
                                      const double *env, double gamma, const double *b, double *x,
                                      int *status, cudaStream_t s);
cudaError_t camp_launch_lu_solve_f64w(const DevMech &m, long long n_cells, const double *state,
                                      const double *env, double gamma, const double *b, double *x,
                                      int *status, cudaStream_t s);

cudaError_t camp_launch_rates(const DevMech &m, long long n_cells, const double *env, double *kf,
                              double *kr, cudaStream_t s);
cudaError_t camp_launch_forcing(const DevMech &m, long long n_cells, const double *state,
                                const double *env, double *f, cudaStream_t s);
cudaError_t camp_launch_jacobian_f32(const DevMech &m, long long n_cells, const double *state,
                                     const double *env, double *jac, cudaStream_t s);
cudaError_t camp_launch_jacobian_f64(const DevMech &m, long long n_cells, const double *state,
                                     const double *env, double *jac, cudaStream_t s);
cudaError_t camp_launch_lu_solve_f32(const DevMech &m, long long n_cells, const double *state,
                                     const double *env, double gamma, const double *b, double *x,
                                     int *status, cudaStream_t s);
cudaError_t camp_launch_lu_solve_f64(const DevMech &m, long long n_cells, const double *state,
                                     const double *env, double gamma, const double *b, double *x,
                                     int *status, cudaStream_t s);

// The block-arrow solve of particle-resolved cells (solve_arrow.cu): one cell
// per thread-block cluster of cl_size CTAs; scratch holds n_clusters cells
// of camp_arrow_cell_bytes each.
#include "arrow.h"
size_t camp_arrow_cell_bytes(const ArrowDev &a, int lu_elem);
cudaError_t camp_arrow_max_clusters(int lu_elem, int cl_size, int *n);
cudaError_t camp_arrow_launch(const DevMech &mt, const ArrowDev &a, const SolveArgs &s, int lu_elem, char *scratch,
                              size_t cell_bytes, int n_clusters, int cl_size, cudaStream_t st);
cudaError_t camp_arrow_forcing(const DevMech &mt, const ArrowDev &a, long long n_cells, const double *state,
                               const double *env, double *f, cudaStream_t st);

// true when camp_solve needs device scratch beyond its arguments and the work
// counter (the block-arrow form's per-cell rows)
bool camp_mech_needs_scratch(const camp_mech *m);

// Record an error message for camp_last_error() and return `code`.
int camp_record_error(int code, const char *msg);
