// Launchers for one LU precision; included by solve_f32.cu and solve_f64.cu
// with CAMP_LT (float / double) and CAMP_SUFFIX (f32 / f64) defined, and by
// solve_f32w.cu / solve_f64w.cu with CAMP_WATER 1 as well (the builds for
// mechanisms with a water parameter, suffix f32w / f64w).
#include "kernels.cuh"

#ifndef CAMP_WATER
#define CAMP_WATER 0
#endif

#define CAMP_CAT2(a, b) a##_##b
#define CAMP_CAT(a, b) CAMP_CAT2(a, b)
#define CAMP_FN(name) CAMP_CAT(name, CAMP_SUFFIX)

namespace {
using LT = CAMP_LT;
constexpr bool W = CAMP_WATER != 0;

// Raise a kernel's dynamic shared-memory limit once to the maximum (the
// block's 227 KB less the kernel's own static shared memory), so that
// launches (possibly inside stream capture) make no further attribute calls.
// One flag per kernel instantiation (the tag), not per function type.  A
// failed call also clears the runtime's last-error state, so that it is not
// reported again by a later, healthy launch.
template <int Tag, class K>
cudaError_t allow_smem(K kern) {
    static int done_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || done_dev == dev) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024 - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) done_dev = dev;
    else (void)cudaGetLastError();
    return e;
}

template <int G, int NPL>
cudaError_t launch_solve_npl(const DevMech &m, const SolveArgs &a, int grid, cudaStream_t s) {
    auto kern = campdev::k_solve<G, NPL, LT, W>;
    int smem = camp_cell_smem_bytes(m, (int)sizeof(LT)) * a.cpb;
    cudaError_t e = allow_smem<G * 16 + NPL>(kern);
    if (e != cudaSuccess) return e;
    kern<<<grid, G * a.cpb, smem, s>>>(m, a);
    return cudaGetLastError();
}

template <int G, int NPL>
cudaError_t occupancy_npl(const DevMech &m, int cpb, int *blocks) {
    auto kern = campdev::k_solve<G, NPL, LT, W>;
    int smem = camp_cell_smem_bytes(m, (int)sizeof(LT)) * cpb;
    cudaError_t e = allow_smem<G * 16 + NPL>(kern);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, G * cpb, smem);
}

template <int G, int NPL>
cudaError_t launch_jac_npl(const DevMech &m, long long n_cells, const double *state,
                           const double *env, double *jac, cudaStream_t s) {
    auto kern = campdev::k_jacobian<G, NPL, LT, W>;
    int smem = camp_cell_smem_bytes(m, (int)sizeof(LT));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)n_cells, G, smem, s>>>(m, n_cells, state, env, jac);
    return cudaGetLastError();
}

template <int G, int NPL>
cudaError_t launch_lu_npl(const DevMech &m, long long n_cells, const double *state,
                          const double *env, double gamma, const double *b, double *x, int *status,
                          cudaStream_t s) {
    auto kern = campdev::k_lu_solve<G, NPL, LT, W>;
    int smem = camp_cell_smem_bytes(m, (int)sizeof(LT));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)n_cells, G, smem, s>>>(m, n_cells, state, env, gamma, b, x, status);
    return cudaGetLastError();
}
}  // namespace

// one case per instantiated cell shape (lanes per cell, register slots per
// lane).  The water builds hold one one-warp shape, with 8 slots: a cell of
// fewer species runs with slots to spare.
#if CAMP_WATER
#define CAMP_DISPATCH_SHAPE(shape)                                \
    switch ((shape) > 0 && (shape) < CAMP_SHAPE_BLOCK ? 8 : (shape)) { \
    case 8: return CALL(32, 8);                                   \
    case CAMP_SHAPE_64X4: return CALL(64, 4);                     \
    case CAMP_SHAPE_BLOCK + 2: return CALL(64, 8);                \
    case CAMP_SHAPE_BLOCK + 4: return CALL(128, 8);               \
    case CAMP_SHAPE_BLOCK + 8: return CALL(256, 8);               \
    default: return cudaErrorInvalidValue;                        \
    }
#else
#define CAMP_DISPATCH_SHAPE(shape)                   \
    switch (shape) {                                 \
    case 1: return CALL(32, 1);                      \
    case 2: return CALL(32, 2);                      \
    case 3: return CALL(32, 3);                      \
    case 4: return CALL(32, 4);                      \
    case 6: return CALL(32, 6);                      \
    case 8: return CALL(32, 8);                      \
    case CAMP_SHAPE_64X4: return CALL(64, 4);        \
    case CAMP_SHAPE_BLOCK + 2: return CALL(64, 8);   \
    case CAMP_SHAPE_BLOCK + 4: return CALL(128, 8);  \
    case CAMP_SHAPE_BLOCK + 8: return CALL(256, 8);  \
    default: return cudaErrorInvalidValue;           \
    }
#endif

cudaError_t CAMP_FN(camp_launch_solve)(const DevMech &m, const SolveArgs &a, int grid, cudaStream_t s) {
#define CALL(G_, N) launch_solve_npl<G_, N>(m, a, grid, s)
    CAMP_DISPATCH_SHAPE(camp_pick_shape(m.n, m.lanes));
#undef CALL
}

cudaError_t CAMP_FN(camp_occupancy)(const DevMech &m, int cpb, int *blocks) {
#define CALL(G_, N) occupancy_npl<G_, N>(m, cpb, blocks)
    CAMP_DISPATCH_SHAPE(camp_pick_shape(m.n, m.lanes));
#undef CALL
}

cudaError_t CAMP_FN(camp_launch_jacobian)(const DevMech &m, long long n_cells, const double *state,
                                          const double *env, double *jac, cudaStream_t s) {
#define CALL(G_, N) launch_jac_npl<G_, N>(m, n_cells, state, env, jac, s)
    CAMP_DISPATCH_SHAPE(camp_pick_shape(m.n, m.lanes));
#undef CALL
}

cudaError_t CAMP_FN(camp_launch_lu_solve)(const DevMech &m, long long n_cells, const double *state,
                                          const double *env, double gamma, const double *b,
                                          double *x, int *status, cudaStream_t s) {
#define CALL(G_, N) launch_lu_npl<G_, N>(m, n_cells, state, env, gamma, b, x, status, s)
    CAMP_DISPATCH_SHAPE(camp_pick_shape(m.n, m.lanes));
#undef CALL
}
