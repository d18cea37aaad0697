// Launchers for one LU precision; included by solve_f32.cu and solve_f64.cu
// with CAMP_LT (float / double) and CAMP_SUFFIX (f32 / f64) defined.
#include "kernels.cuh"

#define CAMP_CAT2(a, b) a##_##b
#define CAMP_CAT(a, b) CAMP_CAT2(a, b)
#define CAMP_FN(name) CAMP_CAT(name, CAMP_SUFFIX)

namespace {
using LT = CAMP_LT;
constexpr int G = 32;

// Raise a kernel's dynamic shared-memory limit once to the maximum, so that
// launches (possibly inside stream capture) make no further attribute calls.
// One flag per kernel instantiation (the tag), not per function type.
template <int Tag, class K>
cudaError_t allow_smem(K kern) {
    static int done_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || done_dev == dev) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e == cudaSuccess) done_dev = dev;
    return e;
}

template <int NPL>
cudaError_t launch_solve_npl(const DevMech &m, const SolveArgs &a, int grid, cudaStream_t s) {
    auto kern = campdev::k_solve<G, NPL, LT>;
    int smem = camp_cell_smem_bytes(m, (int)sizeof(LT)) * a.cpb;
    cudaError_t e = allow_smem<NPL>(kern);
    if (e != cudaSuccess) return e;
    kern<<<grid, G * a.cpb, smem, s>>>(m, a);
    return cudaGetLastError();
}

template <int NPL>
cudaError_t occupancy_npl(const DevMech &m, int cpb, int *blocks) {
    auto kern = campdev::k_solve<G, NPL, LT>;
    int smem = camp_cell_smem_bytes(m, (int)sizeof(LT)) * cpb;
    cudaError_t e = allow_smem<NPL>(kern);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, G * cpb, smem);
}

template <int NPL>
cudaError_t launch_jac_npl(const DevMech &m, long long n_cells, const double *state,
                           const double *env, double *jac, cudaStream_t s) {
    auto kern = campdev::k_jacobian<G, NPL, LT>;
    int smem = camp_cell_smem_bytes(m, (int)sizeof(LT));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)n_cells, G, smem, s>>>(m, n_cells, state, env, jac);
    return cudaGetLastError();
}

template <int NPL>
cudaError_t launch_lu_npl(const DevMech &m, long long n_cells, const double *state,
                          const double *env, double gamma, const double *b, double *x, int *status,
                          cudaStream_t s) {
    auto kern = campdev::k_lu_solve<G, NPL, LT>;
    int smem = camp_cell_smem_bytes(m, (int)sizeof(LT));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)n_cells, G, smem, s>>>(m, n_cells, state, env, gamma, b, x, status);
    return cudaGetLastError();
}
}  // namespace

cudaError_t CAMP_FN(camp_launch_solve)(const DevMech &m, const SolveArgs &a, int grid, cudaStream_t s) {
#define CALL(N) launch_solve_npl<N>(m, a, grid, s)
    switch (camp_pick_npl(m.n)) {
    case 1: return CALL(1);
    case 2: return CALL(2);
    case 3: return CALL(3);
    case 4: return CALL(4);
    case 6: return CALL(6);
    case 8: return CALL(8);
    default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t CAMP_FN(camp_occupancy)(const DevMech &m, int cpb, int *blocks) {
#define CALL(N) occupancy_npl<N>(m, cpb, blocks)
    switch (camp_pick_npl(m.n)) {
    case 1: return CALL(1);
    case 2: return CALL(2);
    case 3: return CALL(3);
    case 4: return CALL(4);
    case 6: return CALL(6);
    case 8: return CALL(8);
    default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t CAMP_FN(camp_launch_jacobian)(const DevMech &m, long long n_cells, const double *state,
                                          const double *env, double *jac, cudaStream_t s) {
#define CALL(N) launch_jac_npl<N>(m, n_cells, state, env, jac, s)
    switch (camp_pick_npl(m.n)) {
    case 1: return CALL(1);
    case 2: return CALL(2);
    case 3: return CALL(3);
    case 4: return CALL(4);
    case 6: return CALL(6);
    case 8: return CALL(8);
    default: return cudaErrorInvalidValue;
    }
#undef CALL
}

cudaError_t CAMP_FN(camp_launch_lu_solve)(const DevMech &m, long long n_cells, const double *state,
                                          const double *env, double gamma, const double *b,
                                          double *x, int *status, cudaStream_t s) {
#define CALL(N) launch_lu_npl<N>(m, n_cells, state, env, gamma, b, x, status, s)
    switch (camp_pick_npl(m.n)) {
    case 1: return CALL(1);
    case 2: return CALL(2);
    case 3: return CALL(3);
    case 4: return CALL(4);
    case 6: return CALL(6);
    case 8: return CALL(8);
    default: return cudaErrorInvalidValue;
    }
#undef CALL
}
