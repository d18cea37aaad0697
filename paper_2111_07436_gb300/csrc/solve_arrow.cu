// Kernels and launchers of the block-arrow solve (arrow.cuh): particle-
// resolved cells, one cell per thread-block cluster.
#include "arrow.cuh"
#include "launch.h"

namespace campdev {

// Every cell over one or more outer steps; clusters take cells round-robin
// (cluster c: cells c, c + clusters, ...), each with its own slice of the
// scratch.  Four CTAs per SM (64 registers a thread): the particle loops are
// chains of dependent global loads, and the extra warps hide their latency
// (measured at 10^4 particles: 2.0x one CTA per SM, 1.3x two).
template <typename LT>
__global__ void __launch_bounds__(ARROW_NT, 4)
    k_arrow(DevMech mt, ArrowDev a, SolveArgs s, char *scratch, size_t cell_bytes) {
    __shared__ ArrowSmem<LT> sm;
    cg::cluster_group cl = cg::this_cluster();
    const long long csz = cl.num_blocks();
    const long long cid = blockIdx.x / csz, ncl = gridDim.x / csz;
    char *mine = scratch + cid * cell_bytes;
    int par = 0;
    for (long long cell = cid; cell < s.n_cells; cell += ncl) {
        CellStats st, tot{0, 0, 0, 0, 0};
        int status = ST_OK;
        for (int o = 0; o < s.n_outer && status == ST_OK; o++) {
            status = arrow_integrate_cell<LT>(mt, a, sm, cl, mine, s.state + cell * a.n, s.env + cell * a.n_env,
                                              s.dt, s.rtol, s.atol, s.atol_len, s.max_steps, s.hmin_frac,
                                              s.step ? s.step + cell : nullptr, par, st,
                                              s.traj ? s.traj + ((long long)o * s.n_cells + cell) * a.n : nullptr);
            tot.steps += st.steps;
            tot.newton += st.newton;
            tot.jac += st.jac;
            tot.errfail += st.errfail;
            tot.ordsum += st.ordsum;
            cl.sync();  // the state written back is the next step's input
        }
        if (cl.block_rank() == 0 && threadIdx.x == 0) {
            s.status[cell] = status;
            if (s.stats) {
                int32_t *o = s.stats + 5 * cell;
                o[0] = tot.steps;
                o[1] = tot.newton;
                o[2] = tot.jac;
                o[3] = tot.errfail;
                o[4] = tot.ordsum;
            }
        }
    }
}

// f(y) of every cell, [cell][n] in declaration order: one block of ARROW_NT
// threads per cell, particles over the threads, gas processes on warp 0,
// the particles' gas sums in a fixed order over warps.
__global__ void __launch_bounds__(ARROW_NT) k_arrow_forcing(DevMech mt, ArrowDev a, long long n_cells,
                                                            const double *state, const double *env, double *f) {
    __shared__ double ygas[CAMP_ARROW_MAX_GAS], part[ARROW_NT / 32][CAMP_ARROW_MAX_C], rsg[ARROW_MAX_RG];
    const long long cell = blockIdx.x;
    if (cell >= n_cells) return;
    const double *y = state + cell * a.n, *e = env + cell * a.n_env;
    double *fo = f + cell * a.n;
    const int tid = threadIdx.x, np = a.n_phi, nc = a.n_c;
    if (tid < a.n_g) ygas[tid] = y[tid];
    __syncthreads();
    double gp[CAMP_ARROW_MAX_C];
    for (int q = 0; q < nc; q++) gp[q] = 0.0;
    double yl[ARROW_MAX_LOC], fl[ARROW_MAX_LOC];
    for (int p = tid; p < a.P; p += ARROW_NT) {
        for (int i = 0; i < np; i++) yl[i] = y[a.n_g + p * np + i];
        for (int q = 0; q < nc; q++) yl[np + q] = ygas[__ldg(a.coupled + q)];
        for (int i = 0; i < a.n_loc; i++) fl[i] = 0.0;
        for (int k = 0; k < a.Rp; k++) {
            const int4 r0 = __ldg(a.prec + 3 * k), r1 = __ldg(a.prec + 3 * k + 1), r2 = __ldg(a.prec + 3 * k + 2);
            double kf, kr;
            rate_constant_at(mt, r0.x, e, e + a.E0 + 3 * p, kf, kr);
            const double r = arrow_rate(r1, r2, kf, kr, yl);
            for (int q = r0.w; q < r1.w; q++) fl[__ldg(a.st_sp + q)] += __ldg(a.st_nu + q) * r;
        }
        for (int i = 0; i < np; i++) fo[a.n_g + p * np + i] = fl[i];
        for (int q = 0; q < nc; q++) gp[q] += fl[np + q];
    }
    for (int q = 0; q < nc; q++) {
        double x = gp[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((tid & 31) == 0) part[tid >> 5][q] = x;
    }
    if (tid < 32)
        for (int k = tid; k < a.Rg; k += 32) {
            const int4 r0 = __ldg(a.grec + 3 * k), r1 = __ldg(a.grec + 3 * k + 1), r2 = __ldg(a.grec + 3 * k + 2);
            double kf, kr;
            rate_constant_at(mt, r0.x, e, e, kf, kr);
            rsg[k] = arrow_rate(r1, r2, kf, kr, ygas);
        }
    __syncthreads();
    if (tid < a.n_g) {
        double s = 0.0;
        for (int q = __ldg(a.gf_ptr + tid); q < __ldg(a.gf_ptr + tid + 1); q++)
            s += __ldg(a.gf_nu + q) * rsg[__ldg(a.gf_k + q)];
        for (int q = 0; q < nc; q++)
            if (__ldg(a.coupled + q) == tid)
                for (int w = 0; w < ARROW_NT / 32; w++) s += part[w][q];
        fo[tid] = s;
    }
}

}  // namespace campdev

namespace {
template <typename LT>
cudaError_t arrow_config(int cl_size, int n_clusters, cudaStream_t st, cudaLaunchConfig_t &cfg,
                         cudaLaunchAttribute *attr) {
    auto kern = campdev::k_arrow<LT>;
    if (cl_size > 8) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3((unsigned)(n_clusters * cl_size));
    cfg.blockDim = dim3(campdev::ARROW_NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl_size;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaSuccess;
}
}  // namespace

size_t camp_arrow_cell_bytes(const ArrowDev &a, int lu_elem) { return campdev::arrow_cell_bytes(a, lu_elem); }

cudaError_t camp_arrow_max_clusters(int lu_elem, int cl_size, int *n) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = lu_elem == 4 ? arrow_config<float>(cl_size, 1, nullptr, cfg, attr)
                                 : arrow_config<double>(cl_size, 1, nullptr, cfg, attr);
    if (e != cudaSuccess) return e;
    return lu_elem == 4 ? cudaOccupancyMaxActiveClusters(n, campdev::k_arrow<float>, &cfg)
                        : cudaOccupancyMaxActiveClusters(n, campdev::k_arrow<double>, &cfg);
}

cudaError_t camp_arrow_launch(const DevMech &mt, const ArrowDev &a, const SolveArgs &s, int lu_elem, char *scratch,
                              size_t cell_bytes, int n_clusters, int cl_size, cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e;
    if (lu_elem == 4) {
        e = arrow_config<float>(cl_size, n_clusters, st, cfg, attr);
        if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, campdev::k_arrow<float>, mt, a, s, scratch, cell_bytes);
    } else {
        e = arrow_config<double>(cl_size, n_clusters, st, cfg, attr);
        if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, campdev::k_arrow<double>, mt, a, s, scratch, cell_bytes);
    }
    return e;
}

cudaError_t camp_arrow_forcing(const DevMech &mt, const ArrowDev &a, long long n_cells, const double *state,
                               const double *env, double *f, cudaStream_t st) {
    campdev::k_arrow_forcing<<<(unsigned)n_cells, campdev::ARROW_NT, 0, st>>>(mt, a, n_cells, state, env, f);
    return cudaGetLastError();
}
