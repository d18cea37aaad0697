// Kernels of the batched solve and of its per-step test entry points,
// templated on the LU precision LT (float: mixed form, double: plain form),
// the lanes per cell G and the register slots per lane NPL; W selects the
// build with the water parameter's per-state work (mechanisms whose section
// constants carry powers of 1/L(y)), so that no other mechanism pays for it.
#pragma once
#include "cellsolve.cuh"
#include "launch.h"

namespace campdev {

template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G >= 32) {
        return 0xffffffffu;
    } else {
        const int sub = (threadIdx.x & 31) / G;
        return ((1u << G) - 1u) << (sub * G);
    }
}

// The whole solve: each group of G lanes integrates one cell at a time.  With
// `queue` null the mapping is static (cell = block * cpb + group); otherwise
// the groups take cells from the counter until it passes n_cells.
// Register caps: the FP32-LU form with one-warp cells is limited by
// registers and shared memory together (168 a lane fits 12 cells per SM;
// 224 fits 9); 64-thread cells with 4 slots take 168 in both forms
// (measured: FP32-LU 6 cells per SM, faster than 128 with spills or 225
// without a cap; FP64 form 7% faster than with 200); 128-thread cells take
// 168 in the FP64 form (3 cells per SM instead of 2: 7% faster despite
// spills; the FP32-LU form gains nothing); the FP64 form and the other
// block cells may take the architectural maximum.
template <int G, int NPL, typename LT, bool W>
__global__ void __maxnreg__((G == 64 && NPL == 4) || (G == 128 && sizeof(LT) == 8) ? 168
                            : ((sizeof(LT) == 8 || G > 32) ? 255 : (NPL >= 6 ? 224 : 168)))
    k_solve(DevMech m, SolveArgs a) {
    extern __shared__ __align__(16) char smem[];
    const int group = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned gm = group_mask<G>();
    const CellSmem L = cell_smem(m.n, m.R, m.n_rev, m.nlu, (int)sizeof(LT), m.n_part, m.n_pw, m.n_pw64);
    CellPtr<LT> c(smem + group * L.bytes, m);
    long long cell = a.queue ? 0 : (long long)blockIdx.x * a.cpb + group;
    for (;;) {
        if (a.queue) {
            if constexpr (G <= 32) {
                unsigned long long v = 0;
                if (lane == 0) v = atomicAdd(a.queue, 1ull);
                cell = (long long)__shfl_sync(gm, v, 0, G);
            } else {  // one cell per block: broadcast through shared memory
                __shared__ unsigned long long next;
                if (threadIdx.x == 0) next = atomicAdd(a.queue, 1ull);
                __syncthreads();
                cell = (long long)next;
                __syncthreads();
            }
        }
        if (cell >= a.n_cells) break;
        CellStats st, tot{0, 0, 0, 0, 0};
        int s = ST_OK;
        // one or more consecutive outer steps of dt, each an independent call
        // of the integrator (a cold start unless step sizes are carried);
        // with a trajectory, the state after each one is also written there
        for (int o = 0; o < a.n_outer && s == ST_OK; o++) {
            s = integrate_cell<G, NPL, LT, W>(m, c, a.state + cell * m.n, a.env + cell * m.n_env, a.dt, a.rtol,
                                              a.atol, a.atol_len, a.max_steps, a.hmin_frac,
                                              a.step ? a.step + cell : nullptr, lane, gm, st,
                                              a.traj ? a.traj + ((long long)o * a.n_cells + cell) * m.n : nullptr);
            tot.steps += st.steps;
            tot.newton += st.newton;
            tot.jac += st.jac;
            tot.errfail += st.errfail;
            tot.ordsum += st.ordsum;
            if (o + 1 < a.n_outer) gsync<G>(gm);  // the state written back is the next step's input
        }
        if (lane == 0) {
            a.status[cell] = s;
            if (a.stats) {
                int32_t *o = a.stats + 5 * cell;
                o[0] = tot.steps;
                o[1] = tot.newton;
                o[2] = tot.jac;
                o[3] = tot.errfail;
                o[4] = tot.ordsum;
            }
        }
        if (!a.queue) break;
        gsync<G>(gm);
    }
}

// Rate constants of every process of every cell, [cell][R] in process order.
template <int G>
__global__ void k_rates(DevMech m, long long n_cells, const double *env, double *kf, double *kr) {
    const long long cell = (long long)blockIdx.x * (blockDim.x / G) + threadIdx.x / G;
    const int lane = threadIdx.x % G;
    if (cell >= n_cells) return;
    for (int k = lane; k < m.R; k += G) {
        double a, b;
        rate_constant(m, k, env + cell * m.n_env, a, b);
        kf[cell * m.R + k] = a;
        kr[cell * m.R + k] = b;
    }
}

template <int G, int NPL, typename LT, bool W>
__device__ __forceinline__ void load_cell(const DevMech &m, const CellPtr<LT> &c, const double *y,
                                          const double *env, double (&yr)[NPL], int lane, unsigned gm) {
    for (int k = lane; k < m.R; k += G) {
        double a, b;
        rate_constant(m, k, env, a, b);
        c.kf[k] = a;
        const int rv = __ldg(m.rrev + k);
        if (rv >= 0) c.kr[rv] = b;
    }
#pragma unroll
    for (int s = 0; s < NPL; s++) {
        int p = lane + G * s;
        yr[s] = p < m.n ? y[__ldg(m.perm + p)] : 0.0;
        if (p < m.n) c.ys[p] = yr[s];
    }
    gsync<G>(gm);
    if constexpr (W) water_setup<G>(m, c.pw, env, lane, gm);
}

// f(y) of every cell, [cell][n] in declaration order.
template <int G, int NPL, typename LT, bool W>
__global__ void k_forcing(DevMech m, long long n_cells, const double *state, const double *env,
                          double *f_out) {
    extern __shared__ __align__(16) char smem[];
    const int group = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned gm = group_mask<G>();
    const long long cell = (long long)blockIdx.x * (blockDim.x / G) + group;
    if (cell >= n_cells) return;
    const CellSmem L = cell_smem(m.n, m.R, m.n_rev, m.nlu, (int)sizeof(LT), m.n_part, m.n_pw, m.n_pw64);
    CellPtr<LT> c(smem + group * L.bytes, m);
    double y[NPL], f[NPL];
    load_cell<G, NPL, LT, W>(m, c, state + cell * m.n, env + cell * m.n_env, y, lane, gm);
    eval_f<G, NPL, LT, W>(m, c, y, f, lane, gm);
#pragma unroll
    for (int s = 0; s < NPL; s++) {
        int p = lane + G * s;
        if (p < m.n) f_out[cell * m.n + __ldg(m.perm + p)] = f[s];
    }
}

// Jacobian values of every cell, [cell][nnzJ] in species-CSR order, computed
// in precision LT (the assembly precision of the corresponding solve form).
template <int G, int NPL, typename LT, bool W>
__global__ void k_jacobian(DevMech m, long long n_cells, const double *state, const double *env,
                           double *jac) {
    extern __shared__ __align__(16) char smem[];
    const int group = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned gm = group_mask<G>();
    const long long cell = (long long)blockIdx.x * (blockDim.x / G) + group;
    if (cell >= n_cells) return;
    const CellSmem L = cell_smem(m.n, m.R, m.n_rev, m.nlu, (int)sizeof(LT), m.n_part, m.n_pw, m.n_pw64);
    CellPtr<LT> c(smem + group * L.bytes, m);
    double y[NPL];
    load_cell<G, NPL, LT, W>(m, c, state + cell * m.n, env + cell * m.n_env, y, lane, gm);
    assemble<G, LT, W>(m, c, 0.0, lane, gm, 1, jac + cell * (long long)m.nnzJ);
}

// Solve (I - gamma J(y)) x = b for every cell with the device LU in
// precision LT; b and x [cell][n] in declaration order; status 4 on a
// tiny pivot (x then left unwritten).
template <int G, int NPL, typename LT, bool W>
__global__ void k_lu_solve(DevMech m, long long n_cells, const double *state, const double *env,
                           double gamma, const double *b, double *x, int *status) {
    extern __shared__ __align__(16) char smem[];
    const int group = threadIdx.x / G, lane = threadIdx.x % G;
    const unsigned gm = group_mask<G>();
    const long long cell = (long long)blockIdx.x * (blockDim.x / G) + group;
    if (cell >= n_cells) return;
    const CellSmem L = cell_smem(m.n, m.R, m.n_rev, m.nlu, (int)sizeof(LT), m.n_part, m.n_pw, m.n_pw64);
    CellPtr<LT> c(smem + group * L.bytes, m);
    double y[NPL];
    load_cell<G, NPL, LT, W>(m, c, state + cell * m.n, env + cell * m.n_env, y, lane, gm);
    assemble<G, LT, W>(m, c, gamma, lane, gm, 0, nullptr);
    bool ok = factor<G, LT>(m, c, lane, gm);
    if (lane == 0) status[cell] = ok ? 0 : ST_SINGULAR;
    if (!ok) return;
    for (int p = lane; p < m.n; p += G) c.x[p] = (LT)b[cell * m.n + __ldg(m.perm + p)];
    substitute<G, LT, subst_pivots<G, NPL, LT>()>(m, c, lane, gm);
    for (int p = lane; p < m.n; p += G) x[cell * m.n + __ldg(m.perm + p)] = (double)c.x[p];
}

}  // namespace campdev
