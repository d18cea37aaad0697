// The block-arrow solve of particle-resolved cells (arrow.h): one cell per
// thread-block cluster, its particles spread over the cluster's threads.
//
// A thread owns the particles p = lane, lane + L, ... (L = threads of the
// cluster) for the whole solve: their Nordsieck rows, corrections, weights,
// rate constants and LU blocks live in global memory laid out [component][P],
// so a warp's loads and stores of one component are contiguous, and no other
// thread ever touches them.  The gas species (at most 32) are the lanes of
// warp 0 of the cluster's first CTA and live in its registers.  The two meet
// only through the arrow: particle -> gas sums (forcing of the exchanged gas
// species, the forward substitution's gas right-hand side, the Schur
// complement of the gas block) go through fixed-order cluster reductions in
// distributed shared memory, and gas -> particle values (the gas state, the
// gas part of each solve) are written into every CTA's shared memory.  Every
// controller decision is taken on reduced values that are bit-identical in
// every thread, so the cluster follows one step sequence; the results depend
// only on the launch shape (threads and CTAs per cluster), not on timing.
//
// Linear algebra (paper Sect. 2.4.1; KLU's sparse LU as prior art): with the
// particle species first, M = I - gamma J = [M_PP M_PG; M_GP M_GG] with
// M_PP block-diagonal.  Per particle: M_pp = L_p U_p (dense, static pivots),
// U_pG = L_p^-1 M_pG, L_Gp = M_Gp U_p^-1; the gas block S = M_GG - sum_p
// L_Gp U_pG.  Solve: y_p = L_p^-1 b_p, b_G' = b_G - sum_p L_Gp y_p,
// x_G = S^-1 b_G', x_p = U_p^-1 (y_p - U_pG x_G).
#pragma once
#include <cooperative_groups.h>

#include "arrow.h"
#include "cellsolve.cuh"

namespace campdev {
namespace cg = cooperative_groups;

constexpr int ARROW_NT = 256;     // threads per CTA
constexpr int ARROW_MAX_CL = 16;  // CTAs per cluster
constexpr int ARROW_MAX_RG = 64;  // gas processes
constexpr int ARROW_RED = CAMP_ARROW_MAX_C * CAMP_ARROW_MAX_C + 2;  // values of one reduction
constexpr int ARROW_MAX_LOC = CAMP_ARROW_MAX_PHI + CAMP_ARROW_MAX_C;

template <typename LT>
struct ArrowSmem {
    double red[2][ARROW_MAX_CL][ARROW_RED];  // CTA 0: the CTAs' partial sums (two buffers)
    double part[ARROW_NT / 32][ARROW_RED];   // this CTA's warps' partial sums
    double res[ARROW_RED];                   // this CTA's copy of a reduction's result
    double ygas[CAMP_ARROW_MAX_GAS];         // gas state at the current iterate (every CTA)
    LT xgas[CAMP_ARROW_MAX_GAS];             // gas part of the current solve (every CTA)
    // CTA 0, warp 0: the gas processes and the factored gas block
    double kfg[ARROW_MAX_RG], krg[ARROW_MAX_RG], rsg[ARROW_MAX_RG];
    LT S[CAMP_ARROW_MAX_GAS * (CAMP_ARROW_MAX_GAS + 1)];
    LT xs[CAMP_ARROW_MAX_GAS];
    long long next_cell;
};

// Per-cell scratch in global memory (one cell per cluster at a time).
template <typename LT>
struct ArrowScratch {
    double *zp;   // [QMAX+1][n_phi][P] Nordsieck rows
    double *ep;   // [n_phi][P] correction
    double *epp;  // [n_phi][P] previous step's correction
    double *wp;   // [n_phi][P] error weights
    double *fp;   // [n_phi][P] forcing (initial step and restarts)
    double *kfp;  // [Rp][P]
    double *krp;  // [Rp][P]
    LT *lu;       // [blk][P]
    LT *xp;       // [n_phi][P] solve scratch
};

__host__ __device__ inline size_t arrow_cell_bytes(const ArrowDev &a, int lu_elem) {
    const size_t P = (size_t)a.P, np = (size_t)a.n_phi;
    size_t d = ((size_t)(QMAX + 1) * np + 4 * np + 2 * (size_t)a.Rp) * P * 8;
    size_t l = ((size_t)a.blk + np) * P * (size_t)lu_elem;
    return ((d + l) + 255) & ~(size_t)255;
}

template <typename LT>
__device__ inline ArrowScratch<LT> arrow_scratch(const ArrowDev &a, char *base) {
    ArrowScratch<LT> c;
    const size_t P = (size_t)a.P, np = (size_t)a.n_phi;
    double *d = (double *)base;
    c.zp = d; d += (size_t)(QMAX + 1) * np * P;
    c.ep = d; d += np * P;
    c.epp = d; d += np * P;
    c.wp = d; d += np * P;
    c.fp = d; d += np * P;
    c.kfp = d; d += (size_t)a.Rp * P;
    c.krp = d; d += (size_t)a.Rp * P;
    LT *l = (LT *)d;
    c.lu = l; l += (size_t)a.blk * P;
    c.xp = l;
    return c;
}

// Cluster-wide sums of K values (K <= ARROW_RED), in a fixed order: warps by
// xor shuffles (lane 0's value), the CTA's warps in order, then the CTAs in
// rank order from CTA 0's shared memory.  Every thread gets identical bits in
// out (want = true).  Two buffers alternate (par), so a buffer is rewritten
// only after every thread has passed the next reduction's barrier.
template <typename LT>
__device__ void cluster_sum(ArrowSmem<LT> &sm, const cg::cluster_group &cl, const double *v, int K, int &par,
                            double *out) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = 0; j < K; j++) {
        double x = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sm.part[warp][j] = x;
    }
    __syncthreads();
    const unsigned r = cl.block_rank();
    if (tid < K) {
        double s = 0.0;
        for (int w = 0; w < ARROW_NT / 32; w++) s += sm.part[w][tid];
        double *dst = cl.map_shared_rank(&sm.red[par][r][tid], 0);
        *dst = s;
    }
    cl.sync();
    if (tid < K) {
        const double *src = cl.map_shared_rank(&sm.red[par][0][0], 0);
        double s = 0.0;
        for (unsigned q = 0; q < cl.num_blocks(); q++) s += src[q * ARROW_RED + tid];
        sm.res[tid] = s;
    }
    __syncthreads();
    for (int j = 0; j < K; j++) out[j] = sm.res[j];
    par ^= 1;
}

template <typename LT>
__device__ inline double cluster_sum1(ArrowSmem<LT> &sm, const cg::cluster_group &cl, double v, int &par) {
    double o;
    cluster_sum(sm, cl, &v, 1, par, &o);
    return o;
}

// rate of a process at local values y (factors f0..f2 forward, b0..b2 reverse)
__device__ __forceinline__ double arrow_rate(const int4 r1, const int4 r2, double kf, double kr, const double *y) {
    double a = kf;
    if (r1.x >= 0) a *= y[r1.x];
    if (r1.y >= 0) a *= y[r1.y];
    if (r1.z >= 0) a *= y[r1.z];
    if (r2.w) {
        double b = kr;
        if (r2.x >= 0) b *= y[r2.x];
        if (r2.y >= 0) b *= y[r2.y];
        if (r2.z >= 0) b *= y[r2.z];
        a -= b;
    }
    return a;
}

// forcing of one particle at local values yl: fl[0..n_loc) (its phase species,
// then the gas species it exchanges with), processes in order
__device__ inline void arrow_particle_forcing(const ArrowDev &a, int p, const double *kfp, const double *krp,
                                              const double *yl, double *fl) {
    for (int i = 0; i < a.n_loc; i++) fl[i] = 0.0;
    for (int k = 0; k < a.Rp; k++) {
        const int4 r0 = __ldg(a.prec + 3 * k), r1 = __ldg(a.prec + 3 * k + 1), r2 = __ldg(a.prec + 3 * k + 2);
        const double r = arrow_rate(r1, r2, kfp[(size_t)k * a.P + p], krp[(size_t)k * a.P + p], yl);
        for (int q = r0.w; q < r1.w; q++) fl[__ldg(a.st_sp + q)] += __ldg(a.st_nu + q) * r;
    }
}

// Jacobian of one particle's processes at yl, as M = I - gamma J pieces:
// the particle block and U_pG / L_Gp (before elimination) into the
// particle's LU storage, the gas-gas part into gg [n_c][n_c] (added)
template <typename LT>
__device__ inline void arrow_particle_assemble(const ArrowDev &a, int p, const double *kfp, const double *krp,
                                               const LT *yl, LT gamma, LT *lu, LT *gg) {
    const int np = a.n_phi, nc = a.n_c;
    const size_t P = (size_t)a.P;
    LT *B = lu, *UpG = lu + (size_t)np * np * P, *LGp = UpG + (size_t)np * nc * P;
    for (int i = 0; i < np; i++)
        for (int j = 0; j < np; j++) B[((size_t)i * np + j) * P + p] = (i == j) ? (LT)1 : (LT)0;
    for (int t = 0; t < np * nc; t++) UpG[(size_t)t * P + p] = (LT)0;
    for (int t = 0; t < nc * np; t++) LGp[(size_t)t * P + p] = (LT)0;
    for (int k = 0; k < a.Rp; k++) {
        const int4 r0 = __ldg(a.prec + 3 * k), r1 = __ldg(a.prec + 3 * k + 1), r2 = __ldg(a.prec + 3 * k + 2);
        const int fac[6] = {r1.x, r1.y, r1.z, r2.x, r2.y, r2.z};
        const LT kf = (LT)kfp[(size_t)k * P + p], kr = (LT)krp[(size_t)k * P + p];
        LT d[6];
#pragma unroll
        for (int q = 0; q < 6; q++) {
            d[q] = (LT)0;
            if (fac[q] < 0 || (q >= 3 && !r2.w)) continue;
            LT v = q < 3 ? kf : -kr;
            const int side = q < 3 ? 0 : 3;
#pragma unroll
            for (int q2 = 0; q2 < 3; q2++)
                if (side + q2 != q && fac[side + q2] >= 0) v *= yl[fac[side + q2]];
            d[q] = v;
        }
        for (int e = r0.w; e < r1.w; e++) {
            const int i = __ldg(a.st_sp + e);
            const LT nu = (LT)__ldg(a.st_nu + e);
#pragma unroll
            for (int q = 0; q < 6; q++) {
                if (fac[q] < 0 || (q >= 3 && !r2.w)) continue;
                const int j = fac[q];
                const LT v = -gamma * nu * d[q];  // M = I - gamma J
                if (i < np && j < np) B[((size_t)i * np + j) * P + p] += v;
                else if (i < np) UpG[((size_t)i * nc + (j - np)) * P + p] += v;
                else if (j < np) LGp[((size_t)(i - np) * np + j) * P + p] += v;
                else gg[(i - np) * nc + (j - np)] += v;
            }
        }
    }
}

// Eliminate one particle: M_pp = L U in place (static pivots, reciprocal
// pivots stored), U_pG <- L^-1 M_pG, L_Gp <- M_Gp U^-1, and gg -= L_Gp U_pG.
// Returns true on a tiny or non-finite pivot.
template <typename LT>
__device__ inline bool arrow_particle_factor(const ArrowDev &a, int p, LT *lu, LT *gg) {
    const int np = a.n_phi, nc = a.n_c;
    const size_t P = (size_t)a.P;
    LT *B = lu, *UpG = lu + (size_t)np * np * P, *LGp = UpG + (size_t)np * nc * P;
    auto b = [&](int i, int j) -> LT & { return B[((size_t)i * np + j) * P + p]; };
    auto u = [&](int i, int c) -> LT & { return UpG[((size_t)i * nc + c) * P + p]; };
    auto l = [&](int c, int j) -> LT & { return LGp[((size_t)c * np + j) * P + p]; };
    bool bad = false;
    for (int k = 0; k < np; k++) {
        const LT piv = b(k, k);
        bad |= bad_pivot(piv);
        const LT rp = recip(piv);
        b(k, k) = rp;
        for (int i = k + 1; i < np; i++) {
            const LT m = b(i, k) * rp;
            b(i, k) = m;
            if (m == (LT)0) continue;
            for (int j = k + 1; j < np; j++) b(i, j) -= m * b(k, j);
            for (int c = 0; c < nc; c++) u(i, c) -= m * u(k, c);  // U_pG = L^-1 M_pG, row by row
        }
        for (int c = 0; c < nc; c++) {  // L_Gp = M_Gp U^-1, column k
            const LT m = l(c, k) * rp;
            l(c, k) = m;
            if (m == (LT)0) continue;
            for (int j = k + 1; j < np; j++) l(c, j) -= m * b(k, j);
        }
    }
    for (int c = 0; c < nc; c++)
        for (int c2 = 0; c2 < nc; c2++) {
            LT s = (LT)0;
            for (int j = 0; j < np; j++) s += l(c, j) * u(j, c2);
            gg[c * nc + c2] -= s;
        }
    return bad;
}

// Forward part for one particle: y_p = L^-1 b_p in xp (b_p given there),
// and sum_p L_Gp y_p added to fw [n_c]
template <typename LT>
__device__ inline void arrow_particle_forward(const ArrowDev &a, int p, const LT *lu, LT *xp, double *fw) {
    const int np = a.n_phi, nc = a.n_c;
    const size_t P = (size_t)a.P;
    const LT *B = lu, *LGp = lu + (size_t)np * np * P + (size_t)np * nc * P;
    LT y[CAMP_ARROW_MAX_PHI];
    for (int i = 0; i < np; i++) {
        LT s = xp[(size_t)i * P + p];
        for (int j = 0; j < i; j++) s -= B[((size_t)i * np + j) * P + p] * y[j];
        y[i] = s;
        xp[(size_t)i * P + p] = s;
    }
    for (int c = 0; c < nc; c++) {
        LT s = (LT)0;
        for (int j = 0; j < np; j++) s += LGp[((size_t)c * np + j) * P + p] * y[j];
        fw[c] += (double)s;
    }
}

// Backward part for one particle: x_p = U^-1 (y_p - U_pG x_G) in xp
template <typename LT>
__device__ inline void arrow_particle_backward(const ArrowDev &a, int p, const LT *lu, LT *xp, const LT *xgas) {
    const int np = a.n_phi, nc = a.n_c;
    const size_t P = (size_t)a.P;
    const LT *B = lu, *UpG = lu + (size_t)np * np * P;
    LT x[CAMP_ARROW_MAX_PHI];
    for (int i = np - 1; i >= 0; i--) {
        LT s = xp[(size_t)i * P + p];
        for (int c = 0; c < nc; c++) s -= UpG[((size_t)i * nc + c) * P + p] * xgas[__ldg(a.coupled + c)];
        for (int j = i + 1; j < np; j++) s -= B[((size_t)i * np + j) * P + p] * x[j];
        x[i] = s * B[((size_t)i * np + i) * P + p];
        xp[(size_t)i * P + p] = x[i];
    }
}

// ---- one cell over [0, dt] ----------------------------------------------------
// The step controller of integrate_cell (cellsolve.cuh), step for step, on
// the block-arrow storage.  Returns the status (uniform over the cluster).
template <typename LT>
__device__ int arrow_integrate_cell(const DevMech &mt, const ArrowDev &a, ArrowSmem<LT> &sm,
                                    const cg::cluster_group &cl, char *scratch, double *__restrict__ y_cell,
                                    const double *__restrict__ env, double dt, double rtol,
                                    const double *__restrict__ atol, int atol_len, int max_steps, double hmin_frac,
                                    double *step_io, int &par, CellStats &st, double *__restrict__ y_copy) {
    constexpr bool EXACT = sizeof(LT) == 8;
    using C = Ctl<EXACT>;
    const ArrowScratch<LT> c = arrow_scratch<LT>(a, scratch);
    const int tid = threadIdx.x;
    const int L = (int)cl.num_blocks() * ARROW_NT;
    const int lane = (int)cl.block_rank() * ARROW_NT + tid;
    const bool gas = cl.block_rank() == 0 && tid < 32;  // warp 0 of CTA 0: the gas species
    const bool gas_own = gas && tid < a.n_g;            // this lane's gas species: tid
    const int np = a.n_phi, nc = a.n_c;
    const size_t P = (size_t)a.P;
    const double h_in = step_io ? *step_io : 0.0;
    st.steps = st.newton = st.jac = st.errfail = st.ordsum = 0;
    auto Z = [&](int j, int i, int p) -> double & { return c.zp[((size_t)j * np + i) * P + p]; };
    auto E = [&](int i, int p) -> double & { return c.ep[(size_t)i * P + p]; };
    auto EP = [&](int i, int p) -> double & { return c.epp[(size_t)i * P + p]; };
    auto Wt = [&](int i, int p) -> double & { return c.wp[(size_t)i * P + p]; };
    auto F = [&](int i, int p) -> double & { return c.fp[(size_t)i * P + p]; };
    auto X = [&](int i, int p) -> LT & { return c.xp[(size_t)i * P + p]; };
    auto species = [&](int i, int p) { return a.n_g + p * np + i; };
    auto atol_of = [&](int s) { return atol_len == 1 ? __ldg(atol) : __ldg(atol + s); };
    // the gas lane's rows
    double zg[QMAX + 1], eg = 0.0, epg = 0.0, wg = 0.0, fg = 0.0;

    // inputs must be finite
    double nbad = 0.0;
    for (int i = lane; i < a.n_env; i += L) nbad += !finite_bits(env[i]);
    for (int p = lane; p < a.P; p += L)
        for (int i = 0; i < np; i++) {
            const double v = y_cell[species(i, p)];
            nbad += !finite_bits(v);
            Z(0, i, p) = v;
            for (int j = 1; j <= QMAX; j++) Z(j, i, p) = 0.0;
            E(i, p) = EP(i, p) = 0.0;
        }
#pragma unroll
    for (int j = 0; j <= QMAX; j++) zg[j] = 0.0;
    if (gas_own) {
        zg[0] = y_cell[tid];
        nbad += !finite_bits(zg[0]);
    }
    auto fail_early = [&](int code) {
        if (step_io && lane == 0) *step_io = 0.0;
        return code;
    };
    if (cluster_sum1(sm, cl, nbad, par) != 0.0) return fail_early(ST_NONFINITE);

    // rate constants: the particles' (own), the gas processes' (gas warp)
    for (int p = lane; p < a.P; p += L) {
        const double *sec = env + a.E0 + 3 * p;
        for (int k = 0; k < a.Rp; k++) {
            double kf, kr;
            rate_constant_at(mt, __ldg(a.prec + 3 * k).x, env, sec, kf, kr);
            c.kfp[(size_t)k * P + p] = kf;
            c.krp[(size_t)k * P + p] = kr;
        }
    }
    if (gas)
        for (int k = tid; k < a.Rg; k += 32) {
            double kf, kr;
            rate_constant_at(mt, __ldg(a.grec + 3 * k).x, env, env, kf, kr);
            sm.kfg[k] = kf;
            sm.krg[k] = kr;
        }

    auto set_weights = [&]() {
        for (int p = lane; p < a.P; p += L)
            for (int i = 0; i < np; i++) Wt(i, p) = C::weight(rtol, Z(0, i, p), atol_of(species(i, p)));
        if (gas_own) wg = C::weight(rtol, zg[0], atol_of(tid));
    };

    // publish the gas state (gas lanes: their value) to every CTA
    auto publish_gas = [&](double yv) {
        if (gas)
            for (unsigned r = 0; r < cl.num_blocks(); r++)
                if (tid < a.n_g) *cl.map_shared_rank(&sm.ygas[tid], r) = yv;
        cl.sync();
    };
    // the gas processes' rates at the published gas state (gas warp)
    auto gas_rates = [&]() {
        if (gas) {
            for (int k = tid; k < a.Rg; k += 32) {
                const int4 r1 = __ldg(a.grec + 3 * k + 1), r2 = __ldg(a.grec + 3 * k + 2);
                sm.rsg[k] = arrow_rate(r1, r2, sm.kfg[k], sm.krg[k], sm.ygas);
            }
            __syncwarp();
        }
    };
    // the gas lane's forcing: its gas processes, then the particles' sums
    auto gas_forcing = [&](const double *red) {
        double s = 0.0;
        for (int q = __ldg(a.gf_ptr + tid); q < __ldg(a.gf_ptr + tid + 1); q++)
            s += __ldg(a.gf_nu + q) * sm.rsg[__ldg(a.gf_k + q)];
        for (int q = 0; q < nc; q++)
            if (__ldg(a.coupled + q) == tid) s += red[q];
        return s;
    };
    // f at y = z0 + b f (b = 0: at z0), into F (particles) and fg (gas
    // lanes); with diff, F and fg are kept and the difference f(y) - f
    // goes to EP and epg instead.  Returns the count of non-finite values.
    auto eval_f = [&](double b, bool diff) -> double {
        publish_gas(gas_own ? zg[0] + b * fg : 0.0);
        double part[CAMP_ARROW_MAX_C + 1];
        for (int q = 0; q <= nc; q++) part[q] = 0.0;
        double yl[ARROW_MAX_LOC], fl[ARROW_MAX_LOC];
        for (int p = lane; p < a.P; p += L) {
            for (int i = 0; i < np; i++) yl[i] = Z(0, i, p) + b * F(i, p);
            for (int q = 0; q < nc; q++) yl[np + q] = sm.ygas[__ldg(a.coupled + q)];
            arrow_particle_forcing(a, p, c.kfp, c.krp, yl, fl);
            for (int i = 0; i < np; i++) {
                part[nc] += !finite_bits(fl[i]);
                if (diff) EP(i, p) = fl[i] - F(i, p);
                else F(i, p) = fl[i];
            }
            for (int q = 0; q < nc; q++) part[q] += fl[np + q];
        }
        gas_rates();
        double red[CAMP_ARROW_MAX_C + 1];
        cluster_sum(sm, cl, part, nc + 1, par, red);
        double gbad = 0.0;
        if (gas_own) {
            const double f1 = gas_forcing(red);
            if (diff) epg = f1 - fg;
            else fg = f1;
            gbad = !finite_bits(f1);
        }
        return red[nc] + cluster_sum1(sm, cl, gbad, par);
    };

    const double T = dt, hmin = hmin_frac * dt;
    set_weights();
    if (eval_f(0.0, false) != 0.0) return fail_early(ST_NONFINITE);

    // weighted sums of squares over every species (cluster reduction)
    auto sumsq2 = [&](auto va, auto vb, double gva, double gvb, double *out2) {
        double s[2] = {0.0, 0.0};
        for (int p = lane; p < a.P; p += L)
            for (int i = 0; i < np; i++) {
                const double w = Wt(i, p);
                const double x = va(i, p) * w, y = vb(i, p) * w;
                s[0] += x * x;
                s[1] += y * y;
            }
        if (gas_own) {
            s[0] += (gva * wg) * (gva * wg);
            s[1] += (gvb * wg) * (gvb * wg);
        }
        cluster_sum(sm, cl, s, 2, par, out2);
    };
    auto rms = [&](double s) { return sqrt(s / (double)a.n); };

    double h;
    if (h_in > 0.0) {
        h = fmin(h_in, T);
    } else {
        double s2[2];
        sumsq2([&](int i, int p) { return Z(0, i, p); }, [&](int i, int p) { return F(i, p); }, zg[0], fg, s2);
        const double d0 = rms(s2[0]), d1 = rms(s2[1]);
        double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
        if (h0 > T) h0 = T;
        eval_f(h0, true);  // f(z0 + h0 f0) - f0 into EP (free until the first step ends)
        sumsq2([&](int i, int p) { return EP(i, p); }, [&](int i, int p) { return 0.0; }, epg, 0.0, s2);
        const double d2 = rms(s2[0]) / h0;
        const double dm = d1 > d2 ? d1 : d2;
        const double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : sqrt(0.01 / dm);
        h = fmin(100.0 * h0, h1);
        if (!(h <= T)) h = T;
    }
    for (int p = lane; p < a.P; p += L)
        for (int i = 0; i < np; i++) {
            Z(1, i, p) = h * F(i, p);
            E(i, p) = 0.0;
        }
    if (gas_own) zg[1] = h * fg;
    eg = 0.0;

    // Nordsieck operations on every own row (the rows of one species in
    // registers, the loops unrolled over QMAX with the order as a guard)
    auto pascal = [&](double (&zz)[QMAX + 1][1], int q, bool up) {
        if (up) nord_predict<1>(zz, q);
        else nord_retract<1>(zz, q);
    };
    auto nord_apply = [&](int q, bool up) {
        for (int p = lane; p < a.P; p += L)
            for (int i = 0; i < np; i++) {
                double zz[QMAX + 1][1];
#pragma unroll
                for (int j = 0; j <= QMAX; j++) zz[j][0] = j <= q ? Z(j, i, p) : 0.0;
                pascal(zz, q, up);
#pragma unroll
                for (int j = 0; j < QMAX; j++)
                    if (j < q) Z(j, i, p) = zz[j][0];
            }
        if (gas_own) {
            double zz[QMAX + 1][1];
#pragma unroll
            for (int j = 0; j <= QMAX; j++) zz[j][0] = zg[j];
            pascal(zz, q, up);
#pragma unroll
            for (int j = 0; j <= QMAX; j++) zg[j] = zz[j][0];
        }
    };
    auto predict = [&](int q) { nord_apply(q, true); };
    auto retract = [&](int q) { nord_apply(q, false); };
    auto rescale = [&](int q, double eta) {
        for (int p = lane; p < a.P; p += L)
            for (int i = 0; i < np; i++) {
                double f = 1.0;
                for (int j = 1; j <= q; j++) {
                    f *= eta;
                    Z(j, i, p) *= f;
                }
            }
        if (gas_own) {
            double f = 1.0;
            for (int j = 1; j <= q; j++) {
                f *= eta;
                zg[j] *= f;
            }
        }
    };

    int q = 1, qwait = 2, nst = 0, nst_lu = 0;
    double h_held = h;
    bool have_lu = false, need_setup = true, ep_valid = false;
    double t = 0.0, gamma_lu = 0.0, rgamma_lu = 0.0;
    int status = ST_OK;
    constexpr double NEWTON_TOL2 = NEWTON_TOL * NEWTON_TOL;
    constexpr double RHO_DIV2 = RHO_DIV * RHO_DIV;

    // J at z0 and the factorisation of M = I - gamma J (particle blocks, then
    // the gas block); returns true if every pivot is usable
    auto setup = [&](double gamma) -> bool {
        publish_gas(gas_own ? zg[0] : 0.0);
        const LT g = (LT)gamma;
        double part[ARROW_RED];
        const int K = nc * nc + 1;
        for (int v = 0; v < K; v++) part[v] = 0.0;
        LT gg[CAMP_ARROW_MAX_C * CAMP_ARROW_MAX_C];
        LT yl[ARROW_MAX_LOC];
        for (int p = lane; p < a.P; p += L) {
            for (int i = 0; i < np; i++) yl[i] = (LT)Z(0, i, p);
            for (int k = 0; k < nc; k++) yl[np + k] = (LT)sm.ygas[__ldg(a.coupled + k)];
            for (int v = 0; v < nc * nc; v++) gg[v] = (LT)0;
            arrow_particle_assemble<LT>(a, p, c.kfp, c.krp, yl, g, c.lu, gg);
            const bool bad = arrow_particle_factor<LT>(a, p, c.lu, gg);
            for (int v = 0; v < nc * nc; v++) part[v] += (double)gg[v];
            part[nc * nc] += bad ? 1.0 : 0.0;
        }
        double red[ARROW_RED];
        cluster_sum(sm, cl, part, K, par, red);
        // the gas block S = I - gamma J_gas + the particles' sums, factored by
        // the gas warp (lane i owns row i)
        double bad_gas = 0.0;
        if (gas) {
            const int ng = a.n_g, LDS = ng + 1;
            if (tid < ng) {
                for (int j = 0; j < ng; j++) sm.S[tid * LDS + j] = (tid == j) ? (LT)1 : (LT)0;
                for (int e = __ldg(a.gf_ptr + tid); e < __ldg(a.gf_ptr + tid + 1); e++) {
                    const int k = __ldg(a.gf_k + e);
                    const LT nu = (LT)__ldg(a.gf_nu + e);
                    const int4 r1 = __ldg(a.grec + 3 * k + 1), r2 = __ldg(a.grec + 3 * k + 2);
                    const int fac[6] = {r1.x, r1.y, r1.z, r2.x, r2.y, r2.z};
                    for (int qq = 0; qq < 6; qq++) {
                        if (fac[qq] < 0 || (qq >= 3 && !r2.w)) continue;
                        LT v = qq < 3 ? (LT)sm.kfg[k] : -(LT)sm.krg[k];
                        const int side = qq < 3 ? 0 : 3;
                        for (int q2 = 0; q2 < 3; q2++)
                            if (side + q2 != qq && fac[side + q2] >= 0) v *= (LT)sm.ygas[fac[side + q2]];
                        sm.S[tid * LDS + fac[qq]] -= g * nu * v;
                    }
                }
                for (int c1 = 0; c1 < nc; c1++)
                    if (__ldg(a.coupled + c1) == tid)
                        for (int c2 = 0; c2 < nc; c2++)
                            sm.S[tid * LDS + __ldg(a.coupled + c2)] += (LT)red[c1 * nc + c2];
            }
            __syncwarp();
            bool bad = false;
            for (int k = 0; k < ng; k++) {
                const LT piv = sm.S[k * LDS + k];
                bad |= bad_pivot(piv);
                const LT rp = recip(piv);
                if (tid > k && tid < ng) {
                    const LT m = sm.S[tid * LDS + k] * rp;
                    sm.S[tid * LDS + k] = m;
                    for (int j = k + 1; j < ng; j++) sm.S[tid * LDS + j] -= m * sm.S[k * LDS + j];
                }
                __syncwarp();
                if (tid == 0) sm.S[k * LDS + k] = rp;
                __syncwarp();
            }
            bad_gas = (tid == 0 && bad) ? 1.0 : 0.0;
        }
        return red[nc * nc] + cluster_sum1(sm, cl, bad_gas, par) == 0.0;
    };

    while (t < T) {
        if (nst >= max_steps) { status = ST_MAXSTEPS; break; }
        // the weights of this step: set before the loop for the first step,
        // by the previous step's accept pass for the others (z0 is not
        // changed between the two)
        int nef = 0, ncf = 0;
        bool last = false;
        double err2 = 0.0;
        bool accepted = false;
        while (!accepted) {
            last = false;
            h_held = h;
            if (t + h >= T) {
                if (t + h > T) {
                    double eta = (T - t) / h;
                    rescale(q, eta);
                    h = T - t;
                }
                last = true;
            }
            predict(q);
            const double rl1 = mt.inv_l1[q];
            const double gamma = C::ratio(h, mt.lcoef[q][1], rl1);
            bool jcur = false, lu_fail = false;
            if (!have_lu || need_setup || nst >= nst_lu + MSBJ ||
                fabs(C::ratio(gamma, gamma_lu, rgamma_lu) - 1.0) > DGMAX) {
                lu_fail = !setup(gamma);
                st.jac++;
                gamma_lu = gamma;
                rgamma_lu = 1.0 / gamma;
                nst_lu = nst;
                have_lu = !lu_fail;
                need_setup = false;
                jcur = true;
            }
            bool conv = false;
            double esum = 0.0;  // sum of (e w)^2 after the latest iteration
            if (!lu_fail) {
                double dprev2 = 0.0;
                eg = 0.0;  // the particles' e is read as zero in the first iteration
                const LT scale = (gamma != gamma_lu)
                                     ? (LT)2 / ((LT)1 + to_lu<LT>(C::ratio(gamma, gamma_lu, rgamma_lu)))
                                     : (LT)1;
                for (int it = 0; it < NEWTON_MAXIT; it++) {
                    publish_gas(gas_own ? zg[0] + eg : 0.0);  // y = z0 + e
                    st.newton++;
                    // particles: forcing, right side, forward substitution
                    double part[2 * CAMP_ARROW_MAX_C + 1];
                    for (int v = 0; v <= 2 * nc; v++) part[v] = 0.0;
                    double yl[ARROW_MAX_LOC], fl[ARROW_MAX_LOC];
                    for (int p = lane; p < a.P; p += L) {
                        for (int i = 0; i < np; i++) yl[i] = Z(0, i, p) + (it ? E(i, p) : 0.0);
                        for (int k = 0; k < nc; k++) yl[np + k] = sm.ygas[__ldg(a.coupled + k)];
                        arrow_particle_forcing(a, p, c.kfp, c.krp, yl, fl);
                        for (int i = 0; i < np; i++) {
                            part[2 * nc] += !finite_bits(fl[i]);
                            X(i, p) = to_lu<LT>(-((it ? E(i, p) : 0.0) - gamma * fl[i] + Z(1, i, p) * rl1));
                        }
                        for (int k = 0; k < nc; k++) part[k] += fl[np + k];
                        arrow_particle_forward<LT>(a, p, c.lu, c.xp, part + nc);
                    }
                    gas_rates();
                    double red[2 * CAMP_ARROW_MAX_C + 1];
                    cluster_sum(sm, cl, part, 2 * nc + 1, par, red);
                    // gas: forcing, right side, y_G = b_G - sum L_Gp y_p, x_G = S^-1 y_G
                    double gnf = 0.0;
                    if (gas) {
                        const int ng = a.n_g, LDS = ng + 1;
                        if (gas_own) {
                            LT fwd = (LT)0;
                            for (int k = 0; k < nc; k++)
                                if (__ldg(a.coupled + k) == tid) fwd = (LT)red[nc + k];
                            fg = gas_forcing(red);
                            gnf = !finite_bits(fg);
                            sm.xs[tid] = to_lu<LT>(-(eg - gamma * fg + zg[1] * rl1)) - fwd;
                        }
                        __syncwarp();
                        for (int k = 0; k < ng; k++) {  // unit lower
                            const LT xk = sm.xs[k];
                            __syncwarp();
                            if (tid > k && tid < ng) sm.xs[tid] -= sm.S[tid * LDS + k] * xk;
                            __syncwarp();
                        }
                        for (int k = ng - 1; k >= 0; k--) {  // upper, reciprocal pivots
                            if (tid == k) sm.xs[k] *= sm.S[k * LDS + k];
                            __syncwarp();
                            const LT xk = sm.xs[k];
                            if (tid < k) sm.xs[tid] -= sm.S[tid * LDS + k] * xk;
                            __syncwarp();
                        }
                        for (unsigned r = 0; r < cl.num_blocks(); r++)
                            if (tid < ng) *cl.map_shared_rank(&sm.xgas[tid], r) = sm.xs[tid];
                    }
                    cl.sync();
                    // particles: backward substitution, the update, its norm
                    // and the weighted sum of squares of e (the error test's,
                    // in the same order as a pass of its own would take)
                    double s2[3] = {0.0, red[2 * nc] + gnf, 0.0};
                    for (int p = lane; p < a.P; p += L) {
                        arrow_particle_backward<LT>(a, p, c.lu, c.xp, sm.xgas);
                        for (int i = 0; i < np; i++) {
                            LT xl = X(i, p) * scale;
                            const double en = (it ? E(i, p) : 0.0) + from_lu(xl), wv = Wt(i, p);
                            E(i, p) = en;
                            s2[0] += (double)upd_term(xl, wv);
                            s2[1] += !isfinite(xl);
                            const double v = en * wv;
                            s2[2] += v * v;
                        }
                    }
                    if (gas_own) {
                        LT xl = sm.xgas[tid] * scale;
                        eg += from_lu(xl);
                        s2[0] += (double)upd_term(xl, wg);
                        s2[1] += !isfinite(xl);
                        s2[2] += (eg * wg) * (eg * wg);
                    }
                    double r2[3];
                    cluster_sum(sm, cl, s2, 3, par, r2);
                    esum = r2[2];
                    if (r2[1] != 0.0) break;  // non-finite forcing or update
                    // (the update's norm: summed in FP64 here; the mixed form
                    // compares squares, the FP64 form the norm itself)
                    const double dn2 = EXACT ? sqrt(r2[0] / (double)a.n) : r2[0] / (double)a.n;
                    if (!isfinite(dn2)) break;
                    double test2 = dn2;
                    if (it > 0) {
                        const double rho2 = dn2 / dprev2;
                        if (rho2 > (EXACT ? RHO_DIV : RHO_DIV2)) break;
                        if (rho2 < 1.0) test2 = dn2 * rho2;
                    }
                    if (test2 <= (EXACT ? NEWTON_TOL : NEWTON_TOL2)) { conv = true; break; }
                    dprev2 = dn2;
                }
            }
            if (!conv) {
                retract(q);
                if (!jcur) { need_setup = true; continue; }
                if (++ncf >= MAX_NCF) { status = lu_fail ? ST_SINGULAR : ST_NEWTON; break; }
                h *= ETA_CF;
                if (h < hmin) { status = ST_ERRTEST; break; }
                rescale(q, ETA_CF);
                need_setup = true;
                qwait = q + 1;
                continue;
            }
            err2 = C::norm(mt.ecoef[q], mt.ecoef2[q], esum, a.n, 1.0 / (double)a.n);
            if (err2 > 1.0) {
                retract(q);
                st.errfail++;
                if (++nef >= MAX_NEF) { status = ST_ERRTEST; break; }
                if (nef >= 3) {
                    h *= 0.1;
                    if (h < hmin) { status = ST_ERRTEST; break; }
                    q = 1;
                    eval_f(0.0, false);
                    for (int p = lane; p < a.P; p += L)
                        for (int i = 0; i < np; i++) Z(1, i, p) = h * F(i, p);
                    if (gas_own) zg[1] = h * fg;
                } else {
                    double eta = C::fail_eta(err2, q + 1);
                    if (eta < 0.2) eta = 0.2;
                    h *= eta;
                    if (h < hmin) { status = ST_ERRTEST; break; }
                    rescale(q, eta);
                }
                qwait = q + 1;
                continue;
            }
            accepted = true;
        }
        if (status != ST_OK) break;

        // accept: z += l (x) e.  The same pass keeps e as the next step's
        // previous e (ep), forms -- when an order selection follows -- its
        // two weighted sums of squares (z_q after the update, e - ep) in the
        // order a pass of their own would take, and then sets the next
        // step's weights from the new z0.
        const double t_new = last ? T : t + h;
        const bool select = qwait - 1 <= 0 && t_new < T;
        double acc[3] = {0.0, 0.0, 0.0};  // non-finite count, sum (z_q w)^2, sum ((e - ep) w)^2
        for (int p = lane; p < a.P; p += L)
            for (int i = 0; i < np; i++) {
                const double ev = E(i, p);
                for (int j = 0; j <= q; j++) Z(j, i, p) += mt.lcoef[q][j] * ev;
                acc[0] += !finite_bits(Z(0, i, p));
                if (select) {
                    const double w = Wt(i, p);
                    const double zq = Z(q, i, p) * w, de = (ev - EP(i, p)) * w;
                    acc[1] += zq * zq;
                    acc[2] += de * de;
                }
                EP(i, p) = ev;
                Wt(i, p) = C::weight(rtol, Z(0, i, p), atol_of(species(i, p)));  // the next step's
            }
        if (gas_own) {
            for (int j = 0; j <= q; j++) zg[j] += mt.lcoef[q][j] * eg;
            acc[0] += !finite_bits(zg[0]);
            if (select) {
                const double zq = zg[q] * wg, de = (eg - epg) * wg;
                acc[1] += zq * zq;
                acc[2] += de * de;
            }
            wg = C::weight(rtol, zg[0], atol_of(tid));
        }
        epg = eg;
        t = t_new;
        nst++;
        st.ordsum += q;
        double r3[3];
        cluster_sum(sm, cl, acc, 3, par, r3);
        if (r3[0] != 0.0) { status = ST_NONFINITE; break; }

        if (--qwait <= 0 && t < T) {
            double eta_q = C::eta(1.2, err2, q + 1);
            double eta_m = 0.0, eta_p = 0.0;
            const double r2[2] = {r3[1], r3[2]};
            if (q > 1) {
                const double ce = mt.ecoef[q - 1] * mt.fact[q];
                const double em2 = C::norm(ce, ce * ce, r2[0], a.n, 1.0 / (double)a.n);
                eta_m = C::eta(1.3, em2, q);
            }
            if (q < QMAX && ep_valid) {
                const double ep2 = C::norm(mt.ecoef[q + 1], mt.ecoef2[q + 1], r2[1], a.n, 1.0 / (double)a.n);
                eta_p = C::eta(1.4, ep2, q + 2);
            }
            double eta = eta_q;
            int qn = q;
            if (eta_m > eta) { eta = eta_m; qn = q - 1; }
            if (eta_p > eta) { eta = eta_p; qn = q + 1; }
            if (eta < ETA_THRESH) {
                qwait = 2;
            } else {
                if (eta > ETA_MAX) eta = ETA_MAX;
                if (qn == q + 1) {
                    const double c_up = mt.lcoef[q][q] / (double)(q + 1);
                    for (int p = lane; p < a.P; p += L)
                        for (int i = 0; i < np; i++) Z(q + 1, i, p) = E(i, p) * c_up;
                    if (gas_own) zg[q + 1] = eg * c_up;
                }
                q = qn;
                h *= eta;
                rescale(q, eta);
                qwait = q + 1;
            }
        }
        ep_valid = true;
    }
    st.steps = nst;
    if (status == ST_OK) {
        for (int p = lane; p < a.P; p += L)
            for (int i = 0; i < np; i++) {
                y_cell[species(i, p)] = Z(0, i, p);
                if (y_copy) y_copy[species(i, p)] = Z(0, i, p);
            }
        if (gas_own) {
            y_cell[tid] = zg[0];
            if (y_copy) y_copy[tid] = zg[0];
        }
    }
    if (step_io && lane == 0) *step_io = status == ST_OK ? h_held : 0.0;
    return status;
}

}  // namespace campdev
