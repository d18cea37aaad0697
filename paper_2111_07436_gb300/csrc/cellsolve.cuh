// Per-cell device routines of the batched chemistry solve (sm_103a).
//
// One group of G lanes (G = 32: one warp) owns one grid cell.  Lane l holds
// the FP64 Nordsieck rows, error weights and corrections of positions
// p = l + G*s (s < NPL) in registers.  Shared memory per cell holds the
// current iterate y, the process rates, the rate constants, the LU values and
// the substitution vector.  Every decision of the step controller is taken on
// group-reduced (hence identical) values, so the lanes of a cell never
// diverge from each other; different cells never synchronise.
//
// Paper references (CAMP, arXiv 2111.07436): rate constants, Table 2;
// forcing f_i = sum_k (dy_i/dt)_k and Jacobian df_i/dy_j = sum_k (...)_k,
// Sect. 2.4.2; the implicit BDF + Newton + sparse LU solve, Sect. 2.4.1.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "devmech.h"

namespace campdev {

// ---- controller constants (identical meaning to the oracle's) ------------
constexpr int QMAX = CAMP_QMAX;
constexpr int NEWTON_MAXIT = 3;
constexpr double NEWTON_TOL = 0.1;
constexpr double RHO_DIV = 2.0;
constexpr double DGMAX = 0.3;
constexpr int MSBJ = 20;
constexpr double ETA_MAX = 10.0;
constexpr double ETA_THRESH = 1.5;
constexpr double ETA_CF = 0.25;
constexpr int MAX_NEF = 7;
constexpr int MAX_NCF = 10;

enum { ST_OK = 0, ST_MAXSTEPS = 1, ST_ERRTEST = 2, ST_NEWTON = 3, ST_SINGULAR = 4, ST_NONFINITE = 5 };

// ---- physical constants (SI 2019, exact) ----------------------------------
constexpr double KB = 1.380649e-23;
constexpr double NAV = 6.02214076e23;
constexpr double RG = KB * NAV;
constexpr double PI_D = 3.14159265358979323846;

// ---- shared-memory layout of one cell --------------------------------------
struct CellSmem {
    int ys, rs, kf, kr, pw, x, lu, bytes;
};
__host__ __device__ inline int align16(int b) { return (b + 15) & ~15; }
// rs holds the R rate terms, then n_part partial sums (of split forcing sums
// inside an f evaluation, of split substitution rows inside a solve)
// pw holds the water parameter's per-cell values (n_pw doubles, and n_pw64
// more in the FP64 form; none without one)
__host__ __device__ inline CellSmem cell_smem(int n, int R, int n_rev, int nlu, int lu_elem, int n_part,
                                              int n_pw, int n_pw64) {
    CellSmem c;
    int o = 0;
    c.ys = o; o = align16(o + 8 * n);
    c.rs = o; o = align16(o + 8 * (R + n_part));
    c.kf = o; o = align16(o + 8 * R);
    c.kr = o; o = align16(o + 8 * n_rev);
    c.pw = o; o = align16(o + 8 * (n_pw + (lu_elem == 8 ? n_pw64 : 0)));
    // the substitution vector shares the rate-term scratch when it fits:
    // the rate terms live only inside one f evaluation, the vector only
    // inside one Newton solve, and the Jacobian assembly keeps its FP32
    // copy of y in ys instead
    if (8 * R >= lu_elem * n) {
        c.x = c.rs;
    } else {
        c.x = o;
        o = align16(o + lu_elem * n);
    }
    c.lu = o; o = align16(o + lu_elem * nlu);
    c.bytes = o;
    return c;
}

template <typename LT>
struct CellPtr {
    double *ys, *rs, *kf, *kr, *pw;
    LT *x, *lu;
    __device__ CellPtr(char *base, const DevMech &m) {
        CellSmem c = cell_smem(m.n, m.R, m.n_rev, m.nlu, (int)sizeof(LT), m.n_part, m.n_pw, m.n_pw64);
        ys = (double *)(base + c.ys);
        rs = (double *)(base + c.rs);
        kf = (double *)(base + c.kf);
        kr = (double *)(base + c.kr);
        pw = (double *)(base + c.pw);
        x = (LT *)(base + c.x);
        lu = (LT *)(base + c.lu);
    }
};

// ---- group primitives --------------------------------------------------------
// A cell is integrated by a group of G lanes: G = 32 lanes of one warp, or a
// whole block of G > 32 threads (one cell per block, for mechanisms too large
// for one warp's registers).  Control flow is uniform across a group, so
// these are safe wherever the group takes them together.
template <int G>
__device__ __forceinline__ void gsync(unsigned gm) {
    if constexpr (G <= 32) __syncwarp(gm);
    else __syncthreads();
}
template <int G>
__device__ __forceinline__ bool gany(bool v, unsigned gm) {
    if constexpr (G <= 32) return __any_sync(gm, v) != 0;
    else return __syncthreads_or(v) != 0;
}
// Sum over the group, the same value in every lane (for a block: a fixed
// order over its warps' partial sums, so every thread gets identical bits)
template <int G, typename T>
__device__ __forceinline__ T gsum_t(T v, unsigned gm) {
    if constexpr (G <= 32) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gm, v, o, G);
        return __shfl_sync(gm, v, 0, G);
    } else {
        __shared__ double part[G / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();  // the previous sum's reads are done
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = (double)v;
        __syncthreads();
        double t = 0.0;
#pragma unroll
        for (int i = 0; i < G / 32; i++) t += part[i];
        return (T)t;
    }
}
template <int G>
__device__ __forceinline__ double gsum(double v, unsigned gm) {
    return gsum_t<G, double>(v, gm);
}

// ---- rate constants (Table 2), per process, from the cell's env ------------
__device__ __forceinline__ double ipowd(double x, int k) {
    double r = 1.0;
    for (int i = 0; i < k; i++) r *= x;
    return r;
}

// A exp(C/T) (T/300)^B: the Arrhenius terms of the Troe and custom rate
// constants (D = 300 K, E = 0)
__device__ __forceinline__ double arr300(const double *par, double T) {
    return __ldg(par) * exp(__ldg(par + 2) / T) * pow(T / 300.0, __ldg(par + 1));
}

// Condensation constant of one section, s^-1: N particles of radius rad,
// each 4 pi rad Dg f_fs(Kn, alpha) with the Fuchs-Sutugin factor and
// Kn = 3 Dg / (cbar rad), cbar = sqrt(8 R T / (pi MW))
__device__ __forceinline__ double condensation(double rad, double Np, double alpha, double Dg,
                                               double MW, double T) {
    double cbar = sqrt(8.0 * RG * T / (PI_D * MW));
    double Kn = 3.0 * Dg / cbar / rad;
    double ffs = 0.75 * alpha * (1.0 + Kn) / (Kn * Kn + Kn + 0.283 * Kn * alpha + 0.75 * alpha);
    return Np * 4.0 * PI_D * rad * Dg * ffs;
}

// Liquid volume of a section in the rate constants: the env value (the
// section's (r, N, L) triple in sec), or 1 when the water parameter makes it a
// function of the state (the constants are then per unit volume and the
// powers of 1/L are applied at each state)
__device__ __forceinline__ double section_volume(const DevMech &m, const double *__restrict__ sec) {
    return m.n_wsec > 0 ? 1.0 : sec[2];
}

// Rate constants of process k: env holds T, P and the runtime rates; sec the
// (radius, number concentration, liquid volume) of the section (or particle)
// a section process acts in (unused by the others)
__device__ inline void rate_constant_at(const DevMech &m, int k, const double *__restrict__ env,
                                        const double *__restrict__ sec, double &kf, double &kr) {
    const double T = env[0], P = env[1];
    const double Mair = P / (KB * T) * 1e-6;  // molec cm^-3
    const double mppb = Mair * 1e-9;          // molec cm^-3 per ppb
    const double *par = m.rpar + CAMP_NPAR * k;
    const int nr = __ldg(m.rnr + k);
    kf = 0.0;
    kr = 0.0;
    switch (__ldg(m.rtype + k)) {
    case CAMP_P_ARRHENIUS: {
        // k = A exp(C/T) (T/D)^B (1 + E P)
        double kk = __ldg(par) * exp(__ldg(par + 2) / T) * pow(T / __ldg(par + 3), __ldg(par + 1)) *
                    (1.0 + __ldg(par + 4) * P);
        kf = kk * ipowd(mppb, nr - 1);
        break;
    }
    case CAMP_P_TROE: {
        // k0[M] / (1 + k0[M]/kinf) * Fc^(1 / (1 + (log10(k0[M]/kinf)/N)^2))
        double k0 = arr300(par, T);
        double ki = arr300(par + 3, T);
        double x = k0 * Mair / ki;
        double lg = log10(x) / __ldg(par + 7);
        double kk = k0 * Mair / (1.0 + x) * pow(__ldg(par + 6), 1.0 / (1.0 + lg * lg));
        kf = kk * ipowd(mppb, nr - 1);
        break;
    }
    case CAMP_P_CUSTOM_H2O2:
        // k1 + k2 [M]
        kf = (arr300(par, T) + arr300(par + 3, T) * Mair) * ipowd(mppb, nr - 1);
        break;
    case CAMP_P_CUSTOM_OH_HNO3: {
        // k0 + k3[M] / (1 + k3[M] / k2)
        double k3M = arr300(par + 6, T) * Mair;
        kf = (arr300(par, T) + k3M / (1.0 + k3M / arr300(par + 3, T))) * ipowd(mppb, nr - 1);
        break;
    }
    case CAMP_P_PHOTOLYSIS:
    case CAMP_P_EMISSION:
    case CAMP_P_LOSS:
        kf = env[__ldg(m.rslot + k)];
        break;
    case CAMP_P_HENRY:
    case CAMP_P_SIMPOL: {
        // condensation k_c per section; evaporation k_c / (H_cc L) with
        // H_cc = 1000 H R T.  Henry: H(T) [M/Pa] from H298 and C.  SIMPOL:
        // H = c_tot / p0 with the SIMPOL.1 vapour pressure
        // log10 p0 [atm] = B1/T + B2 + B3 T + B4 ln T (Raoult's law in a
        // condensed phase of fixed total molarity c_tot)
        const double rad = sec[0];
        const double Np = sec[1];
        const double L = section_volume(m, sec);
        if (!(L > 0.0 && Np > 0.0 && rad > 0.0)) break;
        double H, kb;
        if (__ldg(m.rtype + k) == CAMP_P_HENRY) {
            H = __ldg(par) * exp(__ldg(par + 1) * (1.0 / T - 1.0 / 298.0));
            kb = condensation(rad, Np, __ldg(par + 2), __ldg(par + 3), __ldg(par + 4), T);
        } else {
            double lg = __ldg(par) / T + __ldg(par + 1) + __ldg(par + 2) * T + __ldg(par + 3) * log(T);
            H = __ldg(par + 7) / (101325.0 * exp10(lg));
            kb = condensation(rad, Np, __ldg(par + 4), __ldg(par + 5), __ldg(par + 6), T);
        }
        kf = kb;
        kr = kb / (1000.0 * H * RG * T * L);
        break;
    }
    case CAMP_P_AQREV: {
        // K_eq = A exp(C (1/T - 1/298)); rates in M/s, molarity = y * phi,
        // phi = 1e-9 P / (R T 1000 L) M per ppb
        const double L = section_volume(m, sec);
        if (!(L > 0.0)) break;
        double Keq = __ldg(par) * exp(__ldg(par + 1) * (1.0 / T - 1.0 / 298.0));
        double krev = __ldg(par + 2);
        double phi = 1e-9 * P / (RG * T * 1000.0 * L);
        kf = Keq * krev * ipowd(phi, nr - 1);
        kr = krev * ipowd(phi, __ldg(m.rnp + k) - 1);
        break;
    }
    case CAMP_P_COND_ARRHENIUS: {
        // Arrhenius in the section's condensed phase, M^(1-nr) s^-1:
        // kf = k phi^(nr - 1) in ppb units
        const double L = section_volume(m, sec);
        if (!(L > 0.0)) break;
        double kk = __ldg(par) * exp(__ldg(par + 2) / T) * pow(T / __ldg(par + 3), __ldg(par + 1)) *
                    (1.0 + __ldg(par + 4) * P);
        double phi = 1e-9 * P / (RG * T * 1000.0 * L);
        kf = kk * ipowd(phi, nr - 1);
        break;
    }
    }
}

__device__ __forceinline__ bool section_type(int t) {
    return t == CAMP_P_HENRY || t == CAMP_P_SIMPOL || t == CAMP_P_AQREV || t == CAMP_P_COND_ARRHENIUS;
}

// Rate constants of process k of a compiled mechanism (section processes
// read their section's triple from env)
__device__ __forceinline__ void rate_constant(const DevMech &m, int k, const double *__restrict__ env,
                                              double &kf, double &kr) {
    const int t = __ldg(m.rtype + k);
    const double *sec = section_type(t) ? env + m.env_sec_base + 3 * __ldg(m.rslot + k) : env;
    rate_constant_at(m, k, env, sec, kf, kr);
}

// FP64 values into and out of the LU precision
template <typename LT> __device__ __forceinline__ LT to_lu(double x);
template <> __device__ __forceinline__ float to_lu<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ double to_lu<double>(double x) { return x; }
__device__ __forceinline__ double from_lu(float x) { return (double)x; }
__device__ __forceinline__ double from_lu(double x) { return x; }

// One lane's term (x w)^2 of the Newton update's squared norm, in the LU
// precision.  In FP32 a weight beyond the format's range (atol below ~3e-39
// on a species near zero) is held at its largest value and the product at
// 1e18, so the sum stays finite; either only arises far from convergence.
// A non-finite x is caught separately.
__device__ __forceinline__ float upd_term(float x, double w) {
    const float t = fminf(fabsf(x * fminf((float)w, 3.4e38f)), 1e18f);
    return t * t;
}
__device__ __forceinline__ double upd_term(double x, double w) {
    const double t = x * w;
    return t * t;
}

// finite test on the exponent bits (integer pipe, not the FP64 pipe)
__device__ __forceinline__ bool finite_bits(double x) {
    return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

// ---- forcing f(y): rates of all processes, then a per-position gather --------
// r_k = kf prod(forward factors) - kr prod(reverse factors), from the
// process's packed record (16-bit fields, 0xffff = none).
__device__ __forceinline__ int lo16(int v) { return v & 0xffff; }
__device__ __forceinline__ int hi16(int v) { return (int)((unsigned)v >> 16); }
constexpr int NONE16 = 0xffff;

__device__ __forceinline__ double rate_term(const DevMech &m, int k, const double *ys, double kf,
                                            const double *kr) {
    const int4 rp = __ldg(m.rpack + k);
    const int a0 = lo16(rp.x), a1 = hi16(rp.x), a2 = lo16(rp.y), rv = hi16(rp.y);
    double a = kf;
    if (a0 != NONE16) a *= ys[a0];
    if (a1 != NONE16) a *= ys[a1];
    if (a2 != NONE16) a *= ys[a2];
    if (rv != NONE16) {
        const int b0 = lo16(rp.z), b1 = hi16(rp.z), b2 = lo16(rp.w);
        double b = kr[rv];
        if (b0 != NONE16) b *= ys[b0];
        if (b1 != NONE16) b *= ys[b1];
        if (b2 != NONE16) b *= ys[b2];
        a -= b;
    }
    return a;
}

__device__ __forceinline__ double gather_entry(const DevMech &m, int q, const double *rs) {
    const int g = __ldg(m.fpk + q);
    return __ldg(m.fcoef + hi16(g)) * rs[lo16(g)];
}

// ---- the water parameter (Sect. 2.2.2; Table 4, ZSRAerosolWater) ----------
// With the parameter, the constants of the section processes stay per unit
// volume in kf / kr, and the powers of 1/L(y) are applied where they are
// used (the rate terms, the Jacobian's constants, the chain rule), from each
// process's record: bits 16-26 of rpack.w hold its section + 1 (0: not a
// section process), bits 27-28 la and bits 29-30 lb.  Per-cell scratch c.pw:
// the electrolyte weights, L_env and 1/L of each section (1/L stored as 0
// for a section whose water is not positive: its processes take no part),
// then, in the FP64 form only, the Jacobian's reverse constants.
__device__ __forceinline__ double *pw_wt(const DevMech &, double *pw) { return pw; }
__device__ __forceinline__ double *pw_lenv(const DevMech &m, double *pw) { return pw + m.n_el; }
__device__ __forceinline__ double *pw_invl(const DevMech &m, double *pw) { return pw + m.n_el + m.n_wsec; }
__device__ __forceinline__ double *pw_kr64(const DevMech &m, double *pw) { return pw + m.n_pw; }

struct WaterTag {
    int sec, la, lb;  // sec = -1: not a section process
};
__device__ __forceinline__ WaterTag water_tag(int w) {
    const int h = hi16(w);
    return {(h & 0x7ff) - 1, (h >> 11) & 3, (h >> 13) & 3};
}
// factor of kf (p = la) or kr (p = lb) at the current volumes
__device__ __forceinline__ double water_scale(int sec, int p, const double *invl) {
    if (sec < 0) return 1.0;
    const double il = invl[sec];
    return il > 0.0 ? ipowd(il, p) : 0.0;
}

// Water per ppb of electrolyte e [m^3 per m^3 air]: 1e-9 P / (R T) mol m^-3
// per ppb over the molality m_e(a_w) of its binary solution (ZSR:
// W = sum_i 1000 M_i / (MW_i m_i(a_w)) kg m^-3), over the density of water.
// The molality fit is sqrt(m) = sum_j Y_j a_w^j with a_w = RH, held at the
// fit's lowest activity below it; a fit that gives no positive molality
// holds no water.
__device__ inline double zsr_weight(const DevMech &m, int e, const double *__restrict__ env) {
    const double T = env[0], P = env[1];
    double aw = env[m.rh_slot];
    const double lo = __ldg(m.zsr_low + e);
    if (aw < lo) aw = lo;
    double s = 0.0, p = 1.0;
    for (int j = 0; j < CAMP_ZSR_NY; j++) {
        s += __ldg(m.zsr_Y + CAMP_ZSR_NY * e + j) * p;
        p *= aw;
    }
    const double mol = s * s;
    if (!(mol > 0.0) || !finite_bits(mol)) return 0.0;
    return 1e-9 * P / (RG * T) / mol / 1000.0;
}

// Per cell, once: the electrolyte weights and the sections' env volumes.
template <int G>
__device__ __forceinline__ void water_setup(const DevMech &m, double *pw, const double *__restrict__ env,
                                            int lane, unsigned gm) {
    double *wt = pw_wt(m, pw), *lenv = pw_lenv(m, pw);
    for (int e = lane; e < m.n_el; e += G) wt[e] = zsr_weight(m, e, env);
    for (int b = lane; b < m.n_wsec; b += G) lenv[b] = env[m.env_sec_base + 3 * b + 2];
    gsync<G>(gm);
}

// The parameter at the state in ys: L_b = L_env,b + sum_e w_e y_e, kept as
// 1/L_b (0 for a section whose water is not positive).
template <int G>
__device__ __forceinline__ void water_update(const DevMech &m, double *pw, const double *ys, int lane,
                                             unsigned gm) {
    const double *wt = pw_wt(m, pw), *lenv = pw_lenv(m, pw);
    double *invl = pw_invl(m, pw);
    for (int b = lane; b < m.n_wsec; b += G) {
        double v = lenv[b];
        const int q1 = __ldg(m.pw_ptr + b + 1);
        for (int q = __ldg(m.pw_ptr + b); q < q1; q++) {
            const int w = __ldg(m.pw + q);
            v += wt[hi16(w)] * ys[lo16(w)];
        }
        invl[b] = v > 0.0 ? 1.0 / v : 0.0;
    }
    gsync<G>(gm);
}

// r_k with the powers of 1/L of a section process applied (the water build's
// rate term)
__device__ __forceinline__ double rate_term_water(const DevMech &m, int k, const double *ys, const double *kf,
                                                  const double *kr, const double *invl) {
    const int4 rp = __ldg(m.rpack + k);
    const WaterTag t = water_tag(rp.w);
    double il = 1.0;
    if (t.sec >= 0) {
        il = invl[t.sec];
        if (!(il > 0.0)) return 0.0;
    }
    const int a0 = lo16(rp.x), a1 = hi16(rp.x), a2 = lo16(rp.y), rv = hi16(rp.y);
    double a = kf[k] * ipowd(il, t.la);
    if (a0 != NONE16) a *= ys[a0];
    if (a1 != NONE16) a *= ys[a1];
    if (a2 != NONE16) a *= ys[a2];
    if (rv != NONE16) {
        const int b0 = lo16(rp.z), b1 = hi16(rp.z), b2 = lo16(rp.w);
        double b = kr[rv] * ipowd(il, t.lb);
        if (b0 != NONE16) b *= ys[b0];
        if (b1 != NONE16) b *= ys[b1];
        if (b2 != NONE16) b *= ys[b2];
        a -= b;
    }
    return a;
}

// The chain-rule term J_p P_y of Sect. 2.2.2 after the direct assembly: for
// each (row i, section b) pair g, g = d f_i / d L_b = sum_j nu_ij dr_j/dL_b
// with dr/dL = -(la F - lb B) / L (F, B the forward and reverse terms at the
// assembly's state y), then J_ie += g w_e for each electrolyte e of b.  The
// entries of one g are its n_el consecutive chain records; every record is a
// distinct (row, electrolyte) pair, so lanes need no atomics.
template <int G, typename LT>
__device__ __forceinline__ void water_chain(const DevMech &m, double *pw, const double *kf, const double *kr,
                                            const LT *y, LT *lu, double gamma, int lane, int mode,
                                            double *out) {
    const double *wt = pw_wt(m, pw), *invl = pw_invl(m, pw);
    for (int g = lane; g < m.n_g; g += G) {
        double acc = 0.0;
        const int q1 = __ldg(m.g_ptr + g + 1);
        for (int q = __ldg(m.g_ptr + g); q < q1; q++) {
            const int4 r = __ldg(m.pp + __ldg(m.g_ent + q));
            const double il = invl[r.y];
            if (!(il > 0.0)) continue;
            const int la = r.z & 0xff, lb = r.z >> 8;
            const int4 rp = __ldg(m.rpack + r.x);
            const int a0 = lo16(rp.x), a1 = hi16(rp.x), a2 = lo16(rp.y);
            double F = kf[r.x] * ipowd(il, la);
            if (a0 != NONE16) F *= (double)y[a0];
            if (a1 != NONE16) F *= (double)y[a1];
            if (a2 != NONE16) F *= (double)y[a2];
            double B = 0.0;
            if (r.w >= 0) {
                const int b0 = lo16(rp.z), b1 = hi16(rp.z), b2 = lo16(rp.w);
                B = kr[r.w] * ipowd(il, lb);
                if (b0 != NONE16) B *= (double)y[b0];
                if (b1 != NONE16) B *= (double)y[b1];
                if (b2 != NONE16) B *= (double)y[b2];
            }
            acc += __ldg(m.g_coef + q) * (-((double)la * F - (double)lb * B) * il);
        }
        for (int e = 0; e < m.n_el; e++) {
            const int4 ch = __ldg(m.ch + g * m.n_el + e);
            const double v = acc * wt[e];
            if (mode == 0)
                lu[ch.x] -= to_lu<LT>(gamma * v);
            else
                out[ch.w] += v;
        }
    }
}

// y in c.ys (written by the caller, who also made it visible to the group)
// -> f (own positions).  The per-position sums are spread over the cell's
// lanes by the compiler's balanced assignment (long sums in chunks) and
// handed back through shared memory (reusing ys).
template <int G, int NPL, typename LT, bool W>
__device__ __forceinline__ void eval_f_ys(const DevMech &m, const CellPtr<LT> &c, double (&f)[NPL],
                                          int lane, unsigned gm) {
    if constexpr (W) {
        water_update<G>(m, c.pw, c.ys, lane, gm);
        const double *invl = pw_invl(m, c.pw);
        for (int k = lane; k < m.R; k += G) c.rs[k] = rate_term_water(m, k, c.ys, c.kf, c.kr, invl);
    } else {
        for (int k = lane; k < m.R; k += G) c.rs[k] = rate_term(m, k, c.ys, c.kf[k], c.kr);
    }
    gsync<G>(gm);
    double *fs = c.ys;  // y is no longer needed
    double *fp = c.rs + m.R;
    const int b0 = __ldg(m.flane_ptr + lane), b1 = __ldg(m.flane_ptr + lane + 1);
    for (int i = b0; i < b1; i++) {
        const int2 job = __ldg(m.fjob + i);
        const int end = job.x + hi16(job.y), dst = lo16(job.y);
        double acc = 0.0, acc2 = 0.0;
        int q = job.x;
        for (; q + 1 < end; q += 2) {
            acc += gather_entry(m, q, c.rs);
            acc2 += gather_entry(m, q + 1, c.rs);
        }
        if (q < end) acc += gather_entry(m, q, c.rs);
        if (G == 32 || dst < m.n) fs[dst] = acc + acc2;  // one-warp cells have no split sums
        else fp[dst - m.n] = acc + acc2;
    }
    gsync<G>(gm);
    if (G > 32 && m.n_fsplit > 0) {  // split sums: their partials in a fixed order
        for (int i = lane; i < m.n_fsplit; i += G) {
            const int2 sp = __ldg(m.fsplit + i);
            const int first = lo16(sp.y), cnt = hi16(sp.y);
            double t = 0.0;
            for (int j = 0; j < cnt; j++) t += fp[first + j];
            fs[sp.x] = t;
        }
        gsync<G>(gm);
    }
#pragma unroll
    for (int s = 0; s < NPL; s++) {
        int p = lane + G * s;
        f[s] = (p < m.n) ? fs[p] : 0.0;
    }
    gsync<G>(gm);
}

// y (own positions, registers) -> f (own positions)
template <int G, int NPL, typename LT, bool W>
__device__ __forceinline__ void eval_f(const DevMech &m, const CellPtr<LT> &c, const double (&y)[NPL],
                                       double (&f)[NPL], int lane, unsigned gm) {
#pragma unroll
    for (int s = 0; s < NPL; s++) {
        int p = lane + G * s;
        if (p < m.n) c.ys[p] = y[s];
    }
    gsync<G>(gm);
    eval_f_ys<G, NPL, LT, W>(m, c, f, lane, gm);
}

// f at y = a + b u (own positions), without a register copy of y
template <int G, int NPL, typename LT, bool W>
__device__ __forceinline__ void eval_f_at(const DevMech &m, const CellPtr<LT> &c, const double (&a)[NPL],
                                          double b, const double (&u)[NPL], double (&f)[NPL], int lane,
                                          unsigned gm) {
#pragma unroll
    for (int s = 0; s < NPL; s++) {
        int p = lane + G * s;
        if (p < m.n) c.ys[p] = a[s] + b * u[s];
    }
    gsync<G>(gm);
    eval_f_ys<G, NPL, LT, W>(m, c, f, lane, gm);
}

// ---- Jacobian gather: J (or M = I - gamma J) at ys into LU storage -----------
// mode 0: write M = I - gamma J into c.lu (zeroing fill and block entries)
// mode 1: write J values to out[nnzJ] (species-CSR order)
// In FP32 the rate constants and y are converted once into scratch that is
// free at this point (the rate array and the substitution vector), so the
// per-entry gather does no FP64/FP32 conversion.
template <int G, typename LT, bool W>
__device__ __forceinline__ void assemble(const DevMech &m, const CellPtr<LT> &c, double gamma,
                                         int lane, unsigned gm, int mode, double *out) {
    const LT *kfv, *krv, *yv;
    // the water build: 1/L at this state, and the constants with their
    // powers of 1/L applied (FP64 form: into the rate scratch and the
    // parameter block)
    auto water_constants = [&](LT *kfw, LT *krw) {
        const double *invl = pw_invl(m, c.pw);
        for (int k = lane; k < m.R; k += G) {
            const int4 rp = __ldg(m.rpack + k);
            const WaterTag t = water_tag(rp.w);
            kfw[k] = to_lu<LT>(c.kf[k] * water_scale(t.sec, t.la, invl));
            const int rv = hi16(rp.y);
            if (rv != NONE16) krw[rv] = to_lu<LT>(c.kr[rv] * water_scale(t.sec, t.lb, invl));
        }
    };
    if constexpr (W) water_update<G>(m, c.pw, c.ys, lane, gm);
    if constexpr (sizeof(LT) == 4) {
        LT *kf32 = (LT *)c.rs, *kr32 = kf32 + m.R, *y32 = (LT *)c.ys;
        if constexpr (W) {
            water_constants(kf32, kr32);
        } else {
            for (int k = lane; k < m.R; k += G) kf32[k] = (LT)c.kf[k];
            for (int k = lane; k < m.n_rev; k += G) kr32[k] = (LT)c.kr[k];
        }
        // y to FP32 in place, G positions at a time: a chunk's FP32 values
        // overwrite only FP64 values of this or earlier chunks, and the
        // group reads its chunk before any lane writes it
        for (int b0 = 0; b0 < m.n; b0 += G) {
            const int p = b0 + lane;
            const double v = p < m.n ? c.ys[p] : 0.0;
            gsync<G>(gm);
            if (p < m.n) y32[p] = (LT)v;
        }
        kfv = kf32;
        krv = kr32;
        yv = y32;
    } else {
        if constexpr (W) {
            LT *kf64 = (LT *)c.rs, *kr64 = (LT *)pw_kr64(m, c.pw);
            water_constants(kf64, kr64);
            kfv = kf64;
            krv = kr64;
        } else {
            kfv = (const LT *)c.kf;
            krv = (const LT *)c.kr;
        }
        yv = (const LT *)c.ys;
    }
    if (mode == 0) {  // 16-byte stores: the LU array starts 16-byte aligned
        constexpr int V = 16 / sizeof(LT);
        float4 *z4 = (float4 *)c.lu;
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        const int nv = m.nlu / V;
        for (int i = lane; i < nv; i += G) z4[i] = zero;
        for (int i = nv * V + lane; i < m.nlu; i += G) c.lu[i] = (LT)0;
    }
    gsync<G>(gm);
    const LT g = (LT)gamma;
    if constexpr (sizeof(LT) == 4) {
        {
            // flat per-lane entry list: independent loads, one store per non-zero
            const int b = __ldg(m.jl_ptr + lane), e = __ldg(m.jl_ptr + lane + 1);
            LT acc = (LT)0;
#pragma unroll 4
            for (int i = b; i < e; i++) {
                const int4 r = __ldg(m.jl_rec + i);
                const int k = (int)(short)(r.y & 0xffff);
                const int o1 = hi16(r.y), o2 = lo16(r.w);
                LT v = __int_as_float(r.x) * (k >= 0 ? kfv[k] : krv[-k - 1]);
                if (o1 != NONE16) v *= yv[o1];
                if (o2 != NONE16) v *= yv[o2];
                acc += v;
                if (r.z & (1 << 17)) {
                    if (mode == 0)
                        c.lu[r.z & 0xffff] = ((r.z >> 16) & 1 ? (LT)1 : (LT)0) - g * acc;
                    else
                        out[hi16(r.w)] = (double)acc;
                    acc = (LT)0;
                }
            }
        }
    }
    if constexpr (sizeof(LT) == 8) {  // FP64: one non-zero per lane at a time
        for (int t = lane; t < m.nnzJ; t += G) {
            LT acc = (LT)0;
            const int4 nz = __ldg(m.jnz + t);
            for (int q = nz.x; q < nz.y; q++) {
                const int k = __ldg(m.jk + q);
                LT v = (LT)__ldg(m.jc + q) * (k >= 0 ? kfv[k] : krv[-k - 1]);
                const int o1 = __ldg(m.jo + 2 * q), o2 = __ldg(m.jo + 2 * q + 1);
                if (o1 >= 0) v *= yv[o1];
                if (o2 >= 0) v *= yv[o2];
                acc += v;
            }
            if (mode == 0)
                c.lu[nz.z] = (nz.w ? (LT)1 : (LT)0) - g * acc;
            else
                out[t] = (double)acc;
        }
    }
    gsync<G>(gm);
    if constexpr (W) {
        water_chain<G, LT>(m, c.pw, c.kf, c.kr, yv, c.lu, gamma, lane, mode, out);
        gsync<G>(gm);
    }
}

template <typename LT> __device__ __forceinline__ LT tiny_pivot();
template <> __device__ __forceinline__ float tiny_pivot<float>() { return 1e-30f; }
template <> __device__ __forceinline__ double tiny_pivot<double>() { return 1e-300; }

// ---- LU factorisation in place; returns true if every pivot is usable -------
// Pivots are checked, then replaced by their reciprocals: the substitutions
// and later rows multiply instead of dividing.
// 1 / u, correctly rounded, without the general division's range handling
__device__ __forceinline__ float recip(float u) { return __frcp_rn(u); }
__device__ __forceinline__ double recip(double u) { return 1.0 / u; }

template <typename LT>
__device__ __forceinline__ bool bad_pivot(LT u) {
    return !(fabs(u) > tiny_pivot<LT>()) || !isfinite(u);
}

// Dense trailing block, right-looking in panels of W pivots.  For each
// panel: (1) factor its W columns over the rows below (lane l owns rows
// l + 32 t); (2) forward-substitute the W pivot rows to the right of the
// panel with the panel's unit lower triangle (lane l owns columns l + 32 t);
// (3) one rank-W update of the trailing block, each entry loaded and stored
// once per panel (the W multipliers of a row are broadcast loads).
// Pivots are checked and replaced by their reciprocals.
template <int NS, int W, typename LT>
__device__ __forceinline__ bool dense_factor(LT *A, int D, int LD, int lane, unsigned gm) {
    bool bad = false;
    for (int kp = 0; kp < D; kp += W) {
        const int w = min(W, D - kp);
        // (1) panel columns kp .. kp+w-1
        for (int c = 0; c < w; c++) {
            const int k = kp + c;
            const LT piv = A[k * LD + k];
            bad |= bad_pivot(piv);
            const LT rp = recip(piv);
            LT uk[W];  // the pivot row inside the panel
#pragma unroll
            for (int j = 1; j < W; j++) uk[j] = (c + j < w) ? A[k * LD + k + j] : (LT)0;
#pragma unroll
            for (int t = 0; t < NS; t++) {
                const int i = lane + 32 * t;
                if (i > k && i < D) {
                    LT *row = A + i * LD;
                    const LT l = row[k] * rp;
                    row[k] = l;
#pragma unroll
                    for (int j = 1; j < W; j++)
                        if (c + j < w) row[k + j] -= l * uk[j];
                }
            }
            __syncwarp(gm);
            if (lane == 0) A[k * LD + k] = rp;
        }
        const int j0 = kp + w;
        if (j0 >= D) break;
        // (2) pivot rows of the panel, columns right of it: unit lower solve
        LT u[W][NS];
        bool act[NS];
#pragma unroll
        for (int t = 0; t < NS; t++) {
            const int j = j0 + lane + 32 * t;
            act[t] = j < D;
#pragma unroll
            for (int r = 0; r < W; r++) {
                LT v = (LT)0;
                if (act[t] && r < w) {
                    v = A[(kp + r) * LD + j];
#pragma unroll
                    for (int p = 0; p < r; p++) v -= A[(kp + r) * LD + kp + p] * u[p][t];
                    A[(kp + r) * LD + j] = v;
                }
                u[r][t] = v;
            }
        }
        __syncwarp(gm);
        // (3) trailing block: rank-w update, two rows at a time with every
        // load issued before the stores (rows never alias; the compiler
        // cannot know that)
        int i = j0;
        for (; i + 1 < D; i += 2) {
            const LT *l0p = A + i * LD + kp, *l1p = l0p + LD;
            LT l0[W], l1[W], a0[NS], a1[NS];
#pragma unroll
            for (int r = 0; r < W; r++) {
                l0[r] = r < w ? l0p[r] : (LT)0;
                l1[r] = r < w ? l1p[r] : (LT)0;
            }
#pragma unroll
            for (int t = 0; t < NS; t++) {
                const int col = j0 + lane + 32 * t;
                a0[t] = act[t] ? A[i * LD + col] : (LT)0;
                a1[t] = act[t] ? A[(i + 1) * LD + col] : (LT)0;
            }
#pragma unroll
            for (int t = 0; t < NS; t++) {
#pragma unroll
                for (int r = 0; r < W; r++) {
                    a0[t] -= l0[r] * u[r][t];
                    a1[t] -= l1[r] * u[r][t];
                }
            }
#pragma unroll
            for (int t = 0; t < NS; t++) {
                if (act[t]) {
                    const int col = j0 + lane + 32 * t;
                    A[i * LD + col] = a0[t];
                    A[(i + 1) * LD + col] = a1[t];
                }
            }
        }
        if (i < D) {  // odd number of trailing rows: the last one alone
            const LT *l0p = A + i * LD + kp;
            LT l0[W];
#pragma unroll
            for (int r = 0; r < W; r++) l0[r] = r < w ? l0p[r] : (LT)0;
#pragma unroll
            for (int t = 0; t < NS; t++) {
                if (act[t]) {
                    LT *a = A + i * LD + j0 + lane + 32 * t;
                    LT v = *a;
#pragma unroll
                    for (int r = 0; r < W; r++) v -= l0[r] * u[r][t];
                    *a = v;
                }
            }
        }
        __syncwarp(gm);
    }
    return bad;
}

// panel width of the dense factorisation
constexpr int DENSE_W = 8;

// one op of the row-wise factorisation: a division makes the multiplier l
// (lu[src] holds 1 / U(k,k)), an update subtracts l U(k,j) from its target,
// an LU value or (bit 15 of the target; block cells only) a partial sum
template <bool PART, typename LT>
__device__ __forceinline__ void factor_op(uint32_t op, LT *lu, LT *part, int pbase, LT &l) {
    const int t = CAMP_OP_TGT(op), s = CAMP_OP_SRC(op);
    if (op & CAMP_OP_DIV) {
        l = lu[t] * lu[s];
        lu[t] = l;
    } else if (PART && (t & 0x8000)) {
        part[pbase + (t & 0x7fff)] -= l * lu[s];
    } else {
        lu[t] -= l * lu[s];
    }
}

template <typename LT>
__device__ __forceinline__ bool take_reciprocal(const DevMech &m, LT *lu, int i) {
    const int di = __ldg(m.udiag + i);
    const LT u = lu[di];
    lu[di] = recip(u);
    return bad_pivot(u);
}

template <int G, typename LT>
__device__ bool factor(const DevMech &m, const CellPtr<LT> &c, int lane, unsigned gm) {
    LT *lu = c.lu;
    LT *part = (LT *)(c.rs + m.R);  // chunk partials: the rate scratch is free here
    bool bad = false;
    // sparse rows (and the sparse-pivot updates of the block rows), by level
    for (int L = 0; L < m.n_flev; L++) {
        const int b = __ldg(m.ljob_ptr + L), e = __ldg(m.ljob_ptr + L + 1);
        for (int r = b + lane; r < e; r += G) {
            const int4 jb = __ldg(m.ljob + r);
            const int cnt = lo16(jb.y);
            if constexpr (G > 32) {
                for (int k = 0; k < hi16(jb.y); k++) part[jb.w + k] = (LT)0;
            }
            LT l = (LT)0;
            for (int q = jb.x; q < jb.x + cnt; q++) factor_op<(G > 32)>(__ldg(m.lops + q), lu, part, jb.w, l);
            if (hi16(jb.z) & 1) bad |= take_reciprocal(m, lu, lo16(jb.z));
        }
        gsync<G>(gm);
        if constexpr (G > 32) {  // rows cut into chunks: partials in order, then the tail
            const int rb = __ldg(m.lred_ptr + L), re = __ldg(m.lred_ptr + L + 1);
            for (int k = rb + lane; k < re; k += G) {
                const int4 rd = __ldg(m.lred + k);
                const int ns = lo16(rd.z), nch = hi16(rd.z);
                for (int s = 0; s < ns; s++) {
                    const int off = __ldg(m.lred_off + rd.y + s);
                    LT t = lu[off];
                    for (int ch = 0; ch < nch; ch++) t += part[rd.w + ch * ns + s];
                    lu[off] = t;
                }
                const int2 tl = __ldg(m.ltail + k);
                LT l = (LT)0;
                for (int q = tl.x; q < tl.x + tl.y; q++) factor_op<false>(__ldg(m.lops + q), lu, part, 0, l);
                if (hi16(rd.x) & 1) bad |= take_reciprocal(m, lu, lo16(rd.x));
            }
            if (re > rb) gsync<G>(gm);
        }
    }
    // the dense block is one warp's work (a block group's first warp)
    LT *A = lu + m.dbase;
    if (G <= 32 || lane < 32) {
        const unsigned wm = G <= 32 ? gm : 0xffffffffu;
        switch ((m.D + 31) >> 5) {
        case 0: break;
        case 1: bad |= dense_factor<1, DENSE_W, LT>(A, m.D, m.LD, lane, wm); break;
        case 2: bad |= dense_factor<2, DENSE_W, LT>(A, m.D, m.LD, lane, wm); break;
        case 3: bad |= dense_factor<3, DENSE_W, LT>(A, m.D, m.LD, lane, wm); break;
        default: bad |= dense_factor<4, DENSE_W, LT>(A, m.D, m.LD, lane, wm); break;
        }
    }
    return !gany<G>(bad, gm);
}

// ---- substitution: solves (LU) x = x in place (c.x holds the right side) -----
// Sparse rows go level by level through shared memory.  The dense block's
// right side lives in registers (lane l holds rows l + 32 t); each pivot's
// value is broadcast with a shuffle, and the loops run one 32-row diagonal
// block at a time so that only that block's rows need a comparison.  Rows
// past the block end read the last row (a valid address) and are discarded.
template <int NS, typename LT, int SP>
__device__ __forceinline__ void dense_subst(const LT *A, int D, int LD, LT *xb, int lane, unsigned gm) {
    LT xr[NS];
    int rowc[NS];
#pragma unroll
    for (int t = 0; t < NS; t++) {
        const int i = lane + 32 * t;
        rowc[t] = (i < D ? i : D - 1) * LD;
        xr[t] = i < D ? xb[i] : (LT)0;
    }
    if constexpr (SP == 2) {
    // forward, unit lower, two pivots per round: x_k and the not yet final
    // x_{k+1} come by two independent shuffles, every lane finishes x_{k+1}
    // with the broadcast L(k+1,k), then both columns update the rows below
#pragma unroll
    for (int kb = 0; kb < NS; kb++) {
        const int k0 = 32 * kb, k1 = min(D, k0 + 32);
        int k = k0;
#pragma unroll 2
        for (; k + 1 < k1; k += 2) {
            const int o = k - k0;
            const LT xk = __shfl_sync(gm, xr[kb], o);
            const LT xn = __shfl_sync(gm, xr[kb], o + 1);
            const LT l10 = A[(k + 1) * LD + k];
            const LT xk1 = xn - l10 * xk;
#pragma unroll
            for (int t = kb; t < NS; t++) {
                const LT a0 = A[rowc[t] + k], a1 = A[rowc[t] + k + 1];
                if (t > kb || lane > o + 1) {
                    xr[t] -= a0 * xk;
                    xr[t] -= a1 * xk1;
                } else if (lane == o + 1) {
                    xr[t] = xk1;
                }
            }
        }
        if (k < k1) {  // odd block length: one pivot left
            const int o = k - k0;
            const LT xk = __shfl_sync(gm, xr[kb], o);
#pragma unroll
            for (int t = kb; t < NS; t++) {
                const LT a = A[rowc[t] + k];
                if (t > kb || lane > o) xr[t] -= a * xk;
            }
        }
    }
    // backward, upper with reciprocal diagonal, two pivots per round
#pragma unroll
    for (int kb = NS - 1; kb >= 0; kb--) {
        const int k0 = 32 * kb, k1 = min(D, k0 + 32);
        int k = k1 - 1;
#pragma unroll 2
        for (; k - 1 >= k0; k -= 2) {
            const int o = k - k0;  // pivots k and k-1
            const LT xk = __shfl_sync(gm, xr[kb], o) * A[k * LD + k];
            const LT xp = __shfl_sync(gm, xr[kb], o - 1);
            const LT xk1 = (xp - A[(k - 1) * LD + k] * xk) * A[(k - 1) * LD + k - 1];
#pragma unroll
            for (int t = 0; t <= kb; t++) {
                const LT a0 = A[rowc[t] + k], a1 = A[rowc[t] + k - 1];
                if (t < kb || lane < o - 1) {
                    xr[t] -= a0 * xk;
                    xr[t] -= a1 * xk1;
                } else if (lane == o) {
                    xr[t] = xk;
                } else if (lane == o - 1) {
                    xr[t] = xk1;
                }
            }
        }
        if (k >= k0) {  // one pivot left
            const int o = k - k0;
            const LT xk = __shfl_sync(gm, xr[kb], o) * A[k * LD + k];
#pragma unroll
            for (int t = 0; t <= kb; t++) {
                const LT a = A[rowc[t] + k];
                if (t < kb || lane < o) xr[t] -= a * xk;
                else if (lane == o) xr[t] = xk;
            }
        }
    }
    } else {
    // forward, unit lower, SP pivots per round: the not yet final x_k ..
    // x_{k+SP-1} come by independent shuffles, every lane finishes them with
    // the broadcast L entries of the diagonal block (a chain SP-1 deep), then
    // the SP columns update the rows below
#pragma unroll
    for (int kb = 0; kb < NS; kb++) {
        const int k0 = 32 * kb, k1 = min(D, k0 + 32);
        int k = k0;
#pragma unroll 1
        for (; k + SP <= k1; k += SP) {
            const int o = k - k0;
            LT xf[SP];
#pragma unroll
            for (int p = 0; p < SP; p++) xf[p] = __shfl_sync(gm, xr[kb], o + p);
#pragma unroll
            for (int p = 1; p < SP; p++) {
#pragma unroll
                for (int q = 0; q < p; q++) xf[p] -= A[(k + p) * LD + k + q] * xf[q];
            }
#pragma unroll
            for (int t = kb; t < NS; t++) {
                LT a[SP];
#pragma unroll
                for (int p = 0; p < SP; p++) a[p] = A[rowc[t] + k + p];
                if (t > kb || lane > o + SP - 1) {
#pragma unroll
                    for (int p = 0; p < SP; p++) xr[t] -= a[p] * xf[p];
                } else {
#pragma unroll
                    for (int p = 1; p < SP; p++)
                        if (lane == o + p) xr[t] = xf[p];
                }
            }
        }
        for (; k < k1; k++) {  // the block's last pivots, one at a time
            const int o = k - k0;
            const LT xk = __shfl_sync(gm, xr[kb], o);
#pragma unroll
            for (int t = kb; t < NS; t++) {
                const LT a = A[rowc[t] + k];
                if (t > kb || lane > o) xr[t] -= a * xk;
            }
        }
    }
    // backward, upper with reciprocal diagonal, SP pivots per round (k, k-1,
    // ..., k-SP+1)
#pragma unroll
    for (int kb = NS - 1; kb >= 0; kb--) {
        const int k0 = 32 * kb, k1 = min(D, k0 + 32);
        int k = k1 - 1;
#pragma unroll 1
        for (; k - (SP - 1) >= k0; k -= SP) {
            const int o = k - k0;
            LT xf[SP];
#pragma unroll
            for (int p = 0; p < SP; p++) xf[p] = __shfl_sync(gm, xr[kb], o - p);
#pragma unroll
            for (int p = 0; p < SP; p++) {
#pragma unroll
                for (int q = 0; q < p; q++) xf[p] -= A[(k - p) * LD + k - q] * xf[q];
                xf[p] *= A[(k - p) * LD + k - p];
            }
#pragma unroll
            for (int t = 0; t <= kb; t++) {
                LT a[SP];
#pragma unroll
                for (int p = 0; p < SP; p++) a[p] = A[rowc[t] + k - p];
                if (t < kb || lane < o - (SP - 1)) {
#pragma unroll
                    for (int p = 0; p < SP; p++) xr[t] -= a[p] * xf[p];
                } else {
#pragma unroll
                    for (int p = 0; p < SP; p++)
                        if (lane == o - p) xr[t] = xf[p];
                }
            }
        }
        for (; k >= k0; k--) {  // one pivot at a time
            const int o = k - k0;
            const LT xk = __shfl_sync(gm, xr[kb], o) * A[k * LD + k];
#pragma unroll
            for (int t = 0; t <= kb; t++) {
                const LT a = A[rowc[t] + k];
                if (t < kb || lane < o) xr[t] -= a * xk;
                else if (lane == o) xr[t] = xk;
            }
        }
    }
    }
#pragma unroll
    for (int t = 0; t < NS; t++) {
        const int i = lane + 32 * t;
        if (i < D) xb[i] = xr[t];
    }
}

// Pivots per round of the dense block's triangular solves for a cell shape
// and LU precision: 4 for the FP32 LU of 8-slot lanes (measured:
// multiphase-232 +3.6%, water parameter +2.0%; 8 cost it 1%), 2 otherwise
// (4 cost the 3-slot gas-72 kernel 6.6% and the FP64 8-slot kernels 6-7%,
// 3 cost gas-72 3.5%)
template <int G, int NPL, typename LT>
__host__ __device__ constexpr int subst_pivots() { return (sizeof(LT) == 4 && NPL >= 6) ? 4 : 2; }

// SP: pivots per round of the dense block's triangular solves (2 or 4)
template <int G, typename LT, int SP>
__device__ void substitute(const DevMech &m, const CellPtr<LT> &c, int lane, unsigned gm) {
    LT *x = c.x;
    const LT *lu = c.lu;
    gsync<G>(gm);
    // forward, sparse rows and the L21 part of block rows (rows without L
    // entries keep their value); split rows through partials (LU precision,
    // after the rate terms: free while solving)
    LT *xp = (LT *)(c.rs + m.R);
    for (int L = 0; L < m.n_slev; L++) {
        int b = __ldg(m.slev_ptr + L), e = __ldg(m.slev_ptr + L + 1);
        for (int r = b + lane; r < e; r += G) {
            const int2 job = __ldg(m.sjob + r);
            const int i = lo16(job.y);
            LT s = (G == 32 || i < m.n) ? x[i] : (LT)0, s2 = (LT)0;  // one-warp cells: no split rows
            int qb = job.x, qe = job.x + hi16(job.y);
            int q = qb;
            for (; q + 1 < qe; q += 2) {
                const int e2 = __ldg(m.sl_pack + q), e3 = __ldg(m.sl_pack + q + 1);
                s -= lu[lo16(e2)] * x[hi16(e2)];
                s2 += lu[lo16(e3)] * x[hi16(e3)];
            }
            if (q < qe) {
                const int e2 = __ldg(m.sl_pack + q);
                s -= lu[lo16(e2)] * x[hi16(e2)];
            }
            if (G == 32 || i < m.n) x[i] = s - s2;
            else xp[i - m.n] = s - s2;
        }
        gsync<G>(gm);
        if constexpr (G > 32) {
            const int sb = __ldg(m.ssplit_ptr + L), se = __ldg(m.ssplit_ptr + L + 1);
            if (se > sb) {
                for (int k = sb + lane; k < se; k += G) {
                    const int2 sp = __ldg(m.ssplit + k);
                    const int first = lo16(sp.y), cnt = hi16(sp.y);
                    LT t = x[sp.x];
                    for (int j = 0; j < cnt; j++) t += xp[first + j];
                    x[sp.x] = t;
                }
                gsync<G>(gm);
            }
        }
    }
    const LT *A = lu + m.dbase;
    if (G <= 32 || lane < 32) {
        const unsigned wm = G <= 32 ? gm : 0xffffffffu;
        switch ((m.D + 31) >> 5) {
        case 0: break;
        case 1: dense_subst<1, LT, SP>(A, m.D, m.LD, x + m.d, lane, wm); break;
        case 2: dense_subst<2, LT, SP>(A, m.D, m.LD, x + m.d, lane, wm); break;
        case 3: dense_subst<3, LT, SP>(A, m.D, m.LD, x + m.d, lane, wm); break;
        default: dense_subst<4, LT, SP>(A, m.D, m.LD, x + m.d, lane, wm); break;
        }
    }
    gsync<G>(gm);
    // backward, sparse rows by level
    for (int L = 0; L < m.n_blev; L++) {
        int b = __ldg(m.blev_ptr + L), e = __ldg(m.blev_ptr + L + 1);
        for (int r = b + lane; r < e; r += G) {
            int i = __ldg(m.brow + r);
            LT s = x[i], s2 = (LT)0;
            int qb = __ldg(m.su_ptr + i), qe = __ldg(m.su_ptr + i + 1);
            int q = qb;
            for (; q + 1 < qe; q += 2) {
                const int e2 = __ldg(m.su_pack + q), e3 = __ldg(m.su_pack + q + 1);
                s -= lu[lo16(e2)] * x[hi16(e2)];
                s2 += lu[lo16(e3)] * x[hi16(e3)];
            }
            if (q < qe) {
                const int e2 = __ldg(m.su_pack + q);
                s -= lu[lo16(e2)] * x[hi16(e2)];
            }
            x[i] = (s - s2) * lu[__ldg(m.udiag + i)];
        }
        gsync<G>(gm);
    }
}

template <int G, int NPL>
__device__ __forceinline__ double wrms(const DevMech &m, const double (&v)[NPL], const double (&w)[NPL],
                                       unsigned gm) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < NPL; i++) {
        double a = v[i] * w[i];
        s += a * a;
    }
    return sqrt(gsum<G>(s, gm) / (double)m.n);
}

// ---- Nordsieck array operations (q uniform per cell; rows in registers) -----
template <int NPL>
__device__ __forceinline__ void nord_predict(double (&z)[QMAX + 1][NPL], int q) {
#pragma unroll
    for (int k = 0; k < QMAX; k++) {
        if (k < q) {
#pragma unroll
            for (int j = QMAX; j > k; j--) {
                if (j <= q) {
#pragma unroll
                    for (int s = 0; s < NPL; s++) z[j - 1][s] += z[j][s];
                }
            }
        }
    }
}
template <int NPL>
__device__ __forceinline__ void nord_retract(double (&z)[QMAX + 1][NPL], int q) {
#pragma unroll
    for (int k = QMAX - 1; k >= 0; k--) {
        if (k < q) {
#pragma unroll
            for (int j = 1; j <= QMAX; j++) {
                if (j > k && j <= q) {
#pragma unroll
                    for (int s = 0; s < NPL; s++) z[j - 1][s] -= z[j][s];
                }
            }
        }
    }
}
template <int NPL>
__device__ __forceinline__ void nord_rescale(double (&z)[QMAX + 1][NPL], int q, double eta) {
    double f = 1.0;
#pragma unroll
    for (int j = 1; j <= QMAX; j++) {
        if (j <= q) {
            f *= eta;
#pragma unroll
            for (int s = 0; s < NPL; s++) z[j][s] *= f;
        }
    }
}

// x^p for the step-size and order heuristics of the mixed form.  Only the
// accept/reject tests need FP64; a step-size factor needs a few digits, so
// this takes FP32 log2/exp2 (x = 0 gives 0 for p > 0 and +inf for p < 0).
__device__ __forceinline__ float ctl_powf(float x, float p) {
    return exp2f(p * __log2f(x));
}


// 1/d for d > 0 to ~1e-14 relative: an FP32 estimate refined by one
// Newton-Raphson step w <- w (2 - d w) in FP64; outside the FP32 normal
// range a division
__device__ __forceinline__ double recip_refined(double d) {
    if (d > 1e-37 && d < 1e37) {
        const double w = (double)__frcp_rn((float)d);
        return w * fma(-d, w, 2.0);
    }
    return 1.0 / d;
}

// The step controller's scalar arithmetic.  EXACT (the plain FP64 form)
// takes every scalar decision with the oracle's own FP64 operations --
// divisions, square roots and pow -- so that the two follow the same step
// sequence up to the roundoff of f, J and the LU; otherwise (the mixed form)
// the cheaper forms: reciprocals, squared norms and FP32 powers.  A norm v
// is carried as the norm itself (EXACT: v = c WRMS, from a root) or as its
// square (v = (c WRMS)^2, no root); either way the tests compare v with 1.
template <bool EXACT>
struct Ctl {
    // v from the sum s of n squared weighted terms and the coefficient c
    static __device__ __forceinline__ double norm(double c, double c2, double s, int n, double rn) {
        if constexpr (EXACT) return c * sqrt(s / (double)n);
        else return c2 * (s * rn);
    }
    // the step-size factor of order selection, 1 / ((k err)^(1/p) + 1e-6)
    // (the mixed form entirely in FP32: no FP64 division)
    static __device__ __forceinline__ double eta(double k, double v, int p) {
        if constexpr (EXACT) return 1.0 / (pow(k * v, 1.0 / (double)p) + 1e-6);
        else return (double)(1.0f / (ctl_powf((float)(k * k) * (float)v, 0.5f / (float)p) + 1e-6f));
    }
    // 0.9 err^(-1/p): the step factor after an error-test failure
    static __device__ __forceinline__ double fail_eta(double v, int p) {
        if constexpr (EXACT) return 0.9 * pow(v, -1.0 / (double)p);
        else return (double)(0.9f * ctl_powf((float)v, -0.5f / (float)p));
    }
    // a / b for the ratio of step-size coefficients (rb = 1 / b)
    static __device__ __forceinline__ double ratio(double a, double b, double rb) {
        if constexpr (EXACT) return a / b;
        else return a * rb;
    }
    // the error weight 1 / (rtol |y| + atol)
    static __device__ __forceinline__ double weight(double rtol, double y, double atol) {
        if constexpr (EXACT) return 1.0 / __dadd_rn(__dmul_rn(rtol, fabs(y)), atol);
        else return recip_refined(fma(rtol, fabs(y), atol));
    }
};

struct CellStats {
    int steps, newton, jac, errfail, ordsum;
};

// ---- one cell over [0, dt] ---------------------------------------------------
// y_cell/env_cell: this cell's rows (declaration order).  Returns the status;
// the state is written back only on success.  step_io (null: cold start):
// warm start, in: a value > 0 replaces the initial-step estimate; out: the
// step held before the final cut to dt, 0 on failure.  y_copy (or null)
// receives a second copy of the new state on success.
template <int G, int NPL, typename LT, bool W>
__device__ int integrate_cell(const DevMech &m, const CellPtr<LT> &c, double *__restrict__ y_cell,
                              const double *__restrict__ env_cell, double dt, double rtol,
                              const double *__restrict__ atol, int atol_len, int max_steps,
                              double hmin_frac, double *step_io, int lane, unsigned gm,
                              CellStats &st, double *__restrict__ y_copy = nullptr) {
    const int n = m.n;
    constexpr bool EXACT = sizeof(LT) == 8;  // the plain FP64 form
    using C = Ctl<EXACT>;
    const double h_in = step_io ? *step_io : 0.0;
    st.steps = st.newton = st.jac = st.errfail = st.ordsum = 0;

    // inputs must be finite
    bool bad = false;
    for (int i = lane; i < m.n_env; i += G) bad |= !finite_bits(env_cell[i]);
    double z[QMAX + 1][NPL], e[NPL], ep[NPL], w[NPL], f[NPL];
#pragma unroll
    for (int s = 0; s < NPL; s++) {
        int p = lane + G * s;
        double v = 0.0;
        if (p < n) v = y_cell[__ldg(m.perm + p)];
        bad |= !finite_bits(v);
#pragma unroll
        for (int j = 0; j <= QMAX; j++) z[j][s] = 0.0;
        z[0][s] = v;
        e[s] = ep[s] = 0.0;
    }
    // a cell that fails hands back no step (the next call starts cold)
    auto fail_early = [&](int code) {
        if (step_io && lane == 0) *step_io = 0.0;
        return code;
    };
    if (gany<G>(bad, gm)) return fail_early(ST_NONFINITE);

    for (int k = lane; k < m.R; k += G) {
        double a, b;
        rate_constant(m, k, env_cell, a, b);
        c.kf[k] = a;
        const int rv = __ldg(m.rrev + k);
        if (rv >= 0) c.kr[rv] = b;
    }
    gsync<G>(gm);
    if constexpr (W) water_setup<G>(m, c.pw, env_cell, lane, gm);

    // atol is re-read (an L1 hit) rather than held in registers
    auto set_weights = [&]() {
#pragma unroll
        for (int s = 0; s < NPL; s++) {
            int p = lane + G * s;
            double a = 1.0;
            if (p < n) a = atol_len == 1 ? __ldg(atol) : __ldg(atol + __ldg(m.perm + p));
            w[s] = (p < n) ? C::weight(rtol, z[0][s], a) : 0.0;
        }
    };
    auto any_nonfinite = [&](const double(&v)[NPL]) {
        bool b2 = false;
#pragma unroll
        for (int s = 0; s < NPL; s++) b2 |= !finite_bits(v[s]);
        return gany<G>(b2, gm) != 0;
    };

    const double T = dt, hmin = hmin_frac * dt;
    set_weights();
    eval_f<G, NPL, LT, W>(m, c, z[0], f, lane, gm);
    if (any_nonfinite(f)) return fail_early(ST_NONFINITE);

    // initial step: the carried one, else Hairer, Norsett & Wanner's
    // starting-step estimate for order 1
    double h;
    if (h_in > 0.0) {
        h = fmin(h_in, T);
    } else {
        double d0 = wrms<G, NPL>(m, z[0], w, gm), d1 = wrms<G, NPL>(m, f, w, gm);
        double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
        if (h0 > T) h0 = T;
        eval_f_at<G, NPL, LT, W>(m, c, z[0], h0, f, e, lane, gm);
#pragma unroll
        for (int s = 0; s < NPL; s++) ep[s] = e[s] - f[s];  // ep is free until the first step ends
        double d2 = wrms<G, NPL>(m, ep, w, gm) / h0;
        double dm = d1 > d2 ? d1 : d2;
        double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : sqrt(0.01 / dm);
        h = fmin(100.0 * h0, h1);
        if (!(h <= T)) h = T;
    }
#pragma unroll
    for (int s = 0; s < NPL; s++) {
        z[1][s] = h * f[s];
        e[s] = 0.0;
    }

    int q = 1, qwait = 2, nst = 0, nst_lu = 0;
    double h_held = h;
    bool have_lu = false, need_setup = true, ep_valid = false;
    double t = 0.0, gamma_lu = 0.0, rgamma_lu = 0.0;
    int status = ST_OK;
    // The mixed form takes the controller's tests on squared norms (the same
    // decisions as comparing the norms themselves, without roots): Newton
    // converged when dn^2 min(1, rho^2) <= tol^2, diverged when
    // rho^2 > RHO_DIV^2; the step is accepted when ecoef^2 mean((e w)^2) <= 1.
    // The FP64 form compares the norms themselves, as the oracle does
    // (err2 and dn2 then hold the norms, not their squares).
    constexpr double NEWTON_TOL2 = NEWTON_TOL * NEWTON_TOL;
    constexpr double RHO_DIV2 = RHO_DIV * RHO_DIV;

    while (t < T) {
        if (nst >= max_steps) { status = ST_MAXSTEPS; break; }
        set_weights();
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
                    nord_rescale<NPL>(z, q, eta);
                    h = T - t;
                }
                last = true;
            }
            nord_predict<NPL>(z, q);
            const double rl1 = m.inv_l1[q];
            const double gamma = C::ratio(h, m.lcoef[q][1], rl1);
            bool jcur = false, lu_fail = false;
            if (!have_lu || need_setup || nst >= nst_lu + MSBJ ||
                fabs(C::ratio(gamma, gamma_lu, rgamma_lu) - 1.0) > DGMAX) {
#pragma unroll
                for (int s = 0; s < NPL; s++) {
                    int p = lane + G * s;
                    if (p < n) c.ys[p] = z[0][s];
                }
                gsync<G>(gm);
                assemble<G, LT, W>(m, c, gamma, lane, gm, 0, nullptr);
                lu_fail = !factor<G, LT>(m, c, lane, gm);
                st.jac++;
                gamma_lu = gamma;
                rgamma_lu = 1.0 / gamma;
                nst_lu = nst;
                have_lu = !lu_fail;
                need_setup = false;
                jcur = true;
            }
            // modified Newton on G(e) = e - gamma f(z0 + e) + z1 / l1
            bool conv = false;
            if (!lu_fail) {
                LT dprev2 = (LT)0;
#pragma unroll
                for (int s = 0; s < NPL; s++) e[s] = 0.0;
                const LT scale = (gamma != gamma_lu)
                                     ? (LT)2 / ((LT)1 + to_lu<LT>(C::ratio(gamma, gamma_lu, rgamma_lu)))
                                     : (LT)1;
                for (int it = 0; it < NEWTON_MAXIT; it++) {
                    eval_f_at<G, NPL, LT, W>(m, c, z[0], 1.0, e, f, lane, gm);
                    st.newton++;
                    if (any_nonfinite(f)) break;
#pragma unroll
                    for (int s = 0; s < NPL; s++) {
                        int p = lane + G * s;
                        if (p < n) c.x[p] = to_lu<LT>(-(e[s] - gamma * f[s] + z[1][s] * rl1));
                    }
                    substitute<G, LT, subst_pivots<G, NPL, LT>()>(m, c, lane, gm);
                    // the update's norm in the LU precision (it only steers the iteration)
                    LT dsq = (LT)0;
                    bool nf = false;
#pragma unroll
                    for (int s = 0; s < NPL; s++) {
                        int p = lane + G * s;
                        LT xl = (p < n) ? c.x[p] : (LT)0;
                        xl *= scale;
                        e[s] += from_lu(xl);
                        dsq += upd_term(xl, w[s]);
                        nf |= !isfinite(xl);
                    }
                    // EXACT: the norm itself, as the oracle tests it; mixed:
                    // its square in the LU precision
                    const LT dn2 = EXACT ? (LT)sqrt((double)gsum_t<G, LT>(dsq, gm) / (double)n)
                                         : gsum_t<G, LT>(dsq, gm) * (LT)m.rn;
                    if (gany<G>(nf, gm) || !isfinite(dn2)) break;
                    LT test2 = dn2;
                    if (it > 0) {
                        const LT rho2 = dn2 / dprev2;
                        if (rho2 > (LT)(EXACT ? RHO_DIV : RHO_DIV2)) break;
                        if (rho2 < (LT)1) test2 = dn2 * rho2;
                    }
                    if (test2 <= (LT)(EXACT ? NEWTON_TOL : NEWTON_TOL2)) { conv = true; break; }
                    dprev2 = dn2;
                }
            }
            if (!conv) {
                nord_retract<NPL>(z, q);
                if (!jcur) { need_setup = true; continue; }
                if (++ncf >= MAX_NCF) { status = lu_fail ? ST_SINGULAR : ST_NEWTON; break; }
                h *= ETA_CF;
                if (h < hmin) { status = ST_ERRTEST; break; }
                nord_rescale<NPL>(z, q, ETA_CF);
                need_setup = true;
                qwait = q + 1;
                continue;
            }
            {
                double es = 0.0;
#pragma unroll
                for (int s = 0; s < NPL; s++) { double a = e[s] * w[s]; es += a * a; }
                err2 = C::norm(m.ecoef[q], m.ecoef2[q], gsum<G>(es, gm), n, m.rn);
            }
            if (err2 > 1.0) {
                nord_retract<NPL>(z, q);
                st.errfail++;
                if (++nef >= MAX_NEF) { status = ST_ERRTEST; break; }
                if (nef >= 3) {
                    h *= 0.1;
                    if (h < hmin) { status = ST_ERRTEST; break; }
                    q = 1;
                    eval_f<G, NPL, LT, W>(m, c, z[0], f, lane, gm);
#pragma unroll
                    for (int s = 0; s < NPL; s++) z[1][s] = h * f[s];
                } else {
                    double eta = C::fail_eta(err2, q + 1);
                    if (eta < 0.2) eta = 0.2;
                    h *= eta;
                    if (h < hmin) { status = ST_ERRTEST; break; }
                    nord_rescale<NPL>(z, q, eta);
                }
                qwait = q + 1;
                continue;
            }
            accepted = true;
        }
        if (status != ST_OK) break;

        // accept: z += l (x) e
#pragma unroll
        for (int j = 0; j <= QMAX; j++) {
            if (j <= q) {
                const double lj = m.lcoef[q][j];
#pragma unroll
                for (int s = 0; s < NPL; s++) z[j][s] += lj * e[s];
            }
        }
        t = last ? T : t + h;
        nst++;
        st.ordsum += q;
        if (any_nonfinite(z[0])) { status = ST_NONFINITE; break; }

        if (--qwait <= 0 && t < T) {
            // eta = 1 / ((c err)^(1/(p+1)) + 1e-6), from the squared norms
            double eta_q = C::eta(1.2, err2, q + 1);
            double eta_m = 0.0, eta_p = 0.0;
            if (q > 1) {
                double zs = 0.0;
#pragma unroll
                for (int j = 1; j <= QMAX; j++) {
                    if (j == q) {
#pragma unroll
                        for (int s = 0; s < NPL; s++) { double a = z[j][s] * w[s]; zs += a * a; }
                    }
                }
                const double ce = m.ecoef[q - 1] * m.fact[q];
                const double em2 = C::norm(ce, ce * ce, gsum<G>(zs, gm), n, m.rn);
                eta_m = C::eta(1.3, em2, q);
            }
            if (q < QMAX && ep_valid) {
                double ds = 0.0;
#pragma unroll
                for (int s = 0; s < NPL; s++) { double a = (e[s] - ep[s]) * w[s]; ds += a * a; }
                const double ep2 = C::norm(m.ecoef[q + 1], m.ecoef2[q + 1], gsum<G>(ds, gm), n, m.rn);
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
                    const double c_up = m.lcoef[q][q] / (double)(q + 1);
#pragma unroll
                    for (int j = 2; j <= QMAX; j++) {
                        if (j == q + 1) {
#pragma unroll
                            for (int s = 0; s < NPL; s++) z[j][s] = e[s] * c_up;
                        }
                    }
                }
                q = qn;
                h *= eta;
                nord_rescale<NPL>(z, q, eta);
                qwait = q + 1;
            }
        }
#pragma unroll
        for (int s = 0; s < NPL; s++) ep[s] = e[s];
        ep_valid = true;
    }
    st.steps = nst;
    if (status == ST_OK) {
#pragma unroll
        for (int s = 0; s < NPL; s++) {
            int p = lane + G * s;
            if (p < n) {
                const int i = __ldg(m.perm + p);
                y_cell[i] = z[0][s];
                if (y_copy) y_copy[i] = z[0][s];
            }
        }
    }
    if (step_io && lane == 0) *step_io = status == ST_OK ? h_held : 0.0;
    return status;
}

}  // namespace campdev
