/*
 * camp_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct FP64 CPU reference for the batched CAMP
 * chemistry solve.  It is used by the tests, by __graft_entry__.smoke() and by
 * the CPU-baseline leg of bench.py, never by the product path.  It shares no
 * code with the CUDA path: its own mechanism arrays (filled by oracle/mech.py
 * from the JSON text), a naive loop over reactions, a dense analytic Jacobian,
 * a dense partial-pivot LU, and a variable-order Nordsieck BDF written out in
 * the order the steps are taken.
 *
 * Model (CAMP paper, Sect. 2.4.2): f_i = sum_k (dy_i/dt)_k and
 * df_i/dy_j = sum_k (df_i/dy_j)_k over processes k.  Every process here is a
 * mass-action term r_k = kf_k prod_R y^s - kr_k prod_P y^nu with
 * (dy_i/dt)_k = nu_ik r_k (nu negative for reactants); the per-type physics
 * (Table 2) enters only through the pair (kf_k, kr_k).
 *
 * Parameters (Sect. 2.2.2): a ZSR aerosol-water parameter makes the liquid
 * volume L_b of each section a function of the state; the constants of the
 * section processes then carry powers of 1/L_b(y), and the Jacobian gains
 * the chain-rule term J_p P_y (om_jacobian_env).
 *
 * State units: ppb-equivalent of air for every species (our reading; the
 * paper does not state solver units).  Constants: exact SI 2019 values.
 *
 * Integrator (Sect. 2.4.1 names CVODE's variable-order BDF with Newton
 * iteration; the controller constants below are our own, stated once here):
 *   Nordsieck array z[0..q] of order q <= 5, fixed-step l-vector of
 *   prod_{i=1..q}(1 + x/i), gamma = h / l_1, modified Newton on
 *   G(e) = e - gamma f(y0 + e) + z_1 / l_1 with at most 3 iterations,
 *   local error E = e / ((q+1) l_1), WRMS norms with w = 1/(rtol|y| + atol).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- mechanism arrays (filled from JSON by oracle/mech.py) -------------- */
enum { OM_ARRHENIUS = 0, OM_TROE = 1, OM_PHOTOLYSIS = 2, OM_EMISSION = 3,
       OM_LOSS = 4, OM_HENRY = 5, OM_AQREV = 6, OM_CUSTOM_H2O2 = 7, OM_CUSTOM_OH_HNO3 = 8,
       OM_COND_ARRHENIUS = 9, OM_SIMPOL = 10 };

#define OM_MAXSP 4
typedef struct {
    int type;
    int n_react;            /* distinct reactants */
    int react[OM_MAXSP];    /* species index */
    int rstoich[OM_MAXSP];  /* integer multiplicity */
    int n_prod;             /* distinct products */
    int prod[OM_MAXSP];
    double yield[OM_MAXSP]; /* product yields (integers for reversible types) */
    int env_slot;           /* runtime parameter: index into env */
    int section;            /* section index for section processes, else -1 */
    double p[10];           /* type parameters, see om_rate_constants */
} om_rxn;

#define OM_ZSR_NY 8         /* coefficients of one molality fit */

typedef struct {
    int n_species;
    int n_rxn;
    int n_env;
    int n_sections;
    int env_section_base;   /* env index of section 0's radius */
    const om_rxn *rxn;
    /* ZSR aerosol-water parameter (Sect. 2.2.2, Table 4, ZSRAerosolWater):
     * with n_zsr > 0 the liquid volume of every section is a function of the
     * state, computed from its electrolytes at the cell's relative humidity */
    int rh_slot;              /* env index of the relative humidity (0..1), -1 if none */
    int n_zsr;                /* electrolytes (0: no water parameter) */
    const int *zsr_species;   /* [n_sections][n_zsr] species of electrolyte e in section b */
    const double *zsr_Y;      /* [n_zsr][OM_ZSR_NY] molality fit, sqrt(m) = sum_j Y_j a_w^j */
    const double *zsr_low;    /* [n_zsr] lowest water activity of the fit */
} om_mech;

/* ---- physical constants (SI 2019, exact) -------------------------------- */
static const double KB = 1.380649e-23;     /* J K^-1 */
static const double NA = 6.02214076e23;    /* mol^-1 */
#define RGAS (KB * NA)                      /* J mol^-1 K^-1 */
static const double PI = 3.14159265358979323846;

/* ---- status codes -------------------------------------------------------- */
enum { OM_OK = 0, OM_MAXSTEPS = 1, OM_ERRTEST = 2, OM_NEWTON = 3, OM_SINGULAR = 4,
       OM_NONFINITE = 5 };

/* ---- integrator constants (our choices; the paper gives none) ---------- */
#define QMAX 5
#define NEWTON_MAXIT 3
#define NEWTON_TOL 0.1      /* convergence bound on the WRMS Newton update */
#define RHO_DIV 2.0         /* divergence: ratio of successive updates */
#define DGMAX 0.3           /* refresh J/LU when |gamma/gamma_LU - 1| > DGMAX */
#define MSBJ 20             /* ... or every MSBJ steps */
#define ETA_MAX 10.0
#define ETA_THRESH 1.5      /* step changes smaller than this are skipped */
#define ETA_CF 0.25         /* step factor after a Newton failure */
#define MAX_NEF 7           /* error-test failures in one step -> status 2 */
#define MAX_NCF 10          /* Newton failures in one step -> status 3 */

typedef struct {
    int max_steps;
    double hmin_frac;       /* h_min = hmin_frac * dt */
} om_opts;

/* ======================================================================== */
/* Rate constants: Table 2 of the paper, plus the unit factors of our ppb   */
/* state.  kf multiplies prod_R y^s, kr multiplies prod_P y^nu (ppb s^-1).  */
/* ======================================================================== */
static double ipow(double x, int n) {
    double r = 1.0;
    for (int i = 0; i < n; i++) r *= x;
    return r;
}

/* Arrhenius with D = 300 K and E = 0: A exp(C/T) (T/300)^B, the building
 * block of the Troe and custom rate constants (Table 2) */
static double arr300(double A, double B, double C, double T) {
    return A * exp(C / T) * pow(T / 300.0, B);
}

/* Gas-to-particle mass transfer of one section, s^-1 (Table 2,
 * HenrysLawPhaseTransfer; Zaveri et al. 2008): N particles of radius rad
 * each collect 4 pi rad Dg f_fs(Kn, alpha) with the Fuchs-Sutugin factor
 * f_fs = 0.75 alpha (1 + Kn) / (Kn^2 + Kn + 0.283 Kn alpha + 0.75 alpha),
 * Kn = lambda / rad, mean free path lambda = 3 Dg / cbar and mean speed
 * cbar = sqrt(8 R T / (pi MW)). */
static double mass_transfer(double rad, double Np, double alpha, double Dg, double MW,
                            double T) {
    double cbar = sqrt(8.0 * RGAS * T / (PI * MW));
    double lambda = 3.0 * Dg / cbar;
    double Kn = lambda / rad;
    double ffs = 0.75 * alpha * (1.0 + Kn) / (Kn * Kn + Kn + 0.283 * Kn * alpha + 0.75 * alpha);
    return Np * 4.0 * PI * rad * Dg * ffs;
}

/* Liquid volume of section b [m^3 per m^3 air] that enters the rate
 * constants: the env value, or 1 when a water parameter makes it a function
 * of the state.  In that case kf and kr are per unit volume and the powers of
 * 1/L of water_powers() are applied wherever the state is known. */
static double section_volume(const om_mech *m, const double *env, int b) {
    return m->n_zsr > 0 ? 1.0 : env[m->env_section_base + 3 * b + 2];
}

void om_rate_constants(const om_mech *m, const double *env, double *kf, double *kr) {
    const double T = env[0], P = env[1];
    const double Mair = P / (KB * T) * 1e-6;   /* air number density, molec cm^-3 */
    const double mppb = Mair * 1e-9;            /* molec cm^-3 per ppb */
    for (int k = 0; k < m->n_rxn; k++) {
        const om_rxn *r = &m->rxn[k];
        int nr = 0, np = 0;
        for (int i = 0; i < r->n_react; i++) nr += r->rstoich[i];
        for (int i = 0; i < r->n_prod; i++) np += (int)r->yield[i];
        kf[k] = 0.0;
        kr[k] = 0.0;
        switch (r->type) {
        case OM_ARRHENIUS: {
            /* k = A exp(C/T) (T/D)^B (1 + E P), C = -Ea/k_B  (Table 2, Arrhenius) */
            double A = r->p[0], B = r->p[1], C = r->p[2], D = r->p[3], E = r->p[4];
            double k0 = A * exp(C / T) * pow(T / D, B) * (1.0 + E * P);
            kf[k] = k0 * ipow(mppb, nr - 1);
            break;
        }
        case OM_TROE: {
            /* k = k0[M]/(1 + k0[M]/kinf) * Fc^(1/(1 + (log10(k0[M]/kinf)/N)^2)),
             * k0 and kinf Arrhenius with D = 300, E = 0  (Table 2, Troe) */
            double k0 = r->p[0] * exp(r->p[2] / T) * pow(T / 300.0, r->p[1]);
            double ki = r->p[3] * exp(r->p[5] / T) * pow(T / 300.0, r->p[4]);
            double Fc = r->p[6], N = r->p[7];
            double x = k0 * Mair / ki;
            double lg = log10(x) / N;
            double kt = k0 * Mair / (1.0 + x) * pow(Fc, 1.0 / (1.0 + lg * lg));
            kf[k] = kt * ipow(mppb, nr - 1);
            break;
        }
        case OM_PHOTOLYSIS:  /* first order, J from the host (Table 2, Photolysis) */
        case OM_LOSS:        /* first order (Table 2, FirstOrderLoss) */
        case OM_EMISSION:    /* zero order, ppb s^-1 (Table 2, Emission) */
            kf[k] = env[r->env_slot];
            break;
        case OM_HENRY: {
            /* H(T) = H298 exp(C (1/T - 1/298)) [M Pa^-1]; condensation k_c of
             * the section (Table 2, HenrysLawPhaseTransfer); evaporation
             * k_c / (H_cc L) with the dimensionless H_cc = 1000 H R T, so
             * that at equilibrium y_aq / y_gas = H_cc L. */
            int b = r->section;
            double rad = env[m->env_section_base + 3 * b];
            double Np = env[m->env_section_base + 3 * b + 1];
            double L = section_volume(m, env, b);
            if (!(L > 0.0 && Np > 0.0 && rad > 0.0)) break;
            double H = r->p[0] * exp(r->p[1] * (1.0 / T - 1.0 / 298.0));
            double Hcc = 1000.0 * H * RGAS * T;
            double kb = mass_transfer(rad, Np, r->p[2], r->p[3], r->p[4], T);
            kf[k] = kb;
            kr[k] = kb / (Hcc * L);
            break;
        }
        case OM_SIMPOL: {
            /* Condensation as for Henry's law; evaporation from the SIMPOL.1
             * vapour pressure log10 p0 [atm] = B1/T + B2 + B3 T + B4 ln T
             * (Table 2, SimpolPhaseTransfer).  Reading: the condensed phase
             * is an ideal solution of fixed total molarity c_tot, so Raoult's
             * law p = (c / c_tot) p0 acts as Henry's law with
             * H = c_tot / p0 [M Pa^-1]. */
            int b = r->section;
            double rad = env[m->env_section_base + 3 * b];
            double Np = env[m->env_section_base + 3 * b + 1];
            double L = section_volume(m, env, b);
            if (!(L > 0.0 && Np > 0.0 && rad > 0.0)) break;
            double lg = r->p[0] / T + r->p[1] + r->p[2] * T + r->p[3] * log(T);
            double p0 = 101325.0 * pow(10.0, lg);          /* Pa */
            double H = r->p[7] / p0;
            double Hcc = 1000.0 * H * RGAS * T;
            double kb = mass_transfer(rad, Np, r->p[4], r->p[5], r->p[6], T);
            kf[k] = kb;
            kr[k] = kb / (Hcc * L);
            break;
        }
        case OM_AQREV: {
            /* K_eq = A exp(C (1/T - 1/298)); forward = K_eq kr (Table 2,
             * AqueousReversible).  Molarity c = y * phi with
             * phi = 1e-9 P / (R T 1000 L) [M per ppb]; the rate in M s^-1 is
             * divided by phi to return to ppb s^-1. */
            int b = r->section;
            double L = section_volume(m, env, b);
            if (!(L > 0.0)) break;
            double Keq = r->p[0] * exp(r->p[1] * (1.0 / T - 1.0 / 298.0));
            double krev = r->p[2];
            double phi = 1e-9 * P / (RGAS * T * 1000.0 * L);
            kf[k] = Keq * krev * ipow(phi, nr - 1);
            kr[k] = krev * ipow(phi, np - 1);
            break;
        }
        case OM_CUSTOM_H2O2: {
            /* k = k1 + k2 [M], k1 and k2 Arrhenius with D = 300, E = 0
             * (Table 2, CustomH2o2) */
            double k1 = arr300(r->p[0], r->p[1], r->p[2], T);
            double k2 = arr300(r->p[3], r->p[4], r->p[5], T);
            kf[k] = (k1 + k2 * Mair) * ipow(mppb, nr - 1);
            break;
        }
        case OM_CUSTOM_OH_HNO3: {
            /* k = k0 + k3[M] / (1 + k3[M] / k2), all Arrhenius with D = 300,
             * E = 0 (Table 2, CustomOhHno3) */
            double k0 = arr300(r->p[0], r->p[1], r->p[2], T);
            double k2 = arr300(r->p[3], r->p[4], r->p[5], T);
            double k3M = arr300(r->p[6], r->p[7], r->p[8], T) * Mair;
            kf[k] = (k0 + k3M / (1.0 + k3M / k2)) * ipow(mppb, nr - 1);
            break;
        }
        case OM_COND_ARRHENIUS: {
            /* Arrhenius in a condensed phase instance, M^(1-nr) s^-1 for the
             * aqueous phase (Table 2, CondensedPhaseArrhenius): the rate in
             * M s^-1 is k prod c with c = y phi, returned to ppb s^-1 by
             * dividing by phi, so kf = k phi^(nr - 1). */
            int b = r->section;
            double L = section_volume(m, env, b);
            if (!(L > 0.0)) break;
            double A = r->p[0], B = r->p[1], C = r->p[2], D = r->p[3], E = r->p[4];
            double kk = A * exp(C / T) * pow(T / D, B) * (1.0 + E * P);
            double phi = 1e-9 * P / (RGAS * T * 1000.0 * L);
            kf[k] = kk * ipow(phi, nr - 1);
            break;
        }
        }
    }
}

/* ======================================================================== */
/* Forcing f(y) and dense Jacobian (Sect. 2.4.2): naive loop over processes */
/* ======================================================================== */
static double rate_of(const om_rxn *r, double kf, double kr, const double *y) {
    double a = kf;
    for (int i = 0; i < r->n_react; i++) a *= ipow(y[r->react[i]], r->rstoich[i]);
    double b = 0.0;
    if (kr != 0.0) {
        b = kr;
        for (int i = 0; i < r->n_prod; i++) b *= ipow(y[r->prod[i]], (int)r->yield[i]);
    }
    return a - b;
}

void om_forcing(const om_mech *m, const double *kf, const double *kr, const double *y,
                double *f) {
    for (int i = 0; i < m->n_species; i++) f[i] = 0.0;
    for (int k = 0; k < m->n_rxn; k++) {
        const om_rxn *r = &m->rxn[k];
        double rk = rate_of(r, kf[k], kr[k], y);
        for (int i = 0; i < r->n_react; i++) f[r->react[i]] -= r->rstoich[i] * rk;
        for (int i = 0; i < r->n_prod; i++) f[r->prod[i]] += r->yield[i] * rk;
    }
}

/* d r_k / d y_j for a species j; product rule over integer powers */
static double drate(const om_rxn *r, double kf, double kr, const double *y, int j) {
    double d = 0.0;
    for (int a = 0; a < r->n_react; a++) {
        if (r->react[a] != j) continue;
        double t = kf * r->rstoich[a] * ipow(y[j], r->rstoich[a] - 1);
        for (int i = 0; i < r->n_react; i++)
            if (i != a) t *= ipow(y[r->react[i]], r->rstoich[i]);
        d += t;
    }
    if (kr != 0.0) {
        for (int a = 0; a < r->n_prod; a++) {
            if (r->prod[a] != j) continue;
            int nu = (int)r->yield[a];
            double t = kr * nu * ipow(y[j], nu - 1);
            for (int i = 0; i < r->n_prod; i++)
                if (i != a) t *= ipow(y[r->prod[i]], (int)r->yield[i]);
            d -= t;
        }
    }
    return d;
}

/* J row-major [n][n]: J[i*n + j] = d f_i / d y_j */
void om_jacobian(const om_mech *m, const double *kf, const double *kr, const double *y,
                 double *J) {
    int n = m->n_species;
    memset(J, 0, sizeof(double) * (size_t)n * n);
    for (int k = 0; k < m->n_rxn; k++) {
        const om_rxn *r = &m->rxn[k];
        /* species that appear in r_k */
        int dep[2 * OM_MAXSP], nd = 0;
        for (int i = 0; i < r->n_react; i++) dep[nd++] = r->react[i];
        if (kr[k] != 0.0)
            for (int i = 0; i < r->n_prod; i++) dep[nd++] = r->prod[i];
        for (int a = 0; a < nd; a++) {
            int j = dep[a], seen = 0;
            for (int b = 0; b < a; b++) seen |= (dep[b] == j);
            if (seen) continue;
            double d = drate(r, kf[k], kr[k], y, j);
            for (int i = 0; i < r->n_react; i++) J[r->react[i] * n + j] -= r->rstoich[i] * d;
            for (int i = 0; i < r->n_prod; i++) J[r->prod[i] * n + j] += r->yield[i] * d;
        }
    }
}

/* ======================================================================== */
/* ZSR aerosol water as a parameter (Sect. 2.2.2; Table 4, ZSRAerosolWater) */
/* ======================================================================== */
/* Powers of 1/L in kf (*la) and kr (*lb) of a section process when the
 * liquid volume L is a parameter.  A molarity is y phi with phi proportional
 * to 1/L, and a rate in M s^-1 returns to ppb s^-1 through one division by
 * phi, so a side with f concentration factors carries L^-(f-1); the
 * evaporation constant k_c / (H_cc L) of the phase-transfer types carries
 * L^-1. */
static void water_powers(const om_rxn *r, int *la, int *lb) {
    int nr = 0, np = 0;
    for (int i = 0; i < r->n_react; i++) nr += r->rstoich[i];
    for (int i = 0; i < r->n_prod; i++) np += (int)r->yield[i];
    *la = 0;
    *lb = 0;
    switch (r->type) {
    case OM_HENRY:
    case OM_SIMPOL: *lb = 1; break;
    case OM_AQREV: *la = nr - 1; *lb = np - 1; break;
    case OM_COND_ARRHENIUS: *la = nr - 1; break;
    }
}

/* Molality [mol per kg water] of electrolyte e alone in water at water
 * activity a_w, from a fit of the Jacobson et al. (1996) form
 * sqrt(m) = sum_j Y_j a_w^j; below the fit's lowest activity a_w is held
 * there. */
static double zsr_molality(const om_mech *m, int e, double aw) {
    if (aw < m->zsr_low[e]) aw = m->zsr_low[e];
    double s = 0.0, p = 1.0;
    for (int j = 0; j < OM_ZSR_NY; j++) {
        s += m->zsr_Y[e * OM_ZSR_NY + j] * p;
        p *= aw;
    }
    return s * s;
}

/* Liquid water volume per ppb of electrolyte e [m^3 per m^3 air per ppb]:
 * the ZSR water W = sum_i 1000 M_i / (MW_i m_i(a_w)) (Table 4), in kg per
 * m^3 of air with M_i in kg m^-3 and MW_i in g mol^-1, so that 1000 M_i /
 * MW_i is the electrolyte's molar concentration, 1e-9 P / (R T) mol m^-3 per
 * ppb; divided by the density of water, 1000 kg m^-3.  The water activity
 * is the relative humidity.  An electrolyte whose fitted molality is not
 * positive holds no water. */
static double zsr_weight(const om_mech *m, const double *env, int e) {
    const double T = env[0], P = env[1];
    double mol = zsr_molality(m, e, env[m->rh_slot]);
    if (!(mol > 0.0) || !isfinite(mol)) return 0.0;
    return 1e-9 * P / (RGAS * T) / mol / 1000.0;
}

/* Liquid volume of every section at state y: the env value plus the ZSR
 * water of the section's electrolytes. */
void om_water(const om_mech *m, const double *env, const double *y, double *L) {
    for (int b = 0; b < m->n_sections; b++) {
        double v = env[m->env_section_base + 3 * b + 2];
        for (int e = 0; e < m->n_zsr; e++)
            v += zsr_weight(m, env, e) * y[m->zsr_species[b * m->n_zsr + e]];
        L[b] = v;
    }
}

/* kf, kr of om_rate_constants (per unit volume on the sections) with the
 * powers of 1/L at the current liquid volumes applied.  A section whose
 * water is not positive takes no part, as a section with no water in env
 * does (its processes' constants are 0). */
static void volume_constants(const om_mech *m, const double *kf, const double *kr,
                             const double *L, double *kfe, double *kre) {
    for (int k = 0; k < m->n_rxn; k++) {
        const om_rxn *r = &m->rxn[k];
        kfe[k] = kf[k];
        kre[k] = kr[k];
        if (r->section < 0) continue;
        if (!(L[r->section] > 0.0)) {
            kfe[k] = kre[k] = 0.0;
            continue;
        }
        int la, lb;
        water_powers(r, &la, &lb);
        kfe[k] = kf[k] / ipow(L[r->section], la);
        kre[k] = kr[k] / ipow(L[r->section], lb);
    }
}

/* f(y) of a mechanism whose parameters are evaluated at y first (Sect.
 * 2.2.2: the processes use the parameters' current values). */
void om_forcing_env(const om_mech *m, const double *env, const double *kf, const double *kr,
                    const double *y, double *f) {
    if (m->n_zsr == 0) {
        om_forcing(m, kf, kr, y, f);
        return;
    }
    double *L = malloc(sizeof(double) * (size_t)(m->n_sections + 2 * m->n_rxn));
    double *kfe = L + m->n_sections, *kre = kfe + m->n_rxn;
    om_water(m, env, y, L);
    volume_constants(m, kf, kr, L, kfe, kre);
    om_forcing(m, kfe, kre, y, f);
    free(L);
}

/* The solver's Jacobian by the chain rule of Sect. 2.2.2: the processes'
 * partial derivatives with the parameters held at their values (J_y), plus
 * the partial derivatives of the forcing with respect to the parameters
 * (J_p, n x S) times those of the parameters with respect to the state
 * (P_y, S x n):  J = J_y + J_p P_y.  For the liquid volume of section b,
 * d r_k / d L_b = -(la F_k - lb B_k) / L_b with F_k and B_k the forward and
 * reverse terms of r_k = F_k - B_k, and d L_b / d y_j is electrolyte j's
 * water per ppb. */
void om_jacobian_env(const om_mech *m, const double *env, const double *kf, const double *kr,
                     const double *y, double *J) {
    if (m->n_zsr == 0) {
        om_jacobian(m, kf, kr, y, J);
        return;
    }
    const int n = m->n_species, S = m->n_sections;
    double *L = malloc(sizeof(double) * (size_t)(S + 2 * m->n_rxn));
    double *kfe = L + S, *kre = kfe + m->n_rxn;
    double *Jp = calloc((size_t)n * S, sizeof(double));
    double *Py = calloc((size_t)S * n, sizeof(double));
    om_water(m, env, y, L);
    volume_constants(m, kf, kr, L, kfe, kre);
    om_jacobian(m, kfe, kre, y, J);                        /* J_y */
    for (int k = 0; k < m->n_rxn; k++) {                   /* J_p */
        const om_rxn *r = &m->rxn[k];
        if (r->section < 0) continue;
        int la, lb;
        water_powers(r, &la, &lb);
        if (la == 0 && lb == 0) continue;
        double F = kfe[k], B = 0.0;
        for (int i = 0; i < r->n_react; i++) F *= ipow(y[r->react[i]], r->rstoich[i]);
        if (kre[k] != 0.0) {
            B = kre[k];
            for (int i = 0; i < r->n_prod; i++) B *= ipow(y[r->prod[i]], (int)r->yield[i]);
        }
        const int b = r->section;
        if (!(L[b] > 0.0)) continue;   /* a dry section takes no part */
        double dr = -(la * F - lb * B) / L[b];
        for (int i = 0; i < r->n_react; i++) Jp[r->react[i] * S + b] -= r->rstoich[i] * dr;
        for (int i = 0; i < r->n_prod; i++) Jp[r->prod[i] * S + b] += r->yield[i] * dr;
    }
    for (int b = 0; b < S; b++)                            /* P_y */
        for (int e = 0; e < m->n_zsr; e++)
            Py[b * n + m->zsr_species[b * m->n_zsr + e]] += zsr_weight(m, env, e);
    for (int i = 0; i < n; i++)                            /* J += J_p P_y */
        for (int b = 0; b < S; b++) {
            double a = Jp[i * S + b];
            if (a == 0.0) continue;
            for (int j = 0; j < n; j++) J[i * n + j] += a * Py[b * n + j];
        }
    free(Py);
    free(Jp);
    free(L);
}

/* ======================================================================== */
/* Dense LU with partial pivoting (textbook Doolittle, row swaps)           */
/* ======================================================================== */
/* Factor A (row-major n x n) in place; piv[k] = row swapped into k.  Returns 0
 * on success, 1 if a pivot is exactly zero or not finite. */
int om_lu_factor(int n, double *A, int *piv) {
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(A[k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double v = fabs(A[i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (!(best > 0.0) || !isfinite(best)) return 1;
        if (p != k)
            for (int j = 0; j < n; j++) {
                double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t;
            }
        for (int i = k + 1; i < n; i++) {
            double l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            if (l != 0.0)
                for (int j = k + 1; j < n; j++) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return 0;
}

void om_lu_solve(int n, const double *LU, const int *piv, double *b) {
    for (int k = 0; k < n; k++)
        if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int j = 0; j < i; j++) s -= LU[i * n + j] * b[j];
        b[i] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = b[i];
        for (int j = i + 1; j < n; j++) s -= LU[i * n + j] * b[j];
        b[i] = s / LU[i * n + i];
    }
}

/* ======================================================================== */
/* BDF coefficients                                                          */
/* ======================================================================== */
/* l[q][j]: coefficients of prod_{i=1..q} (1 + x/i); tq[q] = 1/((q+1) l_1(q)),
 * the local-error constant of BDF-q applied to the correction e_n. */
static double LCOEF[QMAX + 2][QMAX + 2];
static double ECOEF[QMAX + 2];
static double FACT[QMAX + 2];
static pthread_once_t coef_once = PTHREAD_ONCE_INIT;

static void coef_init(void) {
    memset(LCOEF, 0, sizeof(LCOEF));
    for (int q = 1; q <= QMAX + 1; q++) {
        double c[QMAX + 2] = {1.0};
        for (int i = 1; i <= q; i++)            /* multiply by (1 + x/i) */
            for (int j = i; j >= 1; j--) c[j] += c[j - 1] / i;
        for (int j = 0; j <= q; j++) LCOEF[q][j] = c[j];
        ECOEF[q] = 1.0 / ((q + 1) * LCOEF[q][1]);
    }
    FACT[0] = 1.0;
    for (int i = 1; i <= QMAX + 1; i++) FACT[i] = FACT[i - 1] * i;
}

void om_bdf_coefficients(int q, double *l, double *ecoef) {
    pthread_once(&coef_once, coef_init);
    for (int j = 0; j <= QMAX + 1; j++) l[j] = LCOEF[q][j];
    *ecoef = ECOEF[q];
}

/* ======================================================================== */
/* Variable-order, variable-step Nordsieck BDF for one cell                  */
/* ======================================================================== */
typedef struct {
    const om_mech *m;
    int n;
    const double *env;
    const double *kf, *kr;
    double *J, *LU, *tmp;
    int *piv;
    int nfe, nje, nni, nef_total;
} om_ctx;

static void fval(om_ctx *c, const double *y, double *f) {
    om_forcing_env(c->m, c->env, c->kf, c->kr, y, f);
    c->nfe++;
}

static double wrms(int n, const double *v, const double *w) {
    double s = 0.0;
    for (int i = 0; i < n; i++) { double a = v[i] * w[i]; s += a * a; }
    return sqrt(s / n);
}

static int all_finite(int n, const double *v) {
    for (int i = 0; i < n; i++) if (!isfinite(v[i])) return 0;
    return 1;
}

/* z[0..q] <- Pascal(z): the Taylor predictor */
static void predict(int n, int q, double *z) {
    for (int k = 0; k < q; k++)
        for (int j = q; j > k; j--)
            for (int i = 0; i < n; i++) z[(j - 1) * n + i] += z[j * n + i];
}

/* exact inverse of predict(): the same elementary updates in reverse order */
static void retract(int n, int q, double *z) {
    for (int k = q - 1; k >= 0; k--)
        for (int j = k + 1; j <= q; j++)
            for (int i = 0; i < n; i++) z[(j - 1) * n + i] -= z[j * n + i];
}

static void rescale(int n, int q, double *z, double eta) {
    double s = 1.0;
    for (int j = 1; j <= q; j++) {
        s *= eta;
        for (int i = 0; i < n; i++) z[j * n + i] *= s;
    }
}

/* Evaluate J at y, form M = I - gamma J and factor it.  Returns 0 on success. */
static int setup(om_ctx *c, const double *y, double gamma) {
    int n = c->n;
    om_jacobian_env(c->m, c->env, c->kf, c->kr, y, c->J);
    for (int i = 0; i < n * n; i++) c->LU[i] = -gamma * c->J[i];
    for (int i = 0; i < n; i++) c->LU[i * n + i] += 1.0;
    c->nje++;
    return om_lu_factor(n, c->LU, c->piv);
}

/* Modified Newton on G(e) = e - gamma f(z0 + e) + z1/l1.  On return e holds the
 * correction; returns 1 if converged. */
static int newton(om_ctx *c, const double *z, int q, double gamma, double gamma_lu,
                  const double *w, double *e, double *ycur, double *f, double *del) {
    int n = c->n;
    double l1 = LCOEF[q][1];
    double dprev = 0.0;
    for (int i = 0; i < n; i++) { e[i] = 0.0; ycur[i] = z[i]; }
    for (int m = 0; m < NEWTON_MAXIT; m++) {
        fval(c, ycur, f);
        c->nni++;
        if (!all_finite(n, f)) return 0;
        for (int i = 0; i < n; i++) del[i] = -(e[i] - gamma * f[i] + z[n + i] / l1);
        om_lu_solve(n, c->LU, c->piv, del);
        if (gamma != gamma_lu) {
            double s = 2.0 / (1.0 + gamma / gamma_lu);
            for (int i = 0; i < n; i++) del[i] *= s;
        }
        for (int i = 0; i < n; i++) { e[i] += del[i]; ycur[i] = z[i] + e[i]; }
        double dn = wrms(n, del, w);
        if (!isfinite(dn)) return 0;
        double test = dn;
        if (m > 0) {
            double rho = dn / dprev;
            if (rho > RHO_DIV) return 0;
            if (rho < 1.0) test = dn * rho;
        }
        if (test <= NEWTON_TOL) return 1;
        dprev = dn;
    }
    return 0;
}

/* Initial step (Hairer, Norsett & Wanner, Solving ODEs I, Sect. II.4, with
 * order 1 and our WRMS norm), capped by dt. */
static double initial_step(om_ctx *c, const double *y0, const double *f0, const double *w,
                           double dt, double *y1, double *f1) {
    int n = c->n;
    double d0 = wrms(n, y0, w), d1 = wrms(n, f0, w);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    if (h0 > dt) h0 = dt;
    for (int i = 0; i < n; i++) y1[i] = y0[i] + h0 * f0[i];
    fval(c, y1, f1);
    for (int i = 0; i < n; i++) y1[i] = f1[i] - f0[i];
    double d2 = wrms(n, y1, w) / h0;
    double dm = d1 > d2 ? d1 : d2;
    double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : sqrt(0.01 / dm);
    double h = fmin(100.0 * h0, h1);
    if (!(h <= dt)) h = dt;   /* also catches NaN */
    return h;
}

/* Integrate one cell over [0, dt].  y in/out (unchanged unless status 0);
 * stats (may be NULL): steps, Newton iterations, Jacobian evaluations,
 * error-test failures.
 * step (may be NULL: every call a cold start, the paper's behaviour): warm
 * start across consecutive calls for the same cell.  On input *step > 0
 * replaces the initial-step estimate (the integration still starts at order
 * 1, with h = min(*step, dt)); on output *step is the step size the
 * controller held before the final step was cut to land on dt, or 0 if the
 * cell failed. */
static int integrate_cell(const om_mech *m, const double *env, double *y, double dt, double rtol,
                          const double *atol, int atol_len, const om_opts *o, int *stats,
                          double *step) {
    const double h_in = step ? *step : 0.0;
    if (step) *step = 0.0;
    int n = m->n_species;
    for (int i = 0; i < n; i++) if (!isfinite(y[i])) return OM_NONFINITE;
    for (int i = 0; i < m->n_env; i++) if (!isfinite(env[i])) return OM_NONFINITE;

    size_t nn = (size_t)n;
    double *buf = calloc((size_t)(QMAX + 2) * nn + 10 * nn + 2 * nn * nn + 2 * (size_t)m->n_rxn, sizeof(double));
    int *piv = calloc(nn, sizeof(int));
    double *z = buf;                     /* (QMAX+2) x n */
    double *w = z + (QMAX + 2) * nn, *e = w + nn, *ep = e + nn, *ycur = ep + nn, *f = ycur + nn;
    double *del = f + nn, *tmp = del + nn, *tmp2 = tmp + nn, *y1 = tmp2 + nn, *f1 = y1 + nn;
    double *J = f1 + nn, *LU = J + nn * nn, *kf = LU + nn * nn, *kr = kf + m->n_rxn;

    om_ctx c = {m, n, env, kf, kr, J, LU, tmp, piv, 0, 0, 0, 0};
    om_rate_constants(m, env, kf, kr);
    int status = OM_OK;
    int q = 1, qwait = 2, nst = 0, have_lu = 0, need_setup = 1, nst_lu = 0, ep_valid = 0;
    double t = 0.0, gamma_lu = 0.0;

    const double T = dt, hmin = o->hmin_frac * dt;
    for (int i = 0; i < n; i++) w[i] = 1.0 / (rtol * fabs(y[i]) + atol[atol_len == 1 ? 0 : i]);
    fval(&c, y, f);
    if (!all_finite(n, f)) { status = OM_NONFINITE; goto done; }
    double h = h_in > 0.0 ? fmin(h_in, dt) : initial_step(&c, y, f, w, dt, y1, f1);
    double h_held = h;  /* the step before any cut to land on dt */
    for (int i = 0; i < n; i++) { z[i] = y[i]; z[n + i] = h * f[i]; }

    while (t < T) {
        if (nst >= o->max_steps) { status = OM_MAXSTEPS; goto done; }
        for (int i = 0; i < n; i++) w[i] = 1.0 / (rtol * fabs(z[i]) + atol[atol_len == 1 ? 0 : i]);
        int nef = 0, ncf = 0, last;
        double err;
        for (;;) {                               /* attempts at one step */
            last = 0;
            h_held = h;
            if (t + h >= T) {
                if (t + h > T) { double eta = (T - t) / h; rescale(n, q, z, eta); h = T - t; }
                last = 1;
            }
            predict(n, q, z);
            double gamma = h / LCOEF[q][1];
            int jcur = 0, lu_fail = 0;
            if (!have_lu || need_setup || nst >= nst_lu + MSBJ ||
                fabs(gamma / gamma_lu - 1.0) > DGMAX) {
                lu_fail = setup(&c, z, gamma);
                gamma_lu = gamma; nst_lu = nst; have_lu = !lu_fail; need_setup = 0; jcur = 1;
            }
            int conv = lu_fail ? 0 : newton(&c, z, q, gamma, gamma_lu, w, e, ycur, f, del);
            if (!conv) {
                retract(n, q, z);
                if (!jcur) { need_setup = 1; continue; }   /* retry with a fresh J */
                if (++ncf >= MAX_NCF) { status = lu_fail ? OM_SINGULAR : OM_NEWTON; goto done; }
                h *= ETA_CF;
                if (h < hmin) { status = OM_ERRTEST; goto done; }
                rescale(n, q, z, ETA_CF);
                need_setup = 1;
                qwait = q + 1;
                continue;
            }
            err = ECOEF[q] * wrms(n, e, w);
            if (err > 1.0) {                      /* error test failed */
                retract(n, q, z);
                c.nef_total++;
                if (++nef >= MAX_NEF) { status = OM_ERRTEST; goto done; }
                if (nef >= 3) {
                    /* repeated failures: restart at order 1 from a fresh derivative */
                    h *= 0.1;
                    if (h < hmin) { status = OM_ERRTEST; goto done; }
                    q = 1;
                    fval(&c, z, f);
                    for (int i = 0; i < n; i++) z[n + i] = h * f[i];
                } else {
                    double eta = 0.9 * pow(err, -1.0 / (q + 1));
                    if (eta < 0.2) eta = 0.2;
                    h *= eta;
                    if (h < hmin) { status = OM_ERRTEST; goto done; }
                    rescale(n, q, z, eta);
                }
                qwait = q + 1;
                continue;
            }
            break;                                 /* accepted */
        }
        /* accept: z <- z_pred + l (x) e */
        for (int j = 0; j <= q; j++)
            for (int i = 0; i < n; i++) z[j * n + i] += LCOEF[q][j] * e[i];
        t = last ? T : t + h;
        nst++;
        if (!all_finite(n, z)) { status = OM_NONFINITE; goto done; }

        /* step size and order selection */
        if (--qwait <= 0 && t < T) {
            double eta_q = 1.0 / (pow(1.2 * err, 1.0 / (q + 1)) + 1e-6);
            double eta_m = 0.0, eta_p = 0.0;
            if (q > 1) {
                double em = ECOEF[q - 1] * FACT[q] * wrms(n, z + (size_t)q * n, w);
                eta_m = 1.0 / (pow(1.3 * em, 1.0 / q) + 1e-6);
            }
            if (q < QMAX && ep_valid) {
                for (int i = 0; i < n; i++) tmp2[i] = e[i] - ep[i];
                double epl = ECOEF[q + 1] * wrms(n, tmp2, w);
                eta_p = 1.0 / (pow(1.4 * epl, 1.0 / (q + 2)) + 1e-6);
            }
            double eta = eta_q;
            int qn = q;
            if (eta_m > eta) { eta = eta_m; qn = q - 1; }
            if (eta_p > eta) { eta = eta_p; qn = q + 1; }
            if (eta < ETA_THRESH) {
                qwait = 2;
            } else {
                if (eta > ETA_MAX) eta = ETA_MAX;
                if (qn == q + 1)
                    for (int i = 0; i < n; i++) z[(q + 1) * n + i] = e[i] * LCOEF[q][q] / (q + 1);
                q = qn;
                h *= eta;
                rescale(n, q, z, eta);
                qwait = q + 1;
            }
        }
        for (int i = 0; i < n; i++) ep[i] = e[i];
        ep_valid = 1;
    }
    for (int i = 0; i < n; i++) y[i] = z[i];
    if (step) *step = h_held;
done:
    if (stats) {
        stats[0] = nst;
        stats[1] = c.nni;
        stats[2] = c.nje;
        stats[3] = c.nef_total;
    }
    free(buf);
    free(piv);
    return status;
}

/* ---- public entry points (called through ctypes) ----------------------- */
int om_integrate(const om_mech *m, const double *env, double *y, double dt, double rtol,
                 const double *atol, int atol_len, int max_steps, double hmin_frac, int *stats,
                 double *step) {
    om_opts o = {max_steps, hmin_frac};
    pthread_once(&coef_once, coef_init);
    if (stats) memset(stats, 0, 4 * sizeof(int));
    return integrate_cell(m, env, y, dt, rtol, atol, atol_len, &o, stats, step);
}

typedef struct {
    const om_mech *m;
    int64_t n_cells;
    double *y;
    const double *env;
    double dt, rtol;
    const double *atol;
    int atol_len;
    om_opts o;
    int *status, *stats;
    double *step;
    int64_t next;
    pthread_mutex_t lock;
} om_job;

static void *worker(void *arg) {
    om_job *j = arg;
    int n = j->m->n_species, ne = j->m->n_env;
    double *yc = malloc(sizeof(double) * n);
    for (;;) {
        pthread_mutex_lock(&j->lock);
        int64_t cell = j->next++;
        pthread_mutex_unlock(&j->lock);
        if (cell >= j->n_cells) break;
        memcpy(yc, j->y + cell * n, sizeof(double) * n);
        int st[4] = {0, 0, 0, 0};
        int s = integrate_cell(j->m, j->env + cell * ne, yc, j->dt, j->rtol, j->atol,
                               j->atol_len, &j->o, st, j->step ? j->step + cell : NULL);
        if (s == OM_OK) memcpy(j->y + cell * n, yc, sizeof(double) * n);
        j->status[cell] = s;
        if (j->stats) memcpy(j->stats + 4 * cell, st, sizeof(st));
    }
    free(yc);
    return NULL;
}

/* Integrate n_cells independent cells, y [n_cells][n] in/out, env
 * [n_cells][n_env], with n_threads host threads.  Cells whose status is not 0
 * keep their input state.  step [n_cells] (may be NULL): warm start, as in
 * integrate_cell. */
void om_solve(const om_mech *m, int64_t n_cells, double *y, const double *env, double dt,
              double rtol, const double *atol, int atol_len, int max_steps, double hmin_frac,
              int *status, int *stats, double *step, int n_threads) {
    pthread_once(&coef_once, coef_init);
    om_job j = {m, n_cells, y, env, dt, rtol, atol, atol_len, {max_steps, hmin_frac},
                status, stats, step, 0, PTHREAD_MUTEX_INITIALIZER};
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * n_threads);
    for (int i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, worker, &j);
    for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&j.lock);
}

/* One BDF step at fixed order q and step h from the Nordsieck array z
 * [(q+1) x n] (test hook for the coefficient pins): predict, fresh Jacobian,
 * Newton to convergence, correct.  Writes the corrected array to z_out, the
 * correction to e_out and returns the WRMS of the local-error estimate
 * (negative if Newton failed). */
double om_bdf_step(const om_mech *m, const double *env, const double *z_in, int q, double h,
                   double rtol, const double *atol, int atol_len, double *z_out, double *e_out) {
    pthread_once(&coef_once, coef_init);
    int n = m->n_species;
    size_t nn = (size_t)n;
    double *buf = calloc(8 * nn + 3 * nn * nn + 2 * (size_t)m->n_rxn, sizeof(double));
    int *piv = calloc(nn, sizeof(int));
    double *w = buf, *ycur = w + nn, *f = ycur + nn, *del = f + nn, *tmp = del + nn;
    double *J = tmp + 3 * nn, *LU = J + nn * nn, *kf = LU + 2 * nn * nn, *kr = kf + m->n_rxn;
    om_ctx c = {m, n, env, kf, kr, J, LU, tmp, piv, 0, 0, 0, 0};
    om_rate_constants(m, env, kf, kr);
    memcpy(z_out, z_in, sizeof(double) * (q + 1) * nn);
    for (int i = 0; i < n; i++) w[i] = 1.0 / (rtol * fabs(z_in[i]) + atol[atol_len == 1 ? 0 : i]);
    predict(n, q, z_out);
    double gamma = h / LCOEF[q][1];
    double res = -1.0;
    if (setup(&c, z_out, gamma) == 0 &&
        newton(&c, z_out, q, gamma, gamma, w, e_out, ycur, f, del)) {
        for (int j = 0; j <= q; j++)
            for (int i = 0; i < n; i++) z_out[j * n + i] += LCOEF[q][j] * e_out[i];
        res = ECOEF[q] * wrms(n, e_out, w);
    }
    free(buf);
    free(piv);
    return res;
}
