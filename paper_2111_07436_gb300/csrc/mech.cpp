// Mechanism compiler (host, once per mechanism).
//
// CAMP paper Sect. 2.2: a mechanism is a set of processes over the gas phase
// and over every instance of an aerosol phase (Sect. 2.2.3: a process
// declared on a phase is applied to each instance of it; here one instance per
// section).  Table 1: each process declares the Jacobian elements it touches
// (get_used_jacobian_elements) and receives the ids of its species and
// Jacobian elements (update_ids).  This file does both, then orders the
// unknowns, computes the LU fill and emits flat device tables.
#include "mech.hpp"

#include <algorithm>
#include <map>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <string>
#include <unordered_map>

#include "json.hpp"

namespace camp {
using campjson::Value;

static const double kBoltzmann = 1.380649e-23;

static int type_code(const std::string &t) {
    if (t == "ARRHENIUS") return CAMP_P_ARRHENIUS;
    if (t == "TROE") return CAMP_P_TROE;
    if (t == "PHOTOLYSIS") return CAMP_P_PHOTOLYSIS;
    if (t == "EMISSION") return CAMP_P_EMISSION;
    if (t == "FIRST_ORDER_LOSS") return CAMP_P_LOSS;
    if (t == "HL_PHASE_TRANSFER") return CAMP_P_HENRY;
    if (t == "AQUEOUS_REVERSIBLE") return CAMP_P_AQREV;
    if (t == "CUSTOM_H2O2") return CAMP_P_CUSTOM_H2O2;
    if (t == "CUSTOM_OH_HNO3") return CAMP_P_CUSTOM_OH_HNO3;
    if (t == "CONDENSED_ARRHENIUS") return CAMP_P_COND_ARRHENIUS;
    if (t == "SIMPOL_PHASE_TRANSFER") return CAMP_P_SIMPOL;
    throw std::runtime_error("unknown reaction type '" + t + "'");
}

static bool is_runtime(int t) {
    return t == CAMP_P_PHOTOLYSIS || t == CAMP_P_EMISSION || t == CAMP_P_LOSS;
}
static bool is_sectioned(int t) {
    return t == CAMP_P_HENRY || t == CAMP_P_AQREV || t == CAMP_P_COND_ARRHENIUS || t == CAMP_P_SIMPOL;
}

// total molarity of a condensed phase when a SIMPOL process names none: water
static const double kWaterMolarity = 1000.0 / 18.015;

// Arrhenius parameters A, B, C (from C or Ea), D, E into par[0..4]
static void arrhenius_params(const Value &r, double *par) {
    par[0] = r.number("A");
    par[1] = r.number_or("B", 0.0);
    par[2] = r.find("C") ? r.number("C") : -r.number_or("Ea", 0.0) / kBoltzmann;
    par[3] = r.number_or("D", 300.0);
    par[4] = r.number_or("E", 0.0);
}

// A, B, C of the Arrhenius terms <prefix>_A/_B/_C (D = 300 K, E = 0)
static void arr300_params(const Value &r, const char *prefix, double *par) {
    const std::string p(prefix);
    par[0] = r.number(p + "_A");
    par[1] = r.number_or(p + "_B", 0.0);
    par[2] = r.number_or(p + "_C", 0.0);
}

template <class T>
static void add_coef(std::vector<std::pair<int, T>> &v, int idx, T c) {
    for (auto &e : v)
        if (e.first == idx) { e.second += c; return; }
    v.emplace_back(idx, c);
}

static int as_multiplicity(double v, const char *what) {
    if (!(v >= 1.0) || v != std::floor(v) || v > 3.0)
        throw std::runtime_error(std::string(what) + " must be an integer in 1..3");
    return (int)v;
}

// ---- species and processes -------------------------------------------------
static void read_processes(const Value &root, HostMech &h, int instances) {
    const Value &sp = root.at("species");
    if (sp.kind != Value::Array) throw std::runtime_error("'species' must be an array");
    for (auto &s : sp.arr) h.species.push_back(s.string("name"));
    h.n_gas = (int)h.species.size();
    std::vector<std::string> phase;
    if (const Value *a = root.find("aerosol")) {
        h.n_sections = instances >= 0 ? instances : (int)a->number("sections");
        if (h.n_sections < 0 || h.n_sections > 1024) throw std::runtime_error("bad section count");
        const Value &ph = root.at("phases").at(a->string("phase"));
        for (auto &p : ph.arr) phase.push_back(p.string("name"));
        for (int b = 0; b < h.n_sections; b++)
            for (auto &p : phase) h.species.push_back("bin" + std::to_string(b) + "." + p);
    }
    h.n = (int)h.species.size();
    std::unordered_map<std::string, int> index;
    for (int i = 0; i < h.n; i++)
        if (!index.emplace(h.species[i], i).second)
            throw std::runtime_error("duplicate species '" + h.species[i] + "'");
    auto idx = [&](const std::string &name) {
        auto it = index.find(name);
        if (it == index.end()) throw std::runtime_error("unknown species '" + name + "'");
        return it->second;
    };

    const Value &rx = root.at("reactions");
    if (rx.kind != Value::Array) throw std::runtime_error("'reactions' must be an array");
    int n_runtime = 0;
    for (auto &r : rx.arr) n_runtime += is_runtime(type_code(r.string("type")));
    // parameters (Sect. 2.2.2): a ZSR aerosol-water parameter of the phase,
    // one instance per section
    if (const Value *pars = root.find("parameters")) {
        if (pars->kind != Value::Array) throw std::runtime_error("'parameters' must be an array");
        for (auto &par : pars->arr) {
            if (par.string("type") != "ZSR_AEROSOL_WATER")
                throw std::runtime_error("unknown parameter type '" + par.string("type") + "'");
            if (!h.el_phase.empty() || h.n_sections == 0)
                throw std::runtime_error("one water parameter, on a mechanism with aerosol sections");
            const Value &els = par.at("electrolytes");
            if (els.kind != Value::Array || els.arr.empty())
                throw std::runtime_error("a water parameter needs electrolytes");
            for (auto &e : els.arr) {
                auto it = std::find(phase.begin(), phase.end(), e.string("species"));
                if (it == phase.end()) throw std::runtime_error("electrolyte '" + e.string("species") + "' is not a phase species");
                h.el_phase.push_back((int)(it - phase.begin()));
                const Value &Y = e.at("Y");
                if (Y.kind != Value::Array || Y.arr.empty() || Y.arr.size() > CAMP_ZSR_NY)
                    throw std::runtime_error("an electrolyte's 'Y' must hold 1 to 8 numbers");
                for (int j = 0; j < CAMP_ZSR_NY; j++) h.zsr_Y.push_back(j < (int)Y.arr.size() ? Y.arr[j].num : 0.0);
                h.zsr_low.push_back(e.number_or("low_RH", 0.0));
            }
        }
    }
    const bool water = !h.el_phase.empty();
    h.rh_slot = water ? 2 + n_runtime : -1;
    h.env_sec_base = 2 + n_runtime + (water ? 1 : 0);
    h.n_env = h.env_sec_base + 3 * h.n_sections;

    int slot = 2;
    for (auto &r : rx.arr) {
        int t = type_code(r.string("type"));
        if (is_sectioned(t)) {
            for (int b = 0; b < h.n_sections; b++) {
                std::string pre = "bin" + std::to_string(b) + ".";
                Process p;
                p.type = t;
                p.slot = b;
                if (t == CAMP_P_HENRY) {
                    p.react.emplace_back(idx(r.string("gas")), 1);
                    p.prod.emplace_back(idx(pre + r.string("aqueous")), 1.0);
                    p.par[0] = r.number("H298");
                    p.par[1] = r.number_or("C_H", 0.0);
                    p.par[2] = r.number("alpha");
                    p.par[3] = r.number("Dg");
                    p.par[4] = r.number("MW");
                } else if (t == CAMP_P_SIMPOL) {
                    p.react.emplace_back(idx(r.string("gas")), 1);
                    p.prod.emplace_back(idx(pre + r.string("aqueous")), 1.0);
                    const Value &B = r.at("B");
                    if (B.kind != Value::Array || B.arr.empty() || B.arr.size() > 4)
                        throw std::runtime_error("SIMPOL 'B' must hold 1 to 4 numbers");
                    for (size_t i = 0; i < B.arr.size(); i++) p.par[i] = B.arr[i].num;
                    p.par[4] = r.number("alpha");
                    p.par[5] = r.number("Dg");
                    p.par[6] = r.number("MW");
                    p.par[7] = r.number_or("c_tot", kWaterMolarity);
                } else if (t == CAMP_P_COND_ARRHENIUS) {
                    for (auto &kv : r.at("reactants").obj)
                        add_coef(p.react, idx(pre + kv.first), as_multiplicity(kv.second.num, "stoichiometry"));
                    if (const Value *pr = r.find("products"))
                        for (auto &kv : pr->obj) add_coef(p.prod, idx(pre + kv.first), kv.second.num);
                    arrhenius_params(r, p.par);
                } else {
                    for (auto &kv : r.at("reactants").obj)
                        add_coef(p.react, idx(pre + kv.first), as_multiplicity(kv.second.num, "stoichiometry"));
                    for (auto &kv : r.at("products").obj)
                        add_coef(p.prod, idx(pre + kv.first), (double)as_multiplicity(kv.second.num, "stoichiometry"));
                    p.par[0] = r.number("A");
                    p.par[1] = r.number_or("C", 0.0);
                    p.par[2] = r.number("kr");
                }
                h.procs.push_back(p);
            }
            continue;
        }
        Process p;
        p.type = t;
        if (t == CAMP_P_EMISSION) {
            p.prod.emplace_back(idx(r.string("species")), 1.0);
        } else if (t == CAMP_P_LOSS) {
            p.react.emplace_back(idx(r.string("species")), 1);
        } else {
            for (auto &kv : r.at("reactants").obj)
                add_coef(p.react, idx(kv.first), as_multiplicity(kv.second.num, "stoichiometry"));
            if (const Value *pr = r.find("products"))
                for (auto &kv : pr->obj) add_coef(p.prod, idx(kv.first), kv.second.num);
            if (t == CAMP_P_ARRHENIUS) {
                arrhenius_params(r, p.par);
            } else if (t == CAMP_P_CUSTOM_H2O2) {
                arr300_params(r, "k1", p.par);
                arr300_params(r, "k2", p.par + 3);
            } else if (t == CAMP_P_CUSTOM_OH_HNO3) {
                arr300_params(r, "k0", p.par);
                arr300_params(r, "k2", p.par + 3);
                arr300_params(r, "k3", p.par + 6);
            } else if (t == CAMP_P_TROE) {
                p.par[0] = r.number("k0_A");
                p.par[1] = r.number_or("k0_B", 0.0);
                p.par[2] = r.number_or("k0_C", 0.0);
                p.par[3] = r.number("kinf_A");
                p.par[4] = r.number_or("kinf_B", 0.0);
                p.par[5] = r.number_or("kinf_C", 0.0);
                p.par[6] = r.number_or("Fc", 0.6);
                p.par[7] = r.number_or("N", 1.0);
            }
        }
        if (is_runtime(t)) p.slot = slot++;
        h.procs.push_back(p);
    }
    for (auto &p : h.procs) {
        int nr = 0, np = 0;
        for (auto &e : p.react) nr += e.second;
        if (nr > CAMP_MAXFAC) throw std::runtime_error("more than 3 reactant factors in one process");
        if (p.reversible()) {
            for (auto &e : p.prod) np += (int)e.second;
            if (np > CAMP_MAXFAC) throw std::runtime_error("more than 3 product factors in a reversible process");
        }
        if ((p.type == CAMP_P_AQREV || p.type == CAMP_P_COND_ARRHENIUS) && nr == 0)
            throw std::runtime_error("a condensed-phase reaction needs reactants");
        if (p.type == CAMP_P_AQREV && np == 0)
            throw std::runtime_error("a reversible aqueous reaction needs products");
        // with a water parameter: powers of 1/L in kf and kr.  A molarity is
        // y phi, phi ~ 1/L, and one division by phi returns a rate in M s^-1
        // to ppb s^-1, so a side with f concentration factors carries
        // L^-(f-1); the evaporation constant k_c / (H_cc L) carries L^-1
        if (water && is_sectioned(p.type)) {
            if (p.type == CAMP_P_HENRY || p.type == CAMP_P_SIMPOL) p.lb = 1;
            if (p.type == CAMP_P_AQREV) { p.la = nr - 1; p.lb = np - 1; }
            if (p.type == CAMP_P_COND_ARRHENIUS) p.la = nr - 1;
        }
    }
}

// species index of electrolyte e in section b
static int electrolyte_species(const HostMech &h, int b, int e) {
    const int n_phase = (h.n - h.n_gas) / h.n_sections;
    return h.n_gas + b * n_phase + h.el_phase[e];
}

// ---- integer structure -----------------------------------------------------
static std::vector<int> dependence(const Process &p) {  // species entering r_k
    std::vector<int> d;
    for (auto &e : p.react) if (std::find(d.begin(), d.end(), e.first) == d.end()) d.push_back(e.first);
    if (p.reversible())
        for (auto &e : p.prod) if (std::find(d.begin(), d.end(), e.first) == d.end()) d.push_back(e.first);
    return d;
}
static std::vector<int> touched(const Process &p) {   // rows of f it changes
    std::vector<int> d;
    for (auto &e : p.react) if (std::find(d.begin(), d.end(), e.first) == d.end()) d.push_back(e.first);
    for (auto &e : p.prod) if (std::find(d.begin(), d.end(), e.first) == d.end()) d.push_back(e.first);
    return d;
}
static double net_coef(const Process &p, int s) {
    double v = 0.0;
    for (auto &e : p.react) if (e.first == s) v -= e.second;
    for (auto &e : p.prod) if (e.first == s) v += e.second;
    return v;
}

static int field16(int v) {
    if (v < -1 || v > 32766) throw std::runtime_error("index does not fit a 16-bit table field");
    return v < 0 ? 0xffff : v;
}

static void pack_records(HostMech &h) {
    const int R = (int)h.procs.size(), n = h.n;
    h.rpack.assign((size_t)R * 4, 0);
    for (int k = 0; k < R; k++) {
        const int *f = &h.rfac[(size_t)k * 6];
        int *o = &h.rpack[(size_t)k * 4];
        o[0] = field16(f[0]) | (field16(f[1]) << 16);
        o[1] = field16(f[2]) | (field16(h.rrev[k]) << 16);
        o[2] = field16(f[3]) | (field16(f[4]) << 16);
        o[3] = field16(f[5]);
        // the water parameter: section + 1 and the powers of 1/L
        const Process &p = h.procs[k];
        if (!h.el_phase.empty() && is_sectioned(p.type)) {
            if (p.slot + 1 > 0x7ff || p.la > 3 || p.lb > 3) throw std::runtime_error("water tag does not fit");
            o[3] |= ((p.slot + 1) | (p.la << 11) | (p.lb << 13)) << 16;
        }
    }
    // gather entries as 4 bytes each: process | index into the table of the
    // mechanism's distinct coefficients << 16
    h.fcoef.clear();
    h.fpk.assign(h.fk.size(), 0);
    {
        std::unordered_map<uint64_t, int> seen;
        for (size_t q = 0; q < h.fk.size(); q++) {
            uint64_t bits;
            std::memcpy(&bits, &h.fc[q], 8);
            auto it = seen.find(bits);
            int ci;
            if (it == seen.end()) {
                ci = (int)h.fcoef.size();
                seen.emplace(bits, ci);
                h.fcoef.push_back(h.fc[q]);
            } else {
                ci = it->second;
            }
            if (h.fk[q] > 0xffff || ci > 0xffff) throw std::runtime_error("forcing table does not fit 16-bit fields");
            h.fpk[q] = h.fk[q] | (ci << 16);
        }
    }

    const int nnzJ = (int)h.colidx.size();
    h.jnz.assign((size_t)nnzJ * 4, 0);
    for (int t = 0; t < nnzJ; t++) {
        h.jnz[(size_t)t * 4 + 0] = h.jptr[t];
        h.jnz[(size_t)t * 4 + 1] = h.jptr[t + 1];
        h.jnz[(size_t)t * 4 + 2] = h.jdst[t];
        h.jnz[(size_t)t * 4 + 3] = h.jdiag[t];
    }
    // per-lane flat Jacobian entry lists, longest-processing-time over the lanes
    {
        const int NL = h.lanes;
        std::vector<int> order(nnzJ);
        for (int t = 0; t < nnzJ; t++) order[t] = t;
        auto cnt = [&](int t) { return std::max(1, h.jptr[t + 1] - h.jptr[t]); };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cnt(a) > cnt(b); });
        std::vector<std::vector<int>> lanes(NL);
        std::vector<int> load(NL, 0);
        for (int t : order) {
            int best = 0;
            for (int l = 1; l < NL; l++)
                if (load[l] < load[best]) best = l;
            lanes[best].push_back(t);
            load[best] += cnt(t);
        }
        if (nnzJ > 65535) throw std::runtime_error("too many Jacobian non-zeros for the packed records");
        h.jl_ptr.assign(1, 0);
        h.jl_rec.clear();
        auto emit = [&](float c, int k, int o1, int o2, int t, bool last) {
            int cb;
            std::memcpy(&cb, &c, 4);
            h.jl_rec.push_back(cb);
            h.jl_rec.push_back((k & 0xffff) | (field16(o1) << 16));
            h.jl_rec.push_back(h.jdst[t] | (h.jdiag[t] << 16) | ((last ? 1 : 0) << 17));
            h.jl_rec.push_back(field16(o2) | (t << 16));
        };
        for (auto &v : lanes) {
            for (int t : v) {
                int b = h.jptr[t], e = h.jptr[t + 1];
                if (b == e) emit(0.0f, 0, -1, -1, t, true);
                for (int q = b; q < e; q++) {
                    if (h.jk[q] < -32768 || h.jk[q] > 32767) throw std::runtime_error("process index too large");
                    emit((float)h.jc[q], h.jk[q], h.jo[2 * q], h.jo[2 * q + 1], t, q == e - 1);
                }
            }
            h.jl_ptr.push_back((int)h.jl_rec.size() / 4);
        }
    }
    h.sl_pack.resize(h.sl_off.size());
    for (size_t q = 0; q < h.sl_off.size(); q++) h.sl_pack[q] = field16(h.sl_off[q]) | (field16(h.sl_col[q]) << 16);
    h.su_pack.resize(h.su_off.size());
    for (size_t q = 0; q < h.su_off.size(); q++) h.su_pack[q] = field16(h.su_off[q]) | (field16(h.su_col[q]) << 16);
}

static void build_structure(HostMech &h) {
    const int n = h.n;
    std::vector<char> pat((size_t)n * n, 0);
    for (int i = 0; i < n; i++) pat[(size_t)i * n + i] = 1;
    for (auto &p : h.procs)
        for (int j : dependence(p))
            for (int i : touched(p)) pat[(size_t)i * n + j] = 1;
    // chain rule through the water parameter (Sect. 2.2.2): a process whose
    // constants carry a power of 1/L_b reaches every electrolyte of section b
    for (auto &p : h.procs)
        if (p.la || p.lb)
            for (size_t e = 0; e < h.el_phase.size(); e++)
                for (int i : touched(p)) pat[(size_t)i * n + electrolyte_species(h, p.slot, (int)e)] = 1;
    h.rowptr.assign(1, 0);
    h.colidx.clear();
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) if (pat[(size_t)i * n + j]) h.colidx.push_back(j);
        h.rowptr.push_back((int)h.colidx.size());
    }
    auto csr_pos = [&](int i, int j) {
        auto b = h.colidx.begin() + h.rowptr[i], e = h.colidx.begin() + h.rowptr[i + 1];
        auto it = std::lower_bound(b, e, j);
        return (int)(it - h.colidx.begin());
    };
    h.rxn_map.clear();
    for (auto &p : h.procs)
        for (int j : dependence(p))
            for (int i : touched(p)) h.rxn_map.push_back(csr_pos(i, j));

    // exact minimum degree on pattern | pattern^T without the diagonal
    std::vector<char> adj((size_t)n * n, 0);
    std::vector<int> deg(n, 0);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            if (i != j && (pat[(size_t)i * n + j] || pat[(size_t)j * n + i])) adj[(size_t)i * n + j] = 1;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) deg[i] += adj[(size_t)i * n + j];
    std::vector<char> alive(n, 1);
    h.perm.clear();
    std::vector<int> nb;
    for (int step = 0; step < n; step++) {
        int v = -1;
        for (int a = 0; a < n; a++)
            if (alive[a] && (v < 0 || deg[a] < deg[v])) v = a;
        h.perm.push_back(v);
        nb.clear();
        for (int a = 0; a < n; a++) if (alive[a] && adj[(size_t)v * n + a]) nb.push_back(a);
        for (int a : nb)
            for (int b : nb)
                if (a != b && !adj[(size_t)a * n + b]) { adj[(size_t)a * n + b] = 1; deg[a]++; }
        for (int a : nb) { adj[(size_t)a * n + v] = 0; deg[a]--; }
        alive[v] = 0;
    }
    h.iperm.assign(n, 0);
    for (int k = 0; k < n; k++) h.iperm[h.perm[k]] = k;

    // symbolic LU of the permuted pattern, no pivoting
    std::vector<char> S((size_t)n * n, 0);
    for (int i = 0; i < n; i++)
        for (int q = h.rowptr[i]; q < h.rowptr[i + 1]; q++)
            S[(size_t)h.iperm[i] * n + h.iperm[h.colidx[q]]] = 1;
    for (int k = 0; k < n; k++)
        for (int i = k + 1; i < n; i++) {
            if (!S[(size_t)i * n + k]) continue;
            for (int j = k + 1; j < n; j++)
                if (S[(size_t)k * n + j]) S[(size_t)i * n + j] = 1;
        }
    h.lu_rowptr.assign(1, 0);
    h.lu_colidx.clear();
    for (int i = 0; i < n; i++) {
        for (int j = 0; j < n; j++) if (S[(size_t)i * n + j]) h.lu_colidx.push_back(j);
        h.lu_rowptr.push_back((int)h.lu_colidx.size());
    }
    h.level_fwd.assign(n, 0);
    for (int i = 0; i < n; i++) {
        int lv = -1;
        for (int q = h.lu_rowptr[i]; q < h.lu_rowptr[i + 1]; q++) {
            int k = h.lu_colidx[q];
            if (k < i) lv = std::max(lv, h.level_fwd[k]);
        }
        h.level_fwd[i] = lv + 1;
    }
    h.level_bwd.assign(n, 0);
    for (int i = n - 1; i >= 0; i--) {
        int lv = -1;
        for (int q = h.lu_rowptr[i]; q < h.lu_rowptr[i + 1]; q++) {
            int j = h.lu_colidx[q];
            if (j > i) lv = std::max(lv, h.level_bwd[j]);
        }
        h.level_bwd[i] = lv + 1;
    }
}

// Order the rows of one level, rows[b, e), so that the G lanes of a cell get
// even work: lane l takes positions b + l, b + l + G, ...  Rows go heaviest
// first to the lane with the least work among those with a free position.
template <class Cost>
static void balance_level(std::vector<int> &rows, int b, int e, int G, Cost cost) {
    const int len = e - b;
    if (len <= G) {  // one row per lane: order only
        std::stable_sort(rows.begin() + b, rows.begin() + e, [&](int x, int y) { return cost(x) > cost(y); });
        return;
    }
    std::vector<int> sorted(rows.begin() + b, rows.begin() + e);
    std::stable_sort(sorted.begin(), sorted.end(), [&](int x, int y) { return cost(x) > cost(y); });
    std::vector<long long> load(G, 0);
    std::vector<std::vector<int>> mine(G);
    std::vector<int> cap(G);
    for (int l = 0; l < G; l++) cap[l] = (len - l + G - 1) / G;
    for (int r : sorted) {
        int best = -1;
        for (int l = 0; l < G; l++)
            if ((int)mine[l].size() < cap[l] && (best < 0 || load[l] < load[best])) best = l;
        mine[best].push_back(r);
        load[best] += cost(r);
    }
    for (int l = 0; l < G; l++)
        for (size_t k = 0; k < mine[l].size(); k++) rows[b + l + G * (int)k] = mine[l][k];
}

// The sparse factorisation as lane jobs, level by level.  A row whose ops
// far exceed its level's mean load per lane (the arrow rows of a
// particle-resolved mechanism: one gas species against every particle) is
// cut at pivot boundaries into chunks that run on different lanes: each
// chunk's pivots read only columns no other chunk writes, and its updates of
// columns that several chunks (or the rest of the row) write go to chunk
// partial sums.  One lane then adds the partials in order and finishes the
// row's remaining pivots (the tail).
// How one long row splits for a chunk length CH: chunks of op indices (at
// pivot boundaries, none writing a column another chunk's pivot reads), the
// first op of the tail, and the shared columns (written by several chunks
// or by the tail), each of which takes one partial slot per chunk.
struct RowSplit {
    std::vector<std::vector<int>> chunks;
    int tail_from = 0;
    std::vector<int> shared;
    std::unordered_map<int, int> slot;
};
static RowSplit split_row(const std::vector<uint32_t> &ops, int CH) {
    auto tgt = [](uint32_t op) { return (int)(op & 0xFFFFu); };
    RowSplit rs;
    std::vector<std::pair<int, int>> groups;  // [begin, end) in ops: a DIV and its updates
    for (int q = 0; q < (int)ops.size(); q++) {
        if ((ops[q] & CAMP_OP_DIV) || groups.empty()) groups.push_back({q, q + 1});
        else groups.back().second = q + 1;
    }
    std::unordered_map<int, std::vector<int>> writers;  // column -> chunks writing it
    std::vector<int> cur;
    rs.tail_from = (int)ops.size();
    for (auto &g : groups) {
        const int c = (int)rs.chunks.size();
        auto it = writers.find(tgt(ops[g.first]));
        bool foreign = false;
        if (it != writers.end())
            for (int w : it->second) foreign |= (w != c);
        if (foreign) { rs.tail_from = g.first; break; }
        for (int q = g.first; q < g.second; q++) {
            cur.push_back(q);
            auto &v = writers[tgt(ops[q])];
            if (v.empty() || v.back() != c) v.push_back(c);
        }
        if ((int)cur.size() >= CH) { rs.chunks.push_back(cur); cur.clear(); }
    }
    if (!cur.empty()) rs.chunks.push_back(cur);
    if (rs.chunks.size() < 2) return rs;
    std::unordered_map<int, int> tail_cols;
    for (int q = rs.tail_from; q < (int)ops.size(); q++) tail_cols[tgt(ops[q])] = 1;
    for (auto &g : groups)
        for (int q = g.first; q < g.second && q < rs.tail_from; q++) {
            const int t = tgt(ops[q]);
            if (rs.slot.count(t)) continue;
            if (writers[t].size() >= 2 || tail_cols.count(t)) {
                rs.slot[t] = (int)rs.shared.size();
                rs.shared.push_back(t);
            }
        }
    return rs;
}

// Partial slots one level may use (FP64 values of per-cell shared memory):
// a longer chunk length is taken when the level's splits would need more.
static const long long kLevelPartials = 2048;

static void build_factor_jobs(HostMech &h) {
    const int NL = h.lanes;
    h.ljob_ptr.assign(1, 0);
    h.ljob.clear();
    h.lops.clear();
    h.lred_ptr.assign(1, 0);
    h.lred.clear();
    h.lred_off.clear();
    h.ltail.clear();
    h.n_lpart = 0;
    auto tgt = [](uint32_t op) { return (int)(op & 0xFFFFu); };
    auto row_ops = [&](int i) {
        return std::vector<uint32_t>(h.fops.begin() + h.fops_ptr[i], h.fops.begin() + h.fops_ptr[i + 1]);
    };
    for (size_t l = 0; l + 1 < h.flev_ptr.size(); l++) {
        const int rb = h.flev_ptr[l], re = h.flev_ptr[l + 1];
        long long total = 0, longest = 0;
        for (int r = rb; r < re; r++) {
            const int i = h.frow[r];
            total += h.fops_ptr[i + 1] - h.fops_ptr[i] + 2;
            longest = std::max<long long>(longest, h.fops_ptr[i + 1] - h.fops_ptr[i]);
        }
        // chunk length: the level's mean load per lane, at least 16 ops, and
        // long enough that the level's partial slots stay within budget
        int CH = std::max(16, (int)((total + NL - 1) / NL));
        if (NL > 32) {
            for (;;) {
                long long need = 0;
                for (int r = rb; r < re; r++) {
                    const std::vector<uint32_t> ops = row_ops(h.frow[r]);
                    if ((int)ops.size() <= 2 * CH) continue;
                    const RowSplit rs = split_row(ops, CH);
                    if (rs.chunks.size() >= 2) need += (long long)rs.chunks.size() * (long long)rs.shared.size();
                }
                if (need <= kLevelPartials || CH >= longest) break;
                CH *= 2;
            }
        }
        struct Job { std::vector<uint32_t> ops; int row, recip, ns, pbase; };
        std::vector<Job> jobs;
        int lpart = 0;
        for (int r = rb; r < re; r++) {
            const int i = h.frow[r];
            const int recip = i < h.d ? 1 : 0;
            std::vector<uint32_t> ops = row_ops(i);
            if (NL <= 32 || (int)ops.size() <= 2 * CH) { jobs.push_back({ops, i, recip, 0, 0}); continue; }
            const RowSplit rs = split_row(ops, CH);
            if (rs.chunks.size() < 2) { jobs.push_back({ops, i, recip, 0, 0}); continue; }
            const int ns = (int)rs.shared.size(), nch = (int)rs.chunks.size();
            if (ns > 0x7fff || nch > 0xffff) throw std::runtime_error("factor chunks do not fit their fields");
            for (int c = 0; c < nch; c++) {
                Job jb{{}, i, 0, ns, lpart + c * ns};
                for (int q : rs.chunks[c]) {
                    uint32_t op = ops[q];
                    auto it = rs.slot.find(tgt(op));
                    if (!(op & CAMP_OP_DIV) && it != rs.slot.end())
                        op = (op & 0xFFFF0000u) | 0x8000u | (uint32_t)it->second;
                    jb.ops.push_back(op);
                }
                jobs.push_back(jb);
            }
            int4 rd;
            rd.x = i | (recip << 16);
            rd.y = (int)h.lred_off.size();
            rd.z = ns | (nch << 16);
            rd.w = lpart;
            for (int t : rs.shared) h.lred_off.push_back(t);
            h.lred.push_back(rd.x); h.lred.push_back(rd.y); h.lred.push_back(rd.z); h.lred.push_back(rd.w);
            // the tail's ops go after the level's jobs; until then x holds
            // -1 - (the tail's first op within the row)
            h.ltail.push_back(-1 - rs.tail_from);
            h.ltail.push_back((int)ops.size() - rs.tail_from);
            h.ltail_rows.push_back(i);
            lpart += nch * ns;
        }
        h.n_lpart = std::max(h.n_lpart, lpart);
        std::vector<int> idx(jobs.size());
        for (size_t j = 0; j < jobs.size(); j++) idx[j] = (int)j;
        balance_level(idx, 0, (int)idx.size(), NL, [&](int j) { return (int)jobs[j].ops.size() + 2; });
        for (int j : idx) {
            const Job &jb = jobs[j];
            if (jb.ops.size() > 0xffff) throw std::runtime_error("factor job too long");
            h.ljob.push_back((int)h.lops.size());
            h.ljob.push_back((int)jb.ops.size() | (jb.ns << 16));
            h.ljob.push_back(jb.row | (jb.recip << 16));
            h.ljob.push_back(jb.pbase);
            h.lops.insert(h.lops.end(), jb.ops.begin(), jb.ops.end());
        }
        h.ljob_ptr.push_back((int)h.ljob.size() / 4);
        // the level's tails, stored after its jobs
        for (size_t k = h.lred_ptr.back(); k < h.lred.size() / 4; k++) {
            const int i = h.ltail_rows[k];
            const int from = -1 - h.ltail[2 * k];
            h.ltail[2 * k] = (int)h.lops.size();
            h.lops.insert(h.lops.end(), h.fops.begin() + h.fops_ptr[i] + from, h.fops.begin() + h.fops_ptr[i + 1]);
        }
        h.lred_ptr.push_back((int)h.lred.size() / 4);
    }
}

// ---- device tables -----------------------------------------------------------
static void build_tables(HostMech &h) {
    const int n = h.n, R = (int)h.procs.size();
    const auto &ip = h.iperm;

    // rate constants and rate terms
    h.rtype.resize(R); h.rslot.resize(R); h.rnr.resize(R); h.rnp.resize(R);
    h.rpar.assign((size_t)R * CAMP_NPAR, 0.0);
    h.rfac.assign((size_t)R * 6, -1);
    h.rrev.assign(R, -1);
    h.n_rev = 0;
    for (int k = 0; k < R; k++)
        if (h.procs[k].reversible()) h.rrev[k] = h.n_rev++;
    for (int k = 0; k < R; k++) {
        const Process &p = h.procs[k];
        h.rtype[k] = p.type;
        h.rslot[k] = p.slot;
        for (int i = 0; i < CAMP_NPAR; i++) h.rpar[(size_t)k * CAMP_NPAR + i] = p.par[i];
        int c = 0, nr = 0, np = 0;
        for (auto &e : p.react)
            for (int m = 0; m < e.second; m++) { h.rfac[(size_t)k * 6 + c++] = ip[e.first]; nr++; }
        if (p.reversible()) {
            c = 3;
            for (auto &e : p.prod)
                for (int m = 0; m < (int)e.second; m++) { h.rfac[(size_t)k * 6 + c++] = ip[e.first]; np++; }
        }
        h.rnr[k] = nr;
        h.rnp[k] = np;
    }

    // forcing gather by position
    std::vector<std::vector<std::pair<int, double>>> fl(n);
    for (int k = 0; k < R; k++)
        for (int s : touched(h.procs[k])) {
            double nu = net_coef(h.procs[k], s);
            if (nu != 0.0) fl[ip[s]].emplace_back(k, nu);
        }
    h.fptr.assign(1, 0);
    h.fk.clear(); h.fc.clear();
    for (int p = 0; p < n; p++) {
        for (auto &e : fl[p]) { h.fk.push_back(e.first); h.fc.push_back(e.second); }
        h.fptr.push_back((int)h.fk.size());
    }
    // the per-position sums over the lanes of one cell, longest processing
    // time first; a sum longer than the lanes' mean load is cut into chunks
    // whose partial sums a second pass adds in a fixed order
    {
        const int NL = h.lanes;
        long long total = 0;
        for (int p = 0; p < n; p++) total += h.fptr[p + 1] - h.fptr[p] + 2;
        // only block cells split (one-warp cells take no second pass)
        const int CH = NL > 32 ? std::max(8, (int)((total + NL - 1) / NL)) : 1 << 30;
        struct Job { int first, count, dst; };
        std::vector<Job> jobs;
        h.fsplit.clear();
        h.n_fpart = 0;
        for (int p = 0; p < n; p++) {
            const int b = h.fptr[p], e = h.fptr[p + 1];
            if (e - b <= CH) { jobs.push_back({b, e - b, p}); continue; }
            const int nch = (e - b + CH - 1) / CH;
            h.fsplit.push_back(p);
            h.fsplit.push_back(h.n_fpart | (nch << 16));
            for (int c = 0; c < nch; c++) {
                const int cb = b + (int)((long long)c * (e - b) / nch), ce = b + (int)((long long)(c + 1) * (e - b) / nch);
                jobs.push_back({cb, ce - cb, n + h.n_fpart + c});
            }
            h.n_fpart += nch;
        }
        std::vector<int> order(jobs.size());
        for (size_t j = 0; j < jobs.size(); j++) order[j] = (int)j;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a].count > jobs[b].count; });
        std::vector<std::vector<int>> lanes(NL);
        std::vector<long long> load(NL, 0);
        for (int j : order) {
            int best = 0;
            for (int l = 1; l < NL; l++)
                if (load[l] < load[best]) best = l;
            lanes[best].push_back(j);
            load[best] += jobs[j].count + 2;  // entries plus the per-sum cost
        }
        h.flane_ptr.assign(1, 0);
        h.flane_pos.clear();
        h.fjob.clear();
        for (auto &v : lanes) {
            for (int j : v) {
                const Job &jb = jobs[j];
                if (jb.dst > 0xffff || jb.count > 0xffff) throw std::runtime_error("forcing jobs do not fit 16-bit fields");
                h.flane_pos.push_back(jb.dst);
                h.fjob.push_back(jb.first);
                h.fjob.push_back(jb.dst | (jb.count << 16));
            }
            h.flane_ptr.push_back((int)h.flane_pos.size());
        }
    }

    // dense trailing block: smallest d with D = n - d >= 8 and fill density >= 0.75
    h.d = n;
    for (int d = 0; d + 8 <= n; d++) {
        long long cnt = 0;
        for (int i = d; i < n; i++)
            for (int q = h.lu_rowptr[i]; q < h.lu_rowptr[i + 1]; q++) cnt += (h.lu_colidx[q] >= d);
        if ((double)cnt >= 0.75 * (double)(n - d) * (double)(n - d)) { h.d = d; break; }
    }
    if (n - h.d > 128) h.d = n - 128;  // the substitution keeps at most 4 block rows per lane
    h.D = n - h.d;
    h.LD = h.D % 2 ? h.D : h.D + 1;

    // storage offsets: sparse rows < d, the L21 part of rows >= d, then the block
    std::vector<int> lu_off(h.lu_colidx.size(), -1);
    int nsp = 0;
    for (int i = 0; i < n; i++)
        for (int q = h.lu_rowptr[i]; q < h.lu_rowptr[i + 1]; q++)
            if (i < h.d || h.lu_colidx[q] < h.d) lu_off[q] = nsp++;
    h.dbase = (nsp + 3) & ~3;
    for (int i = h.d; i < n; i++)
        for (int q = h.lu_rowptr[i]; q < h.lu_rowptr[i + 1]; q++)
            if (h.lu_colidx[q] >= h.d) lu_off[q] = h.dbase + (i - h.d) * h.LD + (h.lu_colidx[q] - h.d);
    h.nlu = h.dbase + h.D * h.LD;
    if (h.nlu > 32767) throw std::runtime_error("LU storage too large for the packed tables (32767 values)");
    auto off = [&](int i, int j) {
        auto b = h.lu_colidx.begin() + h.lu_rowptr[i], e = h.lu_colidx.begin() + h.lu_rowptr[i + 1];
        auto it = std::lower_bound(b, e, j);
        if (it == e || *it != j) throw std::logic_error("entry outside the LU pattern");
        return lu_off[it - h.lu_colidx.begin()];
    };

    // Jacobian gather by species-CSR non-zero
    const int nnzJ = (int)h.colidx.size();
    std::vector<std::vector<int>> jent(nnzJ);  // indices into entry arrays
    std::vector<int> ek, eo;
    std::vector<double> ec;
    auto csr_pos = [&](int i, int j) {
        auto b = h.colidx.begin() + h.rowptr[i], e = h.colidx.begin() + h.rowptr[i + 1];
        return (int)(std::lower_bound(b, e, j) - h.colidx.begin());
    };
    for (int k = 0; k < R; k++) {
        const Process &p = h.procs[k];
        for (int j : dependence(p)) {
            for (int i : touched(p)) {
                double nu = net_coef(p, i);
                if (nu == 0.0) continue;
                int t = csr_pos(i, j);
                // forward term: kf * prod(reactant factors)
                for (int side = 0; side < 2; side++) {
                    if (side == 1 && !p.reversible()) break;
                    const int *fac = &h.rfac[(size_t)k * 6 + 3 * side];
                    int mult = 0;
                    for (int m = 0; m < 3; m++) mult += (fac[m] == ip[j]);
                    if (!mult) continue;
                    int others[2] = {-1, -1}, no = 0;
                    bool skipped = false;
                    for (int m = 0; m < 3; m++) {
                        if (fac[m] < 0) continue;
                        if (fac[m] == ip[j] && !skipped) { skipped = true; continue; }
                        others[no++] = fac[m];
                    }
                    jent[t].push_back((int)ek.size());
                    ek.push_back(side == 0 ? k : -(h.rrev[k] + 1));
                    eo.push_back(others[0]);
                    eo.push_back(others[1]);
                    ec.push_back(side == 0 ? nu * mult : -nu * mult);
                }
            }
        }
    }
    h.jptr.assign(1, 0);
    h.jdst.resize(nnzJ); h.jdiag.resize(nnzJ);
    h.jk.clear(); h.jo.clear(); h.jc.clear();
    for (int i = 0; i < n; i++)
        for (int q = h.rowptr[i]; q < h.rowptr[i + 1]; q++) {
            int j = h.colidx[q];
            h.jdst[q] = off(ip[i], ip[j]);
            h.jdiag[q] = (i == j);
            for (int e : jent[q]) {
                h.jk.push_back(ek[e]);
                h.jo.push_back(eo[2 * e]);
                h.jo.push_back(eo[2 * e + 1]);
                h.jc.push_back(ec[e]);
            }
            h.jptr.push_back((int)h.jk.size());
        }

    // the water parameter: electrolyte lists per section, the processes that
    // carry powers of 1/L, d f_i / d L_b sums and the chain-rule entries
    h.pw_ptr.clear(); h.pw.clear(); h.pp.clear(); h.g_ptr.clear(); h.g_ent.clear();
    h.g_coef.clear(); h.ch.clear();
    h.n_pw = h.n_pw64 = 0;
    if (!h.el_phase.empty()) {
        const int S = h.n_sections, n_el = (int)h.el_phase.size();
        h.pw_ptr.assign(1, 0);
        for (int b = 0; b < S; b++) {
            for (int e = 0; e < n_el; e++) h.pw.push_back(ip[electrolyte_species(h, b, e)] | (e << 16));
            h.pw_ptr.push_back((int)h.pw.size());
        }
        std::map<std::pair<int, int>, int> gidx;  // (species, section) -> g
        std::vector<std::pair<int, int>> grow;    // g -> (species, section)
        std::vector<std::vector<std::pair<int, double>>> gl;
        // the processes with powers of 1/L enter the chain rule
        for (int k = 0; k < R; k++) {
            const Process &p = h.procs[k];
            if (!p.la && !p.lb) continue;
            const int j = (int)h.pp.size() / 4;
            h.pp.push_back(k);
            h.pp.push_back(p.slot);
            h.pp.push_back(p.la | (p.lb << 8));
            h.pp.push_back(h.rrev[k]);
            for (int i : touched(p)) {
                const double nu = net_coef(p, i);
                if (nu == 0.0) continue;
                auto key = std::make_pair(i, p.slot);
                auto it = gidx.find(key);
                int g;
                if (it == gidx.end()) {
                    g = (int)grow.size();
                    gidx.emplace(key, g);
                    grow.push_back(key);
                    gl.emplace_back();
                } else {
                    g = it->second;
                }
                gl[g].emplace_back(j, nu);
            }
        }
        h.g_ptr.assign(1, 0);
        for (auto &v : gl) {
            for (auto &e : v) { h.g_ent.push_back(e.first); h.g_coef.push_back(e.second); }
            h.g_ptr.push_back((int)h.g_ent.size());
        }
        for (int g = 0; g < (int)grow.size(); g++) {
            const int i = grow[g].first, b = grow[g].second;
            for (int e = 0; e < n_el; e++) {
                const int col = electrolyte_species(h, b, e);
                h.ch.push_back(off(ip[i], ip[col]));
                h.ch.push_back(g);
                h.ch.push_back(e);
                h.ch.push_back(csr_pos(i, col));
            }
        }
        // per cell: the weights, L_env and 1 / L per section; the FP64 form
        // also keeps the Jacobian's reverse constants there
        h.n_pw = n_el + 2 * S;
        h.n_pw64 = h.n_rev;
    }

    // sparse factorisation ops, row by row; levels: sparse rows by level, then
    // every block row in one final level (they only need sparse pivots)
    h.fops_ptr.assign(1, 0);
    h.fops.clear();
    h.factor_updates = 0;
    for (int i = 0; i < n; i++) {
        for (int q = h.lu_rowptr[i]; q < h.lu_rowptr[i + 1]; q++) {
            int k = h.lu_colidx[q];
            if (k >= i || k >= h.d) continue;
            h.fops.push_back(CAMP_OP_DIV | ((uint32_t)off(k, k) << 16) | (uint32_t)off(i, k));
            for (int r = h.lu_rowptr[k]; r < h.lu_rowptr[k + 1]; r++) {
                int j = h.lu_colidx[r];
                if (j <= k) continue;
                h.fops.push_back(((uint32_t)off(k, j) << 16) | (uint32_t)off(i, j));
                h.factor_updates++;
            }
        }
        h.fops_ptr.push_back((int)h.fops.size());
    }
    for (long long k = 0; k < h.D; k++) h.factor_updates += (h.D - 1 - k) * (h.D - 1 - k);
    // algorithmic flop counts (structure only, independent of the storage)
    h.flops_forcing = 2LL * (long long)h.fk.size();
    for (int k = 0; k < R; k++) {
        int nf = 0, nb = 0;
        for (int m2 = 0; m2 < 3; m2++) nf += h.rfac[(size_t)k * 6 + m2] >= 0;
        for (int m2 = 3; m2 < 6; m2++) nb += h.rfac[(size_t)k * 6 + m2] >= 0;
        h.flops_forcing += nf + (h.procs[k].reversible() ? nb + 1 : 0);
    }
    h.model_forcing = 0;
    for (const auto &p : h.procs) h.model_forcing += 2LL * (long long)p.react.size() + (long long)p.prod.size();
    h.flops_jacobian = 2LL * (long long)h.colidx.size();
    for (size_t e = 0; e < h.jk.size(); e++)
        h.flops_jacobian += 2 + (h.jo[2 * e] >= 0) + (h.jo[2 * e + 1] >= 0);
    if (!h.el_phase.empty()) {
        // the water parameter per state: a multiply-add per electrolyte and a
        // reciprocal per section, then the powers of 1/L of each process;
        // per assembly also d r / d L, the g sums and the chain-rule entries
        long long upd = 2LL * (long long)h.pw.size() + h.n_sections;
        for (auto &p : h.procs) upd += p.la + p.lb + ((p.la || p.lb) && p.lb ? 1 : 0);
        h.flops_forcing += upd;
        h.flops_jacobian += upd + 10LL * (long long)(h.pp.size() / 4) + 2LL * (long long)h.g_ent.size() +
                            3LL * (long long)(h.ch.size() / 4);
    }
    h.flops_factor = 0;
    {
        std::vector<int> lower(n, 0), upper(n, 0);
        for (int i = 0; i < n; i++)
            for (int q = h.lu_rowptr[i]; q < h.lu_rowptr[i + 1]; q++) {
                int j = h.lu_colidx[q];
                if (j < i) lower[j]++;   // column j of L
                if (j > i) upper[i]++;   // row i of U
            }
        for (int k = 0; k < n; k++) h.flops_factor += 2LL * lower[k] * upper[k] + lower[k];
    }
    h.flops_solve = 2LL * ((long long)h.lu_colidx.size() - n) + n;
    int maxl = -1;
    for (int i = 0; i < h.d; i++) maxl = std::max(maxl, h.level_fwd[i]);
    h.flev_ptr.assign(1, 0);
    h.frow.clear();
    for (int l = 0; l <= maxl; l++) {
        for (int i = 0; i < h.d; i++) if (h.level_fwd[i] == l) h.frow.push_back(i);
        h.flev_ptr.push_back((int)h.frow.size());
    }
    if (h.D > 0) {
        for (int i = h.d; i < n; i++) h.frow.push_back(i);
        h.flev_ptr.push_back((int)h.frow.size());
    }

    // substitution lists
    h.sl_ptr.assign(1, 0);
    h.sl_off.clear(); h.sl_col.clear();
    h.su_ptr.assign(1, 0);
    h.su_off.clear(); h.su_col.clear();
    h.udiag.assign(n, -1);
    for (int i = 0; i < n; i++) {
        for (int q = h.lu_rowptr[i]; q < h.lu_rowptr[i + 1]; q++) {
            int j = h.lu_colidx[q];
            if (j < i && j < h.d) { h.sl_off.push_back(off(i, j)); h.sl_col.push_back(j); }
            if (i < h.d && j > i) { h.su_off.push_back(off(i, j)); h.su_col.push_back(j); }
            if (i < h.d && j == i) h.udiag[i] = off(i, i);
        }
        h.sl_ptr.push_back((int)h.sl_off.size());
        h.su_ptr.push_back((int)h.su_off.size());
    }
    // the factorisation's levels balanced by update count; the forward
    // substitution skips rows without L entries and balances by entry count
    for (size_t l = 0; l + 1 < h.flev_ptr.size(); l++)
        balance_level(h.frow, h.flev_ptr[l], h.flev_ptr[l + 1], h.lanes,
                      [&](int i) { return h.fops_ptr[i + 1] - h.fops_ptr[i] + 1; });
    build_factor_jobs(h);
    // Forward substitution as lane jobs, level by level: a row longer than
    // its level's mean load per lane is cut into chunks whose partial dot
    // products a second pass subtracts in a fixed order.
    {
        const int NL = h.lanes;
        h.slev_ptr.assign(1, 0);
        h.sjob.clear();
        h.ssplit_ptr.assign(1, 0);
        h.ssplit.clear();
        h.n_spart = 0;
        struct Job { int first, count, dst; };
        for (size_t l = 0; l + 1 < h.flev_ptr.size(); l++) {
            std::vector<int> rows;
            long long total = 0;
            for (int r = h.flev_ptr[l]; r < h.flev_ptr[l + 1]; r++) {
                const int i = h.frow[r];
                if (h.sl_ptr[i + 1] > h.sl_ptr[i]) {
                    rows.push_back(i);
                    total += h.sl_ptr[i + 1] - h.sl_ptr[i] + 1;
                }
            }
            if (rows.empty()) continue;
            const int CH = NL > 32 ? std::max(16, (int)((total + NL - 1) / NL)) : 1 << 30;
            std::vector<Job> jobs;
            int np = 0;
            for (int i : rows) {
                const int b = h.sl_ptr[i], e = h.sl_ptr[i + 1];
                if (e - b <= CH) { jobs.push_back({b, e - b, i}); continue; }
                const int nch = (e - b + CH - 1) / CH;
                h.ssplit.push_back(i);
                h.ssplit.push_back(np | (nch << 16));
                for (int c = 0; c < nch; c++) {
                    const int cb = b + (int)((long long)c * (e - b) / nch), ce = b + (int)((long long)(c + 1) * (e - b) / nch);
                    jobs.push_back({cb, ce - cb, n + np + c});
                }
                np += nch;
            }
            h.n_spart = std::max(h.n_spart, np);
            std::vector<int> idx(jobs.size());
            for (size_t j = 0; j < jobs.size(); j++) idx[j] = (int)j;
            balance_level(idx, 0, (int)idx.size(), NL, [&](int j) { return jobs[j].count + 1; });
            for (int j : idx) {
                if (jobs[j].dst > 0xffff || jobs[j].count > 0xffff) throw std::runtime_error("substitution jobs do not fit 16-bit fields");
                h.sjob.push_back(jobs[j].first);
                h.sjob.push_back(jobs[j].dst | (jobs[j].count << 16));
            }
            h.slev_ptr.push_back((int)h.sjob.size() / 2);
            h.ssplit_ptr.push_back((int)h.ssplit.size() / 2);
        }
    }
    std::vector<int> bl(n, 0);
    int maxb = -1;
    for (int i = h.d - 1; i >= 0; i--) {
        int lv = -1;
        for (int q = h.lu_rowptr[i]; q < h.lu_rowptr[i + 1]; q++) {
            int j = h.lu_colidx[q];
            if (j > i && j < h.d) lv = std::max(lv, bl[j]);
        }
        bl[i] = lv + 1;
        maxb = std::max(maxb, bl[i]);
    }
    h.blev_ptr.assign(1, 0);
    h.brow.clear();
    for (int l = 0; l <= maxb; l++) {
        for (int i = 0; i < h.d; i++) if (bl[i] == l) h.brow.push_back(i);
        h.blev_ptr.push_back((int)h.brow.size());
        const int b = h.blev_ptr[h.blev_ptr.size() - 2], e = h.blev_ptr.back();
        balance_level(h.brow, b, e, h.lanes, [&](int i) { return h.su_ptr[i + 1] - h.su_ptr[i] + 1; });
    }
}

// Bounds of every index the device tables hold, checked once per mechanism
// on the host: the kernels index shared memory and the tables with these
// values unchecked, so an out-of-range entry is a compiler bug caught here
// (an exception naming the table) instead of a wrong access on the GPU.
static void validate_tables(const HostMech &h) {
    const int n = h.n, R = (int)h.procs.size(), nlu = h.nlu;
    auto fail = [](const char *what) { throw std::runtime_error(std::string("internal table check failed: ") + what); };
    auto in = [](long long v, long long lo, long long hi) { return v >= lo && v < hi; };
    auto f16 = [](int v) { return v & 0xffff; };
    auto h16 = [](int v) { return (int)((unsigned)v >> 16); };
    const int NONE = 0xffff;
    // permutation and rates
    {
        std::vector<int> seen(n, 0);
        for (int p : h.perm) { if (!in(p, 0, n) || seen[p]++) fail("perm"); }
        if ((int)h.perm.size() != n) fail("perm size");
    }
    for (int k = 0; k < R; k++) {
        for (int c = 0; c < 6; c++) if (!in(h.rfac[6 * k + c], -1, n)) fail("rfac");
        if (!in(h.rrev[k], -1, h.n_rev)) fail("rrev");
        // fwd0 | fwd1, fwd2 | reverse-constant index, rev0 | rev1, rev2
        for (int c = 0; c < 4; c++) {
            const int w = h.rpack[4 * k + c];
            const int lo = f16(w), hi = h16(w);
            if (lo != NONE && !in(lo, 0, n)) fail("rpack");
            if (c == 1 && hi != NONE && !in(hi, 0, h.n_rev)) fail("rpack");
            if ((c == 0 || c == 2) && hi != NONE && !in(hi, 0, n)) fail("rpack");
            if (c == 3) {  // water tag: section + 1, la, lb (0 without the parameter)
                const int sec = (hi & 0x7ff) - 1;
                if (h.el_phase.empty() ? hi != 0 : !in(sec, -1, h.n_sections)) fail("rpack water tag");
                if (sec < 0 && hi != 0) fail("rpack water tag");
            }
        }
    }
    // forcing gather
    const int nf = (int)h.fk.size();
    for (int q = 0; q < nf; q++)
        if (!in(f16(h.fpk[q]), 0, R) || !in(h16(h.fpk[q]), 0, (int)h.fcoef.size())) fail("fpk");
    const int nj = (int)h.fjob.size() / 2;
    if (h.flane_ptr.front() != 0 || h.flane_ptr.back() != nj) fail("flane_ptr");
    for (size_t l = 0; l + 1 < h.flane_ptr.size(); l++) if (h.flane_ptr[l] > h.flane_ptr[l + 1]) fail("flane_ptr order");
    for (int i = 0; i < nj; i++) {
        const int first = h.fjob[2 * i], dst = f16(h.fjob[2 * i + 1]), cnt = h16(h.fjob[2 * i + 1]);
        if (!in(first, 0, nf + 1) || first + cnt > nf || !in(dst, 0, n + h.n_fpart)) fail("fjob");
    }
    for (size_t i = 0; i < h.fsplit.size() / 2; i++) {
        const int pos = h.fsplit[2 * i], first = f16(h.fsplit[2 * i + 1]), cnt = h16(h.fsplit[2 * i + 1]);
        if (!in(pos, 0, n) || first + cnt > h.n_fpart) fail("fsplit");
    }
    // Jacobian lists
    const int nnzJ = (int)h.colidx.size();
    for (size_t i = 0; i < h.jl_rec.size() / 4; i++) {
        const int *r = &h.jl_rec[4 * i];
        const int k = (int)(short)(r[1] & 0xffff), o1 = h16(r[1]), o2 = f16(r[3]), t = h16(r[3]);
        if (!in(k, -h.n_rev, R) || (o1 != NONE && !in(o1, 0, n)) || (o2 != NONE && !in(o2, 0, n))) fail("jl_rec");
        if (!in(r[2] & 0xffff, 0, nlu) || !in(t, 0, nnzJ)) fail("jl_rec target");
    }
    // LU: storage layout, factorisation jobs, substitution lists
    if (h.dbase + h.D * h.LD > nlu || h.d + h.D != n) fail("dense block");
    for (int i = 0; i < h.d; i++) if (!in(h.udiag[i], 0, nlu)) fail("udiag");
    const int nops = (int)h.lops.size();
    for (size_t j = 0; j < h.ljob.size() / 4; j++) {
        const int *jb = &h.ljob[4 * j];
        const int cnt = f16(jb[1]), ns = h16(jb[1]), row = f16(jb[2]);
        if (jb[0] < 0 || jb[0] + cnt > nops || !in(row, 0, n) || (ns > 0 && jb[3] + ns > h.n_lpart))
            fail("ljob");
        for (int q = jb[0]; q < jb[0] + cnt; q++) {
            const uint32_t op = h.lops[q];
            const int t = (int)(op & 0xffffu), src = (int)((op >> 16) & 0x7fffu);
            if (!in(src, 0, nlu)) fail("lops source");
            if ((t & 0x8000) && !(op & CAMP_OP_DIV)) {
                if (!in(jb[3] + (t & 0x7fff), 0, h.n_lpart) || (t & 0x7fff) >= ns) fail("lops partial");
            } else if (!in(t, 0, nlu)) fail("lops target");
        }
    }
    for (size_t k = 0; k < h.lred.size() / 4; k++) {
        const int *rd = &h.lred[4 * k];
        const int ns = f16(rd[2]), nch = h16(rd[2]);
        if (!in(f16(rd[0]), 0, n) || rd[1] + ns > (int)h.lred_off.size() || rd[3] + ns * nch > h.n_lpart) fail("lred");
        for (int s2 = 0; s2 < ns; s2++) if (!in(h.lred_off[rd[1] + s2], 0, nlu)) fail("lred_off");
        if (h.ltail[2 * k] < 0 || h.ltail[2 * k] + h.ltail[2 * k + 1] > nops) fail("ltail");
        for (int q = h.ltail[2 * k]; q < h.ltail[2 * k] + h.ltail[2 * k + 1]; q++)
            if ((h.lops[q] & 0x8000u) && !(h.lops[q] & CAMP_OP_DIV)) fail("tail op with a partial target");
    }
    auto check_pack = [&](const std::vector<int> &pk, const char *what) {
        for (int w : pk) if (!in(f16(w), 0, nlu) || !in(h16(w), 0, n)) fail(what);
    };
    check_pack(h.sl_pack, "sl_pack");
    check_pack(h.su_pack, "su_pack");
    const int nsl = (int)h.sl_pack.size();
    for (size_t r = 0; r < h.sjob.size() / 2; r++) {
        const int first = h.sjob[2 * r], dst = f16(h.sjob[2 * r + 1]), cnt = h16(h.sjob[2 * r + 1]);
        if (first < 0 || first + cnt > nsl || !in(dst, 0, n + h.n_spart)) fail("sjob");
    }
    for (size_t k = 0; k < h.ssplit.size() / 2; k++)
        if (!in(h.ssplit[2 * k], 0, n) || f16(h.ssplit[2 * k + 1]) + h16(h.ssplit[2 * k + 1]) > h.n_spart) fail("ssplit");
    for (int i : h.brow) if (!in(i, 0, h.d)) fail("brow");
    // water parameter
    if (!h.el_phase.empty()) {
        const int S = h.n_sections, n_el = (int)h.el_phase.size(), n_pp = (int)h.pp.size() / 4;
        const int n_g = (int)h.g_ptr.size() - 1;
        if ((int)h.pw_ptr.size() != S + 1 || h.pw_ptr.back() != (int)h.pw.size()) fail("pw_ptr");
        for (int w : h.pw) if (!in(f16(w), 0, n) || !in(h16(w), 0, n_el)) fail("pw");
        for (int j = 0; j < n_pp; j++) {
            const int *r = &h.pp[4 * j];
            if (!in(r[0], 0, R) || !in(r[1], 0, S) || !in(r[3], -1, h.n_rev)) fail("pp");
            if ((r[2] & 0xff) > CAMP_MAXFAC || (r[2] >> 8) > CAMP_MAXFAC) fail("pp powers");
        }
        if (h.g_ptr.front() != 0 || h.g_ptr.back() != (int)h.g_ent.size()) fail("g_ptr");
        for (int j : h.g_ent) if (!in(j, 0, n_pp)) fail("g_ent");
        if ((int)h.ch.size() != 4 * n_g * n_el) fail("ch size");
        for (size_t c = 0; c < h.ch.size() / 4; c++) {
            const int *r = &h.ch[4 * c];
            if (!in(r[0], 0, nlu) || !in(r[1], 0, n_g) || !in(r[2], 0, n_el) || !in(r[3], 0, nnzJ)) fail("ch");
            if (r[1] != (int)c / n_el || r[2] != (int)c % n_el) fail("ch order");
        }
        if (!in(h.rh_slot, 2, h.env_sec_base)) fail("rh_slot");
    }
    for (int i = 0; i < n; i++)
        if (h.su_ptr[i] > h.su_ptr[i + 1] || h.sl_ptr[i] > h.sl_ptr[i + 1]) fail("substitution pointers");
}

HostMech compile_mechanism(const char *json, size_t len, int instances, int lanes) {
    Value root = campjson::parse(json, len);
    HostMech h;
    read_processes(root, h, instances);
    if (h.n < 1) throw std::runtime_error("mechanism has no species");
    h.lanes = lanes > 0 ? lanes : camp_cell_lanes(h.n);
    if ((h.lanes != 32 && h.lanes != 64 && h.lanes != 128 && h.lanes != 256) || h.n > 8 * h.lanes)
        throw std::runtime_error("lanes per cell must be 32, 64, 128 or 256, with at most 8 species a lane");
    build_structure(h);
    build_tables(h);
    pack_records(h);
    validate_tables(h);
    return h;
}

AerosolShape aerosol_shape(const char *json, size_t len) {
    Value root = campjson::parse(json, len);
    AerosolShape s;
    if (const Value *a = root.find("aerosol")) {
        const double k = a->number("sections");
        if (!(k >= 0.0 && k <= 1e6)) throw std::runtime_error("bad section count");
        s.instances = (int)k;
        if (const Value *r = a->find("representation")) s.particles = r->kind == Value::String && r->str == "particles";
        if (const Value *v = a->find("solver")) s.block_arrow = v->kind == Value::String && v->str == "block_arrow";
    }
    if (const Value *p = root.find("parameters")) s.water = p->kind == Value::Array && !p->arr.empty();
    return s;
}

// ---- the block-arrow form ----------------------------------------------------
ArrowHost build_arrow(const HostMech &t, int P) {
    if (t.n_sections != 1) throw std::runtime_error("the block-arrow template holds one instance");
    if (!t.el_phase.empty()) throw std::runtime_error("the block-arrow form has no water parameter");
    ArrowHost a;
    a.P = P;
    a.n_g = t.n_gas;
    a.n_phi = t.n - t.n_gas;
    a.E0 = t.env_sec_base;
    a.n_env = t.env_sec_base + 3 * P;
    if (a.n_g > CAMP_ARROW_MAX_GAS) throw std::runtime_error("block-arrow form: more than 32 gas species");
    if (a.n_phi < 1 || a.n_phi > CAMP_ARROW_MAX_PHI)
        throw std::runtime_error("block-arrow form: 1 to 16 phase species per particle");
    auto local = [&](int s) {  // template species -> particle-local index
        if (s >= a.n_g) return s - a.n_g;
        auto it = std::find(a.coupled.begin(), a.coupled.end(), s);
        if (it != a.coupled.end()) return a.n_phi + (int)(it - a.coupled.begin());
        a.coupled.push_back(s);
        return a.n_phi + (int)a.coupled.size() - 1;
    };
    std::vector<int> gas_index;  // template process -> gas process number
    for (int k = 0; k < (int)t.procs.size(); k++) {
        const Process &p = t.procs[k];
        const bool sec = is_sectioned(p.type);
        for (auto &e : p.react)
            if (!sec && e.first >= a.n_g) throw std::runtime_error("a gas process touches a phase species");
        for (auto &e : p.prod)
            if (!sec && e.first >= a.n_g) throw std::runtime_error("a gas process touches a phase species");
        auto map = [&](int s) { return sec ? local(s) : s; };
        int rec[12];
        std::fill(rec, rec + 12, -1);
        rec[0] = k;
        int nf = 0, nb = 0;
        for (auto &e : p.react)
            for (int m = 0; m < e.second; m++) rec[4 + nf++] = map(e.first);
        if (p.reversible())
            for (auto &e : p.prod)
                for (int m = 0; m < (int)e.second; m++) rec[8 + nb++] = map(e.first);
        rec[1] = nf;
        rec[2] = nb;
        rec[3] = (int)a.st_sp.size();
        for (int s : touched(p)) {
            const double nu = net_coef(p, s);
            if (nu == 0.0) continue;
            a.st_sp.push_back(map(s));
            a.st_nu.push_back(nu);
        }
        rec[7] = (int)a.st_sp.size();
        rec[11] = p.reversible() ? 1 : 0;
        std::vector<int> &dst = sec ? a.prec : a.grec;
        if (!sec) gas_index.push_back(k);
        dst.insert(dst.end(), rec, rec + 12);
        // algorithmic work, per instance for the particle processes
        const long long inst = sec ? P : 1;
        a.model_forcing += inst * (2LL * (long long)p.react.size() + (long long)p.prod.size());
        a.flops_forcing += inst * (nf + (p.reversible() ? nb + 1 : 0) + 2LL * (rec[7] - rec[3]));
        a.flops_jacobian += inst * (long long)(nf + nb) * (long long)(std::max(nf, nb) + 2 * (rec[7] - rec[3]));
    }
    a.Rg = (int)a.grec.size() / 12;
    a.Rp = (int)a.prec.size() / 12;
    if (a.Rg > 64) throw std::runtime_error("block-arrow form: more than 64 gas processes");
    a.n_c = (int)a.coupled.size();
    if (a.n_c > CAMP_ARROW_MAX_C) throw std::runtime_error("block-arrow form: a particle exchanges with more than 8 gas species");
    // gas rows: the gas processes that change each gas species
    a.gf_ptr.assign(a.n_g + 1, 0);
    for (int i = 0; i < a.n_g; i++) {
        for (int g = 0; g < a.Rg; g++) {
            const int *r = &a.grec[(size_t)g * 12];
            for (int q = r[3]; q < r[7]; q++)
                if (a.st_sp[q] == i) {
                    a.gf_k.push_back(g);
                    a.gf_nu.push_back(a.st_nu[q]);
                }
        }
        a.gf_ptr[i + 1] = (int)a.gf_k.size();
    }
    // dense per-particle LU (block, U_pG, L_Gp, Schur) and the gas block
    const long long np = a.n_phi, nc = a.n_c, ng = a.n_g;
    a.flops_factor = (long long)P * (2 * np * np * np / 3 + 2 * np * np * nc * 2 + 2 * nc * nc * np) + 2 * ng * ng * ng / 3;
    a.flops_solve = (long long)P * (2 * np * np + 4 * np * nc) + 2 * ng * ng;
    return a;
}

void bdf_coefficients(DevMech &dm) {
    for (int q = 0; q <= CAMP_QMAX + 1; q++) {
        double c[CAMP_QMAX + 2] = {1.0, 0, 0, 0, 0, 0, 0};
        for (int i = 1; i <= q; i++)  // c(x) *= (1 + x / i)
            for (int j = i; j >= 1; j--) c[j] += c[j - 1] / (double)i;
        for (int j = 0; j <= CAMP_QMAX + 1; j++) dm.lcoef[q][j] = c[j];
        dm.ecoef[q] = q > 0 ? 1.0 / ((double)(q + 1) * c[1]) : 0.0;
    }
    dm.fact[0] = 1.0;
    for (int i = 1; i <= CAMP_QMAX + 1; i++) dm.fact[i] = dm.fact[i - 1] * i;
    for (int q = 0; q <= CAMP_QMAX + 1; q++) {
        dm.inv_l1[q] = q > 0 ? 1.0 / dm.lcoef[q][1] : 0.0;
        dm.ecoef2[q] = dm.ecoef[q] * dm.ecoef[q];
    }
    dm.rn = dm.n > 0 ? 1.0 / (double)dm.n : 0.0;
}

// ---- packing ---------------------------------------------------------------
namespace {
struct Packer {
    std::vector<unsigned char> img;
    const unsigned char *base;
    template <class T>
    const T *put(const std::vector<T> &v) {
        size_t off = (img.size() + 15) & ~(size_t)15;
        img.resize(off + std::max<size_t>(v.size() * sizeof(T), 16), 0);
        if (!v.empty()) std::copy((const unsigned char *)v.data(),
                                  (const unsigned char *)v.data() + v.size() * sizeof(T), img.data() + off);
        return reinterpret_cast<const T *>(reinterpret_cast<uintptr_t>(base) + off);
    }
};
}  // namespace

std::vector<unsigned char> pack_tables(const HostMech &h, DevMech &dm, const unsigned char *base) {
    Packer pk{{}, base};
    dm.n = h.n;
    dm.R = (int)h.procs.size();
    dm.n_env = h.n_env;
    dm.env_sec_base = h.env_sec_base;
    dm.lanes = h.lanes;
    dm.rtype = pk.put(h.rtype);
    dm.rpar = pk.put(h.rpar);
    dm.rslot = pk.put(h.rslot);
    dm.rnr = pk.put(h.rnr);
    dm.rnp = pk.put(h.rnp);
    dm.n_rev = h.n_rev;
    dm.rrev = pk.put(h.rrev);
    dm.flane_ptr = pk.put(h.flane_ptr);
    dm.nnzJ = (int)h.colidx.size();
    dm.jk = pk.put(h.jk);
    dm.jo = pk.put(h.jo);
    dm.jc = pk.put(h.jc);
    dm.nlu = h.nlu;
    dm.d = h.d;
    dm.D = h.D;
    dm.LD = h.LD;
    dm.dbase = h.dbase;
    dm.n_flev = (int)h.flev_ptr.size() - 1;
    dm.ljob_ptr = pk.put(h.ljob_ptr);
    dm.ljob = reinterpret_cast<const int4 *>(pk.put(h.ljob));
    dm.lops = pk.put(h.lops);
    dm.lred_ptr = pk.put(h.lred_ptr);
    dm.lred = reinterpret_cast<const int4 *>(pk.put(h.lred));
    dm.lred_off = pk.put(h.lred_off);
    dm.ltail = reinterpret_cast<const int2 *>(pk.put(h.ltail));
    dm.n_slev = (int)h.slev_ptr.size() - 1;
    dm.slev_ptr = pk.put(h.slev_ptr);
    dm.sjob = reinterpret_cast<const int2 *>(pk.put(h.sjob));
    dm.ssplit_ptr = pk.put(h.ssplit_ptr);
    dm.ssplit = reinterpret_cast<const int2 *>(pk.put(h.ssplit));
    // partials in doubles: the factor's are LU-precision values, at most 8 bytes
    dm.n_part = std::max(std::max(h.n_fpart, h.n_spart), h.n_lpart);
    dm.n_blev = (int)h.blev_ptr.size() - 1;
    dm.blev_ptr = pk.put(h.blev_ptr);
    dm.brow = pk.put(h.brow);
    dm.su_ptr = pk.put(h.su_ptr);
    dm.udiag = pk.put(h.udiag);
    dm.perm = pk.put(h.perm);
    dm.rpack = reinterpret_cast<const int4 *>(pk.put(h.rpack));
    dm.fpk = pk.put(h.fpk);
    dm.fcoef = pk.put(h.fcoef);
    dm.fjob = reinterpret_cast<const int2 *>(pk.put(h.fjob));
    dm.n_fsplit = (int)h.fsplit.size() / 2;
    dm.fsplit = reinterpret_cast<const int2 *>(pk.put(h.fsplit));
    dm.jnz = reinterpret_cast<const int4 *>(pk.put(h.jnz));
    dm.sl_pack = pk.put(h.sl_pack);
    dm.jl_ptr = pk.put(h.jl_ptr);
    dm.jl_rec = reinterpret_cast<const int4 *>(pk.put(h.jl_rec));
    dm.su_pack = pk.put(h.su_pack);
    dm.n_wsec = h.el_phase.empty() ? 0 : h.n_sections;
    dm.n_el = (int)h.el_phase.size();
    dm.rh_slot = h.rh_slot;
    dm.zsr_Y = pk.put(h.zsr_Y);
    dm.zsr_low = pk.put(h.zsr_low);
    dm.pw_ptr = pk.put(h.pw_ptr);
    dm.pw = pk.put(h.pw);
    dm.n_pp = (int)h.pp.size() / 4;
    dm.pp = reinterpret_cast<const int4 *>(pk.put(h.pp));
    dm.n_g = h.g_ptr.empty() ? 0 : (int)h.g_ptr.size() - 1;
    dm.g_ptr = pk.put(h.g_ptr);
    dm.g_ent = pk.put(h.g_ent);
    dm.g_coef = pk.put(h.g_coef);
    dm.n_ch = (int)h.ch.size() / 4;
    dm.ch = reinterpret_cast<const int4 *>(pk.put(h.ch));
    dm.n_pw = h.n_pw;
    dm.n_pw64 = h.n_pw64;
    bdf_coefficients(dm);
    return pk.img;
}

std::vector<unsigned char> pack_arrow(const ArrowHost &a, ArrowDev &ad, const unsigned char *base) {
    Packer pk{{}, base};
    ad.P = a.P;
    ad.n_g = a.n_g;
    ad.n_phi = a.n_phi;
    ad.n_c = a.n_c;
    ad.n_loc = a.n_phi + a.n_c;
    ad.n = a.n_g + a.P * a.n_phi;
    ad.n_env = a.n_env;
    ad.E0 = a.E0;
    ad.Rg = a.Rg;
    ad.Rp = a.Rp;
    ad.grec = reinterpret_cast<const int4 *>(pk.put(a.grec));
    ad.prec = reinterpret_cast<const int4 *>(pk.put(a.prec));
    ad.st_sp = pk.put(a.st_sp);
    ad.st_nu = pk.put(a.st_nu);
    ad.coupled = pk.put(a.coupled);
    ad.gf_ptr = pk.put(a.gf_ptr);
    ad.gf_k = pk.put(a.gf_k);
    ad.gf_nu = pk.put(a.gf_nu);
    ad.blk = a.n_phi * a.n_phi + 2 * a.n_phi * a.n_c;
    return pk.img;
}

}  // namespace camp
