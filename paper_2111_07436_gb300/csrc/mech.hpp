// Mechanism compiler: JSON text -> processes -> sparsity, ordering, symbolic
// LU and the flat device tables (CAMP paper Table 1: get_used_jacobian_elements
// and update_ids happen here, once per mechanism, on the host).
#pragma once
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "arrow.h"
#include "devmech.h"

namespace camp {

struct Process {
    int type = 0;
    std::vector<std::pair<int, int>> react;    // (species, multiplicity), distinct
    std::vector<std::pair<int, double>> prod;  // (species, yield), distinct
    double par[CAMP_NPAR] = {};
    int slot = -1;                             // env slot or section
    int la = 0, lb = 0;                        // powers of 1/L in kf, kr (water parameter)
    bool reversible() const {
        return type == CAMP_P_HENRY || type == CAMP_P_AQREV || type == CAMP_P_SIMPOL;
    }
};

// Host image of one compiled mechanism.  Integer structure follows the rules
// in include/camp.h (camp_mech_structure); the device tables mirror DevMech.
struct HostMech {
    std::vector<std::string> species;
    int n = 0, n_gas = 0, n_env = 0, n_sections = 0, env_sec_base = 0;
    int lanes = 32;  // lanes that integrate one cell: the per-lane tables are built for this many
    std::vector<Process> procs;
    // ZSR aerosol-water parameter (none when el_phase is empty)
    int rh_slot = -1;
    std::vector<int> el_phase;                 // phase-species index per electrolyte
    std::vector<double> zsr_Y, zsr_low;        // [n_el][CAMP_ZSR_NY], [n_el]
    std::vector<int> pw_ptr, pw, pp, g_ptr, g_ent, ch;
    std::vector<double> g_coef;
    int n_pw = 0, n_pw64 = 0;

    // integer structure (species numbering except the LU, which is permuted)
    std::vector<int> rowptr, colidx, rxn_map, perm, iperm;
    std::vector<int> lu_rowptr, lu_colidx, level_fwd, level_bwd;

    // device tables
    std::vector<int> rtype, rslot, rnr, rnp, rfac, rrev;
    int n_rev = 0;
    std::vector<double> rpar;
    std::vector<int> fptr, fk;
    std::vector<double> fc;
    std::vector<int> flane_ptr, flane_pos;
    std::vector<int> rpack, jnz, sl_pack, su_pack;  // int4 records as 4 ints
    std::vector<int> fpk, fjob;   // forcing gather entries and lane jobs (see DevMech)
    std::vector<int> fsplit;      // split sums, 2 ints each (see DevMech)
    int n_fpart = 0;
    std::vector<double> fcoef;
    std::vector<int> jl_ptr, jl_rec;
    std::vector<int> jptr, jdst, jdiag, jk, jo;
    std::vector<double> jc;
    int nlu = 0, d = 0, D = 0, LD = 0, dbase = 0;
    std::vector<int> flev_ptr, frow, fops_ptr;
    std::vector<uint32_t> fops;
    // the factorisation as lane jobs (see DevMech)
    std::vector<int> ljob_ptr, ljob, lred_ptr, lred, lred_off, ltail, ltail_rows;
    std::vector<uint32_t> lops;
    int n_lpart = 0;
    std::vector<int> sl_ptr, sl_off, sl_col;
    // forward substitution: lane jobs by level, split rows (see DevMech)
    std::vector<int> slev_ptr, sjob, ssplit_ptr, ssplit;
    int n_spart = 0;
    std::vector<int> blev_ptr, brow, su_ptr, su_off, su_col, udiag;
    long long factor_updates = 0;  // multiply-adds one device factorisation executes
    // algorithmic work of the method, from the symbolic structure
    long long flops_forcing = 0;   // one f(y): rate products + stoichiometric sums
    long long flops_jacobian = 0;  // one J assembly into I - gamma J
    long long flops_factor = 0;    // one sparse LU factorisation (2 per update + divisions)
    long long flops_solve = 0;     // one pair of triangular solves
    long long model_forcing = 0;   // sum over processes of 2 |reactants| + |products|
};

// Throws std::runtime_error with a message on malformed input.
// instances >= 0 replaces the aerosol's section / particle count (the
// template of the block-arrow form compiles one instance).  lanes > 0
// builds the per-lane tables for that many lanes a cell (32, 64, 128 or
// 256, at most 8 species a lane) instead of camp_cell_lanes(n).
HostMech compile_mechanism(const char *json, size_t len, int instances = -1, int lanes = 0);

// The aerosol instancing of a mechanism, read without compiling it.
struct AerosolShape {
    int instances = 0;        // sections or computational particles
    bool particles = false;   // "representation": "particles"
    bool block_arrow = false; // "solver": "block_arrow" asked for
    bool water = false;       // a ZSR water parameter
};
AerosolShape aerosol_shape(const char *json, size_t len);

// Host image of the block-arrow form (arrow.h), built from the one-instance
// template `t` for P instances.
struct ArrowHost {
    int P = 0, n_g = 0, n_phi = 0, n_c = 0, E0 = 0, n_env = 0, Rg = 0, Rp = 0;
    std::vector<int> grec, prec;  // 12 ints a record
    std::vector<int> st_sp;
    std::vector<double> st_nu;
    std::vector<int> coupled;
    std::vector<int> gf_ptr, gf_k;
    std::vector<double> gf_nu;
    // algorithmic work of the full mechanism (as HostMech's counts)
    long long model_forcing = 0, flops_forcing = 0, flops_jacobian = 0, flops_factor = 0, flops_solve = 0;
};
ArrowHost build_arrow(const HostMech &t, int P);
std::vector<unsigned char> pack_arrow(const ArrowHost &a, ArrowDev &ad, const unsigned char *base);

// Fill the coefficient arrays of a DevMech (host-side arithmetic).
void bdf_coefficients(DevMech &dm);

// Pack all device tables into one byte image; `dm` receives offsets
// relative to `base` (pointers are rebased once the image is on the device).
std::vector<unsigned char> pack_tables(const HostMech &h, DevMech &dm, const unsigned char *base);

}  // namespace camp
