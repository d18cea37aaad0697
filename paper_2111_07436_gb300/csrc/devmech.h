// Device-side mechanism tables, shared by the host compiler (mech.cpp) and the
// CUDA kernels.  Every array lives in one device allocation; the struct is
// passed to kernels by value (it sits in the kernel-parameter constant bank).
//
// All species indices here are POSITIONS in the elimination order chosen by
// the compiler (position p holds species perm[p]); only the state/env/atol
// loads and stores translate back to declaration order.
#pragma once
#include <stdint.h>
#include <vector_types.h>

#define CAMP_QMAX 5
#define CAMP_MAXFAC 3  // at most 3 factors (with multiplicity) per rate term

enum {
    CAMP_P_ARRHENIUS = 0,
    CAMP_P_TROE = 1,
    CAMP_P_PHOTOLYSIS = 2,
    CAMP_P_EMISSION = 3,
    CAMP_P_LOSS = 4,
    CAMP_P_HENRY = 5,
    CAMP_P_AQREV = 6,
    CAMP_P_CUSTOM_H2O2 = 7,
    CAMP_P_CUSTOM_OH_HNO3 = 8,
    CAMP_P_COND_ARRHENIUS = 9,
    CAMP_P_SIMPOL = 10
};

#define CAMP_NPAR 10  // rate parameters per process
#define CAMP_ZSR_NY 8 // coefficients of one electrolyte's molality fit

// Lanes that integrate one cell of an n-species mechanism: one warp up to
// 192 species (up to 6 a lane), else one block of 64 threads (4 species a
// lane up to 256 species, 8 beyond), 128 or 256 threads (8 a lane).  For
// 193-256 species two warps with 4 slots each measured 1.3x one warp with 8
// (fewer registers a lane, more warps a SM).  The per-lane tables below are
// built for this many lanes.
inline int camp_cell_lanes(int n) {
    if (n <= 192) return 32;
    if (n <= 512) return 64;
    if (n <= 1024) return 128;
    return 256;
}

// The other lane count the launch autotuner tries for an n-species
// mechanism (0: none): 129-256 species run on one warp (6 or 8 slots a
// lane) or on 64 threads (4 slots a lane), whichever measures faster.
inline int camp_alt_lanes(int n) {
    if (n > 128 && n <= 192) return 64;
    if (n > 192 && n <= 256) return 32;
    return 0;
}

// LU op encoding for the sparse (row-wise) part of the factorisation
#define CAMP_OP_DIV 0x80000000u
#define CAMP_OP_TGT(op) ((int)((op)&0xFFFFu))
#define CAMP_OP_SRC(op) ((int)(((op) >> 16) & 0x7FFFu))

struct DevMech {
    int n;            // species
    int R;            // process instances
    int n_env;
    int env_sec_base; // env index of section 0's radius
    int lanes;        // lanes per cell the per-lane tables were built for

    // --- rate constants (process order) ---
    const int *rtype;     // [R]
    const double *rpar;   // [R][CAMP_NPAR]
    const int *rslot;     // [R] env slot (runtime types) or section (section types)
    const int *rnr;       // [R] total reactant multiplicity
    const int *rnp;       // [R] total product multiplicity (reversible types)
    int n_rev;            // reversible processes (the only ones with a kr)
    const int *rrev;      // [R] index into the cell's kr array, -1 if irreversible

    // --- rate terms r_k = kf prod(fwd) - kr prod(rev), one 16-byte record each:
    // x = fwd0 | fwd1 << 16, y = fwd2 | rv << 16, z = rev0 | rev1 << 16,
    // w = rev2 (positions; 16-bit fields, 0xffff = none; rv = kr index)
    const int4 *rpack;    // [R]

    // --- forcing gather f_p = sum_q c_q r_k(q), as lane jobs ---
    // entry q: process | index into fcoef << 16
    const int *fpk;       // [nf]
    const double *fcoef;  // the mechanism's distinct net coefficients
    // lane l's jobs: flane_ptr[l] .. flane_ptr[l+1], balanced by entry count.
    // Job: x = first entry, y = destination | entry count << 16; a destination
    // d < n is the position's f, d >= n the partial sum d - n of a position
    // whose sum was split into chunks (block cells only)
    const int *flane_ptr; // [lanes+1]
    const int2 *fjob;
    int n_part;           // partial sums of split forcing sums, substitution
                          // rows and factorisation rows (scratch after the
                          // rate terms; counted in FP64 values)
    int n_fsplit;         // positions whose sums are split
    // split position i: x = position, y = first partial | chunk count << 16
    const int2 *fsplit;   // [n_fsplit]

    // --- Jacobian, assembled straight into I - gamma J ---
    int nnzJ;
    // FP32: per-lane flat entry lists (nonzeros spread over the lanes by
    // entry count).  Record: x = bits of the FP32 coefficient, y = k (signed
    // 16 bits; -(r+1) for a reverse constant) | o1 << 16, z = LU offset |
    // diag << 16 | last-entry-of-nonzero << 17, w = o2 | CSR index << 16
    const int *jl_ptr;    // [lanes+1]
    const int4 *jl_rec;   // [entries + empty non-zeros]
    // FP64: by non-zero t: x = first entry, y = end entry, z = LU offset,
    // w = diagonal; entry q: constant jk (k, or -(r+1) for a reverse constant),
    // other factors jo (positions, -1 = none), coefficient jc
    const int4 *jnz;      // [nnzJ]
    const int *jk;        // [nj]
    const int *jo;        // [nj][2]
    const double *jc;     // [nj]

    // --- LU storage: sparse rows [0, nsp) then a dense trailing block ---
    int nlu;              // storage entries
    int d;                // first position of the dense block (= n when there is none)
    int D;                // dense block size n - d
    int LD;               // dense block row stride (odd, to spread shared-memory banks)
    int dbase;            // storage offset of the dense block

    // factorisation of the sparse part: row-wise (up-looking) ops as lane
    // jobs, by level.  Op: DIV flag | source << 16 | target (LU offsets; a
    // division makes the multiplier, an update subtracts it times the
    // source).  Job: x = first op in lops, y = op count | partial slots << 16,
    // z = row | (1 << 16 if the job ends by taking the row's pivot
    // reciprocal), w = partial base.  An update whose target has bit 15 set
    // adds to partial w + (target & 0x7fff) instead of the LU value.  Per
    // level, the rows cut into chunks then get a reduction (x = row |
    // reciprocal flag << 16, y = first entry of lred_off, z = shared columns
    // ns | chunks << 16, w = partial base; chunk c's slot s is w + c ns + s)
    // and their tail ops (x = first op, y = count).
    int n_flev;
    const int *ljob_ptr;  // [n_flev+1] into ljob
    const int4 *ljob;
    const uint32_t *lops;
    const int *lred_ptr;  // [n_flev+1] into lred / ltail
    const int4 *lred;
    const int *lred_off;  // LU offsets of the shared columns
    const int2 *ltail;

    // substitution entries: LU offset | column << 16
    const int *sl_pack;   // L entries of the sparse rows, row by row
    const int *su_pack;   // U entries of the sparse rows, row by row

    // forward substitution of the sparse part: lane jobs by level (jobs
    // within a level ordered to balance the lanes) over the rows that have L
    // entries.  Job: x = first entry of sl_pack, y = destination | entry count
    // << 16; a destination d < n is row d, finished by the job, d >= n the
    // partial dot product d - n of a row cut into chunks; the level's split
    // rows (x = row, y = first partial | chunk count << 16) then subtract
    // their partials in order.
    int n_slev;
    const int *slev_ptr;  // [n_slev+1] into sjob
    const int2 *sjob;
    const int *ssplit_ptr; // [n_slev+1] into ssplit
    const int2 *ssplit;

    // backward substitution of the sparse rows (i < d), by level
    int n_blev;
    const int *blev_ptr;  // [n_blev+1] into brow
    const int *brow;
    const int *su_ptr;    // [n+1] into su_pack
    const int *udiag;     // [n] storage offset of U(i,i) for sparse rows

    const int *perm;      // [n] position -> species (declaration order)

    // --- ZSR aerosol water as a parameter (Sect. 2.2.2): with n_wsec > 0 the
    // liquid volume of section b is L_b(y) = L_env,b + sum_e w_e y_e over its
    // electrolytes, w_e = 1e-9 P / (R T) / (1000 m_e(a_w)) with the molality
    // fit sqrt(m_e) = sum_j Y_j a_w^j at a_w = RH (held at the fit's lowest
    // activity below it).  Section processes then keep per-unit-volume
    // constants in kf / kr; the kernels apply L^-la, L^-lb where the
    // constants are used (each section process's rpack record carries
    // section + 1 in bits 16-26 of w, la in bits 27-28 and lb in bits 29-30),
    // and the Jacobian adds the chain-rule term J_p P_y.
    int n_wsec;           // sections with a water parameter (0: none)
    int n_el;             // electrolytes
    int rh_slot;          // env index of the relative humidity
    const double *zsr_Y;  // [n_el][CAMP_ZSR_NY]
    const double *zsr_low;// [n_el]
    const int *pw_ptr;    // [n_wsec+1] into pw
    const int *pw;        // electrolyte entries: position | electrolyte << 16
    int n_pp;             // section processes with a power of 1/L (chain rule)
    // x = process, y = section, z = la | lb << 8, w = kr index (-1: none)
    const int4 *pp;       // [n_pp]
    // d f_i / d L_b for each (row, section) pair g: sum over entries of
    // coefficient * d r_j / d L_b of parameterised process j
    int n_g;
    const int *g_ptr;     // [n_g+1] into g_ent, g_coef
    const int *g_ent;     // parameterised process index
    const double *g_coef; // net stoichiometric coefficient
    // chain-rule entries J_ij += g_(i,b) w_e, n_el consecutive records per
    // g: x = LU offset of (i, e), y = g index, z = electrolyte e, w =
    // species-CSR non-zero
    int n_ch;
    const int4 *ch;
    int n_pw;             // per-cell FP64 values of the parameter (0: none)
    int n_pw64;           // more of them in the FP64 form (reverse constants)

    // BDF coefficients: l-vector of prod_{i=1..q}(1 + x/i), local-error
    // constants 1/((q+1) l_1(q)), factorials
    double lcoef[CAMP_QMAX + 2][CAMP_QMAX + 2];
    double ecoef[CAMP_QMAX + 2];
    double fact[CAMP_QMAX + 2];
    // the same, arranged so the step controller multiplies instead of
    // dividing and compares squares instead of taking roots
    double inv_l1[CAMP_QMAX + 2];   // 1 / l_1(q)
    double ecoef2[CAMP_QMAX + 2];   // ecoef(q)^2
    double rn;                      // 1 / n
};
