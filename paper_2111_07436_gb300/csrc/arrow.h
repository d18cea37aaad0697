// The block-arrow form of a mechanism whose condensed phase is instanced once
// per computational particle (the particle-resolved representation, CAMP
// paper Sect. 2.2.3 and Table 6; 10^4 particles in the box model of Sect.
// 4.1).  Every particle carries the same phase species and processes; its
// processes couple its own species and a few gas species (the phase-transfer
// gases), so the Jacobian is block-arrow: one small block per particle, the
// gas rows and columns as the arrow.  Instead of one sparsity pattern over
// all n_g + P n_phi species, the compiler keeps the processes of ONE instance
// (a template mechanism with a single particle) and the kernels apply it to
// every particle.
//
// Local numbering inside a particle: its phase species 0 .. n_phi - 1, then
// the coupled gas species n_phi .. n_phi + n_c - 1 (gas species coupled[c]).
#pragma once
#include <stdint.h>
#include <vector_types.h>

#define CAMP_ARROW_MAX_PHI 16  // phase species per particle
#define CAMP_ARROW_MAX_C 8     // gas species a particle exchanges with
#define CAMP_ARROW_MAX_GAS 32  // gas species (one lane each)

struct ArrowDev {
    int P;       // particles (instances of the phase)
    int n_g;     // gas species
    int n_phi;   // phase species per particle
    int n_c;     // gas species coupled to the particles
    int n_loc;   // n_phi + n_c
    int n;       // species of the full mechanism: n_g + P n_phi
    int n_env;   // env entries of the full mechanism: E0 + 3 P
    int E0;      // env index of particle 0's (radius, number, liquid volume)
    int Rg;      // gas processes
    int Rp;      // processes of one particle
    // process records, three int4 each:
    //   {template process k, forward factors nf, reverse factors nb, first stoichiometry entry}
    //   {forward factor species f0, f1, f2 (-1: none), one past the last entry}
    //   {reverse factor species b0, b1, b2 (-1: none), reversible}
    // factor and stoichiometry species: gas numbering for gas processes,
    // local numbering for particle processes
    const int4 *grec;
    const int4 *prec;
    const int *st_sp;
    const double *st_nu;
    const int *coupled;   // [n_c] gas species of local index n_phi + c
    // gas rows: for gas species i, the gas processes that change it and the
    // net coefficient (gf_ptr [n_g + 1] into gf_k, gf_nu)
    const int *gf_ptr;
    const int *gf_k;
    const double *gf_nu;
    // per-particle LU storage, in LU elements per particle: the particle
    // block n_phi x n_phi (L unit lower + U with reciprocal pivots), then
    // U_pG n_phi x n_c, then L_Gp n_c x n_phi
    int blk;
};
