/*
 * FP64 CPU oracle for dynamic-bonding molecular dynamics (test infrastructure).
 *
 * This library is the correctness reference for the CUDA path.  It is plain,
 * single-threaded C compiled with -ffp-contract=off, indexes everything by
 * particle tag, enumerates neighbours directly (cell grid or all pairs), and
 * shares no source with the CUDA path.  Only the tests, the package smoke
 * check and the benchmark's CPU-baseline leg may load it.
 *
 * Paper: "pySNAP + DyBond-v2" (arXiv 2609.21204), Sec. II (DyBond-v2: theory
 * and implementation).
 */
#ifndef SNAP_ORACLE_H
#define SNAP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_TYPES 8
#define ORC_MAX_BTYPES 8
#define ORC_MAX_RX 8
#define ORC_VMAX 4      /* dynamic-bond slots per particle */
#define ORC_SMAX 4      /* static-bond slots per particle */

enum { ORC_HARMONIC = 0, ORC_FENE = 1, ORC_FENEWCA = 2, ORC_TETHER = 3 };
/* Philox key streams (second key word carries (reaction << 8) | stream) */
enum { ORC_FORM = 1, ORC_BREAK = 2, ORC_MATCH = 3, ORC_ORDER = 4, ORC_LANGEVIN = 5,
       ORC_MH_SEL = 6, ORC_MH_ACC = 7, ORC_MH_OWN = 8 };
enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_FENE = 6, ORC_ERR_NONFINITE = 7 };

typedef struct {
    int32_t type_a, type_b, bond_type;
    double r_min, r_max;
    double p_on0, p_off;       /* per-sweep probabilities, Eq. (2) */
    int32_t self_avoid;        /* 1: sites of one molecule (orc_state.mol) do not react with each other */
    double slip_a;             /* slip bond, Eq. (slip): P_off(r) = p_off exp(a sqrt(U_b(r)/kT)); 0: off */
    int32_t melt;              /* 1: melting switch, Eqs. (gT)-(kT), re-evaluated every sweep at the
                                * kinetic temperature (orc_params.kinetic_T); p_on0/p_off above hold
                                * the set-point rates used otherwise */
    double melt_lambda, melt_t, kon_init, koff_init, kon_melt, koff_melt;
} orc_reaction;

typedef struct {
    int64_t n;
    double box[3];
    double dt, kT, gamma;
    uint64_t seed;
    int32_t ntypes;
    double sigma[ORC_MAX_TYPES];
    double eps[ORC_MAX_TYPES * ORC_MAX_TYPES];
    double rcut[ORC_MAX_TYPES * ORC_MAX_TYPES];  /* <= 0: WCA cut 2^(1/6) sigma_ij */
    int32_t valence[ORC_MAX_TYPES];
    int32_t nbtypes;
    int32_t bkind[ORC_MAX_BTYPES];
    double bk[ORC_MAX_BTYPES], br0[ORC_MAX_BTYPES];   /* harmonic k, r0; FENE(WCA) k, R0; Tether k_b, l_min */
    double bx[ORC_MAX_BTYPES][3];                      /* FENEWCA eps, sigma, delta; Tether l_c1, l_c0, l_max */
    int32_t nrx;
    orc_reaction rx[ORC_MAX_RX];
    int32_t bond_period;
    int32_t kinetic_T;         /* 1: T in Eq. (3), the slip factor and g(T) is the instantaneous kinetic
                                * temperature of the half-step velocities (orc_kinetic_T), evaluated at
                                * the start of every sweep; 0: the set-point kT */
} orc_params;

typedef struct {
    double *x, *y, *z;          /* positions in [0, L) */
    double *vx, *vy, *vz;       /* half-step velocities v_{t-1/2} */
    int32_t *img;               /* 3n periodic image counters */
    const int32_t *type;
    const int32_t *sp;          /* n*ORC_SMAX static partner tags (-1 empty) */
    const int32_t *sbt;         /* n*ORC_SMAX static bond types */
    int32_t *dp;                /* n*ORC_VMAX dynamic partner tags, ascending, -1 last */
    int32_t *drx;               /* n*ORC_VMAX reaction index of each dynamic bond */
    int64_t *dbirth;            /* n*ORC_VMAX step at which the bond formed */
    int32_t *occ;               /* number of dynamic bonds per particle */
    double *fx, *fy, *fz;       /* conservative forces (output of orc_forces) */
    double *pe;                 /* per-particle potential energy (nullable) */
    int64_t *life_hist;         /* lifetime histogram in sweeps (nullable) */
    int32_t nhist;
    int64_t step;
    const int32_t *mol;         /* molecule id per particle: the connected components of the
                                 * static bonds; read by reactions with self_avoid */
    double *fscale;             /* nullable: orc_forces writes, per particle, the sensitivity scale
                                 * G_i = sum_j (|F_ij| + r_ij |dF_ij/dr|) over every pair and bond
                                 * force on it: relative perturbations of at most e in every
                                 * separation and in every term change F_i by at most ~e G_i */
    double vabs;                /* written by orc_forces: sum over pairs and bonds of
                                 * r (|F| + r |dF/dr|), the same scale for the virial */
} orc_state;

typedef struct {
    int64_t scanned;        /* type/occupancy-compatible partners examined */
    int64_t in_window;      /* of those, inside [r_min, r_max] */
    int64_t proposals;      /* free sites that proposed */
    int64_t edges;          /* distinct proposal edges */
    int64_t survivors;      /* edges surviving the matching */
    int64_t formed;
    int64_t break_tested;
    int64_t broken;
} orc_sweep_stats;

/* Optional per-particle record of the first processed reaction of a sweep. */
typedef struct {
    int32_t *prop;          /* proposed partner tag or -1 */
    double *prop_r;         /* separation of the proposal */
    int32_t *matched;       /* partner tag of the surviving matched edge, or -1 */
    uint8_t *formed;        /* 1 if the particle gained a bond */
    int32_t *order;         /* processing order of the reactions (nrx entries) */
} orc_trace;

/* Philox-4x32-10 (Salmon et al., SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* 53-bit uniform in [0,1) from two 32-bit words. */
double orc_u53(uint32_t w0, uint32_t w1);
/* exp(x) by Cody–Waite ln2 reduction and a degree-13 Taylor polynomial. */
double orc_exp(double x);
double orc_log(double x);
/* Instantaneous kinetic temperature of the half-step velocities (Sec. II.B: T
 * is the kinetic temperature when the updater triggers), summed
 * deterministically: every particle's v^2 = (vx^2 + vy^2) + vz^2 is rounded to
 * the nearest multiple of 2^-32 and the integers are added exactly in int64;
 * T = sum 2^-32 / (3 n) (3 n degrees of freedom: the Langevin thermostat
 * conserves no momentum).  Exact for any summation order. */
double orc_kinetic_T(const orc_params *P, const orc_state *S);
/* tanh(x) = (1 - e^{-2|x|}) / (1 + e^{-2|x|}) with the sign of x, with orc_exp. */
double orc_tanh(double x);
/* Bond energy U_b(r) of bond type bt (libm exp and log; +inf outside the
 * potential's finite range). */
double orc_bond_energy(const orc_params *P, int32_t bt, double r);
/* The separation a proposal of a reaction with bond type bt aims at (the
 * minimum of the bond energy; see the sweep). */
double orc_aim_separation(const orc_params *P, int32_t bt);

int orc_sweep(const orc_params *P, orc_state *S, int64_t step, orc_sweep_stats *st,
              orc_trace *tr);
int orc_forces(const orc_params *P, orc_state *S, double *e_pair, double *e_bond,
               double *virial);
int orc_run(const orc_params *P, orc_state *S, int64_t nsteps, double *ke_out);
typedef struct {
    int64_t form_attempts, form_accepts, break_attempts, break_accepts;
} orc_mh_stats;

/* One Metropolis–Hastings sweep with the uniform proposal (reaction 0 only):
 * checkerboard cells of side >= 2 r_max + 0.05 (even count per axis), one
 * initiator per active cell, form or break with the MH ratio of the
 * owned-pair move set.  Returns ORC_ERR_ARG if the box is too small. */
int orc_mh_sweep(const orc_params *P, orc_state *S, int64_t step, orc_mh_stats *st);

/* Pair-distance histogram behind g(r): unordered pairs of types (ta, tb) with
 * r < rmax, bin floor(r / (rmax / nbins)); counts are added to hist[nbins]. */
int orc_rdf(const orc_params *P, const orc_state *S, int32_t ta, int32_t tb, double rmax, int32_t nbins,
            int64_t *hist);
/* All unordered pairs (i<j) with r < rc_ij + extra, written as tag pairs.
   Returns the count (writes at most cap pairs). */
int64_t orc_pairs_within(const orc_params *P, const orc_state *S, double extra,
                         int use_reactive_cut, int32_t *out, int64_t cap);
/* Candidate partners of particle i for reaction slot a: writes tags, returns count. */
int32_t orc_candidates(const orc_params *P, const orc_state *S, int32_t a, int64_t i,
                       int32_t *out, int32_t cap);

#ifdef __cplusplus
}
#endif
#endif
