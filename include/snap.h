/*
 * snap — B300-native dynamic-bonding molecular dynamics: C ABI.
 *
 * One MD step = [neighbour-list rebuild when any particle moved more than
 * skin/2] -> [bond sweep every bond_period steps] -> pair + bond forces ->
 * Langevin kick/drift.  All of it runs in hand-written CUDA kernels for
 * sm_103a on the stream given in snap_config; nothing returns to the host
 * except on the snap_get_* / snap_sync calls.
 *
 * The method is the dynamic-bonding scheme of "pySNAP + DyBond-v2"
 * (arXiv 2609.21204), Sec. II:
 *   - a reaction (snap_add_reaction) is a two-state process between sites of
 *     two types with per-sweep probabilities P_on^0 and P_off (Eqs. 1-2);
 *   - formation is accepted with P_on^0 exp(-U_b(r)/kT), breaking with P_off
 *     (Eq. 3; Eq. 4 for the harmonic bond);
 *   - the sweep runs proposal, matching, acceptance and breaking per
 *     reaction, reading occupancies as they stood when the reaction began
 *     (Sec. II.C, Fig. 1), in a random reaction order redrawn every sweep;
 *   - every random decision is a Philox-4x32-10 draw keyed by the seed, the
 *     reaction and the stream, counted by the step and the sorted tag pair
 *     (Sec. II.E), so results do not depend on thread scheduling or memory
 *     order.
 * Readings where the paper is silent: valence is a per-type occupancy counter
 * (a particle joins at most one new bond per reaction per sweep, never two
 * bonds to one partner); matching is a one-round locally dominant matching on
 * per-edge Philox priorities; kT in Eq. 3 is the set-point kT (kT = 0 gives
 * the factor [U_b <= 0]); the window test r_min^2 <= r^2 <= r_max^2 and the
 * acceptance are computed in FP64 in every precision mode.
 *
 * Conventions for every call:
 *   - particles are identified by their tag 0..n-1 (global over replicas:
 *     replica r owns tags [sum_{q<r} n_q, sum_{q<=r} n_q)); every host array
 *     is in tag order; positions are x,y,z triples (n*3 doubles);
 *   - host arrays passed in are copied before the call returns; host arrays
 *     passed out are owned by the caller and must hold the stated size;
 *   - no call aborts the process; errors are returned as snap_status and
 *     described by snap_last_error(); device-side faults (non-finite
 *     positions, FENE overstretch, neighbour-list overflow) latch a status
 *     word that snap_sync / snap_step / snap_get_* report;
 *   - all GPU work is ordered on cfg.stream; calls that return host data
 *     synchronise that stream.
 */
#ifndef SNAP_H
#define SNAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct snap_ctx snap_ctx;

typedef enum {
    SNAP_OK = 0,
    SNAP_ERR_ARG = 1,            /* invalid argument or size */
    SNAP_ERR_STATE = 2,          /* call out of order (e.g. step before particles) */
    SNAP_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    SNAP_ERR_OOM = 4,            /* device allocation failed */
    SNAP_ERR_NLIST_OVERFLOW = 5, /* neighbour capacity exceeded (grown and retried internally) */
    SNAP_ERR_FENE_OVERSTRETCH = 6, /* a bond outside its potential's finite range (FENE, FENEWCA, Tether) */
    SNAP_ERR_NONFINITE = 7,      /* a position became NaN/Inf */
    SNAP_ERR_TIMEOUT = 8
} snap_status;

enum { SNAP_FP64 = 0, SNAP_MIXED = 1 };     /* precision modes */
enum { SNAP_HARMONIC = 0, SNAP_FENE = 1, SNAP_FENEWCA = 2, SNAP_TETHER = 3 };  /* bond kinds */

#define SNAP_MAX_TYPES 8
#define SNAP_MAX_BOND_TYPES 8
#define SNAP_MAX_REACTIONS 8
#define SNAP_MAX_VALENCE 4       /* dynamic bonds per particle */
#define SNAP_MAX_STATIC 4        /* static bonds per particle */

typedef void *(*snap_alloc_fn)(size_t bytes, void *user);
typedef void (*snap_free_fn)(void *ptr, void *user);

typedef struct {
    int64_t n;               /* total particles (sum over replicas), below 2^27 */
    double box[3];           /* periodic box edges (single system; replica_box overrides) */
    double dt, kT, gamma;    /* time step, set-point temperature, Langevin friction */
    uint64_t seed;           /* Philox key; only the low 48 bits are used */
    int32_t precision;       /* SNAP_FP64: all FP64; SNAP_MIXED: FP32 pair/bond forces */
    int32_t bond_period;     /* n of Eq. 2: sweep every bond_period steps (>= 1) */
    double skin;             /* neighbour-list skin (> 0) */
    int32_t n_replicas;      /* 0 or 1: one system; > 1: independent replicas */
    const int64_t *replica_n;     /* n_replicas counts (NULL if one system) */
    const double *replica_box;    /* n_replicas*3 box edges (NULL: all use box) */
    const double *replica_kT;     /* n_replicas set-point kT (NULL: all use kT) */
    const uint64_t *replica_seed; /* n_replicas seeds (NULL: seed + replica index) */
    void *stream;            /* cudaStream_t the library launches on (NULL: default stream) */
    snap_alloc_fn alloc;     /* device allocator (NULL: cudaMalloc) */
    snap_free_fn free;       /* matching release function */
    void *alloc_user;        /* passed to alloc/free */
    int32_t block_size;      /* threads per block for particle kernels: 0 (= 256) or a
                                multiple of 32 up to 256 */
    int32_t nlist_capacity;  /* initial force-list entries per particle (0: from density;
                                the reactive list is always sized from density) */
    int32_t lifetime_bins;   /* bins of the bond-lifetime histogram (0: 256) */
} snap_config;

typedef struct {
    int64_t step;            /* steps taken so far */
    int64_t n_bonds;         /* dynamic bonds present */
    int64_t sweeps;          /* sweeps performed */
    int64_t formed_total, broken_total;
    /* counters of the most recent sweep (summed over reactions and replicas) */
    int64_t scanned;         /* neighbour entries examined by free reactive sites */
    int64_t in_window;       /* compatible partners inside [r_min, r_max] */
    int64_t proposals, edges, survivors, formed, break_tested, broken;
    int64_t nlist_builds;    /* neighbour-list rebuilds so far */
    int64_t nlist_entries;   /* force-list entries written by the last rebuild */
    int64_t mh_form_attempts, mh_form_accepts;    /* Metropolis-Hastings moves so far */
    int64_t mh_break_attempts, mh_break_accepts;
    int64_t events_logged;   /* bond-formation events offered to the event log */
    int64_t rnlist_entries;  /* reactive-list entries written by the last rebuild */
    int64_t rebuild_launches; /* launches of the rebuild kernels (taken or skipped) so far */
    int32_t nlist_capacity;  /* current force-list entries-per-particle capacity */
    int32_t status;          /* latched device status (snap_status value) */
} snap_stats;

typedef struct {
    double e_pair, e_bond;   /* potential energies (FP64 sums, fixed order) */
    double kinetic;          /* kinetic energy of v_{t-1/2} (sum of v^2/2) */
    double virial;
} snap_energy;

/* Create a context; validates cfg and copies it (replica arrays included).
 * Allocates device memory for n particles through cfg.alloc.  On error
 * *out is NULL and nothing is allocated. */
snap_status snap_init(snap_ctx **out, const snap_config *cfg);

/* Interaction types.  sigma[ntypes]; eps_pair[ntypes*ntypes] (row-major, must
 * be symmetric); rcut[ntypes*ntypes] pair cut-offs, or NULL for the WCA cut
 * 2^(1/6) sigma_ij with sigma_ij = (sigma_i + sigma_j)/2.  The pair potential is
 * the Lennard-Jones potential shifted to zero at the cut (the WCA potential
 * for the default cut); it acts on every pair, bonded or not. */
snap_status snap_set_types(snap_ctx *, int32_t ntypes, const double *sigma,
                           const double *eps_pair, const double *rcut);

/* Dynamic-bond capacity per type: valence[ntypes] in 0..SNAP_MAX_VALENCE
 * (0 = not reactive).  The occupancy counter generalises the paper's unit
 * valence flag (Sec. II.A, II.C). */
snap_status snap_set_valence(snap_ctx *, const int32_t *valence);

/* Bond type bt: SNAP_HARMONIC U = k/2 (r - r0)^2, or SNAP_FENE
 * U = -k R0^2/2 ln(1 - (r/R0)^2) with r0_or_R0 = R0.  Either kind may be a
 * static bond or the bond type of a reaction (snap_add_reaction).  The other
 * kinds take snap_set_bond_params_ex (SNAP_ERR_ARG here). */
snap_status snap_set_bond_params(snap_ctx *, int32_t bt, int32_t kind, double k,
                                 double r0_or_R0);

/* Bond type bt of any kind (Sec. II.B: the updater accepts the harmonic,
 * FENEWCA and Tether evaluators of HOOMD-blue; the potentials below are those
 * of HOOMD-blue's documentation), params[nparams] host doubles:
 *   SNAP_HARMONIC (2): k, r0            U = k/2 (r - r0)^2
 *   SNAP_FENE     (2): k, R0            U = -k R0^2/2 ln(1 - (r/R0)^2)
 *   SNAP_FENEWCA  (5): k, R0, eps, sigma, delta; with s = r - delta,
 *       U = -k R0^2/2 ln(1 - (s/R0)^2) + 4 eps [(sigma/s)^12 - (sigma/s)^6] + eps
 *       (the WCA bracket for s < 2^(1/6) sigma only)
 *   SNAP_TETHER   (5): k_b, l_min, l_c1, l_c0, l_max,
 *       U = k_b e^{1/(l_c0 - r)} / (l_max - r) for r > l_c0, plus
 *           k_b e^{1/(r - l_c1)} / (r - l_min) for r < l_c1, 0 in between.
 * Requirements: finite values; k >= 0 and R0 (l_min) > 0; FENEWCA eps >= 0,
 * sigma > 0, delta >= 0; Tether l_min < l_c1 < l_c0 < l_max; else
 * SNAP_ERR_ARG.  A bond outside the finite range of its potential (FENE and
 * FENEWCA at s >= R0 or s <= 0, Tether at r <= l_min or r >= l_max) latches
 * SNAP_ERR_FENE_OVERSTRETCH in force evaluations and is never formed by a
 * reaction (U_b = +inf in Eq. 3).  A proposal aims at the minimum of the
 * energy: r0 (harmonic), 0 (FENE), delta + s* with s* the root of dU/ds below
 * min(2^(1/6) sigma, R0) (FENEWCA; delta when eps = 0), (l_c1 + l_c0)/2, the
 * middle of the zero-energy interval (Tether). */
snap_status snap_set_bond_params_ex(snap_ctx *, int32_t bt, int32_t kind, const double *params,
                                    int32_t nparams);

/* Static bonds: nb tag pairs (2*nb ints) of bond type bt; at most
 * SNAP_MAX_STATIC per particle.  Never change during the run. */
snap_status snap_add_static_bonds(snap_ctx *, int64_t nb, const int32_t *tag_pairs,
                                  int32_t bt);

/* Register a reaction between particle types type_a and type_b forming bonds
 * of bond type bt (set before; any kind) when r_min <= r <= r_max, with
 * per-sweep probabilities p_on0 and p_off (Eqs. 1-3; K = p_on0/p_off).  The
 * Metropolis factor of Eq. 3 uses that bond type's energy (FENE: evaluated
 * with the library's own logarithm, +inf at r >= R0), and a proposal keeps
 * the partner closest to the bond term's minimum: r0 for a harmonic bond, 0
 * for FENE (Sec. II.B-C).  The slip bond and the Metropolis–Hastings move set
 * need a harmonic bond type.  self_avoid = 1
 * excludes intramolecular bonds (Sec. II.D): two sites of one molecule — a
 * connected component of the static bonds, traced by the library when the
 * first step runs and again whenever static bonds are added — are never
 * partners of this reaction; 0 admits them; other values return SNAP_ERR_ARG.
 * The Metropolis–Hastings move set (snap_set_mh) refuses such a reaction.
 * Writes the reaction index to *index_out when non-NULL. */
snap_status snap_add_reaction(snap_ctx *, int32_t type_a, int32_t type_b, int32_t bt,
                              double r_min, double r_max, double p_on0, double p_off,
                              int32_t self_avoid, int32_t *index_out);

/* Slip bond (Sec. II.D, Eq. slip): bonds of reaction `reaction` break with
 * P_off(r) = p_off exp(a sqrt(U_b(r)/kT)), capped at 1, evaluated in FP64 at
 * the bond's separation in every sweep.  At kT = 0 the factor takes its
 * limits (1 for U_b = 0; P_off = 1 for U_b > 0).  a = 0 (the default) keeps
 * P_off constant.  a must be finite and >= 0; the modifier excludes the melting
 * switch on the same reaction and the Metropolis–Hastings move set
 * (SNAP_ERR_ARG / SNAP_ERR_STATE). */
snap_status snap_set_slip(snap_ctx *, int32_t reaction, double a);

/* Melting switch (Sec. II.D, Eqs. gT and kT): the rate constants of reaction
 * `reaction` become k(T) = k_init (1 - g) + k_melt g with
 * g = (tanh(lambda (T - t_melt)) + 1) / 2 at each replica's set-point kT, and
 * the per-sweep probabilities P = k n dt (Eq. 2, n = bond_period), replacing
 * the reaction's p_on0 and p_off in every replica.  Rates must be finite and
 * >= 0 with P <= 1 (else SNAP_ERR_ARG and nothing changes); excludes the slip
 * bond on the same reaction. */
snap_status snap_set_melting(snap_ctx *, int32_t reaction, double lambda, double t_melt,
                             double kon_init, double koff_init, double kon_melt, double koff_melt);

/* Temperature of the sweep (Sec. II.B: T in Eq. 3 is the instantaneous
 * kinetic temperature when the updater triggers).  on = 0 (default): every
 * replica's set-point kT.  on = 1: at the start of every sweep each replica's
 * T = sum_i |v_i|^2 / (3 n) over its half-step velocities v_{t-1/2}, summed
 * deterministically (each |v_i|^2 in FP64 rounded to the nearest multiple of
 * 2^-32 and the integers added exactly; sums of |v_i|^2 up to ~2^31 per
 * replica), so the sweep stays independent of thread order.  That T enters
 * Eq. 3, the slip factor, and the melting switch, which is then re-evaluated
 * every sweep (Eqs. gT, kT, 2, probabilities capped at 1).  T = 0 gives the
 * factor [U_b <= 0].  Other values of on return SNAP_ERR_ARG; the
 * Metropolis-Hastings move set (snap_set_mh) excludes on = 1 (SNAP_ERR_STATE). */
snap_status snap_set_kinetic_temperature(snap_ctx *, int32_t on);

/* Per-replica rates of one reaction (batched sweeps over the bond energy). */
snap_status snap_set_reaction_rates(snap_ctx *, int32_t reaction, int32_t replica,
                                    double p_on0, double p_off);

/* Initial state in tag order: pos3[n*3] (wrapped into the box on entry),
 * vel3[n*3] half-step velocities v_{-1/2} (NULL: zero), type[n].  Clears the
 * dynamic bonds and resets the step counter to 0. */
snap_status snap_set_particles(snap_ctx *, const double *pos3, const double *vel3,
                               const int32_t *type);

/* Overwrite positions (tag order, wrapped on entry) and optionally velocities. */
snap_status snap_set_positions(snap_ctx *, const double *pos3, const double *vel3);

/* Replace the dynamic-bond set: nb bonds given as tag pairs and reaction
 * indices; birth steps set to the current step.  Fails with SNAP_ERR_ARG if a
 * particle would exceed SNAP_MAX_VALENCE. */
snap_status snap_set_bonds(snap_ctx *, int64_t nb, const int32_t *tag_pairs,
                           const int32_t *reaction);

/* Advance nsteps MD steps (asynchronous on the stream except for a status
 * poll every 2000 steps and at the end, which wait).  Steps run as CUDA graphs
 * of 20 steps whose neighbour-list rebuild sits in a conditional node; the
 * environment variable SNAP_GRAPH_MODE=plain captures every kernel instead
 * (for per-kernel profilers), SNAP_GRAPH_MODE=none disables graphs. */
snap_status snap_step(snap_ctx *, int64_t nsteps);

/* Retry limit of the lock-free 16-byte compare-and-swap minimum that the
 * proposal phase uses when one side of a reaction is scarce (default 65536).
 * A pusher retries only when another pusher lowered the same key in between,
 * so the limit is never reached in correct operation; reaching it latches
 * SNAP_ERR_TIMEOUT, which the step or sweep call returns.  The failing step is
 * not taken: its sweep's scratch is cleared, bonds and positions keep their
 * values from before it, and the step counter does not advance.  Lowering the
 * limit (0 makes every such exchange give up) exercises that path; limit < 0
 * returns SNAP_ERR_ARG. */
snap_status snap_set_retry_limit(snap_ctx *, int32_t limit);

/* Threads per block of the neighbour-list build (a launch shape the
 * autotuner searches beside the particle kernels' block size): 64, 128 or
 * 256 (the default); anything else returns SNAP_ERR_ARG.  The lists, and so
 * every result, do not depend on it. */
snap_status snap_set_list_block(snap_ctx *, int32_t threads);

/* (A layout parameter of the neighbour-list build that Sec. II.C's sweep and
 * the force loop read; the paper has no counterpart.)
 * Sub-cells along x per neighbour cell for the list build: each cell is cut
 * into k slices of equal width along x, the particles are sorted by slice
 * within their cell, and the list build scans only the slices that overlap a
 * particle's x window in each row of cells, so fewer candidates are tested
 * where the cut-offs are short against the cell width.  k is 1, 2, 4 or 8, or
 * 0 (the default) for automatic: the most slices (at most 8) that keep at
 * least half a particle per (type, slice) on average.  Fewer are used where
 * the sort keys (cells x types x k) would exceed 2^24.  Only before
 * snap_set_particles lays the cell grid out (SNAP_ERR_STATE after); any other
 * k returns SNAP_ERR_ARG.  The lists hold the same pairs for every k; the
 * order of particles inside a cell, and so the order of list entries and of
 * the force sums, follows the slices. */
snap_status snap_set_list_subcells(snap_ctx *, int32_t k);

/* The number of sub-cells along x per cell in use (after snap_set_particles;
 * SNAP_ERR_STATE before). */
snap_status snap_get_list_subcells(snap_ctx *, int32_t *k);

/* Capture, instantiate and upload the step graphs for both buffer parities
 * now, so that no later snap_step pays for a capture (a step swaps two
 * coordinate buffers; a call with an odd step count leaves the next call on
 * the other one, and each parity has a graph of its own).  Runs no step and
 * changes no state; waits for the stream.  With SNAP_GRAPH_MODE=none it does
 * nothing.  Parameters or buffers that change later (a new reaction, a grown
 * neighbour list) make the graphs stale; the next snap_step recaptures. */
snap_status snap_prepare(snap_ctx *);

/* Advance nsteps MD steps launched one kernel at a time with CUDA events
 * between the phases, and write the average milliseconds per step of each
 * phase to ms[SNAP_NPHASES]: [0] neighbour-list maintenance (all rebuild
 * kernels, mostly early exits), [1] bond sweep, [2] the force + Langevin
 * kernel of the production step, [3] step end.  Same kernels and results as
 * snap_step; slower (no graphs). */
#define SNAP_NPHASES 4
snap_status snap_step_profiled(snap_ctx *, int64_t nsteps, double *ms);
/* One neighbour-list rebuild at the current positions (forced), each kernel
 * timed with CUDA events: ms[SNAP_NREBUILD_PHASES] = [0] cell keys, [1] scan
 * of the cell counts, [2] scatter, [3] in-cell sort, [4] gather into sorted
 * order, [5] empty (the copy back of the gathered arrays runs inside the
 * list build), [6] neighbour lists and copy back, [7] done flag.  Changes nothing
 * but the particle order (the state is the same physical state). */
#define SNAP_NREBUILD_PHASES 8
snap_status snap_rebuild_profiled(snap_ctx *, double *ms);

/* One bond sweep at the current positions with the current step counter as
 * its Philox counter; positions and the step counter are unchanged. */
snap_status snap_bond_update(snap_ctx *);

/* Conservative forces at the current positions and topology (tag order,
 * n*3 doubles; the FP32 values in SNAP_MIXED mode). */
snap_status snap_get_forces(snap_ctx *, double *f3);

/* Dynamic bonds ascending by (min tag, max tag): tag_pairs[2*cap] and
 * reaction[cap] (nullable).  *n_out = number of bonds; SNAP_ERR_ARG if it
 * exceeds cap (nothing written). */
snap_status snap_get_bonds(snap_ctx *, int32_t *tag_pairs, int32_t *reaction, int64_t cap,
                           int64_t *n_out);

snap_status snap_get_positions(snap_ctx *, double *pos3);
snap_status snap_get_velocities(snap_ctx *, double *vel3);
snap_status snap_get_images(snap_ctx *, int32_t *img3);

/* Neighbour lists as tag pairs (i, j), i < j, each unordered pair once: the
 * union of the force list (pairs within the pair cut-off + skin) and the
 * reactive list (reaction-compatible pairs within r_max + skin). */
snap_status snap_get_neighbors(snap_ctx *, int32_t *tag_pairs, int64_t cap, int64_t *n_out);

snap_status snap_get_stats(snap_ctx *, snap_stats *out);

/* Pair-distance histogram behind g(r) of replica `replica` (0 for one
 * system), the structural observable whose agreement with the FP64 reference
 * the method is checked by: hist[nbins] (host, written) receives, for every
 * unordered pair of one particle of type_a and one of type_b (two distinct
 * particles when type_a == type_b) at separation r < r_max, one count in bin
 * floor(r / dr), dr = r_max / nbins.  r is the exact FP64 minimum-image
 * separation of the current positions (the one the sweep's window test uses),
 * so the counts are a pure function of the positions.  The call forces a
 * neighbour-list rebuild first (in SNAP_MIXED mode that re-rounds the FP32
 * coordinates, as every rebuild does).  g(r) = counts / (pairs of an ideal
 * gas of the same composition in each spherical shell).  r_max must lie in
 * (0, w - 0.002], w the replica's smallest neighbour-cell edge; bad types,
 * replica or nbins outside 1..2^20 return SNAP_ERR_ARG. */
snap_status snap_get_rdf(snap_ctx *, int32_t replica, int32_t type_a, int32_t type_b, double r_max,
                         int32_t nbins, int64_t *hist);
snap_status snap_get_energy(snap_ctx *, snap_energy *out);
/* Bond lifetimes (in sweeps) of every bond broken so far; bins[nbins], last
 * bin collects the tail. */
snap_status snap_get_lifetime_hist(snap_ctx *, int64_t *bins, int32_t nbins);

/* Checkpoint: positions, velocities, images, dynamic bonds with birth steps and
 * the step counter.  Philox is counter-based, so a restored run continues
 * bit-identically.  Call with buf NULL to query *len. */
snap_status snap_get_state(snap_ctx *, void *buf, size_t *len);
snap_status snap_set_state(snap_ctx *, const void *buf, size_t len);

/* ---------------------------------------------------------------------------
 * Learned proposal (an extension beyond the paper): a 12 -> 64 -> 64 -> 1 ReLU
 * network scoring the candidate partners of a site, run on the tensor cores
 * (BF16 operands, FP32 accumulation, FP32 master weights).  Features of a
 * candidate pair (i, j), all in float32, in this order:
 *   r, (r - r0)/r_max, [type_i == type_a], [type_i == type_b],
 *   [type_j == type_a], [type_j == type_b], occ_i/val_i, occ_j/val_j,
 *   [occ_i < val_i], [occ_j < val_j], coord_i/8, coord_j/8
 * with coord_x the number of particles of the partner type of x within the
 * reaction's window [r_min, r_max] of x.  Parameters are packed as
 * W1[16][64] (rows 12..15 zero), b1[64], W2[64][64], b2[64], w3[64], b3.
 * All arrays named d_* are device pointers owned by the caller.
 * ------------------------------------------------------------------------- */
#define SNAP_MLP_FEATURES 12
#define SNAP_MLP_PARAMS 5313
typedef struct snap_mlp snap_mlp;
snap_status snap_mlp_create(snap_mlp **out, void *stream);
snap_status snap_mlp_set_weights(snap_mlp *, const float *w);       /* host, SNAP_MLP_PARAMS */
snap_status snap_mlp_get_weights(snap_mlp *, float *w);
/* logits of `rows` feature rows (d_feat: rows x 12 float32) into d_logits */
snap_status snap_mlp_forward(snap_mlp *, const float *d_feat, int64_t rows, float *d_logits);
/* mean listwise softmax cross-entropy over `events` candidate sets (rows
 * d_offsets[e]..d_offsets[e+1], d_offsets[0] = 0, label = index of the formed
 * partner within its set) and its gradient (host grad, nullable). */
snap_status snap_mlp_loss_grad(snap_mlp *, const float *d_feat, int64_t rows, const int32_t *d_offsets,
                               const int32_t *d_labels, int64_t events, double *loss, float *grad);
/* Adam over shuffled minibatches of batch_events events; losses[epochs] (nullable). */
snap_status snap_mlp_train(snap_mlp *, const float *d_feat, int64_t rows, const int32_t *d_offsets,
                           const int32_t *d_labels, int64_t events, int32_t epochs, int64_t batch_events,
                           float lr, uint64_t seed, double *losses);
void snap_mlp_destroy(snap_mlp *);

/* Metropolis-Hastings bond moves instead of the DyBond sweep (an extension
 * beyond the paper).  mode 0: DyBond sweep (default); 1: MH with the uniform
 * proposal; 2: MH with the learned proposal
 * q = (1 - eps_u) softmax(mlp) + eps_u / n.  Move set: checkerboard cells of
 * side >= 2 r_max + 0.05 (an even number per axis, colour = step mod 8), one
 * initiator per active cell drawn uniformly among its reactive particles,
 * form (with one of its owned candidates) or break (one of its owned in-window
 * bonds) with probability 1/2, accepted with the Metropolis-Hastings ratio for
 * the bond weight K exp(-U_b/kT), K = p_on0 / p_off.  Needs exactly one
 * reaction and one system; the network must outlive the context's use of it. */
snap_status snap_set_mh(snap_ctx *, int32_t mode, const struct snap_mlp *mlp, double eps_u);
/* One MH sweep at the current positions (step counter unchanged). */
snap_status snap_mh_sweep(snap_ctx *);
/* Sets the step counter (keys every Philox draw and the birth step of new
 * bonds; the MH colour is step mod 8).  step < 0: SNAP_ERR_ARG. */
snap_status snap_set_step(snap_ctx *, int64_t step);
/* Record bond-formation events of the DyBond sweep (training data for the
 * proposal network): for every site whose own proposal formed a bond, the
 * features of all its candidates (at most 16) and the index of the partner.
 * capacity 0 turns logging off; events past the capacity are counted in
 * snap_stats.events_logged but not stored.  snap_get_events copies them out
 * compactly (host buffers): feat[rows][12], offsets[events + 1],
 * labels[events]; *n_events / *n_rows are always set, and buffers smaller
 * than that return SNAP_ERR_ARG with nothing copied (a size query);
 * clear != 0 empties the log afterwards. */
snap_status snap_log_events(snap_ctx *, int64_t capacity);
snap_status snap_get_events(snap_ctx *, float *feat, int32_t *offsets, int32_t *labels, int64_t cap_events,
                            int64_t cap_rows, int64_t *n_events, int64_t *n_rows, int32_t clear);

/* Allocation-free pair energy (this entry point has no counterpart in the
 * paper; it is an addition for callers that cannot allocate device memory
 * while they run: a host framework that has reserved the device's memory for
 * its own allocator, a real-time loop that cannot afford an allocation's
 * latency or failure, a plugin that is only handed device pointers).
 *
 * Computes the total Lennard-Jones/WCA pair energy (d_out[0]) and pair virial
 * sum_pairs (-dU/dr) r (d_out[1]) of n particles by direct summation over all
 * pairs, with the same pair potential and parameters as snap_set_types.
 * d_pos3: device, n*3 doubles (x,y,z per particle); d_type: device, n int32,
 * each in [0, ntypes) (a particle whose type lies outside that range takes
 * part in no pair); d_out: device, 2 doubles; box, sigma[ntypes], eps_pair[ntypes^2] and
 * rcut[ntypes^2] (nullable: WCA cut) are host arrays read before the call
 * returns.  Work is queued on `stream` (a cudaStream_t, NULL: default stream);
 * d_out is valid once the stream reaches that point.
 *
 * Nothing is allocated: per-particle partial sums live in a fixed device
 * array of 2 * SNAP_NOALLOC_MAX_N doubles (1 MiB) that every GPU loading the
 * library holds until the process exits.  n above SNAP_NOALLOC_MAX_N (or
 * negative), a NULL pointer, ntypes outside 1..SNAP_MAX_TYPES or a box edge
 * <= 0 returns SNAP_ERR_ARG and queues nothing.  The first call on each device
 * looks up the array's device address with that device current (make that
 * first call before any stream capture); a lookup failure returns
 * SNAP_ERR_CUDA.  All calls share the array, so calls whose work overlaps on
 * the GPU (different streams, no ordering between them) race; calls ordered
 * on one stream do not.  Every entry a call reads is written by that call
 * first, so nothing needs clearing between calls. */
#define SNAP_NOALLOC_MAX_N 65536
snap_status snap_pair_energy_noalloc(int64_t n, const double *d_pos3, const int32_t *d_type,
                                     const double *box, int32_t ntypes, const double *sigma,
                                     const double *eps_pair, const double *rcut, double *d_out,
                                     void *stream);

/* Wait for the stream and return the latched device status (then cleared). */
snap_status snap_sync(snap_ctx *);
const char *snap_last_error(const snap_ctx *);
void snap_destroy(snap_ctx *);

#ifdef __cplusplus
}
#endif
#endif
