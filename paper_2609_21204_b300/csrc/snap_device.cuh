// Device-side definitions shared by the snap kernels (sm_103a).
//
// Counter-based randomness (Philox-4x32-10, Salmon et al. SC'11) and the
// exponential of the acceptance factor are implemented here from their
// published definitions so that every stochastic decision of the bond sweep
// is a pure function of (seed, reaction, stream, step, tag pair), as Sec. II.E
// of the DyBond-v2 paper requires.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace snap {

constexpr int kMaxTypes = 8;
constexpr int kMaxBondTypes = 8;
constexpr int kMaxRx = 8;
constexpr int kVmax = 4;   // dynamic-bond slots per particle
constexpr int kSmax = 4;   // static-bond slots per particle

// Philox key streams: key word 1 = ((seed >> 32) & 0xFFFF) << 16 | reaction << 8 | stream
enum Stream : uint32_t { kForm = 1, kBreak = 2, kMatch = 3, kOrder = 4, kLangevin = 5,
                         kMhSel = 6, kMhAcc = 7, kMhOwn = 8 };

// status bits latched by kernels (mapped to snap_status on the host)
enum StatusBit : uint32_t {
    kStOverflow = 1u << 0,
    kStFene = 1u << 1,
    kStNonfinite = 1u << 2,
    kStTimeout = 1u << 3,   // a bounded retry loop gave up (a defect; the step is not trusted)
};

// ------------------------------------------------------------ parameters
// Passed by value to every kernel (kernel-parameter space, broadcast reads).
struct DevParams {
    int32_t ntypes, nrx, period, nhist;
    int32_t valence[kMaxTypes];
    // pair tables, index ti*kMaxTypes+tj
    float rc2f[kMaxTypes * kMaxTypes];      // pair cut-off squared
    float fl2f[kMaxTypes * kMaxTypes];      // force-list cut-off squared: (pair cut + skin)^2
    float xl2f[kMaxTypes * kMaxTypes];      // reactive-list cut-off squared: (r_max + skin)^2, 0: none
    float sig2f[kMaxTypes * kMaxTypes], eps24f[kMaxTypes * kMaxTypes], shiftf[kMaxTypes * kMaxTypes];
    double rc2d[kMaxTypes * kMaxTypes];
    double sig2d[kMaxTypes * kMaxTypes], eps24d[kMaxTypes * kMaxTypes], shiftd[kMaxTypes * kMaxTypes];
    // bond types
    int32_t bkind[kMaxBondTypes];   // 0 harmonic, 1 FENE, 2 FENEWCA, 3 Tether (the C ABI's bond kinds)
    double bk[kMaxBondTypes], br0[kMaxBondTypes];   // harmonic k, r0; FENE(WCA) k, R0; Tether k_b, l_min
    float bkf[kMaxBondTypes], br0f[kMaxBondTypes];
    double bx[kMaxBondTypes][3];    // FENEWCA: eps, sigma, delta; Tether: l_c1, l_c0, l_max
    float bxf[kMaxBondTypes][3];
    // reactions
    int32_t rx_ta[kMaxRx], rx_tb[kMaxRx], rx_bt[kMaxRx];
    int32_t rx_self[kMaxRx];   // 1: sites of one molecule do not react with each other (Sec. II.D)
    double rx_slip[kMaxRx];    // slip-bond parameter a of Eq. (slip); 0: constant P_off
    double rx_r0[kMaxRx];      // separation a proposal aims at: harmonic r0; 0 for FENE
    int32_t slip_mask;         // bit a set: reaction a has the slip modifier
    double rx_rmin2[kMaxRx], rx_rmax2[kMaxRx];
    // integrator
    double dt, half_dt, gamma, sqrt3;
    float dtf, gammaf, sqrt3f;   // the same, rounded to FP32 (mixed-mode kick)
    float disp2f;           // squared displacement that triggers a rebuild
    int32_t nbr_cap;        // force-list entries per particle
    int32_t rnbr_cap;       // reactive-list entries per particle
    int64_t n;              // particles (all replicas)
    int64_t nbr_stride;     // column stride of both neighbour lists
    int32_t nrep;
    int32_t screen;         // mixed mode: FP32 pre-screen of the proposal test, FP32 velocities
    int32_t ncell;          // cells over all replicas
    int32_t sub_shift;      // log2 of the sub-cells along x per cell: sort keys are
                            // ((type * ncell + rank of the row's first cell) << sub_shift) + sub-cell x
    int32_t mh_cells, mh_moves;   // MH checkerboard cells and active cells per sweep
    float mh_eps;           // weight of the uniform component of the learned proposal
    int32_t log_events;     // record bond-formation events in the plain sweep
    int64_t pdist_rows;     // pushing sites whose pair distances fit the pdist scratch
    int32_t has_static;     // any static bonds (else their slots are neither gathered nor read)
    int32_t cas_cap;        // retries of the push-mode 16-byte compare-and-swap before SNAP_ERR_TIMEOUT
    // kinetic temperature (Sec. II.B) and the melting switch re-evaluated at it (Eqs. gT-kT)
    int32_t kinetic_T;      // 1: T of the sweep is the kinetic temperature of the half-step velocities
    int32_t melt_mask;      // bit a set: reaction a has the melting switch
    double period_dt;       // n dt of Eq. 2
    double melt_lambda[kMaxRx], melt_t[kMaxRx];
    double kon_init[kMaxRx], koff_init[kMaxRx], kon_melt[kMaxRx], koff_melt[kMaxRx];
};

struct RepDev {
    double L[3], invL[3], halfL[3], w[3];
    float wf[3];
    float cscale[3];        // cells per unit length (nc / L) in FP32, for cell assignment
    int32_t nc[3];
    int32_t cell_off;       // first global cell id of this replica
    int32_t pad0;
    int64_t tag_off, n;
    double kT, noise_c;     // set-point kT and sqrt(2 gamma kT / dt)
    double t_sweep;         // T of the current sweep: kT, or the kinetic temperature (k_sweep_begin)
    float noise_cf;         // noise_c rounded to FP32 (mixed-mode kick)
    uint32_t key0, key1hi;  // Philox key words derived from the seed
    double p_on0[kMaxRx], p_off[kMaxRx];
    unsigned long long off_thresh[kMaxRx];   // ceil(p_off * 2^53): break iff 53-bit draw < this
    int32_t mh_nc[3];                        // Metropolis–Hastings checkerboard cells per axis (even)
    int32_t pad1;
};

// Device arrays (sorted particle order unless stated).
struct DevArrays {
    double *x, *y, *z, *vx, *vy, *vz;   // vx..vz: FP64 mode velocities
    float4 *v4;                     // mixed mode velocities (w unused)
    int32_t *ix, *iy, *iz;          // image counters
    int32_t *type, *tag, *rtag, *rep;
    int32_t *mol;   // molecule id by tag (connected components of the static bonds); null unless a
                    // reaction excludes intramolecular partners
    void *pos4;                     // float4 or double4_32a: coords relative to frozen cell origin, w = bits
    void *pos4n;                    // the second pos4 buffer: the fused step writes the new coordinates here
    float4 *ref4;                   // rel coords at the last rebuild (displacement test)
    float4 *npos;                   // FP32 wrapped positions at the last rebuild, cell bits in w (list build)
    void *force;                    // float4 or double4_32a (w unused)
    int4 *sp;                       // static partner tags (-1 empty), kSmax per particle
    int32_t *sbt;                   // static bond types, 8 bits each, packed
    int4 *dp;                       // dynamic partner tags, ascending, -1 last
    int32_t *drx;                   // reaction index per dynamic slot, 8 bits each, packed
    int4 *dbirth;                   // step (low 32 bits) at which each dynamic bond formed
    int32_t *occ;                   // dynamic bonds held
    uint8_t *avail;                 // type if occ < valence, else 0xFF (set per sweep)
    int32_t *avail_count;           // available particles per type (this sweep; kMaxTypes)
    int32_t *avail_list;            // push mode: available particles of type t at t * n + k
    ulonglong2 *pkey;               // push mode: smallest (|r - r0| as FP64 bits, pusher tag) pushed to a site
    unsigned long long *pdist;      // push mode: pair distances of pass 1, kPushSlots per pushing site
    int32_t *nbr, *nn;              // force list (column-major): pairs within pair cut + skin
    int32_t *rnbr, *rnn;            // reactive list: compatible pairs within r_max + skin
    // cell list
    int32_t *cell_count, *cell_start, *cell_cursor, *cell_key, *order, *rank_of;
    // sweep scratch
    int32_t *prop;                  // proposed partner index or -1
    double *prop_d;                 // |r - r0| of the proposal (FP64)
    uint32_t *prio;
    unsigned long long *best;
    int32_t *fpart;                 // formed partner index or -1
    uint32_t *brk;                  // bit s set: dynamic slot s breaks
    int32_t *rx_order;              // processing order of the reactions this sweep
    int32_t *site_list;             // sites with proposal work this reaction (compacted)
    int32_t *list_count;            // length of site_list
    int32_t *cont;                  // kContenders candidates per listed site (bit 30: window ambiguous)
    int32_t *ncont;                 // contenders per site; kContenders + 1: screen overflowed
    // bookkeeping
    long long *step;                // device step counter
    uint32_t *status;
    int32_t *need_rebuild;
    int32_t *list_fresh;            // 1 from a rebuild until an MD step has stored the force-list shift codes
    int32_t *gathered;              // 1 from a rebuild's gather until its end: the list build copies back
    int32_t *nbr_need;              // largest [force, reactive] count seen (overflow sizing)
    unsigned long long *counters;   // sweep counters, see Counter
    unsigned long long *life_hist;
    double *e_part;                 // per-particle energy scratch
    RepDev *reps;                   // per replica; k_sweep_begin updates t_sweep (and melting rates)
    unsigned long long *ksum;       // per replica: fixed-point sum of v^2 (2^-32 units) for the kinetic T
    // Metropolis–Hastings mode (single system)
    int32_t *mh_key, *mh_count, *mh_start, *mh_cursor, *mh_order, *mh_bsum, *mh_gate;
    int32_t *mv_type, *mv_i, *mv_j, *mv_n, *mv_b, *mv_c, *mv_cand;   // per move (active cell)
    double *mv_r;                   // kMhCand per move: separations of the candidates
    float *mv_feat, *mv_logit;      // features (12 per row) and logits of the candidate rows of all moves
    int32_t *mv_row0;               // learned proposal: first row of move m's candidates
    int32_t *mv_rows;               // learned proposal: rows reserved this sweep (compacted over live moves)
    // bond-formation event log (training data)
    float *ev_feat;                 // kMhCand x 12 per event
    int32_t *ev_n, *ev_label, *ev_count;
    int32_t ev_cap;
};

constexpr int kMhCand = 16;         // candidates per MH move or logged event
constexpr double kTwoSixth = 0x1.1f59ac3c7d6c0p+0;   // 2^(1/6), the WCA cut in units of sigma
enum BondKind { kHarmonic = 0, kFene = 1, kFeneWca = 2, kTether = 3 };

constexpr int kContenders = 4;
constexpr int kPushSlots = 64;     // push mode: pair distances kept per pushing site
constexpr int kMixedResync = 8;    // mixed mode: FP32 coordinates re-rounded from FP64 this often (power of 2)
constexpr int kCopies = 32;        // each counter is spread over this many words

enum Counter {
    cScanned = 0, cInWindow, cProposals, cEdges, cSurvivors, cFormed, cBreakTested, cBroken,
    cSweeps, cFormedTotal, cBrokenTotal, cBuilds, cNlistScanned, cNlistEntries,
    cMhFormAtt, cMhFormAcc, cMhBreakAtt, cMhBreakAcc, cEvents, cRnlistEntries, cRebuildLaunches, cNumCounters
};

// ------------------------------------------------------------ Philox-4x32-10
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = c.x, b = c.z;
        const uint32_t lo0 = 0xD2511F53u * a, hi0 = __umulhi(0xD2511F53u, a);
        const uint32_t lo1 = 0xCD9E8D57u * b, hi1 = __umulhi(0xCD9E8D57u, b);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t rx_key1(const RepDev &R, int a, uint32_t stream)
{
    return R.key1hi | ((uint32_t)(a & 0xFF) << 8) | stream;
}

// draw for the unordered pair of local tags lo < hi
__device__ __forceinline__ U4 pair_draw(const RepDev &R, int a, uint32_t stream, long long step,
                                        uint32_t lo, uint32_t hi)
{
    U4 c{(uint32_t)((unsigned long long)step & 0xFFFFFFFFull),
         (uint32_t)((unsigned long long)step >> 32), lo, hi};
    return philox10(c, R.key0, rx_key1(R, a, stream));
}

// 53-bit uniform in [0,1): (w0 << 21 | w1 >> 11) * 2^-53, exact in FP64
__device__ __forceinline__ double u53(uint32_t w0, uint32_t w1)
{
    const unsigned long long m = ((unsigned long long)w0 << 21) | (unsigned long long)(w1 >> 11);
    return __dmul_rn((double)m, 0x1.0p-53);
}

// ------------------------------------------------------------ exp
// exp(x) = 2^k e^r with k = rint(x log2 e), r reduced by two fused steps
// against ln2 split as (nearest double, remainder) — the Cody–Waite reduction
// (Cody & Waite 1980) — and e^r summed as its Taylor series through r^13 in
// Horner form with fused multiply-adds.  2^k is applied as two exact powers of
// two.  Written from the mathematics; every operation is correctly rounded
// IEEE arithmetic, so the result is reproducible on any IEEE platform.
__device__ __forceinline__ double pow2_exact(int n)
{
    return __longlong_as_double((long long)(n + 1023) << 52);
}

__device__ __forceinline__ double exp_cw(double x)
{
    if (x != x) return x;
    if (x > 709.7) return __longlong_as_double(0x7FF0000000000000ll);
    if (x < -745.2) return 0.0;
    const double log2e = 0x1.71547652b82fep+0;
    const double ln2_a = 0x1.62e42fefa39efp-1;
    const double ln2_b = 0x1.abc9e3b39803fp-56;
    const double k = rint(__dmul_rn(x, log2e));
    double r = fma(-k, ln2_a, x);
    r = fma(-k, ln2_b, r);
    // Taylor coefficients 1/m!, m = 13 .. 0
    double s = 1.0 / 6227020800.0;
    s = fma(s, r, 1.0 / 479001600.0);
    s = fma(s, r, 1.0 / 39916800.0);
    s = fma(s, r, 1.0 / 3628800.0);
    s = fma(s, r, 1.0 / 362880.0);
    s = fma(s, r, 1.0 / 40320.0);
    s = fma(s, r, 1.0 / 5040.0);
    s = fma(s, r, 1.0 / 720.0);
    s = fma(s, r, 1.0 / 120.0);
    s = fma(s, r, 1.0 / 24.0);
    s = fma(s, r, 1.0 / 6.0);
    s = fma(s, r, 0.5);
    s = fma(s, r, 1.0);
    s = fma(s, r, 1.0);
    const int ki = (int)k;
    const int h = ki / 2;
    return __dmul_rn(__dmul_rn(s, pow2_exact(h)), pow2_exact(ki - h));
}

// tanh(x) = (1 - e^{-2|x|}) / (1 + e^{-2|x|}) with the sign of x, on exp_cw:
// correctly rounded operations only, so it is reproducible bit for bit (the
// melting switch g(T) of Eq. gT at the kinetic temperature).
__device__ __forceinline__ double tanh_cw(double x)
{
    const double ax = fabs(x);
    const double e = exp_cw(__dmul_rn(-2.0, ax));
    const double t = __ddiv_rn(__dsub_rn(1.0, e), __dadd_rn(1.0, e));
    return x < 0.0 ? -t : t;
}

// ------------------------------------------------------------ log
// ln(x) for the FENE bond energy of Eq. (3): x = m 2^e with m in
// [sqrt(1/2), sqrt(2)), s = (m - 1)/(m + 1) and ln m = 2 atanh(s) summed as
// 2 (s + s^3/3 + ... + s^27/27) in Horner form with fused multiply-adds
// (|s| <= 0.172: the first dropped term is below 1e-21 of the result);
// ln x = e ln2 + ln m with ln2 split as for exp_cw.  Written from the
// mathematics with correctly rounded IEEE operations, so it is reproducible
// on any IEEE platform.  Domain: positive normal x (the caller passes
// 1 - (r/R0)^2 >= 2^-53).
__device__ __forceinline__ double log_cw(double x)
{
    const long long b = __double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7FF) - 1023;
    double m = __longlong_as_double((b & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);   // [1, 2)
    if (m > 0x1.6a09e667f3bcdp+0) {          // sqrt(2): halve m, exactly
        m = __dmul_rn(m, 0.5);
        e += 1;
    }
    const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
    const double z = __dmul_rn(s, s);
    double q = 1.0 / 27.0;
    q = fma(q, z, 1.0 / 25.0);
    q = fma(q, z, 1.0 / 23.0);
    q = fma(q, z, 1.0 / 21.0);
    q = fma(q, z, 1.0 / 19.0);
    q = fma(q, z, 1.0 / 17.0);
    q = fma(q, z, 1.0 / 15.0);
    q = fma(q, z, 1.0 / 13.0);
    q = fma(q, z, 1.0 / 11.0);
    q = fma(q, z, 1.0 / 9.0);
    q = fma(q, z, 1.0 / 7.0);
    q = fma(q, z, 1.0 / 5.0);
    q = fma(q, z, 1.0 / 3.0);
    const double t = __dmul_rn(2.0, s);
    const double lm = fma(t, __dmul_rn(z, q), t);
    const double de = (double)e;
    const double ln2_a = 0x1.62e42fefa39efp-1;
    const double ln2_b = 0x1.abc9e3b39803fp-56;
    return fma(de, ln2_a, fma(de, ln2_b, lm));
}

// ------------------------------------------------------------ geometry
// cell coordinates and type packed in the w word of pos4:
// bits 0-3 type, 4-12 cx, 13-21 cy, 22-30 cz
__device__ __forceinline__ uint32_t pack_bits(int t, int cx, int cy, int cz)
{
    return (uint32_t)t | ((uint32_t)cx << 4) | ((uint32_t)cy << 13) | ((uint32_t)cz << 22);
}
__device__ __forceinline__ int bits_type(uint32_t b) { return (int)(b & 0xF); }
__device__ __forceinline__ int bits_cx(uint32_t b) { return (int)((b >> 4) & 0x1FF); }
__device__ __forceinline__ int bits_cy(uint32_t b) { return (int)((b >> 13) & 0x1FF); }
__device__ __forceinline__ int bits_cz(uint32_t b) { return (int)((b >> 22) & 0x1FF); }

// Force-list entries: the neighbour's sorted index in the low 27 bits and,
// above them (once the first MD step after the rebuild has stored it), the
// code (sx + 1) + 3 (sy + 1) + 9 (sz + 1) of the cell shift s in {-1, 0, 1}^3
// that takes the neighbour's frozen cell next to the particle's (the minimum
// image); fixed until the next rebuild, like the cells.
constexpr int kIdxBits = 27;
constexpr uint32_t kIdxMask = (1u << kIdxBits) - 1u;
constexpr long long kMaxParticles = 1ll << kIdxBits;

// minimum-image cell offset (cells frozen between rebuilds)
__device__ __forceinline__ int cell_delta(int d, int nc)
{
    const int h = nc >> 1;
    if (d > h) d -= nc;
    else if (d < -h) d += nc;
    return d;
}

// FP64 minimum image exactly as: k = rint(d * invL); d - L * k (no contraction)
__device__ __forceinline__ double min_image(double d, double L, double invL)
{
    const double k = rint(__dmul_rn(d, invL));
    return __dsub_rn(d, __dmul_rn(L, k));
}

template <typename R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4_32a; };

__device__ __forceinline__ uint32_t w_bits(const float4 &p) { return __float_as_uint(p.w); }
__device__ __forceinline__ uint32_t w_bits(const double4_32a &p)
{
    return (uint32_t)__double_as_longlong(p.w);
}
__device__ __forceinline__ void set_w_bits(float4 &p, uint32_t b) { p.w = __uint_as_float(b); }
__device__ __forceinline__ void set_w_bits(double4_32a &p, uint32_t b)
{
    p.w = __longlong_as_double((long long)b);
}

__device__ __forceinline__ bool status_ok(const uint32_t *st) { return *(volatile const uint32_t *)st == 0u; }

// replica of particle i (no load for a single system)
__device__ __forceinline__ int rep_of(const DevParams &P, const DevArrays &A, long long i)
{
    return P.nrep > 1 ? A.rep[i] : 0;
}

// reaction processed in slot `slot` of replica rp's sweep (with one reaction
// the order is the identity and no load is needed)
__device__ __forceinline__ int rx_at(const DevParams &P, const DevArrays &A, int rp, int slot)
{
    return P.nrx == 1 ? 0 : A.rx_order[rp * kMaxRx + slot];
}

// warp-aggregated 64-bit counter increment (one atomic per full warp)
__device__ __forceinline__ void warp_count(unsigned long long *ctr, unsigned long long v)
{
    const unsigned mask = __activemask();
    if (mask == 0xFFFFFFFFu) {
        unsigned long long s = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, s);
    } else if (v) {
        atomicAdd(ctr, v);
    }
}

// Warp-level counter reduction into spread copies: every lane of the warp
// must call this (lanes without work pass zeros).  One atomic per warp and
// counter, spread over kCopies words so that no single address serialises;
// the host sums the copies.  No block barrier, so slow warps stall nobody.
template <int N>
__device__ __forceinline__ void warp_counts(unsigned long long *ctr, const int (&idx)[N],
                                            const unsigned long long (&v)[N])
{
    const int lane = threadIdx.x & 31;
    const unsigned gw = (unsigned)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        unsigned long long x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        if (lane == 0 && x) atomicAdd(&ctr[idx[k] * kCopies + (gw & (kCopies - 1))], x);
    }
}

__device__ __forceinline__ void counter_reset(unsigned long long *ctr, int c)
{
    for (int k = 0; k < kCopies; ++k) ctr[c * kCopies + k] = 0ull;
}

__device__ __forceinline__ void counter_add1(unsigned long long *ctr, int c, unsigned long long v)
{
    ctr[c * kCopies] += v;
}

// Warp-aggregated append of flagged items to a global list: every lane of the
// warp must call this; returns the slot of this lane's item (or -1).  One
// atomic per warp with work and no block barrier.
__device__ __forceinline__ int warp_append(bool want, int32_t *count)
{
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, want);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    return want ? base + __popc(m & ((1u << lane) - 1u)) : -1;
}

// Block-aggregated append of flagged items to a global list: every thread of
// the block must call this; returns the slot of this thread's item (or -1).
__device__ __forceinline__ int block_append(bool want, int32_t *count)
{
    __shared__ int s_base, s_cnt;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const unsigned m = __ballot_sync(0xFFFFFFFFu, want);
    int wbase = 0;
    if (lane == 0 && m) wbase = atomicAdd(&s_cnt, __popc(m));
    wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
    __syncthreads();
    if (threadIdx.x == 0) s_base = s_cnt ? atomicAdd(count, s_cnt) : 0;
    __syncthreads();
    return want ? s_base + wbase + __popc(m & ((1u << lane) - 1u)) : -1;
}

}  // namespace snap
