// Bit-reproducible kernels: the bond sweep and the Langevin integrator.
//
// Compiled with -fmad=false and written with explicit round-to-nearest
// intrinsics, so every FP64 operation is a single IEEE rounding in a fixed
// order.  Given identical positions, the sweep therefore takes exactly the
// decisions its definition implies, on any device and any block size.
//
// The sweep follows Sec. II.C of the DyBond-v2 paper (Fig. 1), one kernel per
// phase and per reaction in a random order redrawn every sweep:
//   propose  — every free reactive site scans its reactive neighbour list and
//              keeps the free, type-compatible partner in [r_min, r_max]
//              closest to the rest length (ties to the smaller tag); in mixed
//              mode an FP32 screen keeps the few candidates that may win and
//              k_exact decides among them in FP64;
//   match    — (in k_exact) each proposal edge gets a Philox priority;
//              atomicMax of (priority << 32 | other tag) at both endpoints;
//   accept   — an edge survives iff it holds the maximum at both ends (a
//              locally dominant matching, disjoint by construction, replacing
//              the paper's compare-and-swap race with a scheduling-independent
//              rule) and forms with probability P_on^0 exp(-U_b(r)/kT), Eq. 3;
//   break    — (same kernel as accept) every bond of this reaction present
//              before the reaction began breaks with probability P_off;
//   apply    — per particle, broken slots are removed and the formed partner
//              inserted; occupancies change before the next reaction reads them.
#include <algorithm>

#include "snap_kernels.h"
#include "apply.cuh"

namespace snap {

namespace {

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }

template <bool FORCED>
__device__ __forceinline__ bool sweep_active(const DevParams &P, const DevArrays &A, long long &step)
{
    if (!status_ok(A.status)) return false;
    step = *A.step;
    if (!FORCED && (step % P.period) != 0) return false;
    return true;
}

// grid-stride kernels over the compacted site list use this many blocks
constexpr int kListBlocks = 296;
constexpr int kSweepBeginBlock = 256;

// Sweep start: counters reset, the reaction order per replica
// (Fisher–Yates driven by Philox(ORDER) with counter (step, k), so competing
// reactions are treated evenhandedly), the availability byte of every
// particle (its type while it has a free valence slot, else 0xFF) with the
// count per type.  Each thread takes kBeginItems particles of its block's
// tile, their loads issued together, so that the grid is one wave of resident
// blocks instead of several waves of one dependent load chain each.  The
// per-reaction scratch (best, fpart, brk, prop, the push keys) starts clear
// and k_apply clears it after each reaction: a sweep either runs to its end
// or (a latched status) none of its kernels act.
constexpr int kBeginItems = 4;

template <bool FORCED>
__global__ void __launch_bounds__(kSweepBeginBlock) k_sweep_begin(DevParams P, DevArrays A)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const long long r = gtid();
    if (r == 0) {
        for (int c = cScanned; c <= cBroken; ++c) counter_reset(A.counters, c);
        counter_reset(A.counters, cNlistScanned);
        counter_add1(A.counters, cSweeps, 1ull);
        *A.list_count = 0;
    }
    const long long base = (long long)blockIdx.x * (kSweepBeginBlock * kBeginItems) + threadIdx.x;
    int ty[kBeginItems], oc[kBeginItems], av[kBeginItems];
#pragma unroll
    for (int u = 0; u < kBeginItems; ++u) {
        const long long q = base + u * kSweepBeginBlock;
        ty[u] = q < P.n ? A.type[q] : -1;
        oc[u] = q < P.n ? A.occ[q] : 0;
    }
#pragma unroll
    for (int u = 0; u < kBeginItems; ++u) {
        const long long q = base + u * kSweepBeginBlock;
        av[u] = (ty[u] >= 0 && oc[u] < P.valence[ty[u]]) ? ty[u] : -1;
        if (q < P.n) A.avail[q] = av[u] >= 0 ? (uint8_t)av[u] : (uint8_t)0xFF;
    }
    // per-type counts and (single system, single reaction: the only case push
    // mode serves) compacted lists; one global atomic per block and type
    const bool lists = P.nrep == 1 && P.nrx == 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ int s_cnt[kMaxTypes], s_base[kMaxTypes], s_woff[kBeginItems][kSweepBeginBlock / 32][kMaxTypes];
    if (threadIdx.x < kMaxTypes) s_cnt[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kBeginItems; ++u)
        for (int t = 0; t < P.ntypes; ++t) {
            const unsigned m = __ballot_sync(0xFFFFFFFFu, av[u] == t);
            if (lane == 0) s_woff[u][wid][t] = m ? atomicAdd(&s_cnt[t], __popc(m)) : 0;
        }
    __syncthreads();
    if (threadIdx.x < P.ntypes) {
        const int t = threadIdx.x;
        s_base[t] = s_cnt[t] ? atomicAdd(&A.avail_count[t], s_cnt[t]) : 0;
    }
    __syncthreads();
    if (lists) {
#pragma unroll
        for (int u = 0; u < kBeginItems; ++u)
            for (int t = 0; t < P.ntypes; ++t) {
                const unsigned m = __ballot_sync(0xFFFFFFFFu, av[u] == t);
                if (av[u] == t)
                    A.avail_list[(long long)t * P.n + s_base[t] + s_woff[u][wid][t] + __popc(m & ((1u << lane) - 1u))] =
                        (int)(base + u * kSweepBeginBlock);
            }
    }
    if (r >= P.nrep) return;
    RepDev &R = A.reps[r];
    // the temperature of this sweep (Sec. II.B): the set-point, or the kinetic
    // temperature from the fixed-point sum k_kin_sum left, with the melting
    // switch re-evaluated at it
    double T = R.kT;
    if (P.kinetic_T) {
        const unsigned long long q = A.ksum[r];
        A.ksum[r] = 0ull;
        T = __ddiv_rn(__dmul_rn(__ll2double_rn((long long)q), 0x1.0p-32), (double)(3 * R.n));
        for (int a = 0; a < P.nrx; ++a) {
            if (!((P.melt_mask >> a) & 1)) continue;
            const double g = __dmul_rn(0.5, __dadd_rn(tanh_cw(__dmul_rn(P.melt_lambda[a], __dsub_rn(T, P.melt_t[a]))),
                                                      1.0));
            const double kon = __dadd_rn(__dmul_rn(P.kon_init[a], __dsub_rn(1.0, g)), __dmul_rn(P.kon_melt[a], g));
            const double koff = __dadd_rn(__dmul_rn(P.koff_init[a], __dsub_rn(1.0, g)), __dmul_rn(P.koff_melt[a], g));
            double pon = __dmul_rn(kon, P.period_dt), poff = __dmul_rn(koff, P.period_dt);
            pon = pon < 1.0 ? pon : 1.0;
            poff = poff < 1.0 ? poff : 1.0;
            R.p_on0[a] = pon;
            R.p_off[a] = poff;
            R.off_thresh[a] = (unsigned long long)ceil(__dmul_rn(poff, 0x1.0p53));
        }
    }
    R.t_sweep = T;
    int ord[kMaxRx];
    for (int a = 0; a < P.nrx; ++a) ord[a] = a;
    for (int k = P.nrx - 1; k >= 1; --k) {
        const U4 w = pair_draw(R, 0, kOrder, step, (uint32_t)k, 0u);
        const int j = (int)(((unsigned long long)w.x * (unsigned long long)(k + 1)) >> 32);
        const int t = ord[k];
        ord[k] = ord[j];
        ord[j] = t;
    }
    for (int a = 0; a < kMaxRx; ++a) A.rx_order[r * kMaxRx + a] = a < P.nrx ? ord[a] : 0;
}

// Kinetic temperature of the half-step velocities (Sec. II.B), summed
// deterministically: each particle's v^2 = (vx^2 + vy^2) + vz^2 in FP64 is
// rounded to the nearest multiple of 2^-32 and the integers are added exactly
// (64-bit integer atomics: any order gives the same sum).  k_sweep_begin turns
// the sum into T = sum 2^-32 / (3 n) and clears it.
template <bool FORCED>
__global__ void k_kin_sum(DevParams P, DevArrays A)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const long long i = gtid();
    unsigned long long q = 0ull;
    int rp = 0;
    if (i < P.n) {
        rp = rep_of(P, A, i);
        double vx, vy, vz;
        if (P.screen) {
            const float4 v = A.v4[i];
            vx = v.x; vy = v.y; vz = v.z;
        } else {
            vx = A.vx[i]; vy = A.vy[i]; vz = A.vz[i];
        }
        const double v2 = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
        q = (unsigned long long)__double2ll_rn(__dmul_rn(v2, 0x1.0p32));
    }
    // one atomic per warp when the warp holds one replica, else per lane
    const int rp0 = __shfl_sync(0xFFFFFFFFu, rp, 0);
    if (__all_sync(0xFFFFFFFFu, rp == rp0)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xFFFFFFFFu, q, o);
        if ((threadIdx.x & 31) == 0 && q) atomicAdd(&A.ksum[rp0], q);
    } else if (q) {
        atomicAdd(&A.ksum[rp], q);
    }
}

// exact FP64 squared separation, as the definition states it:
// d = x_j - x_i; d -= L rint(d / L) per axis; r^2 = (dx^2 + dy^2) + dz^2
__device__ __forceinline__ double exact_r2(const DevArrays &A, const RepDev &R, int i, int j)
{
    const double dx = min_image(__dsub_rn(A.x[j], A.x[i]), R.L[0], R.invL[0]);
    const double dy = min_image(__dsub_rn(A.y[j], A.y[i]), R.L[1], R.invL[1]);
    const double dz = min_image(__dsub_rn(A.z[j], A.z[i]), R.L[2], R.invL[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// The same value with the minimum image skipped on axes where it is the
// identity: when the two frozen cells (bits of pos4.w) are neighbours without
// wrapping and there are at least 6 cells, |d| < 2 w + skin < L / 2, so
// rint(d / L) = 0 and d - L * 0 = d exactly.  Valid only while positions stay
// unwrapped between rebuilds (mixed mode); FP64 mode wraps them every step,
// so a particle that crossed a face since the rebuild sits a box edge away
// from its frozen cell and needs the full minimum image.
__device__ __forceinline__ double exact_r2_cells(const DevArrays &A, const RepDev &R, int i, int j, uint32_t bi,
                                                 uint32_t bj)
{
    double dx = __dsub_rn(A.x[j], A.x[i]);
    double dy = __dsub_rn(A.y[j], A.y[i]);
    double dz = __dsub_rn(A.z[j], A.z[i]);
    if (!(R.nc[0] >= 6 && abs(bits_cx(bj) - bits_cx(bi)) <= 1)) dx = min_image(dx, R.L[0], R.invL[0]);
    if (!(R.nc[1] >= 6 && abs(bits_cy(bj) - bits_cy(bi)) <= 1)) dy = min_image(dy, R.L[1], R.invL[1]);
    if (!(R.nc[2] >= 6 && abs(bits_cz(bj) - bits_cz(bi)) <= 1)) dz = min_image(dz, R.L[2], R.invL[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// w bits (type, frozen cell) of particle i from pos4 in either precision
__device__ __forceinline__ uint32_t cell_bits(const DevParams &P, const DevArrays &A, int i)
{
    return P.screen ? w_bits(reinterpret_cast<const float4 *>(A.pos4)[i])
                    : w_bits(reinterpret_cast<const double4_32a *>(A.pos4)[i]);
}

// keep the candidate minimising |r - r0|, ties to the smaller tag
__device__ __forceinline__ void consider(double d, double r, int j, int tgj, int &best, int &best_tag,
                                         double &best_d, double &best_r)
{
    if (best < 0 || d < best_d || (d == best_d && tgj < best_tag)) {
        best = j;
        best_tag = tgj;
        best_d = d;
        best_r = r;
    }
}

// Conservative single-precision screen for the exact FP64 proposal test.
// The cell-relative FP32 coordinates (|rel| < 4) are within 2e-6 of the FP64
// ones (rounded from them at most kMixedResync = 8 steps ago, advanced by FP32
// steps since), so the FP32 separation of a listed pair is within 4.2e-6 per
// component (7.3e-6 in length), r^2 within 3e-5 (r < 2) and |r - r0| within
// 1e-5 when r^2 >= 0.09.  With margins of 1e-4 a candidate is
// dropped in FP32 only when the exact test would reject it or when another
// candidate surely beats it; every candidate that may win is re-evaluated in
// FP64 by k_exact, in dense warps.
constexpr float kScreenR2 = 1e-4f;
constexpr float kScreenD = 1e-4f;

// Push mode.  When one side of a reaction has far fewer available particles
// than the other (a saturated gel: almost every colloid slot is taken), the
// scarce side's sites both make their own proposals and push themselves, as
// candidates, to their available partners on the abundant side; each of
// those picks the smallest |r - r0| among what it received (ties to the
// smaller tag) — exactly the proposal a scan of its own list would make, for
// a small fraction of the neighbour visits.  The pushing sites come from the
// compacted per-type list of k_sweep_begin, so their FP64 work runs in dense
// warps.  Single system with a single reaction (the lists and counts are per
// type and are not updated between reactions).
constexpr int kPushRatio = 4;

// the pushing type of reaction slot `slot`, or -1 for the plain (pull) scan
__device__ __forceinline__ int push_type(const DevParams &P, const DevArrays &A, int slot)
{
    if (P.nrep != 1 || P.nrx != 1) return -1;
    const int a = rx_at(P, A, 0, slot);
    const int ta = P.rx_ta[a], tb = P.rx_tb[a];
    if (ta == tb) return -1;
    const long long ca = A.avail_count[ta], cb = A.avail_count[tb];
    if (ca * kPushRatio <= cb) return ta;
    if (cb * kPushRatio <= ca) return tb;
    return -1;
}

// Partners of site i that may be proposed: available with the partner type
// (one byte load), not already bonded to i (sorted indices of i's partners)
// and, when the reaction excludes intramolecular bonds (Sec. II.D), not of
// i's molecule (mol >= 0 only then).
struct SiteFilter {
    uint8_t pt;
    int b0, b1, b2, b3;
    int mol;
    __device__ __forceinline__ bool ok(const DevArrays &A, int j) const
    {
        return A.avail[j] == pt && j != b0 && j != b1 && j != b2 && j != b3 && (mol < 0 || A.mol[A.tag[j]] != mol);
    }
};

__device__ __forceinline__ SiteFilter site_filter(const DevParams &P, const DevArrays &A, int a, int ti, int ta,
                                                  int tb, int i)
{
    const int4 dp = A.dp[i];
    SiteFilter f;
    f.pt = (uint8_t)(ti == ta ? tb : ta);
    f.mol = P.rx_self[a] ? A.mol[A.tag[i]] : -1;
    f.b0 = dp.x >= 0 ? A.rtag[dp.x] : -1;
    f.b1 = dp.y >= 0 ? A.rtag[dp.y] : -1;
    f.b2 = dp.z >= 0 ? A.rtag[dp.z] : -1;
    f.b3 = dp.w >= 0 ? A.rtag[dp.w] : -1;
    return f;
}

// FP32 separation squared from cell-relative coordinates and frozen cells
__device__ __forceinline__ float screen_r2(const float4 &pi4, const float4 &pj4, const RepDev &R)
{
    const uint32_t bi = w_bits(pi4), bj = w_bits(pj4);
    const float ex = (pj4.x - pi4.x) + (float)cell_delta(bits_cx(bj) - bits_cx(bi), R.nc[0]) * R.wf[0];
    const float ey = (pj4.y - pi4.y) + (float)cell_delta(bits_cy(bj) - bits_cy(bi), R.nc[1]) * R.wf[1];
    const float ez = (pj4.z - pi4.z) + (float)cell_delta(bits_cz(bj) - bits_cz(bi), R.nc[2]) * R.wf[2];
    return ex * ex + ey * ey + ez * ez;
}

// Proposal phase over the reactive list.  FP64 mode decides each site here.
// Mixed mode screens in FP32: a first pass finds the smallest sure upper
// bound of |r - r0| among candidates surely inside the window, a second pass
// keeps (in list order, at most kContenders) every candidate that may still
// win — window-ambiguous, too close for the bound, or within the margin of
// that bound — for k_exact to decide in FP64.
template <bool SCREEN>
__device__ __forceinline__ void pull_propose(const DevParams &P, DevArrays &A, int slot)
{
    unsigned long long scanned = 0, inwin = 0, nscan = 0, nprop = 0;
    // grid-stride with a warp-uniform trip count (a small grid exits cheaply in push mode)
    for (long long base = (long long)blockIdx.x * blockDim.x; base < P.n; base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    bool want = false;
    if (i < P.n) {
        int best = -1, ncont = 0;
        double best_d = 0.0;
        const int rp = rep_of(P, A, i);
        const int a = rx_at(P, A, rp, slot);
        const int ti = A.type[i];
        const int ta = P.rx_ta[a], tb = P.rx_tb[a];
        if ((ti == ta || ti == tb) && A.occ[i] < P.valence[ti]) {
            const RepDev &R = A.reps[rp];
            const SiteFilter flt = site_filter(P, A, a, ti, ta, tb, (int)i);
            const int nn = A.rnn[i];
            const int *nb = A.rnbr + i;
            const long long stride = P.nbr_stride;
            nscan += (unsigned long long)nn;
            if (SCREEN) {
                const float4 *pos4 = reinterpret_cast<const float4 *>(A.pos4);
                const float4 pi4 = pos4[i];
                const float rmin2f = (float)P.rx_rmin2[a], rmax2f = (float)P.rx_rmax2[a];
                const float r0f = (float)P.rx_r0[a];
                float min_upper = 3.0e38f;
                unsigned long long sure_in = 0;
                for (int k = 0; k < nn; ++k) {
                    const int j = __ldg(nb + (long long)k * stride);
                    if (!flt.ok(A, j)) continue;
                    ++scanned;
                    const float r2f = screen_r2(pi4, pos4[j], R);
                    if (r2f < rmin2f - kScreenR2 || r2f > rmax2f + kScreenR2) continue;  // surely outside
                    if (r2f > rmin2f + kScreenR2 && r2f < rmax2f - kScreenR2) {          // surely inside
                        ++sure_in;
                        if (r2f >= 0.09f) min_upper = fminf(min_upper, fabsf(sqrtf(r2f) - r0f) + kScreenD);
                    }
                }
                if (scanned > 0) {
                    for (int k = 0; k < nn; ++k) {
                        const int j = __ldg(nb + (long long)k * stride);
                        if (!flt.ok(A, j)) continue;
                        const float r2f = screen_r2(pi4, pos4[j], R);
                        if (r2f < rmin2f - kScreenR2 || r2f > rmax2f + kScreenR2) continue;
                        const bool amb = !(r2f > rmin2f + kScreenR2 && r2f < rmax2f - kScreenR2);
                        if (!amb && r2f >= 0.09f && fabsf(sqrtf(r2f) - r0f) - kScreenD > min_upper) continue;
                        if (ncont < kContenders) A.cont[i * kContenders + ncont] = j | (amb ? (1 << 30) : 0);
                        ++ncont;
                    }
                }
                if (ncont > kContenders) ncont = kContenders + 1;   // k_exact rescans this site in full
                else inwin += sure_in;
                want = ncont > 0;
            } else {
                const double rmin2 = P.rx_rmin2[a], rmax2 = P.rx_rmax2[a];
                const double r0 = P.rx_r0[a];
                int best_tag = 0;
                double best_r = 0.0;
                for (int k = 0; k < nn; ++k) {
                    const int j = __ldg(nb + (long long)k * stride);
                    if (!flt.ok(A, j)) continue;
                    ++scanned;
                    const double r2 = exact_r2(A, R, (int)i, j);
                    if (r2 < rmin2 || r2 > rmax2) continue;
                    ++inwin;
                    const double r = __dsqrt_rn(r2);
                    consider(fabs(__dsub_rn(r, r0)), r, j, A.tag[j], best, best_tag, best_d, best_r);
                }
                nprop += best >= 0 ? 1ull : 0ull;
                want = best >= 0;
            }
        }
        A.prop[i] = best;
        A.prop_d[i] = best_d;
        A.ncont[i] = ncont;
    }
    const int sl = warp_append(want, A.list_count);
    if (sl >= 0) A.site_list[sl] = (int)i;
    }
    const int idx[4] = {cNlistScanned, cScanned, cInWindow, cProposals};
    const unsigned long long v[4] = {nscan, scanned, inwin, nprop};
    warp_counts<4>(A.counters, idx, v);
}

// Matching: the edge i -> j gets priority w = first word of Philox(MATCH;
// min tag, max tag); atomicMax of (w << 32 | other tag) at both endpoints.
__device__ __forceinline__ void match_edge(DevArrays &A, const RepDev &R, int a, long long step, int i, int j)
{
    if (j < 0) return;
    const uint32_t ti = (uint32_t)(A.tag[i] - R.tag_off), tj = (uint32_t)(A.tag[j] - R.tag_off);
    const uint32_t lo = ti < tj ? ti : tj, hi = ti < tj ? tj : ti;
    const U4 w = pair_draw(R, a, kMatch, step, lo, hi);
    A.prio[i] = w.x;
    const unsigned long long pr = (unsigned long long)w.x << 32;
    atomicMax(&A.best[i], pr | tj);
    atomicMax(&A.best[j], pr | ti);
}

// Exact FP64 evaluation of the screened contenders, one listed site per
// thread, then the matching priority of the site's proposal edge.
__device__ __forceinline__ void pull_exact(const DevParams &P, DevArrays &A, int slot, long long step)
{
    const int nlist = *A.list_count;
    unsigned long long inwin = 0, nprop = 0;
    for (long long q = gtid(); q < nlist; q += (long long)gridDim.x * blockDim.x) {
        const int i = A.site_list[q];
        const int nc = A.ncont[i];
        const int rp = rep_of(P, A, i);
        const int a = rx_at(P, A, rp, slot);
        const RepDev &R = A.reps[rp];
        if (nc == 0) {
            // FP64 mode: the proposal was decided in k_propose
            match_edge(A, R, a, step, i, A.prop[i]);
            continue;
        }
        const double rmin2 = P.rx_rmin2[a], rmax2 = P.rx_rmax2[a];
        const double r0 = P.rx_r0[a];
        int best = -1, best_tag = 0;
        double best_d = 0.0, best_r = 0.0;
        if (nc <= kContenders) {
            for (int c = 0; c < nc; ++c) {
                const int e = A.cont[i * kContenders + c];
                const int j = e & 0x3FFFFFFF;
                const double r2 = exact_r2(A, R, i, j);
                if (r2 < rmin2 || r2 > rmax2) continue;
                if (e >> 30) ++inwin;
                const double r = __dsqrt_rn(r2);
                consider(fabs(__dsub_rn(r, r0)), r, j, A.tag[j], best, best_tag, best_d, best_r);
            }
        } else {
            // screen overflow: the plain exact scan
            const SiteFilter flt = site_filter(P, A, a, A.type[i], P.rx_ta[a], P.rx_tb[a], i);
            const int nn = A.rnn[i];
            for (int k = 0; k < nn; ++k) {
                const int j = A.rnbr[(long long)k * P.nbr_stride + i];
                if (!flt.ok(A, j)) continue;
                const double r2 = exact_r2(A, R, i, j);
                if (r2 < rmin2 || r2 > rmax2) continue;
                ++inwin;
                const double r = __dsqrt_rn(r2);
                consider(fabs(__dsub_rn(r, r0)), r, j, A.tag[j], best, best_tag, best_d, best_r);
            }
        }
        A.prop[i] = best;
        A.prop_d[i] = best_d;
        if (best >= 0) ++nprop;
        match_edge(A, R, a, step, i, best);
    }
    const int idx[2] = {cInWindow, cProposals};
    const unsigned long long v[2] = {inwin, nprop};
    warp_counts<2>(A.counters, idx, v);
}

// (d, tag) keys: d = |r - r0| as FP64 bits (non-negative doubles order like
// their bit patterns), ties to the smaller tag; lexicographic order
__device__ __forceinline__ bool key_less(unsigned long long d, unsigned long long t, unsigned long long d2,
                                        unsigned long long t2)
{
    return d < d2 || (d == d2 && t < t2);
}

// (d, tag) minimum over the warp
__device__ __forceinline__ void warp_min_key(unsigned long long &d, unsigned long long &t)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long d2 = __shfl_xor_sync(0xFFFFFFFFu, d, o);
        const unsigned long long t2 = __shfl_xor_sync(0xFFFFFFFFu, t, o);
        if (key_less(d2, t2, d, t)) {
            d = d2;
            t = t2;
        }
    }
}

// 16-byte compare-and-swap on global memory; returns the previous value
__device__ __forceinline__ ulonglong2 cas128(ulonglong2 *p, ulonglong2 cmp, ulonglong2 val)
{
    ulonglong2 old;
    asm volatile(
        "{\n\t.reg .b128 c, v, d;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 v, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], c, v;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(old.x), "=l"(old.y)
        : "l"(cmp.x), "l"(cmp.y), "l"(val.x), "l"(val.y), "l"(p)
        : "memory");
    return old;
}

// Lowers *p to (d, t) if smaller.  Lock-free: a failed exchange means another
// pusher lowered the key; the retries are bounded by the pushers of one site
// (the cap, 2^16 unless snap_set_retry_limit lowers it, only guards against a
// defect, and latches a status bit).
__device__ __forceinline__ void atomic_min_key(const DevParams &P, const DevArrays &A, int j, unsigned long long d,
                                               unsigned long long t, int cap)
{
    ulonglong2 *p = &A.pkey[j];
    ulonglong2 cur = *p;
    for (int it = 0; it < cap; ++it) {
        if (!key_less(d, t, cur.x, cur.y)) return;
        const ulonglong2 old = cas128(p, cur, make_ulonglong2(d, t));
        if (old.x == cur.x && old.y == cur.y) return;
        cur = old;
    }
    atomicOr(A.status, (uint32_t)kStTimeout);
}

// Push mode, pass 1: one warp per pushing site (from the compacted list),
// its lanes over the site's reactive list.  Every in-window pair lowers the
// candidate's (d, tag) key by a 16-byte atomic; the pushing site's own
// proposal is the warp minimum, made here with its matching priority.  The
// pair distances are kept for pass 2.
__device__ __forceinline__ void push_pass1(const DevParams &P, DevArrays &A, int slot, long long step, int s)
{
    const int a = rx_at(P, A, 0, slot);
    const int ta = P.rx_ta[a], tb = P.rx_tb[a];
    const RepDev &R = A.reps[0];
    const double rmin2 = P.rx_rmin2[a], rmax2 = P.rx_rmax2[a];
    const double r0 = P.rx_r0[a];
    const long long stride = P.nbr_stride;
    const int lane = threadIdx.x & 31;
    unsigned long long scanned = 0, inwin = 0, nscan = 0, nprop = 0;
    const int ns = A.avail_count[s];
    const int32_t *list = A.avail_list + (long long)s * P.n;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const float rmin2f = (float)rmin2, rmax2f = (float)rmax2;
    const float4 *pos4 = reinterpret_cast<const float4 *>(A.pos4);
    for (long long q = gtid() >> 5; q < ns; q += warps) {
        const int i = list[q];
        const SiteFilter flt = site_filter(P, A, a, s, ta, tb, i);
        const int nn = A.rnn[i];
        if (lane == 0) nscan += (unsigned long long)nn;
        const uint32_t bi = cell_bits(P, A, i);
        const float4 pi4 = P.screen ? pos4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const unsigned long long me = (unsigned long long)(uint32_t)A.tag[i];
        unsigned long long bd = ~0ull, bt = ~0ull;     // this site's best (d, partner tag)
        for (int k = lane; k < nn; k += 32) {
            const int j = __ldg(A.rnbr + (long long)k * stride + i);
            unsigned long long d = ~0ull;                // not a candidate
            if (flt.ok(A, j)) {
                scanned += 2;                            // the pair, as both of its sites see it
                bool maybe = true;
                uint32_t bj;
                if (P.screen) {                          // mixed mode: FP32 pre-screen of the window
                    const float4 pj4 = pos4[j];
                    bj = w_bits(pj4);
                    const float r2f = screen_r2(pi4, pj4, R);
                    maybe = !(r2f < rmin2f - kScreenR2 || r2f > rmax2f + kScreenR2);
                } else {
                    bj = 0u;                             // FP64 mode: full minimum image, cells unused
                }
                const double r2 = !maybe ? -1.0
                                  : P.screen ? exact_r2_cells(A, R, i, j, bi, bj) : exact_r2(A, R, i, j);
                if (maybe && r2 >= rmin2 && r2 <= rmax2) {
                    inwin += 2;
                    d = (unsigned long long)__double_as_longlong(fabs(__dsub_rn(__dsqrt_rn(r2), r0)));
                    atomic_min_key(P, A, j, d, me, P.cas_cap);
                    const unsigned long long tj = (unsigned long long)(uint32_t)A.tag[j];
                    if (key_less(d, tj, bd, bt)) {
                        bd = d;
                        bt = tj;
                    }
                }
            }
            if (q < P.pdist_rows && k < kPushSlots) A.pdist[q * kPushSlots + k] = d;
        }
        warp_min_key(bd, bt);
        if (lane == 0 && bd != ~0ull) {
            const int c = A.rtag[(uint32_t)bt];
            A.prop[i] = c;
            A.prop_d[i] = __longlong_as_double((long long)bd);
            match_edge(A, R, a, step, i, c);
            ++nprop;
        }
    }
    const int idx[5] = {cNlistScanned, cScanned, cInWindow, cProposals, cEdges};
    const unsigned long long v[5] = {nscan, scanned, inwin, nprop, nprop};
    warp_counts<5>(A.counters, idx, v);
}

// Push mode, pass 2 (same mapping): the winning pusher of each candidate (its
// (d, tag) is the candidate's key) sets the candidate's proposal and matching
// priority.  The edge is new unless the pushing site proposed it too.  The
// keys are cleared by k_apply.
__device__ __forceinline__ void push_pass2(const DevParams &P, DevArrays &A, int slot, long long step, int s)
{
    const int a = rx_at(P, A, 0, slot);
    const int ta = P.rx_ta[a], tb = P.rx_tb[a];
    const RepDev &R = A.reps[0];
    const double rmin2 = P.rx_rmin2[a], rmax2 = P.rx_rmax2[a];
    const double r0 = P.rx_r0[a];
    const long long stride = P.nbr_stride;
    const int lane = threadIdx.x & 31;
    const int ns = A.avail_count[s];
    const int32_t *list = A.avail_list + (long long)s * P.n;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    unsigned long long nprop = 0, nedge = 0;
    for (long long q = gtid() >> 5; q < ns; q += warps) {
        const int i = list[q];
        if (A.prop[i] < 0) continue;                     // warp-uniform: no candidate in window
        const SiteFilter flt = site_filter(P, A, a, s, ta, tb, i);
        const int nn = A.rnn[i];
        const unsigned long long me = (unsigned long long)(uint32_t)A.tag[i];
        const int pi = A.prop[i];
        for (int k = lane; k < nn; k += 32) {
            const int j = __ldg(A.rnbr + (long long)k * stride + i);
            unsigned long long d;
            if (q < P.pdist_rows && k < kPushSlots) {
                d = A.pdist[q * kPushSlots + k];
                if (d == ~0ull) continue;
            } else {
                if (!flt.ok(A, j)) continue;
                const double r2 = exact_r2(A, R, i, j);
                if (r2 < rmin2 || r2 > rmax2) continue;
                d = (unsigned long long)__double_as_longlong(fabs(__dsub_rn(__dsqrt_rn(r2), r0)));
            }
            const ulonglong2 kj = A.pkey[j];
            if (kj.x != d || kj.y != me) continue;
            A.prop[j] = i;
            A.prop_d[j] = __longlong_as_double((long long)d);
            match_edge(A, R, a, step, j, i);
            ++nprop;
            if (pi != j) ++nedge;
        }
    }
    const int idx[2] = {cProposals, cEdges};
    const unsigned long long v[2] = {nprop, nedge};
    warp_counts<2>(A.counters, idx, v);
}

// Slip bond, Eq. (slip): P_off(r) = P_off^0 exp(a sqrt(U_b(r)/kT)), capped at 1.
// At kT = 0 the factor takes its limits (1 for U_b = 0, infinite for U_b > 0);
// an exponent of 700 or more caps at once.  Every operation is one IEEE
// rounding; exp is this library's own (the acceptance factor's).
__device__ __forceinline__ double slip_p_off(double p0, double k, double r0, double kT, double a, double r)
{
    if (p0 == 0.0) return p0;
    const double dr = __dsub_rn(r, r0);
    const double U = __dmul_rn(__dmul_rn(__dmul_rn(0.5, k), dr), dr);
    double x;
    if (kT > 0.0) x = __ddiv_rn(U, kT);
    else x = U > 0.0 ? __longlong_as_double(0x7FF0000000000000ll) : 0.0;
    const double e = __dmul_rn(a, __dsqrt_rn(x));
    if (!(e < 700.0)) return 1.0;
    const double p = __dmul_rn(p0, exp_cw(e));
    return p < 1.0 ? p : 1.0;
}

// Breaking (Fig. 1d) of particle i's bonds of the reaction in slot `slot`:
// each bond present when the reaction began, owned by its smaller tag,
// breaks iff Philox(BREAK; tags) gives u53 < P_off.  Reads the slots as they
// were before the reaction; writes only the break bits, which k_apply reads.
// SLIP: the draws of slip reactions (Eq. slip), which run in a kernel of
// their own (k_break_slip) so that the proposal kernel, which hosts the
// constant-P_off draws, keeps its registers; each kind skips the other's.
// (dp, me, drx: the particle's slots, tag and packed reactions, loaded by the
// caller so that several particles' loads can be in flight together.)
template <bool SLIP>
__device__ __forceinline__ void break_particle(const DevParams &P, DevArrays &A, int slot, long long step, long long i,
                                               const int4 dp, const int me, const int drx,
                                               unsigned long long &tested)
{
    if (dp.x < 0) return;
    const int rp = rep_of(P, A, i);
    const int a = rx_at(P, A, rp, slot);
    if ((((P.slip_mask >> a) & 1) != 0) != SLIP) return;
    const RepDev &R = A.reps[rp];
    const int pv[4] = {dp.x, dp.y, dp.z, dp.w};
#pragma unroll
    for (int s = 0; s < kVmax; ++s) {
        const int p = pv[s];
        if (p < 0 || p < me) continue;           // the smaller tag owns the bond
        if (((drx >> (8 * s)) & 0xFF) != a) continue;
        ++tested;
        const U4 w = pair_draw(R, a, kBreak, step, (uint32_t)(me - R.tag_off), (uint32_t)(p - R.tag_off));
        // u53 < p_off  <=>  m < ceil(p_off 2^53) with m the 53-bit integer of u53;
        // with the slip modifier P_off depends on r and m < p_off 2^53 is tested in
        // FP64 (both sides exact)
        const unsigned long long m = ((unsigned long long)w.x << 21) | (unsigned long long)(w.y >> 11);
        int j = -1;
        bool brk;
        if (SLIP) {
            j = A.rtag[p];
            const int bt = P.rx_bt[a];
            const double pr = slip_p_off(R.p_off[a], P.bk[bt], P.br0[bt], R.t_sweep, P.rx_slip[a],
                                         __dsqrt_rn(exact_r2(A, R, (int)i, j)));
            brk = (double)m < __dmul_rn(pr, 0x1p53);
        } else {
            brk = m < R.off_thresh[a];
        }
        if (brk) {
            if (!SLIP) j = A.rtag[p];     // the partner's index only for a bond that breaks
            atomicOr(&A.brk[i], 1u << s);
            const int4 q = A.dp[j];
            const int qv[4] = {q.x, q.y, q.z, q.w};
            int sj = 0;
#pragma unroll
            for (int t = 0; t < kVmax; ++t)
                if (qv[t] == me) sj = t;
            atomicOr(&A.brk[j], 1u << sj);
        }
    }
}

// The breaking draws over all particles, grid-stride, kBreakItems particles
// per thread and pass: the slot words of all of them are loaded first, then
// the tags and reactions of the bonded ones, then the draws.
constexpr int kBreakItems = 4;

template <bool SLIP>
__device__ __forceinline__ void break_pass(const DevParams &P, DevArrays &A, int slot, long long step,
                                           unsigned long long &tested)
{
    const long long T = (long long)gridDim.x * blockDim.x;
    for (long long i0 = gtid(); i0 < P.n; i0 += T * kBreakItems) {
        int4 dp[kBreakItems];
        int me[kBreakItems], drx[kBreakItems];
#pragma unroll
        for (int u = 0; u < kBreakItems; ++u) {
            const long long i = i0 + u * T;
            dp[u] = i < P.n ? A.dp[i] : make_int4(-1, -1, -1, -1);
        }
#pragma unroll
        for (int u = 0; u < kBreakItems; ++u) {
            const long long i = i0 + u * T;
            me[u] = dp[u].x >= 0 ? A.tag[i] : 0;
            drx[u] = dp[u].x >= 0 ? A.drx[i] : 0;
        }
#pragma unroll
        for (int u = 0; u < kBreakItems; ++u)
            break_particle<SLIP>(P, A, slot, step, i0 + u * T, dp[u], me[u], drx[u], tested);
    }
}

// The two proposal kernels of a reaction: each runs the scan (pull) or the
// push version of its phase, as push_type decides for this reaction, so the
// mode that is not used costs no launch.  The first also draws the breaking
// of the reaction's existing bonds (independent of the proposals), which
// fills the issue slots that the latency-bound proposal work leaves idle.
template <bool FORCED, bool SCREEN>
__global__ void __launch_bounds__(256, 4) k_proposals(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;   // uniform over the grid
    const int s = push_type(P, A, slot);
    if (s >= 0) push_pass1(P, A, slot, step, s);
    else pull_propose<SCREEN>(P, A, slot);
    unsigned long long tested = 0;
    break_pass<false>(P, A, slot, step, tested);
    const int idx[1] = {cBreakTested};
    const unsigned long long v[1] = {tested};
    warp_counts<1>(A.counters, idx, v);
}

// Breaking draws of slip reactions (launched only when some reaction has the
// slip modifier), between the proposal kernel and the apply phase that reads
// the break bits.
template <bool FORCED>
__global__ void __launch_bounds__(256) k_break_slip(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    unsigned long long tested = 0;
    break_pass<true>(P, A, slot, step, tested);
    const int idx[1] = {cBreakTested};
    const unsigned long long v[1] = {tested};
    warp_counts<1>(A.counters, idx, v);
}

template <bool FORCED>
__global__ void __launch_bounds__(256) k_resolve(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const int s = push_type(P, A, slot);
    if (s >= 0) push_pass2(P, A, slot, step, s);
    else pull_exact(P, A, slot, step);
}

// U_b of a proposed dynamic bond (Eq. 3), every operation one IEEE rounding
// in a fixed order (the oracle evaluates the same expressions).  Harmonic
// from d = |r - r0|: k d^2 / 2 (the sign of r - r0 cancels exactly); FENE,
// whose proposals aim at 0 so that d = r: -k R0^2 ln(1 - (r/R0)^2) / 2 with
// this library's logarithm, +inf at r >= R0.  FENEWCA and Tether from the
// separation r itself (HOOMD-blue's potentials of those names; +inf outside
// their finite range), with this library's exp and log.
__device__ __forceinline__ double dyn_bond_u(const DevParams &P, int bt, double d, double r)
{
    const double inf = __longlong_as_double(0x7FF0000000000000ll);
    const int kind = P.bkind[bt];
    if (kind == kHarmonic) return __dmul_rn(__dmul_rn(__dmul_rn(0.5, P.bk[bt]), d), d);
    const double R0 = P.br0[bt];
    if (kind == kFene) {
        const double q = __ddiv_rn(__dmul_rn(d, d), __dmul_rn(R0, R0));
        if (!(q < 1.0)) return inf;
        return __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(-0.5, P.bk[bt]), R0), R0), log_cw(__dsub_rn(1.0, q)));
    }
    if (kind == kFeneWca) {
        const double eps = P.bx[bt][0], sig = P.bx[bt][1];
        const double s = __dsub_rn(r, P.bx[bt][2]);
        const double q = __ddiv_rn(__dmul_rn(s, s), __dmul_rn(R0, R0));
        if (!(q < 1.0) || !(s > 0.0)) return inf;
        double U = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(-0.5, P.bk[bt]), R0), R0), log_cw(__dsub_rn(1.0, q)));
        if (s < __dmul_rn(sig, kTwoSixth)) {
            const double sr2 = __ddiv_rn(__dmul_rn(sig, sig), __dmul_rn(s, s));
            const double sr6 = __dmul_rn(__dmul_rn(sr2, sr2), sr2);
            U = __dadd_rn(U, __dadd_rn(__dmul_rn(__dmul_rn(4.0, eps), __dsub_rn(__dmul_rn(sr6, sr6), sr6)), eps));
        }
        return U;
    }
    // Tether: k_b = bk, l_min = br0, (l_c1, l_c0, l_max) = bx
    const double lmin = R0, lc1 = P.bx[bt][0], lc0 = P.bx[bt][1], lmax = P.bx[bt][2];
    if (!(r > lmin) || !(r < lmax)) return inf;
    if (r > lc0) {
        const double a = __dsub_rn(lc0, r), b = __dsub_rn(lmax, r);
        return __ddiv_rn(__dmul_rn(P.bk[bt], exp_cw(__ddiv_rn(1.0, a))), b);
    }
    if (r < lc1) {
        const double c = __dsub_rn(r, lc1), e = __dsub_rn(r, lmin);
        return __ddiv_rn(__dmul_rn(P.bk[bt], exp_cw(__ddiv_rn(1.0, c))), e);
    }
    return 0.0;
}

// the separation r of the pair (i, j), needed by the bond kinds whose energy
// is not a function of |r - r0| alone
__device__ __forceinline__ double accept_r(const DevParams &P, const DevArrays &A, const RepDev &R, int bt, int i,
                                          int j)
{
    return P.bkind[bt] >= kFeneWca ? __dsqrt_rn(exact_r2(A, R, i, j)) : 0.0;
}

// Acceptance (Eq. 3) of the surviving edges: in scan mode one thread per
// listed site, in push mode one per pushing site.
template <bool FORCED>
__global__ void k_accept(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    unsigned long long edge = 0, surv = 0, formed = 0;
    const int ps = push_type(P, A, slot);
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (ps >= 0) {
        // push mode: every edge has a pushing end; the edge that can survive at
        // pushing site c is the one its best[] names (its low word is the
        // other end's tag)
        const int ns = A.avail_count[ps];
        for (long long g = gtid(); g < ns; g += stride) {
            const int c = A.avail_list[(long long)ps * P.n + g];
            const unsigned long long bc = A.best[c];
            if (bc != 0ull) {
                const int a = rx_at(P, A, 0, slot);
                const RepDev &R = A.reps[0];
                const uint32_t tc = (uint32_t)(A.tag[c] - R.tag_off), tj = (uint32_t)bc;
                const int j = A.rtag[tj + R.tag_off];
                const unsigned long long pr = bc & 0xFFFFFFFF00000000ull;
                if (A.best[j] == (pr | tc)) {
                    ++surv;
                    const uint32_t lo = tc < tj ? tc : tj, hi = tc < tj ? tj : tc;
                    const U4 w = pair_draw(R, a, kForm, step, lo, hi);
                    const double u = u53(w.x, w.y);
                    // U_b from d = |r - r0| of whichever end proposed the edge
                    const double d = A.prop[c] == j ? A.prop_d[c] : A.prop_d[j];
                    const int bt = P.rx_bt[a];
                    const double U = dyn_bond_u(P, bt, d, accept_r(P, A, R, bt, c, j));
                    double pon;
                    if (R.t_sweep > 0.0) pon = __dmul_rn(R.p_on0[a], exp_cw(-__ddiv_rn(U, R.t_sweep)));
                    else pon = (U <= 0.0) ? R.p_on0[a] : 0.0;
                    if (u < pon) {
                        ++formed;
                        A.fpart[c] = j;
                        A.fpart[j] = c;
                    }
                }
            }
        }
    }
    const int nlist = ps >= 0 ? 0 : *A.list_count;
    for (long long g = gtid(); g < nlist; g += stride) {
        const int i = A.site_list[g];
        const int j = A.prop[i];
        if (j >= 0) {
            const int rp = rep_of(P, A, i);
            const int a = rx_at(P, A, rp, slot);
            const RepDev &R = A.reps[rp];
            const uint32_t ti = (uint32_t)(A.tag[i] - R.tag_off), tj = (uint32_t)(A.tag[j] - R.tag_off);
            // a mutual proposal is one edge, handled by its smaller tag
            if (!(A.prop[j] == i && tj < ti)) {
                ++edge;
                const unsigned long long pr = (unsigned long long)A.prio[i] << 32;
                if (A.best[i] == (pr | tj) && A.best[j] == (pr | ti)) {
                    ++surv;
                    const uint32_t lo = ti < tj ? ti : tj, hi = ti < tj ? tj : ti;
                    const U4 w = pair_draw(R, a, kForm, step, lo, hi);
                    const double u = u53(w.x, w.y);
                    const int bt = P.rx_bt[a];
                    const double U = dyn_bond_u(P, bt, A.prop_d[i], accept_r(P, A, R, bt, i, j));
                    double pon;
                    if (R.t_sweep > 0.0) {
                        const double e = __ddiv_rn(U, R.t_sweep);
                        pon = __dmul_rn(R.p_on0[a], exp_cw(-e));
                    } else {
                        pon = (U <= 0.0) ? R.p_on0[a] : 0.0;
                    }
                    if (u < pon) {
                        ++formed;
                        A.fpart[i] = j;
                        A.fpart[j] = i;
                    }
                }
            }
        }
    }
    const int idx[4] = {cEdges, cSurvivors, cFormed, cFormedTotal};
    const unsigned long long v[4] = {edge, surv, formed, formed};
    warp_counts<4>(A.counters, idx, v);
}

// Apply phase: each thread takes kApplyItems particles of its block's tile,
// the scratch loads of all of them issued before any is used (one wave of
// resident blocks instead of several waves of one load chain each); the few
// particles whose bonds change are updated after.
constexpr int kApplyItems = 4;

template <bool FORCED>
__global__ void k_apply(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const long long g = gtid();
    if (g == 0) *A.list_count = 0;   // next reaction starts an empty list
    if (g < kMaxTypes && slot == P.nrx - 1) A.avail_count[g] = 0;   // the next sweep recounts
    const long long base = (long long)blockIdx.x * (blockDim.x * kApplyItems) + threadIdx.x;
    ApplyIn in[kApplyItems];
#pragma unroll
    for (int u = 0; u < kApplyItems; ++u) {
        const long long i = base + u * blockDim.x;
        if (i < P.n) in[u] = apply_load(A, i);
    }
    unsigned ch = 0u;
#pragma unroll
    for (int u = 0; u < kApplyItems; ++u) {
        const long long i = base + u * blockDim.x;
        if (i < P.n && apply_clear(A, i, in[u])) ch |= 1u << u;
    }
    unsigned long long nbroken = 0;
#pragma unroll
    for (int u = 0; u < kApplyItems; ++u)
        if ((ch >> u) & 1u) apply_update(P, A, slot, step, base + u * blockDim.x, in[u], nbroken);
    const int idx[2] = {cBroken, cBrokenTotal};
    const unsigned long long v[2] = {nbroken, nbroken};
    warp_counts<2>(A.counters, idx, v);
}

// After a latched status the sweep may have stopped part-way (its later
// kernels return early, k_apply among them): clear the per-reaction scratch
// that k_apply would have cleared, so that the next sweep starts clean.  The
// bond slots, occupancies and positions are untouched.
__global__ void k_sweep_reset(DevParams P, DevArrays A)
{
    const long long i = gtid();
    if (i == 0) *A.list_count = 0;
    if (i < kMaxTypes) A.avail_count[i] = 0;
    if (i >= P.n) return;
    A.brk[i] = 0u;
    A.fpart[i] = -1;
    A.best[i] = 0ull;
    A.prop[i] = -1;
    A.pkey[i] = make_ulonglong2(~0ull, ~0ull);
}

__global__ void k_step_end(DevArrays A)
{
    if (!status_ok(A.status)) return;
    *A.step += 1;
    *A.list_fresh = 0;   // the step's MD kernel has stored the force-list shift codes
}

inline unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }

template <bool FORCED>
void sweep_begin(const DevParams &P, const DevArrays &A, Launch L)
{
    if (P.kinetic_T && P.n > 0) k_kin_sum<FORCED><<<grid_for(P.n, 256), 256, 0, L.stream>>>(P, A);
    const long long nb = std::max<long long>((P.n + kSweepBeginBlock * kBeginItems - 1) / (kSweepBeginBlock * kBeginItems),
                                             (P.nrep + kSweepBeginBlock - 1) / kSweepBeginBlock);
    k_sweep_begin<FORCED><<<(unsigned)std::max<long long>(nb, 1), kSweepBeginBlock, 0, L.stream>>>(P, A);
}

template <bool FORCED>
void sweep_reaction(const DevParams &P, const DevArrays &A, int slot, Launch L)
{
    if (P.n == 0) return;
    const unsigned g = grid_for(P.n, L.block);
    const unsigned gl = kListBlocks;
    // grid-stride kernels: enough resident blocks for the scan, and one warp
    // per pushing site in push mode
    const unsigned gprop = (unsigned)std::min<long long>(g, 8LL * sm_count() * (256 / L.block));
    if (P.screen) k_proposals<FORCED, true><<<gprop, L.block, 0, L.stream>>>(P, A, slot);
    else k_proposals<FORCED, false><<<gprop, L.block, 0, L.stream>>>(P, A, slot);
    if (P.slip_mask) k_break_slip<FORCED><<<gprop, L.block, 0, L.stream>>>(P, A, slot);
    k_resolve<FORCED><<<std::max<unsigned>(gl, (unsigned)std::min<long long>(grid_for(P.n, 256), 4LL * sm_count())),
                        256, 0, L.stream>>>(P, A, slot);
    k_accept<FORCED><<<gl, 256, 0, L.stream>>>(P, A, slot);
    if (P.log_events) launch_log_events(P, A, slot, FORCED, L);
    k_apply<FORCED><<<std::max<unsigned>(1u, grid_for(P.n, L.block * kApplyItems)), L.block, 0, L.stream>>>(P, A, slot);
}

}  // namespace

void launch_sweep_begin(const DevParams &P, const DevArrays &A, Launch L) { sweep_begin<false>(P, A, L); }
void launch_sweep_begin_forced(const DevParams &P, const DevArrays &A, Launch L)
{
    sweep_begin<true>(P, A, L);
}
void launch_sweep_reaction(const DevParams &P, const DevArrays &A, int slot, Launch L)
{
    sweep_reaction<false>(P, A, slot, L);
}
void launch_sweep_reaction_forced(const DevParams &P, const DevArrays &A, int slot, Launch L)
{
    sweep_reaction<true>(P, A, slot, L);
}

void launch_step_end(const DevArrays &A, Launch L) { k_step_end<<<1, 1, 0, L.stream>>>(A); }

void launch_sweep_reset(const DevParams &P, const DevArrays &A, Launch L)
{
    k_sweep_reset<<<grid_for(std::max<long long>(P.n, kMaxTypes), 256), 256, 0, L.stream>>>(P, A);
}

}  // namespace snap
