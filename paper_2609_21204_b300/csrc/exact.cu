// Bit-reproducible kernels: the bond sweep and the Langevin integrator.
//
// Compiled with -fmad=false and written with explicit round-to-nearest
// intrinsics, so every FP64 operation is a single IEEE rounding in a fixed
// order.  Given identical positions, the sweep therefore takes exactly the
// decisions its definition implies, on any device and any block size.
//
// The sweep follows Sec. II.C of the DyBond-v2 paper (Fig. 1), one kernel per
// phase and per reaction in a random order redrawn every sweep:
//   propose  — every free reactive site scans its neighbour list and keeps the
//              free, type-compatible partner in [r_min, r_max] closest to the
//              rest length (ties to the smaller tag);
//   match    — each proposal edge gets a Philox priority; atomicMax of
//              (priority << 32 | other tag) at both endpoints;
//   accept   — an edge survives iff it holds the maximum at both ends (a
//              locally dominant matching, disjoint by construction, replacing
//              the paper's compare-and-swap race with a scheduling-independent
//              rule) and forms with probability P_on^0 exp(-U_b(r)/kT), Eq. 3;
//   break    — every bond of this reaction present before the reaction began
//              breaks with probability P_off;
//   apply    — per particle, broken slots are removed and the formed partner
//              inserted; occupancies change before the next reaction reads them.
#include "snap_kernels.h"

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

// Reaction order per replica: Fisher–Yates driven by Philox(ORDER) with
// counter (step, k), so competing reactions are treated evenhandedly.
template <bool FORCED>
__global__ void k_sweep_begin(DevParams P, DevArrays A)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const int r = (int)gtid();
    if (r == 0) {
        for (int c = cScanned; c <= cBroken; ++c) counter_reset(A.counters, c);
        counter_reset(A.counters, cNlistScanned);
        counter_add1(A.counters, cSweeps, 1ull);
        *A.list_count = 0;
    }
    if (r >= P.nrep) return;
    const RepDev &R = A.reps[r];
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

// exact FP64 squared separation, as the definition states it:
// d = x_j - x_i; d -= L rint(d / L) per axis; r^2 = (dx^2 + dy^2) + dz^2
__device__ __forceinline__ double exact_r2(const DevArrays &A, const RepDev &R, int i, int j)
{
    const double dx = min_image(__dsub_rn(A.x[j], A.x[i]), R.L[0], R.invL[0]);
    const double dy = min_image(__dsub_rn(A.y[j], A.y[i]), R.L[1], R.invL[1]);
    const double dz = min_image(__dsub_rn(A.z[j], A.z[i]), R.L[2], R.invL[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
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
// With cell-relative FP32 coordinates (|rel| < 4, each rounded once), the
// FP32 separation of a listed pair differs from the exact one by less than
// 1.3e-6 per component, so r^2 by less than 1.2e-5 (r < 2) and |r - r0| by
// less than 2e-5 when r^2 >= 0.09.  With margins of 1e-4 a candidate is
// dropped in FP32 only when the exact test would reject it or when another
// candidate surely beats it; every candidate that may win is re-evaluated in
// FP64 by k_exact, in dense warps.
constexpr float kScreenR2 = 1e-4f;
constexpr float kScreenD = 1e-4f;

template <bool FORCED, bool SCREEN>
__global__ void __launch_bounds__(256) k_propose(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;   // uniform over the grid
    const long long i = gtid();
    unsigned long long scanned = 0, inwin = 0, nscan = 0, nprop = 0;
    bool want = false;
    int ncont = 0;
    int cont[kContenders];
    if (i < P.n) {
        A.best[i] = 0ull;
        A.fpart[i] = -1;
        A.brk[i] = 0u;
        int best = -1;
        double best_r = 0.0;
        const int rp = A.rep[i];
        const int a = A.rx_order[rp * kMaxRx + slot];
        const int ti = A.type[i];
        const int ta = P.rx_ta[a], tb = P.rx_tb[a];
        if ((ti == ta || ti == tb) && A.occ[i] < P.valence[ti]) {
            const RepDev &R = A.reps[rp];
            const int4 dp = A.dp[i];
            const double rmin2 = P.rx_rmin2[a], rmax2 = P.rx_rmax2[a];
            const double r0 = P.br0[P.rx_bt[a]];
            const float rmin2f = (float)rmin2, rmax2f = (float)rmax2, r0f = (float)r0;
            const float4 *pos4 = reinterpret_cast<const float4 *>(A.pos4);
            float4 pi4 = make_float4(0.f, 0.f, 0.f, 0.f);
            if (SCREEN) pi4 = pos4[i];
            const int nn = A.nn[i];
            const long long stride = P.nbr_stride;
            int best_tag = 0;
            double best_d = 0.0;
            float cd[kContenders];
            float min_upper = 3.0e38f;
            unsigned long long sure_in = 0;
            bool ovf = false;
            nscan = (unsigned long long)nn;
            for (int k0 = 0; k0 < nn; k0 += 8) {
                int jj[8], tt[8], oo[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) jj[u] = (k0 + u < nn) ? A.nbr[(long long)(k0 + u) * stride + i] : -1;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    tt[u] = jj[u] >= 0 ? A.type[jj[u]] : -1;
                    oo[u] = jj[u] >= 0 ? A.occ[jj[u]] : 0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = jj[u];
                    if (j < 0) continue;
                    const int tj = tt[u];
                    const bool compat = (ti == ta && tj == tb) || (ti == tb && tj == ta);
                    if (!compat || oo[u] >= P.valence[tj]) continue;
                    const int tgj = A.tag[j];
                    if (tgj == dp.x || tgj == dp.y || tgj == dp.z || tgj == dp.w) continue;
                    ++scanned;
                    if (SCREEN) {
                        const float4 pj4 = pos4[j];
                        const uint32_t bi = w_bits(pi4), bj = w_bits(pj4);
                        const float ex = (pj4.x - pi4.x) + (float)cell_delta(bits_cx(bj) - bits_cx(bi), R.nc[0]) * R.wf[0];
                        const float ey = (pj4.y - pi4.y) + (float)cell_delta(bits_cy(bj) - bits_cy(bi), R.nc[1]) * R.wf[1];
                        const float ez = (pj4.z - pi4.z) + (float)cell_delta(bits_cz(bj) - bits_cz(bi), R.nc[2]) * R.wf[2];
                        const float r2f = ex * ex + ey * ey + ez * ez;
                        if (r2f < rmin2f - kScreenR2 || r2f > rmax2f + kScreenR2) continue;  // surely outside
                        const bool amb = !(r2f > rmin2f + kScreenR2 && r2f < rmax2f - kScreenR2);
                        const bool small = r2f < 0.09f;
                        const float df = fabsf(sqrtf(r2f) - r0f);
                        if (!amb) {
                            ++sure_in;
                            if (!small) {
                                if (df - kScreenD > min_upper) continue;   // surely beaten
                                min_upper = fminf(min_upper, df + kScreenD);
                            }
                        }
                        // drop kept contenders that are now surely beaten
                        int m = 0;
                        for (int c = 0; c < ncont; ++c) {
                            const bool keep = (cont[c] >> 30) != 0 || cd[c] < 0.f || cd[c] - kScreenD <= min_upper;
                            if (keep) {
                                cont[m] = cont[c];
                                cd[m] = cd[c];
                                ++m;
                            }
                        }
                        ncont = m;
                        if (ncont < kContenders) {
                            cont[ncont] = j | (amb ? (1 << 30) : 0);
                            cd[ncont] = small ? -1.f : df;   // negative: no usable bound
                            ++ncont;
                        } else {
                            ovf = true;
                        }
                    } else {
                        const double r2 = exact_r2(A, R, (int)i, j);
                        if (r2 < rmin2 || r2 > rmax2) continue;
                        ++inwin;
                        const double r = __dsqrt_rn(r2);
                        consider(fabs(__dsub_rn(r, r0)), r, j, tgj, best, best_tag, best_d, best_r);
                    }
                }
            }
            if (SCREEN) {
                if (ovf) ncont = kContenders + 1;          // k_exact rescans this site in full
                else inwin += sure_in;
                want = ncont > 0;
            } else {
                nprop = best >= 0 ? 1ull : 0ull;
                want = best >= 0;
            }
        }
        A.prop[i] = best;
        A.prop_r[i] = best_r;
        A.ncont[i] = ncont;
        if (SCREEN && ncont > 0 && ncont <= kContenders)
            for (int c = 0; c < ncont; ++c) A.cont[i * kContenders + c] = cont[c];
    }
    const int sl = block_append(want, A.list_count);
    if (sl >= 0) A.site_list[sl] = (int)i;
    const int idx[4] = {cNlistScanned, cScanned, cInWindow, cProposals};
    const unsigned long long v[4] = {nscan, scanned, inwin, nprop};
    warp_counts<4>(A.counters, idx, v);
}

// Exact FP64 evaluation of the screened contenders, one listed site per thread.
template <bool FORCED>
__global__ void __launch_bounds__(256) k_exact(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const int nlist = *A.list_count;
    unsigned long long inwin = 0, nprop = 0;
    for (long long q = gtid(); q < nlist; q += (long long)gridDim.x * blockDim.x) {
        const int i = A.site_list[q];
        const int nc = A.ncont[i];
        if (nc == 0) continue;                       // decided without a screen
        const int rp = A.rep[i];
        const int a = A.rx_order[rp * kMaxRx + slot];
        const RepDev &R = A.reps[rp];
        const double rmin2 = P.rx_rmin2[a], rmax2 = P.rx_rmax2[a];
        const double r0 = P.br0[P.rx_bt[a]];
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
            const int ti = A.type[i];
            const int ta = P.rx_ta[a], tb = P.rx_tb[a];
            const int4 dp = A.dp[i];
            const int nn = A.nn[i];
            for (int k = 0; k < nn; ++k) {
                const int j = A.nbr[(long long)k * P.nbr_stride + i];
                const int tj = A.type[j];
                const bool compat = (ti == ta && tj == tb) || (ti == tb && tj == ta);
                if (!compat || A.occ[j] >= P.valence[tj]) continue;
                const int tgj = A.tag[j];
                if (tgj == dp.x || tgj == dp.y || tgj == dp.z || tgj == dp.w) continue;
                const double r2 = exact_r2(A, R, i, j);
                if (r2 < rmin2 || r2 > rmax2) continue;
                ++inwin;
                const double r = __dsqrt_rn(r2);
                consider(fabs(__dsub_rn(r, r0)), r, j, tgj, best, best_tag, best_d, best_r);
            }
        }
        A.prop[i] = best;
        A.prop_r[i] = best_r;
        if (best >= 0) ++nprop;
    }
    const int idx[2] = {cInWindow, cProposals};
    const unsigned long long v[2] = {inwin, nprop};
    warp_counts<2>(A.counters, idx, v);
}

template <bool FORCED>
__global__ void k_match(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const int nlist = *A.list_count;
    for (long long q = gtid(); q < nlist; q += (long long)gridDim.x * blockDim.x) {
        const int i = A.site_list[q];
        const int j = A.prop[i];
        if (j < 0) continue;
        const int rp = A.rep[i];
        const int a = A.rx_order[rp * kMaxRx + slot];
        const RepDev &R = A.reps[rp];
        const uint32_t ti = (uint32_t)(A.tag[i] - R.tag_off), tj = (uint32_t)(A.tag[j] - R.tag_off);
        const uint32_t lo = ti < tj ? ti : tj, hi = ti < tj ? tj : ti;
        const U4 w = pair_draw(R, a, kMatch, step, lo, hi);
        A.prio[i] = w.x;
        const unsigned long long pr = (unsigned long long)w.x << 32;
        atomicMax(&A.best[i], pr | tj);
        atomicMax(&A.best[j], pr | ti);
    }
}

template <bool FORCED>
__global__ void k_accept(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const int nlist = *A.list_count;
    unsigned long long edge = 0, surv = 0, formed = 0;
    for (long long q = gtid(); q < nlist; q += (long long)gridDim.x * blockDim.x) {
        const int i = A.site_list[q];
        const int j = A.prop[i];
        if (j < 0) continue;
        const int rp = A.rep[i];
        const int a = A.rx_order[rp * kMaxRx + slot];
        const RepDev &R = A.reps[rp];
        const uint32_t ti = (uint32_t)(A.tag[i] - R.tag_off), tj = (uint32_t)(A.tag[j] - R.tag_off);
        // a mutual proposal is one edge, handled by its smaller tag
        if (A.prop[j] == i && tj < ti) continue;
        ++edge;
        const unsigned long long pr = (unsigned long long)A.prio[i] << 32;
        if (A.best[i] != (pr | tj) || A.best[j] != (pr | ti)) continue;
        ++surv;
        const uint32_t lo = ti < tj ? ti : tj, hi = ti < tj ? tj : ti;
        const U4 w = pair_draw(R, a, kForm, step, lo, hi);
        const double u = u53(w.x, w.y);
        const int bt = P.rx_bt[a];
        const double dr = __dsub_rn(A.prop_r[i], P.br0[bt]);
        const double U = __dmul_rn(__dmul_rn(__dmul_rn(0.5, P.bk[bt]), dr), dr);
        double pon;
        if (R.kT > 0.0) {
            const double e = __ddiv_rn(U, R.kT);
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
    const int idx[4] = {cEdges, cSurvivors, cFormed, cFormedTotal};
    const unsigned long long v[4] = {edge, surv, formed, formed};
    warp_counts<4>(A.counters, idx, v);
}

template <bool FORCED>
__global__ void k_break(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const long long i = gtid();
    unsigned long long tested = 0;
    const int4 dp = i < P.n ? A.dp[i] : make_int4(-1, -1, -1, -1);
    if (dp.x >= 0) {
        const int rp = A.rep[i];
        const int a = A.rx_order[rp * kMaxRx + slot];
        const RepDev &R = A.reps[rp];
        const int me = A.tag[i];
        const int drx = A.drx[i];
        const int pv[4] = {dp.x, dp.y, dp.z, dp.w};
#pragma unroll
        for (int s = 0; s < kVmax; ++s) {
            const int p = pv[s];
            if (p < 0 || p < me) continue;           // the smaller tag owns the bond
            if (((drx >> (8 * s)) & 0xFF) != a) continue;
            ++tested;
            const U4 w = pair_draw(R, a, kBreak, step, (uint32_t)(me - R.tag_off),
                                   (uint32_t)(p - R.tag_off));
            // u53 < p_off  <=>  m < ceil(p_off 2^53) with m the 53-bit integer of u53
            const unsigned long long m = ((unsigned long long)w.x << 21) | (unsigned long long)(w.y >> 11);
            if (m < R.off_thresh[a]) {
                atomicOr(&A.brk[i], 1u << s);
                const int j = A.rtag[p];
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
    const int idx[1] = {cBreakTested};
    const unsigned long long v[1] = {tested};
    warp_counts<1>(A.counters, idx, v);
}

template <bool FORCED>
__global__ void k_apply(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const long long i = gtid();
    if (i == 0) *A.list_count = 0;   // next reaction starts an empty list
    const uint32_t b = i < P.n ? A.brk[i] : 0u;
    const int f = i < P.n ? A.fpart[i] : -1;
    unsigned long long nbroken = 0;
    if (b != 0u || f >= 0) {
        const int me = A.tag[i];
        const int4 dp = A.dp[i];
        const int4 db = A.dbirth[i];
        const int drx = A.drx[i];
        const int pv[4] = {dp.x, dp.y, dp.z, dp.w};
        const int bv[4] = {db.x, db.y, db.z, db.w};
        int np[4] = {-1, -1, -1, -1}, nb[4] = {0, 0, 0, 0}, nr[4] = {0, 0, 0, 0};
        int m = 0;
        for (int s = 0; s < kVmax; ++s) {
            const int p = pv[s];
            if (p < 0) continue;
            if ((b >> s) & 1u) {
                if (me < p) {
                    ++nbroken;
                    long long life = (long long)((uint32_t)step - (uint32_t)bv[s]) / P.period;
                    if (life >= P.nhist) life = P.nhist - 1;
                    atomicAdd(&A.life_hist[life], 1ull);
                }
                continue;
            }
            np[m] = p; nb[m] = bv[s]; nr[m] = (drx >> (8 * s)) & 0xFF;
            ++m;
        }
        if (f >= 0) {
            const int rp = A.rep[i];
            const int a = A.rx_order[rp * kMaxRx + slot];
            const int pt = A.tag[f];
            int s = m;
            while (s > 0 && np[s - 1] > pt) {
                np[s] = np[s - 1]; nb[s] = nb[s - 1]; nr[s] = nr[s - 1];
                --s;
            }
            np[s] = pt; nb[s] = (int)(uint32_t)step; nr[s] = a;
            ++m;
        }
        A.dp[i] = make_int4(np[0], np[1], np[2], np[3]);
        A.dbirth[i] = make_int4(nb[0], nb[1], nb[2], nb[3]);
        A.drx[i] = (nr[0] & 0xFF) | ((nr[1] & 0xFF) << 8) | ((nr[2] & 0xFF) << 16) | ((nr[3] & 0xFF) << 24);
        A.occ[i] = m;
    }
    const int idx[2] = {cBroken, cBrokenTotal};
    const unsigned long long v[2] = {nbroken, nbroken};
    warp_counts<2>(A.counters, idx, v);
}

// ------------------------------------------------------------ integrator
// a = F_c(x_t) - gamma v_{t-1/2} + sqrt(2 gamma kT/dt) xi,  xi = sqrt(3)(2u - 1)
// v_{t+1/2} = v_{t-1/2} + dt a;  x_{t+1} = x_t + dt v_{t+1/2};  wrap into [0, L)
__device__ __forceinline__ void wrap(double &x, int &img, double L)
{
    if (x >= L) {
        x = __dsub_rn(x, L);
        img += 1;
    } else if (x < 0.0) {
        x = __dadd_rn(x, L);
        img -= 1;
        if (x >= L) {
            x = __dsub_rn(x, L);
            img += 1;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_integrate(DevParams P, DevArrays A)
{
    using V = typename Vec4<R>::T;
    const long long i = gtid();
    if (i >= P.n) return;
    if (!status_ok(A.status)) return;
    const long long step = *A.step;
    const int rp = A.rep[i];
    const RepDev &Rp = A.reps[rp];
    const uint32_t tl = (uint32_t)(A.tag[i] - Rp.tag_off);
    const U4 w = philox10(U4{(uint32_t)((unsigned long long)step & 0xFFFFFFFFull),
                             (uint32_t)((unsigned long long)step >> 32), tl, 0u},
                          Rp.key0, rx_key1(Rp, 0, kLangevin));
    const V f = reinterpret_cast<const V *>(A.force)[i];
    const double fv[3] = {(double)f.x, (double)f.y, (double)f.z};
    const uint32_t wv[3] = {w.x, w.y, w.z};
    double *xs[3] = {A.x, A.y, A.z};
    double *vs[3] = {A.vx, A.vy, A.vz};
    int *is[3] = {A.ix, A.iy, A.iz};
    double xn[3];
    bool finite = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double u = __dadd_rn(__dmul_rn((double)wv[d], 0x1.0p-32), 0x1.0p-33);
        const double xi = __dmul_rn(P.sqrt3, __dsub_rn(__dmul_rn(2.0, u), 1.0));
        const double v0 = vs[d][i];
        const double drag = __dmul_rn(P.gamma, v0);
        const double acc = __dadd_rn(__dsub_rn(fv[d], drag), __dmul_rn(Rp.noise_c, xi));
        const double v1 = __dadd_rn(v0, __dmul_rn(P.dt, acc));
        double x1 = __dadd_rn(xs[d][i], __dmul_rn(P.dt, v1));
        finite = finite && isfinite(x1);
        int img = is[d][i];
        wrap(x1, img, Rp.L[d]);
        vs[d][i] = v1;
        xs[d][i] = x1;
        is[d][i] = img;
        xn[d] = x1;
    }
    if (!finite) {
        atomicOr(A.status, (uint32_t)kStNonfinite);
        return;
    }
    // relative coordinates against the frozen cell origin, minimum image
    V p = reinterpret_cast<V *>(A.pos4)[i];
    const uint32_t bits = w_bits(p);
    const int c[3] = {bits_cx(bits), bits_cy(bits), bits_cz(bits)};
    double rel[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double r = __dsub_rn(xn[d], __dmul_rn((double)c[d], Rp.w[d]));
        if (r > Rp.halfL[d]) r = __dsub_rn(r, Rp.L[d]);
        else if (r < -Rp.halfL[d]) r = __dadd_rn(r, Rp.L[d]);
        rel[d] = r;
    }
    p.x = (R)rel[0]; p.y = (R)rel[1]; p.z = (R)rel[2];
    reinterpret_cast<V *>(A.pos4)[i] = p;
    const float4 ref = A.ref4[i];
    const float ex = (float)rel[0] - ref.x, ey = (float)rel[1] - ref.y, ez = (float)rel[2] - ref.z;
    if (ex * ex + ey * ey + ez * ez > P.disp2f) *A.need_rebuild = 1;
}

// Mixed-precision Langevin step: the kick and the velocity in FP32, the
// position accumulated in FP64 (x += dt v), the cell-relative FP32 coordinate
// as (float)(x - origin) with the FP64 origin of the frozen cell.  Four FP64
// operations per axis; positions stay unwrapped between neighbour-list
// rebuilds (the rebuild wraps them).
__global__ void __launch_bounds__(256) k_integrate_mixed(DevParams P, DevArrays A)
{
    const long long i = gtid();
    if (i >= P.n) return;
    if (!status_ok(A.status)) return;
    const long long step = *A.step;
    const RepDev &Rp = A.reps[A.rep[i]];
    const uint32_t tl = (uint32_t)(A.tag[i] - Rp.tag_off);
    const U4 w = philox10(U4{(uint32_t)((unsigned long long)step & 0xFFFFFFFFull),
                             (uint32_t)((unsigned long long)step >> 32), tl, 0u},
                          Rp.key0, rx_key1(Rp, 0, kLangevin));
    const float4 f = reinterpret_cast<const float4 *>(A.force)[i];
    float4 v = A.v4[i];
    float4 p = reinterpret_cast<float4 *>(A.pos4)[i];
    const float cn = (float)Rp.noise_c, g = (float)P.gamma, s3 = (float)P.sqrt3, dt = (float)P.dt;
    // xi = sqrt(3) (2u - 1) with u = (w >> 8 + 1/2) 2^-24 in (0, 1)
    const float ux = fmaf((float)(w.x >> 8), 0x1.0p-24f, 0x1.0p-25f);
    const float uy = fmaf((float)(w.y >> 8), 0x1.0p-24f, 0x1.0p-25f);
    const float uz = fmaf((float)(w.z >> 8), 0x1.0p-24f, 0x1.0p-25f);
    v.x = fmaf(dt, fmaf(cn, s3 * fmaf(2.0f, ux, -1.0f), fmaf(-g, v.x, f.x)), v.x);
    v.y = fmaf(dt, fmaf(cn, s3 * fmaf(2.0f, uy, -1.0f), fmaf(-g, v.y, f.y)), v.y);
    v.z = fmaf(dt, fmaf(cn, s3 * fmaf(2.0f, uz, -1.0f), fmaf(-g, v.z, f.z)), v.z);
    const double x1 = fma(P.dt, (double)v.x, A.x[i]);
    const double y1 = fma(P.dt, (double)v.y, A.y[i]);
    const double z1 = fma(P.dt, (double)v.z, A.z[i]);
    p.x = (float)(x1 - A.ox[i]);
    p.y = (float)(y1 - A.oy[i]);
    p.z = (float)(z1 - A.oz[i]);
    // finiteness from the exponent bits (no FP64 compare)
    const unsigned long long bad = 0x7FF0000000000000ull;
    if (((unsigned long long)__double_as_longlong(x1) & bad) == bad ||
        ((unsigned long long)__double_as_longlong(y1) & bad) == bad ||
        ((unsigned long long)__double_as_longlong(z1) & bad) == bad) {
        atomicOr(A.status, (uint32_t)kStNonfinite);
        return;
    }
    A.x[i] = x1;
    A.y[i] = y1;
    A.z[i] = z1;
    A.v4[i] = v;
    reinterpret_cast<float4 *>(A.pos4)[i] = p;
    const float4 ref = A.ref4[i];
    const float ex = p.x - ref.x, ey = p.y - ref.y, ez = p.z - ref.z;
    if (ex * ex + ey * ey + ez * ez > P.disp2f) *A.need_rebuild = 1;
}

__global__ void k_step_end(DevArrays A)
{
    if (!status_ok(A.status)) return;
    *A.step += 1;
}

inline unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }

template <bool FORCED>
void sweep_begin(const DevParams &P, const DevArrays &A, Launch L)
{
    k_sweep_begin<FORCED><<<grid_for(P.nrep, 128), 128, 0, L.stream>>>(P, A);
}

template <bool FORCED>
void sweep_reaction(const DevParams &P, const DevArrays &A, int slot, Launch L)
{
    if (P.n == 0) return;
    const unsigned g = grid_for(P.n, L.block);
    const unsigned gl = kListBlocks;
    if (P.screen) {
        k_propose<FORCED, true><<<g, L.block, 0, L.stream>>>(P, A, slot);
        k_exact<FORCED><<<gl, 256, 0, L.stream>>>(P, A, slot);
    } else {
        k_propose<FORCED, false><<<g, L.block, 0, L.stream>>>(P, A, slot);
    }
    k_match<FORCED><<<gl, 256, 0, L.stream>>>(P, A, slot);
    k_accept<FORCED><<<gl, 256, 0, L.stream>>>(P, A, slot);
    if (P.log_events) launch_log_events(P, A, slot, FORCED, L);
    k_break<FORCED><<<g, L.block, 0, L.stream>>>(P, A, slot);
    k_apply<FORCED><<<g, L.block, 0, L.stream>>>(P, A, slot);
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

void launch_integrate(const DevParams &P, const DevArrays &A, bool fp64, Launch L)
{
    if (P.n == 0) return;
    if (fp64) k_integrate<double><<<grid_for(P.n, L.block), L.block, 0, L.stream>>>(P, A);
    else k_integrate_mixed<<<grid_for(P.n, L.block), L.block, 0, L.stream>>>(P, A);
}

void launch_step_end(const DevArrays &A, Launch L) { k_step_end<<<1, 1, 0, L.stream>>>(A); }

}  // namespace snap
