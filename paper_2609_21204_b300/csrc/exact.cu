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

// Reaction order per replica: Fisher–Yates driven by Philox(ORDER) with
// counter (step, k), so competing reactions are treated evenhandedly.
template <bool FORCED>
__global__ void k_sweep_begin(DevParams P, DevArrays A)
{
    long long step;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const int r = (int)gtid();
    if (r == 0) {
        for (int c = cScanned; c <= cBroken; ++c) A.counters[c] = 0ull;
        A.counters[cNlistScanned] = 0ull;
        A.counters[cSweeps] += 1ull;
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

template <bool FORCED>
__global__ void __launch_bounds__(256) k_propose(DevParams P, DevArrays A, int slot)
{
    long long step;
    const long long i = gtid();
    if (i >= P.n) return;
    if (!sweep_active<FORCED>(P, A, step)) return;
    A.best[i] = 0ull;
    A.fpart[i] = -1;
    A.brk[i] = 0u;
    A.prop[i] = -1;
    const int rp = A.rep[i];
    const int a = A.rx_order[rp * kMaxRx + slot];
    const int ti = A.type[i];
    const int ta = P.rx_ta[a], tb = P.rx_tb[a];
    if (ti != ta && ti != tb) return;
    if (A.occ[i] >= P.valence[ti]) return;
    const RepDev &R = A.reps[rp];
    const int4 dp = A.dp[i];
    const double xi = A.x[i], yi = A.y[i], zi = A.z[i];
    const double rmin2 = P.rx_rmin2[a], rmax2 = P.rx_rmax2[a];
    const double r0 = P.br0[P.rx_bt[a]];
    const int nn = A.nn[i];
    const long long stride = P.nbr_stride;
    int best = -1, best_tag = 0;
    double best_d = 0.0, best_r = 0.0;
    unsigned long long scanned = 0, inwin = 0;
    for (int k = 0; k < nn; ++k) {
        const int j = A.nbr[(long long)k * stride + i];
        const int tj = A.type[j];
        const bool compat = (ti == ta && tj == tb) || (ti == tb && tj == ta);
        if (!compat) continue;
        if (A.occ[j] >= P.valence[tj]) continue;
        const int tgj = A.tag[j];
        if (tgj == dp.x || tgj == dp.y || tgj == dp.z || tgj == dp.w) continue;
        ++scanned;
        const double dx = min_image(__dsub_rn(A.x[j], xi), R.L[0], R.invL[0]);
        const double dy = min_image(__dsub_rn(A.y[j], yi), R.L[1], R.invL[1]);
        const double dz = min_image(__dsub_rn(A.z[j], zi), R.L[2], R.invL[2]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (r2 < rmin2 || r2 > rmax2) continue;
        ++inwin;
        const double r = __dsqrt_rn(r2);
        const double d = fabs(__dsub_rn(r, r0));
        if (best < 0 || d < best_d || (d == best_d && tgj < best_tag)) {
            best = j;
            best_tag = tgj;
            best_d = d;
            best_r = r;
        }
    }
    A.prop[i] = best;
    A.prop_r[i] = best_r;
    warp_count(&A.counters[cNlistScanned], (unsigned long long)nn);
    warp_count(&A.counters[cScanned], scanned);
    warp_count(&A.counters[cInWindow], inwin);
    warp_count(&A.counters[cProposals], best >= 0 ? 1ull : 0ull);
}

template <bool FORCED>
__global__ void k_match(DevParams P, DevArrays A, int slot)
{
    long long step;
    const long long i = gtid();
    if (i >= P.n) return;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const int j = A.prop[i];
    if (j < 0) return;
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

template <bool FORCED>
__global__ void k_accept(DevParams P, DevArrays A, int slot)
{
    long long step;
    const long long i = gtid();
    if (i >= P.n) return;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const int j = A.prop[i];
    unsigned long long edge = 0, surv = 0, formed = 0;
    if (j >= 0) {
        const int rp = A.rep[i];
        const int a = A.rx_order[rp * kMaxRx + slot];
        const RepDev &R = A.reps[rp];
        const uint32_t ti = (uint32_t)(A.tag[i] - R.tag_off), tj = (uint32_t)(A.tag[j] - R.tag_off);
        // a mutual proposal is one edge, handled by its smaller tag
        if (!(A.prop[j] == (int)i && tj < ti)) {
            edge = 1;
            const unsigned long long pr = (unsigned long long)A.prio[i] << 32;
            if (A.best[i] == (pr | tj) && A.best[j] == (pr | ti)) {
                surv = 1;
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
                    formed = 1;
                    A.fpart[i] = j;
                    A.fpart[j] = (int)i;
                }
            }
        }
    }
    warp_count(&A.counters[cEdges], edge);
    warp_count(&A.counters[cSurvivors], surv);
    warp_count(&A.counters[cFormed], formed);
    warp_count(&A.counters[cFormedTotal], formed);
}

template <bool FORCED>
__global__ void k_break(DevParams P, DevArrays A, int slot)
{
    long long step;
    const long long i = gtid();
    if (i >= P.n) return;
    if (!sweep_active<FORCED>(P, A, step)) return;
    unsigned long long tested = 0;
    const int4 dp = A.dp[i];
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
            if (u53(w.x, w.y) < R.p_off[a]) {
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
    warp_count(&A.counters[cBreakTested], tested);
}

template <bool FORCED>
__global__ void k_apply(DevParams P, DevArrays A, int slot)
{
    long long step;
    const long long i = gtid();
    if (i >= P.n) return;
    if (!sweep_active<FORCED>(P, A, step)) return;
    const uint32_t b = A.brk[i];
    const int f = A.fpart[i];
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
    warp_count(&A.counters[cBroken], nbroken);
    warp_count(&A.counters[cBrokenTotal], nbroken);
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
    k_propose<FORCED><<<g, L.block, 0, L.stream>>>(P, A, slot);
    k_match<FORCED><<<g, L.block, 0, L.stream>>>(P, A, slot);
    k_accept<FORCED><<<g, L.block, 0, L.stream>>>(P, A, slot);
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
    else k_integrate<float><<<grid_for(P.n, L.block), L.block, 0, L.stream>>>(P, A);
}

void launch_step_end(const DevArrays &A, Launch L) { k_step_end<<<1, 1, 0, L.stream>>>(A); }

}  // namespace snap
