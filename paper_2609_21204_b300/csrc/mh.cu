// Metropolis–Hastings bond moves and bond-event logging (an extension beyond
// the paper: the learned proposal and the uniform proposal it is measured against).
//
// Move set (one reaction, one system): checkerboard cells of side
// >= 2 r_max + 0.05, an even number per axis, colour = parities of the cell
// coordinates; the cells of colour (step mod 8) are active.  In each active
// cell an initiator i is drawn uniformly among its reactive particles
// (ascending tag) and, with probability 1/2 each, tries to
//   form  a bond with one of its owned candidates j (free, compatible,
//         unbonded, r_min <= r <= r_max), drawn from q(j | i; s), or
//   break one of its owned in-window bonds, drawn uniformly.
// Every pair has a fixed owner (one of its two tags, by a step-independent
// Philox bit), so a pair is formed and broken by the same initiator.  With the
// bond weight K exp(-U_b/kT), K = P_on^0 / P_off (Eqs. 1 and 3 of the
// DyBond-v2 paper), detailed balance gives
//   form : min(1, K e / (b_i(s') q(j|i; s)))
//   break: min(1, b_i(s) q(j|i; s \ ij) / (K e))
// where b_i counts i's owned in-window bonds.  The learned proposal is
// q = (1 - eps) softmax(MLP(features)) + eps / n; the uniform one is 1 / n.
// Active cells are more than 2 r_max apart, so their moves touch disjoint
// particles and candidate sets: one thread per active cell.
#include "snap_kernels.h"
#include <algorithm>

#include "snap_mlp.h"

namespace snap {

namespace {

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }

template <bool FORCED>
__device__ __forceinline__ bool mh_active(const DevParams &P, const DevArrays &A, long long &step)
{
    if (!status_ok(A.status)) return false;
    step = *A.step;
    if (!FORCED && (step % P.period) != 0) return false;
    return true;
}

__device__ __forceinline__ double exact_r2(const DevArrays &A, const RepDev &R, int i, int j)
{
    const double dx = min_image(__dsub_rn(A.x[j], A.x[i]), R.L[0], R.invL[0]);
    const double dy = min_image(__dsub_rn(A.y[j], A.y[i]), R.L[1], R.invL[1]);
    const double dz = min_image(__dsub_rn(A.z[j], A.z[i]), R.L[2], R.invL[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__device__ __forceinline__ bool owner_is(const RepDev &R, int ti_local, int tj_local)
{
    const uint32_t lo = (uint32_t)min(ti_local, tj_local), hi = (uint32_t)max(ti_local, tj_local);
    const U4 w = pair_draw(R, 0, kMhOwn, 0ll, lo, hi);
    const uint32_t owner = (w.x & 1u) ? hi : lo;
    return owner == (uint32_t)ti_local;
}

__device__ __forceinline__ bool is_bonded(const int4 &dp, int tag)
{
    return dp.x == tag || dp.y == tag || dp.z == tag || dp.w == tag;
}

// partner type of a particle of type t in reaction a
__device__ __forceinline__ int partner_type(const DevParams &P, int a, int t)
{
    return t == P.rx_ta[a] ? P.rx_tb[a] : P.rx_ta[a];
}

// number of particles of x's partner type inside x's formation window
__device__ int coord_count(const DevParams &P, const DevArrays &A, const RepDev &R, int a, int x)
{
    const int pt = partner_type(P, a, A.type[x]);
    const int nn = A.rnn[x];
    int c = 0;
    for (int k = 0; k < nn; ++k) {
        const int y = A.rnbr[(long long)k * P.nbr_stride + x];
        if (A.type[y] != pt) continue;
        const double r2 = exact_r2(A, R, x, y);
        if (r2 >= P.rx_rmin2[a] && r2 <= P.rx_rmax2[a]) ++c;
    }
    return c;
}

// Twelve pair features (see include/snap.h), with effective occupancies.
__device__ void pair_features(const DevParams &P, const DevArrays &A, int a, int i, int j, int occ_i,
                              int occ_j, int coord_i, int coord_j, double r, float *f)
{
    const int ti = A.type[i], tj = A.type[j];
    const double r0 = P.br0[P.rx_bt[a]];
    const double rmax = sqrt(P.rx_rmax2[a]);
    const float vi = (float)max(P.valence[ti], 1), vj = (float)max(P.valence[tj], 1);
    f[0] = (float)r;
    f[1] = (float)((r - r0) / rmax);
    f[2] = ti == P.rx_ta[a] ? 1.f : 0.f;
    f[3] = ti == P.rx_tb[a] ? 1.f : 0.f;
    f[4] = tj == P.rx_ta[a] ? 1.f : 0.f;
    f[5] = tj == P.rx_tb[a] ? 1.f : 0.f;
    f[6] = (float)occ_i / vi;
    f[7] = (float)occ_j / vj;
    f[8] = occ_i < P.valence[ti] ? 1.f : 0.f;
    f[9] = occ_j < P.valence[tj] ? 1.f : 0.f;
    f[10] = (float)coord_i * 0.125f;
    f[11] = (float)coord_j * 0.125f;
}

// Candidates of i in ascending tag order: compatible, free (freed counts as
// free and unbonded), not bonded to i, inside the window; owned by i when
// 'owned'.  Stores up to kMhCand (index, r); returns the full count.
__device__ int candidates(const DevParams &P, const DevArrays &A, const RepDev &R, int a, int i, int freed,
                          bool owned, int *ci, double *cr)
{
    const int ti = A.type[i];
    const int4 dp = A.dp[i];
    const int tag_i = A.tag[i];
    const int nn = A.rnn[i];
    int n = 0;
    for (int k = 0; k < nn; ++k) {
        const int j = A.rnbr[(long long)k * P.nbr_stride + i];
        const int tj = A.type[j];
        const bool compat = (ti == P.rx_ta[a] && tj == P.rx_tb[a]) || (ti == P.rx_tb[a] && tj == P.rx_ta[a]);
        if (!compat) continue;
        const int tag_j = A.tag[j];
        if (j != freed) {
            if (A.occ[j] >= P.valence[tj]) continue;
            if (is_bonded(dp, tag_j)) continue;
        }
        if (owned && !owner_is(R, tag_i - (int)R.tag_off, tag_j - (int)R.tag_off)) continue;
        const double r2 = exact_r2(A, R, i, j);
        if (r2 < P.rx_rmin2[a] || r2 > P.rx_rmax2[a]) continue;
        if (n < kMhCand) {
            // insertion by tag
            int s = n;
            while (s > 0 && A.tag[ci[s - 1]] > tag_j) {
                ci[s] = ci[s - 1];
                cr[s] = cr[s - 1];
                --s;
            }
            ci[s] = j;
            cr[s] = __dsqrt_rn(r2);
        }
        ++n;
    }
    return n;
}

// owned in-window bonds of i (slots are in ascending partner tag)
__device__ int breakable(const DevParams &P, const DevArrays &A, const RepDev &R, int a, int i, int *bj,
                         double *br)
{
    const int4 dp = A.dp[i];
    const int drx = A.drx[i];
    const int pv[4] = {dp.x, dp.y, dp.z, dp.w};
    const int tag_i = A.tag[i];
    int b = 0;
    for (int s = 0; s < kVmax; ++s) {
        const int p = pv[s];
        if (p < 0 || ((drx >> (8 * s)) & 0xFF) != a) continue;
        if (!owner_is(R, tag_i - (int)R.tag_off, p - (int)R.tag_off)) continue;
        const int j = A.rtag[p];
        const double r2 = exact_r2(A, R, i, j);
        if (r2 < P.rx_rmin2[a] || r2 > P.rx_rmax2[a]) continue;
        bj[b] = j;
        br[b] = __dsqrt_rn(r2);
        ++b;
    }
    return b;
}

// Eq. 3 factor exp(-U_b/kT) (kT = 0: [U_b <= 0]), as in the sweep
__device__ __forceinline__ double bond_factor_exact(const DevParams &P, const RepDev &R, int a, double r)
{
    const int bt = P.rx_bt[a];
    const double dr = __dsub_rn(r, P.br0[bt]);
    const double U = __dmul_rn(__dmul_rn(__dmul_rn(0.5, P.bk[bt]), dr), dr);
    if (R.kT > 0.0) return exp_cw(-__ddiv_rn(U, R.kT));
    return (U <= 0.0) ? 1.0 : 0.0;
}

// --------------------------------------------------------------- MH cells
template <bool FORCED>
__global__ void k_mh_key(DevParams P, DevArrays A)
{
    long long step;
    if (!mh_active<FORCED>(P, A, step)) return;
    const long long i = gtid();
    if (i == 0 && A.mv_rows) *A.mv_rows = 0;   // the learned proposal's row count restarts every sweep
    if (i >= P.n) return;
    const int t = A.type[i];
    A.mh_key[i] = -1;
    if (!((t == P.rx_ta[0] || t == P.rx_tb[0]) && P.valence[t] > 0)) return;
    const RepDev &R = A.reps[0];
    const double xs[3] = {A.x[i], A.y[i], A.z[i]};
    int c3[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double x = xs[d];
        if (!(x >= 0.0 && x < R.L[d])) x = __dsub_rn(x, __dmul_rn(R.L[d], floor(__dmul_rn(x, R.invL[d]))));
        int c = (int)__dmul_rn(__dmul_rn(x, R.invL[d]), (double)R.mh_nc[d]);
        c = min(max(c, 0), R.mh_nc[d] - 1);
        c3[d] = c;
    }
    const int key = (c3[2] * R.mh_nc[1] + c3[1]) * R.mh_nc[0] + c3[0];
    A.mh_key[i] = key;
    atomicAdd(&A.mh_count[key], 1);
}

template <bool FORCED>
__global__ void k_mh_scatter(DevParams P, DevArrays A)
{
    long long step;
    if (!mh_active<FORCED>(P, A, step)) return;
    const long long i = gtid();
    if (i >= P.n) return;
    const int key = A.mh_key[i];
    if (key < 0) return;
    A.mh_order[A.mh_start[key] + atomicAdd(&A.mh_cursor[key], 1)] = (int)i;
}

template <bool FORCED>
__global__ void k_mh_sort(DevParams P, DevArrays A)
{
    long long step;
    if (!mh_active<FORCED>(P, A, step)) return;
    const long long c = gtid();
    if (c >= P.mh_cells) return;
    const int s = A.mh_start[c], e = A.mh_start[c + 1];
    for (int k = s + 1; k < e; ++k) {
        const int v = A.mh_order[k];
        const int tv = A.tag[v];
        int m = k - 1;
        while (m >= s && A.tag[A.mh_order[m]] > tv) {
            A.mh_order[m + 1] = A.mh_order[m];
            --m;
        }
        A.mh_order[m + 1] = v;
    }
    A.mh_count[c] = 0;
    A.mh_cursor[c] = 0;
}

// ------------------------------------------------------------ selection
template <bool FORCED, bool LEARNED>
__global__ void __launch_bounds__(128) k_mh_select(DevParams P, DevArrays A)
{
    long long step;
    if (!mh_active<FORCED>(P, A, step)) return;
    const long long m = gtid();
    unsigned long long fa = 0, ba = 0;
    int nrow = 0;                         // candidate rows this move gives the network
    if (m < P.mh_moves) {
        const RepDev &R = A.reps[0];
        const int a = 0;
        const int hx = R.mh_nc[0] / 2, hy = R.mh_nc[1] / 2;
        const int col = (int)((unsigned long long)step & 7ull);
        const int mx = (int)(m % hx), my = (int)((m / hx) % hy), mz = (int)(m / ((long long)hx * hy));
        const int cx = 2 * mx + (col & 1), cy = 2 * my + ((col >> 1) & 1), cz = 2 * mz + ((col >> 2) & 1);
        const int c = (cz * R.mh_nc[1] + cy) * R.mh_nc[0] + cx;
        const int nc = A.mh_start[c + 1] - A.mh_start[c];
        int type = 0;
        if (nc > 0) {
            const U4 d1 = pair_draw(R, a, kMhSel, step, (uint32_t)c, 0u);
            const int i = A.mh_order[A.mh_start[c] + (int)(((unsigned long long)d1.x * (unsigned long long)nc) >> 32)];
            A.mv_i[m] = i;
            int *cand = A.mv_cand + m * kMhCand;
            double *cr = A.mv_r + m * kMhCand;
            if ((d1.y & 1u) == 0u) {
                ++fa;
                if (A.occ[i] < P.valence[A.type[i]]) {
                    const int n = candidates(P, A, R, a, i, -1, true, cand, cr);
                    if (n > 0 && n <= kMhCand) {
                        int bj[kVmax];
                        double br[kVmax];
                        A.mv_n[m] = n;
                        A.mv_b[m] = breakable(P, A, R, a, i, bj, br) + 1;
                        A.mv_c[m] = (int)(((unsigned long long)d1.z * (unsigned long long)n) >> 32);
                        type = 1;
                        nrow = n;
                    }
                }
            } else {
                ++ba;
                int bj[kVmax];
                double br[kVmax];
                const int b = breakable(P, A, R, a, i, bj, br);
                if (b > 0) {
                    const int pick = (int)(((unsigned long long)d1.z * (unsigned long long)b) >> 32);
                    const int j = bj[pick];
                    // candidates of i in the state without the bond i-j
                    const int n2 = candidates(P, A, R, a, i, j, true, cand, cr);
                    if (n2 <= kMhCand) {
                        int idx = 0;
                        for (int k = 0; k < n2; ++k)
                            if (cand[k] == j) idx = k;
                        A.mv_j[m] = j;
                        A.mv_n[m] = n2;
                        A.mv_b[m] = b;
                        A.mv_c[m] = idx;
                        cr[idx] = br[pick];
                        type = 2;
                        nrow = n2;
                    }
                }
            }
        }
        A.mv_type[m] = type;
    }
    if (LEARNED) {
        // Rows of live moves only, packed: one reservation per warp (moves with
        // no candidate row give the network nothing to score); a row's logit
        // depends on its own features alone, so where it lands does not matter.
        int incl = nrow;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        int base = 0;
        if (lane == 31 && total > 0) base = atomicAdd(A.mv_rows, total);
        base = __shfl_sync(0xFFFFFFFFu, base, 31);
        if (nrow > 0) A.mv_row0[m] = base + incl - nrow;
    }
    const int idx[2] = {cMhFormAtt, cMhBreakAtt};
    const unsigned long long v[2] = {fa, ba};
    warp_counts<2>(A.counters, idx, v);
}

// Features of the learned proposal's candidate rows, one warp per live move:
// the coordination counts of the initiator and of each candidate (partner-type
// particles inside the formation window, exact FP64 distances as everywhere in
// the sweep) are counted by the 32 lanes over the concatenated reactive lists
// of the n + 1 particles (a ballot per list and pass); lane k then writes
// candidate k's row.  (A thread per move counting n + 1 lists one entry at a
// time held the FP64 pipe with one lane active; walking the lists one after
// the other chained n + 1 dependent load sequences.)
template <bool FORCED>
__global__ void __launch_bounds__(128) k_mh_features(DevParams P, DevArrays A)
{
    long long step;
    if (!mh_active<FORCED>(P, A, step)) return;
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    const RepDev &R = A.reps[0];
    const int a = 0;
    for (long long m = gtid() >> 5; m < P.mh_moves; m += nw) {
        const int type = A.mv_type[m];
        if (type == 0) continue;                         // uniform over the warp
        const int i = A.mv_i[m], n = A.mv_n[m], row0 = A.mv_row0[m];
        const int jb = type == 2 ? A.mv_j[m] : -1;       // break: features of the state without i-j
        const int *cand = A.mv_cand + m * kMhCand;
        // the n + 1 reactive lists (list 0: i's, list q: candidate q's), held by
        // lanes 0..n and concatenated: the warp's lanes walk all their entries
        // together, 32 per pass, instead of one list after the other
        int x = -1, len = 0, pt = -1;
        if (lane <= n) {
            x = lane == 0 ? i : cand[lane - 1];
            len = A.rnn[x];
            pt = partner_type(P, a, A.type[x]);
        }
        int off = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, off, o);
            if (lane >= o) off += t;
        }
        const int total = __shfl_sync(0xFFFFFFFFu, off, 31);
        off -= len;                                      // first entry of list `lane`
        int my_cnt = 0;                                  // lane q <= n: list q's count
        for (int e0 = 0; e0 < total; e0 += 32) {
            const int e = e0 + lane;
            int p = 0;                                   // the list of entry e: the last q with off_q <= e
            for (int q = 1; q <= n; ++q)
                if (__shfl_sync(0xFFFFFFFFu, off, q) <= e) p = q;
            const int xp = __shfl_sync(0xFFFFFFFFu, x, p);
            const int ptp = __shfl_sync(0xFFFFFFFFu, pt, p);
            const int k = e - __shfl_sync(0xFFFFFFFFu, off, p);
            bool hit = false;
            if (e < total) {
                const int y = A.rnbr[(long long)k * P.nbr_stride + xp];
                if (A.type[y] == ptp) {
                    const double r2 = exact_r2(A, R, xp, y);
                    hit = r2 >= P.rx_rmin2[a] && r2 <= P.rx_rmax2[a];
                }
            }
            for (int q = 0; q <= n; ++q) {
                const unsigned bq = __ballot_sync(0xFFFFFFFFu, hit && p == q);
                if (lane == q) my_cnt += __popc(bq);
            }
        }
        const int ci = __shfl_sync(0xFFFFFFFFu, my_cnt, 0);
        const int my_c = __shfl_sync(0xFFFFFFFFu, my_cnt, (lane + 1) & 31);   // candidate `lane`'s list
        if (lane < n) {
            const int q = cand[lane];
            const int oi = type == 2 ? A.occ[i] - 1 : A.occ[i];
            const int oq = A.occ[q] - (q == jb ? 1 : 0);
            pair_features(P, A, a, i, q, oi, oq, ci, my_c, A.mv_r[m * kMhCand + lane],
                          A.mv_feat + (long long)(row0 + lane) * kMlpFeatures);
        }
    }
}

// proposal probability of candidate k among n (softmax mixture or uniform)
template <bool LEARNED>
__device__ __forceinline__ double proposal_prob(const DevParams &P, const float *logit, int n, int k)
{
    if (!LEARNED) return 1.0 / (double)n;
    float mx = logit[0];
    for (int c = 1; c < n; ++c) mx = fmaxf(mx, logit[c]);
    double z = 0.0;
    for (int c = 0; c < n; ++c) z += exp((double)(logit[c] - mx));
    const double eps = (double)P.mh_eps;
    return (1.0 - eps) * exp((double)(logit[k] - mx)) / z + eps / (double)n;
}

__device__ void slot_insert(DevArrays &A, int i, int ptag, int a, long long step)
{
    const int4 dp = A.dp[i];
    const int4 db = A.dbirth[i];
    const int drx = A.drx[i];
    int np[4] = {dp.x, dp.y, dp.z, dp.w}, nb[4] = {db.x, db.y, db.z, db.w};
    int nr[4] = {drx & 0xFF, (drx >> 8) & 0xFF, (drx >> 16) & 0xFF, (drx >> 24) & 0xFF};
    int m = 0;
    while (m < 4 && np[m] >= 0) ++m;
    int s = m;
    while (s > 0 && np[s - 1] > ptag) {
        np[s] = np[s - 1]; nb[s] = nb[s - 1]; nr[s] = nr[s - 1];
        --s;
    }
    np[s] = ptag; nb[s] = (int)(uint32_t)step; nr[s] = a;
    A.dp[i] = make_int4(np[0], np[1], np[2], np[3]);
    A.dbirth[i] = make_int4(nb[0], nb[1], nb[2], nb[3]);
    A.drx[i] = (nr[0] & 0xFF) | ((nr[1] & 0xFF) << 8) | ((nr[2] & 0xFF) << 16) | ((nr[3] & 0xFF) << 24);
    A.occ[i] = m + 1;
}

// removes partner ptag from i's slots; returns the birth step of that bond
__device__ int slot_remove(DevArrays &A, int i, int ptag)
{
    const int4 dp = A.dp[i];
    const int4 db = A.dbirth[i];
    const int drx = A.drx[i];
    const int pv[4] = {dp.x, dp.y, dp.z, dp.w}, bv[4] = {db.x, db.y, db.z, db.w};
    int np[4] = {-1, -1, -1, -1}, nb[4] = {0, 0, 0, 0}, nr[4] = {0, 0, 0, 0};
    int m = 0, birth = 0;
    for (int s = 0; s < 4; ++s) {
        if (pv[s] < 0) continue;
        if (pv[s] == ptag) {
            birth = bv[s];
            continue;
        }
        np[m] = pv[s]; nb[m] = bv[s]; nr[m] = (drx >> (8 * s)) & 0xFF;
        ++m;
    }
    A.dp[i] = make_int4(np[0], np[1], np[2], np[3]);
    A.dbirth[i] = make_int4(nb[0], nb[1], nb[2], nb[3]);
    A.drx[i] = (nr[0] & 0xFF) | ((nr[1] & 0xFF) << 8) | ((nr[2] & 0xFF) << 16) | ((nr[3] & 0xFF) << 24);
    A.occ[i] = m;
    return birth;
}

template <bool FORCED, bool LEARNED>
__global__ void __launch_bounds__(128) k_mh_decide(DevParams P, DevArrays A)
{
    long long step;
    if (!mh_active<FORCED>(P, A, step)) return;
    const long long m = gtid();
    unsigned long long facc = 0, bacc = 0, nbroken = 0, nformed = 0;
    if (m < P.mh_moves && A.mv_type[m] != 0) {
        const RepDev &R = A.reps[0];
        const int a = 0;
        const int type = A.mv_type[m];
        const int i = A.mv_i[m], n = A.mv_n[m], b = A.mv_b[m];
        const int hx = R.mh_nc[0] / 2, hy = R.mh_nc[1] / 2;
        const int col = (int)((unsigned long long)step & 7ull);
        const int mx = (int)(m % hx), my = (int)((m / hx) % hy), mz = (int)(m / ((long long)hx * hy));
        const int c = ((2 * mz + ((col >> 2) & 1)) * R.mh_nc[1] + (2 * my + ((col >> 1) & 1))) * R.mh_nc[0] +
                      (2 * mx + (col & 1));
        const U4 d1 = pair_draw(R, a, kMhSel, step, (uint32_t)c, 0u);
        const U4 d2 = pair_draw(R, a, kMhAcc, step, (uint32_t)c, 0u);
        const double u = u53(d2.x, d2.y);
        const double K = __ddiv_rn(R.p_on0[a], R.p_off[a]);
        const float *logit = LEARNED ? A.mv_logit + A.mv_row0[m] : nullptr;
        if (type == 1) {
            int k = A.mv_c[m];
            double pk = 0.0;
            if (LEARNED) {
                // draw from the mixture with a 53-bit uniform; the softmax's max and
                // normaliser once per move, each candidate's probability as
                // proposal_prob evaluates it (the same operations, so the same value)
                const double us = u53(d1.z, d1.w);
                float mxl = logit[0];
                for (int cc = 1; cc < n; ++cc) mxl = fmaxf(mxl, logit[cc]);
                double z = 0.0;
                for (int cc = 0; cc < n; ++cc) z += exp((double)(logit[cc] - mxl));
                const double eps = (double)P.mh_eps;
                double acc = 0.0;
                k = n - 1;
                for (int cc = 0; cc < n; ++cc) {
                    const double pc = (1.0 - eps) * exp((double)(logit[cc] - mxl)) / z + eps / (double)n;
                    acc += pc;
                    pk = pc;
                    if (us < acc) {
                        k = cc;
                        break;
                    }
                }
            }
            const int j = A.mv_cand[m * kMhCand + k];
            const double e = bond_factor_exact(P, R, a, A.mv_r[m * kMhCand + k]);
            double ratio;
            if (LEARNED)
                ratio = __ddiv_rn(__dmul_rn(K, e), __dmul_rn((double)b, pk));
            else
                ratio = __ddiv_rn(__dmul_rn(__dmul_rn(K, e), (double)n), (double)b);
            if (u < ratio) {
                slot_insert(A, i, A.tag[j], a, step);
                slot_insert(A, j, A.tag[i], a, step);
                ++facc;
                ++nformed;
            }
        } else {
            const int j = A.mv_j[m];
            const int k = A.mv_c[m];
            const double e = bond_factor_exact(P, R, a, A.mv_r[m * kMhCand + k]);
            double ratio;
            if (LEARNED)
                ratio = __ddiv_rn(__dmul_rn((double)b, proposal_prob<true>(P, logit, n, k)), __dmul_rn(K, e));
            else
                ratio = __ddiv_rn((double)b, __dmul_rn((double)n, __dmul_rn(K, e)));
            if (u < ratio) {
                const int birth = slot_remove(A, i, A.tag[j]);
                slot_remove(A, j, A.tag[i]);
                long long life = (long long)((uint32_t)step - (uint32_t)birth) / P.period;
                if (life >= P.nhist) life = P.nhist - 1;
                atomicAdd(&A.life_hist[life], 1ull);
                ++bacc;
                ++nbroken;
            }
        }
    }
    const int idx[4] = {cMhFormAcc, cMhBreakAcc, cFormedTotal, cBrokenTotal};
    const unsigned long long v[4] = {facc, bacc, nformed, nbroken};
    warp_counts<4>(A.counters, idx, v);
}

// ------------------------------------------------------------ event log
// After the acceptance phase of a plain sweep: every site whose own proposal
// formed a bond records the features of all its candidates (state before the
// sweep's changes) and the index of the partner it formed with.
template <bool FORCED>
__global__ void k_log_events(DevParams P, DevArrays A, int slot)
{
    long long step;
    if (!mh_active<FORCED>(P, A, step)) return;
    unsigned long long logged = 0;
    for (long long i = gtid(); i < P.n; i += (long long)gridDim.x * blockDim.x) {
        const int j = A.prop[(int)i];
        if (j < 0 || A.fpart[i] != j) continue;
        const int rp = rep_of(P, A, i);
        const int a = rx_at(P, A, rp, slot);
        const RepDev &R = A.reps[rp];
        int ci[kMhCand];
        double cr[kMhCand];
        const int n = candidates(P, A, R, a, i, -1, false, ci, cr);
        if (n == 0 || n > kMhCand) continue;
        int lab = -1;
        for (int k = 0; k < n; ++k)
            if (ci[k] == j) lab = k;
        if (lab < 0) continue;
        const int e = atomicAdd(A.ev_count, 1);
        ++logged;
        if (e >= A.ev_cap) continue;
        const int coord_i = coord_count(P, A, R, a, i);
        for (int k = 0; k < n; ++k)
            pair_features(P, A, a, i, ci[k], A.occ[i], A.occ[ci[k]], coord_i, coord_count(P, A, R, a, ci[k]),
                          cr[k], A.ev_feat + ((long long)e * kMhCand + k) * kMlpFeatures);
        A.ev_n[e] = n;
        A.ev_label[e] = lab;
    }
    const int idx[1] = {cEvents};
    const unsigned long long v[1] = {logged};
    warp_counts<1>(A.counters, idx, v);
}

inline unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }

}  // namespace

void launch_mh_sweep(const DevParams &P, const DevArrays &A, bool forced, const MlpDev *mlp, int32_t *bsum,
                     Launch L)
{
    if (P.n == 0 || P.mh_moves == 0) return;
    const unsigned g = grid_for(P.n, L.block);
    if (forced) k_mh_key<true><<<g, L.block, 0, L.stream>>>(P, A);
    else k_mh_key<false><<<g, L.block, 0, L.stream>>>(P, A);
    launch_scan(A.mh_count, A.mh_start, bsum, P.mh_cells, A.mh_gate, A.status, L);
    if (forced) {
        k_mh_scatter<true><<<g, L.block, 0, L.stream>>>(P, A);
        k_mh_sort<true><<<grid_for(P.mh_cells, 128), 128, 0, L.stream>>>(P, A);
    } else {
        k_mh_scatter<false><<<g, L.block, 0, L.stream>>>(P, A);
        k_mh_sort<false><<<grid_for(P.mh_cells, 128), 128, 0, L.stream>>>(P, A);
    }
    const unsigned gm = grid_for(P.mh_moves, 128);
    if (mlp) {
        if (forced) k_mh_select<true, true><<<gm, 128, 0, L.stream>>>(P, A);
        else k_mh_select<false, true><<<gm, 128, 0, L.stream>>>(P, A);
        const unsigned gf = (unsigned)std::min<long long>((P.mh_moves + 3) / 4, 148LL * 16);
        if (forced) k_mh_features<true><<<gf, 128, 0, L.stream>>>(P, A);
        else k_mh_features<false><<<gf, 128, 0, L.stream>>>(P, A);
        mlp_forward_counted(*mlp, A.mv_feat, A.mv_rows, (long long)P.mh_moves * kMhCand, A.mv_logit, L.stream);
        if (forced) k_mh_decide<true, true><<<gm, 128, 0, L.stream>>>(P, A);
        else k_mh_decide<false, true><<<gm, 128, 0, L.stream>>>(P, A);
    } else {
        if (forced) k_mh_select<true, false><<<gm, 128, 0, L.stream>>>(P, A);
        else k_mh_select<false, false><<<gm, 128, 0, L.stream>>>(P, A);
        if (forced) k_mh_decide<true, false><<<gm, 128, 0, L.stream>>>(P, A);
        else k_mh_decide<false, false><<<gm, 128, 0, L.stream>>>(P, A);
    }
}

void launch_log_events(const DevParams &P, const DevArrays &A, int slot, bool forced, Launch L)
{
    if (P.n == 0) return;
    if (forced) k_log_events<true><<<296, 128, 0, L.stream>>>(P, A, slot);
    else k_log_events<false><<<296, 128, 0, L.stream>>>(P, A, slot);
}

}  // namespace snap
