// Cell list, row-ordered particle sort and the two neighbour lists.
//
// Layout: particles are sorted by (type, rank of their cell, sub-cell along x,
// tag), with cells of side >= the largest neighbour cut-off, ranked x
// innermost and rows in 2-D Morton order of (y, z), each cell cut into 2^s
// slices along x.  Within one type the 27 cells around a particle are nearby
// in memory, so neighbour gathers hit L1/L2, the cells x-1..x+1 of a row (and
// so any run of their slices) are one run of the sorted particles, and a warp
// holds particles of one type, so its lanes do similar work (a colloid has ~2x
// the neighbours of a linker).  The rebuild also stores, per particle, the
// coordinate relative to the origin of its cell (frozen until the next
// rebuild) with the cell coordinates and type packed in the w word, which the
// force loop uses.
#include <algorithm>

#include "snap_kernels.h"

namespace snap {

namespace {

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }

inline unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }

// Cell of a wrapped position, in FP32 (one conversion per axis on the FP64
// pipe instead of five FP64 operations): the cell may be off by one within
// ~1e-4 of a cell face, which the cell size margin absorbs.  The rebuild uses
// this one function for the sort key and for the frozen cell bits.
__device__ __forceinline__ void cell_of(const RepDev &R, double x, double y, double z, int &cx, int &cy,
                                        int &cz)
{
    cx = (int)((float)x * R.cscale[0]);
    cy = (int)((float)y * R.cscale[1]);
    cz = (int)((float)z * R.cscale[2]);
    cx = min(max(cx, 0), R.nc[0] - 1);
    cy = min(max(cy, 0), R.nc[1] - 1);
    cz = min(max(cz, 0), R.nc[2] - 1);
}

// Sub-cell along x: every cell is cut into 2^s slices of equal width along x
// for the sort and the list build.  The scale is the cell scale times 2^s,
// exact in FP32, so that sx >> s is the cell cx that cell_of gives for the
// same coordinate (clamps included).
__device__ __forceinline__ int subcell_x(const RepDev &R, double x, int s)
{
    const float v = (float)x * (R.cscale[0] * (float)(1 << s));
    return (int)fminf(fmaxf(v, 0.f), (float)((R.nc[0] << s) - 1));   // truncation = floor for v >= 0
}

// wrap into [0, L) and count the crossing in the image counter
__device__ __forceinline__ double wrap_img(double x, double L, int &img)
{
    if (x >= L) {
        x -= L;
        img += 1;
    } else if (x < 0.0) {
        x += L;
        img -= 1;
        if (x >= L) {
            x -= L;
            img += 1;
        }
    }
    return x;
}

__global__ void k_cell_key(DevParams P, DevArrays A)
{
    const long long i = gtid();
    if (i == 0) counter_add1(A.counters, cRebuildLaunches, 1ull);   // launches, taken or not
    if (i >= P.n) return;
    if (!status_ok(A.status) || !*A.need_rebuild) return;
    const RepDev &R = A.reps[rep_of(P, A, i)];
    double x = A.x[i], y = A.y[i], z = A.z[i];
    // inside [0, L) on every axis? (non-negative doubles order like their bits)
    const long long bx = __double_as_longlong(x), by = __double_as_longlong(y), bz = __double_as_longlong(z);
    if (!(bx >= 0 && bx < __double_as_longlong(R.L[0]) && by >= 0 && by < __double_as_longlong(R.L[1]) &&
          bz >= 0 && bz < __double_as_longlong(R.L[2]))) {
        int ix = A.ix[i], iy = A.iy[i], iz = A.iz[i];
        x = wrap_img(x, R.L[0], ix);
        y = wrap_img(y, R.L[1], iy);
        z = wrap_img(z, R.L[2], iz);
        A.x[i] = x; A.y[i] = y; A.z[i] = z;
        A.ix[i] = ix; A.iy[i] = iy; A.iz[i] = iz;
    }
    int cx, cy, cz;
    cell_of(R, x, y, z, cx, cy, cz);
    // rank of the row's first cell: the row's cells, and so its sub-cells, follow it in x order
    const int row = A.rank_of[R.cell_off + (cz * R.nc[1] + cy) * R.nc[0]];
    const int c = ((A.type[i] * P.ncell + row) << P.sub_shift) + subcell_x(R, x, P.sub_shift);
    A.cell_key[i] = c;
    // particles are still nearly sorted: lanes of a warp mostly share a key,
    // so one atomic per distinct key and warp
    const unsigned peers = __match_any_sync(__activemask(), c);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&A.cell_count[c], __popc(peers));
    if (i == 0) {
        counter_reset(A.counters, cNlistEntries);
        counter_reset(A.counters, cRnlistEntries);
    }
}

// three-phase exclusive scan of cell_count into cell_start[0..ncell]
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int &total)
{
    constexpr int NW = kScanThreads / 32;
    __shared__ int warp_sums[NW];
    __shared__ int tot;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = lane < NW ? warp_sums[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NW) warp_sums[lane] = wi - w;
        if (lane == NW - 1) tot = wi;
    }
    __syncthreads();
    const int res = incl - v + warp_sums[wid];
    total = tot;
    __syncthreads();
    return res;
}

__global__ void k_scan_tiles(const int32_t *in, int32_t *out, int32_t *bsum, int n, const int32_t *gate,
                             const uint32_t *status)
{
    if (!status_ok(status) || !*gate) return;
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int total;
    int run = block_exclusive_scan(s, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void k_scan_sums(int32_t *bsum, int nb, const int32_t *gate, const uint32_t *status)
{
    if (!status_ok(status) || !*gate) return;
    // one block; nb <= kScanTile
    const int base = threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < nb) ? bsum[base + k] : 0;
        s += v[k];
    }
    int total;
    int run = block_exclusive_scan(s, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < nb) bsum[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) bsum[nb] = total;
}

__global__ void k_scan_add(int32_t *out, const int32_t *bsum, int n, int nb, const int32_t *gate,
                           const uint32_t *status)
{
    if (!status_ok(status) || !*gate) return;
    const long long k = gtid();
    if (k < n) out[k] += bsum[k / kScanTile];
    if (k == 0) out[n] = bsum[nb];
}

// The cell scan leaves in cell_start each key's exclusive prefix within its
// tile of kScanTile keys and in bsum the tiles' offsets; the scatter adds the
// offset itself, and the cell sort (one thread per key) writes the final start.
__global__ void k_scatter(DevParams P, DevArrays A, const int32_t *bsum)
{
    const long long i = gtid();
    if (i >= P.n) return;
    if (!status_ok(A.status) || !*A.need_rebuild) return;
    const int c = A.cell_key[i];
    // one atomic per distinct key and warp; lanes take consecutive slots
    const unsigned peers = __match_any_sync(__activemask(), c);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&A.cell_cursor[c], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int pos = A.cell_start[c] + bsum[c / kScanTile] + base + __popc(peers & ((1u << lane) - 1u));
    A.order[pos] = (int32_t)i;
}

// deterministic order inside a cell: ascending tag (insertion sort, cells are
// small); then the cell's final start (each thread reads and writes only its
// own key's entries)
__global__ void k_cell_sort(DevArrays A, int ncell, const int32_t *bsum)
{
    const long long c = gtid();
    if (c >= ncell) return;
    if (!status_ok(A.status) || !*A.need_rebuild) return;
    const int s = A.cell_start[c] + bsum[c / kScanTile], e = s + A.cell_count[c];
    for (int k = s + 1; k < e; ++k) {
        const int v = A.order[k];
        const int tv = A.tag[v];
        int m = k - 1;
        while (m >= s && A.tag[A.order[m]] > tv) {
            A.order[m + 1] = A.order[m];
            --m;
        }
        A.order[m + 1] = v;
    }
    A.cell_start[c] = s;
    if (c == ncell - 1) A.cell_start[ncell] = e;
    A.cell_count[c] = 0;
    A.cell_cursor[c] = 0;
}

template <typename R>
__global__ void k_gather(DevParams P, DevArrays A, DevArrays B)
{
    using V = typename Vec4<R>::T;
    const long long k = gtid();
    if (k >= P.n) return;
    if (!status_ok(A.status) || !*A.need_rebuild) return;
    if (k == 0) *A.gathered = 1;
    const int i = A.order[k];
    const double x = A.x[i], y = A.y[i], z = A.z[i];
    B.x[k] = x; B.y[k] = y; B.z[k] = z;
    if (sizeof(R) == 8) {
        B.vx[k] = A.vx[i]; B.vy[k] = A.vy[i]; B.vz[k] = A.vz[i];
    } else {
        B.v4[k] = A.v4[i];
    }
    B.ix[k] = A.ix[i]; B.iy[k] = A.iy[i]; B.iz[k] = A.iz[i];
    const int t = A.type[i];
    B.type[k] = t;
    const int tag = A.tag[i];
    B.tag[k] = tag;
    const int rp = rep_of(P, A, i);
    if (P.nrep > 1) B.rep[k] = rp;                  // one system: rep is all zeros and stays so
    if (P.has_static) {
        B.sp[k] = A.sp[i];
        B.sbt[k] = A.sbt[i];
    }
    B.dp[k] = A.dp[i]; B.drx[k] = A.drx[i]; B.dbirth[k] = A.dbirth[i];
    B.occ[k] = A.occ[i];
    A.rtag[tag] = (int32_t)k;
    const RepDev &Rp = A.reps[rp];
    int cx, cy, cz;
    cell_of(Rp, x, y, z, cx, cy, cz);
    const double o0 = (double)cx * Rp.w[0], o1 = (double)cy * Rp.w[1], o2 = (double)cz * Rp.w[2];
    const double rx = x - o0;
    const double ry = y - o1;
    const double rz = z - o2;
    V p;
    p.x = (R)rx; p.y = (R)ry; p.z = (R)rz;
    set_w_bits(p, pack_bits(t, cx, cy, cz));
    reinterpret_cast<V *>(B.pos4)[k] = p;
    A.ref4[k] = make_float4((float)rx, (float)ry, (float)rz, 0.f);
    A.npos[k] = make_float4((float)x, (float)y, (float)z, __uint_as_float(pack_bits(t, cx, cy, cz)));
}

// The gathered particle k copied back from the scratch arrays B into A (run
// by the list build, which reads none of these arrays, at the end of each
// thread's scan: the streaming copy overlaps the latency-bound list work
// instead of taking a kernel of its own).
template <typename R>
__device__ __forceinline__ void copyback_particle(const DevParams &P, DevArrays &A, const DevArrays &B, long long k)
{
    // streaming loads (__ldcs, evicted first): the L1 keeps the candidates'
    // coordinates that the list scans read
    using V = typename Vec4<R>::T;
    A.x[k] = __ldcs(B.x + k); A.y[k] = __ldcs(B.y + k); A.z[k] = __ldcs(B.z + k);
    if (sizeof(R) == 8) {
        A.vx[k] = __ldcs(B.vx + k); A.vy[k] = __ldcs(B.vy + k); A.vz[k] = __ldcs(B.vz + k);
    } else {
        A.v4[k] = __ldcs(B.v4 + k);
    }
    A.ix[k] = __ldcs(B.ix + k); A.iy[k] = __ldcs(B.iy + k); A.iz[k] = __ldcs(B.iz + k);
    A.type[k] = __ldcs(B.type + k); A.tag[k] = __ldcs(B.tag + k);
    if (P.nrep > 1) A.rep[k] = __ldcs(B.rep + k);
    if (P.has_static) {
        A.sp[k] = __ldcs(B.sp + k);
        A.sbt[k] = __ldcs(B.sbt + k);
    }
    A.dp[k] = __ldcs(B.dp + k); A.drx[k] = __ldcs(B.drx + k); A.dbirth[k] = __ldcs(B.dbirth + k);
    A.occ[k] = __ldcs(B.occ + k);
    if (sizeof(R) == 8) {
        const double4_32a *src = reinterpret_cast<const double4_32a *>(B.pos4);
        reinterpret_cast<double4_32a *>(A.pos4)[k] = src[k];
    } else {
        reinterpret_cast<float4 *>(A.pos4)[k] = __ldcs(reinterpret_cast<const float4 *>(B.pos4) + k);
    }
}

// Two neighbour lists, column-major (entry k of particle i at k * stride + i):
// the force list holds every j != i with r^2 < (pair cut + skin + margin)^2
// of the type pair, the reactive list every j of a reaction-compatible type
// with r^2 < (r_max + skin + margin)^2.  The force loop then never visits
// pairs that are only within reach of a bond, and the sweep never visits
// pairs that cannot bond.  Cells are ranked row by row (x innermost, rows in
// 2-D Morton order of (y, z)), and every cell is cut into 2^sub_shift slices
// along x (sub-cells, sorted in x order), so for each of the 9 rows around a
// particle and each type the candidates are one contiguous run of the sorted
// particles: 18 candidate runs per particle instead of 54 single cells.  A
// row is admitted when the particle's distance to the row's (y, z) box is
// below the larger of the two cut-offs of the type pair, and within the row
// only the sub-cells that overlap the x window that distance leaves are
// scanned, so short-ranged pairs (small spheres) and far rows test few
// candidates (on the colloid-linker gel 4 slices per cell cut the candidates
// per particle from ~89 to ~60, 8 slices to ~54).  Separations come from the FP32 wrapped positions
// the rebuild stored (npos) plus a periodic shift per run; their error (a few
// units in the last place of the box edge) is inside the list margin, and the
// lists only need to hold every pair within reach.  (A warp-per-cell variant
// that tests every candidate of the 27 cells against each home particle ran
// 1.8x slower on the colloid-linker gel: without the per-particle culling it
// tests ~4x more pairs.)
// Candidates s0..e-1 against particle i, appended to the force list (F)
// and/or the reactive list (X).  (Two candidates per pass, or running slot
// pointers instead of slot arithmetic, measured no faster: the loop is bound
// by the lanes' different trip counts, not by its instruction count.)
template <bool F, bool X>
__device__ __forceinline__ int2 scan_range(const float4 *npos, int s0, int e, long long i, float ox, float oy,
                                           float oz, float fcut2, float xcut2, int *nbr, int *rnbr, long long stride,
                                           int cap, int rcap, int cnt, int rcnt)
{
    for (int j = s0; j < e; ++j) {
        if (j == i) continue;
        const float4 q = __ldg(npos + j);
        const float ddx = q.x + ox;
        const float ddy = q.y + oy;
        const float ddz = q.z + oz;
        const float r2 = ddx * ddx + ddy * ddy + ddz * ddz;
        if (F && r2 < fcut2) {
            if (cnt < cap) nbr[(long long)cnt * stride + i] = j;
            ++cnt;
        }
        if (X && r2 < xcut2) {
            if (rcnt < rcap) rnbr[(long long)rcnt * stride + i] = j;
            ++rcnt;
        }
    }
    return make_int2(cnt, rcnt);
}

// a zero cut-off takes no pair (r^2 < 0 never holds): that list is skipped,
// the same for every lane of a type-pure warp
__device__ __forceinline__ int2 scan_lists(const float4 *npos, int s0, int e, long long i, float ox, float oy,
                                           float oz, float fcut2, float xcut2, int *nbr, int *rnbr, long long stride,
                                           int cap, int rcap, int2 c)
{
    if (xcut2 <= 0.f)
        return scan_range<true, false>(npos, s0, e, i, ox, oy, oz, fcut2, xcut2, nbr, rnbr, stride, cap, rcap, c.x,
                                       c.y);
    if (fcut2 <= 0.f)
        return scan_range<false, true>(npos, s0, e, i, ox, oy, oz, fcut2, xcut2, nbr, rnbr, stride, cap, rcap, c.x,
                                       c.y);
    return scan_range<true, true>(npos, s0, e, i, ox, oy, oz, fcut2, xcut2, nbr, rnbr, stride, cap, rcap, c.x, c.y);
}

// Slack of the x window of a row (squared and linear, length units): the row
// and sub-cell tests compare FP32 coordinates whose cell faces and roundings
// are off by ~1e-5 at the box sizes the cell bits allow.
constexpr float kWinSlack2 = 5e-4f;
constexpr float kWinSlack = 5e-4f;

template <typename R>
__global__ void __launch_bounds__(256, 8) k_nlist(DevParams P, DevArrays A, DevArrays B)
{
    // uniform: this rebuild's gather ran (the status was clear at its start).
    // Not the status itself: a block that overflows its list latches a status
    // bit, and every block must still copy its particles back.
    if (!*A.gathered) return;
    const long long i = gtid();
    int2 cc = make_int2(0, 0);
    const int cap = P.nbr_cap, rcap = P.rnbr_cap;
    if (i < P.n) {
        const float4 p = A.npos[i];
        const uint32_t b = __float_as_uint(p.w);
        const int ti = bits_type(b), cx = bits_cx(b), cy = bits_cy(b), cz = bits_cz(b);
        const RepDev &Rp = A.reps[rep_of(P, B, i)];   // B: the new order (A is copied back below)
        const int nx = Rp.nc[0], ny = Rp.nc[1], nz = Rp.nc[2];
        const float wy = Rp.wf[1], wz = Rp.wf[2];
        const float Lx = (float)Rp.L[0], Ly = (float)Rp.L[1], Lz = (float)Rp.L[2];
        const long long stride = P.nbr_stride;
        // distances to the faces of the home cell (the cell bits were taken from
        // the same wrapped position: the cell test admits at least what it must)
        const float ry = p.y - (float)cy * wy, rz = p.z - (float)cz * wz;
        const float gyl = fmaxf(ry, 0.f), gyu = fmaxf(wy - ry, 0.f);
        const float gzl = fmaxf(rz, 0.f), gzu = fmaxf(wz - rz, 0.f);
        const int sh = P.sub_shift, nsx = nx << sh;
        const float csk = Rp.cscale[0] * (float)(1 << sh);   // sub-cells per unit length along x
        const float xlo = (float)((cx - 1) << sh), xhi = (float)(((cx + 2) << sh) - 1);
        for (int dz = -1; dz <= 1; ++dz) {
            int zz = cz + dz;
            float oz = -p.z;
            if (zz < 0) { zz += nz; oz -= Lz; }
            if (zz >= nz) { zz -= nz; oz += Lz; }
            const float gz = dz < 0 ? gzl : (dz > 0 ? gzu : 0.f);
            for (int dy = -1; dy <= 1; ++dy) {
                int yy = cy + dy;
                float oy = -p.y;
                if (yy < 0) { yy += ny; oy -= Ly; }
                if (yy >= ny) { yy -= ny; oy += Ly; }
                const float gy = dy < 0 ? gyl : (dy > 0 ? gyu : 0.f);
                const float d2r = gy * gy + gz * gz;
                // rank of the row's cell x = 0: the row's cells follow it in x order
                const int row = __ldg(A.rank_of + Rp.cell_off + (zz * ny + yy) * nx);
                for (int t = 0; t < P.ntypes; ++t) {
                    const float fcut2 = P.fl2f[ti * kMaxTypes + t];
                    const float xcut2 = P.xl2f[ti * kMaxTypes + t];
                    const float cut = fmaxf(fcut2, xcut2);
                    if (d2r >= cut) continue;
                    // x window of the row: |dx|^2 < cut^2 - d2r, widened by slack that
                    // covers the FP32 cell faces and coordinates (~1e-5 here)
                    // (never beyond the cells x-1..x+1, which hold every pair within reach:
                    // this also bounds the indices of a particle whose coordinate has left
                    // the box by more than its edge, e.g. in an exploding system)
                    // (v * rsqrt(v): the approximate root is within a few ulp, far inside the slack)
                    const float v = cut - d2r + kWinSlack2;
                    const float wr = v * rsqrtf(v) + kWinSlack;
                    int xa = (int)fminf(fmaxf(floorf((p.x - wr) * csk), xlo), xhi);
                    int xb = (int)fminf(fmaxf(floorf((p.x + wr) * csk), xlo), xhi);
                    const int kb = (t * P.ncell + row) << sh;
                    // the part of the window across the periodic x boundary is its own
                    // run, kept clear of the main run
                    if (xa < 0) {
                        const int a = min(max(xa + nsx, xb + 1), nsx);
                        cc = scan_lists(A.npos, __ldg(A.cell_start + kb + a), __ldg(A.cell_start + kb + nsx), i,
                                        -p.x - Lx, oy, oz, fcut2, xcut2, A.nbr, A.rnbr, stride, cap, rcap, cc);
                        xa = 0;
                    }
                    if (xb >= nsx) {
                        const int b = min(xb - nsx, xa - 1);
                        cc = scan_lists(A.npos, __ldg(A.cell_start + kb), __ldg(A.cell_start + kb + b + 1), i,
                                        Lx - p.x, oy, oz, fcut2, xcut2, A.nbr, A.rnbr, stride, cap, rcap, cc);
                        xb = nsx - 1;
                    }
                    xa = min(xa, nsx);     // a coordinate outside the box: an empty main run
                    xb = max(xb, -1);
                    cc = scan_lists(A.npos, __ldg(A.cell_start + kb + xa), __ldg(A.cell_start + kb + xb + 1), i, -p.x,
                                    oy, oz, fcut2, xcut2, A.nbr, A.rnbr, stride, cap, rcap, cc);
                }
            }
        }
        A.nn[i] = min(cc.x, cap);
        A.rnn[i] = min(cc.y, rcap);
        if (cc.x > cap || cc.y > rcap) {
            atomicOr(A.status, (uint32_t)kStOverflow);
            atomicMax(&A.nbr_need[0], cc.x);
            atomicMax(&A.nbr_need[1], cc.y);
        }
    }
    const int idx[2] = {cNlistEntries, cRnlistEntries};
    const unsigned long long v[2] = {(unsigned long long)min(cc.x, cap), (unsigned long long)min(cc.y, rcap)};
    warp_counts<2>(A.counters, idx, v);
    if (i < P.n) copyback_particle<R>(P, A, B, i);
}

// Start of a captured step: with end_prev, first the end of the step before
// it in the same graph (what k_step_end does, one launch fewer per step),
// then the rebuild condition.
__global__ void k_set_rebuild_cond(DevArrays A, cudaGraphConditionalHandle h, int end_prev)
{
    const bool ok = status_ok(A.status);
    if (end_prev && ok) {
        *A.step += 1;
        *A.list_fresh = 0;
    }
    cudaGraphSetConditional(h, (ok && *A.need_rebuild) ? 1u : 0u);
}

__global__ void k_rebuild_done(DevArrays A)
{
    *A.gathered = 0;
    if (!status_ok(A.status)) return;
    if (*A.need_rebuild) {
        *A.need_rebuild = 0;
        *A.list_fresh = 1;   // the next MD step stores the pairs' cell shifts
        counter_add1(A.counters, cBuilds, 1ull);
    }
}

}  // namespace

void launch_cell_key(const DevParams &P, const DevArrays &A, Launch L)
{
    if (P.n == 0) return;
    k_cell_key<<<grid_for(P.n, L.block), L.block, 0, L.stream>>>(P, A);
}

// tile-local prefixes and tile offsets only: k_scatter and k_cell_sort add the offsets
void launch_cell_scan(const DevArrays &A, int32_t *block_sums, int ncell, Launch L)
{
    const int nb = (ncell + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<nb, kScanThreads, 0, L.stream>>>(A.cell_count, A.cell_start, block_sums, ncell,
                                                     A.need_rebuild, A.status);
    k_scan_sums<<<1, kScanThreads, 0, L.stream>>>(block_sums, nb, A.need_rebuild, A.status);
}

void launch_scan(const int32_t *in, int32_t *out, int32_t *bsum, int n, const int32_t *gate, const uint32_t *status,
                 Launch L)
{
    if (n <= 0) return;
    const int nb = (n + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<nb, kScanThreads, 0, L.stream>>>(in, out, bsum, n, gate, status);
    k_scan_sums<<<1, kScanThreads, 0, L.stream>>>(bsum, nb, gate, status);
    k_scan_add<<<grid_for(n, 256), 256, 0, L.stream>>>(out, bsum, n, nb, gate, status);
}

void launch_scatter(const DevParams &P, const DevArrays &A, const int32_t *block_sums, Launch L)
{
    if (P.n == 0) return;
    k_scatter<<<grid_for(P.n, L.block), L.block, 0, L.stream>>>(P, A, block_sums);
}

void launch_cell_sort(const DevArrays &A, int ncell, const int32_t *block_sums, Launch L)
{
    k_cell_sort<<<grid_for(ncell, 128), 128, 0, L.stream>>>(A, ncell, block_sums);
}

void launch_gather(const DevParams &P, const DevArrays &A, const DevArrays &B, bool fp64, Launch L)
{
    if (P.n == 0) return;
    if (fp64)
        k_gather<double><<<grid_for(P.n, L.block), L.block, 0, L.stream>>>(P, A, B);
    else
        k_gather<float><<<grid_for(P.n, L.block), L.block, 0, L.stream>>>(P, A, B);
}

// the lists (both precisions list from the FP32 wrapped positions) and the
// copy back of the gathered arrays
void launch_nlist(const DevParams &P, const DevArrays &A, const DevArrays &B, bool fp64, int block, Launch L)
{
    if (P.n == 0) return;
    const unsigned g = grid_for(P.n, block);
    if (fp64) k_nlist<double><<<g, block, 0, L.stream>>>(P, A, B);
    else k_nlist<float><<<g, block, 0, L.stream>>>(P, A, B);
}

void launch_rebuild_done(const DevArrays &A, Launch L) { k_rebuild_done<<<1, 1, 0, L.stream>>>(A); }

void launch_set_rebuild_cond(const DevArrays &A, cudaGraphConditionalHandle h, bool end_prev, Launch L)
{
    k_set_rebuild_cond<<<1, 1, 0, L.stream>>>(A, h, end_prev ? 1 : 0);
}

}  // namespace snap
