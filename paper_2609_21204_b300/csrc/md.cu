// Pair + bond forces and the fused force + Langevin step.
//
// Positions used by the force loop are stored relative to the origin of the
// particle's cell (frozen between rebuilds; nlist.cu lays them out) with the
// cell coordinates and type packed in the w word; a pair's separation is
// (rel_j - rel_i) + (c_j - c_i) * w, which keeps FP32 separations accurate to
// ~1e-7 in any box size.
//
// Pair potential: Lennard-Jones shifted to zero at its cut (WCA for the
// default cut 2^(1/6) sigma_ij); static and dynamic bonds harmonic (Eq. 4 of
// the DyBond-v2 paper names the harmonic form), FENE, FENEWCA or Tether.  No
// pair exclusions: the pair potential acts on bonded pairs too.
#include <algorithm>

#include "snap_kernels.h"
#include "integrate.cuh"

namespace snap {

namespace {

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }

// ------------------------------------------------------------ forces
template <typename R> struct Num;
template <> struct Num<float> {
    __device__ static float rc2(const DevParams &P, int k) { return P.rc2f[k]; }
    __device__ static float sig2(const DevParams &P, int k) { return P.sig2f[k]; }
    __device__ static float eps24(const DevParams &P, int k) { return P.eps24f[k]; }
    __device__ static float bk(const DevParams &P, int k) { return P.bkf[k]; }
    __device__ static float br0(const DevParams &P, int k) { return P.br0f[k]; }
    __device__ static float w(const RepDev &R, int d) { return R.wf[d]; }
    __device__ static float sqrt_(float v) { return sqrtf(v); }
    // approximate reciprocal (MUFU, <= 1 ulp); well inside the FP32 force tolerance
    __device__ static float rcp(float v) { return __fdividef(1.0f, v); }
};
template <> struct Num<double> {
    __device__ static double rc2(const DevParams &P, int k) { return P.rc2d[k]; }
    __device__ static double sig2(const DevParams &P, int k) { return P.sig2d[k]; }
    __device__ static double eps24(const DevParams &P, int k) { return P.eps24d[k]; }
    __device__ static double bk(const DevParams &P, int k) { return P.bk[k]; }
    __device__ static double br0(const DevParams &P, int k) { return P.br0[k]; }
    __device__ static double w(const RepDev &R, int d) { return R.w[d]; }
    __device__ static double sqrt_(double v) { return sqrt(v); }
    __device__ static double rcp(double v) { return 1.0 / v; }
};

// separation (j - i) of two particles from their relative coords and cells;
// returns the code (sx + 1) + 3 (sy + 1) + 9 (sz + 1) of the cell shift
template <typename R, typename V>
__device__ __forceinline__ uint32_t separation(const V &pi, const V &pj, const RepDev &Rp, R &dx, R &dy, R &dz)
{
    const uint32_t bi = w_bits(pi), bj = w_bits(pj);
    const int sx = cell_delta(bits_cx(bj) - bits_cx(bi), Rp.nc[0]);
    const int sy = cell_delta(bits_cy(bj) - bits_cy(bi), Rp.nc[1]);
    const int sz = cell_delta(bits_cz(bj) - bits_cz(bi), Rp.nc[2]);
    dx = (pj.x - pi.x) + (R)sx * Num<R>::w(Rp, 0);
    dy = (pj.y - pi.y) + (R)sy * Num<R>::w(Rp, 1);
    dz = (pj.z - pi.z) + (R)sz * Num<R>::w(Rp, 2);
    return (uint32_t)((sx + 1) + 3 * (sy + 1) + 9 * (sz + 1));
}

template <typename R> __device__ __forceinline__ R exp_(R v);
template <> __device__ __forceinline__ float exp_<float>(float v) { return expf(v); }
template <> __device__ __forceinline__ double exp_<double>(double v) { return exp(v); }

// bond force factor (dU/dr)/r and energy u; returns false when the bond is
// outside the finite range of its potential (FENE / FENEWCA overstretch, a
// Tether bond at or beyond l_min or l_max).  FENEWCA and Tether are the bond
// potentials HOOMD-blue documents under those names (Sec. II.B of the DyBond-v2
// paper lists them as the evaluators it accepts):
//   FENEWCA: U = -k R0^2/2 ln(1 - (s/R0)^2) + [4 eps ((sig/s)^12 - (sig/s)^6) + eps] for
//            s = r - delta < 2^(1/6) sig (the bracket is 0 beyond);
//   Tether:  U = k_b e^{1/(l_c0 - r)} / (l_max - r) for r > l_c0
//              + k_b e^{1/(r - l_c1)} / (r - l_min) for r < l_c1 (0 in between).
template <typename R>
__device__ __forceinline__ bool bond_factor(const DevParams &P, int bt, R r2, R &fb, double &u)
{
    const R k = Num<R>::bk(P, bt), r0 = Num<R>::br0(P, bt);
    const int kind = P.bkind[bt];
    if (kind == kHarmonic) {
        const R r = Num<R>::sqrt_(r2);
        fb = k * (r - r0) / r;
        u = 0.5 * (double)k * ((double)r - (double)r0) * ((double)r - (double)r0);
        return true;
    }
    if (kind == kFene) {
        const R q = r2 / (r0 * r0);
        if (!(q < (R)1)) {
            fb = 0;
            u = 0.0;
            return false;
        }
        fb = k / ((R)1 - q);
        u = -0.5 * (double)k * (double)r0 * (double)r0 * log(1.0 - (double)q);
        return true;
    }
    const R r = Num<R>::sqrt_(r2);
    const R x0 = sizeof(R) == 4 ? (R)P.bxf[bt][0] : (R)P.bx[bt][0];
    const R x1 = sizeof(R) == 4 ? (R)P.bxf[bt][1] : (R)P.bx[bt][1];
    const R x2 = sizeof(R) == 4 ? (R)P.bxf[bt][2] : (R)P.bx[bt][2];
    if (kind == kFeneWca) {
        const R eps = x0, sig = x1, s = r - x2;
        const R q = s * s / (r0 * r0);
        if (!(q < (R)1) || !(s > (R)0)) {
            fb = 0;
            u = 0.0;
            return false;
        }
        R du = k * s / ((R)1 - q);   // dU/dr
        u = -0.5 * (double)k * (double)r0 * (double)r0 * log(1.0 - (double)q);
        if (s < sig * (R)kTwoSixth) {
            const R sr2 = sig * sig / (s * s);
            const R sr6 = sr2 * sr2 * sr2;
            du -= (R)24 * eps * ((R)2 * sr6 * sr6 - sr6) / s;
            const double d6 = (double)sr6;
            u += 4.0 * (double)eps * (d6 * d6 - d6) + (double)eps;
        }
        fb = du / r;
        return true;
    }
    // Tether: k_b = k, l_min = r0, l_c1 = x0, l_c0 = x1, l_max = x2
    if (!(r > r0) || !(r < x2)) {
        fb = 0;
        u = 0.0;
        return false;
    }
    R du = 0;
    u = 0.0;
    if (r > x1) {
        const R a = x1 - r, b = x2 - r;
        const R U = k * exp_<R>((R)1 / a) / b;
        du = U * ((R)1 / (a * a) + (R)1 / b);
        u = (double)U;
    } else if (r < x0) {
        const R c = r - x0, e = r - r0;
        const R U = k * exp_<R>((R)1 / c) / e;
        du = -U * ((R)1 / (c * c) + (R)1 / e);
        u = (double)U;
    }
    fb = du / r;
    return true;
}

// How the force loop finds a pair's cell shift: from the code its list entry
// carries (kShiftCoded), or from the cell bits of both particles, storing the
// code in the entry for the steps that follow (kShiftStore: the first MD step
// after a rebuild) or not (kShiftBits: force read-outs).  Force-list entries
// hold the neighbour's index in the low kIdxBits bits and above them the code
// (sx + 1) + 3 (sy + 1) + 9 (sz + 1) of the minimum-image shift between the
// two frozen cells, fixed until the next rebuild like the cells themselves.
enum ShiftMode { kShiftCoded = 0, kShiftStore = 1, kShiftBits = 2 };

// Force on particle i: WCA/LJ pairs over the force list, static and dynamic
// bonds; the energy terms when E.  Returns false (and latches the status) on
// a FENE overstretch.
template <typename R, bool E, int MODE>
__device__ __forceinline__ bool force_particle(const DevParams &P, const DevArrays &A, long long i,
                                               const typename Vec4<R>::T &pi, const RepDev &Rp,
                                               const float4 *s_shift, R &fx, R &fy, R &fz, double &ep, double &eb,
                                               double &vir)
{
    using V = typename Vec4<R>::T;
    const V *pos = reinterpret_cast<const V *>(A.pos4);
    const int ti = bits_type(w_bits(pi));
    const int nn = __ldcs(A.nn + i);
    const long long stride = P.nbr_stride;
    int *nb = A.nbr + i;
    // bond partners first: their slot words and sorted indices are independent
    // of the pair loop, so the tag -> index loads overlap it
    const int4 dp = __ldcs(A.dp + i);
    const int drx = __ldcs(A.drx + i);
    int dj[kVmax];
    {
        const int dpv[4] = {dp.x, dp.y, dp.z, dp.w};
#pragma unroll
        for (int s = 0; s < kVmax; ++s) dj[s] = dpv[s] >= 0 ? A.rtag[dpv[s]] : -1;
    }
    // pairs in batches of four: four independent position loads, then the
    // arithmetic in list order, while the next batch's four list entries are
    // already in flight; the pair's cell shift comes with its list entry
    // (s_shift: unit shifts by code).  The particle's own words, read once per
    // step, are streaming loads (__ldcs, evicted first) so that the L1 keeps the
    // neighbours' coordinates, which the block's other threads read again.
    const R wx = Num<R>::w(Rp, 0), wy = Num<R>::w(Rp, 1), wz = Num<R>::w(Rp, 2);
    auto entry = [&](int k) -> uint32_t {
        return k >= nn ? (uint32_t)i | (13u << kIdxBits)
               : MODE == kShiftStore ? (uint32_t)nb[(long long)k * stride]   // rewritten below
                                     : (uint32_t)__ldcs(nb + (long long)k * stride);
    };
    uint32_t en[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) en[u] = entry(u);
    for (int k0 = 0; k0 < nn; k0 += 4) {
        uint32_t ee[4];
        V pp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) ee[u] = en[u];
#pragma unroll
        for (int u = 0; u < 4; ++u) pp[u] = pos[ee[u] & kIdxMask];
#pragma unroll
        for (int u = 0; u < 4; ++u) en[u] = entry(k0 + 4 + u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (k0 + u >= nn) break;
            const V pj = pp[u];
            const int tj = bits_type(w_bits(pj));
            R dx, dy, dz;
            if (MODE == kShiftCoded) {
                const float4 sh = s_shift[ee[u] >> kIdxBits];
                dx = (pj.x - pi.x) + (R)sh.x * wx;
                dy = (pj.y - pi.y) + (R)sh.y * wy;
                dz = (pj.z - pi.z) + (R)sh.z * wz;
            } else {
                const uint32_t code = separation<R>(pi, pj, Rp, dx, dy, dz);
                if (MODE == kShiftStore) nb[(long long)(k0 + u) * stride] = (int)((ee[u] & kIdxMask) | (code << kIdxBits));
            }
            const R r2 = dx * dx + dy * dy + dz * dz;
            const int tt = ti * kMaxTypes + tj;
            if (r2 < Num<R>::rc2(P, tt)) {
                const R ir2 = Num<R>::rcp(r2);
                const R s2 = Num<R>::sig2(P, tt) * ir2;
                const R s6 = s2 * s2 * s2;
                const R fr = Num<R>::eps24(P, tt) * (s6 * ((R)2 * s6 - (R)1)) * ir2;
                fx -= fr * dx;
                fy -= fr * dy;
                fz -= fr * dz;
                if (E) {
                    const double s6d = (double)s6;
                    ep += 0.5 * ((double)P.eps24d[tt] / 6.0 * (s6d * s6d - s6d) - P.shiftd[tt]);
                    vir += 0.5 * (double)fr * (double)r2;
                }
            }
        }
    }
    // static bonds
    bool bad = false;
    if (P.has_static) {
        const int4 sp = __ldcs(A.sp + i);
        const int sbt = __ldcs(A.sbt + i);
        const int spv[4] = {sp.x, sp.y, sp.z, sp.w};
#pragma unroll
        for (int s = 0; s < kSmax; ++s) {
            const int ptag = spv[s];
            if (ptag < 0) continue;
            const int j = A.rtag[ptag];
            const V pj = pos[j];
            R dx, dy, dz;
            separation<R>(pi, pj, Rp, dx, dy, dz);
            const R r2 = dx * dx + dy * dy + dz * dz;
            R fb;
            double u;
            if (!bond_factor<R>(P, (sbt >> (8 * s)) & 0xFF, r2, fb, u)) bad = true;
            fx += fb * dx;
            fy += fb * dy;
            fz += fb * dz;
            if (E) { eb += 0.5 * u; vir -= 0.5 * (double)fb * (double)r2; }
        }
    }
    // dynamic bonds
#pragma unroll
    for (int s = 0; s < kVmax; ++s) {
        const int j = dj[s];
        if (j < 0) continue;
        const V pj = pos[j];
        R dx, dy, dz;
        separation<R>(pi, pj, Rp, dx, dy, dz);
        const R r2 = dx * dx + dy * dy + dz * dz;
        R fb;
        double u;
        const int a = (drx >> (8 * s)) & 0xFF;
        if (!bond_factor<R>(P, P.rx_bt[a], r2, fb, u)) bad = true;
        fx += fb * dx;
        fy += fb * dy;
        fz += fb * dz;
        if (E) { eb += 0.5 * u; vir -= 0.5 * (double)fb * (double)r2; }
    }
    if (bad) atomicOr(A.status, (uint32_t)kStFene);
    return !bad;
}

// unit cell shifts by force-list code: code = (sx + 1) + 3 (sy + 1) + 9 (sz + 1)
__device__ __forceinline__ void fill_shift_table(float4 *s_shift)
{
    const int t = threadIdx.x;
    if (t < 27) s_shift[t] = make_float4((float)(t % 3 - 1), (float)(t / 3 % 3 - 1), (float)(t / 9 - 1), 0.f);
    __syncthreads();
}

template <typename R, bool E>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_force(DevParams P, DevArrays A)
{
    using V = typename Vec4<R>::T;
    const long long i = gtid();
    if (i >= P.n) return;
    if (!status_ok(A.status)) return;
    const V pi = reinterpret_cast<const V *>(A.pos4)[i];
    const RepDev &Rp = A.reps[rep_of(P, A, i)];
    R fx = 0, fy = 0, fz = 0;
    double ep = 0.0, eb = 0.0, vir = 0.0;
    force_particle<R, E, kShiftBits>(P, A, i, pi, Rp, nullptr, fx, fy, fz, ep, eb, vir);
    V f;
    f.x = fx; f.y = fy; f.z = fz; f.w = 0;
    reinterpret_cast<V *>(A.force)[i] = f;
    if (E) {
        double vx, vy, vz;
        if (sizeof(R) == 8) {
            vx = A.vx[i]; vy = A.vy[i]; vz = A.vz[i];
        } else {
            const float4 v = A.v4[i];
            vx = v.x; vy = v.y; vz = v.z;
        }
        A.e_part[4 * i + 0] = ep;
        A.e_part[4 * i + 1] = eb;
        A.e_part[4 * i + 2] = vir;
        A.e_part[4 * i + 3] = 0.5 * (vx * vx + vy * vy + vz * vz);
    }
}

// One MD step of a particle after the sweep: its force and its Langevin
// update in one pass (the force never goes to memory).  Neighbours' positions
// are read from pos4 while the new relative coordinate goes to pos4n, the
// other of two buffers, which the host swaps after the step.
template <typename R>
__device__ __forceinline__ void step_md_particle(const DevParams &P, DevArrays &A, const float4 *s_shift)
{
    using V = typename Vec4<R>::T;
    const long long i = gtid();
    if (i >= P.n) return;
    if (!status_ok(A.status)) return;
    const V pi = reinterpret_cast<const V *>(A.pos4)[i];
    const RepDev &Rp = A.reps[rep_of(P, A, i)];
    R fx = 0, fy = 0, fz = 0;
    double ep = 0.0, eb = 0.0, vir = 0.0;
    // the first step after a rebuild works the pairs' cell shifts out and
    // stores them in the list (the flag is the same for the whole grid)
    const bool ok = *A.list_fresh
                        ? force_particle<R, false, kShiftStore>(P, A, i, pi, Rp, s_shift, fx, fy, fz, ep, eb, vir)
                        : force_particle<R, false, kShiftCoded>(P, A, i, pi, Rp, s_shift, fx, fy, fz, ep, eb, vir);
    if (!ok) return;
    const long long step = *A.step;
    if constexpr (sizeof(R) == 8) {
        const double fv[3] = {fx, fy, fz};
        integrate_fp64(P, A, i, step, Rp, fv, pi, reinterpret_cast<double4_32a *>(A.pos4n));
    } else {
        integrate_mixed(P, A, i, step, Rp, fx, fy, fz, pi, reinterpret_cast<float4 *>(A.pos4n));
    }
}

// Mixed precision, capped at 56 registers: one more resident block of 128
// threads per SM than at 64 (9 instead of 8), for a few spilled words (the
// kernel is latency-bound: 78.2 -> 75.4 us on the 10^6 gel; a cap of 48
// spills in the pair loop and is slower).
__global__ void __maxnreg__(56) k_step_md(DevParams P, DevArrays A)
{
    __shared__ float4 s_shift[27];
    fill_shift_table(s_shift);
    step_md_particle<float>(P, A, s_shift);
}

__global__ void __launch_bounds__(256, 2) k_step_md_fp64(DevParams P, DevArrays A)
{
    __shared__ float4 s_shift[27];
    fill_shift_table(s_shift);
    step_md_particle<double>(P, A, s_shift);
}

// deterministic column sums: one block, fixed stride order, fixed tree
__global__ void k_reduce_cols(const double *src, int ncol, long long n, double *out)
{
    __shared__ double sh[1024];
    for (int c = 0; c < ncol; ++c) {
        double s = 0.0;
        for (long long r = threadIdx.x; r < n; r += blockDim.x) s += src[r * ncol + c];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = sh[0];
        __syncthreads();
    }
}

inline unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }


}  // namespace

// multiprocessors of the current device (cached per device)
int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    if (dev >= 0 && dev < 64) cache[dev] = n;
    return n;
}

void launch_step_md(const DevParams &P, const DevArrays &A, bool fp64, Launch L)
{
    if (P.n == 0) return;
    const unsigned g = grid_for(P.n, L.block);
    if (fp64) k_step_md_fp64<<<g, L.block, 0, L.stream>>>(P, A);
    else k_step_md<<<g, L.block, 0, L.stream>>>(P, A);
}

void launch_force(const DevParams &P, const DevArrays &A, bool fp64, bool energy, Launch L)
{
    if (P.n == 0) return;
    const unsigned g = grid_for(P.n, L.block);
    if (fp64) {
        if (energy) k_force<double, true><<<g, L.block, 0, L.stream>>>(P, A);
        else k_force<double, false><<<g, L.block, 0, L.stream>>>(P, A);
    } else {
        if (energy) k_force<float, true><<<g, L.block, 0, L.stream>>>(P, A);
        else k_force<float, false><<<g, L.block, 0, L.stream>>>(P, A);
    }
}


void launch_reduce_cols(const double *src, int ncol, long long n, double *out, Launch L)
{
    k_reduce_cols<<<1, 1024, 0, L.stream>>>(src, ncol, n, out);
}

}  // namespace snap
