// Langevin step of one particle (leapfrog form):
//   a = F_c(x_t) - gamma v_{t-1/2} + sqrt(2 gamma kT/dt) xi,  xi = sqrt(3)(2u - 1)
//   v_{t+1/2} = v_{t-1/2} + dt a;  x_{t+1} = x_t + dt v_{t+1/2}
// with u from Philox(LANGEVIN; step, tag).  Every floating-point operation is
// an explicit intrinsic (one rounding each, no contraction), so the result
// does not depend on the compilation unit.  Used by the fused force +
// integrate kernel; pos_out receives the new cell-relative coordinate (the
// other of two buffers).
#pragma once
#include "snap_device.cuh"

namespace snap {

__device__ __forceinline__ U4 langevin_draw(const RepDev &Rp, const DevArrays &A, long long i, long long step)
{
    const uint32_t tl = (uint32_t)(__ldcs(A.tag + i) - Rp.tag_off);
    return philox10(U4{(uint32_t)((unsigned long long)step & 0xFFFFFFFFull), (uint32_t)((unsigned long long)step >> 32),
                       tl, 0u},
                    Rp.key0, rx_key1(Rp, 0, kLangevin));
}

__device__ __forceinline__ bool moved_past_skin(const DevParams &P, const DevArrays &A, long long i, float rx,
                                                float ry, float rz)
{
    const float4 ref = __ldcs(A.ref4 + i);
    const float ex = __fsub_rn(rx, ref.x), ey = __fsub_rn(ry, ref.y), ez = __fsub_rn(rz, ref.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez)) > P.disp2f;
}

// FP64 mode: everything in FP64; positions wrapped into [0, L) every step.
__device__ __forceinline__ void wrap_step(double &x, int &img, double L)
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

__device__ __forceinline__ void integrate_fp64(const DevParams &P, DevArrays &A, long long i, long long step,
                                               const RepDev &Rp, const double (&fv)[3], double4_32a p,
                                               double4_32a *pos_out)
{
    const U4 w = langevin_draw(Rp, A, i, step);
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
        wrap_step(x1, img, Rp.L[d]);
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
    p.x = rel[0]; p.y = rel[1]; p.z = rel[2];
    pos_out[i] = p;
    if (moved_past_skin(P, A, i, (float)rel[0], (float)rel[1], (float)rel[2])) *A.need_rebuild = 1;
}

// Mixed mode: the kick and the velocity in FP32, the position accumulated in
// FP64 (x += dt v, one FP64 fma and one conversion per axis).  The
// cell-relative FP32 coordinate used by the force loop advances by the same
// FP32 displacement (one FP32 fma), and every kMixedResync steps (and at every
// rebuild) it is reset to (float)(x - origin) from the FP64 position, so it
// never drifts by more than kMixedResync roundings of a coordinate below 4
// (8 x 2.4e-7 < 2e-6).  Positions stay unwrapped between neighbour-list
// rebuilds (the rebuild wraps them).
__device__ __forceinline__ void integrate_mixed(const DevParams &P, DevArrays &A, long long i, long long step,
                                                const RepDev &Rp, float fx, float fy, float fz, float4 p,
                                                float4 *pos_out)
{
    const U4 w = langevin_draw(Rp, A, i, step);
    float4 v = __ldcs(A.v4 + i);   // streaming: read once per step
    const float cn = Rp.noise_cf, g = P.gammaf, s3 = P.sqrt3f, dt = P.dtf;   // rounded on the host
    // xi = sqrt(3) (2u - 1) with u = (w >> 8 + 1/2) 2^-24 in (0, 1)
    const float ux = fmaf((float)(w.x >> 8), 0x1.0p-24f, 0x1.0p-25f);
    const float uy = fmaf((float)(w.y >> 8), 0x1.0p-24f, 0x1.0p-25f);
    const float uz = fmaf((float)(w.z >> 8), 0x1.0p-24f, 0x1.0p-25f);
    v.x = fmaf(dt, fmaf(cn, __fmul_rn(s3, fmaf(2.0f, ux, -1.0f)), fmaf(-g, v.x, fx)), v.x);
    v.y = fmaf(dt, fmaf(cn, __fmul_rn(s3, fmaf(2.0f, uy, -1.0f)), fmaf(-g, v.y, fy)), v.y);
    v.z = fmaf(dt, fmaf(cn, __fmul_rn(s3, fmaf(2.0f, uz, -1.0f)), fmaf(-g, v.z, fz)), v.z);
    const double x1 = fma(P.dt, (double)v.x, __ldcs(A.x + i));
    const double y1 = fma(P.dt, (double)v.y, __ldcs(A.y + i));
    const double z1 = fma(P.dt, (double)v.z, __ldcs(A.z + i));
    if ((step & (kMixedResync - 1)) == 0) {          // uniform over the grid
        // origin of the frozen cell, as the rebuild computed it
        const uint32_t b = w_bits(p);
        p.x = (float)__dsub_rn(x1, __dmul_rn((double)bits_cx(b), Rp.w[0]));
        p.y = (float)__dsub_rn(y1, __dmul_rn((double)bits_cy(b), Rp.w[1]));
        p.z = (float)__dsub_rn(z1, __dmul_rn((double)bits_cz(b), Rp.w[2]));
    } else {
        p.x = fmaf(dt, v.x, p.x);
        p.y = fmaf(dt, v.y, p.y);
        p.z = fmaf(dt, v.z, p.z);
    }
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
    pos_out[i] = p;
    if (moved_past_skin(P, A, i, p.x, p.y, p.z)) *A.need_rebuild = 1;
}

}  // namespace snap
