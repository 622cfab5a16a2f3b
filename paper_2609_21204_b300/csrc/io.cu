// Tag-order <-> memory-order transfers used by the host API.
#include "snap_kernels.h"

namespace snap {

namespace {
template <typename T>
__global__ void k_in(T *dst, const T *src, const int32_t *rtag, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[rtag[t]] = src[t];
}
template <typename T>
__global__ void k_out(T *dst, const T *src, const int32_t *rtag, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = src[rtag[t]];
}
template <typename V>
__global__ void k_force_out(double *dst, const V *f, const int32_t *rtag, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const V v = f[rtag[t]];
    dst[3 * t + 0] = (double)v.x;
    dst[3 * t + 1] = (double)v.y;
    dst[3 * t + 2] = (double)v.z;
}
__global__ void k_iota(int32_t *dst, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dst[t] = (int32_t)t;
}
__global__ void k_v4_in(float4 *v4, const double *vx, const double *vy, const double *vz, const int32_t *rtag,
                        long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) v4[rtag[t]] = make_float4((float)vx[t], (float)vy[t], (float)vz[t], 0.f);
}
__global__ void k_v4_out(double *vx, double *vy, double *vz, const float4 *v4, const int32_t *rtag, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float4 v = v4[rtag[t]];
    vx[t] = v.x;
    vy[t] = v.y;
    vz[t] = v.z;
}
// Wrap into [0, L) counting box crossings: k = floor(x / L), x -= k L, then
// one correction each way (every operation rounded once, as on the host).
__device__ __forceinline__ void wrap_dev(double &x, int32_t &img, double L)
{
    const double k = floor(__ddiv_rn(x, L));
    x = __dsub_rn(x, __dmul_rn(k, L));
    img += (int32_t)k;
    if (x >= L) {
        x = __dsub_rn(x, L);
        img += 1;
    }
    if (x < 0.0) {
        x = __dadd_rn(x, L);
        img -= 1;
    }
    if (x >= L) x = 0.0;
}

__global__ void k_nonfinite(const double *v, long long m, uint32_t *flag)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool bad = t < m && !isfinite(v[t]);
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// tag-ordered (x, y, z) triples -> wrapped sorted-order SoA + image counters
__global__ void k_pos_in(const double *src3, DevParams P, DevArrays A, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = A.rtag[t];
    const RepDev &R = A.reps[rep_of(P, A, i)];
    double x = src3[3 * t], y = src3[3 * t + 1], z = src3[3 * t + 2];
    int32_t ix = 0, iy = 0, iz = 0;
    wrap_dev(x, ix, R.L[0]);
    wrap_dev(y, iy, R.L[1]);
    wrap_dev(z, iz, R.L[2]);
    A.x[i] = x; A.y[i] = y; A.z[i] = z;
    A.ix[i] = ix; A.iy[i] = iy; A.iz[i] = iz;
}

// sorted order -> tag-ordered triples, positions wrapped into [0, L) and
// images including those crossings (either output nullable)
__global__ void k_pos_out(double *dst3, int32_t *img3, DevParams P, DevArrays A, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = A.rtag[t];
    const RepDev &R = A.reps[rep_of(P, A, i)];
    double xs[3] = {A.x[i], A.y[i], A.z[i]};
    int32_t im[3] = {A.ix[i], A.iy[i], A.iz[i]};
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if (!(xs[d] >= 0.0 && xs[d] < R.L[d])) {
            int32_t k = 0;
            wrap_dev(xs[d], k, R.L[d]);
            im[d] += k;
        }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (dst3) dst3[3 * t + d] = xs[d];
        if (img3) img3[3 * t + d] = im[d];
    }
}

// tag-ordered velocity triples <-> sorted order (FP32 float4 in mixed mode)
__global__ void k_vel_in(const double *src3, DevArrays A, bool fp64, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = A.rtag[t];
    const double vx = src3[3 * t], vy = src3[3 * t + 1], vz = src3[3 * t + 2];
    if (fp64) {
        A.vx[i] = vx; A.vy[i] = vy; A.vz[i] = vz;
    } else {
        A.v4[i] = make_float4((float)vx, (float)vy, (float)vz, 0.f);
    }
}

__global__ void k_vel_out(double *dst3, DevArrays A, bool fp64, long long n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int i = A.rtag[t];
    if (fp64) {
        dst3[3 * t] = A.vx[i]; dst3[3 * t + 1] = A.vy[i]; dst3[3 * t + 2] = A.vz[i];
    } else {
        const float4 v = A.v4[i];
        dst3[3 * t] = v.x; dst3[3 * t + 1] = v.y; dst3[3 * t + 2] = v.z;
    }
}

inline unsigned grid_for(long long n) { return (unsigned)((n + 255) / 256); }
}  // namespace

void launch_nonfinite(const double *v, long long m, uint32_t *flag, Launch L)
{
    if (m > 0) k_nonfinite<<<grid_for(m), 256, 0, L.stream>>>(v, m, flag);
}
void launch_pos_in(const double *src3, const DevParams &P, const DevArrays &A, Launch L)
{
    if (P.n > 0) k_pos_in<<<grid_for(P.n), 256, 0, L.stream>>>(src3, P, A, P.n);
}
void launch_pos_out(double *dst3, int32_t *img3, const DevParams &P, const DevArrays &A, Launch L)
{
    if (P.n > 0) k_pos_out<<<grid_for(P.n), 256, 0, L.stream>>>(dst3, img3, P, A, P.n);
}
void launch_vel_in(const double *src3, const DevArrays &A, bool fp64, long long n, Launch L)
{
    if (n > 0) k_vel_in<<<grid_for(n), 256, 0, L.stream>>>(src3, A, fp64, n);
}
void launch_vel_out(double *dst3, const DevArrays &A, bool fp64, long long n, Launch L)
{
    if (n > 0) k_vel_out<<<grid_for(n), 256, 0, L.stream>>>(dst3, A, fp64, n);
}

void launch_v4_in(float4 *v4, const double *vx, const double *vy, const double *vz, const int32_t *rtag,
                  long long n, Launch L)
{
    if (n > 0) k_v4_in<<<grid_for(n), 256, 0, L.stream>>>(v4, vx, vy, vz, rtag, n);
}
void launch_v4_out(double *vx, double *vy, double *vz, const float4 *v4, const int32_t *rtag, long long n,
                   Launch L)
{
    if (n > 0) k_v4_out<<<grid_for(n), 256, 0, L.stream>>>(vx, vy, vz, v4, rtag, n);
}

template <typename T>
void launch_in(T *dst, const T *src, const int32_t *rtag, long long n, Launch L)
{
    if (n > 0) k_in<T><<<grid_for(n), 256, 0, L.stream>>>(dst, src, rtag, n);
}
template <typename T>
void launch_out(T *dst, const T *src, const int32_t *rtag, long long n, Launch L)
{
    if (n > 0) k_out<T><<<grid_for(n), 256, 0, L.stream>>>(dst, src, rtag, n);
}
template void launch_in<double>(double *, const double *, const int32_t *, long long, Launch);
template void launch_in<int32_t>(int32_t *, const int32_t *, const int32_t *, long long, Launch);
template void launch_in<int4>(int4 *, const int4 *, const int32_t *, long long, Launch);
template void launch_out<double>(double *, const double *, const int32_t *, long long, Launch);
template void launch_out<int32_t>(int32_t *, const int32_t *, const int32_t *, long long, Launch);
template void launch_out<int4>(int4 *, const int4 *, const int32_t *, long long, Launch);

void launch_force_out(double *dst3, const void *force, bool fp64, const int32_t *rtag, long long n, Launch L)
{
    if (n <= 0) return;
    if (fp64)
        k_force_out<double4_32a><<<grid_for(n), 256, 0, L.stream>>>(dst3, (const double4_32a *)force, rtag, n);
    else
        k_force_out<float4><<<grid_for(n), 256, 0, L.stream>>>(dst3, (const float4 *)force, rtag, n);
}

void launch_iota(int32_t *dst, long long n, Launch L)
{
    if (n > 0) k_iota<<<grid_for(n), 256, 0, L.stream>>>(dst, n);
}

}  // namespace snap
