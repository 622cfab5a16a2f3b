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
inline unsigned grid_for(long long n) { return (unsigned)((n + 255) / 256); }
}  // namespace

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
