// Allocation-free pair energy: snap_pair_energy_noalloc (see include/snap.h).
//
// Some callers cannot allocate device memory once they are running: a host
// framework that has reserved the whole device pool for its own allocator, a
// real-time loop that cannot afford an allocation's latency or failure, or a
// plugin that is only ever handed device pointers.  This entry point computes
// the total Lennard-Jones/WCA pair energy and virial of caller-provided device
// positions by direct summation over all pairs, keeping its per-particle
// partial sums in the fixed file-scope array below instead of memory obtained
// from cudaMalloc or any allocator.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/snap.h"
#include "snap_device.cuh"

namespace {

constexpr int kNoAllocMax = SNAP_NOALLOC_MAX_N;

// Two doubles per particle (energy, virial halves).  Every GPU that loads the
// library holds this array until the process exits.  In host code its name
// is only a host-side stand-in; kernels are handed the device address
// obtained from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_partial[2 * kNoAllocMax];

struct PairTable {
    int ntypes;
    double L[3];
    double rc2[snap::kMaxTypes * snap::kMaxTypes];
    double sig2[snap::kMaxTypes * snap::kMaxTypes];
    double eps4[snap::kMaxTypes * snap::kMaxTypes];
    double shift[snap::kMaxTypes * snap::kMaxTypes];
};

// Per particle i: half of every pair energy and virial it takes part in.
// Every entry i < n is overwritten, so nothing has to be cleared between calls.
__global__ void k_pair_partial(int n, const double *__restrict__ pos3, const int32_t *__restrict__ type,
                               PairTable T, double *__restrict__ partial)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double xi = pos3[3 * i], yi = pos3[3 * i + 1], zi = pos3[3 * i + 2];
    const int ti = type[i];
    double e = 0.0, w = 0.0;
    // a type outside [0, ntypes) would index past the pair table: such a
    // particle takes part in no pair
    const bool ti_ok = (unsigned)ti < (unsigned)T.ntypes;
    for (int j = 0; ti_ok && j < n; ++j) {
        if (j == i) continue;
        const int tj = type[j];
        if ((unsigned)tj >= (unsigned)T.ntypes) continue;
        double dx = pos3[3 * j] - xi, dy = pos3[3 * j + 1] - yi, dz = pos3[3 * j + 2] - zi;
        dx -= T.L[0] * rint(dx / T.L[0]);
        dy -= T.L[1] * rint(dy / T.L[1]);
        dz -= T.L[2] * rint(dz / T.L[2]);
        const double r2 = dx * dx + dy * dy + dz * dz;
        const int k = ti * snap::kMaxTypes + tj;
        if (r2 >= T.rc2[k]) continue;
        const double s2 = T.sig2[k] / r2;
        const double s6 = s2 * s2 * s2;
        e += 0.5 * (T.eps4[k] * (s6 * s6 - s6) - T.shift[k]);
        w += 0.5 * (6.0 * T.eps4[k] * (2.0 * s6 * s6 - s6));   // (-dU/dr) r
    }
    partial[2 * i] = e;
    partial[2 * i + 1] = w;
}

// One block, fixed stride and tree: the same inputs give the same sums.
__global__ void k_pair_reduce(int n, const double *__restrict__ partial, double *__restrict__ out)
{
    __shared__ double se[512], sw[512];
    double e = 0.0, w = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        e += partial[2 * i];
        w += partial[2 * i + 1];
    }
    se[threadIdx.x] = e;
    sw[threadIdx.x] = w;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            se[threadIdx.x] += se[threadIdx.x + s];
            sw[threadIdx.x] += sw[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = se[0];
        out[1] = sw[0];
    }
}

// device address of the static array, looked up once per device
constexpr int kMaxDevices = 64;
double *g_addr[kMaxDevices] = {};
std::mutex g_addr_mu;

snap_status scratch_address(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SNAP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        // the current device is `dev`, so this is that device's copy of the array
        if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess || !p) {
            cudaGetLastError();
            return SNAP_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return SNAP_OK;
}

}  // namespace

extern "C" snap_status snap_pair_energy_noalloc(int64_t n, const double *d_pos3, const int32_t *d_type,
                                                const double *box, int32_t ntypes, const double *sigma,
                                                const double *eps_pair, const double *rcut, double *d_out,
                                                void *stream)
{
    if (n < 0 || n > kNoAllocMax) return SNAP_ERR_ARG;   // beyond the static array
    if (!box || !sigma || !eps_pair || !d_out || ntypes < 1 || ntypes > snap::kMaxTypes) return SNAP_ERR_ARG;
    if (n > 0 && (!d_pos3 || !d_type)) return SNAP_ERR_ARG;
    PairTable T;
    std::memset(&T, 0, sizeof T);
    T.ntypes = ntypes;
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0.0)) return SNAP_ERR_ARG;
        T.L[d] = box[d];
    }
    for (int a = 0; a < ntypes; ++a)
        for (int b = 0; b < ntypes; ++b) {
            const int k = a * snap::kMaxTypes + b;
            const double sig = 0.5 * (sigma[a] + sigma[b]);
            const double rc = (rcut && rcut[a * ntypes + b] > 0.0) ? rcut[a * ntypes + b] : sig * std::pow(2.0, 1.0 / 6.0);
            const double e = eps_pair[a * ntypes + b];
            const double c2 = (sig * sig) / (rc * rc), c6 = c2 * c2 * c2;
            T.rc2[k] = rc * rc;
            T.sig2[k] = sig * sig;
            T.eps4[k] = 4.0 * e;
            T.shift[k] = 4.0 * e * (c6 * c6 - c6);
        }
    double *partial = nullptr;
    snap_status s = scratch_address(&partial);
    if (s != SNAP_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ni = (int)n;
    if (ni > 0) k_pair_partial<<<(ni + 255) / 256, 256, 0, st>>>(ni, d_pos3, d_type, T, partial);
    k_pair_reduce<<<1, 512, 0, st>>>(ni, partial, d_out);
    if (cudaGetLastError() != cudaSuccess) return SNAP_ERR_CUDA;
    return SNAP_OK;
}
