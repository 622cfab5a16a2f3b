// Observables: the pair-distance histogram behind g(r).
//
// Called right after a forced neighbour-list rebuild, so every particle sits
// in the cell the rebuild filed it under and its FP64 position is wrapped into
// the box; a pair closer than the cell width then lies in neighbouring cells,
// and r_max is limited to that width by the host.  The distance is the exact
// FP64 separation the bond sweep uses (minimum image per axis, (dx^2 + dy^2) +
// dz^2, IEEE square root), and the bin floor(r / dr) is an IEEE division, so
// the integer counts are a pure function of the positions.
#include "snap_kernels.h"

namespace snap {

namespace {

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }

// one thread per particle of type ta in replica rep; each unordered pair once
// (ta == tb: only partners of larger tag)
__global__ void k_rdf(DevParams P, DevArrays A, int rep, int ta, int tb, double rmax, double dr, int nbins,
                      unsigned long long *hist)
{
    const long long i = gtid();
    if (i >= P.n) return;
    if (!status_ok(A.status)) return;
    if (rep_of(P, A, i) != rep || A.type[i] != ta) return;
    const RepDev &R = A.reps[rep];
    const uint32_t bits = P.screen ? w_bits(reinterpret_cast<const float4 *>(A.pos4)[i])
                                   : w_bits(reinterpret_cast<const double4_32a *>(A.pos4)[i]);
    const int cx = bits_cx(bits), cy = bits_cy(bits), cz = bits_cz(bits);
    const int nx = R.nc[0], ny = R.nc[1], nz = R.nc[2];
    const double xi = A.x[i], yi = A.y[i], zi = A.z[i];
    const int tgi = A.tag[i];
    const double rmax2 = __dmul_rn(rmax, rmax);
    for (int dz = -1; dz <= 1; ++dz) {
        const int zz = (cz + dz + nz) % nz;
        for (int dy = -1; dy <= 1; ++dy) {
            const int yy = (cy + dy + ny) % ny;
            for (int dx = -1; dx <= 1; ++dx) {
                const int xx = (cx + dx + nx) % nx;
                // the cell's 2^sub_shift sub-cells are consecutive sort keys
                const int key = (tb * P.ncell + A.rank_of[R.cell_off + (zz * ny + yy) * nx + xx]) << P.sub_shift;
                const int s0 = A.cell_start[key], e = A.cell_start[key + (1 << P.sub_shift)];
                for (int j = s0; j < e; ++j) {
                    if (j == i) continue;
                    if (ta == tb && A.tag[j] <= tgi) continue;
                    const double ax = min_image(__dsub_rn(A.x[j], xi), R.L[0], R.invL[0]);
                    const double ay = min_image(__dsub_rn(A.y[j], yi), R.L[1], R.invL[1]);
                    const double az = min_image(__dsub_rn(A.z[j], zi), R.L[2], R.invL[2]);
                    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
                    if (!(r2 < rmax2)) continue;
                    const double r = __dsqrt_rn(r2);
                    if (!(r < rmax)) continue;
                    const long long b = (long long)__ddiv_rn(r, dr);
                    if (b < nbins) atomicAdd(&hist[b], 1ull);
                }
            }
        }
    }
}

}  // namespace

void launch_rdf(const DevParams &P, const DevArrays &A, int rep, int ta, int tb, double rmax, int nbins,
                unsigned long long *hist, Launch L)
{
    if (P.n == 0) return;
    const double dr = rmax / (double)nbins;
    k_rdf<<<(unsigned)((P.n + 255) / 256), 256, 0, L.stream>>>(P, A, rep, ta, tb, rmax, dr, nbins, hist);
}

}  // namespace snap
