// Kernel launchers (host side) of the snap library.
#pragma once
#include <cuda_runtime.h>

#include "snap_device.cuh"

namespace snap {

struct Launch {
    cudaStream_t stream;
    int block;       // threads per block for particle-parallel kernels
};

// multiprocessors of the current device (cached per device)
int sm_count();

// ---- neighbour-list maintenance (all early-exit unless *need_rebuild) ----
void launch_cell_key(const DevParams &P, const DevArrays &A, Launch L);
void launch_cell_scan(const DevArrays &A, int32_t *block_sums, int ncell, Launch L);
void launch_scatter(const DevParams &P, const DevArrays &A, const int32_t *block_sums, Launch L);
void launch_cell_sort(const DevArrays &A, int ncell, const int32_t *block_sums, Launch L);
void launch_gather(const DevParams &P, const DevArrays &A, const DevArrays &B, bool fp64, Launch L);
void launch_nlist(const DevParams &P, const DevArrays &A, const DevArrays &B, bool fp64, int block, Launch L);
void launch_rebuild_done(const DevArrays &A, Launch L);
// sets a graph conditional to (*need_rebuild && status == 0)
void launch_set_rebuild_cond(const DevArrays &A, cudaGraphConditionalHandle h, bool end_prev, Launch L);

// exclusive scan of in[0..n) into out[0..n] (runs only when *gate != 0 and status is clear)
void launch_scan(const int32_t *in, int32_t *out, int32_t *bsum, int n, const int32_t *gate, const uint32_t *status,
                 Launch L);

// ---- Metropolis–Hastings bond moves (mh.cu); mlp == nullptr: uniform proposal ----
struct MlpDev;
void launch_mh_sweep(const DevParams &P, const DevArrays &A, bool forced, const MlpDev *mlp, int32_t *bsum,
                     Launch L);
void launch_log_events(const DevParams &P, const DevArrays &A, int slot, bool forced, Launch L);

// ---- bond sweep (Sec. II.C), exact FP64 decisions ----
void launch_sweep_begin(const DevParams &P, const DevArrays &A, Launch L);
void launch_sweep_reaction(const DevParams &P, const DevArrays &A, int slot, Launch L);
// forced: run even when step % period != 0 (snap_bond_update)
void launch_sweep_begin_forced(const DevParams &P, const DevArrays &A, Launch L);
void launch_sweep_reaction_forced(const DevParams &P, const DevArrays &A, int slot, Launch L);
// clears the per-reaction sweep scratch after a latched status stopped a sweep part-way
void launch_sweep_reset(const DevParams &P, const DevArrays &A, Launch L);

// ---- forces and integration ----
void launch_force(const DevParams &P, const DevArrays &A, bool fp64, bool energy, Launch L);
// force + Langevin update in one kernel; writes the new coordinates to A.pos4n
// (the caller swaps pos4 and pos4n afterwards)
void launch_step_md(const DevParams &P, const DevArrays &A, bool fp64, Launch L);
void launch_step_end(const DevArrays &A, Launch L);
void launch_reduce_cols(const double *src, int ncol, long long n, double *out, Launch L);

// ---- observables (observe.cu): pair-distance histogram behind g(r) of one replica ----
void launch_rdf(const DevParams &P, const DevArrays &A, int rep, int ta, int tb, double rmax, int nbins,
                unsigned long long *hist, Launch L);

// ---- tag-order I/O: dst[rtag[t]] = src[t] (in), dst[t] = src[rtag[t]] (out) ----
template <typename T> void launch_in(T *dst_sorted, const T *src_tag, const int32_t *rtag, long long n, Launch L);
template <typename T> void launch_out(T *dst_tag, const T *src_sorted, const int32_t *rtag, long long n, Launch L);
void launch_force_out(double *dst3, const void *force, bool fp64, const int32_t *rtag, long long n, Launch L);
void launch_iota(int32_t *dst, long long n, Launch L);
// host I/O in tag-ordered (x, y, z) triples, converted on the device (io.cu)
void launch_nonfinite(const double *v, long long m, uint32_t *flag, Launch L);
void launch_pos_in(const double *src3, const DevParams &P, const DevArrays &A, Launch L);
void launch_pos_out(double *dst3, int32_t *img3, const DevParams &P, const DevArrays &A, Launch L);
void launch_vel_in(const double *src3, const DevArrays &A, bool fp64, long long n, Launch L);
void launch_vel_out(double *dst3, const DevArrays &A, bool fp64, long long n, Launch L);
// mixed-mode FP32 velocities <-> tag-ordered FP64 columns
void launch_v4_in(float4 *v4, const double *vx, const double *vy, const double *vz, const int32_t *rtag,
                  long long n, Launch L);
void launch_v4_out(double *vx, double *vy, double *vz, const float4 *v4, const int32_t *rtag, long long n,
                   Launch L);

}  // namespace snap
