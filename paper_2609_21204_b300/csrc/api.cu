// Host runtime behind the C ABI of include/snap.h: context, device memory,
// CUDA-graph capture of MD steps, error latching and tag-order I/O.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/snap.h"
#include "snap_kernels.h"
#include "snap_mlp.h"

using namespace snap;

namespace {

constexpr int kGraphSteps = 20;     // steps captured per CUDA graph launch
constexpr int kPollSteps = 2000;    // status poll interval inside snap_step

struct RxHost {
    int ta, tb, bt;
    double rmin, rmax, pon, poff;
    int self_avoid;
    double slip_a = 0.0;    // slip-bond modifier, Eq. (slip)
    bool melting = false;   // rates from the melting switch, Eqs. (gT)-(kT)
    double melt[6] = {0, 0, 0, 0, 0, 0};   // lambda, T_melt, k_on^init, k_off^init, k_on^melt, k_off^melt
};

struct RepHost {
    int64_t n, tag_off;
    double L[3];
    double kT;
    uint64_t seed;
    int nc[3];
    int cell_off;
};

}  // namespace

struct snap_ctx {
    snap_config cfg{};
    std::string err;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;     // capture stream for conditional bodies
    bool own_stream = false;
    bool fp64 = false;
    int block = 256;
    int64_t n = 0;
    // model
    int ntypes = 0;
    double sigma[kMaxTypes]{}, eps[kMaxTypes * kMaxTypes]{}, rcut[kMaxTypes * kMaxTypes]{};
    bool types_set = false;
    int valence[kMaxTypes]{};
    int bkind[kMaxBondTypes]{};
    double bk[kMaxBondTypes]{}, br0[kMaxBondTypes]{};
    double bx[kMaxBondTypes][3]{};   // FENEWCA: eps, sigma, delta; Tether: l_c1, l_c0, l_max
    bool bset[kMaxBondTypes]{};
    std::vector<RxHost> rx;
    std::vector<std::vector<double>> rep_pon, rep_poff;  // [reaction][replica]
    std::vector<RepHost> reps;
    std::vector<int32_t> sp_host, sbt_host;  // tag-indexed static slots
    std::vector<int32_t> mol_host;          // molecule id by tag, when a reaction excludes them
    int64_t n_static = 0;                     // static bonds added
    int64_t bonds_base = 0;                  // dynamic bonds set explicitly
    // device
    bool ready = false, particles_set = false;
    int ncell_total = 0;
    int nkeys = 0;
    DevParams P{};
    DevArrays A{}, B{};
    RepDev *d_reps = nullptr;
    int32_t *d_bsum = nullptr;
    double *d_red = nullptr;
    double *io3 = nullptr;           // tag-ordered (x, y, z) staging for host I/O
    int32_t *io_img = nullptr;
    uint32_t *io_flag = nullptr;
    std::vector<void *> allocs;
    // Metropolis–Hastings mode and event log
    int mh_mode = 0;                 // 0: DyBond sweep, 1: MH uniform, 2: MH learned
    const snap_mlp *mlp = nullptr;
    double mh_eps = 0.05;
    int mh_nc[3] = {0, 0, 0};
    bool mh_alloc = false;
    long long ev_cap = 0;
    // graphs
    // One instantiated graph per buffer parity: a step swaps pos4/pos4n, so a
    // call whose step count leaves a remainder starts the next call on the
    // other buffer; its graph is kept rather than recaptured.
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    void *graph_key[2] = {nullptr, nullptr};   // A.pos4 when each graph was captured
    bool graph_dirty = true;                    // both graphs stale (parameters or buffers changed)
    int nbr_cap = 0;
    int rnbr_cap = 0;
    int cas_cap = 1 << 16;           // push-mode compare-and-swap retries (snap_set_retry_limit)
    int list_block = 256;            // threads per block of the list build (snap_set_list_block)
    int list_sub = 0;                // sub-cells along x per cell requested (snap_set_list_subcells; 0: automatic)
    int sub_shift = 0;               // log2 of the sub-cells in use (set when the cell grid is laid out)
    int kinetic_T = 0;               // sweep temperature: 0 set-point, 1 kinetic (snap_set_kinetic_temperature)
};

namespace {

snap_status fail(snap_ctx *c, snap_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

#define CUDA_TRY(c, expr)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail((c), SNAP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void *dalloc(snap_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (c->cfg.alloc) {
        p = c->cfg.alloc(bytes, c->cfg.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocs.push_back(p);
    return p;
}

void dfree(snap_ctx *c, void *p)
{
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    if (c->cfg.free) c->cfg.free(p, c->cfg.alloc_user);
    else cudaFree(p);
}

template <typename T> bool alloc_arr(snap_ctx *c, T *&p, size_t count)
{
    p = static_cast<T *>(dalloc(c, sizeof(T) * count));
    return p != nullptr;
}

Launch launch(snap_ctx *c) { return Launch{c->stream, c->block}; }
Launch launch_on(snap_ctx *c, cudaStream_t s) { return Launch{s, c->block}; }

uint32_t morton2(uint32_t y, uint32_t z)
{
    uint32_t m = 0;
    for (int b = 0; b < 10; ++b) m |= ((y >> b) & 1u) << (2 * b) | ((z >> b) & 1u) << (2 * b + 1);
    return m;
}

// Margin added to every list cut-off: 1e-4, or more where the FP32 wrapped
// positions the list build compares are coarser (8 units in the last place of
// the largest box edge).
double list_margin(const snap_ctx *c)
{
    double lmax = 0.0;
    for (const auto &R : c->reps) lmax = std::max({lmax, R.L[0], R.L[1], R.L[2]});
    return std::max(1e-4, 8.0 * std::ldexp(1.0, std::ilogb(std::max(lmax, 1.0)) - 23));
}

double pair_rc(const snap_ctx *c, int a, int b)
{
    const double rc = c->rcut[a * kMaxTypes + b];
    if (rc > 0.0) return rc;
    const double sig = 0.5 * (c->sigma[a] + c->sigma[b]);
    return sig * std::pow(2.0, 1.0 / 6.0);
}

double reactive_cut(const snap_ctx *c, int a, int b)
{
    double m = 0.0;
    for (const auto &r : c->rx)
        if ((r.ta == a && r.tb == b) || (r.ta == b && r.tb == a)) m = std::max(m, r.rmax);
    return m;
}

snap_status upload_reps(snap_ctx *c)
{
    std::vector<RepDev> h(c->reps.size());
    for (size_t r = 0; r < c->reps.size(); ++r) {
        const RepHost &R = c->reps[r];
        RepDev &D = h[r];
        std::memset(&D, 0, sizeof D);
        for (int d = 0; d < 3; ++d) {
            D.L[d] = R.L[d];
            D.invL[d] = 1.0 / R.L[d];
            D.halfL[d] = 0.5 * R.L[d];
            D.nc[d] = R.nc[d];
            D.w[d] = R.nc[d] > 0 ? R.L[d] / (double)R.nc[d] : R.L[d];
            D.wf[d] = (float)D.w[d];
            D.cscale[d] = (float)((double)R.nc[d] / R.L[d]);
        }
        D.cell_off = R.cell_off;
        D.tag_off = R.tag_off;
        D.n = R.n;
        D.kT = R.kT;
        D.t_sweep = R.kT;
        D.noise_c = std::sqrt(((2.0 * c->cfg.gamma) * R.kT) / c->cfg.dt);
        D.noise_cf = (float)D.noise_c;
        D.key0 = (uint32_t)(R.seed & 0xFFFFFFFFull);
        D.key1hi = (uint32_t)(((R.seed >> 32) & 0xFFFFull) << 16);
        for (int d = 0; d < 3; ++d) D.mh_nc[d] = c->mh_nc[d];
        for (size_t a = 0; a < c->rx.size(); ++a) {
            D.p_on0[a] = c->rep_pon[a][r];
            D.p_off[a] = c->rep_poff[a][r];
            // p_off * 2^53 is exact (scaling by a power of two); u53 = m 2^-53 < p_off
            // holds exactly when the integer m is below its ceiling
            D.off_thresh[a] = (unsigned long long)std::ceil(std::ldexp(D.p_off[a], 53));
        }
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_reps, h.data(), sizeof(RepDev) * h.size(), cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

// The separation a proposal aims at (Sec. II.C: the partner minimising
// |r - r0|, r0 read from the bond potential), read as the minimum of the bond
// energy: r0 (harmonic); 0 (FENE); for FENEWCA delta + s*, s* the root of
// dU/ds on (0, min(2^(1/6) sigma, R0)) found by bisection to the last bit (dU/ds
// rises there from -inf; delta itself when eps = 0); for Tether, whose energy
// is zero on [l_c1, l_c0], the middle of that interval.  The oracle computes
// the same value with the same operations.
double aim_separation(const snap_ctx *c, int bt)
{
    const int kind = c->bkind[bt];
    if (kind == SNAP_HARMONIC) return c->br0[bt];
    if (kind == SNAP_FENE) return 0.0;
    if (kind == SNAP_TETHER) return 0.5 * (c->bx[bt][0] + c->bx[bt][1]);
    const double k = c->bk[bt], R0 = c->br0[bt], eps = c->bx[bt][0], sig = c->bx[bt][1], delta = c->bx[bt][2];
    if (eps == 0.0) return delta;
    double lo = 0.0, hi = std::min(sig * kTwoSixth, R0);
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        const double q = (mid * mid) / (R0 * R0);
        const double f1 = (k * mid) / (1.0 - q);
        const double sr2 = (sig * sig) / (mid * mid);
        const double sr6 = (sr2 * sr2) * sr2;
        const double f2 = ((24.0 * eps) * ((2.0 * sr6) * sr6 - sr6)) / mid;
        if (f1 - f2 > 0.0) hi = mid;
        else lo = mid;
    }
    return delta + hi;
}

void fill_params(snap_ctx *c)
{
    DevParams &P = c->P;
    std::memset(&P, 0, sizeof P);
    P.ntypes = c->ntypes;
    P.nrx = (int)c->rx.size();
    P.period = c->cfg.bond_period;
    P.nhist = c->cfg.lifetime_bins;
    for (int t = 0; t < kMaxTypes; ++t) P.valence[t] = c->valence[t];
    const double skin = c->cfg.skin;
    const double margin = list_margin(c);
    for (int a = 0; a < c->ntypes; ++a)
        for (int b = 0; b < c->ntypes; ++b) {
            const int k = a * kMaxTypes + b;
            const double rc = pair_rc(c, a, b);
            const double sig = 0.5 * (c->sigma[a] + c->sigma[b]);
            const double e = c->eps[k];
            const double fl = rc + skin + margin;
            const double xc = reactive_cut(c, a, b);
            const double xl = xc > 0.0 ? xc + skin + margin : 0.0;
            P.rc2d[k] = rc * rc;
            P.rc2f[k] = (float)(rc * rc);
            P.fl2f[k] = (float)(fl * fl);
            P.xl2f[k] = (float)(xl * xl);
            P.sig2d[k] = sig * sig;
            P.sig2f[k] = (float)(sig * sig);
            P.eps24d[k] = 24.0 * e;
            P.eps24f[k] = (float)(24.0 * e);
            const double c2 = (sig * sig) / (rc * rc), c6 = c2 * c2 * c2;
            P.shiftd[k] = 4.0 * e * (c6 * c6 - c6);
            P.shiftf[k] = (float)P.shiftd[k];
        }
    for (int b = 0; b < kMaxBondTypes; ++b) {
        P.bkind[b] = c->bkind[b];
        P.bk[b] = c->bk[b];
        P.br0[b] = c->br0[b];
        P.bkf[b] = (float)c->bk[b];
        P.br0f[b] = (float)c->br0[b];
        for (int k = 0; k < 3; ++k) {
            P.bx[b][k] = c->bx[b][k];
            P.bxf[b][k] = (float)c->bx[b][k];
        }
    }
    for (size_t a = 0; a < c->rx.size(); ++a) {
        P.rx_ta[a] = c->rx[a].ta;
        P.rx_tb[a] = c->rx[a].tb;
        P.rx_bt[a] = c->rx[a].bt;
        P.rx_self[a] = c->rx[a].self_avoid;
        P.rx_slip[a] = c->rx[a].slip_a;
        // proposals aim at the minimum of the bond energy
        P.rx_r0[a] = aim_separation(c, c->rx[a].bt);
        if (c->rx[a].slip_a != 0.0) P.slip_mask |= 1 << a;
        P.rx_rmin2[a] = c->rx[a].rmin * c->rx[a].rmin;
        P.rx_rmax2[a] = c->rx[a].rmax * c->rx[a].rmax;
    }
    P.dt = c->cfg.dt;
    P.half_dt = 0.5 * c->cfg.dt;
    P.gamma = c->cfg.gamma;
    P.sqrt3 = std::sqrt(3.0);
    P.dtf = (float)P.dt;
    P.gammaf = (float)P.gamma;
    P.sqrt3f = (float)P.sqrt3;
    const double dmax = 0.5 * skin - 1e-4;
    P.disp2f = (float)(dmax * dmax);
    P.nbr_cap = c->nbr_cap;
    P.rnbr_cap = c->rnbr_cap;
    P.n = c->n;
    P.nbr_stride = ((c->n + 31) / 32) * 32;
    P.nrep = (int)c->reps.size();
    P.screen = c->fp64 ? 0 : 1;
    P.ncell = c->ncell_total;
    P.sub_shift = c->sub_shift;
    P.mh_cells = c->mh_mode ? c->mh_nc[0] * c->mh_nc[1] * c->mh_nc[2] : 0;
    P.mh_moves = c->mh_mode ? P.mh_cells / 8 : 0;
    P.mh_eps = (float)c->mh_eps;
    P.log_events = c->ev_cap > 0 ? 1 : 0;
    P.pdist_rows = std::max<int64_t>(c->n, 1) / 5 + 1;
    P.has_static = c->n_static > 0 ? 1 : 0;   // push mode needs a side 4x scarcer: <= n / 5 sites
    P.cas_cap = c->cas_cap;
    P.kinetic_T = c->kinetic_T;
    P.period_dt = (double)c->cfg.bond_period * c->cfg.dt;
    for (size_t a = 0; a < c->rx.size(); ++a) {
        if (!c->rx[a].melting) continue;
        P.melt_mask |= 1 << a;
        P.melt_lambda[a] = c->rx[a].melt[0];
        P.melt_t[a] = c->rx[a].melt[1];
        P.kon_init[a] = c->rx[a].melt[2];
        P.koff_init[a] = c->rx[a].melt[3];
        P.kon_melt[a] = c->rx[a].melt[4];
        P.koff_melt[a] = c->rx[a].melt[5];
    }
}

// everything that depends on the model (cut-offs -> cell grids -> capacities)
// Molecule ids (Sec. II.D): connected components of the static bonds by
// union-find over tags, each labelled by its smallest tag; uploaded by tag
// when some reaction excludes intramolecular partners, else nothing.
snap_status upload_molecules(snap_ctx *c)
{
    bool any = false;
    for (const auto &r : c->rx) any = any || r.self_avoid;
    if (!any) return SNAP_OK;
    const int64_t n = c->n;
    std::vector<int32_t> up((size_t)n);
    for (int64_t t = 0; t < n; ++t) up[t] = (int32_t)t;
    auto root = [&](int32_t x) {
        while (up[x] != x) {
            up[x] = up[up[x]];
            x = up[x];
        }
        return x;
    };
    for (int64_t t = 0; t < n; ++t)
        for (int s = 0; s < kSmax; ++s) {
            const int32_t u = c->sp_host[4 * (size_t)t + s];
            if (u < 0) continue;
            const int32_t ra = root((int32_t)t), rb = root(u);
            if (ra != rb) up[std::max(ra, rb)] = std::min(ra, rb);   // the smaller tag stays the root
        }
    c->mol_host.resize((size_t)n);
    for (int64_t t = 0; t < n; ++t) c->mol_host[t] = root((int32_t)t);
    if (!c->A.mol && !alloc_arr(c, c->A.mol, (size_t)std::max<int64_t>(n, 1)))
        return fail(c, SNAP_ERR_OOM, "molecule ids");
    CUDA_TRY(c, cudaMemcpyAsync(c->A.mol, c->mol_host.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

snap_status ensure_ready(snap_ctx *c)
{
    if (c->ready) return SNAP_OK;
    if (!c->types_set) return fail(c, SNAP_ERR_STATE, "snap_set_types has not been called");
    double rl_max = 0.0, rf_max = 0.0, rx_max = 0.0;
    for (int a = 0; a < c->ntypes; ++a)
        for (int b = 0; b < c->ntypes; ++b) {
            rf_max = std::max(rf_max, pair_rc(c, a, b));
            rx_max = std::max(rx_max, reactive_cut(c, a, b));
        }
    rl_max = std::max(rf_max, rx_max);
    // the 1e-3 margin covers the FP32 cell assignment (a particle may sit up to
    // ~1e-4 outside the cell it is filed under)
    const double cell_min = rl_max + c->cfg.skin + list_margin(c) + 1e-3;
    int off = 0;
    double dens_max = 0.0;
    for (auto &R : c->reps) {
        for (int d = 0; d < 3; ++d) {
            R.nc[d] = (int)std::floor(R.L[d] / cell_min);
            if (R.nc[d] < 3)
                return fail(c, SNAP_ERR_ARG, "box edge shorter than three neighbour cells (3 x " +
                                                 std::to_string(cell_min) + ")");
            if (R.nc[d] > 511) return fail(c, SNAP_ERR_ARG, "more than 511 cells along an axis");
        }
        R.cell_off = off;
        off += R.nc[0] * R.nc[1] * R.nc[2];
        dens_max = std::max(dens_max, (double)R.n / (R.L[0] * R.L[1] * R.L[2]));
    }
    c->ncell_total = off;
    // capacities: expected neighbours within each list's largest cut-off, doubled, + margin
    auto expect_cap = [&](double cut) {
        const double rl = cut + c->cfg.skin + 1e-4;
        const int cap = (int)std::ceil(dens_max * 4.0 / 3.0 * M_PI * rl * rl * rl * 2.0 + 16.0);
        return (cap + 7) & ~7;
    };
    if (c->nbr_cap <= 0) c->nbr_cap = expect_cap(rf_max);
    if (c->rnbr_cap <= 0) c->rnbr_cap = rx_max > 0.0 ? expect_cap(rx_max) : 8;
    // cell tables: cells ranked x innermost (the three cells of a row around a
    // particle are one run of the sorted particles), rows in 2-D Morton order
    // of (y, z) so that neighbouring rows stay close in memory
    std::vector<int32_t> rank_of(off);
    for (const auto &R : c->reps) {
        const int nx = R.nc[0], ny = R.nc[1], nz = R.nc[2];
        std::vector<std::pair<uint32_t, int>> rows;
        rows.reserve((size_t)ny * nz);
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y) rows.emplace_back(morton2(y, z), z * ny + y);
        std::sort(rows.begin(), rows.end());
        for (size_t k = 0; k < rows.size(); ++k)
            for (int x = 0; x < nx; ++x)
                rank_of[R.cell_off + rows[k].second * nx + x] = R.cell_off + (int)k * nx + x;
    }
    DevArrays &A = c->A;
    // sort keys: (type, cell, sub-cell along x).  Sub-cells per cell: as
    // requested, else the most (<= 8) that keep at least half a particle per key
    // on average; fewer where the key count would pass the scan's limit.
    constexpr long long kMaxKeys = (long long)4096 * 4096;
    const long long ncoarse = (long long)off * c->ntypes;
    if (ncoarse > kMaxKeys) return fail(c, SNAP_ERR_ARG, "too many cells x types");
    int sh = 0;
    if (c->list_sub > 0) {
        while ((1 << sh) < c->list_sub) ++sh;
    } else {
        while (sh < 3 && (ncoarse << (sh + 1)) <= 2 * (long long)c->n) ++sh;
    }
    while (sh > 0 && (ncoarse << sh) > kMaxKeys) --sh;
    c->sub_shift = sh;
    const long long nkeys = ncoarse << sh;
    c->nkeys = (int)nkeys;
    const int nb = (int)((nkeys + 4095) / 4096) + 1;
    if (!alloc_arr(c, A.cell_count, nkeys) || !alloc_arr(c, A.cell_start, nkeys + 1) ||
        !alloc_arr(c, A.cell_cursor, nkeys) || !alloc_arr(c, A.rank_of, off) || !alloc_arr(c, c->d_bsum, nb + 1))
        return fail(c, SNAP_ERR_OOM, "cell arrays");
    CUDA_TRY(c, cudaMemsetAsync(A.cell_count, 0, sizeof(int32_t) * nkeys, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(A.cell_cursor, 0, sizeof(int32_t) * nkeys, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(A.rank_of, rank_of.data(), sizeof(int32_t) * off, cudaMemcpyHostToDevice,
                                c->stream));
    const int64_t stride = ((c->n + 31) / 32) * 32;
    if (!alloc_arr(c, A.nbr, (size_t)stride * c->nbr_cap) || !alloc_arr(c, A.rnbr, (size_t)stride * c->rnbr_cap))
        return fail(c, SNAP_ERR_OOM, "neighbour lists");
    fill_params(c);
    snap_status s = upload_reps(c);
    if (s != SNAP_OK) return s;
    if ((s = upload_molecules(c)) != SNAP_OK) return s;
    c->ready = true;
    c->graph_dirty = true;
    return SNAP_OK;
}

// ---- kernel sequences -------------------------------------------------
void seq_rebuild(snap_ctx *c, cudaStream_t stream = nullptr)
{
    const Launch L = launch_on(c, stream ? stream : c->stream);
    launch_cell_key(c->P, c->A, L);
    launch_cell_scan(c->A, c->d_bsum, c->nkeys, L);
    launch_scatter(c->P, c->A, c->d_bsum, L);
    launch_cell_sort(c->A, c->nkeys, c->d_bsum, L);
    launch_gather(c->P, c->A, c->B, c->fp64, L);
    launch_nlist(c->P, c->A, c->B, c->fp64, c->list_block, L);   // copies the gathered arrays back too
    launch_rebuild_done(c->A, L);
}

void seq_sweep(snap_ctx *c, bool forced)
{
    if (c->rx.empty()) return;
    const Launch L = launch(c);
    if (c->mh_mode) {
        launch_mh_sweep(c->P, c->A, forced, c->mh_mode == 2 ? &c->mlp->dev : nullptr, c->A.mh_bsum, L);
        return;
    }
    if (forced) launch_sweep_begin_forced(c->P, c->A, L);
    else launch_sweep_begin(c->P, c->A, L);
    for (int s = 0; s < (int)c->rx.size(); ++s) {
        if (forced) launch_sweep_reaction_forced(c->P, c->A, s, L);
        else launch_sweep_reaction(c->P, c->A, s, L);
    }
}

// force + integration in one kernel that writes the new coordinates to the
// second buffer; the host swaps the two buffers after queueing it
void seq_md(snap_ctx *c, Launch L)
{
    launch_step_md(c->P, c->A, c->fp64, L);
    std::swap(c->A.pos4, c->A.pos4n);
}

void seq_step(snap_ctx *c)
{
    const Launch L = launch(c);
    seq_rebuild(c);
    seq_sweep(c, false);
    seq_md(c, L);
    launch_step_end(c->A, L);
}

// One captured step whose neighbour-list rebuild is the body of a conditional
// (IF) node: between rebuilds the eight rebuild kernels are not launched at all.
// first: the graph's first step; the others end the step before them in the
// condition kernel, last: the graph's last step, which ends with k_step_end.
cudaError_t capture_step_conditional(snap_ctx *c, bool first, bool last)
{
    const Launch L = launch(c);
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
    if (e != cudaSuccess) return e;
    launch_set_rebuild_cond(c->A, h, !first, L);
    e = cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
    if (e != cudaSuccess) return e;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCaptureToGraph(c->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    seq_rebuild(c, c->side);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(c->side, &out);
    if (e != cudaSuccess) return e;
    seq_sweep(c, false);
    seq_md(c, L);
    if (last) launch_step_end(c->A, L);
    return cudaGetLastError();
}

// Graph mode: SNAP_GRAPH_MODE=conditional (default: rebuild kernels inside an
// IF node), plain (every kernel in the graph, rebuild kernels exit early when
// no rebuild is due; kernels in such graphs can be profiled one by one), none
// (no graphs, one launch per kernel).
int graph_mode()
{
    const char *m = std::getenv("SNAP_GRAPH_MODE");
    if (!m) return 0;
    if (!std::strcmp(m, "plain")) return 1;
    if (!std::strcmp(m, "none")) return 2;
    return 0;
}

void end_dangling_capture(cudaStream_t s)
{
    if (!s) return;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
        cudaGraph_t g = nullptr;
        if (cudaStreamEndCapture(s, &g) == cudaSuccess && g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
}

void drop_graphs(snap_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
        c->graph_key[k] = nullptr;
    }
}

// Capture kGraphSteps steps starting from the current buffer parity into
// graph slot k.  Capturing queues nothing: the stream runs no work until the
// graph is launched.
snap_status build_graph(snap_ctx *c, int k)
{
    if (c->graph[k]) {
        cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
        c->graph_key[k] = nullptr;
    }
    const int mode = graph_mode();
    if (!c->side) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    static_assert(kGraphSteps % 2 == 0, "a graph must swap pos4/pos4n an even number of times");
    void *const pos4_0 = c->A.pos4, *const pos4_1 = c->A.pos4n;   // restored after the capture
    CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    for (int s = 0; s < kGraphSteps && ce == cudaSuccess; ++s) {
        if (mode == 1) {
            seq_step(c);
            ce = cudaGetLastError();
        } else {
            ce = capture_step_conditional(c, s == 0, s == kGraphSteps - 1);
        }
    }
    c->A.pos4 = pos4_0;   // an even number of swaps; also undoes a capture that stopped early
    c->A.pos4n = pos4_1;
    if (ce != cudaSuccess) {
        end_dangling_capture(c->side);
        end_dangling_capture(c->stream);
        return fail(c, SNAP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    }
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) return fail(c, SNAP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, SNAP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    c->graph[k] = ex;
    c->graph_key[k] = pos4_0;
    return SNAP_OK;
}

// The graph for the current buffer parity, captured on first use (*out is
// its slot).  Stale graphs are dropped first.
snap_status graph_for_parity(snap_ctx *c, int &out)
{
    if (c->graph_dirty) {
        drop_graphs(c);
        c->graph_dirty = false;
    }
    for (int k = 0; k < 2; ++k)
        if (c->graph[k] && c->graph_key[k] == c->A.pos4) {
            out = k;
            return SNAP_OK;
        }
    const int k = c->graph[0] ? 1 : 0;
    snap_status s = build_graph(c, k);
    if (s != SNAP_OK) {
        c->graph_dirty = true;
        return s;
    }
    out = k;
    return SNAP_OK;
}

snap_status read_status(snap_ctx *c, uint32_t &st)
{
    CUDA_TRY(c, cudaMemcpyAsync(&st, c->A.status, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

snap_status clear_status(snap_ctx *c)
{
    CUDA_TRY(c, cudaMemsetAsync(c->A.status, 0, sizeof(uint32_t), c->stream));
    return SNAP_OK;
}

// After a latched status: clear it and the sweep scratch a stopped sweep may
// have left behind.  The step that latched it did not complete (the step
// counter did not advance).
snap_status recover_status(snap_ctx *c)
{
    snap_status s = clear_status(c);
    if (s != SNAP_OK) return s;
    if (c->ready && c->particles_set) launch_sweep_reset(c->P, c->A, launch(c));
    CUDA_TRY(c, cudaGetLastError());
    return SNAP_OK;
}

snap_status set_need_rebuild(snap_ctx *c)
{
    const int32_t one = 1;
    CUDA_TRY(c, cudaMemcpyAsync(c->A.need_rebuild, &one, sizeof one, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

// Neighbour capacity exceeded: grow, force a rebuild, clear the status.  The
// rebuild happens at the start of a step before any state changes, and every
// kernel after it returns early while the status is set, so the step is
// simply retried.
snap_status grow_nlist(snap_ctx *c)
{
    int32_t need[2] = {0, 0};
    CUDA_TRY(c, cudaMemcpyAsync(need, c->A.nbr_need, sizeof need, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int64_t stride = ((c->n + 31) / 32) * 32;
    int *caps[2] = {&c->nbr_cap, &c->rnbr_cap};
    int32_t **lists[2] = {&c->A.nbr, &c->A.rnbr};
    for (int l = 0; l < 2; ++l) {
        if (need[l] <= *caps[l]) continue;
        int cap = std::max(need[l] + need[l] / 4 + 8, *caps[l] + 8);
        cap = (cap + 7) & ~7;
        dfree(c, *lists[l]);
        *lists[l] = nullptr;
        if (!alloc_arr(c, *lists[l], (size_t)stride * cap)) return fail(c, SNAP_ERR_OOM, "neighbour list regrow");
        *caps[l] = cap;
    }
    c->P.nbr_cap = c->nbr_cap;
    c->P.rnbr_cap = c->rnbr_cap;
    c->graph_dirty = true;
    snap_status s = clear_status(c);
    if (s != SNAP_OK) return s;
    return set_need_rebuild(c);
}

snap_status status_to_code(snap_ctx *c, uint32_t st)
{
    if (st == 0) return SNAP_OK;
    if (st & kStNonfinite) return fail(c, SNAP_ERR_NONFINITE, "non-finite position");
    if (st & kStFene)
        return fail(c, SNAP_ERR_FENE_OVERSTRETCH,
                    "a bond outside the finite range of its potential (FENE/FENEWCA beyond R0, Tether at l_min or l_max)");
    if (st & kStOverflow) return fail(c, SNAP_ERR_NLIST_OVERFLOW, "neighbour list overflow");
    if (st & kStTimeout) return fail(c, SNAP_ERR_TIMEOUT, "a bounded device retry loop gave up");
    return fail(c, SNAP_ERR_STATE, "unknown device status");
}

// run a non-graph sequence with overflow retry (rebuild + f)
template <typename F> snap_status run_with_retry(snap_ctx *c, F f)
{
    for (int attempt = 0; attempt < 8; ++attempt) {
        f();
        CUDA_TRY(c, cudaGetLastError());
        uint32_t st = 0;
        snap_status s = read_status(c, st);
        if (s != SNAP_OK) return s;
        if (st == kStOverflow) {
            s = grow_nlist(c);
            if (s != SNAP_OK) return s;
            continue;
        }
        if (st) {
            recover_status(c);
            return status_to_code(c, st);
        }
        return SNAP_OK;
    }
    return fail(c, SNAP_ERR_NLIST_OVERFLOW, "neighbour list kept overflowing");
}

snap_status check_ready(snap_ctx *c)
{
    if (!c) return SNAP_ERR_ARG;
    snap_status s = ensure_ready(c);
    if (s != SNAP_OK) return s;
    if (!c->particles_set) return fail(c, SNAP_ERR_STATE, "snap_set_particles has not been called");
    return SNAP_OK;
}

void wrap_host(double &x, int32_t &img, double L)
{
    const double k = std::floor(x / L);
    x -= k * L;
    img += (int32_t)k;
    if (x >= L) { x -= L; img += 1; }
    if (x < 0.0) { x += L; img -= 1; }
    if (x >= L) x = 0.0;
}

int rep_of_tag(const snap_ctx *c, int64_t t)
{
    int lo = 0, hi = (int)c->reps.size() - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (c->reps[mid].tag_off <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// upload tag-ordered host data into the current memory order through staging
template <typename T> snap_status upload_in(snap_ctx *c, T *dst, T *stage, const T *host, size_t count)
{
    CUDA_TRY(c, cudaMemcpyAsync(stage, host, sizeof(T) * count, cudaMemcpyHostToDevice, c->stream));
    launch_in<T>(dst, stage, c->A.rtag, (long long)count, launch(c));
    CUDA_TRY(c, cudaGetLastError());
    return SNAP_OK;
}

template <typename T> snap_status download_out(snap_ctx *c, T *host, const T *src, T *stage, size_t count)
{
    launch_out<T>(stage, src, c->A.rtag, (long long)count, launch(c));
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(host, stage, sizeof(T) * count, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

snap_status upload_static(snap_ctx *c)
{
    std::vector<int4> sp(c->n);
    std::vector<int32_t> sbt(c->n);
    for (int64_t t = 0; t < c->n; ++t) {
        sp[t] = make_int4(c->sp_host[4 * t], c->sp_host[4 * t + 1], c->sp_host[4 * t + 2], c->sp_host[4 * t + 3]);
        sbt[t] = c->sbt_host[t];
    }
    snap_status s = upload_in<int4>(c, c->A.sp, c->B.sp, sp.data(), c->n);
    if (s != SNAP_OK) return s;
    s = upload_in<int32_t>(c, c->A.sbt, c->B.sbt, sbt.data(), c->n);
    if (s != SNAP_OK) return s;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

snap_status positions_in(snap_ctx *c, const double *pos3, std::vector<int32_t> *img)
{
    std::vector<double> xs[3];
    for (int d = 0; d < 3; ++d) xs[d].resize(c->n);
    for (int64_t t = 0; t < c->n; ++t) {
        const RepHost &R = c->reps[rep_of_tag(c, t)];
        for (int d = 0; d < 3; ++d) {
            double x = pos3[3 * t + d];
            if (!std::isfinite(x)) return fail(c, SNAP_ERR_NONFINITE, "non-finite input position");
            int32_t im = 0;
            wrap_host(x, im, R.L[d]);
            xs[d][t] = x;
            if (img) (*img)[3 * t + d] = im;
        }
    }
    double *dst[3] = {c->A.x, c->A.y, c->A.z};
    double *stg[3] = {c->B.x, c->B.y, c->B.z};
    for (int d = 0; d < 3; ++d) {
        snap_status s = upload_in<double>(c, dst[d], stg[d], xs[d].data(), c->n);
        if (s != SNAP_OK) return s;
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

snap_status velocities_in(snap_ctx *c, const double *vel3)
{
    std::vector<double> vs[3];
    for (int d = 0; d < 3; ++d) vs[d].assign(c->n, 0.0);
    if (vel3)
        for (int64_t t = 0; t < c->n; ++t)
            for (int d = 0; d < 3; ++d) vs[d][t] = vel3[3 * t + d];
    double *dst[3] = {c->A.vx, c->A.vy, c->A.vz};
    double *stg[3] = {c->B.vx, c->B.vy, c->B.vz};
    if (c->fp64) {
        for (int d = 0; d < 3; ++d) {
            snap_status s = upload_in<double>(c, dst[d], stg[d], vs[d].data(), c->n);
            if (s != SNAP_OK) return s;
        }
    } else {
        // FP32 velocities in mixed mode: stage in tag order, convert and scatter
        for (int d = 0; d < 3; ++d)
            CUDA_TRY(c, cudaMemcpyAsync(stg[d], vs[d].data(), sizeof(double) * c->n, cudaMemcpyHostToDevice,
                                        c->stream));
        launch_v4_in(c->A.v4, stg[0], stg[1], stg[2], c->A.rtag, c->n, launch(c));
        CUDA_TRY(c, cudaGetLastError());
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

struct BondRec {
    int32_t a, b, rx, birth;
};

snap_status bonds_in(snap_ctx *c, const std::vector<BondRec> &bonds)
{
    std::vector<std::vector<BondRec>> per(c->n);
    for (const auto &bd : bonds) {
        per[bd.a].push_back(bd);
        per[bd.b].push_back(BondRec{bd.b, bd.a, bd.rx, bd.birth});
    }
    std::vector<int4> dp(c->n), db(c->n);
    std::vector<int32_t> drx(c->n), occ(c->n);
    for (int64_t t = 0; t < c->n; ++t) {
        auto &v = per[t];
        if ((int)v.size() > kVmax) return fail(c, SNAP_ERR_ARG, "more than SNAP_MAX_VALENCE dynamic bonds on a particle");
        std::sort(v.begin(), v.end(), [](const BondRec &x, const BondRec &y) { return x.b < y.b; });
        int p[4] = {-1, -1, -1, -1}, bi[4] = {0, 0, 0, 0}, r[4] = {0, 0, 0, 0};
        for (size_t s = 0; s < v.size(); ++s) {
            if (s > 0 && v[s].b == v[s - 1].b) return fail(c, SNAP_ERR_ARG, "duplicate dynamic bond");
            p[s] = v[s].b;
            bi[s] = v[s].birth;
            r[s] = v[s].rx;
        }
        dp[t] = make_int4(p[0], p[1], p[2], p[3]);
        db[t] = make_int4(bi[0], bi[1], bi[2], bi[3]);
        drx[t] = (r[0] & 0xFF) | ((r[1] & 0xFF) << 8) | ((r[2] & 0xFF) << 16) | ((r[3] & 0xFF) << 24);
        occ[t] = (int32_t)v.size();
    }
    snap_status s;
    if ((s = upload_in<int4>(c, c->A.dp, c->B.dp, dp.data(), c->n)) != SNAP_OK) return s;
    if ((s = upload_in<int4>(c, c->A.dbirth, c->B.dbirth, db.data(), c->n)) != SNAP_OK) return s;
    if ((s = upload_in<int32_t>(c, c->A.drx, c->B.drx, drx.data(), c->n)) != SNAP_OK) return s;
    if ((s = upload_in<int32_t>(c, c->A.occ, c->B.occ, occ.data(), c->n)) != SNAP_OK) return s;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

snap_status bonds_out(snap_ctx *c, std::vector<BondRec> &out)
{
    std::vector<int4> dp(c->n), db(c->n);
    std::vector<int32_t> drx(c->n);
    snap_status s;
    if ((s = download_out<int4>(c, dp.data(), c->A.dp, c->B.dp, c->n)) != SNAP_OK) return s;
    if ((s = download_out<int4>(c, db.data(), c->A.dbirth, c->B.dbirth, c->n)) != SNAP_OK) return s;
    if ((s = download_out<int32_t>(c, drx.data(), c->A.drx, c->B.drx, c->n)) != SNAP_OK) return s;
    out.clear();
    for (int64_t t = 0; t < c->n; ++t) {
        const int p[4] = {dp[t].x, dp[t].y, dp[t].z, dp[t].w};
        const int b[4] = {db[t].x, db[t].y, db[t].z, db[t].w};
        for (int k = 0; k < kVmax; ++k)
            if (p[k] > t) out.push_back(BondRec{(int32_t)t, p[k], (drx[t] >> (8 * k)) & 0xFF, b[k]});
    }
    std::sort(out.begin(), out.end(),
              [](const BondRec &x, const BondRec &y) { return x.a != y.a ? x.a < y.a : x.b < y.b; });
    return SNAP_OK;
}

snap_status counters_out(snap_ctx *c, unsigned long long *h)
{
    std::vector<unsigned long long> raw((size_t)cNumCounters * kCopies);
    CUDA_TRY(c, cudaMemcpyAsync(raw.data(), c->A.counters, sizeof(unsigned long long) * raw.size(),
                                cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < cNumCounters; ++k) {
        h[k] = 0ull;
        for (int q = 0; q < kCopies; ++q) h[k] += raw[(size_t)k * kCopies + q];
    }
    return SNAP_OK;
}

}  // namespace

// ====================================================================== ABI

extern "C" snap_status snap_init(snap_ctx **out, const snap_config *cfg)
{
    if (!out) return SNAP_ERR_ARG;
    *out = nullptr;
    if (!cfg) return SNAP_ERR_ARG;
    if (cfg->n < 0 || cfg->n >= kMaxParticles) return SNAP_ERR_ARG;
    if (!(cfg->dt > 0.0) || !(cfg->kT >= 0.0) || !(cfg->gamma >= 0.0) || !(cfg->skin > 0.0)) return SNAP_ERR_ARG;
    if (cfg->precision != SNAP_FP64 && cfg->precision != SNAP_MIXED) return SNAP_ERR_ARG;
    if (cfg->bond_period < 1) return SNAP_ERR_ARG;
    if (cfg->block_size < 0 || cfg->block_size > 256 || (cfg->block_size % 32) != 0) return SNAP_ERR_ARG;
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr)) return SNAP_ERR_ARG;
    const int nrep = cfg->n_replicas > 1 ? cfg->n_replicas : 1;
    if (cfg->n_replicas > 1 && !cfg->replica_n) return SNAP_ERR_ARG;
    std::vector<RepHost> reps(nrep);
    int64_t off = 0;
    for (int r = 0; r < nrep; ++r) {
        RepHost &R = reps[r];
        R.n = cfg->n_replicas > 1 ? cfg->replica_n[r] : cfg->n;
        if (R.n < 0) return SNAP_ERR_ARG;
        R.tag_off = off;
        off += R.n;
        for (int d = 0; d < 3; ++d) {
            R.L[d] = (cfg->n_replicas > 1 && cfg->replica_box) ? cfg->replica_box[3 * r + d] : cfg->box[d];
            if (!(R.L[d] > 0.0) || !std::isfinite(R.L[d])) return SNAP_ERR_ARG;
        }
        R.kT = (cfg->n_replicas > 1 && cfg->replica_kT) ? cfg->replica_kT[r] : cfg->kT;
        if (!(R.kT >= 0.0)) return SNAP_ERR_ARG;
        R.seed = (cfg->n_replicas > 1 && cfg->replica_seed) ? cfg->replica_seed[r] : cfg->seed + (uint64_t)r;
        R.nc[0] = R.nc[1] = R.nc[2] = 0;
        R.cell_off = 0;
    }
    if (off != cfg->n) return SNAP_ERR_ARG;

    snap_ctx *c = new snap_ctx();
    c->cfg = *cfg;
    c->cfg.replica_n = nullptr;
    c->cfg.replica_box = nullptr;
    c->cfg.replica_kT = nullptr;
    c->cfg.replica_seed = nullptr;
    if (c->cfg.lifetime_bins <= 0) c->cfg.lifetime_bins = 256;
    c->reps = reps;
    c->n = cfg->n;
    c->fp64 = cfg->precision == SNAP_FP64;
    c->block = cfg->block_size > 0 ? cfg->block_size : 256;
    c->nbr_cap = cfg->nlist_capacity > 0 ? ((cfg->nlist_capacity + 7) & ~7) : 0;
    c->sp_host.assign((size_t)c->n * 4, -1);
    c->sbt_host.assign((size_t)c->n, 0);
    for (int t = 0; t < kMaxTypes * kMaxTypes; ++t) c->eps[t] = 1.0;

    auto bail = [&](snap_status s, const char *what) {
        (void)what;
        snap_destroy(c);
        return s;
    };
    if (cfg->stream) {
        c->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return SNAP_ERR_CUDA;
        }
        c->own_stream = true;
    }
    const size_t n = (size_t)std::max<int64_t>(c->n, 1);
    const size_t v4 = c->fp64 ? sizeof(double4_32a) : sizeof(float4);
    for (DevArrays *D : {&c->A, &c->B}) {
        bool ok = alloc_arr(c, D->x, n) && alloc_arr(c, D->y, n) && alloc_arr(c, D->z, n) &&
                  alloc_arr(c, D->vx, n) && alloc_arr(c, D->vy, n) && alloc_arr(c, D->vz, n) &&
                  alloc_arr(c, D->ix, n) && alloc_arr(c, D->iy, n) && alloc_arr(c, D->iz, n) &&
                  alloc_arr(c, D->type, n) && alloc_arr(c, D->tag, n) && alloc_arr(c, D->rep, n) &&
                  alloc_arr(c, D->sp, n) && alloc_arr(c, D->sbt, n) && alloc_arr(c, D->dp, n) &&
                  alloc_arr(c, D->drx, n) && alloc_arr(c, D->dbirth, n) && alloc_arr(c, D->occ, n);
        D->pos4 = dalloc(c, v4 * n);
        if (D == &c->A) D->pos4n = dalloc(c, v4 * n);
        if (!ok || !D->pos4 || (D == &c->A && !D->pos4n)) return bail(SNAP_ERR_OOM, "particles");
        if (!c->fp64 && !alloc_arr(c, D->v4, n)) return bail(SNAP_ERR_OOM, "velocities");
    }
    DevArrays &A = c->A;
    A.force = dalloc(c, v4 * n);
    bool ok = A.force && alloc_arr(c, A.rtag, n) && alloc_arr(c, A.ref4, n) && alloc_arr(c, A.npos, n) && alloc_arr(c, A.nn, n) && alloc_arr(c, A.rnn, n) && alloc_arr(c, A.avail, n) && alloc_arr(c, A.avail_count, kMaxTypes) &&
              alloc_arr(c, A.avail_list, (size_t)kMaxTypes * n) &&
              alloc_arr(c, A.pkey, n) &&
              alloc_arr(c, A.pdist, (n / 5 + 1) * kPushSlots) &&
              alloc_arr(c, A.cell_key, n) && alloc_arr(c, A.order, n) && alloc_arr(c, A.prop, n) &&
              alloc_arr(c, A.prop_d, n) && alloc_arr(c, A.prio, n) && alloc_arr(c, A.best, n) &&
              alloc_arr(c, A.fpart, n) && alloc_arr(c, A.brk, n) && alloc_arr(c, A.rx_order, (size_t)nrep * kMaxRx) &&
              alloc_arr(c, A.step, 1) && alloc_arr(c, A.status, 1) && alloc_arr(c, A.need_rebuild, 1) && alloc_arr(c, A.list_fresh, 1) &&
              alloc_arr(c, A.gathered, 1) &&
              alloc_arr(c, A.nbr_need, 2) && alloc_arr(c, A.counters, (size_t)cNumCounters * kCopies) &&
              alloc_arr(c, A.site_list, n) && alloc_arr(c, A.list_count, 1) &&
              alloc_arr(c, A.cont, n * kContenders) && alloc_arr(c, A.ncont, n) &&
              alloc_arr(c, A.life_hist, (size_t)c->cfg.lifetime_bins) && alloc_arr(c, A.e_part, 4 * n) &&
              alloc_arr(c, A.ksum, (size_t)nrep) && alloc_arr(c, c->d_red, 8);
    c->d_reps = static_cast<RepDev *>(dalloc(c, sizeof(RepDev) * nrep));
    if (!ok || !c->d_reps) return bail(SNAP_ERR_OOM, "work arrays");
    A.reps = c->d_reps;
    // B shares the non-permuted arrays with A
    DevArrays &B = c->B;
    B.rtag = A.rtag; B.ref4 = A.ref4; B.npos = A.npos; B.force = A.force; B.status = A.status; B.need_rebuild = A.need_rebuild;
    B.step = A.step; B.reps = A.reps; B.order = A.order; B.ksum = A.ksum; B.gathered = A.gathered;
    if (cudaMemsetAsync(A.status, 0, 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.step, 0, 8, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.need_rebuild, 0, 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.list_fresh, 0, 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.gathered, 0, 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.nbr_need, 0, 8, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.counters, 0, sizeof(unsigned long long) * cNumCounters * kCopies, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.list_count, 0, 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.avail_count, 0, sizeof(int32_t) * kMaxTypes, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.pkey, 0xFF, sizeof(ulonglong2) * n, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.prop, 0xFF, sizeof(int32_t) * n, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.fpart, 0xFF, sizeof(int32_t) * n, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.brk, 0, sizeof(uint32_t) * n, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.best, 0, sizeof(unsigned long long) * n, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.life_hist, 0, sizeof(unsigned long long) * c->cfg.lifetime_bins, c->stream) != cudaSuccess ||
        cudaMemsetAsync(A.ksum, 0, sizeof(unsigned long long) * nrep, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(SNAP_ERR_CUDA, "init memset");
    }
    *out = c;
    return SNAP_OK;
}

extern "C" snap_status snap_set_types(snap_ctx *c, int32_t ntypes, const double *sigma, const double *eps_pair,
                                      const double *rcut)
{
    if (!c) return SNAP_ERR_ARG;
    if (ntypes < 1 || ntypes > kMaxTypes || !sigma || !eps_pair) return fail(c, SNAP_ERR_ARG, "bad types");
    for (int a = 0; a < ntypes; ++a) {
        if (!(sigma[a] > 0.0)) return fail(c, SNAP_ERR_ARG, "sigma must be > 0");
        for (int b = 0; b < ntypes; ++b) {
            if (!(eps_pair[a * ntypes + b] >= 0.0) || eps_pair[a * ntypes + b] != eps_pair[b * ntypes + a])
                return fail(c, SNAP_ERR_ARG, "eps_pair must be symmetric and >= 0");
            if (rcut && (rcut[a * ntypes + b] != rcut[b * ntypes + a]))
                return fail(c, SNAP_ERR_ARG, "rcut must be symmetric");
        }
    }
    c->ntypes = ntypes;
    for (int a = 0; a < ntypes; ++a) {
        c->sigma[a] = sigma[a];
        for (int b = 0; b < ntypes; ++b) {
            c->eps[a * kMaxTypes + b] = eps_pair[a * ntypes + b];
            c->rcut[a * kMaxTypes + b] = rcut ? rcut[a * ntypes + b] : 0.0;
        }
    }
    c->types_set = true;
    if (c->ready) return fail(c, SNAP_ERR_STATE, "types cannot change after the first step");
    return SNAP_OK;
}

extern "C" snap_status snap_set_valence(snap_ctx *c, const int32_t *valence)
{
    if (!c || !valence) return SNAP_ERR_ARG;
    if (!c->types_set) return fail(c, SNAP_ERR_STATE, "call snap_set_types first");
    for (int a = 0; a < c->ntypes; ++a)
        if (valence[a] < 0 || valence[a] > kVmax) return fail(c, SNAP_ERR_ARG, "valence out of range");
    for (int a = 0; a < c->ntypes; ++a) c->valence[a] = valence[a];
    if (c->ready) {
        fill_params(c);
        c->graph_dirty = true;
    }
    return SNAP_OK;
}

extern "C" snap_status snap_set_bond_params_ex(snap_ctx *c, int32_t bt, int32_t kind, const double *params,
                                               int32_t nparams)
{
    if (!c) return SNAP_ERR_ARG;
    if (bt < 0 || bt >= kMaxBondTypes) return fail(c, SNAP_ERR_ARG, "bond type out of range");
    const int need = (kind == SNAP_HARMONIC || kind == SNAP_FENE) ? 2 : (kind == SNAP_FENEWCA || kind == SNAP_TETHER) ? 5 : -1;
    if (need < 0) return fail(c, SNAP_ERR_ARG, "unknown bond kind");
    if (!params || nparams != need) return fail(c, SNAP_ERR_ARG, "wrong number of bond parameters for this kind");
    for (int q = 0; q < need; ++q)
        if (!std::isfinite(params[q])) return fail(c, SNAP_ERR_ARG, "bond parameters must be finite");
    const double k = params[0], r0 = params[1];
    if (!(k >= 0.0) || !(r0 > 0.0)) return fail(c, SNAP_ERR_ARG, "bond parameters need k >= 0 and a length > 0");
    double x[3] = {0.0, 0.0, 0.0};
    if (kind == SNAP_FENEWCA) {
        x[0] = params[2]; x[1] = params[3]; x[2] = params[4];
        if (!(x[0] >= 0.0) || !(x[1] > 0.0) || !(x[2] >= 0.0))
            return fail(c, SNAP_ERR_ARG, "FENEWCA needs eps >= 0, sigma > 0, delta >= 0");
    } else if (kind == SNAP_TETHER) {
        x[0] = params[2]; x[1] = params[3]; x[2] = params[4];
        if (!(r0 < x[0] && x[0] < x[1] && x[1] < x[2]))
            return fail(c, SNAP_ERR_ARG, "Tether needs l_min < l_c1 < l_c0 < l_max");
    }
    for (const auto &r : c->rx)
        if (r.bt == bt && kind != SNAP_HARMONIC && (r.slip_a != 0.0 || c->mh_mode != 0))
            return fail(c, SNAP_ERR_ARG, "the slip bond and Metropolis-Hastings moves need a harmonic bond type");
    c->bkind[bt] = kind;
    c->bk[bt] = k;
    c->br0[bt] = r0;
    for (int q = 0; q < 3; ++q) c->bx[bt][q] = x[q];
    c->bset[bt] = true;
    if (c->ready) {
        fill_params(c);
        c->graph_dirty = true;
    }
    return SNAP_OK;
}

extern "C" snap_status snap_set_bond_params(snap_ctx *c, int32_t bt, int32_t kind, double k, double r0)
{
    if (c && kind != SNAP_HARMONIC && kind != SNAP_FENE)
        return fail(c, SNAP_ERR_ARG, "FENEWCA and Tether take their parameters through snap_set_bond_params_ex");
    const double p[2] = {k, r0};
    return snap_set_bond_params_ex(c, bt, kind, p, 2);
}

extern "C" snap_status snap_add_static_bonds(snap_ctx *c, int64_t nb, const int32_t *pairs, int32_t bt)
{
    if (!c) return SNAP_ERR_ARG;
    if (nb < 0 || (nb > 0 && !pairs)) return fail(c, SNAP_ERR_ARG, "bad bond list");
    if (bt < 0 || bt >= kMaxBondTypes || !c->bset[bt]) return fail(c, SNAP_ERR_ARG, "bond type not set");
    std::vector<int32_t> sp = c->sp_host, sbt = c->sbt_host;
    for (int64_t q = 0; q < nb; ++q) {
        const int32_t a = pairs[2 * q], b = pairs[2 * q + 1];
        if (a < 0 || b < 0 || a >= c->n || b >= c->n || a == b) return fail(c, SNAP_ERR_ARG, "bond tag out of range");
        if (rep_of_tag(c, a) != rep_of_tag(c, b)) return fail(c, SNAP_ERR_ARG, "bond across replicas");
        for (int32_t u : {a, b}) {
            const int32_t v = (u == a) ? b : a;
            int s = 0;
            while (s < kSmax && sp[4 * (size_t)u + s] >= 0) ++s;
            if (s == kSmax) return fail(c, SNAP_ERR_ARG, "more than SNAP_MAX_STATIC static bonds on a particle");
            sp[4 * (size_t)u + s] = v;
            sbt[u] |= (bt & 0xFF) << (8 * s);
        }
    }
    c->sp_host.swap(sp);
    c->sbt_host.swap(sbt);
    c->n_static += nb;
    c->P.has_static = c->n_static > 0 ? 1 : 0;
    c->graph_dirty = true;
    if (c->ready) {
        snap_status s = upload_molecules(c);
        if (s != SNAP_OK) return s;
    }
    if (c->particles_set) return upload_static(c);
    return SNAP_OK;
}

extern "C" snap_status snap_add_reaction(snap_ctx *c, int32_t ta, int32_t tb, int32_t bt, double rmin, double rmax,
                                         double pon, double poff, int32_t self_avoid, int32_t *index_out)
{
    if (!c) return SNAP_ERR_ARG;
    if (!c->types_set) return fail(c, SNAP_ERR_STATE, "call snap_set_types first");
    if (c->ready) return fail(c, SNAP_ERR_STATE, "reactions must be registered before the first step");
    if ((int)c->rx.size() >= kMaxRx) return fail(c, SNAP_ERR_ARG, "too many reactions");
    if (ta < 0 || tb < 0 || ta >= c->ntypes || tb >= c->ntypes) return fail(c, SNAP_ERR_ARG, "reaction type out of range");
    if (bt < 0 || bt >= kMaxBondTypes || !c->bset[bt])
        return fail(c, SNAP_ERR_ARG, "reaction bond type must be a bond type that has been set");
    if (!(rmin >= 0.0) || !(rmax > rmin) || !std::isfinite(rmax)) return fail(c, SNAP_ERR_ARG, "bad formation window");
    if (!(pon >= 0.0 && pon <= 1.0) || !(poff >= 0.0 && poff <= 1.0))
        return fail(c, SNAP_ERR_ARG, "per-sweep probabilities must lie in [0, 1] (Eq. 2)");
    if (self_avoid != 0 && self_avoid != 1) return fail(c, SNAP_ERR_ARG, "self_avoid must be 0 or 1");
    c->rx.push_back(RxHost{ta, tb, bt, rmin, rmax, pon, poff, self_avoid});
    c->rep_pon.push_back(std::vector<double>(c->reps.size(), pon));
    c->rep_poff.push_back(std::vector<double>(c->reps.size(), poff));
    if (index_out) *index_out = (int32_t)c->rx.size() - 1;
    return SNAP_OK;
}

extern "C" snap_status snap_set_slip(snap_ctx *c, int32_t a, double slip_a)
{
    if (!c) return SNAP_ERR_ARG;
    if (a < 0 || a >= (int)c->rx.size()) return fail(c, SNAP_ERR_ARG, "reaction out of range");
    if (!(slip_a >= 0.0) || !std::isfinite(slip_a)) return fail(c, SNAP_ERR_ARG, "slip parameter must be finite and >= 0");
    if (slip_a != 0.0 && c->rx[a].melting)
        return fail(c, SNAP_ERR_ARG, "the slip bond and the melting switch are mutually exclusive");
    if (slip_a != 0.0 && c->bkind[c->rx[a].bt] != SNAP_HARMONIC)
        return fail(c, SNAP_ERR_ARG, "the slip bond needs a harmonic bond type");
    if (slip_a != 0.0 && c->mh_mode != 0)
        return fail(c, SNAP_ERR_STATE, "Metropolis-Hastings mode does not support the slip bond");
    c->rx[a].slip_a = slip_a;
    c->P.rx_slip[a] = slip_a;
    if (slip_a != 0.0) c->P.slip_mask |= 1 << a;
    else c->P.slip_mask &= ~(1 << a);
    c->graph_dirty = true;
    return SNAP_OK;
}

// Eqs. (gT)-(kT) at each replica's set-point temperature, then Eq. (2).
extern "C" snap_status snap_set_melting(snap_ctx *c, int32_t a, double lambda, double t_melt, double kon_init,
                                        double koff_init, double kon_melt, double koff_melt)
{
    if (!c) return SNAP_ERR_ARG;
    if (a < 0 || a >= (int)c->rx.size()) return fail(c, SNAP_ERR_ARG, "reaction out of range");
    if (c->rx[a].slip_a != 0.0)
        return fail(c, SNAP_ERR_ARG, "the slip bond and the melting switch are mutually exclusive");
    const double v[6] = {lambda, t_melt, kon_init, koff_init, kon_melt, koff_melt};
    for (double x : v)
        if (!std::isfinite(x)) return fail(c, SNAP_ERR_ARG, "melting parameters must be finite");
    if (kon_init < 0.0 || koff_init < 0.0 || kon_melt < 0.0 || koff_melt < 0.0)
        return fail(c, SNAP_ERR_ARG, "rate constants must be >= 0");
    const double ndt = (double)c->cfg.bond_period;
    std::vector<double> pon(c->reps.size()), poff(c->reps.size());
    for (size_t r = 0; r < c->reps.size(); ++r) {
        const double g = 0.5 * (std::tanh(lambda * (c->reps[r].kT - t_melt)) + 1.0);
        const double kon = kon_init * (1.0 - g) + kon_melt * g;
        const double koff = koff_init * (1.0 - g) + koff_melt * g;
        pon[r] = kon * ndt * c->cfg.dt;
        poff[r] = koff * ndt * c->cfg.dt;
        if (!(pon[r] <= 1.0 && poff[r] <= 1.0))
            return fail(c, SNAP_ERR_ARG, "a rate times n dt exceeds 1 (Eq. 2): lower the rates or the bond period");
    }
    for (size_t r = 0; r < c->reps.size(); ++r) {
        c->rep_pon[a][r] = pon[r];
        c->rep_poff[a][r] = poff[r];
    }
    c->rx[a].pon = pon[0];
    c->rx[a].poff = poff[0];
    c->rx[a].melting = true;
    for (int k = 0; k < 6; ++k) c->rx[a].melt[k] = v[k];
    if (c->ready) {
        fill_params(c);       // the switch's parameters, for the kinetic temperature
        c->graph_dirty = true;
        return upload_reps(c);
    }
    return SNAP_OK;
}

extern "C" snap_status snap_set_reaction_rates(snap_ctx *c, int32_t a, int32_t r, double pon, double poff)
{
    if (!c) return SNAP_ERR_ARG;
    if (a < 0 || a >= (int)c->rx.size() || r < 0 || r >= (int)c->reps.size())
        return fail(c, SNAP_ERR_ARG, "reaction or replica out of range");
    if (!(pon >= 0.0 && pon <= 1.0) || !(poff >= 0.0 && poff <= 1.0))
        return fail(c, SNAP_ERR_ARG, "per-sweep probabilities must lie in [0, 1] (Eq. 2)");
    c->rep_pon[a][r] = pon;
    c->rep_poff[a][r] = poff;
    if (c->ready) return upload_reps(c);
    return SNAP_OK;
}

extern "C" snap_status snap_set_particles(snap_ctx *c, const double *pos3, const double *vel3, const int32_t *type)
{
    if (!c) return SNAP_ERR_ARG;
    if (c->n > 0 && (!pos3 || !type)) return fail(c, SNAP_ERR_ARG, "positions and types are required");
    snap_status s = ensure_ready(c);
    if (s != SNAP_OK) return s;
    for (int64_t t = 0; t < c->n; ++t)
        if (type[t] < 0 || type[t] >= c->ntypes) return fail(c, SNAP_ERR_ARG, "particle type out of range");
    const Launch L = launch(c);
    launch_iota(c->A.tag, c->n, L);
    launch_iota(c->A.rtag, c->n, L);
    CUDA_TRY(c, cudaGetLastError());
    std::vector<int32_t> img((size_t)c->n * 3, 0), rep(c->n);
    for (int64_t t = 0; t < c->n; ++t) rep[t] = rep_of_tag(c, t);
    if ((s = positions_in(c, pos3, &img)) != SNAP_OK) return s;
    if ((s = velocities_in(c, vel3)) != SNAP_OK) return s;
    std::vector<int32_t> ic[3];
    for (int d = 0; d < 3; ++d) {
        ic[d].resize(c->n);
        for (int64_t t = 0; t < c->n; ++t) ic[d][t] = img[3 * t + d];
    }
    int32_t *idst[3] = {c->A.ix, c->A.iy, c->A.iz};
    int32_t *istg[3] = {c->B.ix, c->B.iy, c->B.iz};
    for (int d = 0; d < 3; ++d)
        if ((s = upload_in<int32_t>(c, idst[d], istg[d], ic[d].data(), c->n)) != SNAP_OK) return s;
    if ((s = upload_in<int32_t>(c, c->A.type, c->B.type, type, c->n)) != SNAP_OK) return s;
    if ((s = upload_in<int32_t>(c, c->A.rep, c->B.rep, rep.data(), c->n)) != SNAP_OK) return s;
    if ((s = upload_static(c)) != SNAP_OK) return s;
    if ((s = bonds_in(c, {})) != SNAP_OK) return s;
    c->bonds_base = 0;
    CUDA_TRY(c, cudaMemsetAsync(c->A.step, 0, 8, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->A.status, 0, 4, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->A.counters, 0, sizeof(unsigned long long) * cNumCounters * kCopies, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->A.life_hist, 0, sizeof(unsigned long long) * c->cfg.lifetime_bins, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->A.force, 0, (c->fp64 ? sizeof(double4_32a) : sizeof(float4)) * c->n, c->stream));
    c->particles_set = true;
    return set_need_rebuild(c);
}

// device staging for the host I/O calls (allocated on first use)
snap_status ensure_io(snap_ctx *c)
{
    if (c->io3) return SNAP_OK;
    const size_t n = (size_t)std::max<int64_t>(c->n, 1);
    if (!alloc_arr(c, c->io3, 3 * n) || !alloc_arr(c, c->io_img, 3 * n) || !alloc_arr(c, c->io_flag, 1))
        return fail(c, SNAP_ERR_OOM, "I/O staging");
    return SNAP_OK;
}

// One copy of the tag-ordered triples in each direction; the reordering,
// wrapping and image bookkeeping run on the device (io.cu).
extern "C" snap_status snap_set_positions(snap_ctx *c, const double *pos3, const double *vel3)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (c->n > 0 && !pos3) return fail(c, SNAP_ERR_ARG, "positions are required");
    if (c->n == 0) return SNAP_OK;
    if ((s = ensure_io(c)) != SNAP_OK) return s;
    const Launch L = launch(c);
    const size_t bytes = sizeof(double) * 3 * (size_t)c->n;
    CUDA_TRY(c, cudaMemcpyAsync(c->io3, pos3, bytes, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->io_flag, 0, sizeof(uint32_t), c->stream));
    launch_nonfinite(c->io3, 3 * c->n, c->io_flag, L);
    uint32_t bad = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&bad, c->io_flag, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (bad) return fail(c, SNAP_ERR_NONFINITE, "non-finite input position");
    launch_pos_in(c->io3, c->P, c->A, L);
    if (vel3) {
        CUDA_TRY(c, cudaMemcpyAsync(c->io3, vel3, bytes, cudaMemcpyHostToDevice, c->stream));
        launch_vel_in(c->io3, c->A, c->fp64, c->n, L);
    }
    CUDA_TRY(c, cudaGetLastError());
    return set_need_rebuild(c);
}

extern "C" snap_status snap_set_bonds(snap_ctx *c, int64_t nb, const int32_t *pairs, const int32_t *reaction)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (nb < 0 || (nb > 0 && !pairs)) return fail(c, SNAP_ERR_ARG, "bad bond list");
    long long step = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&step, c->A.step, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::vector<BondRec> bonds;
    bonds.reserve(nb);
    for (int64_t q = 0; q < nb; ++q) {
        int32_t a = pairs[2 * q], b = pairs[2 * q + 1];
        const int32_t r = reaction ? reaction[q] : 0;
        if (a < 0 || b < 0 || a >= c->n || b >= c->n || a == b) return fail(c, SNAP_ERR_ARG, "bond tag out of range");
        if (r < 0 || r >= (int)c->rx.size()) return fail(c, SNAP_ERR_ARG, "bond reaction out of range");
        if (rep_of_tag(c, a) != rep_of_tag(c, b)) return fail(c, SNAP_ERR_ARG, "bond across replicas");
        if (a > b) std::swap(a, b);
        bonds.push_back(BondRec{a, b, r, (int32_t)(uint32_t)step});
    }
    if ((s = bonds_in(c, bonds)) != SNAP_OK) return s;
    unsigned long long h[cNumCounters];
    if ((s = counters_out(c, h)) != SNAP_OK) return s;
    c->bonds_base = nb - (int64_t)h[cFormedTotal] + (int64_t)h[cBrokenTotal];
    return SNAP_OK;
}

extern "C" snap_status snap_step(snap_ctx *c, int64_t nsteps)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (nsteps < 0) return fail(c, SNAP_ERR_ARG, "nsteps < 0");
    long long step0 = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&step0, c->A.step, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const long long target = step0 + nsteps;
    long long cur = step0;
    int retries = 0;
    while (cur < target) {
        long long todo = std::min<long long>(target - cur, kPollSteps);
        long long ngraph = graph_mode() == 2 ? 0 : todo / kGraphSteps;
        int gk = 0;
        if (ngraph > 0 && (s = graph_for_parity(c, gk)) != SNAP_OK) return s;
        for (long long g = 0; g < ngraph; ++g) CUDA_TRY(c, cudaGraphLaunch(c->graph[gk], c->stream));
        for (long long r = ngraph * kGraphSteps; r < todo; ++r) seq_step(c);
        CUDA_TRY(c, cudaGetLastError());
        uint32_t st = 0;
        if ((s = read_status(c, st)) != SNAP_OK) return s;
        CUDA_TRY(c, cudaMemcpyAsync(&cur, c->A.step, 8, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (st == kStOverflow) {
            if (++retries > 16) return fail(c, SNAP_ERR_NLIST_OVERFLOW, "neighbour list kept overflowing");
            if ((s = grow_nlist(c)) != SNAP_OK) return s;
            continue;
        }
        if (st) {
            // the step stopped part-way: regenerate the relative coordinates
            // from the FP64 positions at the next step
            recover_status(c);
            const snap_status code = status_to_code(c, st);
            set_need_rebuild(c);
            return code;
        }
    }
    return SNAP_OK;
}

extern "C" snap_status snap_set_kinetic_temperature(snap_ctx *c, int32_t on)
{
    if (!c) return SNAP_ERR_ARG;
    if (on != 0 && on != 1) return fail(c, SNAP_ERR_ARG, "on must be 0 or 1");
    if (on && c->mh_mode) return fail(c, SNAP_ERR_STATE, "Metropolis-Hastings mode uses the set-point temperature");
    c->kinetic_T = on;
    c->graph_dirty = true;
    if (c->ready) {
        fill_params(c);
        return upload_reps(c);   // set-point rates back in place (the kinetic sweeps overwrite melting rates)
    }
    return SNAP_OK;
}

extern "C" snap_status snap_set_retry_limit(snap_ctx *c, int32_t limit)
{
    if (!c) return SNAP_ERR_ARG;
    if (limit < 0) return fail(c, SNAP_ERR_ARG, "retry limit < 0");
    c->cas_cap = limit;
    c->P.cas_cap = limit;     // kernel parameters are captured by value: recapture the graphs
    c->graph_dirty = true;
    return SNAP_OK;
}

extern "C" snap_status snap_set_list_block(snap_ctx *c, int32_t threads)
{
    if (!c) return SNAP_ERR_ARG;
    if (threads != 64 && threads != 128 && threads != 256)
        return fail(c, SNAP_ERR_ARG, "list-build block size must be 64, 128 or 256");
    c->list_block = threads;
    c->graph_dirty = true;    // the launch shape is captured in the step graphs
    return SNAP_OK;
}

extern "C" snap_status snap_set_list_subcells(snap_ctx *c, int32_t k)
{
    if (!c) return SNAP_ERR_ARG;
    if (k != 0 && k != 1 && k != 2 && k != 4 && k != 8)
        return fail(c, SNAP_ERR_ARG, "sub-cells per cell must be 0 (automatic), 1, 2, 4 or 8");
    if (c->ready) return fail(c, SNAP_ERR_STATE, "the cell grid is laid out: set the sub-cells before snap_set_particles");
    c->list_sub = k;
    return SNAP_OK;
}

extern "C" snap_status snap_get_list_subcells(snap_ctx *c, int32_t *k)
{
    if (!c || !k) return SNAP_ERR_ARG;
    if (!c->ready) return fail(c, SNAP_ERR_STATE, "the cell grid is laid out by snap_set_particles");
    *k = 1 << c->sub_shift;
    return SNAP_OK;
}

extern "C" snap_status snap_prepare(snap_ctx *c)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (graph_mode() == 2) return SNAP_OK;
    for (int parity = 0; parity < 2; ++parity) {
        int k = 0;
        s = graph_for_parity(c, k);
        if (s == SNAP_OK && cudaGraphUpload(c->graph[k], c->stream) != cudaSuccess) {
            cudaGetLastError();
            s = fail(c, SNAP_ERR_CUDA, "cudaGraphUpload failed");
        }
        std::swap(c->A.pos4, c->A.pos4n);   // the other parity; two swaps restore the buffers
        if (s != SNAP_OK) {
            if (parity == 0) std::swap(c->A.pos4, c->A.pos4n);
            return s;
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

extern "C" snap_status snap_step_profiled(snap_ctx *c, int64_t nsteps, double *ms)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (nsteps < 0 || !ms) return fail(c, SNAP_ERR_ARG, "bad arguments");
    for (int k = 0; k < SNAP_NPHASES; ++k) ms[k] = 0.0;
    if (nsteps == 0) return SNAP_OK;
    std::vector<cudaEvent_t> ev((size_t)nsteps * (SNAP_NPHASES + 1));
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            for (auto &x : ev)
                if (x) cudaEventDestroy(x);
            return fail(c, SNAP_ERR_CUDA, "event create");
        }
    const Launch L = launch(c);
    for (int64_t t = 0; t < nsteps; ++t) {
        cudaEvent_t *e = &ev[(size_t)t * (SNAP_NPHASES + 1)];
        cudaEventRecord(e[0], c->stream);
        seq_rebuild(c);
        cudaEventRecord(e[1], c->stream);
        seq_sweep(c, false);
        cudaEventRecord(e[2], c->stream);
        seq_md(c, L);
        cudaEventRecord(e[3], c->stream);
        launch_step_end(c->A, L);
        cudaEventRecord(e[4], c->stream);
    }
    cudaError_t err = cudaStreamSynchronize(c->stream);
    for (int64_t t = 0; t < nsteps && err == cudaSuccess; ++t)
        for (int k = 0; k < SNAP_NPHASES; ++k) {
            float x = 0.f;
            err = cudaEventElapsedTime(&x, ev[(size_t)t * (SNAP_NPHASES + 1) + k],
                                       ev[(size_t)t * (SNAP_NPHASES + 1) + k + 1]);
            ms[k] += x;
        }
    for (auto &e : ev) cudaEventDestroy(e);
    if (err != cudaSuccess) return fail(c, SNAP_ERR_CUDA, cudaGetErrorString(err));
    for (int k = 0; k < SNAP_NPHASES; ++k) ms[k] /= (double)nsteps;
    uint32_t st = 0;
    if ((s = read_status(c, st)) != SNAP_OK) return s;
    if (st) {
        clear_status(c);
        return status_to_code(c, st);
    }
    return SNAP_OK;
}

extern "C" snap_status snap_rebuild_profiled(snap_ctx *c, double *ms)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (!ms) return fail(c, SNAP_ERR_ARG, "ms is NULL");
    if ((s = set_need_rebuild(c)) != SNAP_OK) return s;
    cudaEvent_t ev[SNAP_NREBUILD_PHASES + 1] = {};
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            for (auto &x : ev)
                if (x) cudaEventDestroy(x);
            return fail(c, SNAP_ERR_CUDA, "event create");
        }
    const Launch L = launch(c);
    cudaEventRecord(ev[0], c->stream);
    launch_cell_key(c->P, c->A, L);
    cudaEventRecord(ev[1], c->stream);
    launch_cell_scan(c->A, c->d_bsum, c->nkeys, L);
    cudaEventRecord(ev[2], c->stream);
    launch_scatter(c->P, c->A, c->d_bsum, L);
    cudaEventRecord(ev[3], c->stream);
    launch_cell_sort(c->A, c->nkeys, c->d_bsum, L);
    cudaEventRecord(ev[4], c->stream);
    launch_gather(c->P, c->A, c->B, c->fp64, L);
    cudaEventRecord(ev[5], c->stream);
    cudaEventRecord(ev[6], c->stream);             // the copy back runs inside the list build
    launch_nlist(c->P, c->A, c->B, c->fp64, c->list_block, L);
    cudaEventRecord(ev[7], c->stream);
    launch_rebuild_done(c->A, L);
    cudaEventRecord(ev[8], c->stream);
    cudaError_t err = cudaStreamSynchronize(c->stream);
    for (int k = 0; k < SNAP_NREBUILD_PHASES && err == cudaSuccess; ++k) {
        float x = 0.f;
        err = cudaEventElapsedTime(&x, ev[k], ev[k + 1]);
        ms[k] = x;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (err != cudaSuccess) return fail(c, SNAP_ERR_CUDA, cudaGetErrorString(err));
    uint32_t st = 0;
    if ((s = read_status(c, st)) != SNAP_OK) return s;
    if (st == kStOverflow) {
        if ((s = grow_nlist(c)) != SNAP_OK) return s;
        return snap_rebuild_profiled(c, ms);
    }
    if (st) {
        clear_status(c);
        return status_to_code(c, st);
    }
    return SNAP_OK;
}

extern "C" snap_status snap_bond_update(snap_ctx *c)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    return run_with_retry(c, [&] {
        seq_rebuild(c);
        seq_sweep(c, true);
    });
}

extern "C" snap_status snap_get_forces(snap_ctx *c, double *f3)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (c->n > 0 && !f3) return fail(c, SNAP_ERR_ARG, "f3 is NULL");
    s = run_with_retry(c, [&] {
        seq_rebuild(c);
        launch_force(c->P, c->A, c->fp64, false, launch(c));
    });
    if (s != SNAP_OK) return s;
    double *tmp = static_cast<double *>(dalloc(c, sizeof(double) * 3 * std::max<int64_t>(c->n, 1)));
    if (!tmp) return fail(c, SNAP_ERR_OOM, "force staging");
    launch_force_out(tmp, c->A.force, c->fp64, c->A.rtag, c->n, launch(c));
    cudaError_t e = cudaMemcpyAsync(f3, tmp, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, tmp);
    if (e != cudaSuccess) return fail(c, SNAP_ERR_CUDA, cudaGetErrorString(e));
    return SNAP_OK;
}

extern "C" snap_status snap_get_bonds(snap_ctx *c, int32_t *pairs, int32_t *reaction, int64_t cap, int64_t *n_out)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    std::vector<BondRec> b;
    if ((s = bonds_out(c, b)) != SNAP_OK) return s;
    if (n_out) *n_out = (int64_t)b.size();
    if ((int64_t)b.size() > cap) return fail(c, SNAP_ERR_ARG, "bond buffer too small");
    if (b.size() > 0 && !pairs) return fail(c, SNAP_ERR_ARG, "tag_pairs is NULL");
    for (size_t q = 0; q < b.size(); ++q) {
        pairs[2 * q] = b[q].a;
        pairs[2 * q + 1] = b[q].b;
        if (reaction) reaction[q] = b[q].rx;
    }
    return SNAP_OK;
}

// raw device positions and images in tag order (positions may lie outside
// the box between rebuilds in mixed mode)
snap_status raw_positions_images(snap_ctx *c, double *pos3, int32_t *img3)
{
    snap_status s;
    std::vector<double> v(c->n);
    std::vector<int32_t> w(c->n);
    const double *src[3] = {c->A.x, c->A.y, c->A.z};
    double *stg[3] = {c->B.x, c->B.y, c->B.z};
    const int32_t *isrc[3] = {c->A.ix, c->A.iy, c->A.iz};
    int32_t *istg[3] = {c->B.ix, c->B.iy, c->B.iz};
    for (int d = 0; d < 3; ++d) {
        if ((s = download_out<double>(c, v.data(), src[d], stg[d], c->n)) != SNAP_OK) return s;
        if ((s = download_out<int32_t>(c, w.data(), isrc[d], istg[d], c->n)) != SNAP_OK) return s;
        for (int64_t t = 0; t < c->n; ++t) {
            pos3[3 * t + d] = v[t];
            img3[3 * t + d] = w[t];
        }
    }
    return SNAP_OK;
}

extern "C" snap_status snap_get_positions(snap_ctx *c, double *pos3)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (c->n > 0 && !pos3) return fail(c, SNAP_ERR_ARG, "pos3 is NULL");
    if (c->n == 0) return SNAP_OK;
    if ((s = ensure_io(c)) != SNAP_OK) return s;
    launch_pos_out(c->io3, nullptr, c->P, c->A, launch(c));
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(pos3, c->io3, sizeof(double) * 3 * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

extern "C" snap_status snap_get_velocities(snap_ctx *c, double *vel3)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (c->n > 0 && !vel3) return fail(c, SNAP_ERR_ARG, "vel3 is NULL");
    if (c->n == 0) return SNAP_OK;
    if ((s = ensure_io(c)) != SNAP_OK) return s;
    launch_vel_out(c->io3, c->A, c->fp64, c->n, launch(c));
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(vel3, c->io3, sizeof(double) * 3 * (size_t)c->n, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

extern "C" snap_status snap_get_images(snap_ctx *c, int32_t *img3)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (c->n > 0 && !img3) return fail(c, SNAP_ERR_ARG, "img3 is NULL");
    if (c->n == 0) return SNAP_OK;
    if ((s = ensure_io(c)) != SNAP_OK) return s;
    launch_pos_out(nullptr, c->io_img, c->P, c->A, launch(c));
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(img3, c->io_img, sizeof(int32_t) * 3 * (size_t)c->n, cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

extern "C" snap_status snap_get_neighbors(snap_ctx *c, int32_t *pairs, int64_t cap, int64_t *n_out)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    s = run_with_retry(c, [&] { seq_rebuild(c); });
    if (s != SNAP_OK) return s;
    // the union of the force and the reactive list
    const int64_t stride = c->P.nbr_stride;
    std::vector<int32_t> tag(c->n);
    CUDA_TRY(c, cudaMemcpyAsync(tag.data(), c->A.tag, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->stream));
    std::vector<std::pair<int32_t, int32_t>> out;
    const int32_t *lists[2] = {c->A.nbr, c->A.rnbr};
    const int32_t *counts[2] = {c->A.nn, c->A.rnn};
    const int caps[2] = {c->nbr_cap, c->rnbr_cap};
    for (int l = 0; l < 2; ++l) {
        std::vector<int32_t> nbr((size_t)stride * caps[l]), nn(c->n);
        CUDA_TRY(c, cudaMemcpyAsync(nbr.data(), lists[l], sizeof(int32_t) * nbr.size(), cudaMemcpyDeviceToHost,
                                    c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(nn.data(), counts[l], sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        for (int64_t i = 0; i < c->n; ++i)
            for (int k = 0; k < nn[i]; ++k) {
                // force-list entries carry the pair's cell shift above the index
                const int32_t a = tag[i], b = tag[(uint32_t)nbr[(size_t)k * stride + i] & kIdxMask];
                if (a < b) out.emplace_back(a, b);
            }
    }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    if (n_out) *n_out = (int64_t)out.size();
    if ((int64_t)out.size() > cap) return fail(c, SNAP_ERR_ARG, "pair buffer too small");
    for (size_t q = 0; q < out.size(); ++q) {
        pairs[2 * q] = out[q].first;
        pairs[2 * q + 1] = out[q].second;
    }
    return SNAP_OK;
}

extern "C" snap_status snap_get_rdf(snap_ctx *c, int32_t replica, int32_t type_a, int32_t type_b, double r_max,
                                    int32_t nbins, int64_t *hist)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (!hist) return fail(c, SNAP_ERR_ARG, "hist is NULL");
    if (replica < 0 || replica >= (int)c->reps.size()) return fail(c, SNAP_ERR_ARG, "replica out of range");
    if (type_a < 0 || type_a >= c->ntypes || type_b < 0 || type_b >= c->ntypes)
        return fail(c, SNAP_ERR_ARG, "type out of range");
    if (nbins < 1 || nbins > (1 << 20)) return fail(c, SNAP_ERR_ARG, "nbins must lie in 1..2^20");
    const RepHost &R = c->reps[replica];
    double wmin = 1e300;
    for (int d = 0; d < 3; ++d) wmin = std::min(wmin, R.L[d] / (double)R.nc[d]);
    if (!(r_max > 0.0) || !(r_max <= wmin - 2e-3))
        return fail(c, SNAP_ERR_ARG, "r_max must lie in (0, cell width - 0.002] (cell width " + std::to_string(wmin) + ")");
    // a forced rebuild files every particle in its current cell
    if ((s = set_need_rebuild(c)) != SNAP_OK) return s;
    s = run_with_retry(c, [&] { seq_rebuild(c); });
    if (s != SNAP_OK) return s;
    unsigned long long *d_hist = static_cast<unsigned long long *>(dalloc(c, sizeof(unsigned long long) * nbins));
    if (!d_hist) return fail(c, SNAP_ERR_OOM, "histogram");
    std::vector<unsigned long long> h(nbins);
    cudaError_t e = cudaMemsetAsync(d_hist, 0, sizeof(unsigned long long) * nbins, c->stream);
    if (e == cudaSuccess) {
        launch_rdf(c->P, c->A, replica, type_a, type_b, r_max, nbins, d_hist, launch(c));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_hist, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, d_hist);
    if (e != cudaSuccess) return fail(c, SNAP_ERR_CUDA, cudaGetErrorString(e));
    for (int b = 0; b < nbins; ++b) hist[b] = (int64_t)h[b];
    return SNAP_OK;
}

extern "C" snap_status snap_get_stats(snap_ctx *c, snap_stats *out)
{
    if (!c || !out) return SNAP_ERR_ARG;
    std::memset(out, 0, sizeof *out);
    if (!c->ready || !c->particles_set) return SNAP_OK;
    unsigned long long h[cNumCounters];
    snap_status s = counters_out(c, h);
    if (s != SNAP_OK) return s;
    long long step = 0;
    uint32_t st = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&step, c->A.step, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(&st, c->A.status, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    out->step = step;
    out->formed_total = (int64_t)h[cFormedTotal];
    out->broken_total = (int64_t)h[cBrokenTotal];
    out->n_bonds = c->bonds_base + out->formed_total - out->broken_total;
    out->sweeps = (int64_t)h[cSweeps];
    out->scanned = (int64_t)h[cNlistScanned];
    out->in_window = (int64_t)h[cInWindow];
    out->proposals = (int64_t)h[cProposals];
    out->edges = (int64_t)h[cEdges];
    out->survivors = (int64_t)h[cSurvivors];
    out->formed = (int64_t)h[cFormed];
    out->break_tested = (int64_t)h[cBreakTested];
    out->broken = (int64_t)h[cBroken];
    out->nlist_builds = (int64_t)h[cBuilds];
    out->nlist_entries = (int64_t)h[cNlistEntries];
    out->mh_form_attempts = (int64_t)h[cMhFormAtt];
    out->mh_form_accepts = (int64_t)h[cMhFormAcc];
    out->mh_break_attempts = (int64_t)h[cMhBreakAtt];
    out->mh_break_accepts = (int64_t)h[cMhBreakAcc];
    out->events_logged = (int64_t)h[cEvents];
    out->rnlist_entries = (int64_t)h[cRnlistEntries];
    out->rebuild_launches = (int64_t)h[cRebuildLaunches];
    out->nlist_capacity = c->nbr_cap;
    out->status = (int32_t)status_to_code(c, st);
    return SNAP_OK;
}

extern "C" snap_status snap_get_energy(snap_ctx *c, snap_energy *out)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (!out) return fail(c, SNAP_ERR_ARG, "out is NULL");
    s = run_with_retry(c, [&] {
        seq_rebuild(c);
        launch_force(c->P, c->A, c->fp64, true, launch(c));
        launch_reduce_cols(c->A.e_part, 4, c->n, c->d_red, launch(c));
    });
    if (s != SNAP_OK) return s;
    double h[4];
    CUDA_TRY(c, cudaMemcpyAsync(h, c->d_red, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    out->e_pair = h[0];
    out->e_bond = h[1];
    out->virial = h[2];
    out->kinetic = h[3];
    return SNAP_OK;
}

extern "C" snap_status snap_get_lifetime_hist(snap_ctx *c, int64_t *bins, int32_t nbins)
{
    if (!c || !bins || nbins <= 0) return SNAP_ERR_ARG;
    std::vector<unsigned long long> h(c->cfg.lifetime_bins);
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), c->A.life_hist, sizeof(unsigned long long) * h.size(),
                                cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < nbins; ++k) bins[k] = 0;
    for (size_t k = 0; k < h.size(); ++k) bins[std::min<size_t>(k, nbins - 1)] += (int64_t)h[k];
    return SNAP_OK;
}

namespace {
constexpr uint64_t kStateMagic = 0x31706e73ull;  // "snp1"
}

extern "C" snap_status snap_get_state(snap_ctx *c, void *buf, size_t *len)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (!len) return fail(c, SNAP_ERR_ARG, "len is NULL");
    std::vector<BondRec> b;
    if ((s = bonds_out(c, b)) != SNAP_OK) return s;
    const size_t n = (size_t)c->n;
    const size_t need = 4 * sizeof(uint64_t) + n * (6 * sizeof(double) + 3 * sizeof(int32_t)) + b.size() * sizeof(BondRec);
    if (!buf) {
        *len = need;
        return SNAP_OK;
    }
    if (*len < need) {
        *len = need;
        return fail(c, SNAP_ERR_ARG, "state buffer too small");
    }
    long long step = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&step, c->A.step, 8, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    char *p = static_cast<char *>(buf);
    const uint64_t hdr[4] = {kStateMagic, (uint64_t)n, (uint64_t)step, (uint64_t)b.size()};
    std::memcpy(p, hdr, sizeof hdr);
    p += sizeof hdr;
    // raw (possibly unwrapped) positions and images, so a restore continues bit-identically
    std::vector<double> v3(3 * n);
    std::vector<int32_t> i3(3 * n);
    if ((s = raw_positions_images(c, v3.data(), i3.data())) != SNAP_OK) return s;
    std::memcpy(p, v3.data(), sizeof(double) * 3 * n);
    p += sizeof(double) * 3 * n;
    if ((s = snap_get_velocities(c, v3.data())) != SNAP_OK) return s;
    std::memcpy(p, v3.data(), sizeof(double) * 3 * n);
    p += sizeof(double) * 3 * n;
    std::memcpy(p, i3.data(), sizeof(int32_t) * 3 * n);
    p += sizeof(int32_t) * 3 * n;
    if (!b.empty()) std::memcpy(p, b.data(), sizeof(BondRec) * b.size());
    *len = need;
    // A restore rebuilds the cell list before its first step; rebuild here too,
    // so that the saved run and every run restored from this state continue
    // with the same cell origins and memory order, bit for bit.
    return set_need_rebuild(c);
}

extern "C" snap_status snap_set_state(snap_ctx *c, const void *buf, size_t len)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (!buf || len < 4 * sizeof(uint64_t)) return fail(c, SNAP_ERR_ARG, "state buffer too small");
    uint64_t hdr[4];
    std::memcpy(hdr, buf, sizeof hdr);
    const size_t n = (size_t)c->n;
    if (hdr[0] != kStateMagic || hdr[1] != (uint64_t)n) return fail(c, SNAP_ERR_ARG, "state does not match this context");
    const size_t need = 4 * sizeof(uint64_t) + n * (6 * sizeof(double) + 3 * sizeof(int32_t)) + hdr[3] * sizeof(BondRec);
    if (len < need) return fail(c, SNAP_ERR_ARG, "state buffer truncated");
    const char *p = static_cast<const char *>(buf) + sizeof hdr;
    std::vector<double> pos(3 * n), vel(3 * n);
    std::memcpy(pos.data(), p, sizeof(double) * 3 * n);
    p += sizeof(double) * 3 * n;
    std::memcpy(vel.data(), p, sizeof(double) * 3 * n);
    p += sizeof(double) * 3 * n;
    std::vector<int32_t> img(3 * n);
    std::memcpy(img.data(), p, sizeof(int32_t) * 3 * n);
    p += sizeof(int32_t) * 3 * n;
    std::vector<BondRec> b(hdr[3]);
    if (!b.empty()) std::memcpy(b.data(), p, sizeof(BondRec) * b.size());
    // positions are already wrapped; upload them verbatim so the run continues bit-identically
    double *dst[3] = {c->A.x, c->A.y, c->A.z};
    double *stg[3] = {c->B.x, c->B.y, c->B.z};
    int32_t *idst[3] = {c->A.ix, c->A.iy, c->A.iz};
    int32_t *istg[3] = {c->B.ix, c->B.iy, c->B.iz};
    std::vector<double> col(n);
    std::vector<int32_t> icol(n);
    for (int d = 0; d < 3; ++d) {
        for (size_t t = 0; t < n; ++t) col[t] = pos[3 * t + d];
        if ((s = upload_in<double>(c, dst[d], stg[d], col.data(), n)) != SNAP_OK) return s;
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        for (size_t t = 0; t < n; ++t) icol[t] = img[3 * t + d];
        if ((s = upload_in<int32_t>(c, idst[d], istg[d], icol.data(), n)) != SNAP_OK) return s;
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    if ((s = velocities_in(c, vel.data())) != SNAP_OK) return s;
    if ((s = bonds_in(c, b)) != SNAP_OK) return s;
    const long long step = (long long)hdr[2];
    CUDA_TRY(c, cudaMemcpyAsync(c->A.step, &step, 8, cudaMemcpyHostToDevice, c->stream));
    unsigned long long h[cNumCounters];
    if ((s = counters_out(c, h)) != SNAP_OK) return s;
    c->bonds_base = (int64_t)b.size() - (int64_t)h[cFormedTotal] + (int64_t)h[cBrokenTotal];
    return set_need_rebuild(c);
}

extern "C" snap_status snap_set_mh(snap_ctx *c, int32_t mode, const snap_mlp *mlp, double eps_u)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (mode < 0 || mode > 2) return fail(c, SNAP_ERR_ARG, "mode must be 0, 1 or 2");
    if (mode == 2 && !mlp) return fail(c, SNAP_ERR_ARG, "the learned proposal needs a network");
    if (!(eps_u > 0.0 && eps_u <= 1.0)) return fail(c, SNAP_ERR_ARG, "eps_u must lie in (0, 1]");
    if (mode != 0) {
        if (c->rx.size() != 1 || c->reps.size() != 1)
            return fail(c, SNAP_ERR_ARG, "Metropolis-Hastings mode supports one reaction in one system");
        if (c->rx[0].self_avoid)
            return fail(c, SNAP_ERR_ARG, "Metropolis-Hastings mode does not support intramolecular exclusion");
        if (c->rx[0].slip_a != 0.0)
            return fail(c, SNAP_ERR_ARG, "Metropolis-Hastings mode does not support the slip bond");
        if (c->bkind[c->rx[0].bt] != SNAP_HARMONIC)
            return fail(c, SNAP_ERR_ARG, "Metropolis-Hastings mode needs a harmonic bond type");
        if (c->kinetic_T)
            return fail(c, SNAP_ERR_STATE, "Metropolis-Hastings mode uses the set-point temperature");
        const double side = 2.0 * c->rx[0].rmax + 0.05;
        int nc[3];
        for (int d = 0; d < 3; ++d) {
            nc[d] = (int)std::floor(c->reps[0].L[d] / side);
            if (nc[d] % 2) nc[d] -= 1;
            if (nc[d] < 2) return fail(c, SNAP_ERR_ARG, "box too small for Metropolis-Hastings cells (2 per axis)");
        }
        const int cells = nc[0] * nc[1] * nc[2];
        if (!c->mh_alloc || cells != c->mh_nc[0] * c->mh_nc[1] * c->mh_nc[2]) {
            DevArrays &A = c->A;
            const size_t n = (size_t)std::max<int64_t>(c->n, 1);
            const size_t moves = (size_t)std::max(cells / 8, 1);
            const int nb = (cells + 4095) / 4096 + 1;
            for (void *p : {(void *)A.mh_key, (void *)A.mh_count, (void *)A.mh_start, (void *)A.mh_cursor,
                            (void *)A.mh_order, (void *)A.mh_bsum, (void *)A.mh_gate, (void *)A.mv_type,
                            (void *)A.mv_i, (void *)A.mv_j, (void *)A.mv_n, (void *)A.mv_b, (void *)A.mv_c,
                            (void *)A.mv_cand, (void *)A.mv_r, (void *)A.mv_feat, (void *)A.mv_logit,
                            (void *)A.mv_row0, (void *)A.mv_rows})
                dfree(c, p);
            bool ok = alloc_arr(c, A.mh_key, n) && alloc_arr(c, A.mh_count, cells) &&
                      alloc_arr(c, A.mh_start, cells + 1) && alloc_arr(c, A.mh_cursor, cells) &&
                      alloc_arr(c, A.mh_order, n) && alloc_arr(c, A.mh_bsum, nb + 1) && alloc_arr(c, A.mh_gate, 1) &&
                      alloc_arr(c, A.mv_type, moves) && alloc_arr(c, A.mv_i, moves) && alloc_arr(c, A.mv_j, moves) &&
                      alloc_arr(c, A.mv_n, moves) && alloc_arr(c, A.mv_b, moves) && alloc_arr(c, A.mv_c, moves) &&
                      alloc_arr(c, A.mv_cand, moves * kMhCand) && alloc_arr(c, A.mv_r, moves * kMhCand) &&
                      alloc_arr(c, A.mv_feat, moves * kMhCand * kMlpFeatures) &&
                      alloc_arr(c, A.mv_logit, moves * kMhCand) && alloc_arr(c, A.mv_row0, moves) &&
                      alloc_arr(c, A.mv_rows, 1);
            if (!ok) return fail(c, SNAP_ERR_OOM, "Metropolis-Hastings arrays");
            const int32_t one = 1;
            CUDA_TRY(c, cudaMemsetAsync(A.mh_count, 0, sizeof(int32_t) * cells, c->stream));
            CUDA_TRY(c, cudaMemsetAsync(A.mh_cursor, 0, sizeof(int32_t) * cells, c->stream));
            CUDA_TRY(c, cudaMemsetAsync(A.mv_feat, 0, sizeof(float) * moves * kMhCand * kMlpFeatures, c->stream));
            CUDA_TRY(c, cudaMemsetAsync(A.mv_rows, 0, sizeof(int32_t), c->stream));
            CUDA_TRY(c, cudaMemsetAsync(A.mv_row0, 0, sizeof(int32_t) * moves, c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(A.mh_gate, &one, sizeof one, cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            c->mh_alloc = true;
        }
        for (int d = 0; d < 3; ++d) c->mh_nc[d] = nc[d];
    }
    c->mh_mode = mode;
    c->mlp = mlp;
    c->mh_eps = eps_u;
    fill_params(c);
    c->graph_dirty = true;
    return upload_reps(c);
}

extern "C" snap_status snap_mh_sweep(snap_ctx *c)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (!c->mh_mode) return fail(c, SNAP_ERR_STATE, "Metropolis-Hastings mode is off (snap_set_mh)");
    return run_with_retry(c, [&] {
        seq_rebuild(c);
        seq_sweep(c, true);
    });
}

extern "C" snap_status snap_set_step(snap_ctx *c, int64_t step)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (step < 0) return fail(c, SNAP_ERR_ARG, "step must be >= 0");
    const long long v = (long long)step;
    CUDA_TRY(c, cudaMemcpyAsync(c->A.step, &v, sizeof v, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNAP_OK;
}

extern "C" snap_status snap_log_events(snap_ctx *c, int64_t capacity)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (capacity < 0 || capacity > (int64_t)INT32_MAX / kMhCand) return fail(c, SNAP_ERR_ARG, "bad capacity");
    DevArrays &A = c->A;
    for (void *p : {(void *)A.ev_feat, (void *)A.ev_n, (void *)A.ev_label, (void *)A.ev_count}) dfree(c, p);
    A.ev_feat = nullptr;
    A.ev_n = A.ev_label = A.ev_count = nullptr;
    A.ev_cap = 0;
    c->ev_cap = 0;
    if (capacity > 0) {
        bool ok = alloc_arr(c, A.ev_feat, (size_t)capacity * kMhCand * kMlpFeatures) &&
                  alloc_arr(c, A.ev_n, capacity) && alloc_arr(c, A.ev_label, capacity) && alloc_arr(c, A.ev_count, 1);
        if (!ok) return fail(c, SNAP_ERR_OOM, "event log");
        CUDA_TRY(c, cudaMemsetAsync(A.ev_count, 0, sizeof(int32_t), c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        A.ev_cap = (int32_t)capacity;
        c->ev_cap = capacity;
    }
    fill_params(c);
    c->graph_dirty = true;
    return SNAP_OK;
}

extern "C" snap_status snap_get_events(snap_ctx *c, float *feat, int32_t *offsets, int32_t *labels, int64_t cap_events,
                                       int64_t cap_rows, int64_t *n_events, int64_t *n_rows, int32_t clear)
{
    snap_status s = check_ready(c);
    if (s != SNAP_OK) return s;
    if (c->ev_cap == 0) return fail(c, SNAP_ERR_STATE, "event logging is off (snap_log_events)");
    int32_t cnt = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&cnt, c->A.ev_count, sizeof cnt, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const long long ne = std::min<long long>(cnt, c->ev_cap);
    std::vector<int32_t> nv(ne), lv(ne);
    std::vector<float> fv((size_t)ne * kMhCand * kMlpFeatures);
    if (ne > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(nv.data(), c->A.ev_n, sizeof(int32_t) * ne, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(lv.data(), c->A.ev_label, sizeof(int32_t) * ne, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(fv.data(), c->A.ev_feat, sizeof(float) * fv.size(), cudaMemcpyDeviceToHost,
                                    c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    long long rows = 0;
    for (long long e = 0; e < ne; ++e) rows += nv[e];
    if (n_events) *n_events = ne;
    if (n_rows) *n_rows = rows;
    if (ne > cap_events || rows > cap_rows) return fail(c, SNAP_ERR_ARG, "event buffers too small");
    if (ne > 0 && (!feat || !offsets || !labels)) return fail(c, SNAP_ERR_ARG, "NULL event buffer");
    long long r = 0;
    if (offsets) offsets[0] = 0;
    for (long long e = 0; e < ne; ++e) {
        std::memcpy(feat + r * kMlpFeatures, fv.data() + (size_t)e * kMhCand * kMlpFeatures,
                    sizeof(float) * kMlpFeatures * nv[e]);
        r += nv[e];
        offsets[e + 1] = (int32_t)r;
        labels[e] = lv[e];
    }
    if (clear) CUDA_TRY(c, cudaMemsetAsync(c->A.ev_count, 0, sizeof(int32_t), c->stream));
    return SNAP_OK;
}

extern "C" snap_status snap_sync(snap_ctx *c)
{
    if (!c) return SNAP_ERR_ARG;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (!c->ready || !c->particles_set) return SNAP_OK;
    uint32_t st = 0;
    snap_status s = read_status(c, st);
    if (s != SNAP_OK) return s;
    if (st) clear_status(c);
    return status_to_code(c, st);
}

extern "C" const char *snap_last_error(const snap_ctx *c)
{
    if (!c) return "null context";
    return c->err.c_str();
}

extern "C" void snap_destroy(snap_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    std::vector<void *> all = c->allocs;
    for (void *p : all) dfree(c, p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->side) cudaStreamDestroy(c->side);
    delete c;
}
