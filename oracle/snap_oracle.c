/*
 * FP64 CPU oracle for dynamic-bonding MD — TEST INFRASTRUCTURE ONLY.
 *
 * Follows "pySNAP + DyBond-v2" (arXiv 2609.21204):
 *   Sec. II.A  two-state reaction, Eq. (1) K = k_on/k_off, eps = ln K
 *   Sec. II.A  per-sweep probabilities, Eq. (2)
 *   Sec. II.B  Metropolis factor on formation only, Eqs. (3)-(4)
 *   Sec. II.C  the bonding sweep (Fig. 1): proposal, matching, acceptance,
 *              breaking; occupancy read as it stood when the reaction began
 *   Sec. II.E  counter-based Philox keyed by seed, step and stream, counted by
 *              the sorted tag pair
 * plus a plain WCA/LJ + FENE/harmonic force field and a Langevin integrator
 * for the MD around the sweep.
 *
 * Readings where the paper is silent (shared with the CUDA path only as a
 * written specification, never as code):
 *   - valence > 1 is an occupancy counter with a per-type capacity; a particle
 *     joins at most one new bond per reaction per sweep and never a second
 *     bond to a partner it is already bonded to;
 *   - the matching phase is a one-round locally dominant matching: every
 *     proposal edge gets the priority word Philox(MATCH; min tag, max tag)[0];
 *     an edge survives iff at both endpoints its key (priority << 32 | other
 *     tag) is the largest among the edges touching that endpoint;
 *   - the proposal keeps the partner minimising |r - r0|, ties to the smaller
 *     tag; the window test is r_min^2 <= r^2 <= r_max^2 in FP64;
 *   - T in Eq. (3) is the set-point kT; at kT = 0 the factor is [U_b <= 0];
 *   - exp() in Eq. (3) is this file's own (Cody–Waite + Taylor), and so is
 *     the log() of a FENE dynamic bond's energy (atanh series), so that the
 *     CUDA path, which implements the same published recipes, decides alike;
 *   - a proposal aims at the minimum of the reaction's bond term: r0 for a
 *     harmonic bond, 0 for FENE;
 *   - Langevin: leapfrog form of velocity Verlet with drag -gamma v_{t-1/2}
 *     and a uniform random force sqrt(2 gamma kT / dt) * sqrt(3) (2u - 1);
 *   - no pair exclusions: WCA acts on bonded pairs too;
 *   - a molecule is a connected component of the static-bond graph (a
 *     particle without static bonds is a molecule of its own); the
 *     self-avoid flag of a reaction removes same-molecule partners from its
 *     candidates, in the proposal phase and in the MH move set alike.
 *
 * Parity unpinned: none of the functions below is left without a test that
 * ties it to the paper or to mathematics (closed forms, brute force,
 * invariants); see tests/test_oracle_*.py.
 */
#include "snap_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox-4x32 with 10 rounds: multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key
 * increments 0x9E3779B9 / 0xBB67AE85 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_u53(uint32_t w0, uint32_t w1)
{
    uint64_t m = ((uint64_t)w0 << 21) | (uint64_t)(w1 >> 11);
    return (double)m * 0x1.0p-53;
}

static void orc_key(const orc_params *P, int32_t rx, int32_t stream, uint32_t key[2])
{
    key[0] = (uint32_t)(P->seed & 0xFFFFFFFFull);
    key[1] = (uint32_t)(((P->seed >> 32) & 0xFFFFull) << 16) |
             ((uint32_t)(rx & 0xFF) << 8) | (uint32_t)(stream & 0xFF);
}

/* Draw for the unordered tag pair (a < b) at a step on one stream of one reaction. */
static void orc_pair_draw(const orc_params *P, int32_t rx, int32_t stream, int64_t step,
                          int64_t a, int64_t b, uint32_t out[4])
{
    uint32_t key[2], ctr[4];
    orc_key(P, rx, stream, key);
    ctr[0] = (uint32_t)((uint64_t)step & 0xFFFFFFFFull);
    ctr[1] = (uint32_t)((uint64_t)step >> 32);
    ctr[2] = (uint32_t)a;
    ctr[3] = (uint32_t)b;
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------ exp */

/* exp(x) = 2^k exp(r), k = rint(x / ln2), r = x - k ln2 reduced in two fma
 * steps with ln2 split into its nearest double and the remainder (Cody and
 * Waite, "Software Manual for the Elementary Functions", 1980); exp(r) by its
 * Taylor series to degree 13 (truncation < 5e-18 for |r| <= ln2/2), Horner
 * form with fused multiply-adds; 2^k applied as two exact powers of two. */
static const double ORC_INV_LN2 = 0x1.71547652b82fep+0;
static const double ORC_LN2_HI = 0x1.62e42fefa39efp-1;
static const double ORC_LN2_LO = 0x1.abc9e3b39803fp-56;

static double orc_pow2i(int n)
{
    uint64_t bits = (uint64_t)(n + 1023) << 52;
    double d;
    memcpy(&d, &bits, sizeof d);
    return d;
}

double orc_exp(double x)
{
    if (x != x) return x;
    if (x > 709.7) return INFINITY;
    if (x < -745.2) return 0.0;
    double k = rint(x * ORC_INV_LN2);
    double r = fma(-k, ORC_LN2_HI, x);
    r = fma(-k, ORC_LN2_LO, r);
    double p = 1.0 / 6227020800.0;            /* 1/13! */
    p = fma(p, r, 1.0 / 479001600.0);         /* 1/12! */
    p = fma(p, r, 1.0 / 39916800.0);          /* 1/11! */
    p = fma(p, r, 1.0 / 3628800.0);           /* 1/10! */
    p = fma(p, r, 1.0 / 362880.0);            /* 1/9!  */
    p = fma(p, r, 1.0 / 40320.0);             /* 1/8!  */
    p = fma(p, r, 1.0 / 5040.0);              /* 1/7!  */
    p = fma(p, r, 1.0 / 720.0);               /* 1/6!  */
    p = fma(p, r, 1.0 / 120.0);               /* 1/5!  */
    p = fma(p, r, 1.0 / 24.0);                /* 1/4!  */
    p = fma(p, r, 1.0 / 6.0);                 /* 1/3!  */
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p = fma(p, r, 1.0);
    int ki = (int)k;
    int k1 = ki / 2;
    int k2 = ki - k1;
    return (p * orc_pow2i(k1)) * orc_pow2i(k2);
}

/* Natural logarithm for the FENE bond energy of Eq. (3), this file's own so
 * that the CUDA path, which follows the same published recipe, decides alike:
 * x = m 2^e with m in [sqrt(1/2), sqrt(2)), s = (m - 1)/(m + 1) and
 * ln m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), the series kept to s^27
 * (|s| <= 0.172, so the next term is below 1e-21 of the result);
 * ln x = e ln2 + ln m with ln2 split in two words.  Positive normal and
 * subnormal x; 0 -> -inf, negative or NaN -> NaN, +inf -> +inf. */
double orc_log(double x)
{
    if (x != x || x < 0.0) return NAN;
    if (x == 0.0) return -INFINITY;
    if (x == INFINITY) return INFINITY;
    int e = 0;
    if (x < 0x1.0p-1022) {                    /* subnormal: scale into the normal range */
        x *= 0x1.0p54;
        e = -54;
    }
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    e += (int)((b >> 52) & 0x7FF) - 1023;
    b = (b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;   /* m in [1, 2) */
    double m;
    memcpy(&m, &b, sizeof m);
    if (m > 0x1.6a09e667f3bcdp+0) {           /* sqrt(2): halve m, exactly */
        m *= 0.5;
        e += 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double q = 1.0 / 27.0;
    q = fma(q, z, 1.0 / 25.0);
    q = fma(q, z, 1.0 / 23.0);
    q = fma(q, z, 1.0 / 21.0);
    q = fma(q, z, 1.0 / 19.0);
    q = fma(q, z, 1.0 / 17.0);
    q = fma(q, z, 1.0 / 15.0);
    q = fma(q, z, 1.0 / 13.0);
    q = fma(q, z, 1.0 / 11.0);
    q = fma(q, z, 1.0 / 9.0);
    q = fma(q, z, 1.0 / 7.0);
    q = fma(q, z, 1.0 / 5.0);
    q = fma(q, z, 1.0 / 3.0);
    double t = 2.0 * s;
    double lm = fma(t, z * q, t);
    double de = (double)e;
    return fma(de, ORC_LN2_HI, fma(de, ORC_LN2_LO, lm));
}

/* ------------------------------------------------------- bond energies */

/* FENEWCA and Tether: the bond potentials HOOMD-blue documents under those
 * names, which Sec. II.B names as evaluators the updater accepts.
 *   FENEWCA (k, R0, eps, sigma, delta), s = r - delta:
 *     U = -k R0^2/2 ln(1 - (s/R0)^2) + [4 eps ((sigma/s)^12 - (sigma/s)^6) + eps] for s < 2^(1/6) sigma
 *   Tether (k_b, l_min, l_c1, l_c0, l_max):
 *     U = k_b e^{1/(l_c0 - r)} / (l_max - r) for r > l_c0 and k_b e^{1/(r - l_c1)} / (r - l_min)
 *     for r < l_c1, 0 in between.
 * U, dU/dr and d2U/dr2 with libm; returns ORC_ERR_FENE outside the finite
 * range (s <= 0 or s >= R0; r <= l_min or r >= l_max). */
static const double ORC_TWO_SIXTH = 0x1.1f59ac3c7d6c0p+0;   /* 2^(1/6) */

static int orc_bond_terms(const orc_params *P, int32_t bt, double r, double *U, double *dU, double *d2U)
{
    double k = P->bk[bt], r0 = P->br0[bt];
    int kind = P->bkind[bt];
    *U = *dU = *d2U = 0.0;
    if (kind == ORC_HARMONIC) {
        *U = 0.5 * k * (r - r0) * (r - r0);
        *dU = k * (r - r0);
        *d2U = k;
        return ORC_OK;
    }
    if (kind == ORC_FENE || kind == ORC_FENEWCA) {
        double s = kind == ORC_FENE ? r : r - P->bx[bt][2];
        double q = (s * s) / (r0 * r0);
        if (q >= 1.0 || (kind == ORC_FENEWCA && s <= 0.0)) return ORC_ERR_FENE;
        *U = -0.5 * k * r0 * r0 * log(1.0 - q);
        *dU = k * s / (1.0 - q);
        *d2U = k * (1.0 + q) / ((1.0 - q) * (1.0 - q));
        if (kind == ORC_FENEWCA) {
            double eps = P->bx[bt][0], sig = P->bx[bt][1];
            if (s < sig * ORC_TWO_SIXTH) {
                double sr6 = pow(sig / s, 6.0), sr12 = sr6 * sr6;
                *U += 4.0 * eps * (sr12 - sr6) + eps;
                *dU -= 24.0 * eps * (2.0 * sr12 - sr6) / s;
                *d2U += 24.0 * eps * (26.0 * sr12 - 7.0 * sr6) / (s * s);
            }
        }
        return ORC_OK;
    }
    /* Tether */
    double lmin = r0, lc1 = P->bx[bt][0], lc0 = P->bx[bt][1], lmax = P->bx[bt][2];
    if (r <= lmin || r >= lmax) return ORC_ERR_FENE;
    if (r > lc0) {
        double a = lc0 - r, b = lmax - r;
        double h = 1.0 / (a * a) + 1.0 / b;
        *U = k * exp(1.0 / a) / b;
        *dU = *U * h;
        *d2U = *dU * h + *U * (2.0 / (a * a * a) + 1.0 / (b * b));
    } else if (r < lc1) {
        double c = r - lc1, e = r - lmin;
        double h = 1.0 / (c * c) + 1.0 / e;
        *U = k * exp(1.0 / c) / e;
        *dU = -*U * h;
        *d2U = -*dU * h + *U * (2.0 / (c * c * c) + 1.0 / (e * e));
    }
    return ORC_OK;
}

double orc_bond_energy(const orc_params *P, int32_t bt, double r)
{
    double U, dU, d2U;
    if (orc_bond_terms(P, bt, r, &U, &dU, &d2U) != ORC_OK) return INFINITY;
    return U;
}

/* U_b of a dynamic bond for Eq. (3): harmonic 1/2 k (r - r0)^2, or FENE
 * -1/2 k R0^2 ln(1 - (r/R0)^2) with this file's logarithm (+inf at r >= R0). */
static double orc_dyn_energy(const orc_params *P, int32_t bt, double r)
{
    double k = P->bk[bt], r0 = P->br0[bt];
    int kind = P->bkind[bt];
    if (kind == ORC_HARMONIC) {
        double dr = r - r0;
        return 0.5 * k * dr * dr;
    }
    if (kind == ORC_FENE) {
        double q = (r * r) / (r0 * r0);
        if (!(q < 1.0)) return INFINITY;
        return -0.5 * k * r0 * r0 * orc_log(1.0 - q);
    }
    if (kind == ORC_FENEWCA) {
        double eps = P->bx[bt][0], sig = P->bx[bt][1];
        double s = r - P->bx[bt][2];
        double q = (s * s) / (r0 * r0);
        if (!(q < 1.0) || !(s > 0.0)) return INFINITY;
        double U = -0.5 * k * r0 * r0 * orc_log(1.0 - q);
        if (s < sig * ORC_TWO_SIXTH) {
            double sr2 = (sig * sig) / (s * s);
            double sr6 = (sr2 * sr2) * sr2;
            U = U + (4.0 * eps * (sr6 * sr6 - sr6) + eps);
        }
        return U;
    }
    /* Tether */
    double lmin = r0, lc1 = P->bx[bt][0], lc0 = P->bx[bt][1], lmax = P->bx[bt][2];
    if (!(r > lmin) || !(r < lmax)) return INFINITY;
    if (r > lc0) {
        double a = lc0 - r, b = lmax - r;
        return (k * orc_exp(1.0 / a)) / b;
    }
    if (r < lc1) {
        double c = r - lc1, e = r - lmin;
        return (k * orc_exp(1.0 / c)) / e;
    }
    return 0.0;
}

/* The separation a proposal aims at (Sec. II.C: |r - r0| is minimised, r0
 * read from the bond potential), read as the minimum of the bond energy: the
 * rest length (harmonic); 0 (FENE); for FENEWCA delta + s*, s* the root of
 * dU/ds on (0, min(2^(1/6) sigma, R0)) by bisection to the last bit (delta when
 * eps = 0); for Tether the middle of its zero-energy interval [l_c1, l_c0]. */
static double orc_rest_length(const orc_params *P, int32_t bt)
{
    int kind = P->bkind[bt];
    if (kind == ORC_HARMONIC) return P->br0[bt];
    if (kind == ORC_FENE) return 0.0;
    if (kind == ORC_TETHER) return 0.5 * (P->bx[bt][0] + P->bx[bt][1]);
    double k = P->bk[bt], R0 = P->br0[bt], eps = P->bx[bt][0], sig = P->bx[bt][1], delta = P->bx[bt][2];
    if (eps == 0.0) return delta;
    double lo = 0.0, hi = sig * ORC_TWO_SIXTH;
    if (R0 < hi) hi = R0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        double q = (mid * mid) / (R0 * R0);
        double f1 = (k * mid) / (1.0 - q);
        double sr2 = (sig * sig) / (mid * mid);
        double sr6 = (sr2 * sr2) * sr2;
        double f2 = ((24.0 * eps) * ((2.0 * sr6) * sr6 - sr6)) / mid;
        if (f1 - f2 > 0.0) hi = mid;
        else lo = mid;
    }
    return delta + hi;
}

double orc_aim_separation(const orc_params *P, int32_t bt) { return orc_rest_length(P, bt); }

/* Eq. (3): P_on(r) = P_on^0 exp(-U_b(r)/kT); at kT = 0 the factor is [U_b <= 0].
 * T is the sweep's temperature (set-point or kinetic) and p_on0 the sweep's rate. */
static double orc_p_on(const orc_params *P, const orc_reaction *R, double r, double T, double p_on0)
{
    double U = orc_dyn_energy(P, R->bond_type, r);
    if (T > 0.0) {
        double a = U / T;
        return p_on0 * orc_exp(-a);
    }
    return (U <= 0.0) ? p_on0 : 0.0;
}

double orc_kinetic_T(const orc_params *P, const orc_state *S)
{
    int64_t n = P->n;
    if (n <= 0) return 0.0;
    uint64_t sum = 0;
    for (int64_t i = 0; i < n; ++i) {
        double v2 = (S->vx[i] * S->vx[i] + S->vy[i] * S->vy[i]) + S->vz[i] * S->vz[i];
        sum += (uint64_t)llrint(v2 * 0x1.0p32);
    }
    return ((double)(int64_t)sum * 0x1.0p-32) / (double)(3 * n);
}

double orc_tanh(double x)
{
    double ax = fabs(x);
    double e = orc_exp(-2.0 * ax);
    double t = (1.0 - e) / (1.0 + e);
    return x < 0.0 ? -t : t;
}

/* Melting switch, Eqs. (gT)-(kT), at temperature T, with Eq. (2):
 * g = (tanh(lambda (T - T_melt)) + 1) / 2, k = k_init (1 - g) + k_melt g,
 * P = k n dt (capped at 1). */
static void orc_melt_rates(const orc_params *P, const orc_reaction *R, double T, double *pon, double *poff)
{
    double nd = (double)P->bond_period * P->dt;
    double g = 0.5 * (orc_tanh(R->melt_lambda * (T - R->melt_t)) + 1.0);
    double kon = R->kon_init * (1.0 - g) + R->kon_melt * g;
    double koff = R->koff_init * (1.0 - g) + R->koff_melt * g;
    double a = kon * nd, b = koff * nd;
    *pon = a < 1.0 ? a : 1.0;
    *poff = b < 1.0 ? b : 1.0;
}

/* Slip bond, Eq. (slip): a bond at separation r breaks with
 * P_off(r) = P_off^0 exp(a sqrt(U_b(r)/kT)), capped at 1.  As kT -> 0 the
 * factor tends to 1 for U_b = 0 and to infinity (P_off -> 1) for U_b > 0; at
 * kT = 0 it takes those limits.  An exponent of 700 or more caps at once. */
static double orc_p_off(const orc_params *P, const orc_reaction *R, double r, double T, double p_off)
{
    if (R->slip_a == 0.0 || p_off == 0.0) return p_off;
    double U = orc_dyn_energy(P, R->bond_type, r);
    double x;
    if (T > 0.0) x = U / T;
    else x = (U > 0.0) ? INFINITY : 0.0;
    double e = R->slip_a * sqrt(x);
    if (!(e < 700.0)) return 1.0;
    double p = p_off * orc_exp(e);
    return p < 1.0 ? p : 1.0;
}

/* ------------------------------------------------------------ geometry */

static double orc_min_image(double d, double L, double invL)
{
    double k = rint(d * invL);
    double s = L * k;
    return d - s;
}

static double orc_dist2(const orc_params *P, const orc_state *S, int64_t i, int64_t j,
                        double *dx, double *dy, double *dz)
{
    double ix = 1.0 / P->box[0], iy = 1.0 / P->box[1], iz = 1.0 / P->box[2];
    double a = orc_min_image(S->x[j] - S->x[i], P->box[0], ix);
    double b = orc_min_image(S->y[j] - S->y[i], P->box[1], iy);
    double c = orc_min_image(S->z[j] - S->z[i], P->box[2], iz);
    *dx = a; *dy = b; *dz = c;
    double aa = a * a;
    double bb = b * b;
    double cc = c * c;
    return (aa + bb) + cc;
}

/* Cell grid with head/next linked lists; falls back to all pairs when any
 * axis has fewer than three cells. */
typedef struct {
    int nc[3];
    int brute;
    int64_t *head, *next;
} orc_grid;

static int orc_grid_build(const orc_params *P, const orc_state *S, double cut, orc_grid *g)
{
    g->head = g->next = NULL;
    g->brute = 0;
    for (int d = 0; d < 3; ++d) {
        g->nc[d] = (int)floor(P->box[d] / cut);
        if (g->nc[d] < 3) g->brute = 1;
    }
    if (g->brute) return 0;
    int64_t ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2];
    g->head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    g->next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P->n > 0 ? P->n : 1));
    if (!g->head || !g->next) return -1;
    for (int64_t c = 0; c < ncell; ++c) g->head[c] = -1;
    for (int64_t i = P->n - 1; i >= 0; --i) {
        int cx = (int)floor(S->x[i] / P->box[0] * g->nc[0]);
        int cy = (int)floor(S->y[i] / P->box[1] * g->nc[1]);
        int cz = (int)floor(S->z[i] / P->box[2] * g->nc[2]);
        cx = ((cx % g->nc[0]) + g->nc[0]) % g->nc[0];
        cy = ((cy % g->nc[1]) + g->nc[1]) % g->nc[1];
        cz = ((cz % g->nc[2]) + g->nc[2]) % g->nc[2];
        int64_t c = ((int64_t)cz * g->nc[1] + cy) * g->nc[0] + cx;
        g->next[i] = g->head[c];
        g->head[c] = i;
    }
    return 0;
}

static void orc_grid_free(orc_grid *g)
{
    free(g->head);
    free(g->next);
    g->head = g->next = NULL;
}

/* Calls fn(j, ctx) for every particle j != i in the 27 cells around i
 * (every j != i when the grid is in all-pairs mode). */
typedef void (*orc_visit)(int64_t j, void *ctx);

static void orc_grid_visit(const orc_params *P, const orc_state *S, const orc_grid *g,
                           int64_t i, orc_visit fn, void *ctx)
{
    if (g->brute) {
        for (int64_t j = 0; j < P->n; ++j)
            if (j != i) fn(j, ctx);
        return;
    }
    int cx = (int)floor(S->x[i] / P->box[0] * g->nc[0]);
    int cy = (int)floor(S->y[i] / P->box[1] * g->nc[1]);
    int cz = (int)floor(S->z[i] / P->box[2] * g->nc[2]);
    cx = ((cx % g->nc[0]) + g->nc[0]) % g->nc[0];
    cy = ((cy % g->nc[1]) + g->nc[1]) % g->nc[1];
    cz = ((cz % g->nc[2]) + g->nc[2]) % g->nc[2];
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int x = (cx + dx + g->nc[0]) % g->nc[0];
                int y = (cy + dy + g->nc[1]) % g->nc[1];
                int z = (cz + dz + g->nc[2]) % g->nc[2];
                int64_t c = ((int64_t)z * g->nc[1] + y) * g->nc[0] + x;
                for (int64_t j = g->head[c]; j >= 0; j = g->next[j])
                    if (j != i) fn(j, ctx);
            }
}

/* ----------------------------------------------------------- the sweep */

static int orc_partner_type_ok(const orc_reaction *R, int32_t ti, int32_t tj)
{
    if (ti == R->type_a && tj == R->type_b) return 1;
    if (ti == R->type_b && tj == R->type_a) return 1;
    return 0;
}

static int orc_is_bonded(const orc_state *S, int64_t i, int64_t j)
{
    for (int s = 0; s < ORC_VMAX; ++s)
        if (S->dp[i * ORC_VMAX + s] == (int32_t)j) return 1;
    return 0;
}

/* Intramolecular exclusion (Sec. II.D): with the reaction's self-avoid flag
 * set, two sites of the same molecule (traced through the static bonds) are
 * not partners of each other. */
static int orc_same_molecule(const orc_reaction *R, const orc_state *S, int64_t i, int64_t j)
{
    return R->self_avoid && S->mol[i] == S->mol[j];
}

typedef struct {
    const orc_params *P;
    const orc_state *S;
    const orc_reaction *R;
    int64_t i;
    double rmin2, rmax2, r0;
    int64_t best;
    double best_d, best_r;
    int64_t scanned, in_window;
    int32_t *list;      /* optional candidate list */
    int32_t cap, count;
} orc_prop_ctx;

/* Proposal phase (Sec. II.C, Fig. 1a): a free site keeps the free,
 * type-compatible partner inside [r_min, r_max] whose separation is closest
 * to the rest length r0 of the reaction's bond. */
static void orc_prop_visit(int64_t j, void *vctx)
{
    orc_prop_ctx *c = (orc_prop_ctx *)vctx;
    const orc_state *S = c->S;
    const orc_params *P = c->P;
    int32_t ti = S->type[c->i], tj = S->type[j];
    if (!orc_partner_type_ok(c->R, ti, tj)) return;
    if (S->occ[j] >= P->valence[tj]) return;
    if (orc_is_bonded(S, c->i, j)) return;
    if (orc_same_molecule(c->R, S, c->i, j)) return;
    c->scanned++;
    double dx, dy, dz;
    double r2 = orc_dist2(P, S, c->i, j, &dx, &dy, &dz);
    if (r2 < c->rmin2 || r2 > c->rmax2) return;
    c->in_window++;
    if (c->list && c->count < c->cap) c->list[c->count] = (int32_t)j;
    c->count++;
    double r = sqrt(r2);
    double d = fabs(r - c->r0);
    if (c->best < 0 || d < c->best_d || (d == c->best_d && j < c->best)) {
        c->best = j;
        c->best_d = d;
        c->best_r = r;
    }
}

static double orc_max_rmax(const orc_params *P)
{
    double m = 0.0;
    for (int a = 0; a < P->nrx; ++a)
        if (P->rx[a].r_max > m) m = P->rx[a].r_max;
    return m;
}

static void orc_slot_remove(orc_state *S, int64_t i, int64_t j)
{
    int32_t *p = S->dp + i * ORC_VMAX;
    int32_t *x = S->drx + i * ORC_VMAX;
    int64_t *b = S->dbirth + i * ORC_VMAX;
    int w = 0;
    for (int s = 0; s < ORC_VMAX; ++s) {
        if (p[s] < 0 || p[s] == (int32_t)j) continue;
        p[w] = p[s]; x[w] = x[s]; b[w] = b[s];
        ++w;
    }
    for (; w < ORC_VMAX; ++w) { p[w] = -1; x[w] = -1; b[w] = 0; }
    S->occ[i] -= 1;
}

static void orc_slot_insert(orc_state *S, int64_t i, int64_t j, int32_t rx, int64_t step)
{
    int32_t *p = S->dp + i * ORC_VMAX;
    int32_t *x = S->drx + i * ORC_VMAX;
    int64_t *b = S->dbirth + i * ORC_VMAX;
    int s = ORC_VMAX - 1;
    /* shift larger partners right; the caller guarantees a free slot */
    while (s > 0 && (p[s - 1] < 0 || p[s - 1] > (int32_t)j)) {
        p[s] = p[s - 1]; x[s] = x[s - 1]; b[s] = b[s - 1];
        --s;
    }
    p[s] = (int32_t)j; x[s] = rx; b[s] = step;
    S->occ[i] += 1;
}

int32_t orc_candidates(const orc_params *P, const orc_state *S, int32_t a, int64_t i,
                       int32_t *out, int32_t cap)
{
    if (a < 0 || a >= P->nrx) return -1;
    orc_grid g;
    if (orc_grid_build(P, S, orc_max_rmax(P), &g) != 0) return -1;
    const orc_reaction *R = &P->rx[a];
    orc_prop_ctx c;
    memset(&c, 0, sizeof c);
    c.P = P; c.S = S; c.R = R; c.i = i;
    c.rmin2 = R->r_min * R->r_min;
    c.rmax2 = R->r_max * R->r_max;
    c.r0 = orc_rest_length(P, R->bond_type);
    c.best = -1;
    c.list = out; c.cap = cap;
    int32_t ti = S->type[i];
    if ((ti == R->type_a || ti == R->type_b) && S->occ[i] < P->valence[ti])
        orc_grid_visit(P, S, &g, i, orc_prop_visit, &c);
    orc_grid_free(&g);
    return c.count;
}

int orc_sweep(const orc_params *P, orc_state *S, int64_t step, orc_sweep_stats *st,
              orc_trace *tr)
{
    int64_t n = P->n;
    if (P->nrx <= 0 || n <= 0) return ORC_OK;
    orc_sweep_stats local;
    memset(&local, 0, sizeof local);
    orc_grid g;
    if (orc_grid_build(P, S, orc_max_rmax(P), &g) != 0) return ORC_ERR_ARG;

    int32_t *prop = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *prop_r = (double *)malloc(sizeof(double) * (size_t)n);
    uint64_t *bestkey = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    int32_t *fpart = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t *brk = (uint8_t *)malloc((size_t)n * ORC_VMAX);
    int64_t nb_max = n * ORC_VMAX / 2 + 1;
    int64_t *brk_i = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb_max);
    int64_t *brk_j = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb_max);
    int64_t *brk_life = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb_max);

    /* reaction order: Fisher–Yates driven by Philox(ORDER), redrawn every sweep
     * so that no reaction is favoured by its registration order (Sec. II.C) */
    int32_t order[ORC_MAX_RX];
    for (int a = 0; a < P->nrx; ++a) order[a] = a;
    for (int k = P->nrx - 1; k >= 1; --k) {
        uint32_t w[4];
        orc_pair_draw(P, 0, ORC_ORDER, step, k, 0, w);
        int j = (int)(((uint64_t)w[0] * (uint64_t)(k + 1)) >> 32);
        int32_t t = order[k]; order[k] = order[j]; order[j] = t;
    }
    if (tr && tr->order)
        for (int a = 0; a < P->nrx; ++a) tr->order[a] = order[a];

    /* the temperature of this sweep (Sec. II.B): kinetic, from the velocities
     * as the sweep begins, or the set-point; with the kinetic temperature a
     * melting switch is re-evaluated at it */
    double T = P->kinetic_T ? orc_kinetic_T(P, S) : P->kT;

    for (int slot = 0; slot < P->nrx; ++slot) {
        int32_t a = order[slot];
        const orc_reaction *R = &P->rx[a];
        double rmin2 = R->r_min * R->r_min, rmax2 = R->r_max * R->r_max;
        double r0 = orc_rest_length(P, R->bond_type);
        double p_on0 = R->p_on0, p_off0 = R->p_off;
        if (P->kinetic_T && R->melt) orc_melt_rates(P, R, T, &p_on0, &p_off0);

        /* (a) proposal — occupancies as they stand when the reaction begins */
        for (int64_t i = 0; i < n; ++i) {
            prop[i] = -1;
            prop_r[i] = 0.0;
            bestkey[i] = 0;
            fpart[i] = -1;
            int32_t ti = S->type[i];
            if (ti != R->type_a && ti != R->type_b) continue;
            if (S->occ[i] >= P->valence[ti]) continue;
            orc_prop_ctx c;
            memset(&c, 0, sizeof c);
            c.P = P; c.S = S; c.R = R; c.i = i;
            c.rmin2 = rmin2; c.rmax2 = rmax2; c.r0 = r0;
            c.best = -1;
            orc_grid_visit(P, S, &g, i, orc_prop_visit, &c);
            local.scanned += c.scanned;
            local.in_window += c.in_window;
            if (c.best >= 0) {
                prop[i] = (int32_t)c.best;
                prop_r[i] = c.best_r;
                local.proposals++;
            }
        }
        /* (b) matching — per-edge Philox priority, locally dominant edges win */
        for (int64_t i = 0; i < n; ++i) {
            if (prop[i] < 0) continue;
            int64_t j = prop[i];
            int64_t lo = i < j ? i : j, hi = i < j ? j : i;
            uint32_t w[4];
            orc_pair_draw(P, a, ORC_MATCH, step, lo, hi, w);
            uint64_t ki = ((uint64_t)w[0] << 32) | (uint64_t)(uint32_t)j;
            uint64_t kj = ((uint64_t)w[0] << 32) | (uint64_t)(uint32_t)i;
            if (ki > bestkey[i]) bestkey[i] = ki;
            if (kj > bestkey[j]) bestkey[j] = kj;
        }
        /* (c) acceptance of surviving edges with Eq. (3) */
        for (int64_t i = 0; i < n; ++i) {
            if (prop[i] < 0) continue;
            int64_t j = prop[i];
            if (prop[j] == (int32_t)i && j < i) continue;   /* mutual edge: handled once */
            local.edges++;
            int64_t lo = i < j ? i : j, hi = i < j ? j : i;
            uint32_t w[4];
            orc_pair_draw(P, a, ORC_MATCH, step, lo, hi, w);
            uint64_t ki = ((uint64_t)w[0] << 32) | (uint64_t)(uint32_t)j;
            uint64_t kj = ((uint64_t)w[0] << 32) | (uint64_t)(uint32_t)i;
            if (bestkey[i] != ki || bestkey[j] != kj) continue;
            local.survivors++;
            if (tr && slot == 0 && tr->matched) { tr->matched[i] = (int32_t)j; tr->matched[j] = (int32_t)i; }
            orc_pair_draw(P, a, ORC_FORM, step, lo, hi, w);
            double u = orc_u53(w[0], w[1]);
            double pon = orc_p_on(P, R, prop_r[i], T, p_on0);
            if (u < pon) {
                fpart[i] = (int32_t)j;
                fpart[j] = (int32_t)i;
                local.formed++;
            }
        }
        if (tr && slot == 0) {
            for (int64_t i = 0; i < n; ++i) {
                if (tr->prop) tr->prop[i] = prop[i];
                if (tr->prop_r) tr->prop_r[i] = prop_r[i];
                if (tr->formed) tr->formed[i] = (uint8_t)(fpart[i] >= 0);
            }
        }
        /* (d) breaking of this reaction's pre-existing bonds with P_off */
        memset(brk, 0, (size_t)n * ORC_VMAX);
        for (int64_t i = 0; i < n; ++i) {
            for (int s = 0; s < ORC_VMAX; ++s) {
                int32_t j = S->dp[i * ORC_VMAX + s];
                if (j < 0 || j < i) continue;
                if (S->drx[i * ORC_VMAX + s] != a) continue;
                local.break_tested++;
                uint32_t w[4];
                orc_pair_draw(P, a, ORC_BREAK, step, i, j, w);
                double p_off = p_off0;
                if (R->slip_a != 0.0) {
                    double dx, dy, dz;
                    p_off = orc_p_off(P, R, sqrt(orc_dist2(P, S, i, j, &dx, &dy, &dz)), T, p_off0);
                }
                if (orc_u53(w[0], w[1]) < p_off) brk[i * ORC_VMAX + s] = 1;
            }
        }
        /* apply: breaks first, then the formed bonds (occupancy updated for the
         * reactions processed later in this sweep).  Broken pairs are listed
         * before any slot moves so that the flags keep their meaning. */
        int64_t nbrk = 0;
        for (int64_t i = 0; i < n; ++i)
            for (int s = 0; s < ORC_VMAX; ++s)
                if (brk[i * ORC_VMAX + s]) {
                    brk_i[nbrk] = i;
                    brk_j[nbrk] = S->dp[i * ORC_VMAX + s];
                    brk_life[nbrk] = step - S->dbirth[i * ORC_VMAX + s];
                    ++nbrk;
                }
        for (int64_t q = 0; q < nbrk; ++q) {
            if (S->life_hist && S->nhist > 0) {
                int64_t per = P->bond_period > 0 ? P->bond_period : 1;
                int64_t b = brk_life[q] / per;
                if (b >= S->nhist) b = S->nhist - 1;
                if (b < 0) b = 0;
                S->life_hist[b]++;
            }
            orc_slot_remove(S, brk_i[q], brk_j[q]);
            orc_slot_remove(S, brk_j[q], brk_i[q]);
            local.broken++;
        }
        for (int64_t i = 0; i < n; ++i)
            if (fpart[i] >= 0) orc_slot_insert(S, i, fpart[i], a, step);
    }
    free(prop); free(prop_r); free(bestkey); free(fpart); free(brk);
    free(brk_i); free(brk_j); free(brk_life);
    orc_grid_free(&g);
    if (st) {
        st->scanned += local.scanned;
        st->in_window += local.in_window;
        st->proposals += local.proposals;
        st->edges += local.edges;
        st->survivors += local.survivors;
        st->formed += local.formed;
        st->break_tested += local.break_tested;
        st->broken += local.broken;
    }
    return ORC_OK;
}

/* ------------------------------------------------------- MH sweep */
/*
 * Metropolis–Hastings bond moves (an extension beyond the paper, the baseline
 * a learned proposal is measured against).  Move set: an initiator i, drawn uniformly among
 * the reactive particles of an active checkerboard cell, either forms a bond
 * with one of its owned candidates j (free, compatible, unbonded, inside
 * [r_min, r_max]) chosen with probability q(j | i) — here uniform — or breaks
 * one of its owned in-window bonds chosen uniformly.  Each pair has a fixed
 * owner (one of the two tags, by a step-independent Philox bit), so forming
 * and breaking a pair are always initiated by the same particle.  The target
 * weight of a bond is K exp(-U_b/kT) with K = P_on^0 / P_off (Eqs. 1, 3), so
 *   form : min(1, K e / (b_i(s') q(j|i; s)))
 *   break: min(1, b_i(s) q(j|i; s \ ij) / (K e))
 * with b_i the number of owned in-window bonds of i.  Cells of one colour are
 * more than 2 r_max apart, so their moves touch disjoint particles and
 * candidate sets and can run in parallel.
 */
static int orc_owner_is(const orc_params *P, int64_t i, int64_t j)
{
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    uint32_t w[4];
    orc_pair_draw(P, 0, ORC_MH_OWN, 0, lo, hi, w);
    int64_t owner = (w[0] & 1u) ? hi : lo;
    return owner == i;
}

static double orc_factor(const orc_params *P, const orc_reaction *R, double r)
{
    double U = orc_dyn_energy(P, R->bond_type, r);
    if (P->kT > 0.0) {
        double a = U / P->kT;
        return orc_exp(-a);
    }
    return (U <= 0.0) ? 1.0 : 0.0;
}

#define ORC_MH_CMAX 16

/* owned candidates of i (ascending tag); 'as_free' treats i as free and
 * 'freed' (or -1) as an unbonded free partner (the state without bond i-freed).
 * Returns the count (may exceed ORC_MH_CMAX; only the first ones are stored). */
static int orc_mh_candidates(const orc_params *P, const orc_state *S, const orc_grid *g,
                             const orc_reaction *R, int64_t i, int64_t freed, int32_t *out, double *rout)
{
    int count = 0;
    double rmin2 = R->r_min * R->r_min, rmax2 = R->r_max * R->r_max;
    int64_t cand[4096];
    int nc = 0;
    /* gather every particle in the 27 cells (or all) first, then filter */
    if (g->brute) {
        for (int64_t j = 0; j < P->n && nc < 4096; ++j)
            if (j != i) cand[nc++] = j;
    } else {
        int cx = (int)floor(S->x[i] / P->box[0] * g->nc[0]);
        int cy = (int)floor(S->y[i] / P->box[1] * g->nc[1]);
        int cz = (int)floor(S->z[i] / P->box[2] * g->nc[2]);
        cx = ((cx % g->nc[0]) + g->nc[0]) % g->nc[0];
        cy = ((cy % g->nc[1]) + g->nc[1]) % g->nc[1];
        cz = ((cz % g->nc[2]) + g->nc[2]) % g->nc[2];
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int x = (cx + dx + g->nc[0]) % g->nc[0];
                    int y = (cy + dy + g->nc[1]) % g->nc[1];
                    int z = (cz + dz + g->nc[2]) % g->nc[2];
                    int64_t c = ((int64_t)z * g->nc[1] + y) * g->nc[0] + x;
                    for (int64_t j = g->head[c]; j >= 0 && nc < 4096; j = g->next[j])
                        if (j != i) cand[nc++] = j;
                }
    }
    /* ascending tag */
    for (int a = 1; a < nc; ++a) {
        int64_t v = cand[a];
        int b = a - 1;
        while (b >= 0 && cand[b] > v) { cand[b + 1] = cand[b]; --b; }
        cand[b + 1] = v;
    }
    int32_t ti = S->type[i];
    for (int k = 0; k < nc; ++k) {
        int64_t j = cand[k];
        int32_t tj = S->type[j];
        if (!orc_partner_type_ok(R, ti, tj)) continue;
        if (j != freed) {
            if (S->occ[j] >= P->valence[tj]) continue;
            if (orc_is_bonded(S, i, j)) continue;
        }
        if (orc_same_molecule(R, S, i, j)) continue;
        if (!orc_owner_is(P, i, j)) continue;
        double dx, dy, dz;
        double r2 = orc_dist2(P, S, i, j, &dx, &dy, &dz);
        if (r2 < rmin2 || r2 > rmax2) continue;
        if (count < ORC_MH_CMAX) {
            out[count] = (int32_t)j;
            rout[count] = sqrt(r2);
        }
        count++;
    }
    return count;
}

/* owned in-window bonds of i of reaction a (ascending partner tag) */
static int orc_mh_breakable(const orc_params *P, const orc_state *S, const orc_reaction *R, int32_t a,
                            int64_t i, int32_t *out, double *rout)
{
    int count = 0;
    double rmin2 = R->r_min * R->r_min, rmax2 = R->r_max * R->r_max;
    for (int s = 0; s < ORC_VMAX; ++s) {
        int32_t j = S->dp[i * ORC_VMAX + s];
        if (j < 0 || S->drx[i * ORC_VMAX + s] != a) continue;
        if (!orc_owner_is(P, i, j)) continue;
        double dx, dy, dz;
        double r2 = orc_dist2(P, S, i, j, &dx, &dy, &dz);
        if (r2 < rmin2 || r2 > rmax2) continue;
        out[count] = j;
        rout[count] = sqrt(r2);
        count++;
    }
    return count;
}

int orc_mh_sweep(const orc_params *P, orc_state *S, int64_t step, orc_mh_stats *st)
{
    if (P->nrx < 1 || P->n <= 0) return ORC_OK;
    const int32_t a = 0;
    const orc_reaction *R = &P->rx[0];
    double side = 2.0 * R->r_max + 0.05;
    int nc[3];
    for (int d = 0; d < 3; ++d) {
        nc[d] = (int)floor(P->box[d] / side);
        if (nc[d] % 2) nc[d] -= 1;
        if (nc[d] < 2) return ORC_ERR_ARG;
    }
    orc_grid g;
    if (orc_grid_build(P, S, R->r_max, &g) != 0) return ORC_ERR_ARG;
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    /* reactive particles per MH cell, ascending tag (tags visited in order) */
    int64_t *cnt = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)P->n);
    for (int64_t i = 0; i < P->n; ++i) {
        int32_t t = S->type[i];
        cell_of[i] = -1;
        if (!((t == R->type_a || t == R->type_b) && P->valence[t] > 0)) continue;
        int c3[3];
        const double xs[3] = {S->x[i], S->y[i], S->z[i]};
        for (int d = 0; d < 3; ++d) {
            double invL = 1.0 / P->box[d];
            int c = (int)((xs[d] * invL) * (double)nc[d]);
            if (c < 0) c = 0;
            if (c >= nc[d]) c = nc[d] - 1;
            c3[d] = c;
        }
        int64_t c = ((int64_t)c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
        cell_of[i] = c;
        cnt[c + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
    int64_t *lst = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt[ncell] + 1));
    int64_t *fill = (int64_t *)calloc((size_t)ncell, sizeof(int64_t));
    for (int64_t i = 0; i < P->n; ++i)
        if (cell_of[i] >= 0) lst[cnt[cell_of[i]] + fill[cell_of[i]]++] = i;
    const uint32_t colour = (uint32_t)((uint64_t)step & 7u);
    const double K = R->p_on0 / R->p_off;
    for (int cz = 0; cz < nc[2]; ++cz)
        for (int cy = 0; cy < nc[1]; ++cy)
            for (int cx = 0; cx < nc[0]; ++cx) {
                uint32_t col = (uint32_t)(cx & 1) | ((uint32_t)(cy & 1) << 1) | ((uint32_t)(cz & 1) << 2);
                if (col != colour) continue;
                int64_t c = ((int64_t)cz * nc[1] + cy) * nc[0] + cx;
                int64_t nci = cnt[c + 1] - cnt[c];
                if (nci == 0) continue;
                uint32_t d1[4], d2[4];
                orc_pair_draw(P, a, ORC_MH_SEL, step, c, 0, d1);
                orc_pair_draw(P, a, ORC_MH_ACC, step, c, 0, d2);
                int64_t k = (int64_t)(((uint64_t)d1[0] * (uint64_t)nci) >> 32);
                int64_t i = lst[cnt[c] + k];
                double u = orc_u53(d2[0], d2[1]);
                int32_t cands[ORC_MH_CMAX], bonds[ORC_VMAX];
                double crs[ORC_MH_CMAX], brs[ORC_VMAX];
                if ((d1[1] & 1u) == 0u) {
                    if (st) st->form_attempts++;
                    if (S->occ[i] >= P->valence[S->type[i]]) continue;
                    int n = orc_mh_candidates(P, S, &g, R, i, -1, cands, crs);
                    if (n == 0 || n > ORC_MH_CMAX) continue;
                    int ci = (int)(((uint64_t)d1[2] * (uint64_t)n) >> 32);
                    int64_t j = cands[ci];
                    int bnew = orc_mh_breakable(P, S, R, a, i, bonds, brs) + 1;
                    double e = orc_factor(P, R, crs[ci]);
                    double ratio = ((K * e) * (double)n) / (double)bnew;
                    if (u < ratio) {
                        orc_slot_insert(S, i, j, a, step);
                        orc_slot_insert(S, j, i, a, step);
                        if (st) st->form_accepts++;
                    }
                } else {
                    if (st) st->break_attempts++;
                    int b = orc_mh_breakable(P, S, R, a, i, bonds, brs);
                    if (b == 0) continue;
                    int ci = (int)(((uint64_t)d1[2] * (uint64_t)b) >> 32);
                    int64_t j = bonds[ci];
                    int n2 = orc_mh_candidates(P, S, &g, R, i, j, cands, crs);
                    if (n2 > ORC_MH_CMAX) continue;
                    double e = orc_factor(P, R, brs[ci]);
                    double ratio = (double)b / ((double)n2 * (K * e));
                    if (u < ratio) {
                        int64_t birth = 0;
                        for (int s = 0; s < ORC_VMAX; ++s)
                            if (S->dp[i * ORC_VMAX + s] == (int32_t)j) birth = S->dbirth[i * ORC_VMAX + s];
                        if (S->life_hist && S->nhist > 0) {
                            int64_t per = P->bond_period > 0 ? P->bond_period : 1;
                            int64_t lb = (step - birth) / per;
                            if (lb >= S->nhist) lb = S->nhist - 1;
                            if (lb < 0) lb = 0;
                            S->life_hist[lb]++;
                        }
                        orc_slot_remove(S, i, j);
                        orc_slot_remove(S, j, i);
                        if (st) st->break_accepts++;
                    }
                }
            }
    free(cnt); free(cell_of); free(lst); free(fill);
    orc_grid_free(&g);
    return ORC_OK;
}

/* --------------------------------------------------------------- forces */

static double orc_pair_rc(const orc_params *P, int32_t ti, int32_t tj)
{
    double rc = P->rcut[ti * ORC_MAX_TYPES + tj];
    if (rc > 0.0) return rc;
    double sig = 0.5 * (P->sigma[ti] + P->sigma[tj]);
    return sig * pow(2.0, 1.0 / 6.0);
}

typedef struct {
    const orc_params *P;
    orc_state *S;
    int64_t i;
    double epair, vir;
} orc_force_ctx;

/* Shifted Lennard-Jones, U = 4 eps [(s/r)^12 - (s/r)^6] - U(r_c) for r < r_c;
 * with r_c = 2^(1/6) s this is the WCA potential. */
static void orc_force_visit(int64_t j, void *vctx)
{
    orc_force_ctx *c = (orc_force_ctx *)vctx;
    const orc_params *P = c->P;
    orc_state *S = c->S;
    int64_t i = c->i;
    if (j <= i) return;
    int32_t ti = S->type[i], tj = S->type[j];
    double rc = orc_pair_rc(P, ti, tj);
    double dx, dy, dz;
    double r2 = orc_dist2(P, S, i, j, &dx, &dy, &dz);
    if (r2 >= rc * rc) return;
    double eps = P->eps[ti * ORC_MAX_TYPES + tj];
    double sig = 0.5 * (P->sigma[ti] + P->sigma[tj]);
    double s2 = (sig * sig) / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    double fr = 24.0 * eps * (2.0 * s12 - s6) / r2;   /* -(dU/dr)/r */
    double c2 = (sig * sig) / (rc * rc);
    double c6 = c2 * c2 * c2;
    double u = 4.0 * eps * (s12 - s6) - 4.0 * eps * (c6 * c6 - c6);
    S->fx[i] -= fr * dx; S->fy[i] -= fr * dy; S->fz[i] -= fr * dz;
    S->fx[j] += fr * dx; S->fy[j] += fr * dy; S->fz[j] += fr * dz;
    if (S->pe) { S->pe[i] += 0.5 * u; S->pe[j] += 0.5 * u; }
    {
        /* |F| and r |dF/dr| of the pair force F(r) = 24 eps (2 s12 - s6) / r */
        double r = sqrt(r2);
        double f = fabs(fr) * r;
        double g = 24.0 * eps * fabs(7.0 * s6 - 26.0 * s12) / r;
        if (S->fscale) { S->fscale[i] += f + g; S->fscale[j] += f + g; }
        S->vabs += r * (f + g);
    }
    c->epair += u;
    c->vir += fr * r2;
}

/* Bond force between i and j (j > i) of bond type bt; returns 0 or ORC_ERR_FENE. */
static int orc_bond_pair(const orc_params *P, orc_state *S, int64_t i, int64_t j, int32_t bt,
                         double *eb, double *vir)
{
    double dx, dy, dz;
    double r2 = orc_dist2(P, S, i, j, &dx, &dy, &dz);
    double k = P->bk[bt], r0 = P->br0[bt];
    double fb, u, g;   /* g = r |dF/dr| of the bond force F(r) = -dU/dr */
    if (P->bkind[bt] >= ORC_FENEWCA) {
        double r = sqrt(r2), dU, d2U;
        if (orc_bond_terms(P, bt, r, &u, &dU, &d2U) != ORC_OK) return ORC_ERR_FENE;
        fb = dU / r;
        g = r * fabs(d2U);
    } else if (P->bkind[bt] == ORC_HARMONIC) {
        double r = sqrt(r2);
        fb = k * (r - r0) / r;       /* (dU/dr)/r, pulls i towards j when stretched */
        u = 0.5 * k * (r - r0) * (r - r0);
        g = k * r;
    } else {
        double q = r2 / (r0 * r0);
        if (q >= 1.0) return ORC_ERR_FENE;
        fb = k / (1.0 - q);
        u = -0.5 * k * r0 * r0 * log(1.0 - q);
        g = k * sqrt(r2) * (1.0 + q) / ((1.0 - q) * (1.0 - q));
    }
    S->fx[i] += fb * dx; S->fy[i] += fb * dy; S->fz[i] += fb * dz;
    S->fx[j] -= fb * dx; S->fy[j] -= fb * dy; S->fz[j] -= fb * dz;
    if (S->pe) { S->pe[i] += 0.5 * u; S->pe[j] += 0.5 * u; }
    {
        double r = sqrt(r2);
        double f = fabs(fb) * r;
        if (S->fscale) { S->fscale[i] += f + g; S->fscale[j] += f + g; }
        S->vabs += r * (f + g);
    }
    *eb += u;
    *vir -= fb * r2;
    return 0;
}

int orc_forces(const orc_params *P, orc_state *S, double *e_pair, double *e_bond,
               double *virial)
{
    int64_t n = P->n;
    double rcmax = 0.0;
    for (int a = 0; a < P->ntypes; ++a)
        for (int b = 0; b < P->ntypes; ++b) {
            double rc = orc_pair_rc(P, a, b);
            if (rc > rcmax) rcmax = rc;
        }
    for (int64_t i = 0; i < n; ++i) {
        S->fx[i] = S->fy[i] = S->fz[i] = 0.0;
        if (S->pe) S->pe[i] = 0.0;
        if (S->fscale) S->fscale[i] = 0.0;
    }
    S->vabs = 0.0;
    orc_grid g;
    if (orc_grid_build(P, S, rcmax > 0 ? rcmax : 1.0, &g) != 0) return ORC_ERR_ARG;
    orc_force_ctx c;
    c.P = P; c.S = S; c.epair = 0.0; c.vir = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        c.i = i;
        orc_grid_visit(P, S, &g, i, orc_force_visit, &c);
    }
    orc_grid_free(&g);
    double eb = 0.0, vir = c.vir;
    int err = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int s = 0; s < ORC_SMAX; ++s) {
            int32_t j = S->sp[i * ORC_SMAX + s];
            if (j <= i) continue;
            if (orc_bond_pair(P, S, i, j, S->sbt[i * ORC_SMAX + s], &eb, &vir)) err = ORC_ERR_FENE;
        }
        for (int s = 0; s < ORC_VMAX; ++s) {
            int32_t j = S->dp[i * ORC_VMAX + s];
            if (j <= i) continue;
            int32_t bt = P->rx[S->drx[i * ORC_VMAX + s]].bond_type;
            if (orc_bond_pair(P, S, i, j, bt, &eb, &vir)) err = ORC_ERR_FENE;
        }
    }
    if (e_pair) *e_pair = c.epair;
    if (e_bond) *e_bond = eb;
    if (virial) *virial = vir;
    return err;
}

/* ----------------------------------------------------------- integrator */

static void orc_wrap(double *x, int32_t *img, double L)
{
    if (*x >= L) {
        *x -= L;
        *img += 1;
    } else if (*x < 0.0) {
        *x += L;
        *img -= 1;
        if (*x >= L) {
            *x -= L;
            *img += 1;
        }
    }
}

/* One MD step per iteration: [bond sweep if step % period == 0] ->
 * conservative forces at x_t -> Langevin kick with drag on v_{t-1/2} and a
 * counter-based random force -> drift -> wrap. */
int orc_run(const orc_params *P, orc_state *S, int64_t nsteps, double *ke_out)
{
    int64_t n = P->n;
    double c = sqrt(((2.0 * P->gamma) * P->kT) / P->dt);
    double s3 = sqrt(3.0);
    uint32_t key[2];
    orc_key(P, 0, ORC_LANGEVIN, key);
    int err = 0;
    double ke = 0.0;
    for (int64_t it = 0; it < nsteps; ++it) {
        int64_t t = S->step;
        int64_t per = P->bond_period > 0 ? P->bond_period : 1;
        if (P->nrx > 0 && t % per == 0) orc_sweep(P, S, t, NULL, NULL);
        int e = orc_forces(P, S, NULL, NULL, NULL);
        if (e) err = e;
        ke = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            uint32_t ctr[4] = {(uint32_t)((uint64_t)t & 0xFFFFFFFFull), (uint32_t)((uint64_t)t >> 32),
                               (uint32_t)i, 0u};
            uint32_t w[4];
            orc_philox4x32_10(ctr, key, w);
            double xi[3];
            for (int d = 0; d < 3; ++d) {
                double u = (double)w[d] * 0x1.0p-32 + 0x1.0p-33;
                xi[d] = s3 * (2.0 * u - 1.0);
            }
            double f[3] = {S->fx[i], S->fy[i], S->fz[i]};
            double *v[3] = {&S->vx[i], &S->vy[i], &S->vz[i]};
            double *x[3] = {&S->x[i], &S->y[i], &S->z[i]};
            for (int d = 0; d < 3; ++d) {
                double drag = P->gamma * *v[d];
                double acc = (f[d] - drag) + c * xi[d];
                double vs = *v[d] + (0.5 * P->dt) * acc;   /* synchronised v_t */
                ke += 0.5 * vs * vs;
                *v[d] = *v[d] + P->dt * acc;
                *x[d] = *x[d] + P->dt * *v[d];
                if (!isfinite(*x[d])) err = ORC_ERR_NONFINITE;
                orc_wrap(x[d], &S->img[3 * i + d], P->box[d]);
            }
        }
        S->step = t + 1;
    }
    if (ke_out) *ke_out = ke;
    return err;
}

/* ---------------------------------------------------------- observables */

typedef struct {
    const orc_params *P;
    const orc_state *S;
    int64_t i;
    int32_t tb, same;
    double rmax2, rmax, dr;
    int32_t nbins;
    int64_t *hist;
} orc_rdf_ctx;

static void orc_rdf_visit(int64_t j, void *vctx)
{
    orc_rdf_ctx *c = (orc_rdf_ctx *)vctx;
    if (c->S->type[j] != c->tb) return;
    if (c->same && j <= c->i) return;
    double dx, dy, dz;
    double r2 = orc_dist2(c->P, c->S, c->i, j, &dx, &dy, &dz);
    if (!(r2 < c->rmax2)) return;
    double r = sqrt(r2);
    if (!(r < c->rmax)) return;
    int64_t b = (int64_t)(r / c->dr);
    if (b < c->nbins) c->hist[b]++;
}

/* Pair-distance histogram behind g(r): every unordered pair of one particle
 * of type ta and one of type tb (two distinct particles of type ta when
 * ta == tb) with r < r_max adds one to bin floor(r / dr), dr = r_max / nbins;
 * r = sqrt of the same FP64 r^2 as the sweep's window test.  Counts are added
 * to hist (the caller clears it). */
int orc_rdf(const orc_params *P, const orc_state *S, int32_t ta, int32_t tb, double rmax, int32_t nbins,
            int64_t *hist)
{
    if (!(rmax > 0.0) || nbins <= 0 || !hist) return ORC_ERR_ARG;
    orc_grid g;
    if (orc_grid_build(P, S, rmax, &g) != 0) return ORC_ERR_ARG;
    orc_rdf_ctx c;
    c.P = P; c.S = S; c.tb = tb; c.same = ta == tb;
    c.rmax = rmax; c.rmax2 = rmax * rmax; c.dr = rmax / (double)nbins; c.nbins = nbins; c.hist = hist;
    for (int64_t i = 0; i < P->n; ++i) {
        if (S->type[i] != ta) continue;
        c.i = i;
        orc_grid_visit(P, S, &g, i, orc_rdf_visit, &c);
    }
    orc_grid_free(&g);
    return ORC_OK;
}

/* ------------------------------------------------------------ pair sets */

typedef struct {
    const orc_params *P;
    const orc_state *S;
    int64_t i;
    double extra;
    int use_rx;
    int32_t *out;
    int64_t cap, count;
} orc_pairs_ctx;

static double orc_reactive_cut(const orc_params *P, int32_t ti, int32_t tj)
{
    double m = 0.0;
    for (int a = 0; a < P->nrx; ++a)
        if (orc_partner_type_ok(&P->rx[a], ti, tj) && P->rx[a].r_max > m) m = P->rx[a].r_max;
    return m;
}

static void orc_pairs_visit(int64_t j, void *vctx)
{
    orc_pairs_ctx *c = (orc_pairs_ctx *)vctx;
    if (j <= c->i) return;
    int32_t ti = c->S->type[c->i], tj = c->S->type[j];
    double rc = orc_pair_rc(c->P, ti, tj);
    if (c->use_rx) {
        double rr = orc_reactive_cut(c->P, ti, tj);
        if (rr > rc) rc = rr;
    }
    rc += c->extra;
    double dx, dy, dz;
    double r2 = orc_dist2(c->P, c->S, c->i, j, &dx, &dy, &dz);
    if (r2 >= rc * rc) return;
    if (c->count < c->cap) {
        c->out[2 * c->count] = (int32_t)c->i;
        c->out[2 * c->count + 1] = (int32_t)j;
    }
    c->count++;
}

int64_t orc_pairs_within(const orc_params *P, const orc_state *S, double extra,
                         int use_reactive_cut, int32_t *out, int64_t cap)
{
    double cut = 0.0;
    for (int a = 0; a < P->ntypes; ++a)
        for (int b = 0; b < P->ntypes; ++b) {
            double rc = orc_pair_rc(P, a, b);
            if (use_reactive_cut) {
                double rr = orc_reactive_cut(P, a, b);
                if (rr > rc) rc = rr;
            }
            if (rc > cut) cut = rc;
        }
    orc_grid g;
    if (orc_grid_build(P, S, cut + extra, &g) != 0) return -1;
    orc_pairs_ctx c;
    c.P = P; c.S = S; c.extra = extra; c.use_rx = use_reactive_cut;
    c.out = out; c.cap = cap; c.count = 0;
    for (int64_t i = 0; i < P->n; ++i) {
        c.i = i;
        orc_grid_visit(P, S, &g, i, orc_pairs_visit, &c);
    }
    orc_grid_free(&g);
    return c.count;
}
