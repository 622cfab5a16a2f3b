// Apply phase of the bond sweep for one particle (Sec. II.C, last step of a
// reaction): broken slots are removed (their lifetimes histogrammed by the
// smaller tag of each pair), the formed partner is inserted in ascending tag
// order with the current step as its birth, occupancy and availability are
// updated, and the per-reaction scratch of the particle is cleared for the
// next reaction.  Integer work only.  (Fusing it into the force kernel that
// follows measured no faster on the colloid-linker gel: the force loop is
// latency-bound and the extra loads only lengthen it.)
#pragma once
#include "snap_device.cuh"

namespace snap {

// The scratch words of one particle that the apply phase reads.
struct ApplyIn {
    uint32_t b;        // break bits
    int f;             // formed partner (sorted index) or -1
    ulonglong2 k;      // push key
    int4 dp;           // dynamic partners (tags)
};

__device__ __forceinline__ ApplyIn apply_load(const DevArrays &A, long long i)
{
    ApplyIn v;
    v.b = A.brk[i];
    v.f = A.fpart[i];
    v.k = A.pkey[i];
    v.dp = A.dp[i];
    return v;
}

// The scratch of particle i cleared for the next reaction; returns whether
// its bond slots change.
__device__ __forceinline__ bool apply_clear(DevArrays &A, long long i, const ApplyIn &v)
{
    if (v.b != 0u) A.brk[i] = 0u;
    if (v.f >= 0) A.fpart[i] = -1;
    A.best[i] = 0ull;
    A.prop[i] = -1;
    if (v.k.x != ~0ull || v.k.y != ~0ull) A.pkey[i] = make_ulonglong2(~0ull, ~0ull);
    return v.b != 0u || v.f >= 0;
}

// The slot update of a particle whose bonds change.
__device__ __forceinline__ void apply_update(const DevParams &P, DevArrays &A, int slot, long long step, long long i,
                                             const ApplyIn &v, unsigned long long &nbroken)
{
    const int me = A.tag[i];
    const int4 db = A.dbirth[i];
    const int drx = A.drx[i];
    const int pv[4] = {v.dp.x, v.dp.y, v.dp.z, v.dp.w};
    const int bv[4] = {db.x, db.y, db.z, db.w};
    int np[4] = {-1, -1, -1, -1}, nb[4] = {0, 0, 0, 0}, nr[4] = {0, 0, 0, 0};
    int m = 0;
#pragma unroll
    for (int s = 0; s < kVmax; ++s) {
        const int p = pv[s];
        if (p < 0) continue;
        if ((v.b >> s) & 1u) {
            if (me < p) {
                ++nbroken;
                long long life = (long long)((uint32_t)step - (uint32_t)bv[s]) / P.period;
                if (life >= P.nhist) life = P.nhist - 1;
                atomicAdd(&A.life_hist[life], 1ull);
            }
            continue;
        }
        np[m] = p; nb[m] = bv[s]; nr[m] = (drx >> (8 * s)) & 0xFF;
        ++m;
    }
    if (v.f >= 0) {
        const int rp = rep_of(P, A, i);
        const int a = rx_at(P, A, rp, slot);
        const int pt = A.tag[v.f];
        int s = m;
        while (s > 0 && np[s - 1] > pt) {
            np[s] = np[s - 1]; nb[s] = nb[s - 1]; nr[s] = nr[s - 1];
            --s;
        }
        np[s] = pt; nb[s] = (int)(uint32_t)step; nr[s] = a;
        ++m;
    }
    A.dp[i] = make_int4(np[0], np[1], np[2], np[3]);
    A.dbirth[i] = make_int4(nb[0], nb[1], nb[2], nb[3]);
    A.drx[i] = (nr[0] & 0xFF) | ((nr[1] & 0xFF) << 8) | ((nr[2] & 0xFF) << 16) | ((nr[3] & 0xFF) << 24);
    A.occ[i] = m;
    const int t = A.type[i];
    A.avail[i] = m < P.valence[t] ? (uint8_t)t : (uint8_t)0xFF;
}

}  // namespace snap
