// Deferred epilogue stores for the chunked (split-TF32) tcgen05 GEMMs.
//
// With chunked accumulation the epilogue warps must drain every chunk of the
// next tile from TMEM as soon as the MMA finishes it. If they first stored the
// whole finished tile to global memory, the MMA would stall after one chunk
// of the next tile. Instead the finished sums are parked in a TMEM sum buffer
// (tcgen05.st, one row per lane) and stored four columns at a time between the
// chunk drains of the next tile, so the stores overlap the MMAs.
#pragma once

#include "epilogue.cuh"
#include "tc_ptx.cuh"

namespace cdmpt {
namespace tc {

template <int BN>
struct PendingTile {
    const EpiParams<float>* p = nullptr;   // null: nothing pending
    uint32_t sbuf = 0;                     // TMEM address of this warp's lanes, buffer column 0
    int m = 0, n0 = 0, next = 0;           // row of this lane, first column, next 4-column group
    bool vec4 = false;
    bool diag = false;                     // diagonal tile of a symmetric result

    // Parks a finished tile: acc holds this lane's row, columns n0 .. n0 + BN - 1.
    __device__ __forceinline__ void park(const EpiParams<float>* pp, uint32_t sb, int mm, int nn0,
                                         bool dg, const float (&acc)[BN]) {
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 32) tmem_st32(sb + (uint32_t)c0, acc + c0);
        tmem_wait_st();
        p = pp;
        sbuf = sb;
        m = mm;
        n0 = nn0;
        next = 0;
        diag = dg;
        vec4 = epi_vec4_ok(*pp) && nn0 + BN <= pp->N && !(pp->sym && dg);
    }

    // Stores up to `groups` groups of four columns (warp-collective); adds the
    // D * E contributions to dsum. Returns true when the tile is complete.
    __device__ __forceinline__ bool drain(int groups, double& dsum) {
        for (int k = 0; k < groups && next < BN / 4; ++k, ++next) {
            uint32_t v[4];
            tmem_ld4(sbuf + (uint32_t)(4 * next), v);
            if (m < p->M) {
                const int n = n0 + 4 * next;
                float local = 0.f;
                if (vec4) {
                    local = epi_apply4(*p, m, n, __uint_as_float(v[0]), __uint_as_float(v[1]),
                                       __uint_as_float(v[2]), __uint_as_float(v[3]));
                } else if (p->sym) {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (n + i < p->N)
                            local += epi_apply_sym(*p, m, n + i, __uint_as_float(v[i]), diag);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (n + i < p->N) local += epi_apply(*p, m, n + i, __uint_as_float(v[i]));
                }
                dsum += (double)local;
            }
        }
        return next >= BN / 4;
    }
};

}  // namespace tc
}  // namespace cdmpt
