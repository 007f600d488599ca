// Epilogue stores of the tcgen05 kernels through a per-warp shared-memory transpose.
//
// tcgen05.ld leaves one output row per lane (TMEM lane = row), so a lane that applies the
// epilogue where it stands writes 16 bytes into each of 32 different rows per instruction,
// and every load of C or E that follows a store has to wait for it (the compiler cannot
// move a load of C above a store to D that may alias it). On short-K tiles, the grouped
// products of a batch, those dependent row-strided accesses cost more than the tile's
// MMAs. Here a 32 x 32 block goes through a 32 x 33 shared-memory buffer instead: lanes
// then take 32 consecutive columns of one row, so each access of C, D, Dhi, Dlo and E is a
// 128-byte row segment, and the loads of a batch of rows are issued before its first store.
// Symmetric results send the values back through the buffer for the mirrored block, whose
// rows are the block's columns: those stores are row segments as well.
//
// A single warp per scheduler runs this code while the tensor pipe works, so it is written
// for few instructions and no divergent branches: the symmetric mirror and the TF32 split
// copies are template parameters chosen once per tile, beta C, gamma I and the dot enter
// through selects, and out-of-range elements are masked by predicated stores.
#pragma once

#include <cstdint>

#include "epilogue.cuh"

namespace cdmpt {
namespace tc {

// Words of one warp's transpose buffer: 32 rows of 33, the pad word keeping both the
// row-wise and the column-wise passes free of bank conflicts.
constexpr int kXposeWords = 32 * 33;

__device__ __forceinline__ void split_tf32(float v, float& h, float& l) {
    uint32_t hb, lb;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v));
    h = __uint_as_float(hb);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(v - h));
    l = __uint_as_float(lb);
}

// The block through the buffer: S[row][col] = a, lane = row on entry.
__device__ __forceinline__ void xpose_in(const float (&a)[32], float* S, int lane) {
#pragma unroll
    for (int j = 0; j < 32; ++j) S[lane * 33 + j] = a[j];
    __syncwarp();
}

template <bool SYM, bool SPLIT>
__device__ __forceinline__ float epi_block32_plain(const EpiParams<float>& p, int m0, int n,
                                                   bool diag, float* S, int lane) {
    constexpr int RB = 8;   // rows whose loads are issued together
    // every field the loops use, read once (p may live in global memory, where the
    // stores below could alias it)
    const int M = p.M, N = p.N;
    const size_t ldd = (size_t)p.ldd, ldc = (size_t)p.ldc, lde = (size_t)p.lde;
    float* const D = p.D;
    float* const Dhi = p.Dhi;
    float* const Dlo = p.Dlo;
    const int c = n + lane;
    const bool col_ok = c < N;
    const float alpha = p.alpha, beta = p.beta, gamma = p.gamma;
    const bool has_c = beta != 0.f, has_g = gamma != 0.f, has_dot = p.dot != nullptr;
    const bool has_e = has_dot && p.E != nullptr;
    const int db = p.diag_block;
    int mm = has_g ? m0 % db : -1;   // (m0 + r) % diag_block, advanced row by row
    const size_t o0 = (size_t)m0 * ldd + c;
    const float* Cp = has_c ? p.C + (size_t)m0 * ldc + c : nullptr;
    const float* Ep = has_e ? p.E + (size_t)m0 * lde + c : nullptr;
    float local = 0.f;
#pragma unroll 1
    for (int r0 = 0; r0 < 32; r0 += RB) {
        float cv[RB], ev[RB];
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int m = m0 + r0 + i;
            const bool ok = col_ok && m < M && !(diag && c < m);
            cv[i] = (ok && has_c) ? Cp[(size_t)(r0 + i) * ldc] : 0.f;
            ev[i] = (ok && has_e) ? Ep[(size_t)(r0 + i) * lde] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            const int m = m0 + r0 + i;
            const bool ok = col_ok && m < M && !(diag && c < m);
            float v = alpha * S[(r0 + i) * 33 + lane];
            v = has_c ? fmaf(beta, cv[i], v) : v;
            v = (has_g && mm == c) ? v + gamma : v;
            mm = (mm + 1 == db) ? 0 : mm + 1;
            if constexpr (SYM) S[(r0 + i) * 33 + lane] = v;
            const size_t o = o0 + (size_t)(r0 + i) * ldd;
            if (ok) D[o] = v;
            if constexpr (SPLIT) {
                float h, l;
                split_tf32(v, h, l);
                if (ok) {
                    Dhi[o] = h;
                    Dlo[o] = l;
                }
            }
            const float d = v * (has_e ? ev[i] : v);
            const float w = (SYM && m != c) ? 2.f * d : d;
            local += (ok && has_dot) ? w : 0.f;
        }
    }
    if constexpr (SYM) {
        // the mirrored block: lane l on row m0 + l again, column n + j goes to row n + j
        __syncwarp();
        const int m = m0 + lane;
        const bool row_ok = m < M;
        const size_t q0 = (size_t)n * ldd + m;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const int cj = n + j;
            const bool ok = row_ok && cj < N && cj != m && !(diag && cj < m);
            const float w = S[lane * 33 + j];
            const size_t o = q0 + (size_t)j * ldd;
            if (ok) D[o] = w;
            if constexpr (SPLIT) {
                float h, l;
                split_tf32(w, h, l);
                if (ok) {
                    Dhi[o] = h;
                    Dlo[o] = l;
                }
            }
        }
    }
    return local;
}

// Applies the epilogue (alpha, beta C, gamma I, transposed placement, TF32 split copies,
// symmetric mirror, Frobenius dot; the same arithmetic as epi_apply and epi_apply_sym) to
// the block of an output tile with rows m0 .. m0 + 31 and columns n .. n + 31. Lane l holds
// row m0 + l in a[0 .. 31]. diag: a diagonal tile of a symmetric result, whose elements
// below the diagonal are not taken. S: this warp's kXposeWords-word buffer. Returns the
// lane's share of the D * E sum (mirrored elements counted twice). Warp-collective.
__device__ __forceinline__ float epi_block32(const EpiParams<float>& p, int m0, int n,
                                             bool diag, const float (&a)[32], float* S,
                                             int lane) {
    float local = 0.f;
    xpose_in(a, S, lane);
    if (p.trans_block > 0) {
        // transposed placement (never symmetric): element by element, lane = row
#pragma unroll 1
        for (int j = 0; j < 32; ++j)
            if (m0 + lane < p.M && n + j < p.N)
                local += epi_apply(p, m0 + lane, n + j, S[lane * 33 + j]);
        __syncwarp();
        return local;
    }
    const bool split = p.Dhi != nullptr;
    if (p.sym)
        local = split ? epi_block32_plain<true, true>(p, m0, n, diag, S, lane)
                      : epi_block32_plain<true, false>(p, m0, n, diag, S, lane);
    else
        local = split ? epi_block32_plain<false, true>(p, m0, n, diag, S, lane)
                      : epi_block32_plain<false, false>(p, m0, n, diag, S, lane);
    __syncwarp();   // the buffer is reused by the next block
    return local;
}

}  // namespace tc
}  // namespace cdmpt
