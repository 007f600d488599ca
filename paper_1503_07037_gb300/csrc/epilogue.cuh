// Epilogue shared by the CUDA-core and tcgen05 GEMMs:
//   D = alpha * acc + beta * C + gamma * I_blocks,
// stored at (m, n) or, with trans_block > 0, at the transposed position inside
// the row block of height trans_block that holds m; C is read at the same
// position. Optionally accumulates sum D * E (E = D when E is null).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cdmpt {

template <typename T>
struct EpiParams {
    T alpha, beta, gamma;
    const T* C;
    int ldc;
    T* D;
    int ldd;
    int M, N;
    int diag_block;
    int trans_block;
    double* dot;
    const T* E;
    int lde;
    T* Dhi;   // optional TF32 split of D (float only), same ld as D
    T* Dlo;
    int sym;  // symmetric result: upper-triangular tiles only, mirrored (see epi_apply_sym)
};

template <typename T>
__device__ __forceinline__ void epi_position(const EpiParams<T>& p, int m, int n, size_t& r,
                                             size_t& c) {
    if (p.trans_block > 0) {
        const int b = m / p.trans_block;
        r = (size_t)b * p.trans_block + n;
        c = (size_t)(m - b * p.trans_block);
    } else {
        r = (size_t)m;
        c = (size_t)n;
    }
}

// Applies the epilogue to one element; returns the D * E contribution.
template <typename T>
__device__ __forceinline__ T epi_apply(const EpiParams<T>& p, int m, int n, T acc) {
    size_t r, c;
    epi_position(p, m, n, r, c);
    T v = p.alpha * acc;
    if (p.beta != T(0)) v = fma(p.beta, p.C[r * p.ldc + c], v);
    if (p.gamma != T(0) && (m % p.diag_block) == n) v += p.gamma;
    p.D[r * p.ldd + c] = v;
    if constexpr (sizeof(T) == 4) {
        if (p.Dhi) {
            uint32_t h, l;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
            const float hv = __uint_as_float(h);
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(v - hv));
            p.Dhi[r * p.ldd + c] = hv;
            p.Dlo[r * p.ldd + c] = __uint_as_float(l);
        }
    }
    if (p.dot) return v * (p.E ? p.E[r * p.lde + c] : v);
    return T(0);
}

// Symmetric-result epilogue for element (m, n) of an upper-triangular tile:
// on a diagonal tile only n >= m is taken; the value goes to (m, n) and, off
// the diagonal, to (n, m) as well (C and E symmetric, no transposed placement).
// Returns the D * E contribution of both positions.
template <typename T>
__device__ __forceinline__ T epi_apply_sym(const EpiParams<T>& p, int m, int n, T acc,
                                           bool diag_tile) {
    if (diag_tile && n < m) return T(0);
    T v = p.alpha * acc;
    if (p.beta != T(0)) v = fma(p.beta, p.C[(size_t)m * p.ldc + n], v);
    if (p.gamma != T(0) && (m % p.diag_block) == n) v += p.gamma;
    const size_t a = (size_t)m * p.ldd + n, b = (size_t)n * p.ldd + m;
    p.D[a] = v;
    if (m != n) p.D[b] = v;
    if constexpr (sizeof(T) == 4) {
        if (p.Dhi) {
            uint32_t h, l;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
            const float hv = __uint_as_float(h);
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(v - hv));
            p.Dhi[a] = hv;
            p.Dlo[a] = __uint_as_float(l);
            if (m != n) {
                p.Dhi[b] = hv;
                p.Dlo[b] = __uint_as_float(l);
            }
        }
    }
    if (p.dot) {
        const T e = p.E ? p.E[(size_t)m * p.lde + n] : v;
        return (m != n ? T(2) : T(1)) * v * e;
    }
    return T(0);
}

// True when four consecutive columns of a row can be handled with 16-byte
// accesses: no transposed placement, leading dimensions multiples of 4 and
// 16-byte aligned arrays.
__device__ __forceinline__ bool epi_vec4_ok(const EpiParams<float>& p) {
    const int lds = p.ldd | (p.C ? p.ldc : 0) | (p.E ? p.lde : 0);
    const uintptr_t a = (uintptr_t)p.D | (uintptr_t)p.C | (uintptr_t)p.E | (uintptr_t)p.Dhi |
                        (uintptr_t)p.Dlo;
    return p.trans_block <= 0 && (lds & 3) == 0 && (a & 15) == 0;
}

// epi_apply for columns n .. n + 3 of row m (n % 4 == 0, n + 3 < N, and
// epi_vec4_ok); returns the D * E contribution of the four elements. With
// p.sym (only on off-diagonal tiles) the four values are mirrored to (n + i, m).
__device__ __forceinline__ float epi_apply4(const EpiParams<float>& p, int m, int n, float a0,
                                            float a1, float a2, float a3) {
    float v[4] = {p.alpha * a0, p.alpha * a1, p.alpha * a2, p.alpha * a3};
    if (p.beta != 0.f) {
        const float4 c = *(const float4*)(p.C + (size_t)m * p.ldc + n);
        v[0] = fmaf(p.beta, c.x, v[0]);
        v[1] = fmaf(p.beta, c.y, v[1]);
        v[2] = fmaf(p.beta, c.z, v[2]);
        v[3] = fmaf(p.beta, c.w, v[3]);
    }
    if (p.gamma != 0.f) {
        const int d = (m % p.diag_block) - n;
        v[0] += d == 0 ? p.gamma : 0.f;
        v[1] += d == 1 ? p.gamma : 0.f;
        v[2] += d == 2 ? p.gamma : 0.f;
        v[3] += d == 3 ? p.gamma : 0.f;
    }
    const size_t o = (size_t)m * p.ldd + n;
    *(float4*)(p.D + o) = make_float4(v[0], v[1], v[2], v[3]);
    if (p.sym) {
        // mirror of an off-diagonal tile: column n + i of row m to row n + i (the
        // 32 lanes of a warp hold consecutive rows, so these stores coalesce)
#pragma unroll
        for (int i = 0; i < 4; ++i) p.D[(size_t)(n + i) * p.ldd + m] = v[i];
    }
    if (p.Dhi) {
        float h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t hb, lb;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(v[i]));
            h[i] = __uint_as_float(hb);
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"(v[i] - h[i]));
            l[i] = __uint_as_float(lb);
        }
        *(float4*)(p.Dhi + o) = make_float4(h[0], h[1], h[2], h[3]);
        *(float4*)(p.Dlo + o) = make_float4(l[0], l[1], l[2], l[3]);
        if (p.sym) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                p.Dhi[(size_t)(n + i) * p.ldd + m] = h[i];
                p.Dlo[(size_t)(n + i) * p.ldd + m] = l[i];
            }
        }
    }
    if (p.dot) {
        float d;
        if (p.E) {
            const float4 e = *(const float4*)(p.E + (size_t)m * p.lde + n);
            d = v[0] * e.x + v[1] * e.y + v[2] * e.z + v[3] * e.w;
        } else {
            d = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
        }
        return p.sym ? 2.f * d : d;   // off-diagonal tile: the mirror counts too
    }
    return 0.f;
}

}  // namespace cdmpt
