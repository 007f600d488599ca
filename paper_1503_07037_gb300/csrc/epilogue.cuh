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

}  // namespace cdmpt
