// HBM-bound kernels on pair-stored matrices (value = hi + lo, two FP32 arrays) for the
// mixed-precision trajectory: the exact start Z_0 from the FP64 Hamiltonian, the step
// residual's linear part, corrections added without rounding the sum back to FP32,
// symmetrisation, diagonal shifts (Newton steps on mu), traces and FP64 output.
// Every kernel that changes hi also writes its TF32 split (thi, tlo) when given, so the
// split-TF32 engine can read the updated operand. Layout as elsewhere: N-row blocks with
// leading dimension ld (a multiple of 32), zero padding preserved.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "dd.cuh"
#include "internal.cuh"

namespace cdmpt {

namespace {

constexpr int kThreads = 256;

int grid_for(size_t items) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    const size_t want = (items + kThreads - 1) / kThreads;
    return (int)std::max<size_t>(1, std::min(want, (size_t)sms * 8));
}

__device__ __forceinline__ void put(float* thi, float* tlo, size_t i, float v) {
    if (thi) {
        float h, l;
        dd::tf32_split(v, h, l);
        thi[i] = h;
        if (tlo) tlo[i] = l;
    }
}

// (hi, lo)[r][j] = scale (H[r][j] - shift [j == r mod N]) rounded to a pair, 0 in the padding
__global__ void k_pair_init(float* __restrict__ hi, float* __restrict__ lo, const double* __restrict__ H,
                            int N, int ld, int ldh, size_t rows, double scale, double shift,
                            float* __restrict__ thi, float* __restrict__ tlo) {
    const size_t total = rows * (size_t)ld;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / ld;
        const int j = (int)(e - r * ld);
        double v = 0.0;
        if (j < N) {
            v = H[r * ldh + j];
            if ((size_t)j == r % (size_t)N) v -= shift;
            v *= scale;
        }
        const float h = (float)v;
        hi[e] = h;
        lo[e] = (float)(v - (double)h);
        put(thi, tlo, e, h);
    }
}

// out = a x + b y in double-float, rounded to FP32 (a, b powers of two or zero, so the
// scalings are exact)
__global__ void k_pair_lincomb(float* __restrict__ out, float a, const float* __restrict__ xh,
                               const float* __restrict__ xl, float b, const float* __restrict__ yh,
                               const float* __restrict__ yl, size_t nvec) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvec;
         v += (size_t)gridDim.x * blockDim.x) {
        const size_t i = v * 4;
        const float4 x1 = *(const float4*)(xh + i), x2 = *(const float4*)(xl + i);
        const float4 y1 = *(const float4*)(yh + i), y2 = *(const float4*)(yl + i);
        const float X1[4] = {x1.x, x1.y, x1.z, x1.w}, X2[4] = {x2.x, x2.y, x2.z, x2.w};
        const float Y1[4] = {y1.x, y1.y, y1.z, y1.w}, Y2[4] = {y2.x, y2.y, y2.z, y2.w};
        float o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float h, l;
            dd::add(__fmul_rn(a, X1[k]), __fmul_rn(a, X2[k]), __fmul_rn(b, Y1[k]),
                    __fmul_rn(b, Y2[k]), h, l);
            o[k] = __fadd_rn(h, l);
        }
        *(float4*)(out + i) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// (hi, lo) += d, renormalised; split of the new hi
__global__ void k_pair_add(float* __restrict__ hi, float* __restrict__ lo, const float* __restrict__ d,
                           size_t nvec, float* __restrict__ thi, float* __restrict__ tlo) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < nvec;
         v += (size_t)gridDim.x * blockDim.x) {
        const size_t i = v * 4;
        const float4 h4 = *(const float4*)(hi + i), l4 = *(const float4*)(lo + i);
        const float4 d4 = *(const float4*)(d + i);
        const float H[4] = {h4.x, h4.y, h4.z, h4.w}, L[4] = {l4.x, l4.y, l4.z, l4.w};
        const float Dd[4] = {d4.x, d4.y, d4.z, d4.w};
        float oh[4], ol[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) dd::add1(H[k], L[k], Dd[k], oh[k], ol[k]);
        *(float4*)(hi + i) = make_float4(oh[0], oh[1], oh[2], oh[3]);
        *(float4*)(lo + i) = make_float4(ol[0], ol[1], ol[2], ol[3]);
        if (thi) {
#pragma unroll
            for (int k = 0; k < 4; ++k) put(thi, tlo, i + k, oh[k]);
        }
    }
}

constexpr int TT = 32;

// (hi, lo)_b = ((hi, lo)_b + (hi, lo)_b^T) / 2 in double-float, in place; block (bx, by) with
// bx < by exits, the other one owns the tile pair
__global__ void k_pair_symmetrize(float* __restrict__ hi, float* __restrict__ lo, int N, int ld,
                                  float* __restrict__ thi, float* __restrict__ tlo) {
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bi > bj) return;
    __shared__ float ah[TT][TT + 1], al[TT][TT + 1], bh[TT][TT + 1], bl[TT][TT + 1];
    const size_t base = (size_t)blockIdx.z * N * ld;
    const int i0 = bi * TT, j0 = bj * TT;
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        int r = i0 + y, c = j0 + threadIdx.x;
        bool in = r < N && c < N;
        ah[y][threadIdx.x] = in ? hi[base + (size_t)r * ld + c] : 0.f;
        al[y][threadIdx.x] = in ? lo[base + (size_t)r * ld + c] : 0.f;
        r = j0 + y;
        c = i0 + threadIdx.x;
        in = r < N && c < N;
        bh[y][threadIdx.x] = in ? hi[base + (size_t)r * ld + c] : 0.f;
        bl[y][threadIdx.x] = in ? lo[base + (size_t)r * ld + c] : 0.f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < TT; y += blockDim.y) {
        const int x = threadIdx.x;
        float h1, l1, h2, l2;
        dd::add(ah[y][x], al[y][x], bh[x][y], bl[x][y], h1, l1);   // position (i0 + y, j0 + x)
        dd::add(bh[y][x], bl[y][x], ah[x][y], al[x][y], h2, l2);   // position (j0 + y, i0 + x)
        h1 *= 0.5f;
        l1 *= 0.5f;
        h2 *= 0.5f;
        l2 *= 0.5f;
        int r = i0 + y, c = j0 + x;
        if (r < N && c < N) {
            const size_t i = base + (size_t)r * ld + c;
            hi[i] = h1;
            lo[i] = l1;
            put(thi, tlo, i, h1);
        }
        if (bi != bj) {
            r = j0 + y;
            c = i0 + x;
            if (r < N && c < N) {
                const size_t i = base + (size_t)r * ld + c;
                hi[i] = h2;
                lo[i] = l2;
                put(thi, tlo, i, h2);
            }
        }
    }
}

// diagonal of every N x N block += (sh + sl)
__global__ void k_pair_add_diag(float* __restrict__ hi, float* __restrict__ lo, int N, int ld,
                                size_t rows, float sh, float sl, float* __restrict__ thi,
                                float* __restrict__ tlo) {
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < rows;
         r += (size_t)gridDim.x * blockDim.x) {
        const size_t i = r * ld + (r % (size_t)N);
        float h, l;
        dd::add(hi[i], lo[i], sh, sl, h, l);
        hi[i] = h;
        lo[i] = l;
        put(thi, tlo, i, h);
    }
}

// out[r][j] = a (hi + lo)[r][j] + bd [j == r mod N] in FP64 (leading dimension ldo)
__global__ void k_pair_to_f64(double* __restrict__ out, int ldo, const float* __restrict__ hi,
                              const float* __restrict__ lo, int ldi, int N, size_t rows, double a,
                              double bd) {
    const size_t total = rows * (size_t)N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e / N;
        const int j = (int)(e - r * N);
        double v = a * ((double)hi[r * ldi + j] + (double)lo[r * ldi + j]);
        if ((size_t)j == r % (size_t)N) v += bd;
        out[r * ldo + j] = v;
    }
}

}  // namespace

#define PAIR_LAUNCH_CHECK()                                                              \
    do {                                                                                 \
        cudaError_t _e = cudaGetLastError();                                             \
        if (_e != cudaSuccess) {                                                         \
            set_error(std::string("pair kernel launch: ") + cudaGetErrorString(_e));    \
            return CDMPT_ERR_CUDA;                                                       \
        }                                                                                \
    } while (0)

namespace pair {

cdmpt_status init(float* hi, float* lo, const double* H, int N, int ld, int ldh, int blocks,
                  double scale, double shift, cudaStream_t s, float* thi, float* tlo) {
    const size_t rows = (size_t)blocks * N;
    k_pair_init<<<grid_for(rows * ld), kThreads, 0, s>>>(hi, lo, H, N, ld, ldh, rows, scale, shift,
                                                         thi, tlo);
    PAIR_LAUNCH_CHECK();
    return CDMPT_OK;
}

static bool pow2_or_zero(double a) {
    if (a == 0.0) return true;
    int e = 0;
    const double m = std::frexp(std::fabs(a), &e);
    return m == 0.5;
}

cdmpt_status lincomb(float* out, double a, const float* xh, const float* xl, double b,
                     const float* yh, const float* yl, size_t count, cudaStream_t s) {
    if (!pow2_or_zero(a) || !pow2_or_zero(b) || (count & 3)) {
        set_error("pair lincomb: coefficients must be powers of two and count a multiple of 4");
        return CDMPT_ERR_ARG;
    }
    const size_t nvec = count / 4;
    k_pair_lincomb<<<grid_for(nvec), kThreads, 0, s>>>(out, (float)a, xh, xl, (float)b, yh, yl,
                                                        nvec);
    PAIR_LAUNCH_CHECK();
    return CDMPT_OK;
}

cdmpt_status add(float* hi, float* lo, const float* d, size_t count, cudaStream_t s, float* thi,
                 float* tlo) {
    if (count & 3) {
        set_error("pair add: count must be a multiple of 4");
        return CDMPT_ERR_ARG;
    }
    const size_t nvec = count / 4;
    k_pair_add<<<grid_for(nvec), kThreads, 0, s>>>(hi, lo, d, nvec, thi, tlo);
    PAIR_LAUNCH_CHECK();
    return CDMPT_OK;
}

cdmpt_status symmetrize(float* hi, float* lo, int N, int ld, int blocks, cudaStream_t s,
                        float* thi, float* tlo) {
    const int nt = (N + TT - 1) / TT;
    dim3 grid(nt, nt, blocks), block(TT, 8);
    k_pair_symmetrize<<<grid, block, 0, s>>>(hi, lo, N, ld, thi, tlo);
    PAIR_LAUNCH_CHECK();
    return CDMPT_OK;
}

cdmpt_status add_diag(float* hi, float* lo, int N, int ld, int blocks, double shift,
                      cudaStream_t s, float* thi, float* tlo) {
    const size_t rows = (size_t)blocks * N;
    const float sh = (float)shift;
    const float sl = (float)(shift - (double)sh);
    k_pair_add_diag<<<grid_for(rows), kThreads, 0, s>>>(hi, lo, N, ld, rows, sh, sl, thi, tlo);
    PAIR_LAUNCH_CHECK();
    return CDMPT_OK;
}

cdmpt_status to_f64(double* out, int ldo, const float* hi, const float* lo, int ldi, int N,
                    int rows, double a, double b_diag, cudaStream_t s) {
    k_pair_to_f64<<<grid_for((size_t)rows * N), kThreads, 0, s>>>(out, ldo, hi, lo, ldi, N,
                                                                   (size_t)rows, a, b_diag);
    PAIR_LAUNCH_CHECK();
    return CDMPT_OK;
}

}  // namespace pair

}  // namespace cdmpt
