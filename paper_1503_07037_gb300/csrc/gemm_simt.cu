// CUDA-core GEMM D = alpha X Y^T + beta C + gamma I (FFMA for float, DFMA for
// double). This is the FP64 engine of the recursion (tcgen05 has no FP64
// kind) and an independent cross-check of the tcgen05 engines.
#include <cuda_runtime.h>

#include <string>

#include "epilogue.cuh"
#include "internal.cuh"

namespace cdmpt {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_simt(const T* __restrict__ X, int ldx,
                                                   const T* __restrict__ Y, int ldy, int K,
                                                   EpiParams<T> p, const double* skip) {
    if (skip && *skip != 0.0) return;
    __shared__ T Xs[BK][BM + 4];
    __shared__ T Ys[BK][BN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    // loader mapping: 64 rows x 16 k = 1024 elements, 4 per thread
    const int lr = threadIdx.x >> 2, lk = (threadIdx.x & 3) * 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + lk + q;
            const int mx = m0 + lr, ny = n0 + lr;
            Xs[lk + q][lr] = (mx < p.M && k < K) ? X[(size_t)mx * ldx + k] : T(0);
            Ys[lk + q][lr] = (ny < p.N && k < K) ? Y[(size_t)ny * ldy + k] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Xs[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Ys[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }

    double dsum = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= p.M) continue;
        T local = T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n < p.N) local += epi_apply(p, m, n, acc[i][j]);
        }
        dsum += (double)local;
    }
    if (p.dot) {
        __shared__ double part[8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = dsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += part[w];
            if (s != 0.0) atomicAdd(p.dot, s);
        }
    }
}

}  // namespace

template <typename T>
cdmpt_status gemm_simt(int M, int N, int K, const T* X, int ldx, const T* Y, int ldy, T* D,
                       int ldd, const Epilogue<T>& ep, const double* skip, cudaStream_t s) {
    if (M <= 0 || N <= 0) return CDMPT_OK;
    EpiParams<T> p;
    p.alpha = (T)ep.alpha;
    p.beta = (T)ep.beta;
    p.gamma = (T)ep.gamma;
    p.C = ep.C;
    p.ldc = ep.ldc;
    p.D = D;
    p.ldd = ldd;
    p.M = M;
    p.N = N;
    p.diag_block = ep.diag_block > 0 ? ep.diag_block : M;
    p.trans_block = ep.trans_block;
    p.dot = ep.dot;
    p.E = ep.E;
    p.lde = ep.lde;
    p.Dhi = ep.Dhi;
    p.Dlo = ep.Dlo;
    p.sym = 0;   // every element is computed here
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    k_gemm_simt<T><<<grid, 256, 0, s>>>(X, ldx, Y, ldy, K, p, skip);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("gemm_simt launch: ") + cudaGetErrorString(e));
        return CDMPT_ERR_CUDA;
    }
    return CDMPT_OK;
}

template cdmpt_status gemm_simt<float>(int, int, int, const float*, int, const float*, int,
                                       float*, int, const Epilogue<float>&, const double*,
                                       cudaStream_t);
template cdmpt_status gemm_simt<double>(int, int, int, const double*, int, const double*, int,
                                        double*, int, const Epilogue<double>&, const double*,
                                        cudaStream_t);

}  // namespace cdmpt
