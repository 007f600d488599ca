// Self-consistent charge kernels and the Anderson mixer (see scc.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "scc.cuh"

namespace cdmpt {

namespace {

constexpr int kRows = 8;   // rows per 256-thread block (one warp per row)

__global__ void k_scc_charges(const double* __restrict__ D, int ldd, const double* __restrict__ S,
                              int lds, const double* __restrict__ q0, int N,
                              double* __restrict__ dq) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kRows + (threadIdx.x >> 5);
    if (i >= N) return;
    double acc = 0.0;
    if (S) {
        for (int j = lane; j < N; j += 32) acc += D[(size_t)i * ldd + j] * S[(size_t)i * lds + j];
    } else if (lane == 0) {
        acc = D[(size_t)i * ldd + i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) dq[i] = 2.0 * acc - (q0 ? q0[i] : 0.0);
}

__global__ void k_scc_gemv(const double* __restrict__ A, int lda, const double* __restrict__ x,
                           int N, double* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kRows + (threadIdx.x >> 5);
    if (i >= N) return;
    double acc = 0.0;
    for (int j = lane; j < N; j += 32) acc += A[(size_t)i * lda + j] * x[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) y[i] = acc;
}

__global__ void k_scc_fock(const double* __restrict__ h, int ldh, const double* __restrict__ S,
                           int lds, const double* __restrict__ V, int N, double* __restrict__ F,
                           int ldf) {
    const size_t total = (size_t)N * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e - (size_t)i * N);
        double g;
        if (S)
            g = 0.5 * S[(size_t)i * lds + j] * (V[i] + V[j]);
        else
            g = i == j ? V[i] : 0.0;
        F[(size_t)i * ldf + j] = h[(size_t)i * ldh + j] + g;
    }
}

__global__ void k_scc_dot(const double* __restrict__ A, const double* __restrict__ B,
                          size_t count, double* __restrict__ out) {
    double acc = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
         e += (size_t)gridDim.x * blockDim.x)
        acc += A[e] * B[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += part[w];
        atomicAdd(out, t);
    }
}

}  // namespace

cdmpt_status scc_dot(const double* A, const double* B, size_t count, double* out,
                     cudaStream_t s) {
    const int blocks = (int)std::min<size_t>((count + 255) / 256, 1024);
    k_scc_dot<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(A, B, count, out);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? CDMPT_OK : CDMPT_ERR_CUDA;
}

cdmpt_status scc_charges(const double* D, int ldd, const double* S, int lds, const double* q0,
                         int N, double* dq, cudaStream_t s) {
    k_scc_charges<<<(N + kRows - 1) / kRows, 32 * kRows, 0, s>>>(D, ldd, S, lds, q0, N, dq);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? CDMPT_OK : CDMPT_ERR_CUDA;
}

cdmpt_status scc_gemv(const double* A, int lda, const double* x, int N, double* y,
                      cudaStream_t s) {
    k_scc_gemv<<<(N + kRows - 1) / kRows, 32 * kRows, 0, s>>>(A, lda, x, N, y);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? CDMPT_OK : CDMPT_ERR_CUDA;
}

cdmpt_status scc_fock(const double* h, int ldh, const double* S, int lds, const double* V,
                      int N, double* F, int ldf, cudaStream_t s) {
    const size_t total = (size_t)N * N;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
    k_scc_fock<<<blocks, 256, 0, s>>>(h, ldh, S, lds, V, N, F, ldf);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? CDMPT_OK : CDMPT_ERR_CUDA;
}

// Anderson (Pulay) mixing: with the differences dX, dR of the last iterates and residuals,
// gamma = argmin ||r - dR gamma||_2 (normal equations, Tikhonov-guarded), and
// x <- x + mix r - (dX + mix dR) gamma.
void Anderson::next(std::vector<double>& x, const std::vector<double>& r) {
    if (!xp_.empty()) {
        std::vector<double> a(n_), b(n_);
        for (int i = 0; i < n_; ++i) {
            a[i] = x[i] - xp_[i];
            b[i] = r[i] - rp_[i];
        }
        dx_.push_back(a);
        dr_.push_back(b);
        if ((int)dx_.size() > depth_) {
            dx_.erase(dx_.begin());
            dr_.erase(dr_.begin());
        }
    }
    xp_ = x;
    rp_ = r;
    const int m = (int)dr_.size();
    std::vector<double> gam(m, 0.0);
    if (m > 0) {
        std::vector<double> G(m * m), c(m);
        double tr = 0.0;
        for (int p = 0; p < m; ++p) {
            for (int q = 0; q < m; ++q) {
                double v = 0.0;
                for (int i = 0; i < n_; ++i) v += dr_[p][i] * dr_[q][i];
                G[p * m + q] = v;
            }
            double v = 0.0;
            for (int i = 0; i < n_; ++i) v += dr_[p][i] * r[i];
            c[p] = v;
            tr += G[p * m + p];
        }
        for (int p = 0; p < m; ++p) G[p * m + p] += 1e-12 * (tr > 0 ? tr : 1.0);
        // Gaussian elimination with partial pivoting (m <= depth, small)
        for (int k = 0; k < m; ++k) {
            int piv = k;
            for (int p = k + 1; p < m; ++p)
                if (std::fabs(G[p * m + k]) > std::fabs(G[piv * m + k])) piv = p;
            if (piv != k) {
                for (int q = 0; q < m; ++q) std::swap(G[k * m + q], G[piv * m + q]);
                std::swap(c[k], c[piv]);
            }
            const double d = G[k * m + k];
            if (d == 0.0) continue;
            for (int p = k + 1; p < m; ++p) {
                const double f = G[p * m + k] / d;
                for (int q = k; q < m; ++q) G[p * m + q] -= f * G[k * m + q];
                c[p] -= f * c[k];
            }
        }
        for (int k = m - 1; k >= 0; --k) {
            double v = c[k];
            for (int q = k + 1; q < m; ++q) v -= G[k * m + q] * gam[q];
            gam[k] = G[k * m + k] != 0.0 ? v / G[k * m + k] : 0.0;
        }
    }
    for (int i = 0; i < n_; ++i) {
        double v = x[i] + mix_ * r[i];
        for (int p = 0; p < m; ++p) v -= (dx_[p][i] + mix_ * dr_[p][i]) * gam[p];
        x[i] = v;
    }
}

}  // namespace cdmpt
