// Device-resident solver of one canonical DMPT problem (Algorithm 1 to first
// order) for storage type T. Host code here only sequences kernel launches
// and reads back a handful of FP64 scalars (traces, CG status).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "internal.cuh"

namespace cdmpt {

struct Context {
    cudaStream_t stream = nullptr;
    int engine = CDMPT_GEMM_AUTO;   // float storage only
    bool profile = false;
    // statistics of the running solve
    cdmpt_stats* st = nullptr;
    // event pairs for GEMM timing (profile mode)
    std::vector<cudaEvent_t> ev;
    std::vector<char> ev_ok;        // pair i timed a GEMM that did its work
    size_t ev_used = 0;
    double* pinned = nullptr;       // host scalar readback (64 doubles)
};

template <typename T>
class Solver {
public:
    ~Solver();
    // (Re)allocate for N x N problems with D directions and n steps.
    cdmpt_status reserve(int N, int D, int n);
    cdmpt_status solve(Context& cx, const double* H0, const double* H1, int N, int D,
                       double gmin, double gmax, double trH0, const cdmpt_opts& o, double beta,
                       double nocc, int n, double* P0, double* P1, double* mu_out,
                       double* mu1_out, int out_on_device, double* alpha_out);

    int ld = 0;

private:
    cdmpt_status gemm(Context& cx, int M, int Nc, int K, const T* X, const T* Y, T* D,
                      const Epilogue<T>& ep, const double* skip, int engine_override = 0);
    cdmpt_status cg(Context& cx, T* X, const T* A, const T* rhs_base, double rhs_scale, int rows,
                    double tol, int maxit, int* iters_out, int engine_override = 0);
    cdmpt_status sweep(Context& cx, const double* H0, double mu, double s2, const cdmpt_opts& o,
                       int n, int* cg_iters, int engine_override);
    cdmpt_status read_scalars(Context& cx, const double* dev, int count);

    int N_ = 0, D_ = 0, n_ = 0;
    size_t blk_ = 0;                 // N * ld elements
    std::vector<T*> Z_, A_;          // trajectory Z_0..Z_n and A_0..A_{n-1}
    T *R_ = nullptr, *P_ = nullptr, *Q_ = nullptr;       // CG work (D' * N rows)
    T *S_ = nullptr, *A1_ = nullptr, *RHS_ = nullptr;    // response work
    T *Z1a_ = nullptr, *Z1b_ = nullptr;                  // response iterates
    T *Qmu_ = nullptr, *Mq_ = nullptr;                   // dP/dmu and I - Z_0^2
    double* sc_ = nullptr;           // device scalars
    std::vector<void*> allocs_;
    int rows_cap_ = 0;               // row capacity of the CG work buffers
};

}  // namespace cdmpt
