// Self-consistent charge tight binding (a synthetic G(D) for the self-consistent layer of
// Sec. IV): Mulliken charges, the charge potential and the Fock build, plus the Anderson
// mixer of the charge fixed point.
#pragma once

#include <vector>

#include "internal.cuh"

namespace cdmpt {

// dq_i = 2 sum_j D_ij S_ij - q0_i (Mulliken populations of the restricted density D; S null
// means S = I; q0 null means zero). D and S are FP64 with leading dimensions ldd and lds.
cdmpt_status scc_charges(const double* D, int ldd, const double* S, int lds, const double* q0,
                         int N, double* dq, cudaStream_t s);

// y = A x for a symmetric N x N FP64 A with leading dimension lda.
cdmpt_status scc_gemv(const double* A, int lda, const double* x, int N, double* y,
                      cudaStream_t s);

// F_ij = h_ij + (S_ij / 2)(V_i + V_j) (S null: F_ij = h_ij + V_i delta_ij) on N x N; the
// padding columns of F (up to ldf) are left as they are.
cdmpt_status scc_fock(const double* h, int ldh, const double* S, int lds, const double* V,
                      int N, double* F, int ldf, cudaStream_t s);

// out += sum_e A[e] B[e] over count contiguous FP64 elements (no alignment or length
// requirement: scalar loads).
cdmpt_status scc_dot(const double* A, const double* B, size_t count, double* out, cudaStream_t s);

// Anderson mixing of a fixed point x = g(x) given x and the residual r = g(x) - x: returns the
// next x from the last `depth` (x, r) pairs (weight `mix` on the residual).
class Anderson {
public:
    Anderson(int n, int depth, double mix) : n_(n), depth_(depth), mix_(mix) {}
    void next(std::vector<double>& x, const std::vector<double>& r);

private:
    int n_, depth_;
    double mix_;
    std::vector<std::vector<double>> dx_, dr_;
    std::vector<double> xp_, rp_;
};

}  // namespace cdmpt
