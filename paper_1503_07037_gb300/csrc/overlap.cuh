// Non-orthogonal basis: the Loewdin factor Z = S^(-1/2) and the congruence X -> Z X Z.
#pragma once

#include "internal.cuh"

namespace cdmpt {

// Z = S^(-1/2) for symmetric positive definite S (N x N, leading dimension ld, zero
// padding), by coupled Newton-Schulz on S / c (c >= the largest eigenvalue of S). work holds
// 4 N x ld doubles, dscal one device double. Stops when ||Z Y - I||_F / sqrt(N) < tol.
cdmpt_status lowdin_factor(const double* S, int N, int ld, double c, double* Z, double* work,
                           double* dscal, int maxit, double tol, int* iters, double* resid,
                           cudaStream_t s);

// out = Z X Z for symmetric X (FP64; tmp holds N x ldz doubles; out may alias X, which is
// read only by the first of the two products).
cdmpt_status congruence(const double* Z, int ldz, int N, const double* X, int ldx, double* out,
                        int ldo, double* tmp, cudaStream_t s);

}  // namespace cdmpt
