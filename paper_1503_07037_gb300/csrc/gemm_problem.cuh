// One problem of a (possibly grouped) tcgen05 GEMM launch, shared by the
// kernel (gemm_tc.cu) and the batched solver that builds descriptor arrays.
#pragma once

#include <cuda.h>

#include "epilogue.cuh"

namespace cdmpt {

struct GemmProblem {
    EpiParams<float> p;        // M, N, D, C, alpha, beta, gamma, dot, ...
    int K;
    int tile_begin;            // first launch-wide tile index of this problem
    int num_mt;                // output tiles along M
    const double* skip;        // the problem is skipped while *skip != 0
    const CUtensorMap* maps;   // grouped launches: X hi, Y hi, X lo, Y lo (device memory)
    // Block-norm screening (single launches with 128-column tiles only; mask null:
    // dense). Bit kb of mask[(I * nnt + J) * nmw + kb / 32] says whether k-slice kb (32
    // columns of K) of output tile (I, J) is computed; nnt tiles per tile row, nmw words
    // per tile. counts, if not null, receives += [slices computed, slices examined].
    const uint32_t* mask;
    int nnt, nmw;
    unsigned long long* counts;
};

// Tensor map of an FP32 operand (rows x cols, leading dimension ld) as the X
// (box 128 rows) or the Y operand (box of bn rows, 0 = the engine's tile
// width) of the tcgen05 kernel. Returns false if the driver rejects it.
bool tc_encode_operand(CUtensorMap* map, const float* base, int rows, int cols, int ld,
                       bool as_y, int engine, int bn = 0);

}  // namespace cdmpt
