// Grouped elementwise kernels of the batched solve: one launch covers every
// system of a batch, blockIdx.y (or .z) selecting the system.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cdmpt.h"

namespace cdmpt {

// Per-system operands of one grouped elementwise launch.
struct GrpEw {
    float* p0;
    float* p1;
    float* p2;
    float* p3;
    float* p4;            // pair operations only
    const double* h;      // FP64 input (init_z / dot with H)
    double* sc;           // this system's device scalars
    long long count;      // elements (rows x ld) of the operation
    int N, ld, rows;
    double s0, s1;        // op coefficients
    const double* skip;   // system skipped while *skip != 0 (may be null)
    double s2;            // CG init: tolerance^2 on the reference norm in slot kCgRefSlot (0: none)
};

// Per-system scalar slot that holds ||ref||^2 of a CG solve's absolute tolerance.
constexpr int kCgRefSlot = 11;

enum GrpOp {
    G_AXPBY = 0,      // p0 = s0 p1 + s1 p0, split to (p2, p3) when given
    G_LINCOMB = 1,    // p0 = s0 p1 + s1 p2
    G_CG_UPDATE = 2,  // X=p0, R=p1, P=p2, Q=p3 with alpha from sc
    G_CG_DIR = 3,     // P=p0, R=p1, split to (p2, p3)
    G_DOT = 4,        // sc[(int)s0] += <p0, p1>
    G_SPLIT = 5,      // (p2, p3) = split(p0)
    G_ZERO = 6,       // p0 = 0
    G_INIT_Z = 7,     // p0 = s0 (h - s1 I), split to (p2, p3)
    G_DOT_H = 8,      // sc[(int)s0] += <p0, h>   (N x N block of p0 against FP64 h, ld of h = ld)
    // pair-stored matrices (value = hi + lo, double-float arithmetic)
    G_PAIR_INIT = 9,      // (p0, p1) = s0 (h - s1 I) rounded to a pair, split of p0 to (p2, p3)
    G_PAIR_LINCOMB = 10,  // p0 = FP32(s0 (p1 + p2) + s1 (p3 + p4)), s0 and s1 powers of two
    G_PAIR_ADD = 11,      // (p0, p1) += p2 without rounding to FP32, split of p0 to (p3, p4)
};

cdmpt_status grouped_ew(int op, const GrpEw* dev_desc, int G, long long max_count,
                        cudaStream_t s);
// Tiled ops over the N x N blocks (rows / N blocks per system)
cdmpt_status grouped_symmetrize(const GrpEw* dev_desc, int G, int max_N, int max_blocks,
                                cudaStream_t s);            // p0 in place, split to (p2, p3)
cdmpt_status grouped_transpose_add(const GrpEw* dev_desc, int G, int max_N, int max_blocks,
                                   cudaStream_t s);         // p0 = p1 + p1^T, split (p2, p3)
cdmpt_status grouped_trace(const GrpEw* dev_desc, int G, int max_N, int max_blocks,
                           cudaStream_t s);                 // sc[(int)s0 + b] += Tr block b of p0
// (p0, p1) = ((p0, p1) + (p0, p1)^T) / 2 for pair-stored blocks, split of p0 to (p2, p3)
cdmpt_status grouped_pair_symmetrize(const GrpEw* dev_desc, int G, int max_N, int max_blocks,
                                     cudaStream_t s);
// CG scalar steps: one thread per system; init also sets done for skipped systems
cdmpt_status grouped_cg_init(const GrpEw* dev_desc, int G, cudaStream_t s);
cdmpt_status grouped_cg_step(const GrpEw* dev_desc, int G, cudaStream_t s);

}  // namespace cdmpt
