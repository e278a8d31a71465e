// Internal interface between the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>   // header-only NVTX v3: no library to link; a no-op without a tool attached
#include <stdint.h>

namespace bfint {

// A named NVTX range for the lifetime of the object: profilers (Nsight
// Systems, ncu's NVTX filters) show each entry point and kernel launch of the
// library under its name.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// One level of a 2D (quadtree) factorization on the tensor-core core
// (bf_tc.cuh, load/store kinds LD_QUAD / ST_QUAD): planar 128-RHS tiles of R
// positions in and out; group g = A nB + B reads blocks ain A + bin B + c sin
// (bszi positions each, c = 0..3) and writes aout A + bout B + c sout (bszo
// each); `parts` output parts of Nout and `chunks` K-chunks of Kin per group,
// blocks [Re F; Im F] (2 Nout x Kin, K-major core-matrix layout) per
// (group, part, chunk) in that order.
struct QuadTc {
    const float *fac;
    const uint16_t *fac16;   // BF16 rungs: the blocks split into BF16 parts
    const float2 *in;
    float2 *out;
    long long R;
    unsigned *err;
    long long ain, bin, sin, aout, bout, sout;
    int bszi, bszo, nB, ngroups, parts, chunks, Kin, Nout, nrhs;
    int split, bf16;         // as bf_plan_set_precision's rungs
    int stall;               // failure-detection test hook (no copies: every wait expires)
};

// Sets the tensor-core kernel's shared-memory attribute (once per plan).
cudaError_t tc_prepare();
cudaError_t quad_tc_launch(const QuadTc &q, int num_sms, cudaStream_t s);
// Splits nblocks FP32 blocks (rows x Kin, K-major core-matrix layout) into
// `parts` BF16 parts each (legacy default stream; the caller synchronizes).
cudaError_t bf16_split(const float *fac, uint16_t *out, long long nblocks, int rows, int Kin, int parts,
                       int num_sms);
// Byte offset of (row n, column k) in the FP32 operand layout of `rows` rows.
int tc_boff(int n, int k, int rows);

}  // namespace bfint
