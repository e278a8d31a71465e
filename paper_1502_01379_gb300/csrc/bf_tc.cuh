// Tensor-core (tcgen05) multi-RHS core, sm_103a.
//
// Pass structure.  The h transfer levels of each half act, inside one
// middle-level node's segment of m r-blocks, like the stages of a radix-2
// FFT (mirror of Eq. RSh2; the in-place slot order of bf_wide.cuh): merging
// level t pairs the slots that differ in bit t-1.  Two consecutive levels
// t, t+1 therefore act on closed groups of four slots (bits t-1 and t), and
// their product on such a group is one dense (4r) x (4r) complex block --
// with exactly as many entries, and as many multiply-adds per RHS, as the
// four r x 2r butterfly blocks it replaces (16 r^2).  The leaf factor folds
// into the first down pass (and the last up pass) the same way, and the real
// diagonal S^h of M^h (Eq. KeqUMV) into the first up pass.  The host forms
// these products in FP64 when the plan is created; each pass of the apply is
// then one dense complex block per (node, group of G <= 4 slots) applied to
// a tile of W <= 128 RHS at a time:  Y = F X with F of Nout x Kin (Nout,
// Kin <= 64).
//
// Tensor-core mapping.  The RHS sit on the MMA M dimension (M = 128; rows
// W .. 127 of a narrower tile are never read out): the
// activation tile X (128 RHS x Kin) is the A operand, read from tensor
// memory, and the block F is the B operand, streamed by TMA into shared
// memory as one K-major operand [Re F; Im F] of 2 Nout rows.  Two real
// accumulators
//     D = Re X [Re F; Im F]^T,   E = Im X [Re F; Im F]^T
// give Re Y = D[:, o] - E[:, Nout+o] and Im Y = D[:, Nout+o] + E[:, o]; the
// epilogue combines them, so no rearranged copy of F is needed.  Each MMA is
// 128 x 2 Nout x 8 (kind::tf32, FP32 accumulation).  FP32 accuracy comes from
// the 3xTF32 split x = x_hi + x_lo with x_hi = x rounded to the nearest TF32
// value (which the tensor core's truncation leaves unchanged) and
// x_lo = x - x_hi exactly: every product is formed as
// a_hi b_hi + a_hi b_lo + a_lo b_hi.  With rounding rather than truncation the
// low parts take either sign, so the dropped a_lo b_lo (~2^-24 relative) and
// the truncation of the low parts to TF32 average out over the sums instead
// of adding up pass after pass.  X_lo lives next to X in tensor memory; the
// prep warp rounds each streamed F in shared memory and builds F_lo there.
// A plan may instead ask for plain TF32 products (split = 1: one MMA per
// product, no low parts), or for BF16 operands (kind::f16, K = 16 per MMA,
// the template flag BF): plain, hi/lo (3 products) or a three-way split
// hi + mid + lo (6 products); the BF16 blocks are split once per plan into
// their parts (bf16_split_kernel) and streamed as they are, the activations
// are split by the epilogue warps as they enter tensor memory.
//
// 2D levels (LD_QUAD / ST_QUAD): the same item pipeline on one quadtree level
// of a 2D factorization -- a group's four input blocks gathered as runs of
// positions, its stack split into output parts and K-chunks of at most 64;
// the K-chunks of a work item are consecutive sub-items of one CTA that
// accumulate in tensor memory, and the epilogue reads D and E after the last.
// Items whose tile fits half the staging area get two staging buffers.
//
// Tensor memory (512 columns): Re X | Im X | Re X_lo | Im X_lo (64 each) |
// D (128) | E (128).  BF16 operands pack two values per column, so each X
// part needs Kin/2 <= 32 columns; the three-way split keeps X_mid in the
// upper 32 columns of the X_hi range.
//
// Pass intermediates are W-RHS tiles stored position-major, planar, in quads
// of positions: positions 4k .. 4k+3 of tile t hold the real parts (RHS-major,
// each RHS's four values adjacent: 16 W bytes), then the imaginary parts, so
// an r-block (r a multiple of 8) is one contiguous copy and each warp access
// is one 16-byte vector per lane, 512 contiguous bytes.  (2D levels keep one
// position per row: W real parts, then W imaginary parts.)  The host takes W
// as the RHS count over the ceil(nrhs / 128) tiles, rounded up to a multiple
// of 32, so a call with fewer than 128 vectors moves only the columns it has.
//
// Warp roles (one persistent CTA per SM, looping over work items
// (node, group, RHS tile)):
//  * producer warp: TMA bulk copies of each item's block F into a two-slot
//    ring and of the item's input tile into a shared-memory staging buffer
//    (one copy per slot for pass intermediates; for the input vectors, 2-D
//    tensor copies of W RHS rows x 128 bytes with the 128-byte swizzle, or
//    one copy per RHS row when no tensor map could be made); when it issues
//    item i's copies it also prefetches item
//    i+1's block and tile into L2, so the staging copy of item i+1 (issued
//    once item i's tile is converted) reads from L2;
//  * prep warp: F_lo for each ring slot;
//  * MMA warp: one thread issues the item's MMAs in two groups, first the
//    3 Kin/8 that accumulate D (they read Re X, Re X_lo), then the 3 Kin/8
//    for E (Im X, Im X_lo), and commits each group;
//  * eight epilogue warps (two per tensor-memory lane quarter).  While the
//    E group of item i-1 runs they read item i-1's D into registers and
//    convert the real part of item i's staged tile into Re X, Re X_lo; while
//    the D group of item i runs they read item i-1's E, combine and store its
//    outputs, and convert the imaginary part.  So the tensor pipe does not
//    wait for the epilogue.
// They meet on mbarriers; every wait is bounded (bf_kernels.cuh), and on
// expiry the CTA runs its remaining control flow without waiting or
// computing and the producer drains the copies it issued.
#pragma once

#include <cuda.h>   // CUtensorMap (type only; the map is encoded through the runtime's driver entry point)
#include <cuda_bf16.h>

#include "bf_kernels.cuh"

namespace bftc {

constexpr int NR = 128;                  // RHS per work item = MMA M
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxDim = 64;              // Kin, Nout (complex) per block
constexpr uint32_t kXr = 0, kXi = 64, kXrl = 128, kXil = 192, kD = 256, kE = 384;
constexpr int kStages = 2;
constexpr uint32_t kSlotBytes = 2u * kMaxDim * kMaxDim * 4u;                  // 32 KB
constexpr uint32_t kPointRow = kMaxDim * 8u + 16u;                           // padded staging row
constexpr uint32_t kStageBytes = (uint32_t)NR * kPointRow;                   // >= Kin * NR * 8
constexpr uint32_t kTrBytes = 32u * 64u;                                     // per-warp transpose tile

// A kernel instance with EPI epilogue warps (8 or 16: EPI / 4 per
// tensor-memory lane quarter, each taking every (EPI / 4)-th chunk of 8
// positions or outputs), then the MMA, producer and prep warps.  Tiles of up
// to 96 RHS run with 16 (their conversions and stores fall on fewer lane
// quarters, so more warps per quarter hide more latency); 128-RHS tiles with
// 8 (measured faster there: 3.79 against 4.05 ms per 128-RHS apply at
// N = 2^20).
template <int EPI>
struct Epi {
    static constexpr int warps = EPI;
    static constexpr int split = EPI / 4;          // epilogue warps per lane quarter
    static constexpr int chunks = 64 / 8 / split;  // 8-output chunks of a block per epilogue warp
    static constexpr int mma_warp = EPI, prod_warp = EPI + 1, prep_warp = EPI + 2;
    static constexpr int threads = (EPI + 3) * 32;
    static constexpr size_t smem = 2ull * kStages * kSlotBytes + kStageBytes + EPI * kTrBytes + 256;
};

enum LoadKind : int { LD_POINTS = 0, LD_SLOTS = 1, LD_GATHER = 2, LD_QUAD = 3 };
enum StoreKind : int { ST_SLOTS = 0, ST_LOGICAL = 1, ST_POINTS = 2, ST_QUAD = 3 };

// Passed as a __grid_constant__ kernel parameter: the TMA reads the tensor
// map from parameter space.
struct alignas(64) TcParams {
    CUtensorMap tmap;       // LD_POINTS with use_tmap: the input vectors as {2 N floats, nrhs rows}
    const float *fac;       // per (node, group): [Re F; Im F], 2 Nout x Kin, K-major no-swizzle
    const uint16_t *fac16;  // BF16 rungs: per (node, group) the split parts (hi, then lo or mid, lo) of
                            // the same block, each 2 Nout x Kin BF16 in the 8-element core-row layout
    const float2 *in;       // LD_POINTS: vectors, RHS j at in + j ld_in; else tiles [t][R][re 128 | im 128]
    long long ld_in;
    float2 *out;            // ST_POINTS: vectors, RHS j at out + j ld_out; else tiles [t][R][re 128 | im 128]
    long long ld_out;
    long long R;            // positions per RHS in an intermediate (2^L r)
    unsigned *err;
    int load_kind, store_kind;
    int m, r, n0, h;
    int a, kb, G, ngroups;  // the group's slots differ in node-slot bits a .. a+kb-1
    int Kin, Nout;
    int nrhs;
    int W;                  // RHS per tile (a multiple of 32, <= NR): tile t holds RHS t W .. t W + W - 1;
                            // intermediates hold R positions x W RHS per tile (layout above)
    int split;              // products per real product: 1 plain; 3 hi/lo split; 6 (BF16 only) hi/mid/lo split
    int stall;              // failure-detection test hook: the producer issues no copies, so every
                            // consumer wait runs into its bound and the launch reports BF_ERR_TIMEOUT
    int bf16;               // operand type: 0 TF32 (kind::tf32, K = 8), 1 BF16 (kind::f16, K = 16)
    int use_tmap;           // LD_POINTS: load the tile by tensor-map copies (else one copy per row)
    // LD_QUAD / ST_QUAD: one level of a 2D (quadtree) factorization.  Group g = A q_nB + B
    // reads the four blocks q_ain A + q_bin B + c q_sin (c = 0..3, q_bszi positions each)
    // and writes q_aout A + q_bout B + c q_sout (q_bszo each).  A work item is
    // (group, output part, RHS tile): Nout of the group's 4 q_bszo outputs, accumulated
    // over q_chunks K-chunks of Kin inputs each (consecutive sub-items of one CTA).
    long long q_ain, q_bin, q_sin, q_aout, q_bout, q_sout;
    int q_bszi, q_bszo, q_nB, q_ngroups, q_parts, q_chunks;
};

// Byte offset of (row n, col k) in a K-major no-swizzle operand of `rows`
// rows: K-adjacent 8x16-byte core matrices rows/8*128 B apart (LBO), 8-row
// groups 128 B apart (SBO).
__host__ __device__ inline int boff(int n, int k, int rows) {
    return (k >> 2) * (rows >> 3) * 128 + (n >> 3) * 128 + (n & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ int slot_of(const TcParams &p, int g, int j) {
    return ((g >> p.a) << (p.a + p.kb)) | (j << p.a) | (g & ((1 << p.a) - 1));
}
__device__ __forceinline__ int bitrev(int x, int bits) {
    return bits ? (int)(__brev((unsigned)x) >> (32 - bits)) : 0;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// kind::tf32, FP32 accumulator, A and B K-major, N = n, M = 128.
__device__ __forceinline__ uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(NR >> 4) << 24);
}
// kind::f16 with A and B both BF16, FP32 accumulator, K-major, N = n, M = 128.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(NR >> 4) << 24);
}
// D[tmem] (+)= A[tmem] * B[smem], BF16 operands (K = 16)
__device__ __forceinline__ void mma_ts_bf16(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}
// D[tmem] (+)= A[tmem] * B[smem]
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bfk::smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Two 32x32b.x8 tensor-memory loads and their wait in one asm statement, so
// no register is read before the data has arrived.
__device__ __forceinline__ void tmem_ld8x2(uint32_t a0, uint32_t a1, float (&v0)[8], float (&v1)[8]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(a0), "r"(a1)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        v0[i] = __uint_as_float(r[i]);
        v1[i] = __uint_as_float(r[8 + i]);
    }
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t (&v)[4]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// Part of x below the TF32 mantissa (the tensor core truncates the low 13 bits).
// x rounded to the nearest TF32 value (10-bit mantissa; ties away from zero).
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x00001000u) & 0xFFFFE000u);
}
// x rounded to the nearest BF16 value (ties away from zero), as FP32 bits
// whose low 16 bits are zero: two integer ALU operations.
__device__ __forceinline__ uint32_t bf16_hi_bits(float x) { return (__float_as_uint(x) + 0x8000u) & 0xFFFF0000u; }
// Two values rounded to BF16 (to nearest even) and packed, a in the low half
// (the lower K index of an operand pair): one conversion instruction.
__device__ __forceinline__ uint32_t pack_bf16_rn(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}
// The splits below take the high (and middle) parts by integer rounding and
// only the last part by a conversion, so the work is shared between the
// integer and conversion pipes; every difference is exact in FP32.
// Eight values -> BF16 pairs: x rounded (plain rung).
__device__ __forceinline__ void round_bf16x8(const float (&v)[8], uint32_t (&hi)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) hi[i] = pack_bf16_rn(v[2 * i], v[2 * i + 1]);
}
// Eight values -> BF16 high parts (x rounded) and low parts (x - hi, rounded): 16 mantissa bits.
__device__ __forceinline__ void split_bf16x8(const float (&v)[8], uint32_t (&hi)[4], uint32_t (&lo)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t h0 = bf16_hi_bits(v[2 * i]), h1 = bf16_hi_bits(v[2 * i + 1]);
        hi[i] = __byte_perm(h0, h1, 0x7632);
        lo[i] = pack_bf16_rn(v[2 * i] - __uint_as_float(h0), v[2 * i + 1] - __uint_as_float(h1));
    }
}
// Three-way split x = hi + mid + lo: 24 mantissa bits.
__device__ __forceinline__ void split3_bf16x8(const float (&v)[8], uint32_t (&hi)[4], uint32_t (&mid)[4],
                                              uint32_t (&lo)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t h0 = bf16_hi_bits(v[2 * i]), h1 = bf16_hi_bits(v[2 * i + 1]);
        const float r0 = v[2 * i] - __uint_as_float(h0), r1 = v[2 * i + 1] - __uint_as_float(h1);
        const uint32_t m0 = bf16_hi_bits(r0), m1 = bf16_hi_bits(r1);
        hi[i] = __byte_perm(h0, h1, 0x7632);
        mid[i] = __byte_perm(m0, m1, 0x7632);
        lo[i] = pack_bf16_rn(r0 - __uint_as_float(m0), r1 - __uint_as_float(m1));
    }
}

struct Smem {
    float *ring, *blo;                 // kStages slots of kSlotBytes each
    unsigned char *xs;                 // input staging
    float4 *tr;                        // per-warp transpose tiles (output rows)
    uint64_t *full, *empty, *bready;   // [kStages]
    uint64_t *xfull, *xfree;           // [2]: staging buffer landed / consumed
    uint64_t *xrready, *xiready;       // Re X / Im X written (and D / E of the last item read)
    uint64_t *ddone, *edone;           // D group / E group of MMAs completed
    uint32_t *tmem_slot;
    volatile int *abort_flag;
};

// Lane 0 waits on an mbarrier phase; the result is broadcast to the warp.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, unsigned *err) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = !*abort_flag && bfk::mbar_wait(bar, parity, abort_flag, err);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}
__device__ __forceinline__ void warp_arrive(uint64_t *bar) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) bfk::mbar_arrive(bar);
}

struct Item {
    int n, g, t, nt;
    int part, chunk;   // LD_QUAD: output part and K-chunk (0 otherwise)
    bool last;         // last K-chunk: the accumulators hold the item's result
    long long blk;     // index of the item's block F
};
__device__ __forceinline__ int nchunks(const TcParams &p) { return p.q_chunks > 1 ? p.q_chunks : 1; }
__device__ __forceinline__ int nwork(const TcParams &p, int ntiles) {
    return (p.load_kind == LD_QUAD ? p.q_ngroups * p.q_parts : p.m * p.ngroups) * ntiles;
}
// Work item of this CTA's sub-item s: work items blockIdx.x, + gridDim.x, ..., each
// taken as nchunks consecutive sub-items (its K-chunks).
// (Every warp decodes every item, so the common cases avoid integer division.)
__device__ __forceinline__ int sub_item(const TcParams &p, int s) {
    return blockIdx.x + (p.q_chunks > 1 ? s / p.q_chunks : s) * gridDim.x;
}
__device__ __forceinline__ int chunk_of(const TcParams &p, int s) { return p.q_chunks > 1 ? s % p.q_chunks : 0; }
__device__ __forceinline__ Item decode(const TcParams &p, int item, int chunk, int ntiles) {
    Item it;
    it.t = ntiles == 1 ? 0 : item % ntiles;
    const int ng = ntiles == 1 ? item : item / ntiles;
    it.chunk = chunk;
    it.last = chunk == nchunks(p) - 1;
    if (p.load_kind == LD_QUAD) {
        it.n = 0;
        it.g = ng / p.q_parts;
        it.part = ng - it.g * p.q_parts;
        it.blk = (long long)ng * nchunks(p) + chunk;
    } else if ((p.ngroups & (p.ngroups - 1)) == 0) {   // 1D: a power of two
        it.n = ng >> (__ffs(p.ngroups) - 1);
        it.g = ng & (p.ngroups - 1);
        it.part = 0;
        it.blk = (long long)ng;
    } else {
        it.n = ng / p.ngroups;
        it.g = ng - it.n * p.ngroups;
        it.part = 0;
        it.blk = (long long)it.n * p.ngroups + it.g;
    }
    it.nt = min(p.W, p.nrhs - it.t * p.W);
    return it;
}
// Input staging buffers: two halves of the staging area when an item's tile
// (Kin positions x p.W RHS) fits one -- tiles of up to 64 RHS, and passes or
// 2D K-chunks of at most 32 positions -- so the next tile's copy overlaps this
// tile's conversion; else one.
constexpr uint32_t kHalfStage = kStageBytes / 2;
__device__ __forceinline__ int nbufs(const TcParams &p) {
    const uint32_t need = p.load_kind == LD_POINTS && !p.use_tmap ? (uint32_t)p.W * kPointRow
                                                                  : (uint32_t)p.Kin * p.W * 8u;
    return need <= kHalfStage ? 2 : 1;
}
// LD_QUAD / ST_QUAD: first input / output block index of the item's group.
__device__ __forceinline__ long long quad_in_base(const TcParams &p, const Item &w) {
    const int A = w.g / p.q_nB, B = w.g - A * p.q_nB;
    return p.q_ain * A + p.q_bin * B;
}
__device__ __forceinline__ long long quad_out_base(const TcParams &p, const Item &w) {
    const int A = w.g / p.q_nB, B = w.g - A * p.q_nB;
    return p.q_aout * A + p.q_bout * B;
}

// Position (in the intermediate) of the first entry of local slot j's r-block.
__device__ __forceinline__ long long slot_pos(const TcParams &p, const Item &it, int j) {
    const int ps = slot_of(p, it.g, j);
    if (p.load_kind == LD_GATHER) return ((long long)bitrev(ps, p.h) * p.m + it.n) * p.r;   // M^h: block q of row node n
    return ((long long)it.n * p.m + ps) * p.r;
}

// One 2-D tensor-map tile (TMA) into shared memory, counted on `bar`.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            bfk::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bfk::smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void prefetch_tile_2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}
// One tensor-map tile: W RHS rows x 128 bytes (16 points).
__device__ __forceinline__ uint32_t box_bytes(const TcParams &p) { return (uint32_t)p.W * 128u; }

__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Bounded wait that ignores the abort flag (drains before exit).
__device__ __forceinline__ void drain_wait(uint64_t *bar, uint32_t parity) {
    if (bfk::mbar_try_wait(bar, parity)) return;
    const unsigned long long t0 = bfk::globaltimer();
    while (!bfk::mbar_try_wait(bar, parity) && bfk::globaltimer() - t0 < bfk::kWaitNs) {
    }
}

// The copies of an item's input tile: `fn(staging offset, src, bytes)` per copy,
// distributed over the warp's lanes.
template <class Fn>
__device__ __forceinline__ void tile_copies(const TcParams &p, const Item &w, int lane, Fn fn) {
    if (p.load_kind == LD_POINTS) {
        const float2 *src = p.in + (long long)(w.t * p.W) * p.ld_in + ((long long)w.n * p.m + slot_of(p, w.g, 0)) * p.n0;
        for (int row = lane; row < w.nt; row += 32)
            fn((uint32_t)row * kPointRow, src + (long long)row * p.ld_in, (uint32_t)p.Kin * 8u);
    } else if (p.load_kind == LD_QUAD) {
        // inputs chunk*Kin .. +Kin of the group's stack: runs inside its four blocks
        const int k0 = w.chunk * p.Kin, c0 = k0 / p.q_bszi, c1 = (k0 + p.Kin - 1) / p.q_bszi;
        const long long base = quad_in_base(p, w);
        for (int c = c0 + lane; c <= c1; c += 32) {
            const int ka = max(k0, c * p.q_bszi), kb = min(k0 + p.Kin, (c + 1) * p.q_bszi);
            const long long pos = (base + c * p.q_sin) * p.q_bszi + (ka - c * p.q_bszi);
            fn((uint32_t)(ka - k0) * p.W * 8u, p.in + ((long long)w.t * p.R + pos) * p.W, (uint32_t)(kb - ka) * p.W * 8u);
        }
    } else {
        for (int j = lane; j < p.G; j += 32)
            fn((uint32_t)j * p.r * p.W * 8u, p.in + ((long long)w.t * p.R + slot_pos(p, w, j)) * p.W,
               (uint32_t)p.r * p.W * 8u);
    }
}
__device__ __forceinline__ uint32_t tile_bytes(const TcParams &p, const Item &w) {
    if (p.load_kind == LD_POINTS)
        return p.use_tmap ? (uint32_t)(p.Kin / 16) * box_bytes(p) : (uint32_t)p.Kin * 8u * (uint32_t)w.nt;
    if (p.load_kind == LD_QUAD) return (uint32_t)p.Kin * p.W * 8u;
    return (uint32_t)p.r * p.W * 8u * (uint32_t)p.G;
}
// Tensor-map coordinates of an LD_POINTS item: x (floats) of its first point, y (row) of its first RHS.
__device__ __forceinline__ int points_x(const TcParams &p, const Item &w) {
    return (int)(2 * (((long long)w.n * p.m + slot_of(p, w.g, 0)) * p.n0));
}
__device__ __forceinline__ const float *block_src(const TcParams &p, const Item &w) {
    return p.fac + w.blk * (2ll * p.Nout * p.Kin);
}
// BF16 rungs: split parts per block and bytes per part.
__device__ __forceinline__ int bf16_parts(const TcParams &p) { return p.split == 6 ? 3 : p.split == 3 ? 2 : 1; }
__device__ __forceinline__ uint32_t part_bytes(const TcParams &p) { return 2u * p.Nout * p.Kin * 2u; }
__device__ __forceinline__ const uint16_t *block_src16(const TcParams &p, const Item &w) {
    return p.fac16 + w.blk * (2ll * p.Nout * p.Kin) * bf16_parts(p);
}
// Bytes of one item's block as streamed: FP32, or the BF16 parts.
template <bool BF>
__device__ __forceinline__ uint32_t block_bytes(const TcParams &p) {
    return BF ? part_bytes(p) * (uint32_t)bf16_parts(p) : 2u * p.Nout * p.Kin * 4u;
}

// Producer warp: the item's block F into ring slot (it % kStages), then its
// input tile into the staging buffer once the epilogue warps have converted
// the previous one; with the copies of item i, L2 prefetches of item i+1.
template <bool BF>
__device__ __forceinline__ void producer(const TcParams &p, const Smem &s, int ntiles, int nitems) {
    const int lane = threadIdx.x & 31;
    const uint32_t ubytes = block_bytes<BF>(p);
    uint32_t nf = 0, nx = 0;   // factor copies / staging groups issued
    const uint32_t nb = (uint32_t)nbufs(p);
    for (int sub = 0; !p.stall && sub_item(p, sub) < nitems; ++sub) {
        const Item w = decode(p, sub_item(p, sub), chunk_of(p, sub), ntiles);
        const uint32_t slot = nf % kStages, use = nf / kStages;
        bool ok = true;
        if (lane == 0) {
            ok = !*s.abort_flag && (use == 0 || bfk::mbar_wait(&s.empty[slot], (use - 1) & 1, s.abort_flag, p.err));
            if (ok) {
                bfk::mbar_arrive_expect_tx(&s.full[slot], ubytes);
                if (!BF) {
                    bfk::bulk_g2s(s.ring + (size_t)slot * (kSlotBytes / 4), block_src(p, w), ubytes, &s.full[slot]);
                } else {   // parts 0, 1 into the ring slot, part 2 (three-way split) into the second buffer
                    const uint32_t pb = part_bytes(p), n01 = min(ubytes, 2u * pb);
                    bfk::bulk_g2s(s.ring + (size_t)slot * (kSlotBytes / 4), block_src16(p, w), n01, &s.full[slot]);
                    if (ubytes > n01)
                        bfk::bulk_g2s(s.blo + (size_t)slot * (kSlotBytes / 4),
                                      reinterpret_cast<const unsigned char *>(block_src16(p, w)) + n01, ubytes - n01,
                                      &s.full[slot]);
                }
            }
        }
        if (__shfl_sync(0xffffffffu, ok ? 1 : 0, 0) == 0) break;
        ++nf;
        const uint32_t xb = nx % nb, xuse = nx / nb;
        if (xuse > 0 && !warp_wait(&s.xfree[xb], (xuse - 1) & 1, s.abort_flag, p.err)) break;
        if (lane == 0) bfk::mbar_arrive_expect_tx(&s.xfull[xb], tile_bytes(p, w));
        __syncwarp();
        unsigned char *xs = s.xs + xb * kHalfStage;
        if (p.load_kind == LD_POINTS && p.use_tmap) {
            if (lane < p.Kin / 16)
                tma_load_2d(xs + (size_t)lane * box_bytes(p), &p.tmap, points_x(p, w) + 32 * lane, w.t * p.W, &s.xfull[xb]);
        } else
            tile_copies(p, w, lane, [&](uint32_t off, const void *src, uint32_t b) { bfk::bulk_g2s(xs + off, src, b, &s.xfull[xb]); });
        ++nx;
        if (sub_item(p, sub + 1) < nitems) {   // next item of this CTA: into L2
            const Item w2 = decode(p, sub_item(p, sub + 1), chunk_of(p, sub + 1), ntiles);
            if (lane == 0) prefetch_l2(BF ? (const void *)block_src16(p, w2) : (const void *)block_src(p, w2), ubytes);
            if (p.load_kind == LD_POINTS && p.use_tmap) {
                if (lane < p.Kin / 16) prefetch_tile_2d(&p.tmap, points_x(p, w2) + 32 * lane, w2.t * p.W);
            } else {
                tile_copies(p, w2, lane, [&](uint32_t, const void *src, uint32_t b) { prefetch_l2(src, b); });
            }
        }
    }
    // Every copy issued must land before the CTA may exit.
    if (lane == 0) {
        for (uint32_t k = nf > (uint32_t)kStages ? nf - kStages : 0; k < nf; ++k)
            drain_wait(&s.full[k % kStages], (k / kStages) & 1);
        for (uint32_t k = nx > nb ? nx - nb : 0; k < nx; ++k) drain_wait(&s.xfull[k % nb], (k / nb) & 1);
    }
}

// Prep warp: each streamed block rounded to TF32 in place and its low part
// F_lo, in the same operand layout.
template <bool BF>
__device__ __forceinline__ void prep(const TcParams &p, const Smem &s, int nitems) {
    const int lane = threadIdx.x & 31;
    const int n4 = 2 * p.Nout * p.Kin / 4;
    uint32_t it = 0;
    for (int sub = 0; sub_item(p, sub) < nitems; ++sub, ++it) {
        const uint32_t slot = it % kStages;
        const bool ok = warp_wait(&s.full[slot], (it / kStages) & 1, s.abort_flag, p.err);
        if (ok && !BF) {   // (BF16 rungs stream blocks already split: nothing to do)
            // the block rounded to TF32 in place (the MMAs read it), F_lo = F - round(F)
            float4 *hi = reinterpret_cast<float4 *>(s.ring + (size_t)slot * (kSlotBytes / 4));
            float4 *lo = reinterpret_cast<float4 *>(s.blo + (size_t)slot * (kSlotBytes / 4));
            for (int i = lane; i < n4; i += 32) {
                const float4 v = hi[i];
                const float4 r = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
                hi[i] = r;
                if (p.split > 1) lo[i] = make_float4(v.x - r.x, v.y - r.y, v.z - r.z, v.w - r.w);
            }
            fence_async_smem();
        }
        warp_arrive(&s.bready[slot]);
    }
}

// MMA warp (one thread): per item the D group (Re X) then the E group (Im X).
template <bool BF>
__device__ __forceinline__ void mma_issuer(const TcParams &p, const Smem &s, uint32_t tmem, int nitems) {
    const int rows = 2 * p.Nout;
    const uint32_t lbo = (uint32_t)(rows >> 3) * 128u;
    const uint32_t idesc = idesc_tf32(rows);
    uint32_t it = 0;
    for (int sub = 0; sub_item(p, sub) < nitems; ++sub, ++it) {
        const uint32_t acc0 = chunk_of(p, sub) ? 1u : 0u;   // later K-chunks accumulate
        const uint32_t slot = it % kStages;
        const uint32_t b1 = bfk::smem_u32(s.ring) + slot * kSlotBytes;
        const uint32_t bl = bfk::smem_u32(s.blo) + slot * kSlotBytes;
        bool ok = !*s.abort_flag && bfk::mbar_wait(s.xrready, it & 1, s.abort_flag, p.err);
        ok = ok && bfk::mbar_wait(&s.bready[slot], (it / kStages) & 1, s.abort_flag, p.err);
        tc_fence_after();
        for (int grp = 0; grp < 2; ++grp) {
            if (grp == 1) {
                ok = ok && bfk::mbar_wait(s.xiready, it & 1, s.abort_flag, p.err);
                tc_fence_after();
            }
            const uint32_t d = tmem + (grp ? kE : kD);
            const uint32_t xh = tmem + (grp ? kXi : kXr), xl = tmem + (grp ? kXil : kXrl);
            if (BF && ok && p.split == 6) {
                // BF16 three-way split: the terms of order 2^-16 (hi lo, lo hi, mid mid),
                // then 2^-8 (hi mid, mid hi), then hi hi.  X_mid sits 32 columns after X_hi.
                const uint32_t pb = 2u * p.Nout * p.Kin * 2u;
                const uint32_t idesc16 = idesc_bf16(rows), bhi = b1, bmid = b1 + pb, blow = bl;
                const int nk = p.Kin / 16;
                for (int kk = 0; kk < nk; ++kk) {
                    const uint32_t bo = (uint32_t)(2 * kk) * lbo, c = (uint32_t)(8 * kk);
                    mma_ts_bf16(d, xh + c, sdesc(blow + bo, lbo, 128), idesc16, (kk || acc0) ? 1u : 0u);
                    mma_ts_bf16(d, xl + c, sdesc(bhi + bo, lbo, 128), idesc16, 1);
                    mma_ts_bf16(d, xh + 32 + c, sdesc(bmid + bo, lbo, 128), idesc16, 1);
                }
                for (int kk = 0; kk < nk; ++kk) {
                    const uint32_t bo = (uint32_t)(2 * kk) * lbo, c = (uint32_t)(8 * kk);
                    mma_ts_bf16(d, xh + c, sdesc(bmid + bo, lbo, 128), idesc16, 1);
                    mma_ts_bf16(d, xh + 32 + c, sdesc(bhi + bo, lbo, 128), idesc16, 1);
                }
                for (int kk = 0; kk < nk; ++kk)
                    mma_ts_bf16(d, xh + (uint32_t)(8 * kk), sdesc(bhi + (uint32_t)(2 * kk) * lbo, lbo, 128), idesc16, 1);
            } else if (BF && ok) {
                // BF16: K = 16 per MMA; F_hi, F_lo consecutive in the ring slot
                const uint32_t idesc16 = idesc_bf16(rows), bhi = b1, blow = b1 + 2u * p.Nout * p.Kin * 2u;
                bool first = true;
                if (p.split > 1) {
                    for (int kk = 0; kk < p.Kin / 16; ++kk) {
                        const uint32_t bo = (uint32_t)(2 * kk) * lbo;
                        const uint32_t c = (uint32_t)(8 * kk);
                        mma_ts_bf16(d, xh + c, sdesc(blow + bo, lbo, 128), idesc16, first ? acc0 : 1u);
                        mma_ts_bf16(d, xl + c, sdesc(bhi + bo, lbo, 128), idesc16, 1);
                        first = false;
                    }
                }
                for (int kk = 0; kk < p.Kin / 16; ++kk) {
                    const uint32_t bo = (uint32_t)(2 * kk) * lbo;
                    mma_ts_bf16(d, xh + (uint32_t)(8 * kk), sdesc(bhi + bo, lbo, 128), idesc16, first ? acc0 : 1u);
                    first = false;
                }
            } else if (ok) {
                // Correction products first, main products last: the tensor core's
                // FP32 accumulation rounds each step toward zero relative to the
                // running sum, so the small terms are added while the sum is small
                // and the large sum sees only Kin/8 accumulation steps.
                bool first = true;
                if (p.split > 1) {
                    for (int kk = 0; kk < p.Kin / 8; ++kk) {
                        const uint32_t bo = (uint32_t)(2 * kk) * lbo;
                        const uint32_t c = (uint32_t)(8 * kk);
                        mma_ts(d, xh + c, sdesc(bl + bo, lbo, 128), idesc, first ? acc0 : 1u);
                        mma_ts(d, xl + c, sdesc(b1 + bo, lbo, 128), idesc, 1);
                        first = false;
                    }
                }
                for (int kk = 0; kk < p.Kin / 8; ++kk) {
                    const uint32_t bo = (uint32_t)(2 * kk) * lbo;
                    mma_ts(d, xh + (uint32_t)(8 * kk), sdesc(b1 + bo, lbo, 128), idesc, first ? acc0 : 1u);
                    first = false;
                }
            }
            if (grp == 1) mma_commit(&s.empty[slot]);   // ring slot and F_lo free once both groups completed
            mma_commit(grp ? s.edone : s.ddone);
        }
    }
    if (it > 0) drain_wait(s.edone, (it - 1) & 1);   // no MMA in flight when tensor memory is freed
}

// One part (0 = real, 1 = imaginary) of the staged input tile -> X and X_lo
// in tensor memory (this thread's RHS lane; the warp's chunks of 8 positions,
// e = 8 (hf + SPLIT c)).  WT is the tile width p.W as a compile-time constant
// (the staged strides).
template <bool BF, int WT, int SPLIT>
__device__ __forceinline__ void convert(const TcParams &p, const unsigned char *xs, uint32_t lb, int mlane, int hf,
                                        int part) {
    const uint32_t ch = part ? kXi : kXr, cl = part ? kXil : kXrl;
    for (int e = 8 * hf; e < p.Kin; e += 8 * SPLIT) {
        float v[8], vl[8];
        if (p.load_kind == LD_POINTS && p.use_tmap) {
            // tile e/16, row mlane (128 B), 16-byte chunk c stored at c ^ (mlane % 8)
            const unsigned char *row = xs + (size_t)(e >> 4) * (WT * 128) + (size_t)mlane * 128;
            const int c0 = (e & 15) >> 1;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 q = *reinterpret_cast<const float4 *>(row + (((c0 + i) ^ (mlane & 7)) << 4));
                v[2 * i] = part ? q.y : q.x;
                v[2 * i + 1] = part ? q.w : q.z;
            }
        } else if (p.load_kind == LD_POINTS) {
            const float4 *row = reinterpret_cast<const float4 *>(xs + (size_t)mlane * kPointRow) + (e >> 1);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 q = row[i];
                v[2 * i] = part ? q.y : q.x;
                v[2 * i + 1] = part ? q.w : q.z;
            }
        } else if (p.load_kind == LD_QUAD) {   // planar positions
            const float *col = reinterpret_cast<const float *>(xs) + (size_t)e * 2 * WT + part * WT + mlane;
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = col[i * 2 * WT];
        } else {   // quads of positions: this lane's 4 consecutive values are one 16-byte load
            const float4 *q4 = reinterpret_cast<const float4 *>(xs) + (size_t)(e >> 2) * 2 * WT + part * WT + mlane;
            const float4 a = q4[0], b = q4[2 * WT];
            v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
            v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
        }
        if (BF) {   // BF16 pairs: element e + 2i in the low half of column (e / 2) + i
            uint32_t h[4], m[4], l[4];
            if (p.split == 6) {
                split3_bf16x8(v, h, m, l);
                tmem_st4(lb + ch + 32 + (uint32_t)(e >> 1), m);   // X_mid 32 columns after X_hi
            } else if (p.split == 3) {
                split_bf16x8(v, h, l);
            } else {
                round_bf16x8(v, h);
            }
            tmem_st4(lb + ch + (uint32_t)(e >> 1), h);
            if (p.split > 1) tmem_st4(lb + cl + (uint32_t)(e >> 1), l);
            continue;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float hi = tf32_round(v[i]);
            vl[i] = v[i] - hi;
            v[i] = hi;
        }
        tmem_st8(lb + ch + (uint32_t)e, v);
        if (p.split > 1) tmem_st8(lb + cl + (uint32_t)e, vl);
    }
    tmem_wait_st();
}

// Accumulator registers of one thread: the outputs of its warp's chunks
// o = 8 (hf + SPLIT c) < Nout, eight per chunk.
template <int SPLIT>
struct Acc {
    static constexpr int chunks = 64 / 8 / SPLIT;
    float re[chunks][8], im[chunks][8];
};

// D of the item -> registers (D[:, o] into re, D[:, Nout+o] into im).
template <int SPLIT>
__device__ __forceinline__ void read_d(const TcParams &p, uint32_t lb, int hf, Acc<SPLIT> &a) {
#pragma unroll
    for (int c = 0; c < Acc<SPLIT>::chunks; ++c) {
        const int o = 8 * (hf + SPLIT * c);
        if (o < p.Nout) tmem_ld8x2(lb + kD + (uint32_t)o, lb + kD + (uint32_t)(p.Nout + o), a.re[c], a.im[c]);
    }
}

// Stores 8 consecutive outputs of this thread's RHS row (ST_POINTS) through
// the warp's transpose tile: each lane writes its 64-byte row segment, then
// each store instruction writes eight rows' 64-byte segments (whole sectors).
// The tile's 16-byte chunks are XOR-swizzled so both phases are conflict-free.
template <int WT>
__device__ __forceinline__ void store_points8(const TcParams &p, const Smem &s, const Item &w, int q, int o,
                                              const float (&re)[8], const float (&im)[8]) {
    const int lane = threadIdx.x & 31;
    float4 *tr = s.tr + (size_t)(threadIdx.x >> 5) * (kTrBytes / 16);
    const int sw = (lane >> 1) & 3;
#pragma unroll
    for (int c = 0; c < 4; ++c) tr[lane * 4 + (c ^ sw)] = make_float4(re[2 * c], im[2 * c], re[2 * c + 1], im[2 * c + 1]);
    __syncwarp();
    const int j = o / p.n0, pt = o - j * p.n0;
    const long long col = ((long long)w.n * p.m + slot_of(p, w.g, j)) * p.n0 + pt;   // first of the 8 points
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        const int row = 8 * st + (lane >> 2), c = lane & 3;
        const float4 v = tr[row * 4 + (c ^ ((row >> 1) & 3))];
        if (q * 32 + row < w.nt)
            *reinterpret_cast<float4 *>(p.out + (long long)(w.t * WT + q * 32 + row) * p.ld_out + col + 2 * c) = v;
    }
    __syncwarp();
}

// E of the item combined with its D (registers): Re Y = D[:, o] - E[:, Nout+o],
// Im Y = D[:, Nout+o] + E[:, o], in place.  After this the E columns are free.
template <int SPLIT>
__device__ __forceinline__ void combine_e(const TcParams &p, uint32_t lb, int hf, Acc<SPLIT> &a) {
#pragma unroll
    for (int c = 0; c < Acc<SPLIT>::chunks; ++c) {
        const int o = 8 * (hf + SPLIT * c);
        if (o >= p.Nout) continue;
        float er[8], ei[8];
        tmem_ld8x2(lb + kE + (uint32_t)o, lb + kE + (uint32_t)(p.Nout + o), er, ei);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            a.re[c][i] -= ei[i];
            a.im[c][i] += er[i];
        }
    }
}

// The item's outputs (combined, in registers) stored.
template <int WT, int SPLIT>
__device__ __forceinline__ void store_out(const TcParams &p, const Smem &s, const Item &w, int q, int mlane, int hf,
                                          const Acc<SPLIT> &a) {
    const bool live = mlane < w.nt;
#pragma unroll
    for (int c = 0; c < Acc<SPLIT>::chunks; ++c) {
        const int o = 8 * (hf + SPLIT * c);
        if (o >= p.Nout) continue;
        const float(&re)[8] = a.re[c];
        const float(&im)[8] = a.im[c];
        if (p.store_kind == ST_POINTS) {
            store_points8<WT>(p, s, w, q, o, re, im);
        } else if (p.store_kind == ST_QUAD) {
            if (live) {
                const long long base = quad_out_base(p, w);
                constexpr int W2 = 2 * WT;
                float *dst = reinterpret_cast<float *>(p.out) + (long long)w.t * p.R * W2 + mlane;
                const int oo0 = w.part * p.Nout + o;
                if ((p.q_bszo & 7) == 0) {   // the 8 outputs lie in one block: one index computation
                    const int c = oo0 / p.q_bszo;
                    const long long pos0 = (base + c * p.q_sout) * p.q_bszo + (oo0 - c * p.q_bszo);
                    float *d0 = dst + pos0 * W2;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        d0[i * W2] = re[i];
                        d0[i * W2 + WT] = im[i];
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int oo = oo0 + i, c = oo / p.q_bszo;
                        const long long pos = (base + c * p.q_sout) * p.q_bszo + (oo - c * p.q_bszo);
                        dst[pos * W2] = re[i];
                        dst[pos * W2 + WT] = im[i];
                    }
                }
            }
        } else if (live) {
            const int j = o / p.r, kk = o - j * p.r;
            const int ps = slot_of(p, w.g, j);
            const int blk = p.store_kind == ST_LOGICAL ? bitrev(ps, p.h) : ps;
            // quads of positions (kk is a multiple of 8): four 16-byte stores
            const long long pos = (long long)w.t * p.R + ((long long)w.n * p.m + blk) * p.r + kk;
            float4 *dst = reinterpret_cast<float4 *>(p.out) + (pos >> 2) * 2 * WT + mlane;
            dst[0] = make_float4(re[0], re[1], re[2], re[3]);
            dst[WT] = make_float4(im[0], im[1], im[2], im[3]);
            dst[2 * WT] = make_float4(re[4], re[5], re[6], re[7]);
            dst[3 * WT] = make_float4(im[4], im[5], im[6], im[7]);
        }
    }
}

// Epilogue warps, per item i (WT = p.W): D of item i-1 into registers; the
// real half of item i's tile into tensor memory (D(i) may start); E of item
// i-1 combined into the registers; the imaginary half (E(i) may start, and
// the staging buffer is released); then item i-1's outputs stored.  The
// stores come last so that the E chain (E(i-1) done -> E(i) issued) holds
// only the combine and the conversion, and the next tile's copy overlaps
// them.
template <bool BF, int WT, int EPI>
__device__ __forceinline__ void epilogue(const TcParams &p, const Smem &s, uint32_t tmem, int ntiles, int nitems) {
    constexpr int SPLIT = Epi<EPI>::split;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int q = warp & 3, hf = warp >> 2;
    const int mlane = q * 32 + (tid & 31);
    const uint32_t lb = tmem + ((uint32_t)(q * 32) << 16);
    const uint32_t nb = (uint32_t)nbufs(p);
    // Warps whose lane quarter lies beyond the tile width only keep the
    // barrier count: their tensor-memory rows are never read out.
    const bool active = q * 32 < WT;
    uint32_t it = 0;
    Item prev{};
    Acc<SPLIT> acc;
    for (int sub = 0; sub_item(p, sub) < nitems; ++sub, ++it) {
        const Item w = decode(p, sub_item(p, sub), chunk_of(p, sub), ntiles);
        bool okd = false;
        if (it > 0) {   // item it-1: D -> registers (its E group is running) once its last K-chunk is in
            okd = warp_wait(s.ddone, (it - 1) & 1, s.abort_flag, p.err);
            tc_fence_after();
            if (okd && prev.last && active) read_d(p, lb, hf, acc);
        }
        const uint32_t xb = it % nb;
        const unsigned char *xs = s.xs + xb * kHalfStage;
        const bool okx = warp_wait(&s.xfull[xb], (it / nb) & 1, s.abort_flag, p.err);
        if (okx && active) convert<BF, WT, SPLIT>(p, xs, lb, mlane, hf, 0);
        tc_fence_before();
        warp_arrive(s.xrready);
        bool oke = false;
        if (it > 0) {   // item it-1: E combined (item it's D group is running)
            oke = warp_wait(s.edone, (it - 1) & 1, s.abort_flag, p.err);
            tc_fence_after();
            if (okd && oke && prev.last && active) combine_e(p, lb, hf, acc);
        }
        if (okx && active) convert<BF, WT, SPLIT>(p, xs, lb, mlane, hf, 1);
        tc_fence_before();
        warp_arrive(s.xiready);
        warp_arrive(&s.xfree[xb]);
        if (okd && oke && prev.last && active) store_out<WT, SPLIT>(p, s, prev, q, mlane, hf, acc);   // item it-1's outputs
        prev = w;
    }
    if (it > 0) {
        const bool okd = warp_wait(s.ddone, (it - 1) & 1, s.abort_flag, p.err);
        tc_fence_after();
        if (okd && active) read_d(p, lb, hf, acc);
        const bool oke = warp_wait(s.edone, (it - 1) & 1, s.abort_flag, p.err);
        tc_fence_after();
        if (okd && oke && active) {
            combine_e(p, lb, hf, acc);
            store_out<WT, SPLIT>(p, s, prev, q, mlane, hf, acc);
        }
    }
}

// The blocks of one tensor-core pass split for a BF16 rung, once per plan
// and rung: block b's FP32 [Re F; Im F] (rows = 2 Nout, the layout of boff)
// becomes its `parts` BF16 parts (hi; hi, lo; or hi, mid, lo), each in the
// 8-element core-row layout the MMAs read, so the kernel streams them as
// they are.  One 16-byte chunk (8 values of one row) of every part per
// thread; chunk c of a part is K chunk c / rows of row c % rows, whose 8
// values are the FP32 layout's chunks 2 kc rows + n and (2 kc + 1) rows + n.
__global__ void bf16_split_kernel(const float *fac, uint4 *out, long long nblocks, int rows, int Kin, int parts) {
    const long long per = (long long)rows * Kin / 8;
    const long long total = nblocks * per;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / per;
        const int c = (int)(i - b * per);
        const int kc = c / rows, n = c - kc * rows;
        const float4 *src = reinterpret_cast<const float4 *>(fac + b * rows * Kin);
        const float4 x = src[(2 * kc) * rows + n], y = src[(2 * kc + 1) * rows + n];
        const float v[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
        uint4 *dst = out + b * per * parts + c;
        uint32_t h[4], m[4], l[4];
        if (parts == 3) {
            split3_bf16x8(v, h, m, l);
            dst[per] = make_uint4(m[0], m[1], m[2], m[3]);
            dst[2 * per] = make_uint4(l[0], l[1], l[2], l[3]);
        } else if (parts == 2) {
            split_bf16x8(v, h, l);
            dst[per] = make_uint4(l[0], l[1], l[2], l[3]);
        } else {
            round_bf16x8(v, h);
        }
        dst[0] = make_uint4(h[0], h[1], h[2], h[3]);
    }
}

// BF: the BF16 rungs (p.bf16 = 1) or the TF32 rungs, one instantiation each.
template <bool BF, int EPI>
__global__ void __launch_bounds__(Epi<EPI>::threads, 1) bf_tc_kernel(const __grid_constant__ TcParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Smem s;
    s.ring = reinterpret_cast<float *>(smem_raw);
    s.blo = s.ring + (size_t)kStages * (kSlotBytes / 4);
    s.xs = reinterpret_cast<unsigned char *>(s.blo + (size_t)kStages * (kSlotBytes / 4));
    s.tr = reinterpret_cast<float4 *>(s.xs + kStageBytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(s.xs + kStageBytes + EPI * kTrBytes);
    s.full = bars;
    s.empty = bars + kStages;
    s.bready = bars + 2 * kStages;
    s.xfull = bars + 3 * kStages;
    s.xfree = s.xfull + 2;
    s.xrready = s.xfull + 4;
    s.xiready = s.xfull + 5;
    s.ddone = s.xfull + 6;
    s.edone = s.xfull + 7;
    s.tmem_slot = reinterpret_cast<uint32_t *>(s.xfull + 8);
    s.abort_flag = reinterpret_cast<volatile int *>(s.tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            bfk::mbar_init(&s.full[i], 1);
            bfk::mbar_init(&s.empty[i], 1);
            bfk::mbar_init(&s.bready[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            bfk::mbar_init(&s.xfull[b], 1);
            bfk::mbar_init(&s.xfree[b], EPI);
        }
        bfk::mbar_init(s.xrready, EPI);
        bfk::mbar_init(s.xiready, EPI);
        bfk::mbar_init(s.ddone, 1);
        bfk::mbar_init(s.edone, 1);
        *s.abort_flag = 0;
        bfk::fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         bfk::smem_u32(s.tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s.tmem_slot;
    const int ntiles = (p.nrhs + p.W - 1) / p.W;
    const int nitems = nwork(p, ntiles);
    if (warp == Epi<EPI>::prod_warp) {
        producer<BF>(p, s, ntiles, nitems);
    } else if (warp == Epi<EPI>::prep_warp) {
        prep<BF>(p, s, nitems);
    } else if (warp == Epi<EPI>::mma_warp) {
        if ((tid & 31) == 0) mma_issuer<BF>(p, s, tmem, nitems);
    } else if (EPI == 16) {   // tiles of 32, 64 or 96 RHS
        if (p.W == 32)
            epilogue<BF, 32, EPI>(p, s, tmem, ntiles, nitems);
        else if (p.W == 64)
            epilogue<BF, 64, EPI>(p, s, tmem, ntiles, nitems);
        else
            epilogue<BF, 96, EPI>(p, s, tmem, ntiles, nitems);
    } else {                  // 128-RHS tiles
        epilogue<BF, NR, EPI>(p, s, tmem, ntiles, nitems);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace bftc
