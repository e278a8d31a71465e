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
// 128 RHS at a time:  Y = F X with F of Nout x Kin (Nout, Kin <= 64).
//
// Tensor-core mapping.  The RHS sit on the MMA M dimension (M = 128): the
// activation tile X (128 RHS x Kin) is the A operand, read from tensor
// memory, and the block F is the B operand, streamed by TMA into shared
// memory as one K-major operand [Re F; Im F] of 2 Nout rows.  Two real
// accumulators
//     D = Re X [Re F; Im F]^T,   E = Im X [Re F; Im F]^T
// give Re Y = D[:, o] - E[:, Nout+o] and Im Y = D[:, Nout+o] + E[:, o]; the
// epilogue combines them, so no rearranged copy of F is needed.  Each MMA is
// 128 x 2 Nout x 8 (kind::tf32, FP32 accumulation).  FP32 accuracy comes from
// the 3xTF32 split: the tensor core truncates FP32 operands to TF32, so with
// x_lo = x - trunc(x) every product is formed as a b + a b_lo + a_lo b (the
// dropped a_lo b_lo is ~2^-22 relative).  X_lo lives next to X in tensor
// memory; F_lo is built in shared memory by one warp per streamed block.
//
// Tensor memory (512 columns): Re X | Im X | Re X_lo | Im X_lo (64 each) |
// D (128) | E (128).
//
// Warp roles (one persistent CTA per SM, looping over work items
// (node, group, 128-RHS tile)):
//  * producer warp: TMA bulk copies of each item's block F into a two-slot
//    ring and of the item's input tile into a shared-memory staging buffer
//    (one copy per slot for pass intermediates, one per RHS row for the
//    input vectors), so HBM reads for item i+1 overlap item i's MMAs;
//  * prep warp: F_lo for each ring slot;
//  * MMA warp: one thread issues the item's 6 Kin/8 MMAs and commits them;
//  * eight epilogue warps (two per tensor-memory lane quarter): read item
//    i-1's accumulators, combine and store its outputs to global memory,
//    then convert item i's staged tile into X and X_lo in tensor memory.
// They meet on mbarriers; every wait is bounded (bf_kernels.cuh), and on
// expiry the CTA runs its remaining control flow without waiting or
// computing and the producer drains the copies it issued.
#pragma once

#include "bf_kernels.cuh"

namespace bftc {

constexpr int NR = 128;                  // RHS per work item = MMA M
constexpr int kEpiWarps = 8;
constexpr int kMmaWarp = kEpiWarps;
constexpr int kProdWarp = kEpiWarps + 1;
constexpr int kPrepWarp = kEpiWarps + 2;
constexpr int kThreads = (kEpiWarps + 3) * 32;
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxDim = 64;              // Kin, Nout (complex) per block
constexpr uint32_t kXr = 0, kXi = 64, kXrl = 128, kXil = 192, kD = 256, kE = 384;
constexpr int kStages = 2;
constexpr uint32_t kSlotBytes = 2u * kMaxDim * kMaxDim * 4u;                  // 32 KB
constexpr uint32_t kPointRow = kMaxDim * 8u + 16u;                           // padded staging row
constexpr uint32_t kStageBytes = (uint32_t)NR * kPointRow;                   // >= Kin * NR * 8
constexpr size_t kSmemBytes = 2ull * kStages * kSlotBytes + kStageBytes + 256;

enum LoadKind : int { LD_POINTS = 0, LD_SLOTS = 1, LD_GATHER = 2 };
enum StoreKind : int { ST_SLOTS = 0, ST_LOGICAL = 1, ST_POINTS = 2 };

struct TcParams {
    const float *fac;       // per (node, group): [Re F; Im F], 2 Nout x Kin, K-major no-swizzle
    const float2 *in;       // LD_POINTS: vectors, RHS j at in + j ld_in; else tiles [t][R][128]
    long long ld_in;
    float2 *out;            // ST_POINTS: vectors, RHS j at out + j ld_out; else tiles [t][R][128]
    long long ld_out;
    long long R;            // positions per RHS in an intermediate (2^L r)
    unsigned *err;
    int load_kind, store_kind;
    int m, r, n0, h;
    int a, kb, G, ngroups;  // the group's slots differ in node-slot bits a .. a+kb-1
    int Kin, Nout;
    int nrhs;
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
// Four 32x32b.x8 tensor-memory loads and their wait in one asm statement, so
// no register is read before the data has arrived.
__device__ __forceinline__ void tmem_ld8x4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, float (&v0)[8],
                                           float (&v1)[8], float (&v2)[8], float (&v3)[8]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%33];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%34];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%35];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        v0[i] = __uint_as_float(r[i]);
        v1[i] = __uint_as_float(r[8 + i]);
        v2[i] = __uint_as_float(r[16 + i]);
        v3[i] = __uint_as_float(r[24 + i]);
    }
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// Part of x below the TF32 mantissa (the tensor core truncates the low 13 bits).
__device__ __forceinline__ float lo_part(float x) { return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

struct Smem {
    float *ring, *blo;                 // kStages slots of kSlotBytes each
    unsigned char *xs;                 // input staging
    uint64_t *full, *empty, *bready;   // [kStages]
    uint64_t *xfull, *xfree, *xready, *dfull;
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
};
__device__ __forceinline__ Item decode(const TcParams &p, int item, int ntiles) {
    Item it;
    it.t = item % ntiles;
    const int ng = item / ntiles;
    it.n = ng / p.ngroups;
    it.g = ng - it.n * p.ngroups;
    it.nt = min(NR, p.nrhs - it.t * NR);
    return it;
}

// Position (in the intermediate) of the first entry of local slot j's r-block.
__device__ __forceinline__ long long slot_pos(const TcParams &p, const Item &it, int j) {
    const int ps = slot_of(p, it.g, j);
    if (p.load_kind == LD_GATHER) return ((long long)bitrev(ps, p.h) * p.m + it.n) * p.r;   // M^h: block q of row node n
    return ((long long)it.n * p.m + ps) * p.r;
}

// Bounded wait that ignores the abort flag (drains before exit).
__device__ __forceinline__ void drain_wait(uint64_t *bar, uint32_t parity) {
    if (bfk::mbar_try_wait(bar, parity)) return;
    const unsigned long long t0 = bfk::globaltimer();
    while (!bfk::mbar_try_wait(bar, parity) && bfk::globaltimer() - t0 < bfk::kWaitNs) {
    }
}

// Producer warp: the item's block F into ring slot (it % kStages), then its
// input tile into the staging buffer once the epilogue warps have converted
// the previous one.
__device__ __forceinline__ void producer(const TcParams &p, const Smem &s, int ntiles, int nitems) {
    const int lane = threadIdx.x & 31;
    const uint32_t ubytes = 2u * p.Nout * p.Kin * 4u;
    uint32_t nf = 0, nx = 0;   // factor copies / staging groups issued
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const Item w = decode(p, item, ntiles);
        const long long ng = (long long)w.n * p.ngroups + w.g;
        const uint32_t slot = nf % kStages, use = nf / kStages;
        bool ok = true;
        if (lane == 0) {
            ok = !*s.abort_flag && (use == 0 || bfk::mbar_wait(&s.empty[slot], (use - 1) & 1, s.abort_flag, p.err));
            if (ok) {
                bfk::mbar_arrive_expect_tx(&s.full[slot], ubytes);
                bfk::bulk_g2s(s.ring + (size_t)slot * (kSlotBytes / 4), p.fac + ng * (2ll * p.Nout * p.Kin), ubytes,
                              &s.full[slot]);
            }
        }
        if (__shfl_sync(0xffffffffu, ok ? 1 : 0, 0) == 0) break;
        ++nf;
        if (nx > 0 && !warp_wait(s.xfree, (nx - 1) & 1, s.abort_flag, p.err)) break;
        if (p.load_kind == LD_POINTS) {
            const uint32_t rowb = (uint32_t)p.Kin * 8u;
            if (lane == 0) bfk::mbar_arrive_expect_tx(s.xfull, rowb * (uint32_t)w.nt);
            __syncwarp();
            const float2 *src = p.in + (long long)(w.t * NR) * p.ld_in + ((long long)w.n * p.m + slot_of(p, w.g, 0)) * p.n0;
            for (int row = lane; row < w.nt; row += 32)
                bfk::bulk_g2s(s.xs + (size_t)row * kPointRow, src + (long long)row * p.ld_in, rowb, s.xfull);
        } else {
            const uint32_t slotb = (uint32_t)p.r * NR * 8u;
            if (lane == 0) bfk::mbar_arrive_expect_tx(s.xfull, slotb * (uint32_t)p.G);
            __syncwarp();
            for (int j = lane; j < p.G; j += 32)
                bfk::bulk_g2s(s.xs + (size_t)j * slotb, p.in + ((long long)w.t * p.R + slot_pos(p, w, j)) * NR, slotb,
                              s.xfull);
        }
        ++nx;
    }
    // Every copy issued must land before the CTA may exit.
    if (lane == 0) {
        for (uint32_t k = nf > (uint32_t)kStages ? nf - kStages : 0; k < nf; ++k)
            drain_wait(&s.full[k % kStages], (k / kStages) & 1);
        if (nx > 0) drain_wait(s.xfull, (nx - 1) & 1);
    }
}

// Prep warp: F_lo of each streamed block, in the same operand layout.
__device__ __forceinline__ void prep(const TcParams &p, const Smem &s, int nitems) {
    const int lane = threadIdx.x & 31;
    const int n4 = 2 * p.Nout * p.Kin / 4;
    uint32_t it = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
        const uint32_t slot = it % kStages;
        if (warp_wait(&s.full[slot], (it / kStages) & 1, s.abort_flag, p.err)) {
            const float4 *src = reinterpret_cast<const float4 *>(s.ring + (size_t)slot * (kSlotBytes / 4));
            float4 *dst = reinterpret_cast<float4 *>(s.blo + (size_t)slot * (kSlotBytes / 4));
            for (int i = lane; i < n4; i += 32) {
                const float4 v = src[i];
                dst[i] = make_float4(lo_part(v.x), lo_part(v.y), lo_part(v.z), lo_part(v.w));
            }
            fence_async_smem();
        }
        warp_arrive(&s.bready[slot]);
    }
}

// MMA warp (one thread): the item's 6 Kin/8 MMAs into D and E.
__device__ __forceinline__ void mma_issuer(const TcParams &p, const Smem &s, uint32_t tmem, int nitems) {
    const int rows = 2 * p.Nout;
    const uint32_t lbo = (uint32_t)(rows >> 3) * 128u;
    const uint32_t idesc = idesc_tf32(rows);
    const uint32_t d = tmem + kD, e = tmem + kE;
    uint32_t it = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
        const uint32_t slot = it % kStages;
        bool ok = !*s.abort_flag && bfk::mbar_wait(s.xready, it & 1, s.abort_flag, p.err);
        ok = ok && bfk::mbar_wait(&s.bready[slot], (it / kStages) & 1, s.abort_flag, p.err);
        tc_fence_after();
        if (ok) {
            const uint32_t b1 = bfk::smem_u32(s.ring) + slot * kSlotBytes;
            const uint32_t bl = bfk::smem_u32(s.blo) + slot * kSlotBytes;
            for (int kk = 0; kk < p.Kin / 8; ++kk) {
                const uint32_t bo = (uint32_t)(2 * kk) * lbo;
                const uint64_t B = sdesc(b1 + bo, lbo, 128), Bl = sdesc(bl + bo, lbo, 128);
                const uint32_t c = (uint32_t)(8 * kk);
                const uint32_t acc = kk > 0 ? 1u : 0u;
                mma_ts(d, tmem + kXr + c, B, idesc, acc);
                mma_ts(d, tmem + kXr + c, Bl, idesc, 1);
                mma_ts(d, tmem + kXrl + c, B, idesc, 1);
                mma_ts(e, tmem + kXi + c, B, idesc, acc);
                mma_ts(e, tmem + kXi + c, Bl, idesc, 1);
                mma_ts(e, tmem + kXil + c, B, idesc, 1);
            }
        }
        mma_commit(&s.empty[slot]);   // ring slot and F_lo free once these MMAs completed
        mma_commit(s.dfull);
    }
    if (it > 0) drain_wait(s.dfull, (it - 1) & 1);   // no MMA in flight when tensor memory is freed
}

// Staged input tile -> X and X_lo in tensor memory (this thread's RHS lane,
// positions of its half).
__device__ __forceinline__ void convert(const TcParams &p, const Smem &s, uint32_t lb, int mlane, int hf) {
    const int half = p.Kin >> 1;
    for (int e = hf * half; e < (hf + 1) * half; e += 8) {
        float re[8], im[8], rl[8], il[8];
        if (p.load_kind == LD_POINTS) {
            const float4 *row = reinterpret_cast<const float4 *>(s.xs + (size_t)mlane * kPointRow) + (e >> 1);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 v = row[i];
                re[2 * i] = v.x;
                im[2 * i] = v.y;
                re[2 * i + 1] = v.z;
                im[2 * i + 1] = v.w;
            }
        } else {
            const float2 *col = reinterpret_cast<const float2 *>(s.xs) + (size_t)e * NR + mlane;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float2 v = col[(size_t)i * NR];
                re[i] = v.x;
                im[i] = v.y;
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            rl[i] = lo_part(re[i]);
            il[i] = lo_part(im[i]);
        }
        tmem_st8(lb + kXr + (uint32_t)e, re);
        tmem_st8(lb + kXi + (uint32_t)e, im);
        tmem_st8(lb + kXrl + (uint32_t)e, rl);
        tmem_st8(lb + kXil + (uint32_t)e, il);
    }
    tmem_wait_st();
}

// Item's accumulators -> outputs (this thread's RHS lane, outputs of its half).
__device__ __forceinline__ void epilogue(const TcParams &p, const Item &w, uint32_t lb, int mlane, int hf) {
    const int half = p.Nout >> 1;
    const bool live = mlane < w.nt;
    for (int o = hf * half; o < (hf + 1) * half; o += 8) {
        float dr[8], di[8], er[8], ei[8];
        tmem_ld8x4(lb + kD + (uint32_t)o, lb + kD + (uint32_t)(p.Nout + o), lb + kE + (uint32_t)o,
                   lb + kE + (uint32_t)(p.Nout + o), dr, di, er, ei);
        if (!live) continue;
        float re[8], im[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            re[i] = dr[i] - ei[i];
            im[i] = di[i] + er[i];
        }
        if (p.store_kind == ST_POINTS) {
            const int j = o / p.n0, pt = o - j * p.n0;
            float4 *dst = reinterpret_cast<float4 *>(p.out + (long long)(w.t * NR + mlane) * p.ld_out +
                                                     ((long long)w.n * p.m + slot_of(p, w.g, j)) * p.n0 + pt);
#pragma unroll
            for (int i = 0; i < 4; ++i) dst[i] = make_float4(re[2 * i], im[2 * i], re[2 * i + 1], im[2 * i + 1]);
        } else {
            const int j = o / p.r, kk = o - j * p.r;
            const int ps = slot_of(p, w.g, j);
            const int blk = p.store_kind == ST_LOGICAL ? bitrev(ps, p.h) : ps;
            float2 *dst = p.out + ((long long)w.t * p.R + ((long long)w.n * p.m + blk) * p.r + kk) * NR + mlane;
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[(size_t)i * NR] = make_float2(re[i], im[i]);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1) bf_tc_kernel(const TcParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    Smem s;
    s.ring = reinterpret_cast<float *>(smem_raw);
    s.blo = s.ring + (size_t)kStages * (kSlotBytes / 4);
    s.xs = reinterpret_cast<unsigned char *>(s.blo + (size_t)kStages * (kSlotBytes / 4));
    uint64_t *bars = reinterpret_cast<uint64_t *>(s.xs + kStageBytes);
    s.full = bars;
    s.empty = bars + kStages;
    s.bready = bars + 2 * kStages;
    s.xfull = bars + 3 * kStages;
    s.xfree = s.xfull + 1;
    s.xready = s.xfull + 2;
    s.dfull = s.xfull + 3;
    s.tmem_slot = reinterpret_cast<uint32_t *>(s.xfull + 4);
    s.abort_flag = reinterpret_cast<volatile int *>(s.tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            bfk::mbar_init(&s.full[i], 1);
            bfk::mbar_init(&s.empty[i], 1);
            bfk::mbar_init(&s.bready[i], 1);
        }
        bfk::mbar_init(s.xfull, 1);
        bfk::mbar_init(s.xfree, kEpiWarps);
        bfk::mbar_init(s.xready, kEpiWarps);
        bfk::mbar_init(s.dfull, 1);
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
    const int ntiles = (p.nrhs + NR - 1) / NR;
    const int nitems = p.m * p.ngroups * ntiles;
    if (warp == kProdWarp) {
        producer(p, s, ntiles, nitems);
    } else if (warp == kPrepWarp) {
        prep(p, s, nitems);
    } else if (warp == kMmaWarp) {
        if ((tid & 31) == 0) mma_issuer(p, s, tmem, nitems);
    } else {
        const int q = warp & 3, hf = warp >> 2;
        const int mlane = q * 32 + (tid & 31);
        const uint32_t lb = tmem + ((uint32_t)(q * 32) << 16);
        uint32_t it = 0;
        Item prev{};
        for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++it) {
            if (it > 0) {
                const bool ok = warp_wait(s.dfull, (it - 1) & 1, s.abort_flag, p.err);
                tc_fence_after();
                if (ok) epilogue(p, prev, lb, mlane, hf);
            }
            const Item w = decode(p, item, ntiles);
            if (warp_wait(s.xfull, it & 1, s.abort_flag, p.err)) convert(p, s, lb, mlane, hf);
            tc_fence_before();
            warp_arrive(s.xfree);
            warp_arrive(s.xready);
            prev = w;
        }
        if (it > 0) {
            const bool ok = warp_wait(s.dfull, (it - 1) & 1, s.abort_flag, p.err);
            tc_fence_after();
            if (ok) epilogue(p, prev, lb, mlane, hf);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace bftc
