// Tensor-core (tcgen05) compute core of the multi-RHS path, sm_103a.
//
// Same passes, groups and in-place slot order as bf_wide.cuh, with 128 RHS
// per CTA.  Each unit -- a 2r x 2r butterfly [X_{2n,q}; X_{2n+1,q}] (Eq. RSh2
// and its mirror) or a leaf block, N output rows by K inputs -- is applied
// as Y^T = X^T B^T with the RHS on the MMA M dimension (M = 128):
//     [D_re | D_im] = Xr [Br | Bi]^T + Xi [-Bi | Br]^T
// two real tcgen05.mma kind::tf32 groups with N' = 2N, FP32 accumulation in
// tensor memory.  FP32 accuracy comes from the 3xTF32 split: the tensor core
// truncates FP32 inputs to TF32, so with x_lo = x - trunc(x) every product is
// formed as A B + A B_lo + A_lo B (the dropped A_lo B_lo is ~2^-22 relative).
//
// The activation tile lives in tensor memory, not shared memory: column
// c*P + pos of plane c in {re, re_lo, im, im_lo} holds position pos for the
// 128 RHS (one per lane), and the MMAs read A straight from there.  Shared
// memory holds only the factor units ([Br; Bi] as one canonical K-major
// no-swizzle operand of 2N rows, streamed by TMA) and, per unit, the four B
// operands [Br; Bi], its low part, [-Bi; Br] and its low part.
//
// Warp roles (persistent CTA, one per SM, looping over (node, group, RHS
// tile) items): a producer warp streams factor stages with TMA; one MMA warp
// issues each unit's 24 MMAs (r = 16) from a single thread; eight epilogue
// warps load/store the tile, build the B operands of unit u+1 and read back
// unit u-1's accumulators (tcgen05.ld), splitting them into value and low
// part and writing them over u-1's input positions (tcgen05.st).  They meet
// on mbarriers: bready (B operands built), dfull (MMAs committed), dfree
// (accumulator read back) -- double-buffered -- and tready (tile complete for
// the next level).  All waits are bounded.
#pragma once

#include "bf_wide.cuh"

namespace bftc {

using bfk::Level;
using bfw::WideParams;

constexpr int NR = 128;                 // RHS per CTA = MMA M
constexpr uint32_t kTmemCols = 512;

// byte offset of (row n, col k) in a B operand of `rows` rows (K-major,
// no swizzle): K-adjacent core matrices rows/8*128 B apart (LBO), 8-row
// groups 128 B apart (SBO).
__host__ __device__ inline int boff(int n, int k, int rows) {
    return (k >> 2) * (rows >> 3) * 128 + (n >> 3) * 128 + (n & 7) * 16 + (k & 3) * 4;
}

// Shared memory: ring + 2 B-scratch buffers of 4 operands of 2*nk floats + barriers.
__host__ __device__ inline size_t tc_smem_bytes(int stages, int slot_len, int nk_max) {
    return (size_t)stages * slot_len * 8 + 2ull * 4 * 2 * nk_max * 4 + (2ull * stages + 8) * 8 + 32;
}
constexpr int kEpiWarps = 8;                 // epilogue warps (2 per tensor-memory lane quarter)
constexpr int kTcThreads = (kEpiWarps + 2) * 32;
// Tensor-memory columns: 4 planes of P positions + 2 accumulators of dn columns.
__host__ __device__ inline bool tc_tmem_fits(int P, int dn) { return 4 * P + 2 * dn <= (int)kTmemCols; }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ uint32_t idesc_tf32(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(NR >> 4) << 24);
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
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ float lo_part(float x) { return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Writes 8 positions (value and low part, re and im) of this thread's lane.
__device__ __forceinline__ void tile_put8(uint32_t lane_base, int P, int pos, const float (&re)[8],
                                          const float (&im)[8]) {
    float rl[8], il[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        rl[i] = lo_part(re[i]);
        il[i] = lo_part(im[i]);
    }
    tmem_st8(lane_base + (uint32_t)pos, re);
    tmem_st8(lane_base + (uint32_t)(P + pos), rl);
    tmem_st8(lane_base + (uint32_t)(2 * P + pos), im);
    tmem_st8(lane_base + (uint32_t)(3 * P + pos), il);
}

struct TcSmem {
    float2 *ring;
    float *bs[2];                       // per buffer: B', B'_lo, B'', B''_lo, each 2*nk floats
    uint64_t *full, *empty;             // factor ring: producer <-> epilogue warps
    uint64_t *bready, *dfull, *dfree;   // [2] each: B built / MMAs done / accumulator free
    uint64_t *tready;                   // tile complete (epilogue warps -> MMA warp)
    volatile int *abort_flag;
    uint32_t *tmem_slot;
};

struct TcGeom {
    int P;         // tile positions
    int dn;        // accumulator columns per buffer
    int nk;        // max unit N*K
    uint32_t tmem; // allocation base
};

// Lane 0 of a warp waits on an mbarrier phase; the result is broadcast to the warp.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, unsigned *err) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = !*abort_flag && bfk::mbar_wait(bar, parity, abort_flag, err);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}
__device__ __forceinline__ void warp_arrive(uint64_t *bar) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) bfk::mbar_arrive(bar);
}

// Fills the tile: warp (quarter q, half hf) handles lanes 32q.. and 8-position
// chunks c8 = hf (mod 2); each lane loads its RHS's positions, up to four
// chunks of loads in flight before the tensor-memory stores.
__device__ __forceinline__ void tc_load(const WideParams &p, const TcGeom &G, int n, int g, int rhs0, int nt) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3, hf = warp >> 2;
    const int m = q * 32 + lane;
    const uint32_t lb = G.tmem + ((uint32_t)(q * 32) << 16);
    const bool points = p.load_kind == bfw::LD_POINTS;
    const int npos = points ? p.G * p.n0 : p.G * p.r;
    const int off = points ? p.G * (p.W - p.n0) : 0;
    const int nch = npos / 8;
    // 16-byte loads when every 8-position chunk starts on a 16-byte boundary
    const bool vec16 = ((reinterpret_cast<unsigned long long>(p.in) & 15) == 0) && ((p.ld_in & 1) == 0);
    for (int c0 = hf; c0 < nch; c0 += 8) {
        float re[4][8], im[4][8];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c8 = c0 + 2 * b;
            const int e = c8 * 8;
            if (m < nt && c8 < nch) {
                const float2 *src;
                float w[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) w[i] = 1.f;
                if (points) {
                    src = p.in + ((long long)n * p.m + bfw::slot_of(p, g, 0)) * p.n0 + e;
                } else {
                    const int j = e / p.r, k = e - j * p.r;
                    const int ps = bfw::slot_of(p, g, j);
                    if (p.load_kind == bfw::LD_SLOTS) {
                        src = p.in + ((long long)n * p.m + ps) * p.r + k;
                    } else {
                        const int qq = bfw::bitrev(ps, p.h);
                        const float *ws = p.S + ((long long)n * p.m + qq) * p.r + k;
#pragma unroll
                        for (int i = 0; i < 8; ++i) w[i] = __ldg(ws + i);
                        src = p.in + ((long long)qq * p.m + n) * p.r + k;
                    }
                }
                if (p.in_t) {   // [position][RHS]: the warp's lanes read consecutive RHS
                    const float2 *col = p.in + (long long)(src - p.in) * p.ld_in + rhs0 + m;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float2 v = __ldg(col + (long long)i * p.ld_in);
                        re[b][i] = w[i] * v.x;
                        im[b][i] = w[i] * v.y;
                    }
                    continue;
                }
                src += (long long)(rhs0 + m) * p.ld_in;
                if (vec16) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(src) + i);
                        re[b][2 * i] = w[2 * i] * v.x;
                        im[b][2 * i] = w[2 * i] * v.y;
                        re[b][2 * i + 1] = w[2 * i + 1] * v.z;
                        im[b][2 * i + 1] = w[2 * i + 1] * v.w;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float2 v = __ldg(src + i);
                        re[b][i] = w[i] * v.x;
                        im[b][i] = w[i] * v.y;
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) re[b][i] = im[b][i] = 0.f;
            }
        }
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (c0 + 2 * b < nch) tile_put8(lb, G.P, off + (c0 + 2 * b) * 8, re[b], im[b]);
    }
    tmem_wait_st();
}

__device__ __forceinline__ void tc_store(const WideParams &p, const TcGeom &G, int n, int g, int rhs0, int nt) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3, hf = warp >> 2;
    const int m = q * 32 + lane;
    const uint32_t lb = G.tmem + ((uint32_t)(q * 32) << 16);
    const int npos = p.G * p.r;
    const bool vec16 = ((reinterpret_cast<unsigned long long>(p.out) & 15) == 0) && ((p.ld_out & 1) == 0);
    for (int c8 = hf; c8 < npos / 8; c8 += 2) {
        const int e = c8 * 8;
        float re[8], im[8];
        tmem_ld8(lb + (uint32_t)e, re);
        tmem_ld8(lb + (uint32_t)(2 * G.P + e), im);
        if (m < nt) {
            const int j = e / p.r, k = e - j * p.r;
            const int ps = bfw::slot_of(p, g, j);
            const int blk = p.store_kind == bfw::ST_LOGICAL ? bfw::bitrev(ps, p.h) : ps;
            const long long pos = ((long long)n * p.m + blk) * p.r + k;
            if (p.out_t) {   // [position][RHS]: the warp's lanes write consecutive RHS
                float2 *col = p.out + pos * p.ld_out + rhs0 + m;
#pragma unroll
                for (int i = 0; i < 8; ++i) col[(long long)i * p.ld_out] = make_float2(re[i], im[i]);
                continue;
            }
            float2 *dst = p.out + (long long)(rhs0 + m) * p.ld_out + pos;
            if (vec16) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    reinterpret_cast<float4 *>(dst)[i] = make_float4(re[2 * i], im[2 * i], re[2 * i + 1], im[2 * i + 1]);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) dst[i] = make_float2(re[i], im[i]);
            }
        }
    }
}

// B operands of one unit (N x K; stage holds [Br; Bi] as 2N rows) into buffer b.
__device__ __forceinline__ void tc_prep(const TcSmem &s, int b, const float *bu, int N, int K, int nc) {
    const int rows = 2 * N;
    const int nchunk = rows * K / 4;   // 16-byte chunks: 4 k values of one row
    float *B1 = s.bs[b], *B1l = B1 + rows * K, *B2 = B1l + rows * K, *B2l = B2 + rows * K;
    for (int idx = threadIdx.x; idx < nchunk; idx += nc) {
        // chunk idx <-> (k4, row): offset = k4*(rows/8)*128 + (row/8)*128 + (row%8)*16 bytes
        const int k4 = idx / rows, row = idx - k4 * rows;
        const int o = (k4 * (rows >> 3) * 128 + (row >> 3) * 128 + (row & 7) * 16) >> 2;
        const float4 v = *reinterpret_cast<const float4 *>(bu + o);
        *reinterpret_cast<float4 *>(B1 + o) = v;
        *reinterpret_cast<float4 *>(B1l + o) = make_float4(lo_part(v.x), lo_part(v.y), lo_part(v.z), lo_part(v.w));
        // [-Bi; Br]: row < N takes -(row N + row), row >= N takes row - N
        const int src_row = row < N ? row + N : row - N;
        const int os = (k4 * (rows >> 3) * 128 + (src_row >> 3) * 128 + (src_row & 7) * 16) >> 2;
        float4 w = *reinterpret_cast<const float4 *>(bu + os);
        if (row < N) w = make_float4(-w.x, -w.y, -w.z, -w.w);
        *reinterpret_cast<float4 *>(B2 + o) = w;
        *reinterpret_cast<float4 *>(B2l + o) = make_float4(lo_part(w.x), lo_part(w.y), lo_part(w.z), lo_part(w.w));
    }
    fence_async_smem();
}

struct UnitGeo {
    int pa, pb, half, j0, j1, u;
};

template <int KIND>
__device__ __forceinline__ UnitGeo unit_geo(const WideParams &p, const Level &lv, int u) {
    UnitGeo q;
    q.u = u;
    q.j0 = q.j1 = 0;
    if (KIND == bfk::LEAF_IN) {
        q.pa = p.G * (p.W - p.n0) + u * p.n0;
        q.pb = q.pa;
        q.half = lv.K;
    } else if (KIND == bfk::LEAF_OUT) {
        q.pa = u * p.r;
        q.pb = q.pa;
        q.half = lv.K;
    } else {
        q.j0 = bfw::insert0(u, lv.s);
        q.j1 = q.j0 | (1 << lv.s);
        q.pa = q.j0 * p.r;
        q.pb = q.j1 * p.r;
        q.half = p.r;
    }
    return q;
}

// One thread issues unit u's MMAs into accumulator b and commits them.
__device__ __forceinline__ void tc_issue(const TcSmem &s, const TcGeom &G, int b, const UnitGeo &q, int N, int K) {
    tc_fence_after();
    const int rows = 2 * N;
    const uint32_t lbo = (uint32_t)(rows >> 3) * 128;
    const uint32_t idesc = idesc_tf32(rows);
    const uint32_t d = G.tmem + (uint32_t)(4 * G.P + b * G.dn);
    const uint32_t b1 = bfk::smem_u32(s.bs[b]), plane = (uint32_t)(rows * K * 4);
    for (int kk = 0; kk < (K >> 3); ++kk) {
        const int k = kk * 8;
        const int pos = k < q.half ? q.pa + k : q.pb + (k - q.half);
        const uint32_t bo = (uint32_t)(k >> 2) * lbo;
        const uint64_t B1 = sdesc(b1 + bo, lbo, 128), B1l = sdesc(b1 + plane + bo, lbo, 128);
        const uint64_t B2 = sdesc(b1 + 2 * plane + bo, lbo, 128), B2l = sdesc(b1 + 3 * plane + bo, lbo, 128);
        const uint32_t are = G.tmem + (uint32_t)pos, arl = are + (uint32_t)G.P;
        const uint32_t aim = are + (uint32_t)(2 * G.P), ail = are + (uint32_t)(3 * G.P);
        mma_ts(d, are, B1, idesc, kk == 0 ? 0u : 1u);
        mma_ts(d, are, B1l, idesc, 1);
        mma_ts(d, arl, B1, idesc, 1);
        mma_ts(d, aim, B2, idesc, 1);
        mma_ts(d, aim, B2l, idesc, 1);
        mma_ts(d, ail, B2, idesc, 1);
    }
    mma_commit(&s.dfull[b]);
}

// Reads unit q's accumulator b and writes its N outputs: over its input
// positions in the tile, or (leaf U^L / V^L) to global memory.
template <int KIND>
__device__ __forceinline__ void tc_epilogue(const WideParams &p, const TcGeom &G, int b, const UnitGeo &q, int N,
                                            int n, int g, int rhs0, int nt) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, hf = warp >> 2;
    const int m = quarter * 32 + lane;
    const uint32_t lb = G.tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t d = lb + (uint32_t)(4 * G.P + b * G.dn);
    for (int c0 = hf * 8; c0 < N; c0 += 16) {
        float re[8], im[8];
        tmem_ld8(d + (uint32_t)c0, re);
        tmem_ld8(d + (uint32_t)(N + c0), im);
        if (KIND == bfk::LEAF_OUT) {
            if (m < nt) {
                const int ps = bfw::slot_of(p, g, q.u);
                float2 *dst = p.out + (long long)(rhs0 + m) * p.ld_out + ((long long)n * p.m + ps) * p.n0 + c0;
#pragma unroll
                for (int i = 0; i < 8; ++i) dst[i] = make_float2(re[i], im[i]);
            }
        } else {
            int pos;
            if (KIND == bfk::LEAF_IN) {
                pos = q.u * p.r + c0;
            } else {
                const int o = c0 >= p.r ? 1 : 0;
                pos = (o ? q.j1 : q.j0) * p.r + (c0 - o * p.r);
            }
            tile_put8(lb, G.P, pos, re, im);
        }
    }
    if (KIND != bfk::LEAF_OUT) tmem_wait_st();
    tc_fence_before();
}

// Epilogue warps: all units of one level.  Order: prep(0), then for u >= 1
// prep(u) and the epilogue of u-1, then the epilogue of the last unit; so
// B scratch b is rebuilt only after the MMAs that read it have completed.
template <int KIND>
__device__ __forceinline__ void epi_level(const WideParams &p, const TcSmem &s, const TcGeom &G, const Level &lv,
                                          uint32_t &gs, uint32_t (&dph)[2], int n, int g, int rhs0, int nt, int ne) {
    const int N = lv.rpu, K = lv.K;
    const int nunits = lv.nstages * lv.upb;
    UnitGeo prev{};
    for (int u = 0; u <= nunits; ++u) {
        if (u < nunits) {
            const int st = u / lv.upb, ui = u - st * lv.upb;
            const uint32_t slot = (gs + st) % p.stages, use = (gs + st) / p.stages;
            const int b = u & 1;
            bool ok = true;
            if (ui == 0) ok = warp_wait(&s.full[slot], use & 1, s.abort_flag, p.err);
            if (ok && !*s.abort_flag) {
                const float *bu = reinterpret_cast<const float *>(s.ring + (long long)slot * p.slot_len) +
                                  (long long)ui * 2 * N * K;
                tc_prep(s, b, bu, N, K, ne);
            }
            warp_arrive(&s.bready[b]);
            if (ui == lv.upb - 1) warp_arrive(&s.empty[slot]);
        }
        if (u > 0) {
            const int b = (u - 1) & 1;
            const bool ok = warp_wait(&s.dfull[b], dph[b] & 1, s.abort_flag, p.err);
            ++dph[b];
            tc_fence_after();
            if (ok) tc_epilogue<KIND>(p, G, b, prev, N, n, g, rhs0, nt);
            else tc_fence_before();
            warp_arrive(&s.dfree[b]);
        }
        if (u < nunits) prev = unit_geo<KIND>(p, lv, u);
    }
    gs += lv.nstages;
}

// MMA warp (one thread): all units of one level.
__device__ __forceinline__ void mma_level(const WideParams &p, const TcSmem &s, const TcGeom &G, const Level &lv,
                                          uint32_t &tph, uint32_t (&bph)[2], uint32_t (&issued)[2],
                                          uint32_t (&fph)[2]) {
    const int N = lv.rpu, K = lv.K;
    const int nunits = lv.nstages * lv.upb;
    bool ok = !*s.abort_flag && bfk::mbar_wait(s.tready, tph & 1, s.abort_flag, p.err);
    ++tph;
    for (int u = 0; u < nunits; ++u) {
        const int b = u & 1;
        ok = ok && bfk::mbar_wait(&s.bready[b], bph[b] & 1, s.abort_flag, p.err);
        ++bph[b];
        if (issued[b] > 0) {
            ok = ok && bfk::mbar_wait(&s.dfree[b], fph[b] & 1, s.abort_flag, p.err);
            ++fph[b];
        }
        ++issued[b];
        UnitGeo q;
        switch (lv.kind) {
            case bfk::LEAF_IN: q = unit_geo<bfk::LEAF_IN>(p, lv, u); break;
            case bfk::LEAF_OUT: q = unit_geo<bfk::LEAF_OUT>(p, lv, u); break;
            default: q = unit_geo<bfk::MERGE>(p, lv, u); break;
        }
        if (ok) {
            tc_issue(s, G, b, q, N, K);
        } else {
            mma_commit(&s.dfull[b]);   // keeps the epilogue warps' phases moving
        }
    }
}

// Persistent: each CTA loops over work items (node, group, RHS tile) with
// stride gridDim.x; tensor memory is allocated once and the producer streams
// the factor chunks of the CTA's items back to back.
__global__ void __launch_bounds__(kTcThreads, 1) bf_tc_kernel(const WideParams p, int nk_max, int dn) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int ne = kEpiWarps * 32;
    TcSmem s;
    s.ring = reinterpret_cast<float2 *>(smem_raw);
    float *bsbase = reinterpret_cast<float *>(s.ring + (long long)p.stages * p.slot_len);
    s.bs[0] = bsbase;
    s.bs[1] = bsbase + 4ll * 2 * nk_max;
    s.full = reinterpret_cast<uint64_t *>(bsbase + 2ll * 4 * 2 * nk_max);
    s.empty = s.full + p.stages;
    s.bready = s.empty + p.stages;
    s.dfull = s.bready + 2;
    s.dfree = s.dfull + 2;
    s.tready = s.dfree + 2;
    s.tmem_slot = reinterpret_cast<uint32_t *>(s.tready + 1);
    s.abort_flag = reinterpret_cast<volatile int *>(s.tmem_slot + 1);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < p.stages; ++i) {
            bfk::mbar_init(&s.full[i], 1);
            bfk::mbar_init(&s.empty[i], kEpiWarps);
        }
        for (int b = 0; b < 2; ++b) {
            bfk::mbar_init(&s.bready[b], kEpiWarps);
            bfk::mbar_init(&s.dfull[b], 1);
            bfk::mbar_init(&s.dfree[b], kEpiWarps);
        }
        bfk::mbar_init(s.tready, kEpiWarps);
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
    TcGeom G;
    G.P = p.G * p.W;
    G.dn = dn;
    G.nk = nk_max;
    G.tmem = *s.tmem_slot;
    const int ntiles = (p.nrhs + NR - 1) / NR;
    const int nitems = p.m * p.ngroups * ntiles;
    if (warp == kEpiWarps + 1) {                 // producer
        if ((tid & 31) == 0) {
            uint32_t gs = 0;
            for (int item = blockIdx.x; item < nitems; item += gridDim.x)
                if (!bfk::produce_chunk(p, item / ntiles, gs, s.ring, s.full, s.empty, s.abort_flag)) break;
            bfk::produce_drain(p, gs, s.full, s.abort_flag);
        }
    } else if (warp == kEpiWarps) {              // MMA issuer
        if ((tid & 31) == 0) {
            uint32_t tph = 0, bph[2] = {0, 0}, issued[2] = {0, 0}, fph[2] = {0, 0};
            for (int item = blockIdx.x; item < nitems; item += gridDim.x)
                for (int l = 0; l < p.nlev; ++l) mma_level(p, s, G, p.lev[l], tph, bph, issued, fph);
        }
    } else {                                     // epilogue warps
        uint32_t gs = 0, dph[2] = {0, 0};
        for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
            const int tile = item % ntiles, ng = item / ntiles;
            const int n = ng / p.ngroups;
            const int g = ng - n * p.ngroups;
            const int rhs0 = tile * NR;
            const int nt = min(NR, p.nrhs - rhs0);
            tc_load(p, G, n, g, rhs0, nt);
            tc_fence_before();
            warp_arrive(s.tready);
            for (int l = 0; l < p.nlev; ++l) {
                const Level lv = p.lev[l];
                switch (lv.kind) {
                    case bfk::LEAF_IN: epi_level<bfk::LEAF_IN>(p, s, G, lv, gs, dph, n, g, rhs0, nt, ne); break;
                    case bfk::MERGE: epi_level<bfk::MERGE>(p, s, G, lv, gs, dph, n, g, rhs0, nt, ne); break;
                    case bfk::SPLIT: epi_level<bfk::SPLIT>(p, s, G, lv, gs, dph, n, g, rhs0, nt, ne); break;
                    default: epi_level<bfk::LEAF_OUT>(p, s, G, lv, gs, dph, n, g, rhs0, nt, ne); break;
                }
                if (l + 1 < p.nlev) warp_arrive(s.tready);   // epilogues wrote the tile (wait::st + fence done)
            }
            tc_fence_after();
            if (p.store_kind != bfw::ST_NONE) tc_store(p, G, n, g, rhs0, nt);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(G.tmem), "r"(kTmemCols) : "memory");
}

}  // namespace bftc
