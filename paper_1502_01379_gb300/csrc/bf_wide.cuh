// Multi-RHS ("wide") apply kernels for sm_103a.
//
// The fused kernels of bf_kernels.cuh keep a whole middle-level node's
// segment (m r-blocks) per RHS in shared memory, which limits them to a few
// RHS per CTA.  For batches, each half of the chain is instead run in two
// passes over small groups of r-blocks that hold NR (16..64) RHS each:
//
// The level-l intermediate is kept "in place": a butterfly writes its two
// output r-blocks over its two input r-blocks.  Then, inside one middle-level
// node's segment of m = 2^h r-blocks, the butterflies of merging level t
// (segments of s = 2^t blocks, factor level l = L - t, mirror of Eq. RSh2)
// pair the slots that differ in bit t-1 of the slot index, exactly like the
// stages of a radix-2 FFT, and after all h levels slot p holds logical block
// bitrev_h(p).  So levels 1..k touch only bits 0..k-1 (contiguous groups of
// 2^k slots) and levels k+1..h only bits k..h-1 (groups of 2^(h-k) slots at
// stride 2^k): pass D1 = leaf + levels 1..k, pass D2 = levels k+1..h (and in
// general any split of the h levels into chunks of slot bits a..a+kb-1, one
// pass per chunk).  The up half mirrors this: its first pass gathers the M^h
// block transpose (Eq. KeqUMV) into bit-reversed slots and runs the top
// splitting levels, its last pass runs the lowest levels and the leaf U^L.
//
// Each CTA = (node, group, RHS tile of NR).  Factor units are the same 2r x 2r
// butterflies and leaf blocks as in the fused path, packed per CTA in the
// order this CTA consumes them and streamed by the same TMA producer.  The
// compute core is CUDA-core FP32: a thread owns RB (2 or 1) output rows of a
// unit for 4 RHS, reading the factor rows with one 16-byte shared load and the
// inputs with two 16-byte loads from an XOR-swizzled [position][RHS] tile
// whose quads are split in halves so that each load is contiguous across lanes.
#pragma once

#include "bf_kernels.cuh"

namespace bfw {

using bfk::Level;

enum LoadKind : int { LD_POINTS = 0, LD_SLOTS = 1, LD_GATHER = 2 };
enum StoreKind : int { ST_SLOTS = 0, ST_LOGICAL = 1, ST_NONE = 2 };

struct WideParams {
    const float2 *fac;      // packed factor stream, one chunk per (node, group)
    long long cta_len;
    const float2 *in;
    long long ld_in;
    float2 *out;
    long long ld_out;
    const float *S;         // LD_GATHER: weights (node, q, k)
    unsigned *err;
    int nlev, load_kind, store_kind;
    int m, r, n0, W, h;
    int G;                  // r-block slots per group (2^kb)
    int a, kb;              // the group's slots differ in node-slot bits a .. a+kb-1
    int ngroups;
    int nrhs, stages, slot_len;
    Level lev[bfk::kMaxLevels];   // MERGE / SPLIT: lev.s holds the local slot bit
};

__host__ __device__ inline size_t wide_smem_bytes(int stages, int slot_len, int G, int W, int NR) {
    return (size_t)stages * slot_len * 8 + (size_t)G * W * NR * 8 + 2ull * stages * 8 + 16;
}

// Tile layout: position pos holds NR complex values as two halves of NR/2;
// RHS t = 4 tq + 2 half + i lives at xh(pos, tq, half) + i.  Quads are
// XOR-swizzled by pos so that lanes reading one position at different quads,
// and lanes writing different positions at one quad, hit distinct banks.
template <int NR>
__device__ __forceinline__ int xh(int pos, int tq, int half) {
    constexpr int NQ = NR / 4;
    return pos * NR + half * (NR / 2) + (((tq ^ pos) & (NQ - 1)) << 1);
}
// Node slot of local slot j of group g: bits a..a+kb-1 from j, the others from g.
__device__ __forceinline__ int slot_of(const WideParams &p, int g, int j) {
    return ((g >> p.a) << (p.a + p.kb)) | (j << p.a) | (g & ((1 << p.a) - 1));
}
__device__ __forceinline__ int insert0(int v, int b) { return ((v >> b) << (b + 1)) | (v & ((1 << b) - 1)); }
__device__ __forceinline__ int bitrev(int x, int bits) {
    return bits ? (int)(__brev((unsigned)x) >> (32 - bits)) : 0;
}
__device__ __forceinline__ void cmac(float2 &a, float2 f, float2 x) {
    a.x = fmaf(f.x, x.x, a.x);
    a.x = fmaf(-f.y, x.y, a.x);
    a.y = fmaf(f.x, x.y, a.y);
    a.y = fmaf(f.y, x.x, a.y);
}

struct WideSmem {
    float2 *ring, *X;
    uint64_t *full, *empty;
    volatile int *abort_flag;
};

template <int NR>
__device__ __forceinline__ void put_quad(float2 *X, int pos, int tq, float2 a, float2 b, float2 c, float2 d) {
    *reinterpret_cast<float4 *>(X + xh<NR>(pos, tq, 0)) = make_float4(a.x, a.y, b.x, b.y);
    *reinterpret_cast<float4 *>(X + xh<NR>(pos, tq, 1)) = make_float4(c.x, c.y, d.x, d.y);
}

// Fills the tile: each thread takes tile positions and loads all NR RHS of
// a position (independent global loads, coalesced across threads).
template <int NR>
__device__ __forceinline__ void wide_load(const WideParams &p, float2 *X, int n, int g, int rhs0, int nt, int nc) {
    constexpr int NQ = NR / 4;
    const int tid = threadIdx.x;
    const float2 zero = make_float2(0.f, 0.f);
    const bool points = p.load_kind == LD_POINTS;
    const int npos = points ? p.G * p.n0 : p.G * p.r;
    const int off = points ? p.G * (p.W - p.n0) : 0;
    for (int e = tid; e < npos; e += nc) {
        const float2 *src;
        float w = 1.f;
        if (points) {
            src = p.in + ((long long)n * p.m + slot_of(p, g, 0)) * p.n0 + e;   // a = 0: contiguous
        } else {
            const int j = e / p.r, k = e - j * p.r;
            const int ps = slot_of(p, g, j);
            if (p.load_kind == LD_SLOTS) {
                src = p.in + ((long long)n * p.m + ps) * p.r + k;
            } else {   // M^h: slot ps holds logical block q = bitrev_h(ps) of this row node
                const int q = bitrev(ps, p.h);
                w = __ldg(p.S + ((long long)n * p.m + q) * p.r + k);
                src = p.in + ((long long)q * p.m + n) * p.r + k;
            }
        }
        src += (long long)rhs0 * p.ld_in;
#pragma unroll 4
        for (int tq = 0; tq < NQ; ++tq) {
            float2 v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int t = 4 * tq + i;
                v[i] = t < nt ? __ldg(src + (long long)t * p.ld_in) : zero;
                v[i].x *= w;
                v[i].y *= w;
            }
            put_quad<NR>(X, off + e, tq, v[0], v[1], v[2], v[3]);
        }
    }
}

template <int NR>
__device__ __forceinline__ void wide_store(const WideParams &p, const float2 *X, int n, int g, int rhs0, int nt,
                                           int nc) {
    constexpr int NQ = NR / 4;
    const int tid = threadIdx.x;
    const int npos = p.G * p.r;
    for (int e = tid; e < npos; e += nc) {
        const int j = e / p.r, k = e - j * p.r;
        const int ps = slot_of(p, g, j);
        const int blk = p.store_kind == ST_LOGICAL ? bitrev(ps, p.h) : ps;
        float2 *dst = p.out + (long long)rhs0 * p.ld_out + ((long long)n * p.m + blk) * p.r + k;
#pragma unroll 4
        for (int tq = 0; tq < NQ; ++tq) {
            const float4 a = *reinterpret_cast<const float4 *>(X + xh<NR>(e, tq, 0));
            const float4 b = *reinterpret_cast<const float4 *>(X + xh<NR>(e, tq, 1));
            const float2 v[4] = {make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y),
                                 make_float2(b.z, b.w)};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int t = 4 * tq + i;
                if (t < nt) dst[(long long)t * p.ld_out] = v[i];
            }
        }
    }
}

// One level: all stages; per stage, batches of units computed by all
// consumers, barrier, then written in place.
template <int NR, int KIND, int RB>
__device__ __forceinline__ void wide_level(const WideParams &p, const WideSmem &s, float2 *X, const Level &lv,
                                           uint32_t &gs, int n, int g, int rhs0, int nt, int nc) {
    constexpr int NQ = NR / 4;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int rows = lv.upb * lv.rpu;
    const int tpu = (lv.rpu / RB) * NQ;     // threads per unit (host: tpu <= nc)
    const int upar = max(1, nc / tpu);    // >= 1 so the batch loop always advances
    const int ub = tid / tpu;
    const int item = tid - ub * tpu;
    const int rp = item / NQ, tq = item - rp * NQ;
    const int row0 = rp * RB;
    const int off_in = p.G * (p.W - p.n0);
    for (int st = 0; st < lv.nstages; ++st, ++gs) {
        const uint32_t slot = gs % p.stages;
        const uint32_t use = gs / p.stages;
        const bool ready = !*s.abort_flag && bfk::mbar_wait(&s.full[slot], use & 1, s.abort_flag, p.err);
        const float2 *stg = s.ring + (long long)slot * p.slot_len;
        for (int u0 = 0; u0 < lv.upb; u0 += upar) {
            const int ui = u0 + ub;
            const bool active = ready && ub < upar && ui < lv.upb;
            const int u = st * lv.upb + ui;
            float2 acc[RB][4];
#pragma unroll
            for (int a = 0; a < RB; ++a)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[a][i] = make_float2(0.f, 0.f);
            int j0 = 0, j1 = 0;
            if (active) {
                int pa, pb, half;
                if (KIND == bfk::LEAF_IN) {
                    pa = off_in + u * p.n0;
                    pb = pa;
                    half = lv.K;
                } else if (KIND == bfk::LEAF_OUT) {
                    pa = u * p.r;
                    pb = pa;
                    half = lv.K;
                } else {
                    j0 = insert0(u, lv.s);
                    j1 = j0 | (1 << lv.s);
                    pa = j0 * p.r;
                    pb = j1 * p.r;
                    half = p.r;
                }
                const float2 *f = stg + ui * lv.rpu + row0;
#pragma unroll 4
                for (int k = 0; k < lv.K; ++k) {
                    float2 fr[RB];
                    if (RB == 2) {
                        const float4 v = *reinterpret_cast<const float4 *>(f + k * rows);
                        fr[0] = make_float2(v.x, v.y);
                        fr[RB - 1] = make_float2(v.z, v.w);
                    } else {
                        fr[0] = f[k * rows];
                    }
                    const int pos = k < half ? pa + k : pb + (k - half);
                    const float4 x01 = *reinterpret_cast<const float4 *>(X + xh<NR>(pos, tq, 0));
                    const float4 x23 = *reinterpret_cast<const float4 *>(X + xh<NR>(pos, tq, 1));
                    const float2 xs[4] = {make_float2(x01.x, x01.y), make_float2(x01.z, x01.w),
                                          make_float2(x23.x, x23.y), make_float2(x23.z, x23.w)};
#pragma unroll
                    for (int a = 0; a < RB; ++a)
#pragma unroll
                        for (int i = 0; i < 4; ++i) cmac(acc[a][i], fr[a], xs[i]);
                }
            }
            if (KIND != bfk::LEAF_OUT) bfk::consumer_sync(nc);   // all inputs read before in-place writes
            if (active) {
#pragma unroll
                for (int a = 0; a < RB; ++a) {
                    const int rr = row0 + a;
                    if (KIND == bfk::LEAF_OUT) {
                        const int ps = slot_of(p, g, u);
                        const long long pt = ((long long)n * p.m + ps) * p.n0 + rr;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int t = tq * 4 + i;
                            if (t < nt) p.out[(long long)(rhs0 + t) * p.ld_out + pt] = acc[a][i];
                        }
                    } else {
                        int pos;
                        if (KIND == bfk::LEAF_IN) {
                            pos = u * p.r + rr;
                        } else {
                            const int o = rr >= p.r ? 1 : 0;
                            pos = (o ? j1 : j0) * p.r + (rr - o * p.r);
                        }
                        put_quad<NR>(X, pos, tq, acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) bfk::mbar_arrive(&s.empty[slot]);
    }
}

template <int NR, int KIND>
__device__ __forceinline__ void wide_level_rb(const WideParams &p, const WideSmem &s, float2 *X, const Level &lv,
                                              uint32_t &gs, int n, int g, int rhs0, int nt, int nc) {
    if ((lv.rpu & 1) == 0) wide_level<NR, KIND, 2>(p, s, X, lv, gs, n, g, rhs0, nt, nc);
    else wide_level<NR, KIND, 1>(p, s, X, lv, gs, n, g, rhs0, nt, nc);
}

template <int NR>
__global__ void __launch_bounds__(288, 1) bf_wide_kernel(const WideParams p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nc = blockDim.x - 32;
    WideSmem s;
    s.ring = reinterpret_cast<float2 *>(smem_raw);
    s.X = s.ring + (long long)p.stages * p.slot_len;
    s.full = reinterpret_cast<uint64_t *>(s.X + (long long)p.G * p.W * NR);
    s.empty = s.full + p.stages;
    s.abort_flag = reinterpret_cast<volatile int *>(s.empty + p.stages);
    if (threadIdx.x == 0) {
        for (int i = 0; i < p.stages; ++i) {
            bfk::mbar_init(&s.full[i], 1);
            bfk::mbar_init(&s.empty[i], nc / 32);
        }
        *s.abort_flag = 0;
        bfk::fence_mbar_init();
    }
    __syncthreads();
    const int tid = threadIdx.x;
    const int n = blockIdx.y / p.ngroups;
    const int g = blockIdx.y - n * p.ngroups;
    const int rhs0 = blockIdx.x * NR;
    const int nt = min(NR, p.nrhs - rhs0);
    if (tid >= nc) {
        if (tid == nc) bfk::produce(p, blockIdx.y, s.ring, s.full, s.empty, s.abort_flag);
    } else {
        wide_load<NR>(p, s.X, n, g, rhs0, nt, nc);
        bfk::consumer_sync(nc);
        uint32_t gs = 0;
        for (int l = 0; l < p.nlev; ++l) {
            const Level lv = p.lev[l];
            switch (lv.kind) {
                case bfk::LEAF_IN: wide_level_rb<NR, bfk::LEAF_IN>(p, s, s.X, lv, gs, n, g, rhs0, nt, nc); break;
                case bfk::MERGE: wide_level_rb<NR, bfk::MERGE>(p, s, s.X, lv, gs, n, g, rhs0, nt, nc); break;
                case bfk::SPLIT: wide_level_rb<NR, bfk::SPLIT>(p, s, s.X, lv, gs, n, g, rhs0, nt, nc); break;
                default: wide_level_rb<NR, bfk::LEAF_OUT>(p, s, s.X, lv, gs, n, g, rhs0, nt, nc); break;
            }
            bfk::consumer_sync(nc);
        }
        if (p.store_kind != ST_NONE) wide_store<NR>(p, s.X, n, g, rhs0, nt, nc);
    }
    __syncthreads();
}

}  // namespace bfw
