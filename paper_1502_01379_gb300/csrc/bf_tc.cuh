// Tensor-core (tcgen05) compute core of the multi-RHS path, sm_103a.
//
// Same passes, groups and in-place slot order as bf_wide.cuh, with 128 RHS
// per CTA.  Each unit -- a 2r x 2r butterfly [X_{2n,q}; X_{2n+1,q}] (Eq. RSh2
// and its mirror) or a leaf block -- is applied as Y^T = X^T B^T with the RHS
// on the MMA M dimension (M = 128) and the unit's rows on N:
//     D_re = Xr Br^T - Xi Bi^T,   D_im = Xr Bi^T + Xi Br^T        (per unit)
// four real tcgen05.mma kind::tf32 groups (the minus sign through the
// instruction's A-negate bit), accumulated in FP32 in tensor memory.  FP32
// accuracy comes from the 3xTF32 split: the tensor core truncates its FP32
// inputs to TF32, so with x_lo = x - trunc(x) each product is formed as
// A B + A B_lo + A_lo B (the dropped A_lo B_lo is ~2^-22 relative).  The
// activation tile (two planes, re and im) and the factor units are stored in
// the MMA's canonical K-major no-swizzle layout (8-row x 16-byte core
// matrices) so that descriptors address them in place; per unit the consumer
// warps write A_lo and B_lo into scratch planes, one thread issues the 48
// MMAs (r = 16) and commits them to an mbarrier, and the warps read D back
// with tcgen05.ld and write the outputs over the unit's input slots.
#pragma once

#include "bf_wide.cuh"

namespace bftc {

using bfk::Level;
using bfw::WideParams;

constexpr int NR = 128;   // RHS per CTA = MMA M
constexpr uint32_t kTmemCols = 128;

// byte offset of (row m, position k) in a canonical K-major plane whose
// rows hold `kdim` positions: core matrix (8 rows x 4 positions) = 128 B,
// K-adjacent core matrices 128 B apart (LBO), 8-row groups kdim/4*128 B apart (SBO).
__host__ __device__ inline int aoff(int m, int k, int kdim) {
    return (m >> 3) * (kdim >> 2) * 128 + (k >> 2) * 128 + (m & 7) * 16 + (k & 3) * 4;
}
// byte offset of (row n, col k) in a factor plane of N rows: K-adjacent core
// matrices N/8*128 B apart (LBO), 8-row groups 128 B apart (SBO).
__host__ __device__ inline int boff(int n, int k, int N) {
    return (k >> 2) * (N >> 3) * 128 + (n >> 3) * 128 + (n & 7) * 16 + (k & 3) * 4;
}

__host__ __device__ inline size_t tc_smem_bytes(int stages, int slot_len, int G, int W, int kmax_unit, int nk_max) {
    // ring + tile (2 planes x 128 x G*W) + A_lo (2 x 128 x kmax_unit) + B_lo (2 x nk_max) + barriers
    return (size_t)stages * slot_len * 8 + 2ull * NR * G * W * 4 + 2ull * NR * kmax_unit * 4 + 2ull * nk_max * 4 +
           (2ull * stages + 1) * 8 + 32;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ uint32_t idesc_tf32(int N, bool neg_a) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(NR >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
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
__device__ __forceinline__ float lo_part(float x) { return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

struct TcSmem {
    float2 *ring;
    float *tile_re, *tile_im;   // canonical planes, kdim = G*W positions
    float *alo_re, *alo_im;     // canonical planes, kdim = kmax_unit positions
    float *blo;                 // re plane then im plane of one unit
    uint64_t *full, *empty, *mma_bar;
    uint32_t *tmem_slot;
    volatile int *abort_flag;
};

// Tile load: a warp task is 8 RHS rows x 16 positions; lane -> (row, 4-position chunk).
__device__ __forceinline__ void tc_load(const WideParams &p, const TcSmem &s, int kdim, int n, int g, int rhs0, int nt,
                                        int nc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = nc >> 5;
    const bool points = p.load_kind == bfw::LD_POINTS;
    const int npos = points ? p.G * p.n0 : p.G * p.r;
    const int off = points ? p.G * (p.W - p.n0) : 0;
    const int ntask = (NR / 8) * (npos / 16);
    for (int task = warp; task < ntask; task += nwarps) {
        const int rg = task % (NR / 8), cg = task / (NR / 8);
        const int m = rg * 8 + (lane & 7);
        const int e = cg * 16 + (lane >> 3) * 4;   // first of 4 positions
        float4 re = make_float4(0.f, 0.f, 0.f, 0.f), im = re;
        if (m < nt) {
            const float2 *src;
            float4 w = make_float4(1.f, 1.f, 1.f, 1.f);
            if (points) {
                src = p.in + ((long long)n * p.m + bfw::slot_of(p, g, 0)) * p.n0 + e;
            } else {
                const int j = e / p.r, k = e - j * p.r;
                const int ps = bfw::slot_of(p, g, j);
                if (p.load_kind == bfw::LD_SLOTS) {
                    src = p.in + ((long long)n * p.m + ps) * p.r + k;
                } else {
                    const int q = bfw::bitrev(ps, p.h);
                    w = *reinterpret_cast<const float4 *>(p.S + ((long long)n * p.m + q) * p.r + k);
                    src = p.in + ((long long)q * p.m + n) * p.r + k;
                }
            }
            src += (long long)(rhs0 + m) * p.ld_in;   // complex64: 8-byte accesses whatever ld is
            const float2 a0 = __ldg(src), a1 = __ldg(src + 1), a2 = __ldg(src + 2), a3 = __ldg(src + 3);
            re = make_float4(w.x * a0.x, w.y * a1.x, w.z * a2.x, w.w * a3.x);
            im = make_float4(w.x * a0.y, w.y * a1.y, w.z * a2.y, w.w * a3.y);
        }
        const int o = aoff(m, off + e, kdim) >> 2;
        *reinterpret_cast<float4 *>(s.tile_re + o) = re;
        *reinterpret_cast<float4 *>(s.tile_im + o) = im;
    }
}

__device__ __forceinline__ void tc_store(const WideParams &p, const TcSmem &s, int kdim, int n, int g, int rhs0,
                                         int nt, int nc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = nc >> 5;
    const int npos = p.G * p.r;
    const int ntask = (NR / 8) * (npos / 16);
    for (int task = warp; task < ntask; task += nwarps) {
        const int rg = task % (NR / 8), cg = task / (NR / 8);
        const int m = rg * 8 + (lane & 7);
        const int e = cg * 16 + (lane >> 3) * 4;
        if (m >= nt) continue;
        const int j = e / p.r, k = e - j * p.r;
        const int ps = bfw::slot_of(p, g, j);
        const int blk = p.store_kind == bfw::ST_LOGICAL ? bfw::bitrev(ps, p.h) : ps;
        const int o = aoff(m, e, kdim) >> 2;
        const float4 re = *reinterpret_cast<const float4 *>(s.tile_re + o);
        const float4 im = *reinterpret_cast<const float4 *>(s.tile_im + o);
        float2 *dst = p.out + (long long)(rhs0 + m) * p.ld_out + ((long long)n * p.m + blk) * p.r + k;
        dst[0] = make_float2(re.x, im.x);
        dst[1] = make_float2(re.y, im.y);
        dst[2] = make_float2(re.z, im.z);
        dst[3] = make_float2(re.w, im.w);
    }
}

// One unit: A positions (K of them) are pa.. (first half) and pb.. (second
// half, from position `half` on); factor unit (N x K) at `bu`.
template <int KIND>
__device__ __forceinline__ bool tc_unit(const WideParams &p, const TcSmem &s, int kdim, int kmax_unit, const float *bu,
                                        int N, int K, int pa, int pb, int half, int j0, int j1, int u, int n, int g,
                                        int rhs0, int nt, int nc, uint32_t tmem, uint32_t &mma_phase) {
    const int tid = threadIdx.x;
    // 1. A_lo of the unit's K positions and B_lo of its factor into scratch.
    {
        const int nchunk = K >> 2;   // 4-position chunks
        for (int idx = tid; idx < NR * nchunk; idx += nc) {
            const int m = idx % NR, c = idx / NR;
            const int k = 4 * c;
            const int pos = k < half ? pa + k : pb + (k - half);
            const int src = aoff(m, pos, kdim) >> 2, dst = aoff(m, k, kmax_unit) >> 2;
            const float4 a = *reinterpret_cast<const float4 *>(s.tile_re + src);
            const float4 b = *reinterpret_cast<const float4 *>(s.tile_im + src);
            *reinterpret_cast<float4 *>(s.alo_re + dst) = make_float4(lo_part(a.x), lo_part(a.y), lo_part(a.z), lo_part(a.w));
            *reinterpret_cast<float4 *>(s.alo_im + dst) = make_float4(lo_part(b.x), lo_part(b.y), lo_part(b.z), lo_part(b.w));
        }
        const int nb = 2 * N * K / 4;
        for (int idx = tid; idx < nb; idx += nc) {
            const float4 v = reinterpret_cast<const float4 *>(bu)[idx];
            reinterpret_cast<float4 *>(s.blo)[idx] = make_float4(lo_part(v.x), lo_part(v.y), lo_part(v.z), lo_part(v.w));
        }
    }
    fence_async_smem();
    bfk::consumer_sync(nc);
    // After the barrier every consumer sees the same abort flag: issue and
    // wait only if no thread of the CTA has given up.
    const bool go = !*s.abort_flag;
    // 2. One thread issues the MMAs: 12 groups per K step of 8.
    if (go && tid == 0) {
        tc_fence_after();
        const uint32_t lboB = (uint32_t)(N >> 3) * 128, sboA = (uint32_t)(kdim >> 2) * 128,
                       sboS = (uint32_t)(kmax_unit >> 2) * 128;
        const uint32_t id_pos = idesc_tf32(N, false), id_neg = idesc_tf32(N, true);
        const uint32_t d_re = tmem, d_im = tmem + (uint32_t)N;
        const uint32_t br = bfk::smem_u32(bu), bi = br + (uint32_t)(N * K * 4);
        const uint32_t blr = bfk::smem_u32(s.blo), bli = blr + (uint32_t)(N * K * 4);
        const uint32_t tre = bfk::smem_u32(s.tile_re), tim = bfk::smem_u32(s.tile_im);
        const uint32_t lre = bfk::smem_u32(s.alo_re), lim = bfk::smem_u32(s.alo_im);
        for (int kk = 0; kk < (K >> 3); ++kk) {
            const int k = kk * 8;
            const int pos = k < half ? pa + k : pb + (k - half);
            const uint32_t ao = (uint32_t)(pos >> 2) * 128, so = (uint32_t)(k >> 2) * 128,
                           bo = (uint32_t)(k >> 2) * lboB;
            const uint64_t xr = sdesc(tre + ao, 128, sboA), xi = sdesc(tim + ao, 128, sboA);
            const uint64_t xrl = sdesc(lre + so, 128, sboS), xil = sdesc(lim + so, 128, sboS);
            const uint64_t Br = sdesc(br + bo, lboB, 128), Bi = sdesc(bi + bo, lboB, 128);
            const uint64_t Brl = sdesc(blr + bo, lboB, 128), Bil = sdesc(bli + bo, lboB, 128);
            const uint32_t first = kk == 0 ? 0u : 1u;
            mma_tf32(d_re, xr, Br, id_pos, first);
            mma_tf32(d_re, xr, Brl, id_pos, 1);
            mma_tf32(d_re, xrl, Br, id_pos, 1);
            mma_tf32(d_re, xi, Bi, id_neg, 1);
            mma_tf32(d_re, xi, Bil, id_neg, 1);
            mma_tf32(d_re, xil, Bi, id_neg, 1);
            mma_tf32(d_im, xr, Bi, id_pos, first);
            mma_tf32(d_im, xr, Bil, id_pos, 1);
            mma_tf32(d_im, xrl, Bi, id_pos, 1);
            mma_tf32(d_im, xi, Br, id_pos, 1);
            mma_tf32(d_im, xi, Brl, id_pos, 1);
            mma_tf32(d_im, xil, Br, id_pos, 1);
        }
        mma_commit(s.mma_bar);
    }
    // 3. Wait for the MMAs, read D, write the outputs over the unit's inputs.
    const bool ok = go && bfk::mbar_wait(s.mma_bar, mma_phase & 1, s.abort_flag, p.err);
    if (go) ++mma_phase;
    tc_fence_after();
    const int warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, chalf = warp >> 2;      // 8 consumer warps: 4 lane quarters x 2 column halves
    const int m = quarter * 32 + lane;
    const int ncol = N >> 1;
    if (ok && chalf < (nc >> 7)) {
        for (int c0 = chalf * ncol; c0 < (chalf + 1) * ncol; c0 += 8) {
            float vr[8], vi[8];
            const uint32_t lane_addr = ((uint32_t)(quarter * 32) << 16);
            tmem_ld8(tmem + lane_addr + (uint32_t)c0, vr);
            tmem_ld8(tmem + lane_addr + (uint32_t)(N + c0), vi);
            if (KIND == bfk::LEAF_OUT) {
                if (m < nt) {
                    const int ps = bfw::slot_of(p, g, u);
                    float2 *dst = p.out + (long long)(rhs0 + m) * p.ld_out + ((long long)n * p.m + ps) * p.n0 + c0;
#pragma unroll
                    for (int i = 0; i < 8; ++i) dst[i] = make_float2(vr[i], vi[i]);
                }
            } else {
                int pos;
                if (KIND == bfk::LEAF_IN) {
                    pos = u * p.r + c0;
                } else {
                    const int o = c0 >= p.r ? 1 : 0;
                    pos = (o ? j1 : j0) * p.r + (c0 - o * p.r);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int off = aoff(m, pos + 4 * i, kdim) >> 2;
                    *reinterpret_cast<float4 *>(s.tile_re + off) =
                        make_float4(vr[4 * i], vr[4 * i + 1], vr[4 * i + 2], vr[4 * i + 3]);
                    *reinterpret_cast<float4 *>(s.tile_im + off) =
                        make_float4(vi[4 * i], vi[4 * i + 1], vi[4 * i + 2], vi[4 * i + 3]);
                }
            }
        }
    }
    tc_fence_before();
    bfk::consumer_sync(nc);
    return ok;
}

template <int KIND>
__device__ __forceinline__ void tc_level(const WideParams &p, const TcSmem &s, int kdim, int kmax_unit,
                                         const Level &lv, uint32_t &gs, int n, int g, int rhs0, int nt, int nc,
                                         uint32_t tmem, uint32_t &mma_phase) {
    const int lane = threadIdx.x & 31;
    const int off_in = p.G * (p.W - p.n0);
    const int N = lv.rpu, K = lv.K;
    for (int st = 0; st < lv.nstages; ++st, ++gs) {
        const uint32_t slot = gs % p.stages;
        const uint32_t use = gs / p.stages;
        if (!*s.abort_flag) bfk::mbar_wait(&s.full[slot], use & 1, s.abort_flag, p.err);
        bfk::consumer_sync(nc);
        const bool ready = !*s.abort_flag;   // uniform: read after the barrier
        const float *stg = reinterpret_cast<const float *>(s.ring + (long long)slot * p.slot_len);
        for (int ui = 0; ui < lv.upb; ++ui) {
            const int u = st * lv.upb + ui;
            int pa, pb, half, j0 = 0, j1 = 0;
            if (KIND == bfk::LEAF_IN) {
                pa = off_in + u * p.n0;
                pb = pa;
                half = K;
            } else if (KIND == bfk::LEAF_OUT) {
                pa = u * p.r;
                pb = pa;
                half = K;
            } else {
                j0 = bfw::insert0(u, lv.s);
                j1 = j0 | (1 << lv.s);
                pa = j0 * p.r;
                pb = j1 * p.r;
                half = p.r;
            }
            if (ready)
                tc_unit<KIND>(p, s, kdim, kmax_unit, stg + (long long)ui * 2 * N * K, N, K, pa, pb, half, j0, j1, u, n,
                              g, rhs0, nt, nc, tmem, mma_phase);
        }
        __syncwarp();
        if (lane == 0) bfk::mbar_arrive(&s.empty[slot]);
    }
}

__global__ void __launch_bounds__(288, 1) bf_tc_kernel(const WideParams p, int kmax_unit, int nk_max) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int nc = blockDim.x - 32;   // 256 consumers = 8 warps
    const int kdim = p.G * p.W;
    TcSmem s;
    s.ring = reinterpret_cast<float2 *>(smem_raw);
    s.tile_re = reinterpret_cast<float *>(s.ring + (long long)p.stages * p.slot_len);
    s.tile_im = s.tile_re + (long long)NR * kdim;
    s.alo_re = s.tile_im + (long long)NR * kdim;
    s.alo_im = s.alo_re + (long long)NR * kmax_unit;
    s.blo = s.alo_im + (long long)NR * kmax_unit;
    s.full = reinterpret_cast<uint64_t *>(s.blo + 2ll * nk_max);
    s.empty = s.full + p.stages;
    s.mma_bar = s.empty + p.stages;
    s.tmem_slot = reinterpret_cast<uint32_t *>(s.mma_bar + 1);
    s.abort_flag = reinterpret_cast<volatile int *>(s.tmem_slot + 1);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int i = 0; i < p.stages; ++i) {
            bfk::mbar_init(&s.full[i], 1);
            bfk::mbar_init(&s.empty[i], nc / 32);
        }
        bfk::mbar_init(s.mma_bar, 1);
        *s.abort_flag = 0;
        bfk::fence_mbar_init();
    }
    if (tid < 32) {
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
    const int n = blockIdx.y / p.ngroups;
    const int g = blockIdx.y - n * p.ngroups;
    const int rhs0 = blockIdx.x * NR;
    const int nt = min(NR, p.nrhs - rhs0);
    if (tid >= nc) {
        if (tid == nc) bfk::produce(p, blockIdx.y, s.ring, s.full, s.empty, s.abort_flag);
    } else {
        tc_load(p, s, kdim, n, g, rhs0, nt, nc);
        bfk::consumer_sync(nc);
        uint32_t gs = 0, mma_phase = 0;
        for (int l = 0; l < p.nlev; ++l) {
            const Level lv = p.lev[l];
            switch (lv.kind) {
                case bfk::LEAF_IN: tc_level<bfk::LEAF_IN>(p, s, kdim, kmax_unit, lv, gs, n, g, rhs0, nt, nc, tmem, mma_phase); break;
                case bfk::MERGE: tc_level<bfk::MERGE>(p, s, kdim, kmax_unit, lv, gs, n, g, rhs0, nt, nc, tmem, mma_phase); break;
                case bfk::SPLIT: tc_level<bfk::SPLIT>(p, s, kdim, kmax_unit, lv, gs, n, g, rhs0, nt, nc, tmem, mma_phase); break;
                default: tc_level<bfk::LEAF_OUT>(p, s, kdim, kmax_unit, lv, gs, n, g, rhs0, nt, nc, tmem, mma_phase); break;
            }
            bfk::consumer_sync(nc);
        }
        if (p.store_kind != bfw::ST_NONE) tc_store(p, s, kdim, n, g, rhs0, nt, nc);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace bftc
