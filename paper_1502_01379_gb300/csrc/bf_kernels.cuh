// Butterfly-factorization apply kernels for sm_103a.
//
// The factorization K ~ U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^*
// (Eq. Kfactors) splits at the middle level h = L/2 into two halves that are
// local to one tree node each (Sec. 3.1-3.2):
//
//  * "down" kernel: for column node j of T_Omega at level h, the leaf factor
//    (V^L)^* on the n0*m points of B^h_j and the transfer factors
//    (H^{L-1})^* ... (H^h)^* only ever touch the m r-blocks of segment j of the
//    intermediate vector (each (H^l)^* is a set of 2r x 2r butterflies that
//    merge two half-segments, mirror of Eq. RSh2).  One CTA keeps that segment
//    in shared memory across all levels and writes it out once.
//  * M^h is a block transpose of the m x m grid of r-blocks times a real
//    diagonal (Eq. KeqUMV): the "up" kernel of row node i gathers blocks
//    (q m + i), q < m, scaled by S^h_{i,q}.
//  * "up" kernel: G^h ... G^{L-1} (butterflies that split a segment in two,
//    Eq. RSh2) and the leaf factor U^L for row node i, writing N/m outputs.
//
// The adjoint uses the same two kernels with the conjugate-transposed factors
// (packed separately) and S^T.  Every factor entry is read from HBM exactly
// once per launch (per RHS tile): the factor stream of each CTA is laid out
// contiguously in consumption order and streamed through a ring of shared-
// memory slots by a producer warp issuing cp.async.bulk (TMA) copies that
// complete on mbarriers; consumer warps compute one output row per thread
// with the factor read from shared memory (coalesced, k-major within a stage)
// and the input entry broadcast from the segment buffer.
//
// All waits are bounded (globaltimer, ~2 s).  On expiry a thread sets a shared
// abort flag and the plan's error word; every thread then runs the remaining
// control flow without waiting or computing, so all barriers are still met,
// and the producer drains the copies it issued before the CTA exits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bfk {

constexpr int kMaxLevels = 16;
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned long long kWaitNs = 2000000000ull;

enum LevelKind : int { LEAF_IN = 0, MERGE = 1, SPLIT = 2, LEAF_OUT = 3 };

struct Level {
    int kind;
    int K;          // inner dimension of one unit (n0, 2r or r)
    int rpu;        // output rows of one unit (r, 2r or n0)
    int upb;        // units per stage
    int nstages;    // stages of this level per CTA
    int stage_len;  // complex elements per stage (even: 16-byte multiple)
    int s;          // MERGE/SPLIT: segment size in r-blocks at this level
    int pad_;
};

struct Params {
    const float2 *fac;      // packed factor stream, one chunk of cta_len per CTA
    long long cta_len;
    const float2 *in;       // down: vectors (N x nrhs); up: workspace (R x nrhs)
    long long ld_in;
    float2 *out;            // down: workspace; up: vectors
    long long ld_out;
    const float *S;         // up: S rows of this direction, (node, q, k)
    unsigned *err;
    int nlev;
    int m, r, n0, W;        // W = max(n0, r)
    int nrhs;               // vectors in this launch
    int stages;             // ring depth
    int slot_len;           // complex elements per ring slot
    Level lev[kMaxLevels];
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared (TMA engine), completion counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void consumer_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Bounded wait on one mbarrier phase.  Returns false (after flagging the
// abort) if the phase did not complete within kWaitNs or another thread of
// the CTA has already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned *err) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (*abort_flag) return false;
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicOr(err, kErrTimeout);
            return false;
        }
    }
}

__device__ __forceinline__ void cfma(float2 &acc, float2 f, float2 x) {
    acc.x = fmaf(f.x, x.x, acc.x);
    acc.x = fmaf(-f.y, x.y, acc.x);
    acc.y = fmaf(f.x, x.y, acc.y);
    acc.y = fmaf(f.y, x.x, acc.y);
}

// --------------------------------------------------------------- producer
// One thread streams this CTA's factor chunk, stage by stage, into the ring.
__device__ __forceinline__ void produce(const Params &p, float2 *ring, uint64_t *full, uint64_t *empty,
                                       volatile int *abort_flag) {
    const float2 *src = p.fac + (long long)blockIdx.y * p.cta_len;
    uint32_t gs = 0;
    bool ok = true;
    for (int l = 0; l < p.nlev && ok; ++l) {
        const Level &lv = p.lev[l];
        for (int st = 0; st < lv.nstages; ++st) {
            const uint32_t slot = gs % p.stages;
            const uint32_t use = gs / p.stages;
            if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1, abort_flag, p.err)) {
                ok = false;
                break;
            }
            const uint32_t bytes = (uint32_t)lv.stage_len * 8u;
            mbar_arrive_expect_tx(&full[slot], bytes);
            bulk_g2s(ring + (long long)slot * p.slot_len, src, bytes, &full[slot]);
            src += lv.stage_len;
            ++gs;
        }
    }
    // Drain: every copy issued must have landed before the CTA may exit.
    for (uint32_t slot = 0; slot < (uint32_t)p.stages && slot < gs; ++slot) {
        const uint32_t last_use = (gs - 1 - slot) / p.stages;
        if (!mbar_try_wait(&full[slot], last_use & 1)) {
            const unsigned long long t0 = globaltimer();
            while (!mbar_try_wait(&full[slot], last_use & 1)) {
                if (globaltimer() - t0 > kWaitNs) {
                    *abort_flag = 1;
                    atomicOr(p.err, kErrTimeout);
                    break;
                }
            }
        }
    }
}

// ------------------------------------------------------- consumer: one stage
// Output rows `row` of the stage's units: acc[t] = sum_k F[k][row] * x_t[k],
// with x[k] taken from xa for k < half and from xb above.
template <int T>
__device__ __forceinline__ void stage_dot(const float2 *__restrict__ stg, int rows, int row, int K,
                                          const float2 *xa, const float2 *xb, int half, float2 (&acc)[T]) {
#pragma unroll
    for (int t = 0; t < T; ++t) acc[t] = make_float2(0.f, 0.f);
    const float2 *f = stg + row;
#pragma unroll 4
    for (int k = 0; k < half; ++k) {
        const float2 fk = f[(long long)k * rows];
#pragma unroll
        for (int t = 0; t < T; ++t) cfma(acc[t], fk, xa[k * T + t]);
    }
#pragma unroll 4
    for (int k = half; k < K; ++k) {
        const float2 fk = f[(long long)k * rows];
#pragma unroll
        for (int t = 0; t < T; ++t) cfma(acc[t], fk, xb[(k - half) * T + t]);
    }
}

struct Smem {
    float2 *ring, *buf0, *buf1;
    uint64_t *full, *empty;
    volatile int *abort_flag;
};

template <int T>
__device__ __forceinline__ Smem carve(const Params &p, unsigned char *smem) {
    Smem s;
    s.ring = reinterpret_cast<float2 *>(smem);
    s.buf0 = s.ring + (long long)p.stages * p.slot_len;
    s.buf1 = s.buf0 + (long long)p.m * p.W * T;
    s.full = reinterpret_cast<uint64_t *>(s.buf1 + (long long)p.m * p.W * T);
    s.empty = s.full + p.stages;
    s.abort_flag = reinterpret_cast<volatile int *>(s.empty + p.stages);
    return s;
}

__host__ __device__ inline size_t smem_bytes(int stages, int slot_len, int m, int W, int T) {
    return (size_t)stages * slot_len * 8 + 2ull * m * W * T * 8 + 2ull * stages * 8 + 16;
}

template <int T>
__device__ __forceinline__ void setup(const Params &p, const Smem &s, int nconsumers) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < p.stages; ++i) {
            mbar_init(&s.full[i], 1);
            mbar_init(&s.empty[i], nconsumers / 32);
        }
        *s.abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
}

// Runs the levels [0, nlev) of this CTA on the segment buffers; returns the
// buffer that holds the last level's output.
template <int T, bool kDown>
__device__ __forceinline__ float2 *run_levels(const Params &p, const Smem &s, int nconsumers, int rhs0,
                                              int nt) {
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int node = blockIdx.y;
    float2 *xin = s.buf0, *xout = s.buf1;
    uint32_t gs = 0;
    for (int l = 0; l < p.nlev; ++l) {
        const Level lv = p.lev[l];
        const int rows = lv.upb * lv.rpu;
        for (int st = 0; st < lv.nstages; ++st, ++gs) {
            const uint32_t slot = gs % p.stages;
            const uint32_t use = gs / p.stages;
            const bool ready = !*s.abort_flag && mbar_wait(&s.full[slot], use & 1, s.abort_flag, p.err);
            if (ready) {
                const float2 *stg = s.ring + (long long)slot * p.slot_len;
                for (int row = tid; row < rows; row += nconsumers) {
                    const int u = st * lv.upb + row / lv.rpu;
                    const int rr = row % lv.rpu;
                    float2 acc[T];
                    if (lv.kind == LEAF_IN) {
                        // unit = leaf u of this node, output r-block u
                        stage_dot<T>(stg, rows, row, lv.K, xin + (long long)u * p.n0 * T, nullptr, lv.K, acc);
#pragma unroll
                        for (int t = 0; t < T; ++t) xout[((long long)u * p.r + rr) * T + t] = acc[t];
                    } else if (lv.kind == MERGE) {
                        // inputs: blocks seg*s + c*s/2 + q (c = 0, 1); outputs seg*s + 2q + d
                        const int hs = lv.s >> 1, seg = u / hs, q = u - seg * hs;
                        const long long b0 = (long long)seg * lv.s + q;
                        stage_dot<T>(stg, rows, row, lv.K, xin + b0 * p.r * T, xin + (b0 + hs) * p.r * T, p.r,
                                     acc);
                        const long long o = ((long long)seg * lv.s + 2 * q) * p.r + rr;
#pragma unroll
                        for (int t = 0; t < T; ++t) xout[o * T + t] = acc[t];
                    } else if (lv.kind == SPLIT) {
                        // inputs: blocks seg*s + 2q + d; outputs seg*s + c*s/2 + q
                        const int hs = lv.s >> 1, seg = u / hs, q = u - seg * hs;
                        const long long b0 = (long long)seg * lv.s + 2 * q;
                        stage_dot<T>(stg, rows, row, lv.K, xin + b0 * p.r * T, nullptr, lv.K, acc);
                        const int c = rr / p.r, kk = rr - c * p.r;
                        const long long o = ((long long)seg * lv.s + c * hs + q) * p.r + kk;
#pragma unroll
                        for (int t = 0; t < T; ++t) xout[o * T + t] = acc[t];
                    } else {  // LEAF_OUT: unit = leaf u of this node, n0 outputs to global
                        stage_dot<T>(stg, rows, row, lv.K, xin + (long long)u * p.r * T, nullptr, lv.K, acc);
                        const long long o = (long long)node * p.n0 * p.m + (long long)u * p.n0 + rr;
#pragma unroll
                        for (int t = 0; t < T; ++t)
                            if (t < nt) p.out[(long long)(rhs0 + t) * p.ld_out + o] = acc[t];
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&s.empty[slot]);
        }
        consumer_sync(nconsumers);
        float2 *tmp = xin;
        xin = xout;
        xout = tmp;
    }
    return xin;
}

// ------------------------------------------------------------------ kernels
template <int T>
__global__ void __launch_bounds__(288, 1) bf_down_kernel(const Params p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nconsumers = blockDim.x - 32;
    const Smem s = carve<T>(p, smem_raw);
    setup<T>(p, s, nconsumers);
    const int tid = threadIdx.x;
    const int node = blockIdx.y;          // tree node at level h
    const int rhs0 = blockIdx.x * T;      // RHS tile (fastest: tiles of one node share its factors in L2)
    const int nt = min(T, p.nrhs - rhs0);
    if (tid >= nconsumers) {
        if (tid == nconsumers) produce(p, s.ring, s.full, s.empty, s.abort_flag);
    } else {
        // Input points of column node `node`: n0*m consecutive entries per RHS.
        const int nin = p.n0 * p.m;
        const long long base = (long long)node * nin;
        for (int e = tid; e < nin * T; e += nconsumers) {
            const int t = e % T, ee = e / T;
            s.buf0[e] = (t < nt) ? __ldg(p.in + (long long)(rhs0 + t) * p.ld_in + base + ee) : make_float2(0.f, 0.f);
        }
        consumer_sync(nconsumers);
        const float2 *res = run_levels<T, true>(p, s, nconsumers, rhs0, nt);
        // Segment `node` of the level-h vector: m*r consecutive entries per RHS.
        const int nseg = p.m * p.r;
        const long long obase = (long long)node * nseg;
        for (int e = tid; e < nseg * T; e += nconsumers) {
            const int t = e % T, ee = e / T;
            if (t < nt) p.out[(long long)(rhs0 + t) * p.ld_out + obase + ee] = res[e];
        }
    }
    __syncthreads();
}

template <int T>
__global__ void __launch_bounds__(288, 1) bf_up_kernel(const Params p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int nconsumers = blockDim.x - 32;
    const Smem s = carve<T>(p, smem_raw);
    setup<T>(p, s, nconsumers);
    const int tid = threadIdx.x;
    const int node = blockIdx.y;          // tree node at level h
    const int rhs0 = blockIdx.x * T;      // RHS tile (fastest: tiles of one node share its factors in L2)
    const int nt = min(T, p.nrhs - rhs0);
    if (tid >= nconsumers) {
        if (tid == nconsumers) produce(p, s.ring, s.full, s.empty, s.abort_flag);
    } else {
        // M^h: local block q <- S[node, q] * (block q*m + node of the level-h vector).
        const int nseg = p.m * p.r;
        for (int e = tid; e < nseg * T; e += nconsumers) {
            const int t = e % T, ee = e / T;
            const int q = ee / p.r, k = ee - q * p.r;
            float2 v = make_float2(0.f, 0.f);
            if (t < nt) {
                const float w = __ldg(p.S + (long long)node * nseg + ee);
                const float2 x = __ldg(p.in + (long long)(rhs0 + t) * p.ld_in + ((long long)q * p.m + node) * p.r + k);
                v = make_float2(w * x.x, w * x.y);
            }
            s.buf0[e] = v;
        }
        consumer_sync(nconsumers);
        run_levels<T, false>(p, s, nconsumers, rhs0, nt);
    }
    __syncthreads();
}

}  // namespace bfk
