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
    int stall;              // failure-detection test hook: the producer issues no copies
    // Extents (elements) of the buffers behind fac, in, out and S: what the launch's
    // arguments define.  Checked builds (BF_CHECKED) test every global index against
    // them; other builds ignore them.
    long long fac_elems, in_elems, out_elems, s_elems;
    Level lev[kMaxLevels];
};

// Checked builds: a global index outside its buffer's extent sets kErrBounds
// in the error word and the access is skipped (a load reads zero), so a
// kernel indexing mistake shows up as a status instead of a memory fault.
constexpr unsigned kErrBounds = 2u;
#ifdef BF_CHECKED
__device__ __forceinline__ bool in_extent(unsigned *err, long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicOr(err, kErrBounds);
    return false;
}
#else
__device__ __forceinline__ bool in_extent(unsigned *, long long, long long) { return true; }
#endif

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

// --------------------------------------------------------------- producer
// One thread streams this CTA's factor chunk, stage by stage, into the ring.
// Streams one factor chunk (all levels of one CTA work item) into the ring;
// Extent of a producer's factor stream (checked builds; parameter types
// without one are not checked).
__device__ __forceinline__ long long fac_extent(const Params &p) { return p.fac_elems; }
template <class P>
__device__ __forceinline__ long long fac_extent(const P &) { return 1LL << 62; }

// `gs` counts stages across calls.  Returns false if a wait gave up.
template <class P>
__device__ __forceinline__ bool produce_chunk(const P &p, long long chunk, uint32_t &gs, float2 *ring, uint64_t *full,
                                              uint64_t *empty, volatile int *abort_flag) {
    const float2 *src = p.fac + chunk * p.cta_len;
    for (int l = 0; l < p.nlev; ++l) {
        const Level &lv = p.lev[l];
        for (int st = 0; st < lv.nstages; ++st) {
            const uint32_t slot = gs % p.stages;
            const uint32_t use = gs / p.stages;
            if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1, abort_flag, p.err)) return false;
            const uint32_t bytes = (uint32_t)lv.stage_len * 8u;
            if (!in_extent(p.err, (long long)(src - p.fac) + lv.stage_len - 1, fac_extent(p))) {
                *abort_flag = 1;   // consumers stop waiting; nothing is copied
                return false;
            }
            mbar_arrive_expect_tx(&full[slot], bytes);
            bulk_g2s(ring + (long long)slot * p.slot_len, src, bytes, &full[slot]);
            src += lv.stage_len;
            ++gs;
        }
    }
    return true;
}

// Every copy issued must have landed before the CTA may exit.
template <class P>
__device__ __forceinline__ void produce_drain(const P &p, uint32_t gs, uint64_t *full, volatile int *abort_flag) {
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

// One thread streams this CTA's factor chunk, stage by stage, into the ring.
// With the stall hook set it issues nothing: every consumer wait then runs
// into its bound and the launch ends with the error word set.
__device__ __forceinline__ bool stalled(const Params &p) { return p.stall != 0; }
template <class P>
__device__ __forceinline__ bool stalled(const P &) { return false; }
template <class P>
__device__ __forceinline__ void produce(const P &p, long long chunk, float2 *ring, uint64_t *full, uint64_t *empty,
                                       volatile int *abort_flag) {
    if (stalled(p)) return;
    uint32_t gs = 0;
    produce_chunk(p, chunk, gs, ring, full, empty, abort_flag);
    produce_drain(p, gs, full, abort_flag);
}

// ------------------------------------------------------- consumer: one stage
// One complex output for T right-hand sides, kept as four independent FMA
// chains (re*re, im*im, re*im, im*re) so consecutive k do not serialize.
template <int T>
struct Acc {
    float rr[T], ii[T], ri[T], ir[T];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int t = 0; t < T; ++t) rr[t] = ii[t] = ri[t] = ir[t] = 0.f;
    }
    __device__ __forceinline__ void mac(int t, float2 f, float2 x) {
        rr[t] = fmaf(f.x, x.x, rr[t]);
        ii[t] = fmaf(f.y, x.y, ii[t]);
        ri[t] = fmaf(f.x, x.y, ri[t]);
        ir[t] = fmaf(f.y, x.x, ir[t]);
    }
    __device__ __forceinline__ float2 get(int t) const { return make_float2(rr[t] - ii[t], ri[t] + ir[t]); }
};

// Rows r0 (and r0 + 1 when kPair) of a stage: a[t] = sum_k F[k][row] x_t[k],
// x[k] from xa for k < half and from xb above.  In pair mode both rows belong
// to the same unit, share x, and their factors arrive in one 16-byte load.
template <int T, bool kPair>
__device__ __forceinline__ void stage_dot(const float2 *__restrict__ stg, int rows, int r0, int K,
                                          const float2 *xa, const float2 *xb, int half, Acc<T> &a0, Acc<T> &a1) {
    a0.zero();
    if (kPair) a1.zero();
    const float2 *f = stg + r0;
#pragma unroll 8
    for (int k = 0; k < half; ++k) {
        float2 f0, f1;
        if (kPair) {
            const float4 v = *reinterpret_cast<const float4 *>(f + k * rows);
            f0 = make_float2(v.x, v.y);
            f1 = make_float2(v.z, v.w);
        } else {
            f0 = f[k * rows];
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float2 x = xa[k * T + t];
            a0.mac(t, f0, x);
            if (kPair) a1.mac(t, f1, x);
        }
    }
#pragma unroll 8
    for (int k = half; k < K; ++k) {
        float2 f0, f1;
        if (kPair) {
            const float4 v = *reinterpret_cast<const float4 *>(f + k * rows);
            f0 = make_float2(v.x, v.y);
            f1 = make_float2(v.z, v.w);
        } else {
            f0 = f[k * rows];
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float2 x = xb[(k - half) * T + t];
            a0.mac(t, f0, x);
            if (kPair) a1.mac(t, f1, x);
        }
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

// Output position (in r-blocks * r + row, without the RHS interleave) of row
// rr of unit u at a level of kind KIND, and the unit's input pointers.
template <int T, int KIND>
__device__ __forceinline__ void unit_io(const Params &p, const Level &lv, int lg_hs, float2 *xin, int u,
                                        const float2 *&xa, const float2 *&xb, int &half, long long &obase) {
    if (KIND == LEAF_IN) {
        xa = xin + (long long)u * p.n0 * T;
        xb = xa;
        half = lv.K;
        obase = (long long)u * p.r;
    } else if (KIND == MERGE) {
        // inputs: blocks seg*s + c*s/2 + q (c = 0, 1); outputs seg*s + 2q + d
        const int hs = lv.s >> 1, seg = u >> lg_hs, q = u & (hs - 1);
        const long long b0 = (long long)seg * lv.s + q;
        xa = xin + b0 * p.r * T;
        xb = xin + (b0 + hs) * p.r * T;
        half = p.r;
        obase = ((long long)seg * lv.s + 2 * q) * p.r;
    } else if (KIND == SPLIT) {
        // inputs: blocks seg*s + 2q + d; outputs seg*s + c*s/2 + q
        const int hs = lv.s >> 1, seg = u >> lg_hs, q = u & (hs - 1);
        xa = xin + ((long long)seg * lv.s + 2 * q) * p.r * T;
        xb = xa;
        half = lv.K;
        obase = ((long long)seg * lv.s + q) * p.r;   // + c*hs*r + kk per row
    } else {  // LEAF_OUT
        xa = xin + (long long)u * p.r * T;
        xb = xa;
        half = lv.K;
        obase = (long long)u * p.n0;
    }
}

template <int T, int KIND>
__device__ __forceinline__ void store_row(const Params &p, const Level &lv, float2 *xout, long long obase, int rr,
                                          const Acc<T> &a, int node, int rhs0, int nt) {
    if (KIND == LEAF_IN || KIND == MERGE) {
#pragma unroll
        for (int t = 0; t < T; ++t) xout[(obase + rr) * T + t] = a.get(t);
    } else if (KIND == SPLIT) {
        const int c = rr >= p.r ? 1 : 0;
        const long long o = obase + (long long)c * (lv.s >> 1) * p.r + (rr - c * p.r);
#pragma unroll
        for (int t = 0; t < T; ++t) xout[o * T + t] = a.get(t);
    } else {
        const long long o = (long long)node * p.n0 * p.m + obase + rr;
#pragma unroll
        for (int t = 0; t < T; ++t)
            if (t < nt) {
                const long long i = (long long)(rhs0 + t) * p.ld_out + o;
                if (in_extent(p.err, i, p.out_elems)) p.out[i] = a.get(t);
            }
    }
}

// All stages of one level.  Work items are single rows, or pairs of
// adjacent rows of one unit when the unit's row count is even.
template <int T, int KIND>
__device__ __forceinline__ void run_level(const Params &p, const Smem &s, const Level &lv, float2 *xin,
                                          float2 *xout, uint32_t &gs, int nconsumers, int node, int rhs0, int nt) {
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int rows = lv.upb * lv.rpu;
    const bool pair = (lv.rpu & 1) == 0;
    const int nitems = pair ? rows >> 1 : rows;
    const int lg_hs = lv.s > 1 ? __ffs(lv.s >> 1) - 1 : 0;
    // The first item of this thread has the same (unit-in-stage, row) in every stage.
    const int r_first = pair ? 2 * tid : tid;
    const int ui_first = r_first / lv.rpu;
    const int rr_first = r_first - ui_first * lv.rpu;
    for (int st = 0; st < lv.nstages; ++st, ++gs) {
        const uint32_t slot = gs % p.stages;
        const uint32_t use = gs / p.stages;
        const bool ready = !*s.abort_flag && mbar_wait(&s.full[slot], use & 1, s.abort_flag, p.err);
        if (ready) {
            const float2 *stg = s.ring + (long long)slot * p.slot_len;
            for (int it = tid; it < nitems; it += nconsumers) {
                int r0, ui, rr;
                if (it == tid) {
                    r0 = r_first;
                    ui = ui_first;
                    rr = rr_first;
                } else {
                    r0 = pair ? 2 * it : it;
                    ui = r0 / lv.rpu;
                    rr = r0 - ui * lv.rpu;
                }
                const int u = st * lv.upb + ui;
                const float2 *xa, *xb;
                int half;
                long long obase;
                unit_io<T, KIND>(p, lv, lg_hs, xin, u, xa, xb, half, obase);
                Acc<T> a0, a1;
                if (pair) {
                    stage_dot<T, true>(stg, rows, r0, lv.K, xa, xb, half, a0, a1);
                    store_row<T, KIND>(p, lv, xout, obase, rr, a0, node, rhs0, nt);
                    store_row<T, KIND>(p, lv, xout, obase, rr + 1, a1, node, rhs0, nt);
                } else {
                    stage_dot<T, false>(stg, rows, r0, lv.K, xa, xb, half, a0, a1);
                    store_row<T, KIND>(p, lv, xout, obase, rr, a0, node, rhs0, nt);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.empty[slot]);
    }
}

// Runs the levels [0, nlev) of this CTA on the segment buffers; returns the
// buffer that holds the last level's output.
template <int T>
__device__ __forceinline__ float2 *run_levels(const Params &p, const Smem &s, int nconsumers, int node, int rhs0,
                                              int nt) {
    float2 *xin = s.buf0, *xout = s.buf1;
    uint32_t gs = 0;
    for (int l = 0; l < p.nlev; ++l) {
        const Level lv = p.lev[l];
        switch (lv.kind) {
            case LEAF_IN: run_level<T, LEAF_IN>(p, s, lv, xin, xout, gs, nconsumers, node, rhs0, nt); break;
            case MERGE: run_level<T, MERGE>(p, s, lv, xin, xout, gs, nconsumers, node, rhs0, nt); break;
            case SPLIT: run_level<T, SPLIT>(p, s, lv, xin, xout, gs, nconsumers, node, rhs0, nt); break;
            default: run_level<T, LEAF_OUT>(p, s, lv, xin, xout, gs, nconsumers, node, rhs0, nt); break;
        }
        consumer_sync(nconsumers);
        float2 *tmp = xin;
        xin = xout;
        xout = tmp;
    }
    return xin;
}

// ------------------------------------------------------------------ kernels
// Down half of one CTA: column node `node` (tree node at level h), RHS tile
// starting at rhs0 (tiles of one node are adjacent in the grid, so they share
// its factors in L2).
template <int T>
__device__ __forceinline__ void down_body(const Params &p, unsigned char *smem_raw, int node, int rhs0) {
    const int nconsumers = blockDim.x - 32;
    const Smem s = carve<T>(p, smem_raw);
    setup<T>(p, s, nconsumers);
    const int tid = threadIdx.x;
    const int nt = min(T, p.nrhs - rhs0);
    if (tid >= nconsumers) {
        if (tid == nconsumers) produce(p, node, s.ring, s.full, s.empty, s.abort_flag);
    } else {
        // Input points of column node `node`: n0*m consecutive entries per RHS.
        const int nin = p.n0 * p.m;
        const long long base = (long long)node * nin;
        for (int e = tid; e < nin * T; e += nconsumers) {
            const int t = e % T, ee = e / T;
            const long long i = (long long)(rhs0 + t) * p.ld_in + base + ee;
            s.buf0[e] = (t < nt && in_extent(p.err, i, p.in_elems)) ? __ldg(p.in + i) : make_float2(0.f, 0.f);
        }
        consumer_sync(nconsumers);
        const float2 *res = run_levels<T>(p, s, nconsumers, node, rhs0, nt);
        // Segment `node` of the level-h vector: m*r consecutive entries per RHS.
        const int nseg = p.m * p.r;
        const long long obase = (long long)node * nseg;
        for (int e = tid; e < nseg * T; e += nconsumers) {
            const int t = e % T, ee = e / T;
            if (t < nt) {
                const long long i = (long long)(rhs0 + t) * p.ld_out + obase + ee;
                if (in_extent(p.err, i, p.out_elems)) p.out[i] = res[e];
            }
        }
    }
    __syncthreads();
}

// Up half of one CTA: row node `node`, RHS tile starting at rhs0.
template <int T>
__device__ __forceinline__ void up_body(const Params &p, unsigned char *smem_raw, int node, int rhs0) {
    const int nconsumers = blockDim.x - 32;
    const Smem s = carve<T>(p, smem_raw);
    setup<T>(p, s, nconsumers);
    const int tid = threadIdx.x;
    const int nt = min(T, p.nrhs - rhs0);
    if (tid >= nconsumers) {
        if (tid == nconsumers) produce(p, node, s.ring, s.full, s.empty, s.abort_flag);
    } else {
        // M^h: local block q <- S[node, q] * (block q*m + node of the level-h vector).
        const int nseg = p.m * p.r;
        for (int e = tid; e < nseg * T; e += nconsumers) {
            const int t = e % T, ee = e / T;
            const int q = ee / p.r, k = ee - q * p.r;
            float2 v = make_float2(0.f, 0.f);
            if (t < nt) {
                const long long is = (long long)node * nseg + ee;
                const long long ix = (long long)(rhs0 + t) * p.ld_in + ((long long)q * p.m + node) * p.r + k;
                if (in_extent(p.err, is, p.s_elems) && in_extent(p.err, ix, p.in_elems)) {
                    const float w = __ldg(p.S + is);
                    const float2 x = __ldg(p.in + ix);
                    v = make_float2(w * x.x, w * x.y);
                }
            }
            s.buf0[e] = v;
        }
        consumer_sync(nconsumers);
        run_levels<T>(p, s, nconsumers, node, rhs0, nt);
    }
    __syncthreads();
}

template <int T>
__global__ void __launch_bounds__(288, 1) bf_down_kernel(const Params p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    down_body<T>(p, smem_raw, blockIdx.y, blockIdx.x * T);
}

template <int T>
__global__ void __launch_bounds__(288, 1) bf_up_kernel(const Params p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    up_body<T>(p, smem_raw, blockIdx.y, blockIdx.x * T);
}

// Grouped launches: many operators (each its own Params) in one grid.  CTA i
// runs work item items[i] = (operator, node, RHS tile) with that operator's
// Params, copied to shared memory first.  Register-bounded for two CTAs per
// SM up to 4 RHS per tile (batches are mostly small operators whose CTAs need
// little shared memory); 8-RHS tiles hold 8 vectors of a node segment (up to
// 128 KB) and take one CTA per SM.
struct GroupItem {
    int op, node, rhs0, pad_;
};

template <int T>
__global__ void __launch_bounds__(288, (T >= 8 ? 1 : 2)) bf_down_grouped(const Params *plist, const GroupItem *items) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Params sp;
    const GroupItem it = items[blockIdx.x];
    if (threadIdx.x == 0) sp = plist[it.op];
    __syncthreads();
    down_body<T>(sp, smem_raw, it.node, it.rhs0);
}

template <int T>
__global__ void __launch_bounds__(288, (T >= 8 ? 1 : 2)) bf_up_grouped(const Params *plist, const GroupItem *items) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Params sp;
    const GroupItem it = items[blockIdx.x];
    if (threadIdx.x == 0) sp = plist[it.op];
    __syncthreads();
    up_body<T>(sp, smem_raw, it.node, it.rhs0);
}

}  // namespace bfk
