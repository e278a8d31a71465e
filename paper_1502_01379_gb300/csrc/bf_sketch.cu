// Sketch products of a 1D kernel matrix, evaluated entry by entry on the GPU.
//
// K(x_j, xi_k) = exp(2 pi i (x_j xi_k + c_j |xi_k|)),  x_j = j / N,  xi_k = k - N/2
// (Sec. 4, Eq. 1D-FIO-kernal with c_j = c(x_j); c = 0 is the Fourier matrix of
// Sec. 1.1 up to the column shift).  The construction from products (Sec. 3.1,
// first case; Sec. 2.1) needs K_ij C_jj and K_ij^* R_ii for Gaussian blocks
// C_jj, R_ii supported on one middle-level node each; with no fast apply of K
// at hand these are formed here directly: O(N^2 k) multiply-adds, entries
// generated in registers and never stored.
//
// Phase reduction.  frac(Phi) is carried as a 64-bit fixed-point fraction,
// exact modulo 1: x_j xi_k = j xi_k / N is (j xi_k mod N) 2^(64 - log2 N), a
// wrapping 64-bit product of j << (64 - log2 N) and xi_k; c_j |xi_k| is the
// wrapping product of c_j 2^64 (an exact integer for an FP64 c_j in [2^-10, 1),
// computed by the caller) and |xi_k|.  The sum is rounded to 24 bits (2^-25
// turn, 1.9e-7 rad) and sin / cos taken in FP32 (sincospif).
//
// Layout: two output indices o per thread (rows x for the forward products,
// columns xi for the adjoint ones), 256 per CTA; blockIdx.y is the sketch
// block (node); the node's nb summation indices stream through shared memory
// in chunks of 64 together with the block's rows (broadcast reads: every
// thread of the CTA reads the same entry), each thread accumulating k complex
// sums in registers.  Every output is written once, coalesced.

#include "bfly.h"

#include <cstdint>

namespace bfs {

constexpr int TPB = 128;
constexpr int SCHUNK = 64;

struct Args {
    const unsigned long long *c;   // N fixed-point c_j, or null (c = 0)
    const float2 *blocks;          // (nodes, nb, k)
    float2 *out;                   // (nodes, k, hi - lo)
    long long lo, hi;
    int log2N, nb, k, node0;
};

// Two outputs per thread (o and o + TPB): each staged sketch entry feeds both
// from one shared-memory load, halving the loads per multiply-add.
constexpr int ROWS = 2;

template <int KP, bool ADJ>
__global__ void __launch_bounds__(TPB) sketch_kernel(Args a) {
    __shared__ float2 sb[SCHUNK][KP];
    __shared__ unsigned long long sc[SCHUNK];
    const int b = blockIdx.y;
    const long long s0 = (long long)(a.node0 + b) * a.nb;
    const float2 *blk = a.blocks + (long long)b * a.nb * a.k;
    const int sh = 64 - a.log2N;
    const long long half = 1LL << (a.log2N - 1);
    long long o[ROWS];
    bool valid[ROWS];
    unsigned long long mul[ROWS], cx[ROWS], axi[ROWS];
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
        o[q] = a.lo + (long long)blockIdx.x * (TPB * ROWS) + q * TPB + threadIdx.x;
        valid[q] = o[q] < a.hi;
        const long long oo = valid[q] ? o[q] : 0;
        if (!ADJ) {
            mul[q] = (unsigned long long)oo << sh;                    // x << sh, times xi' below
            cx[q] = (a.c && valid[q]) ? a.c[oo] : 0ULL;
            axi[q] = 0;
        } else {
            const long long xi = oo - half;
            mul[q] = (unsigned long long)xi << sh;                    // xi' << sh, times x below
            axi[q] = (unsigned long long)(xi < 0 ? -xi : xi);
            cx[q] = 0;
        }
    }
    float2 acc[ROWS][KP];
#pragma unroll
    for (int q = 0; q < ROWS; ++q)
#pragma unroll
        for (int c = 0; c < KP; ++c) acc[q][c] = make_float2(0.f, 0.f);
    for (int t0 = 0; t0 < a.nb; t0 += SCHUNK) {
        const int tn = min(SCHUNK, a.nb - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < SCHUNK * KP; e += TPB) {
            const int t = e / KP, c = e - t * KP;
            sb[t][c] = (t < tn && c < a.k) ? blk[(long long)(t0 + t) * a.k + c] : make_float2(0.f, 0.f);
        }
        if (ADJ)
            for (int t = threadIdx.x; t < SCHUNK; t += TPB) sc[t] = (a.c && t < tn) ? a.c[s0 + t0 + t] : 0ULL;
        __syncthreads();
        for (int t = 0; t < tn; ++t) {
            const long long s = s0 + t0 + t;
            float sn[ROWS], cs[ROWS];
#pragma unroll
            for (int q = 0; q < ROWS; ++q) {
                unsigned long long P;
                if (!ADJ) {
                    const long long xi = s - half;
                    P = mul[q] * (unsigned long long)xi + cx[q] * (unsigned long long)(xi < 0 ? -xi : xi);
                } else {
                    P = (unsigned long long)s * mul[q] + sc[t] * axi[q];
                }
                // 2 frac(Phi) in [0, 2), rounded to 24 bits (a wrap to 2^24 is 2 = 0 turns)
                const unsigned w = (unsigned)(((P + (1ULL << 39)) >> 40) & 0xFFFFFFULL);
                sincospif((float)w * (1.0f / 8388608.0f), &sn[q], &cs[q]);
                if (ADJ) sn[q] = -sn[q];                                  // conj(K)
            }
#pragma unroll
            for (int c = 0; c < KP; ++c) {
                const float2 v = sb[t][c];
#pragma unroll
                for (int q = 0; q < ROWS; ++q) {
                    acc[q][c].x = fmaf(cs[q], v.x, fmaf(-sn[q], v.y, acc[q][c].x));
                    acc[q][c].y = fmaf(cs[q], v.y, fmaf(sn[q], v.x, acc[q][c].y));
                }
            }
        }
    }
    const long long rows = a.hi - a.lo;
#pragma unroll
    for (int q = 0; q < ROWS; ++q) {
        if (!valid[q]) continue;
        float2 *dst = a.out + (long long)b * a.k * rows + (o[q] - a.lo);
#pragma unroll
        for (int c = 0; c < KP; ++c)
            if (c < a.k) dst[(long long)c * rows] = acc[q][c];
    }
}

template <int KP>
cudaError_t launch(const Args &a, int nodes, bool adjoint, cudaStream_t s) {
    const dim3 grid((unsigned)((a.hi - a.lo + TPB * ROWS - 1) / (TPB * ROWS)), (unsigned)nodes);
    if (adjoint)
        sketch_kernel<KP, true><<<grid, TPB, 0, s>>>(a);
    else
        sketch_kernel<KP, false><<<grid, TPB, 0, s>>>(a);
    return cudaGetLastError();
}

bool is_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace bfs

extern "C" bf_status bf_sketch_products(const bf_sketch_desc *d, const unsigned long long *c_fixed,
                                        const void *blocks, void *out, cudaStream_t stream) {
    if (!d || !blocks || !out) return BF_ERR_INVALID;
    if (d->log2N < 1 || d->log2N > 30 || d->k < 1 || d->nb < 1 || d->nodes < 1 || d->node0 < 0)
        return BF_ERR_INVALID;
    const long long N = 1LL << d->log2N;
    if ((d->nb & (d->nb - 1)) || d->nb > N || (long long)(d->node0 + d->nodes) * d->nb > N) return BF_ERR_INVALID;
    if (d->lo < 0 || d->hi > N || d->lo >= d->hi) return BF_ERR_INVALID;
    if (d->k > 32 || d->nodes > 65535) return BF_ERR_UNSUPPORTED;
    if (!bfs::is_device(blocks) || !bfs::is_device(out) || (c_fixed && !bfs::is_device(c_fixed)))
        return BF_ERR_INVALID;
    bfs::Args a;
    a.c = c_fixed;
    a.blocks = static_cast<const float2 *>(blocks);
    a.out = static_cast<float2 *>(out);
    a.lo = d->lo;
    a.hi = d->hi;
    a.log2N = d->log2N;
    a.nb = d->nb;
    a.k = d->k;
    a.node0 = d->node0;
    const bool adj = d->adjoint != 0;
    // exact widths for k = r + 5 at r = 8, 12, 16 (the construction's sketches), else padded
    cudaError_t e = d->k <= 8    ? bfs::launch<8>(a, d->nodes, adj, stream)
                  : d->k == 13 ? bfs::launch<13>(a, d->nodes, adj, stream)
                  : d->k <= 16 ? bfs::launch<16>(a, d->nodes, adj, stream)
                  : d->k == 17 ? bfs::launch<17>(a, d->nodes, adj, stream)
                  : d->k == 21 ? bfs::launch<21>(a, d->nodes, adj, stream)
                  : d->k <= 24 ? bfs::launch<24>(a, d->nodes, adj, stream)
                               : bfs::launch<32>(a, d->nodes, adj, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA;
    }
    return BF_OK;
}
