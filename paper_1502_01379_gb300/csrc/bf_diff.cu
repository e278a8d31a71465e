// Reverse-mode differentiation of the butterfly apply (sm_103a): the
// gradient of a real loss with respect to the input vectors and to every
// factor block, behind the bf_diff_* entry points of bfly.h.
//
// u = K g with K = U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^*
// (Eq. Kfactors) is linear in the input and in each factor separately, so
// for one factor step y = A x with upstream gradient ybar:
//     xbar = A^* ybar,   Abar = sum over RHS of ybar x^*,
// and a block used through its conjugate transpose, y = B^* x, has
// Bbar = sum over RHS of x ybar^*  (PyTorch's convention for complex tensors:
// grad = dL/dRe + i dL/dIm).  Every step of the chain is a set of
// independent units that share this form.  A unit has `count` parameter
// blocks X_c of p x q, a "P side" of count p-vectors and a "Q side" of one
// q-vector:
//     leaf V^L, U^L:  count 1, p = n0 (the leaf's points), q = r;
//     butterfly of transfer level l (Eq. RSh2 and its mirror for H):
//                     count 2, p = r (the two r-blocks X_c = H^l_{2a+c,b} or
//                     G^l_{2a+c,b} act on / produce), q = 2r (the two r-blocks
//                     on the other side of the butterfly),
// and one of two forms,  "XH": Q = sum_c X_c^* P_c   or   "X": P_c = X_c Q,
// with the parameter gradient always Xbar_c = sum over RHS of P_c Qbar^*
// (P_c and Q being the step's P-side and Q-side vectors, one of them the
// saved forward input and the other the upstream gradient):
//     forward V:  t = V^* g        XH       backward: gbar = V tbar (X),  Vbar = g tbar^*
//     forward H:  out = sum H^* in XH       backward: inbar = H outbar,   Hbar = in outbar^*
//     forward G:  out = G in       X        backward: inbar = sum G^* outbar (XH), Gbar = outbar in^*
//     forward U:  u = U w          X        backward: wbar = U^* ubar (XH), Ubar = ubar w^*
// The Q side of unit u is always the contiguous positions [u q, (u+1) q) of
// its vector (leaf r-block u, or the two adjacent r-blocks 2u, 2u+1 of the
// butterfly's two-block side); the P side is leaf block u, or r-blocks
// (2a+c) C + b with (a, b) = (u / C, u % C), C = 2^{L-l-1}.  M^h (Eq. KeqUMV)
// is its own elementwise kernel.
//
// Vectors inside are position-major: entry (position, RHS j) at
// position * nrhs + j, so a warp reads 32 RHS of one position contiguously;
// the caller's column-major vectors are transposed at entry and exit.
// The forward pass keeps the input of every k-th factor (the "saved" buffer
// the caller owns); the backward pass recomputes the others segment by
// segment from those checkpoints.  k = 1 keeps every level; the plan picks
// k from a memory budget.
#include "bfly.h"
#include "bf_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

namespace bfd {

constexpr int kThreads = 256;
constexpr int kChunk = 32;          // RHS per chunk
constexpr int kPad = kChunk + 1;    // padded chunk row (float2), conflict-free column reads
constexpr int kMaxGradPerThread = 16;

enum Form : int { FORM_XH = 0, FORM_X = 1 };

struct Unit {
    const float2 *X;    // parameter blocks, p x q row-major, block index first
    const float2 *src;  // input of the step: P side (XH) or Q side (X)
    float2 *dst;        // output of the step
    const float2 *ga;   // gradient: P-side vector (or null)
    const float2 *gb;   // gradient: Q-side vector
    float2 *grad;       // gradient output in the parameter layout (or null)
    int count, p, q, C; // C = 0 for a leaf
    int form, nrhs;
};

__device__ __forceinline__ int p_block(const Unit &a, int u, int c) {
    if (a.C == 0) return u;
    const int hi = u / a.C, lo = u - hi * a.C;
    return (2 * hi + c) * a.C + lo;
}
__device__ __forceinline__ float2 cmul(float2 x, float2 y) {
    return make_float2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
}
__device__ __forceinline__ float2 cmul_conj_a(float2 x, float2 y) {   // conj(x) * y
    return make_float2(x.x * y.x + x.y * y.y, x.x * y.y - x.y * y.x);
}
__device__ __forceinline__ float2 cmul_conj_b(float2 x, float2 y) {   // x * conj(y)
    return make_float2(x.x * y.x + x.y * y.y, x.y * y.x - x.x * y.y);
}
__device__ __forceinline__ void cadd(float2 &a, float2 b) {
    a.x += b.x;
    a.y += b.y;
}
// y += x * z, y += conj(x) * z, y += x * conj(z): four FMAs each.
__device__ __forceinline__ void cmac(float2 &y, float2 x, float2 z) {
    y.x = fmaf(x.x, z.x, fmaf(-x.y, z.y, y.x));
    y.y = fmaf(x.x, z.y, fmaf(x.y, z.x, y.y));
}
__device__ __forceinline__ void cmac_conj_a(float2 &y, float2 x, float2 z) {
    y.x = fmaf(x.x, z.x, fmaf(x.y, z.y, y.x));
    y.y = fmaf(x.x, z.y, fmaf(-x.y, z.x, y.y));
}
__device__ __forceinline__ void cmac_conj_b(float2 &y, float2 x, float2 z) {
    y.x = fmaf(x.x, z.x, fmaf(x.y, z.y, y.x));
    y.y = fmaf(x.y, z.x, fmaf(-x.x, z.y, y.y));
}
constexpr int kTile = 4;   // outputs per warp lane in the step loops (register tile)

// One CTA per unit; RHS in chunks of kChunk.  Shared memory: the unit's
// parameter blocks, its P-side chunk (count p rows) and Q-side chunk (q rows).
// GPT: gradient entries per thread (0 for a forward step), so a step's
// registers, and with them the CTAs per SM, follow its block size.
template <int GPT>
__global__ void __launch_bounds__(kThreads) unit_kernel(const Unit a) {
    extern __shared__ float2 sm[];
    const int u = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int np = a.count * a.p, nx = np * a.q;
    float2 *Xs = sm;                    // [c][row][col]
    float2 *Ps = Xs + nx;               // [c*p + row][kPad]
    float2 *Qs = Ps + (size_t)np * kPad;   // [col][kPad]
    for (int e = tid; e < nx; e += kThreads) {
        const int c = e / (a.p * a.q), rem = e - c * a.p * a.q;
        Xs[e] = a.X[(size_t)p_block(a, u, c) * a.p * a.q + rem];
    }
    constexpr bool grad = GPT > 0;
    constexpr int NG = GPT > 0 ? GPT : 1;
    const float2 *pv = a.form == FORM_XH ? a.src : a.ga;
    const float2 *qv = a.form == FORM_X ? a.src : a.gb;
    const bool needP = a.form == FORM_XH || grad, needQ = a.form == FORM_X || grad;
    float2 acc[NG];
#pragma unroll
    for (int t = 0; t < NG; ++t) acc[t] = make_float2(0.f, 0.f);
    for (int j0 = 0; j0 < a.nrhs; j0 += kChunk) {
        const int nc = min(kChunk, a.nrhs - j0);
        __syncthreads();
        if (needP)
            for (int rr = warp; rr < np; rr += kThreads / 32) {
                const int c = rr / a.p, row = rr - c * a.p;
                const size_t pos = (size_t)p_block(a, u, c) * a.p + row;
                Ps[rr * kPad + lane] = lane < nc ? pv[pos * a.nrhs + j0 + lane] : make_float2(0.f, 0.f);
            }
        if (needQ)
            for (int o = warp; o < a.q; o += kThreads / 32) {
                const size_t pos = (size_t)u * a.q + o;
                Qs[o * kPad + lane] = lane < nc ? qv[pos * a.nrhs + j0 + lane] : make_float2(0.f, 0.f);
            }
        __syncthreads();
        // Each lane is one RHS; a warp takes kTile consecutive outputs at a time
        // (fewer when there are too few to give every warp kTile), so each
        // shared-memory value of the lane's vector feeds kTile multiply-adds.
        if (a.form == FORM_XH) {   // Q[o][j] = sum_c sum_row conj(X_c[row][o]) P_c[row][j]
            const int tile = max(1, min(kTile, a.q / (kThreads / 32)));
            for (int ob = warp * tile; ob < a.q; ob += tile * (kThreads / 32)) {
                float2 y[kTile];
#pragma unroll
                for (int i = 0; i < kTile; ++i) y[i] = make_float2(0.f, 0.f);
                for (int rr = 0; rr < np; ++rr) {
                    const float2 pv = Ps[rr * kPad + lane];
                    const float2 *xr = Xs + rr * a.q + ob;
#pragma unroll
                    for (int i = 0; i < kTile; ++i)
                        if (i < tile && ob + i < a.q) cmac_conj_a(y[i], xr[i], pv);
                }
#pragma unroll
                for (int i = 0; i < kTile; ++i)
                    if (i < tile && ob + i < a.q && lane < nc)
                        a.dst[((size_t)u * a.q + ob + i) * a.nrhs + j0 + lane] = y[i];
            }
        } else {                   // P_c[row][j] = sum_o X_c[row][o] Q[o][j]
            const int tile = max(1, min(kTile, np / (kThreads / 32)));
            for (int rb = warp * tile; rb < np; rb += tile * (kThreads / 32)) {
                float2 y[kTile];
#pragma unroll
                for (int i = 0; i < kTile; ++i) y[i] = make_float2(0.f, 0.f);
                for (int o = 0; o < a.q; ++o) {
                    const float2 qv = Qs[o * kPad + lane];
#pragma unroll
                    for (int i = 0; i < kTile; ++i)
                        if (i < tile && rb + i < np) cmac(y[i], Xs[(rb + i) * a.q + o], qv);
                }
#pragma unroll
                for (int i = 0; i < kTile; ++i) {
                    const int rr = rb + i;
                    if (i < tile && rr < np && lane < nc) {
                        const int c = rr / a.p, row = rr - c * a.p;
                        a.dst[((size_t)p_block(a, u, c) * a.p + row) * a.nrhs + j0 + lane] = y[i];
                    }
                }
            }
        }
        if (grad) {                // Xbar_c[row][o] += sum_j P_c[row][j] conj(Q[o][j])
#pragma unroll
            for (int t = 0; t < NG; ++t) {
                const int e = tid + t * kThreads;
                if (e < nx) {
                    const int rr = e / a.q, o = e - rr * a.q;
                    const float2 *pr = Ps + rr * kPad, *qr = Qs + o * kPad;
                    float2 s = acc[t];
                    for (int j = 0; j < nc; ++j) cmac_conj_b(s, pr[j], qr[j]);
                    acc[t] = s;
                }
            }
        }
    }
    if (grad) {
#pragma unroll
        for (int t = 0; t < NG; ++t) {
            const int e = tid + t * kThreads;
            if (e < nx) {
                const int c = e / (a.p * a.q), rem = e - c * a.p * a.q;
                a.grad[(size_t)p_block(a, u, c) * a.p * a.q + rem] = acc[t];
            }
        }
    }
}

// M^h (Eq. KeqUMV): forward w_{i,j} = S_{i,j} t_{j,i}; backward
// tbar_{j,i} = S_{i,j} wbar_{i,j} and Sbar_{i,j} = Re sum over RHS conj(wbar_{i,j}) t_{j,i}.
// One warp per (i, j, k), lanes over the RHS.
__global__ void middle_kernel(const float *S, const float2 *src, float2 *dst, const float2 *t_saved, float *gradS,
                              int m, int r, int nrhs, int backward) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (long long)m * m * r) return;
    const int k = (int)(w % r);
    const long long ij = w / r;
    const int i = (int)(ij / m), j = (int)(ij - (long long)i * m);
    const long long pw = ((long long)i * m + j) * r + k;   // w_{i,j} entry k
    const long long pt = ((long long)j * m + i) * r + k;   // t_{j,i} entry k
    const float s = S[pw];
    float g = 0.f;
    for (int n = lane; n < nrhs; n += 32) {
        if (!backward) {
            const float2 v = src[pt * nrhs + n];
            dst[pw * nrhs + n] = make_float2(s * v.x, s * v.y);
        } else {
            const float2 wb = src[pw * nrhs + n];
            dst[pt * nrhs + n] = make_float2(s * wb.x, s * wb.y);
            const float2 t = t_saved[pt * nrhs + n];
            g += wb.x * t.x + wb.y * t.y;
        }
    }
    if (backward) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) g += __shfl_xor_sync(0xffffffffu, g, off);
        if (lane == 0) gradS[pw] = g;
    }
}

// Column-major (RHS j at in + j ld) <-> position-major (position * nrhs + j).
__global__ void to_posmajor(const float2 *in, long long ld, float2 *out, long long P, int nrhs) {
    __shared__ float2 tile[32][33];
    const long long p0 = (long long)blockIdx.x * 32;
    const int j0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const long long p = p0 + threadIdx.x;
        const int j = j0 + y;
        if (p < P && j < nrhs) tile[y][threadIdx.x] = in[(long long)j * ld + p];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const long long p = p0 + y;
        const int j = j0 + threadIdx.x;
        if (p < P && j < nrhs) out[p * nrhs + j] = tile[threadIdx.x][y];
    }
}
__global__ void from_posmajor(const float2 *in, float2 *out, long long ld, long long P, int nrhs) {
    __shared__ float2 tile[32][33];
    const long long p0 = (long long)blockIdx.x * 32;
    const int j0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const long long p = p0 + y;
        const int j = j0 + threadIdx.x;
        if (p < P && j < nrhs) tile[y][threadIdx.x] = in[p * nrhs + j];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int j = j0 + y;
        const long long p = p0 + threadIdx.x;
        if (p < P && j < nrhs) out[(long long)j * ld + p] = tile[threadIdx.x][y];
    }
}

size_t unit_smem(int count, int p, int q) {
    return ((size_t)count * p * q + (size_t)count * p * kPad + (size_t)q * kPad) * sizeof(float2);
}

}  // namespace bfd

struct bf_diff_s {
    int L, n0, r, h, m, nrhs_max, nf, k;
    long long N, R;
    float2 *work = nullptr;   // 2 temporaries + (k-1) segment vectors, each max(N, R) x nrhs_max
    size_t work_vec = 0;      // entries per work vector
};

namespace {

bf_status cuda_status(cudaError_t e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA;
}

long long vec_len(const bf_diff_s &P, int f) { return (f == 0 || f == P.nf) ? P.N : P.R; }

// Offsets (entries) of the saved inputs x_f, f % k == 0; total in *total.
std::vector<long long> saved_offsets(const bf_diff_s &P, int k, int nrhs, long long *total) {
    std::vector<long long> off(P.nf, -1);
    long long acc = 0;
    for (int f = 0; f < P.nf; f += k) {
        off[f] = acc;
        acc += vec_len(P, f) * nrhs;
    }
    *total = acc;
    return off;
}

struct Ctx {
    const bf_diff_s &P;
    const bf_dfactors &F;
    int nrhs;
    cudaStream_t s;
};

cudaError_t launch_unit(const Ctx &c, int f, int form, const float2 *src, float2 *dst, const float2 *ga,
                        const float2 *gb, float2 *grad) {
    const bf_diff_s &P = c.P;
    bfd::Unit a;
    std::memset(&a, 0, sizeof(a));
    a.src = src;
    a.dst = dst;
    a.ga = ga;
    a.gb = gb;
    a.grad = grad;
    a.form = form;
    a.nrhs = c.nrhs;
    long long nunits;
    if (f == 0 || f == P.nf - 1) {   // leaf V^L (f = 0) or U^L
        a.X = static_cast<const float2 *>(f == 0 ? c.F.VL : c.F.UL);
        a.count = 1;
        a.p = P.n0;
        a.q = P.r;
        a.C = 0;
        nunits = 1LL << P.L;
    } else {                          // transfer level
        const bool is_h = f <= P.h;
        const int l = is_h ? P.L - f : f - 2;
        a.X = static_cast<const float2 *>(is_h ? c.F.H[l - P.h] : c.F.G[l - P.h]);
        a.count = 2;
        a.p = P.r;
        a.q = 2 * P.r;
        a.C = 1 << (P.L - l - 1);
        nunits = 1LL << (P.L - 1);
    }
    const size_t smem = bfd::unit_smem(a.count, a.p, a.q);
    const int nx = a.count * a.p * a.q;
    if (!grad) bfd::unit_kernel<0><<<(unsigned)nunits, bfd::kThreads, smem, c.s>>>(a);
    else if (nx <= 4 * bfd::kThreads) bfd::unit_kernel<4><<<(unsigned)nunits, bfd::kThreads, smem, c.s>>>(a);
    else if (nx <= 8 * bfd::kThreads) bfd::unit_kernel<8><<<(unsigned)nunits, bfd::kThreads, smem, c.s>>>(a);
    else bfd::unit_kernel<16><<<(unsigned)nunits, bfd::kThreads, smem, c.s>>>(a);
    return cudaGetLastError();
}

// Forward step f: x_{f+1} = factor_f(x_f).
cudaError_t step_forward(const Ctx &c, int f, const float2 *x, float2 *y) {
    const bf_diff_s &P = c.P;
    if (f == P.h + 1) {
        const long long warps = (long long)P.m * P.m * P.r;
        bfd::middle_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, c.s>>>(c.F.S, x, y, nullptr, nullptr, P.m,
                                                                                  P.r, c.nrhs, 0);
        return cudaGetLastError();
    }
    const bool form_xh = f <= P.h;   // V^L and the H levels use their blocks conjugate-transposed
    return launch_unit(c, f, form_xh ? bfd::FORM_XH : bfd::FORM_X, x, y, nullptr, nullptr, nullptr);
}

// Backward step f: xbar_f from xbar_{f+1} (= yb), the factor's gradient from
// its saved input x_f.
cudaError_t step_backward(const Ctx &c, const bf_dgrads &G, int f, const float2 *x, const float2 *yb, float2 *xb) {
    const bf_diff_s &P = c.P;
    if (f == P.h + 1) {
        const long long warps = (long long)P.m * P.m * P.r;
        bfd::middle_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, c.s>>>(c.F.S, yb, xb, x, G.S, P.m, P.r,
                                                                                  c.nrhs, 1);
        return cudaGetLastError();
    }
    float2 *grad;
    if (f == 0) grad = static_cast<float2 *>(G.VL);
    else if (f == P.nf - 1) grad = static_cast<float2 *>(G.UL);
    else if (f <= P.h) grad = static_cast<float2 *>(G.H[P.L - f - P.h]);
    else grad = static_cast<float2 *>(G.G[f - 2 - P.h]);
    if (f <= P.h)   // V, H: xbar = X ybar (form X: Q side = ybar), Xbar = x ybar^*
        return launch_unit(c, f, bfd::FORM_X, yb, xb, x, yb, grad);
    // G, U: xbar = X^* ybar (form XH: P side = ybar), Xbar = ybar x^*
    return launch_unit(c, f, bfd::FORM_XH, yb, xb, yb, x, grad);
}

bool valid_factors(const bf_diff_s &P, const bf_dfactors *f) {
    if (!f || !f->VL || !f->UL || !f->S) return false;
    if (P.h > 0 && (!f->H || !f->G)) return false;
    for (int t = 0; t < P.h; ++t)
        if (!f->H[t] || !f->G[t]) return false;
    return true;
}

cudaError_t transpose_in(const bf_diff_s &P, const float2 *in, long long ld, float2 *out, long long len, int nrhs,
                         cudaStream_t s) {
    const dim3 grid((unsigned)((len + 31) / 32), (unsigned)((nrhs + 31) / 32));
    bfd::to_posmajor<<<grid, dim3(32, 8), 0, s>>>(in, ld, out, len, nrhs);
    (void)P;
    return cudaGetLastError();
}
cudaError_t transpose_out(const bf_diff_s &P, const float2 *in, float2 *out, long long ld, long long len, int nrhs,
                          cudaStream_t s) {
    const dim3 grid((unsigned)((len + 31) / 32), (unsigned)((nrhs + 31) / 32));
    bfd::from_posmajor<<<grid, dim3(32, 8), 0, s>>>(in, out, ld, len, nrhs);
    (void)P;
    return cudaGetLastError();
}

}  // namespace

extern "C" {

bf_status bf_diff_create(bf_diff *out, const bf_diff_desc *d) {
    if (!out) return BF_ERR_INVALID;
    *out = nullptr;
    if (!d || d->L < 0 || (d->L & 1) || d->leaf < 1 || d->r < 1 || d->nrhs_max < 1 || d->stride < 0)
        return BF_ERR_INVALID;
    if (d->L > 24 || d->r > 32 || d->leaf > 64) return BF_ERR_UNSUPPORTED;
    const int p = std::max(d->leaf, d->r), q = 2 * d->r;
    if ((size_t)std::max(2 * d->r * q, d->leaf * d->r) > (size_t)bfd::kMaxGradPerThread * bfd::kThreads)
        return BF_ERR_UNSUPPORTED;
    if (bfd::unit_smem(2, d->r, q) > 227 * 1024 || bfd::unit_smem(1, d->leaf, d->r) > 227 * 1024)
        return BF_ERR_UNSUPPORTED;
    (void)p;
    bf_diff_s *P = new (std::nothrow) bf_diff_s();
    if (!P) return BF_ERR_NOMEM;
    P->L = d->L;
    P->n0 = d->leaf;
    P->r = d->r;
    P->h = d->L / 2;
    P->m = 1 << P->h;
    P->nrhs_max = d->nrhs_max;
    P->nf = d->L + 3;
    P->N = (long long)d->leaf << d->L;
    P->R = (1LL << d->L) * d->r;
    const long long vec = std::max(P->N, P->R) * d->nrhs_max;
    // Checkpoint stride: forced, or the smallest k whose saved inputs plus
    // recompute segment (k - 1 vectors) fit the budget (0: keep every input),
    // else the k with the least memory.
    int k = d->stride;
    if (k == 0) {
        k = 1;
        if (d->saved_budget > 0) {
            long long best = -1;
            int bestk = 1;
            bool found = false;
            for (int cand = 1; cand <= P->nf; ++cand) {
                long long tot = 0;
                saved_offsets(*P, cand, d->nrhs_max, &tot);
                const long long mem = (tot + (long long)(cand - 1) * P->R * d->nrhs_max) * 8;
                if (mem <= (long long)d->saved_budget) {
                    k = cand;
                    found = true;
                    break;
                }
                if (best < 0 || mem < best) {
                    best = mem;
                    bestk = cand;
                }
            }
            if (!found) k = bestk;
        }
    }
    P->k = std::min(std::max(k, 1), P->nf);
    P->work_vec = (size_t)vec;
    const size_t nvec = 2 + (size_t)(P->k - 1);
    // One attribute value shared by every plan: the opt-in maximum (an upper
    // bound; each launch requests only its unit's shared memory).
    if (cudaFuncSetAttribute(bfd::unit_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(bfd::unit_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(bfd::unit_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess ||
        cudaFuncSetAttribute(bfd::unit_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess) {
        cudaGetLastError();
        delete P;
        return BF_ERR_CUDA;
    }
    cudaError_t e = cudaMalloc(&P->work, nvec * P->work_vec * sizeof(float2));
    if (e != cudaSuccess) {
        delete P;
        return cuda_status(e);
    }
    *out = P;
    return BF_OK;
}

bf_status bf_diff_destroy(bf_diff p) {
    if (!p) return BF_OK;
    cudaDeviceSynchronize();
    cudaFree(p->work);
    cudaGetLastError();
    delete p;
    return BF_OK;
}

int bf_diff_stride(bf_diff p) { return p ? p->k : 0; }

size_t bf_diff_saved_bytes(bf_diff p, int nrhs) {
    if (!p || nrhs < 1 || nrhs > p->nrhs_max) return 0;
    long long tot = 0;
    saved_offsets(*p, p->k, nrhs, &tot);
    return (size_t)tot * sizeof(float2);
}

bf_status bf_diff_forward(bf_diff p, const bf_dfactors *f, const void *g, void *u, int nrhs, long long ld,
                          void *saved, cudaStream_t s) {
    bfint::NvtxRange range("bf_diff_forward");
    if (!p || !g || !u || !saved || nrhs < 1 || nrhs > p->nrhs_max || ld < p->N || !valid_factors(*p, f))
        return BF_ERR_INVALID;
    long long tot = 0;
    const std::vector<long long> off = saved_offsets(*p, p->k, nrhs, &tot);
    float2 *sv = static_cast<float2 *>(saved);
    float2 *tmp[2] = {p->work, p->work + p->work_vec};
    const Ctx c{*p, *f, nrhs, s};
    cudaError_t e = transpose_in(*p, static_cast<const float2 *>(g), ld, sv + off[0], p->N, nrhs, s);
    const float2 *cur = sv + off[0];
    int ti = 0;
    for (int fi = 0; fi < p->nf && e == cudaSuccess; ++fi) {
        float2 *next = (fi + 1 < p->nf && off[fi + 1] >= 0) ? sv + off[fi + 1] : tmp[ti];
        if (next == tmp[ti]) ti ^= 1;
        e = step_forward(c, fi, cur, next);
        cur = next;
    }
    if (e == cudaSuccess) e = transpose_out(*p, cur, static_cast<float2 *>(u), ld, p->N, nrhs, s);
    return e == cudaSuccess ? BF_OK : cuda_status(e);
}

bf_status bf_diff_backward(bf_diff p, const bf_dfactors *f, const void *ubar, void *gbar, int nrhs, long long ld,
                           const void *saved, const bf_dgrads *grads, cudaStream_t s) {
    bfint::NvtxRange range("bf_diff_backward");
    if (!p || !ubar || !gbar || !saved || !grads || nrhs < 1 || nrhs > p->nrhs_max || ld < p->N ||
        !valid_factors(*p, f))
        return BF_ERR_INVALID;
    if (!grads->VL || !grads->UL || !grads->S || (p->h > 0 && (!grads->H || !grads->G))) return BF_ERR_INVALID;
    for (int t = 0; t < p->h; ++t)
        if (!grads->H[t] || !grads->G[t]) return BF_ERR_INVALID;
    long long tot = 0;
    const std::vector<long long> off = saved_offsets(*p, p->k, nrhs, &tot);
    const float2 *sv = static_cast<const float2 *>(saved);
    float2 *tmp[2] = {p->work, p->work + p->work_vec};
    float2 *seg = p->work + 2 * p->work_vec;   // x_{s+1} .. x_{s+k-1} of the current segment
    const Ctx c{*p, *f, nrhs, s};
    cudaError_t e = transpose_in(*p, static_cast<const float2 *>(ubar), ld, tmp[0], p->N, nrhs, s);
    int di = 0;   // tmp[di] holds the current upstream gradient
    for (int fi = p->nf - 1; fi >= 0 && e == cudaSuccess;) {
        const int s0 = (fi / p->k) * p->k;   // segment start (a checkpoint)
        const float2 *xs = sv + off[s0];
        const float2 *cur = xs;
        for (int q = s0; q < fi && e == cudaSuccess; ++q) {   // recompute x_{s0+1} .. x_fi
            float2 *next = seg + (size_t)(q - s0) * p->work_vec;
            e = step_forward(c, q, cur, next);
            cur = next;
        }
        for (int q = fi; q >= s0 && e == cudaSuccess; --q) {
            const float2 *x = q == s0 ? xs : seg + (size_t)(q - s0 - 1) * p->work_vec;
            e = step_backward(c, *grads, q, x, tmp[di], tmp[di ^ 1]);
            di ^= 1;
        }
        fi = s0 - 1;
    }
    if (e == cudaSuccess) e = transpose_out(*p, tmp[di], static_cast<float2 *>(gbar), ld, p->N, nrhs, s);
    return e == cudaSuccess ? BF_OK : cuda_status(e);
}

}  // extern "C"
