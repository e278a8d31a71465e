// 2D (quadtree) butterfly factorizations: plan and apply, sm_103a.
//
// The 2D factorization has the 1D form K ~ U^L G^{L-1} ... G^h M^h
// (H^h)^* ... (H^{L-1})^* (V^L)^* with four children per tree node (the
// extension to higher dimensions that Sec. 1.2 points to).  Level l carries,
// for every pair (node of one tree at level l, node of the other at level
// L-l), a vector of r_l = min(r, N/4^l) entries.  One transfer level acts on
// closed groups of four such vectors:
//   splitting (G^l):  [w_{i,4j'} .. w_{i,4j'+3}] -> w_{4i+c,j'} = G^l_{4i+c,j'} [..],
//   merging ((H^l)^*): t_{4j+c,i'} (c = 0..3) -> [t_{j,4i'} .. t_{j,4i'+3}] = sum_c (H^l_{4j+c,i'})^* t_{4j+c,i'},
// i.e. per group one dense complex block of (4 r_out) x (4 r_in).  The plan
// forms these blocks in FP64 when it is created -- the leaf factor folded
// into the first and last pass, the real diagonal S^h of M^h into the first
// splitting pass -- so the apply is L passes of the same operation:
//     out_stack(group) = F(group) in_stack(group),
// where the four input (output) blocks of group (A, B) sit at block indices
// a A + b B + c s (c = 0..3) of the level's vector, with block size r_in
// (r_out) or n0 at the leaves.  The vectors at level l are ordered (node of
// the first tree, node of the second), so a group's four blocks are either
// consecutive or 4^{L-l-1} apart; the first splitting pass reads the merging
// half's output transposed (M^h).
//
// Kernels.  Thread o of a group accumulates output o of the stack in FP32
// while it streams column o of F (stored k-major, F^T, so a warp's loads of
// one k are contiguous), the input stack staged in shared memory:
//  * one vector (quad_gemv_kernel): one group per thread block, a stream over
//    the blocks (HBM-bound);
//  * 2..31 vectors and the two levels that touch the caller's vectors in
//    larger calls (quad_pass_kernel<NT>): tiles of NT vectors, several groups
//    per block for small stacks, planar-tile outputs staged through shared
//    memory;
//  * 32 or more vectors: every other level on the tensor-core core
//    (bf_tc.cuh, LD_QUAD / ST_QUAD, launched through bf_internal.h), with
//    planar 128-vector tiles between all levels.
#include <cuda_runtime.h>

#include <algorithm>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "../../include/bfly.h"
#include "bf_internal.h"

namespace bfq {

constexpr int kMaxL = 12;
constexpr int kMaxStack = 128;   // Kin, Nout per group (4 r_l, 4 n0)

struct Pass {
    const float2 *F;             // per group: Kin x Nout complex, k-major (F^T)
    int nA, nB;                  // groups (A, B): A < nA, B < nB
    long long ain, bin, sin;     // block index of input child c: ain A + bin B + c sin
    long long aout, bout, sout;
    int bsz_in, bsz_out;         // entries per block
    int Kin, Nout;               // 4 bsz_in, 4 bsz_out
    int in_planar, out_planar;   // vectors as planar 128-RHS tiles of R positions (else RHS-major with ld)
    long long R;
};

// Address of (vector j, position pos) in a planar tile buffer: tile j / 128
// holds, per position, the 128 real parts then the 128 imaginary parts.
__device__ __forceinline__ long long planar_at(long long R, long long j, long long pos) {
    return ((j >> 7) * R + pos) * 256 + (j & 127);
}

// One vector at a time: a stream over the blocks, one group per thread block
// (as many thread blocks in flight as the SM holds), one output row per thread.
__global__ void __launch_bounds__(128) quad_gemv_kernel(const Pass p, const float2 *__restrict__ in,
                                                        float2 *__restrict__ out) {
    extern __shared__ float2 xs[];   // [Kin]
    const long long g = blockIdx.x;
    const int A = (int)(g / p.nB), B = (int)(g - (long long)A * p.nB);
    const long long in_base = p.ain * A + p.bin * B;
    for (int k = threadIdx.x; k < p.Kin; k += blockDim.x) {
        const int c = k / p.bsz_in, x = k - c * p.bsz_in;
        xs[k] = in[(in_base + c * p.sin) * p.bsz_in + x];
    }
    __syncthreads();
    const long long out_base = p.aout * A + p.bout * B;
    const float2 *Fg = p.F + g * (long long)p.Kin * p.Nout;
    for (int o = threadIdx.x; o < p.Nout; o += blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        const float2 *f = Fg + o;
#pragma unroll 4
        for (int k = 0; k < p.Kin; ++k) {
            const float2 fv = __ldg(f + (long long)k * p.Nout);
            const float2 xv = xs[k];
            acc.x = fmaf(fv.x, xv.x, fmaf(-fv.y, xv.y, acc.x));
            acc.y = fmaf(fv.x, xv.y, fmaf(fv.y, xv.x, acc.y));
        }
        const int c = o / p.bsz_out, x = o - c * p.bsz_out;
        out[(out_base + c * p.sout) * p.bsz_out + x] = acc;
    }
}

// NT vectors per thread block (2..32), RHS-major or planar tiles.
template <int NT>
__global__ void __launch_bounds__(128) quad_pass_kernel(const Pass p, const float2 *__restrict__ in, long long ld_in,
                                                        float2 *__restrict__ out, long long ld_out, int nrhs, int gpb,
                                                        int tpg) {
    // gpb consecutive groups per thread block, tpg threads per group (small stacks
    // share a block so its threads stay busy and its accesses stay contiguous)
    extern __shared__ float2 xs[];   // [gpb][Kin][NT] inputs, then (planar stores) [gpb][Nout][NT] outputs
    const int ntiles = (nrhs + NT - 1) / NT;
    const long long gb = blockIdx.x / ntiles;
    const int tile = (int)(blockIdx.x - gb * ntiles);
    const long long ngroups = (long long)p.nA * p.nB, g0 = gb * gpb;
    const int rhs0 = tile * NT, nt = min(NT, nrhs - rhs0);
    const int per = p.Kin * NT;
    for (int idx = threadIdx.x; idx < gpb * per; idx += blockDim.x) {
        // consecutive threads: consecutive positions of consecutive groups of one
        // vector (RHS-major), or consecutive vectors at one position (planar)
        int gi, j, k;
        if (NT >= 8 && p.in_planar) {
            j = idx % NT;
            k = (idx / NT) % p.Kin;
            gi = idx / per;
        } else {
            k = idx % p.Kin;
            gi = (idx / p.Kin) % gpb;
            j = idx / (p.Kin * gpb);
        }
        const long long g = g0 + gi;
        float2 v = make_float2(0.f, 0.f);
        if (j < nt && g < ngroups) {
            const int A = (int)(g / p.nB), B = (int)(g - (long long)A * p.nB);
            const int c = k / p.bsz_in, x = k - c * p.bsz_in;
            const long long pos = (p.ain * A + p.bin * B + c * p.sin) * p.bsz_in + x;
            if (NT >= 8 && p.in_planar) {
                const float *f = reinterpret_cast<const float *>(in) + planar_at(p.R, rhs0 + j, pos);
                v = make_float2(f[0], f[128]);
            } else {
                v = in[(long long)(rhs0 + j) * ld_in + pos];
            }
        }
        xs[(gi * p.Kin + k) * NT + j] = v;
    }
    __syncthreads();
    const int gi = threadIdx.x / tpg;
    const long long g = g0 + gi;
    const bool active = gi < gpb && g < ngroups;
    const int A = (int)(g / p.nB), B = (int)(g - (long long)A * p.nB);
    const long long out_base = p.aout * A + p.bout * B;
    const float2 *Fg = p.F + g * (long long)p.Kin * p.Nout;
    const float2 *xg = xs + gi * per;
    float2 *ys = xs + (size_t)gpb * per;   // planar stores: outputs staged here
    for (int o = threadIdx.x - gi * tpg; active && o < p.Nout; o += tpg) {
        float2 acc[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j] = make_float2(0.f, 0.f);
        const float2 *f = Fg + o;
#pragma unroll 4
        for (int k = 0; k < p.Kin; ++k) {
            const float2 fv = __ldg(f + (long long)k * p.Nout);
            const float2 *xk = xg + k * NT;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const float2 xv = xk[j];
                acc[j].x = fmaf(fv.x, xv.x, fmaf(-fv.y, xv.y, acc[j].x));
                acc[j].y = fmaf(fv.x, xv.y, fmaf(fv.y, xv.x, acc[j].y));
            }
        }
        if (NT >= 8 && p.out_planar) {
#pragma unroll
            for (int j = 0; j < NT; ++j) ys[(gi * p.Nout + o) * NT + j] = acc[j];
            continue;
        }
        const int c = o / p.bsz_out, x = o - c * p.bsz_out;
        const long long pos = (out_base + c * p.sout) * p.bsz_out + x;
#pragma unroll
        for (int j = 0; j < NT; ++j)
            if (j < nt) out[(long long)(rhs0 + j) * ld_out + pos] = acc[j];
    }
    // (planar tiles are used only between the tensor-core levels, with 32 or more
    // vectors per call and so tiles of NT >= 8)
    if constexpr (NT < 8) return;
    if (!p.out_planar) return;
    // planar stores through shared memory: consecutive threads write consecutive
    // vectors of one output position (contiguous floats of one tile row)
    __syncthreads();
    for (int idx = threadIdx.x; idx < gpb * p.Nout * NT; idx += blockDim.x) {
        const int j = idx % NT, row = idx / NT, gj = row / p.Nout, oo = row - gj * p.Nout;
        const long long gg = g0 + gj;
        if (j >= nt || gg >= ngroups) continue;
        const int A2 = (int)(gg / p.nB), B2 = (int)(gg - (long long)A2 * p.nB);
        const int c = oo / p.bsz_out, x = oo - c * p.bsz_out;
        const long long pos = ((p.aout * A2 + p.bout * B2) + c * p.sout) * p.bsz_out + x;
        float *f = reinterpret_cast<float *>(out) + planar_at(p.R, rhs0 + j, pos);
        const float2 v = ys[idx];
        f[0] = v.x;
        f[128] = v.y;
    }
}

struct HostPass {
    Pass p;
    float2 *d = nullptr;
    // tensor-core form of the same level (batches of 32 or more vectors)
    bool tc = false;
    int parts = 1, chunks = 1, Nc = 0, Kc = 0;   // output parts of Nc, K-chunks of Kc
    float *dtc = nullptr;                        // [Re F; Im F] per (group, part, chunk)
    uint16_t *d16 = nullptr;                     // the same split into BF16 parts (BF16 rungs)
    int d16_parts = 0;
};

}  // namespace

struct bf_quad_s {
    int L = 0, n0 = 0, r = 0, h = 0, nrhs_max = 0;
    long long N = 0, m = 0, Rmax = 0;
    int ranks[bfq::kMaxL + 1] = {};
    std::vector<bfq::HostPass> fwd, adj;
    float2 *ws[2] = {nullptr, nullptr};
    size_t device_bytes = 0;
    int num_sms = 1;
    bool tc = false;          // tensor-core passes built (nrhs_max >= 32)
    int tc_min = 32;          // smallest chunk of vectors the tensor-core path serves
    int tc_split = 3, tc_bf16 = 0;
    int kc_max = 64;          // tensor-core K-chunk limit (BF_QUAD_KC: 32 or 64)
    int inject_stall = 0;     // failure-detection test hook (BF_INJECT_STALL=1 at creation)
    int device = -1;          // CUDA device the plan's memory lives on
    unsigned *d_err = nullptr;
};

namespace {

using cd = std::complex<double>;

bf_status qfail(cudaError_t) {
    cudaGetLastError();
    return BF_ERR_CUDA;
}

// Factor entry readers over the caller's host arrays (complex64 or complex128).
struct Reader {
    int dtype;
    cd at(const void *base, long long idx) const {
        if (dtype == BF_C128) {
            const double *p = static_cast<const double *>(base) + 2 * idx;
            return cd(p[0], p[1]);
        }
        const float *p = static_cast<const float *>(base) + 2 * idx;
        return cd(p[0], p[1]);
    }
    double real(const void *base, long long idx) const {
        return dtype == BF_C128 ? static_cast<const double *>(base)[idx] : (double)static_cast<const float *>(base)[idx];
    }
};

long long pow4(int e) { return 1LL << (2 * e); }

// Runs fn(g) for g in [0, n) on the host's cores.
template <class Fn>
void parallel_for(long long n, Fn fn) {
    const int nt = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t)
        pool.emplace_back([&, t] {
            for (long long g = n * t / nt; g < n * (t + 1) / nt; ++g) fn(g);
        });
    for (auto &th : pool) th.join();
}

// The passes of one direction.  Forward: merging with (H, V^L), splitting with
// (G, U^L), S[i][j]; adjoint: merging with (G, U^L), splitting with (H, V^L),
// S transposed (K^* = V^L H ... (M^h)^* (G^h)^* ... (U^L)^*).
bf_status build_direction(bf_quad_s &Q, const bf_factors &f, bool adjoint, std::vector<bfq::HostPass> &out) {
    const Reader rd{f.dtype};
    const int L = Q.L, h = Q.h, n0 = Q.n0;
    const int *rk = Q.ranks;
    const void *const *Dn = adjoint ? f.G : f.H;     // merging transfer blocks
    const void *leafDn = adjoint ? f.UL : f.VL;
    const void *const *Up = adjoint ? f.H : f.G;     // splitting transfer blocks
    const void *leafUp = adjoint ? f.VL : f.UL;
    const long long m = Q.m;
    for (int half = 0; half < 2; ++half) {
        for (int s = 0; s < L - h; ++s) {
            const int lv = half == 0 ? L - 1 - s : h + s;
            const long long nA = pow4(lv), nB = pow4(L - lv - 1);
            bfq::Pass p{};
            p.nA = (int)nA;
            p.nB = (int)nB;
            const int r0 = rk[lv], r1 = rk[lv + 1];
            const bool leaf = lv == L - 1;
            if (half == 0) {   // merging: in blocks (4A + c) nB + B, out A 4nB + 4B + c
                p.ain = 4 * nB, p.bin = 1, p.sin = nB;
                p.aout = 4 * nB, p.bout = 4, p.sout = 1;
                p.bsz_in = leaf ? n0 : r1;
                p.bsz_out = r0;
            } else {           // splitting: in A 4nB + 4B + c (or M^h's transpose), out (4A + c) nB + B
                if (lv == h) p.ain = 1, p.bin = 4 * m, p.sin = m;
                else p.ain = 4 * nB, p.bin = 4, p.sin = 1;
                p.aout = 4 * nB, p.bout = 1, p.sout = nB;
                p.bsz_in = r0;
                p.bsz_out = leaf ? n0 : r1;
            }
            p.Kin = 4 * p.bsz_in;
            p.Nout = 4 * p.bsz_out;
            if (p.Kin > bfq::kMaxStack || p.Nout > bfq::kMaxStack) return BF_ERR_UNSUPPORTED;
            const long long ngroups = nA * nB;
            const size_t per = (size_t)p.Kin * p.Nout;
            // Tensor-core form: every pass but the two that touch the caller's vectors,
            // when the stack splits into parts / K-chunks of at most 64 that are
            // multiples of 16.
            bfq::HostPass hp;
            hp.p = p;
            const bool edge = (half == 0 && s == 0) || (half == 1 && s == L - h - 1);
            auto split64 = [](int D, int &n, int &each) {
                n = (D + 63) / 64;
                each = D / n;
                return D % n == 0 && each % 16 == 0;
            };
            // K-chunks of at most Q.kc_max.  Chunks of at most 32 positions get two
            // staging buffers (the next tile's copy overlaps this one's conversion),
            // but splitting a 96-wide stack into three of them instead of two of 48
            // measured slower (9.1 vs 7.7 ms per 128-vector apply at 256 x 256), so
            // the default is 64.
            auto split_k = [&](int D, int &n, int &each) {
                for (n = 1; n <= D / 16; ++n)
                    if (D % n == 0 && (each = D / n) <= Q.kc_max && each % 16 == 0) return true;
                return split64(D, n, each);
            };
            hp.tc = Q.tc && !edge && split_k(p.Kin, hp.chunks, hp.Kc) && split64(p.Nout, hp.parts, hp.Nc);
            const size_t tper = (size_t)2 * hp.Nc * hp.Kc;   // floats per (group, part, chunk) block
            std::vector<float> tch;
            if (hp.tc) {
                try {
                    tch.assign(tper * hp.parts * hp.chunks * ngroups, 0.f);
                } catch (const std::bad_alloc &) {
                    return BF_ERR_NOMEM;
                }
            }
            std::vector<float2> host;
            try {
                host.resize(per * ngroups);
            } catch (const std::bad_alloc &) {
                return BF_ERR_NOMEM;
            }
            const void *T = half == 0 ? Dn[lv - h] : Up[lv - h];
            parallel_for(ngroups, [&](long long g) {
                const long long A = g / nB, B = g - A * nB;
                float2 *Fg = host.data() + per * g;   // Fg[k * Nout + o]
                std::vector<cd> blk((size_t)p.Kin * p.Nout);   // blk[o * Kin + k]
                for (int c = 0; c < 4; ++c) {
                    const long long b = (4 * A + c) * nB + B;   // transfer block index of child c
                    const long long tb = b * r1 * 4 * r0;       // its first entry (r1 x 4 r0, row-major)
                    if (half == 0) {
                        // column block c: (T_b)^* (4 r0 x r1), times (leaf_{4A+c})^* (r_L x n0) at the leaves
                        for (int o = 0; o < 4 * r0; ++o)
                            for (int k = 0; k < p.bsz_in; ++k) {
                                cd v;
                                if (!leaf) {
                                    v = std::conj(rd.at(T, tb + (long long)k * 4 * r0 + o));
                                } else {
                                    for (int a = 0; a < r1; ++a)
                                        v += std::conj(rd.at(T, tb + (long long)a * 4 * r0 + o)) *
                                             std::conj(rd.at(leafDn, (b * n0 + k) * r1 + a));
                                }
                                blk[(size_t)o * p.Kin + c * p.bsz_in + k] = v;
                            }
                    } else {
                        // row block c: T_b (r1 x 4 r0), times leaf_{4A+c} (n0 x r_L) on the left at the leaves
                        for (int o = 0; o < p.bsz_out; ++o)
                            for (int k = 0; k < 4 * r0; ++k) {
                                cd v;
                                if (!leaf) {
                                    v = rd.at(T, tb + (long long)o * 4 * r0 + k);
                                } else {
                                    for (int a = 0; a < r1; ++a)
                                        v += rd.at(leafUp, (b * n0 + o) * r1 + a) * rd.at(T, tb + (long long)a * 4 * r0 + k);
                                }
                                if (lv == h) {   // M^h: column c' r_h + x carries S of block (row node, column node)
                                    const int cp = k / r0, x = k - cp * r0;
                                    const long long i = adjoint ? 4 * B + cp : A, j = adjoint ? A : 4 * B + cp;
                                    v *= rd.real(f.S, (i * m + j) * r0 + x);
                                }
                                blk[(size_t)(c * p.bsz_out + o) * p.Kin + k] = v;
                            }
                    }
                }
                for (int o = 0; o < p.Nout; ++o)
                    for (int k = 0; k < p.Kin; ++k) {
                        const cd v = blk[(size_t)o * p.Kin + k];
                        Fg[(size_t)k * p.Nout + o] = make_float2((float)v.real(), (float)v.imag());
                    }
                if (!hp.tc) return;
                // [Re F; Im F] of rows part*Nc.., columns chunk*Kc.. in the MMA operand layout
                for (int pp = 0; pp < hp.parts; ++pp)
                    for (int cc = 0; cc < hp.chunks; ++cc) {
                        float *tb = tch.data() + ((g * hp.parts + pp) * hp.chunks + cc) * tper;
                        for (int n = 0; n < 2 * hp.Nc; ++n)
                            for (int k = 0; k < hp.Kc; ++k) {
                                const cd v = blk[(size_t)(pp * hp.Nc + n % hp.Nc) * p.Kin + cc * hp.Kc + k];
                                tb[bfint::tc_boff(n, k, 2 * hp.Nc) / 4] = (float)(n < hp.Nc ? v.real() : v.imag());
                            }
                    }
            });
            if (cudaMalloc(&hp.d, host.size() * sizeof(float2)) != cudaSuccess) {
                cudaGetLastError();
                return BF_ERR_NOMEM;
            }
            out.push_back(hp);
            Q.device_bytes += host.size() * sizeof(float2);
            if (cudaMemcpy(hp.d, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
                return qfail(cudaErrorUnknown);
            out.back().p.F = hp.d;
            if (hp.tc) {
                if (cudaMalloc(&out.back().dtc, tch.size() * sizeof(float)) != cudaSuccess) {
                    cudaGetLastError();
                    out.back().dtc = nullptr;
                    return BF_ERR_NOMEM;
                }
                Q.device_bytes += tch.size() * sizeof(float);
                if (cudaMemcpy(out.back().dtc, tch.data(), tch.size() * sizeof(float), cudaMemcpyHostToDevice) !=
                    cudaSuccess)
                    return qfail(cudaErrorUnknown);
            }
        }
    }
    return BF_OK;
}

void free_quad(bf_quad_s *Q) {
    if (!Q) return;
    for (auto *d : {&Q->fwd, &Q->adj})
        for (auto &hp : *d) {
            cudaFree(hp.d);
            cudaFree(hp.dtc);
            cudaFree(hp.d16);
        }
    cudaFree(Q->ws[0]);
    cudaFree(Q->ws[1]);
    cudaFree(Q->d_err);
    delete Q;
}

template <int NT>
cudaError_t launch_pass(const bfq::Pass &p, const float2 *in, long long ld_in, float2 *out, long long ld_out, int nrhs,
                        cudaStream_t s) {
    const long long ntiles = (nrhs + NT - 1) / NT;
    // threads per group: Nout rounded up to a power of 2 (at most 128); groups per
    // block: as many as fill 128 threads within 48 KB of staging
    int tpg = 1;
    while (tpg < p.Nout && tpg < 128) tpg <<= 1;
    const size_t per = (size_t)(p.Kin + (p.out_planar ? p.Nout : 0)) * NT * sizeof(float2);
    const int gpb = (int)std::max<size_t>(1, std::min<size_t>(128 / tpg, 49152 / per));
    const int threads = gpb > 1 ? gpb * tpg : std::min(128, (p.Nout + 31) / 32 * 32);
    if (gpb == 1) tpg = threads;
    const long long ngroups = (long long)p.nA * p.nB;
    const long long blocks = (ngroups + gpb - 1) / gpb * ntiles;
    bfq::quad_pass_kernel<NT><<<(unsigned)blocks, threads, per * gpb, s>>>(p, in, ld_in, out, ld_out, nrhs, gpb, tpg);
    return cudaGetLastError();
}

cudaError_t run_gemv(const bfq::Pass &p, const float2 *in, float2 *out, cudaStream_t s) {
    const int threads = std::min(128, (p.Nout + 31) / 32 * 32);
    bfq::quad_gemv_kernel<<<(unsigned)((long long)p.nA * p.nB), threads, (size_t)p.Kin * sizeof(float2), s>>>(p, in,
                                                                                                           out);
    return cudaGetLastError();
}

cudaError_t run_pass(const bfq::Pass &p, const float2 *in, long long ld_in, float2 *out, long long ld_out, int nrhs,
                     cudaStream_t s) {
    // a small stack (few outputs) gets a narrower RHS tile, so that 128 threads'
    // worth of its groups fit 48 KB of staging
    int tpg = 1;
    while (tpg < p.Nout && tpg < 128) tpg <<= 1;
    const long long fit = 49152 / ((long long)(p.Kin + p.Nout) * 8 * (128 / tpg));
    const int cap = fit >= 32 ? 32 : fit >= 16 ? 16 : fit >= 8 ? 8 : 32;   // (below 8: one group per block)
    if (nrhs >= 32 && cap >= 32) return launch_pass<32>(p, in, ld_in, out, ld_out, nrhs, s);
    if (nrhs >= 16 && cap >= 16) return launch_pass<16>(p, in, ld_in, out, ld_out, nrhs, s);
    if (nrhs >= 8) return launch_pass<8>(p, in, ld_in, out, ld_out, nrhs, s);
    if (nrhs >= 4) return launch_pass<4>(p, in, ld_in, out, ld_out, nrhs, s);
    if (nrhs >= 2) return launch_pass<2>(p, in, ld_in, out, ld_out, nrhs, s);
    // one vector: the streaming kernel (0.71 ms per apply at 256 x 256 against 0.90 for
    // the tiled kernel with one-vector tiles)
    if (!p.in_planar && !p.out_planar) return run_gemv(p, in, out, s);
    return launch_pass<1>(p, in, ld_in, out, ld_out, nrhs, s);
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

bf_status bf_quad_create(bf_quad *out, const bf_desc *desc, const bf_factors *f, cudaStream_t stream) {
    if (!out) return BF_ERR_INVALID;
    *out = nullptr;
    if (!desc || !f || !f->VL || !f->UL || !f->S || !f->H || !f->G) return BF_ERR_INVALID;
    if (f->dtype != BF_C64 && f->dtype != BF_C128) return BF_ERR_INVALID;
    const int L = desc->L, n0 = desc->leaf, r = desc->r;
    if (L < 2 || L % 2 || desc->nrhs_max < 1 || r < 1 || n0 < 1) return BF_ERR_INVALID;
    if ((n0 & (n0 - 1)) || (n0 & 0xAAAAAAAA)) return BF_ERR_INVALID;   // a power of 4
    if (L > bfq::kMaxL || r > 32 || n0 > 16) return BF_ERR_UNSUPPORTED;
    for (int t = 0; t < L / 2; ++t)
        if (!f->H[t] || !f->G[t]) return BF_ERR_INVALID;
    bf_quad_s *Q = new (std::nothrow) bf_quad_s;
    if (!Q) return BF_ERR_NOMEM;
    Q->L = L;
    Q->n0 = n0;
    Q->r = r;
    Q->h = L / 2;
    Q->nrhs_max = desc->nrhs_max;
    Q->N = (long long)n0 << (2 * L);
    Q->m = pow4(Q->h);
    for (int lv = Q->h; lv <= L; ++lv) Q->ranks[lv] = (int)std::min<long long>(r, Q->N >> (2 * lv));
    Q->Rmax = pow4(L) * Q->ranks[Q->h];
    int dev = 0;
    cudaGetDevice(&dev);
    Q->device = dev;
    cudaDeviceGetAttribute(&Q->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (const char *e = std::getenv("BF_TC_MIN")) Q->tc_min = std::max(8, std::atoi(e));   // planar tiles need NT >= 8
    Q->tc = Q->nrhs_max >= Q->tc_min;
    if (const char *e = std::getenv("BF_QUAD_KC")) Q->kc_max = std::atoi(e) <= 32 ? 32 : 64;
    if (const char *e = std::getenv("BF_INJECT_STALL")) Q->inject_stall = std::atoi(e) == 1 ? 1 : 0;
    if (Q->tc && bfint::tc_prepare() != cudaSuccess) {
        delete Q;
        return qfail(cudaErrorUnknown);
    }
    bf_status st = build_direction(*Q, *f, false, Q->fwd);
    if (st == BF_OK) st = build_direction(*Q, *f, true, Q->adj);
    if (st == BF_OK) {
        // planar 128-vector tiles on the tensor-core path: room for whole tiles
        const long long cols = Q->tc ? (Q->nrhs_max + 127) / 128 * 128 : Q->nrhs_max;
        const size_t ws = (size_t)Q->Rmax * cols * sizeof(float2);
        for (auto &w : Q->ws)
            if (st == BF_OK && cudaMalloc(&w, ws) != cudaSuccess) {
                cudaGetLastError();
                w = nullptr;
                st = BF_ERR_NOMEM;
            }
        if (st == BF_OK) Q->device_bytes += 2 * ws;
        if (st == BF_OK && cudaMalloc(&Q->d_err, sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            Q->d_err = nullptr;
            st = BF_ERR_NOMEM;
        }
        if (st == BF_OK && cudaMemset(Q->d_err, 0, sizeof(unsigned)) != cudaSuccess) st = qfail(cudaErrorUnknown);
    }
    if (st == BF_OK && cudaStreamSynchronize(stream) != cudaSuccess) st = qfail(cudaErrorUnknown);
    if (st != BF_OK) {
        free_quad(Q);
        return st;
    }
    *out = Q;
    return BF_OK;
}

bf_status bf_quad_apply(bf_quad Q, const void *in, void *out, int nrhs, long long ld, int adjoint,
                        cudaStream_t stream) {
    bfint::NvtxRange range(adjoint ? "bf_quad_apply (adjoint)" : "bf_quad_apply");
    if (!Q || nrhs < 0) return BF_ERR_INVALID;
    if (nrhs == 0) return BF_OK;
    if (!in || !out || ld < Q->N) return BF_ERR_INVALID;
    const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
    const long long span = ((long long)(nrhs - 1) * ld + Q->N) * 8;
    if (a < b + span && b < a + span) return BF_ERR_INVALID;
    if (!is_device_ptr(in) || !is_device_ptr(out)) return BF_ERR_INVALID;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != Q->device) {   // the plan's memory is on Q->device
        cudaGetLastError();
        return BF_ERR_INVALID;
    }
    const auto &D = adjoint ? Q->adj : Q->fwd;
    const int np = (int)D.size();
    for (int k0 = 0; k0 < nrhs; k0 += Q->nrhs_max) {
        const int nc = std::min(Q->nrhs_max, nrhs - k0);
        const float2 *src = static_cast<const float2 *>(in) + (long long)k0 * ld;
        float2 *dst = static_cast<float2 *>(out) + (long long)k0 * ld;
        const bool tc = Q->tc && nc >= Q->tc_min;   // planar tiles between the passes, tensor cores where built
        for (int ps = 0; ps < np; ++ps) {
            const bfq::HostPass &hp = D[ps];
            const float2 *pin = ps == 0 ? src : Q->ws[(ps - 1) & 1];
            float2 *pout = ps == np - 1 ? dst : Q->ws[ps & 1];
            const long long lin = ps == 0 ? ld : Q->Rmax, lout = ps == np - 1 ? ld : Q->Rmax;
            cudaError_t e;
            if (tc && hp.tc) {
                bfint::QuadTc q{};
                q.fac = hp.dtc;
                q.fac16 = hp.d16;
                q.in = pin;
                q.out = pout;
                q.R = Q->Rmax;
                q.err = Q->d_err;
                q.ain = hp.p.ain, q.bin = hp.p.bin, q.sin = hp.p.sin;
                q.aout = hp.p.aout, q.bout = hp.p.bout, q.sout = hp.p.sout;
                q.bszi = hp.p.bsz_in, q.bszo = hp.p.bsz_out, q.nB = hp.p.nB;
                q.ngroups = hp.p.nA * hp.p.nB;
                q.parts = hp.parts, q.chunks = hp.chunks, q.Kin = hp.Kc, q.Nout = hp.Nc, q.nrhs = nc;
                q.split = Q->tc_split, q.bf16 = Q->tc_bf16;
                q.stall = Q->inject_stall;
                e = bfint::quad_tc_launch(q, Q->num_sms, stream);
            } else {
                bfq::Pass pp = hp.p;
                pp.in_planar = tc && ps > 0;
                pp.out_planar = tc && ps < np - 1;
                pp.R = Q->Rmax;
                e = run_pass(pp, pin, lin, pout, lout, nc, stream);
            }
            if (e != cudaSuccess) return qfail(e);
        }
    }
    return BF_OK;
}

size_t bf_quad_device_bytes(bf_quad Q) { return Q ? Q->device_bytes : 0; }

int bf_quad_tc_passes(bf_quad Q) {
    int n = 0;
    if (Q)
        for (const auto &hp : Q->fwd) n += hp.tc ? 1 : 0;
    return n;
}

bf_status bf_quad_check(bf_quad Q, cudaStream_t stream) {
    if (!Q) return BF_ERR_INVALID;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return qfail(cudaErrorUnknown);
    unsigned e = 0;
    if (cudaMemcpy(&e, Q->d_err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess) return qfail(cudaErrorUnknown);
    if (e && cudaMemset(Q->d_err, 0, sizeof(unsigned)) != cudaSuccess) return qfail(cudaErrorUnknown);
    return e ? BF_ERR_TIMEOUT : BF_OK;
}

bf_status bf_quad_set_precision(bf_quad Q, int precision) {
    if (!Q) return BF_ERR_INVALID;
    int split, bf16;
    switch (precision) {
    case BF_PREC_FP32: split = 3; bf16 = 0; break;
    case BF_PREC_TF32: split = 1; bf16 = 0; break;
    case BF_PREC_BF16X3: split = 3; bf16 = 1; break;
    case BF_PREC_BF16: split = 1; bf16 = 1; break;
    case BF_PREC_BF16X6: split = 6; bf16 = 1; break;
    default: return BF_ERR_INVALID;
    }
    const int parts = bf16 ? (split == 6 ? 3 : split == 3 ? 2 : 1) : 0;
    std::vector<bfq::HostPass *> todo;
    for (auto *D : {&Q->fwd, &Q->adj})
        for (auto &hp : *D)
            if (hp.tc && hp.d16_parts != parts) todo.push_back(&hp);
    auto part_bytes = [](const bfq::HostPass &hp) {
        return (size_t)hp.p.nA * hp.p.nB * hp.parts * hp.chunks * 2 * hp.Nc * hp.Kc * sizeof(uint16_t);
    };
    std::vector<uint16_t *> fresh(todo.size(), nullptr);   // allocate all first: on failure the plan is unchanged
    if (parts > 0)
        for (size_t i = 0; i < todo.size(); ++i)
            if (cudaMalloc(&fresh[i], part_bytes(*todo[i]) * parts) != cudaSuccess) {
                cudaGetLastError();
                for (uint16_t *q : fresh) cudaFree(q);
                return BF_ERR_NOMEM;
            }
    if (!todo.empty() && cudaDeviceSynchronize() != cudaSuccess) return qfail(cudaErrorUnknown);
    for (size_t i = 0; i < todo.size(); ++i) {
        bfq::HostPass &hp = *todo[i];
        cudaFree(hp.d16);
        Q->device_bytes -= part_bytes(hp) * hp.d16_parts;
        hp.d16 = fresh[i];
        hp.d16_parts = parts;
        Q->device_bytes += part_bytes(hp) * parts;
    }
    // the rung matches the installed buffers before any split runs: a failure
    // below can leave wrong values, never a rung reading more parts than exist
    Q->tc_split = split;
    Q->tc_bf16 = bf16;
    if (parts == 0 || todo.empty()) return BF_OK;
    for (bfq::HostPass *hp : todo)
        if (bfint::bf16_split(hp->dtc, hp->d16, (long long)hp->p.nA * hp->p.nB * hp->parts * hp->chunks, 2 * hp->Nc,
                              hp->Kc, parts, Q->num_sms) != cudaSuccess)
            return qfail(cudaErrorUnknown);
    if (cudaDeviceSynchronize() != cudaSuccess) return qfail(cudaErrorUnknown);
    return BF_OK;
}

int bf_quad_passes(bf_quad Q) { return Q ? (int)Q->fwd.size() : 0; }

bf_status bf_quad_destroy(bf_quad Q) {
    if (!Q) return BF_OK;
    cudaDeviceSynchronize();
    free_quad(Q);
    return BF_OK;
}

}  // extern "C"
