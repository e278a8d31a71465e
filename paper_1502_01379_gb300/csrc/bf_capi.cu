// C ABI of the butterfly apply library: plan creation (validation, factor
// packing, upload), apply / adjoint launches, profiling and error checks.
// Declarations and argument documentation: include/bfly.h.
#include "bfly.h"
#include "bf_kernels.cuh"
#include "bf_wide.cuh"
#include "bf_tc.cuh"
#include "bf_internal.h"

#include <algorithm>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <utility>
#include <vector>

namespace bfint {
cudaError_t tc_launch(const bftc::TcParams &p, int grid, cudaStream_t s);
}

namespace {

using bfk::Level;
using bfk::Params;

constexpr int kMaxSmem = 232448;  // 227 KB opt-in per block on sm_100/sm_103

// One packed factor stream: the factors one kernel reads, chunked per CTA.
struct Stream {
    float2 *d = nullptr;
    long long cta_len = 0;
    int nlev = 0;
    Level lev[bfk::kMaxLevels];
};

// Forward or adjoint direction: the down and up kernels' streams and the S rows.
struct Direction {
    Stream down, up;
    float *d_S = nullptr;  // (node, q, k) weights for the up kernel's gather
};

struct Timing {
    cudaEvent_t a, b, c;
};

// One pass of the multi-RHS path (bf_wide.cuh): its packed stream and group
// geometry (the group's slots differ in node-slot bits a .. a+kb-1).
struct WidePass {
    Stream st;
    bool down = true;
    int load_kind = 0, store_kind = 0;
    int a = 0, kb = 0, G = 1, ngroups = 1;
    int Kin = 0, Nout = 0;   // tensor-core core: dense block per (node, group), Nout x Kin complex
    uint16_t *d16 = nullptr; // tensor-core core, BF16 rungs: the blocks split into d16_parts BF16 parts
    int d16_parts = 0;
};

// Configuration of one multi-RHS core: CUDA-core (bf_wide.cuh) or tensor-core (bf_tc.cuh).
struct WideCfg {
    bool tc = false;
    int kmax = 1;          // slot bits per pass
    int slot_len = 0;      // ring slot, complex entries
    int stages = 2;
    int nr_max = 0;        // CUDA-core: largest RHS tile
};

// The passes of one direction: down half (leaf first), then up half.
struct WideDirection {
    WideCfg cfg;
    std::vector<WidePass> pass;
};

}  // namespace

struct bf_plan_s {
    int L, n0, r, h, m, W, nrhs_max;
    int device = -1;                              // CUDA device the plan's memory lives on
    long long N, R;
    int stages, slot_len, consumers;
    Direction fwd, adj;
    float2 *d_ws = nullptr;                       // R x nrhs_max level-h vectors
    float2 *d_stage_in = nullptr, *d_stage_out = nullptr;  // host-pointer staging, N x nrhs_max
    // host-pointer calls on the fused path: node groups on side streams (created on first use)
    static constexpr int kGroups = 4;
    cudaStream_t gstream[kGroups] = {};
    cudaEvent_t gfork = nullptr, gjoin[kGroups] = {};
    unsigned *d_err = nullptr;
    size_t device_bytes = 0;
    bool profiling = false;
    std::vector<Timing> timings;
    size_t timing_used = 0;
    // multi-RHS path
    bool wide = false, tc = false;           // which multi-RHS cores were built
    int wide_min = 0, tc_min = 0;             // smallest batch each core serves
    int num_sms = 1;
    int tc_split = 3;                         // tensor-core products per real product: 1 plain, 3 hi/lo, 6 hi/mid/lo
    int tc_bf16 = 0;                          // tensor-core operand type: 0 = TF32, 1 = BF16
    int inject_stall = 0;                     // failure-detection test hook (BF_INJECT_STALL=1 at creation)
    WideDirection wfwd, wadj;                 // CUDA-core multi-RHS passes
    WideDirection tfwd, tadj;                 // tensor-core multi-RHS passes
    float2 *d_wsA = nullptr;                       // R x nrhs_max pass intermediate
};

namespace {

int env_int(const char *name, int dflt) {
    const char *v = std::getenv(name);
    if (!v || !*v) return dflt;
    char *end = nullptr;
    long x = std::strtol(v, &end, 10);
    return (end && *end == 0 && x > 0 && x < (1 << 30)) ? (int)x : dflt;
}

bf_status cuda_fail(cudaError_t e) {
    (void)e;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? BF_ERR_NOMEM : BF_ERR_CUDA;
}

#define BF_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_);    \
    } while (0)

// Reads element (block, row, col) of a canonical row-major factor array.
struct Src {
    const void *p;
    int dtype;
    int rows, cols;
    inline float2 at(long long blk, int row, int col) const {
        const long long i = (blk * rows + row) * (long long)cols + col;
        if (dtype == BF_C64) return static_cast<const float2 *>(p)[i];
        const double2 v = static_cast<const double2 *>(p)[i];
        return make_float2((float)v.x, (float)v.y);
    }
    inline std::complex<double> atd(long long blk, int row, int col) const {
        const long long i = (blk * rows + row) * (long long)cols + col;
        if (dtype == BF_C64) {
            const float2 v = static_cast<const float2 *>(p)[i];
            return {(double)v.x, (double)v.y};
        }
        const double2 v = static_cast<const double2 *>(p)[i];
        return {v.x, v.y};
    }
};

inline float2 conjf2(float2 v) { return make_float2(v.x, -v.y); }

// Level table of one stream.  Down: leaf then merging levels t = 1..h
// (segments of s = 2^t blocks, i.e. factor level l = L - t).  Up: splitting
// levels t = h..1 then the leaf.
void make_levels(Stream &st, bool down, int h, int m, int n0, int r, int slot_len) {
    auto fill = [&](Level &lv, int kind, int K, int rpu, int nunits, int s) {
        int upb = 1;
        while (upb * 2 <= nunits && (long long)(upb * 2) * K * rpu <= slot_len) upb *= 2;
        lv.kind = kind;
        lv.K = K;
        lv.rpu = rpu;
        lv.upb = upb;
        lv.nstages = nunits / upb;
        lv.stage_len = (upb * K * rpu + 1) & ~1;
        lv.s = s;
        lv.pad_ = 0;
    };
    int n = 0;
    if (down) {
        fill(st.lev[n++], bfk::LEAF_IN, n0, r, m, 1);
        for (int t = 1; t <= h; ++t) fill(st.lev[n++], bfk::MERGE, 2 * r, 2 * r, m / 2, 1 << t);
    } else {
        for (int t = h; t >= 1; --t) fill(st.lev[n++], bfk::SPLIT, 2 * r, 2 * r, m / 2, 1 << t);
        fill(st.lev[n++], bfk::LEAF_OUT, r, n0, m, 1);
    }
    st.nlev = n;
    st.cta_len = 0;
    for (int i = 0; i < n; ++i) st.cta_len += (long long)st.lev[i].nstages * st.lev[i].stage_len;
}

// Which factor a stream packs.
enum StreamKind { FWD_DOWN, FWD_UP, ADJ_DOWN, ADJ_UP };

// Packs one stream: for CTA (node) c, level by level, stage by stage, the
// units' matrices B (rpu x K) stored k-major over the stage's rows:
// dst[k * (upb*rpu) + u_in * rpu + rr] = B_u[rr][k].
void pack_stream(float2 *dst, const Stream &st, StreamKind kind, const bf_plan_s &P, const bf_factors &f) {
    const int L = P.L, h = P.h, m = P.m, n0 = P.n0, r = P.r;
    const Src VL{f.VL, f.dtype, n0, r}, UL{f.UL, f.dtype, n0, r};
    auto work = [&](int c0, int c1) {
        for (int c = c0; c < c1; ++c) {
            float2 *o = dst + (long long)c * st.cta_len;
            for (int li = 0; li < st.nlev; ++li) {
                const Level &lv = st.lev[li];
                const int rows = lv.upb * lv.rpu;
                for (int stg = 0; stg < lv.nstages; ++stg) {
                    for (int ui = 0; ui < lv.upb; ++ui) {
                        const int u = stg * lv.upb + ui;
                        for (int rr = 0; rr < lv.rpu; ++rr) {
                            for (int k = 0; k < lv.K; ++k) {
                                float2 v;
                                if (lv.kind == bfk::LEAF_IN || lv.kind == bfk::LEAF_OUT) {
                                    const long long b = (long long)c * m + u;
                                    const Src &S = (kind == FWD_DOWN || kind == ADJ_UP) ? VL : UL;
                                    if (lv.kind == bfk::LEAF_IN) v = conjf2(S.at(b, k, rr));  // (X^L_b)^*: rr = col k, k = point p
                                    else v = S.at(b, rr, k);                                   // X^L_b: rr = point p, k = col
                                } else {
                                    const int s = lv.s, hs = s >> 1;
                                    const int l = L - __builtin_ctz(s);        // factor level
                                    const int seg = u / hs, q = u % hs;
                                    const long long nodel = (long long)c * (m / s) + seg;  // tree node at level l
                                    const bool is_h = (kind == FWD_DOWN || kind == ADJ_UP);
                                    const Src X{is_h ? f.H[l - h] : f.G[l - h], f.dtype, r, 2 * r};
                                    if (lv.kind == bfk::MERGE) {
                                        // rr = d*r + kk (output block 2q+d), k = c'*r + k' (input block c'*hs+q)
                                        const int cc = k / r, kp = k % r;
                                        const long long blk = (2 * nodel + cc) * hs + q;
                                        // (X^l_{2n+c',q})^*: entry (d*r+kk, k') = conj(X[k'][d*r+kk])
                                        v = conjf2(X.at(blk, kp, rr));
                                    } else {
                                        // rr = c'*r + kk (output block c'*hs+q), k = d*r + k' (input block 2q+d)
                                        const int cc = rr / r, kk = rr % r;
                                        const long long blk = (2 * nodel + cc) * hs + q;
                                        v = X.at(blk, kk, k);
                                    }
                                }
                                o[(long long)k * rows + (long long)ui * lv.rpu + rr] = v;
                            }
                        }
                    }
                    if (lv.stage_len > rows * lv.K) o[lv.stage_len - 1] = make_float2(0.f, 0.f);
                    o += lv.stage_len;
                }
            }
        }
    };
    int nthreads = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    nthreads = std::min(nthreads, m);
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t) pool.emplace_back(work, (int)((long long)m * t / nthreads), (int)((long long)m * (t + 1) / nthreads));
    for (auto &th : pool) th.join();
}

bf_status upload_stream(bf_plan_s &P, Stream &st, StreamKind kind, const bf_factors &f) {
    const size_t n = (size_t)P.m * st.cta_len;
    std::vector<float2> host;
    try {
        host.resize(n);
    } catch (const std::bad_alloc &) {
        return BF_ERR_NOMEM;
    }
    pack_stream(host.data(), st, kind, P, f);
    BF_CUDA(cudaMalloc(&st.d, n * sizeof(float2)));
    P.device_bytes += n * sizeof(float2);
    BF_CUDA(cudaMemcpy(st.d, host.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
    return BF_OK;
}

bf_status upload_S(bf_plan_s &P, const bf_factors &f) {
    const int m = P.m, r = P.r;
    const size_t n = (size_t)m * m * r;
    std::vector<float> fw(n), ad(n);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j)
            for (int k = 0; k < r; ++k) {
                const size_t src = ((size_t)i * m + j) * r + k;
                const float v = f.dtype == BF_C64 ? static_cast<const float *>(f.S)[src]
                                                  : (float)static_cast<const double *>(f.S)[src];
                fw[src] = v;                               // forward: row node i gathers q = j
                ad[((size_t)j * m + i) * r + k] = v;       // adjoint: column node j gathers q = i
            }
    BF_CUDA(cudaMalloc(&P.fwd.d_S, n * sizeof(float)));
    BF_CUDA(cudaMalloc(&P.adj.d_S, n * sizeof(float)));
    P.device_bytes += 2 * n * sizeof(float);
    BF_CUDA(cudaMemcpy(P.fwd.d_S, fw.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    BF_CUDA(cudaMemcpy(P.adj.d_S, ad.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    return BF_OK;
}

// ------------------------------------------------------------ multi-RHS path
inline int host_insert0(int v, int b) { return ((v >> b) << (b + 1)) | (v & ((1 << b) - 1)); }
inline int host_bitrev(int x, int bits) {
    int y = 0;
    for (int i = 0; i < bits; ++i) y |= ((x >> i) & 1) << (bits - 1 - i);
    return y;
}

// Pass geometry and level tables.  The h levels of each half are cut into
// chunks of at most kmax slot bits, [a, a+kb).  Down half, chunks in
// increasing a: merging levels t = a+1..a+kb (local bit t-1-a); the first
// pass also loads the input points and runs the leaf, the last one stores the
// level-h vector in logical order.  Up half, chunks in decreasing a:
// splitting levels t = a+kb..a+1; the first pass gathers M^h, the last one
// runs the leaf and writes the output.  Level.s = local slot bit, Level.pad_ = t.
void make_wide_passes(WideDirection &D, const bf_plan_s &P, const WideCfg &cfg) {
    const int h = P.h, m = P.m, r = P.r, n0 = P.n0;
    const int kmax = cfg.kmax;
    D.cfg = cfg;
    std::vector<std::pair<int, int>> chunks;   // (a, kb)
    for (int a = 0; a < h || chunks.empty(); a += std::max(1, kmax)) chunks.push_back({a, std::min(kmax, h - a)});
    if (h == 0) chunks = {{0, 0}};
    auto fill = [&](Level &lv, int kind, int K, int rpu, int nunits, int bit, int t) {
        int upb = 1;
        while (upb * 2 <= nunits && (long long)(upb * 2) * K * rpu <= cfg.slot_len) upb *= 2;
        lv.kind = kind;
        lv.K = K;
        lv.rpu = rpu;
        lv.upb = upb;
        lv.nstages = nunits / upb;
        lv.stage_len = (upb * K * rpu + 1) & ~1;
        lv.s = bit;
        lv.pad_ = t;
    };
    D.pass.clear();
    const int nc = (int)chunks.size();
    for (int half = 0; half < 2; ++half) {
        for (int ci = 0; ci < nc; ++ci) {
            const auto ch = half == 0 ? chunks[ci] : chunks[nc - 1 - ci];
            const bool first = ci == 0, last = ci == nc - 1;
            WidePass wp;
            wp.down = half == 0;
            wp.a = ch.first;
            wp.kb = ch.second;
            wp.G = 1 << wp.kb;
            wp.ngroups = m >> wp.kb;
            Stream &st = wp.st;
            int n = 0;
            if (wp.down) {
                wp.load_kind = first ? bfw::LD_POINTS : bfw::LD_SLOTS;
                wp.store_kind = last ? bfw::ST_LOGICAL : bfw::ST_SLOTS;
                if (first) fill(st.lev[n++], bfk::LEAF_IN, n0, r, wp.G, 0, 0);
                for (int t = wp.a + 1; t <= wp.a + wp.kb; ++t)
                    fill(st.lev[n++], bfk::MERGE, 2 * r, 2 * r, wp.G / 2, t - 1 - wp.a, t);
            } else {
                wp.load_kind = first ? bfw::LD_GATHER : bfw::LD_SLOTS;
                wp.store_kind = last ? bfw::ST_NONE : bfw::ST_SLOTS;
                for (int t = wp.a + wp.kb; t >= wp.a + 1; --t)
                    fill(st.lev[n++], bfk::SPLIT, 2 * r, 2 * r, wp.G / 2, t - 1 - wp.a, t);
                if (last) fill(st.lev[n++], bfk::LEAF_OUT, r, n0, wp.G, 0, 0);
            }
            st.nlev = n;
            st.cta_len = 0;
            for (int i = 0; i < n; ++i) st.cta_len += (long long)st.lev[i].nstages * st.lev[i].stage_len;
            D.pass.push_back(wp);
        }
    }
}

inline int host_slot_of(const WidePass &wp, int g, int j) {
    return ((g >> wp.a) << (wp.a + wp.kb)) | (j << wp.a) | (g & ((1 << wp.a) - 1));
}

// Entry (rr, k) of unit u of level lv in pass wp, chunk (node c, group g):
// the same unit matrices as the fused path (rows = the unit's outputs, cols =
// its inputs).  Down half: (V^L)^* and (H^l)^* forward, (U^L)^* and (G^l)^*
// adjoint; up half the others.
struct UnitSource {
    const WidePass &wp;
    const bf_plan_s &P;
    const bf_factors &f;
    bool use_v;
    UnitSource(const WidePass &w, bool adjoint, const bf_plan_s &pl, const bf_factors &fa)
        : wp(w), P(pl), f(fa), use_v(w.down != adjoint) {}
    std::complex<double> operator()(const Level &lv, int c, int g, int u, int rr, int k) const {
        const int L = P.L, h = P.h, m = P.m, n0 = P.n0, r = P.r;
        if (lv.kind == bfk::LEAF_IN || lv.kind == bfk::LEAF_OUT) {
            const Src LEAF{use_v ? f.VL : f.UL, f.dtype, n0, r};
            const long long b = (long long)c * m + host_slot_of(wp, g, u);
            return lv.kind == bfk::LEAF_IN ? std::conj(LEAF.atd(b, k, rr)) : LEAF.atd(b, rr, k);
        }
        const int t = lv.pad_, sz = 1 << t, hs = sz >> 1;
        const int j0 = host_insert0(u, lv.s);
        const int p0 = host_slot_of(wp, g, j0);
        const int seg = p0 >> t;
        const int q = host_bitrev(p0 & (hs - 1), t - 1);
        const long long nodel = (long long)c * (m / sz) + seg;
        const int l = L - t;
        const Src X{use_v ? f.H[l - h] : f.G[l - h], f.dtype, r, 2 * r};
        if (lv.kind == bfk::MERGE) {
            const int cc = k / r, kp = k % r;
            return std::conj(X.atd((2 * nodel + cc) * hs + q, kp, rr));
        }
        const int cc = rr / r, kk = rr % r;
        return X.atd((2 * nodel + cc) * hs + q, kk, k);
    }
};

// Packs one pass: chunk (node c, group g) = c * ngroups + g; units in the
// order the CTA runs them; the unit matrices are the fused path's.
void pack_wide(float2 *dst, const WidePass &wp, bool adjoint, const bf_plan_s &P, const bf_factors &f) {
    const int m = P.m;
    const UnitSource unit(wp, adjoint, P, f);
    const Stream &st = wp.st;
    auto work = [&](int c0, int c1) {
        for (int c = c0; c < c1; ++c) {
            for (int g = 0; g < wp.ngroups; ++g) {
                float2 *o = dst + ((long long)c * wp.ngroups + g) * st.cta_len;
                for (int li = 0; li < st.nlev; ++li) {
                    const Level &lv = st.lev[li];
                    const int rows = lv.upb * lv.rpu;
                    for (int stg = 0; stg < lv.nstages; ++stg) {
                        for (int ui = 0; ui < lv.upb; ++ui) {
                            const int u = stg * lv.upb + ui;
                            for (int rr = 0; rr < lv.rpu; ++rr)
                                for (int k = 0; k < lv.K; ++k) {
                                    const std::complex<double> v = unit(lv, c, g, u, rr, k);
                                    o[(long long)k * rows + (long long)ui * lv.rpu + rr] =
                                        make_float2((float)v.real(), (float)v.imag());
                                }
                        }
                        if (lv.stage_len > rows * lv.K) o[lv.stage_len - 1] = make_float2(0.f, 0.f);
                        o += lv.stage_len;
                    }
                }
            }
        }
    };
    int nthreads = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    nthreads = std::min(nthreads, m);
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t)
        pool.emplace_back(work, (int)((long long)m * t / nthreads), (int)((long long)m * (t + 1) / nthreads));
    for (auto &th : pool) th.join();
}

// Tensor-core core: the pass's levels (and the leaf, and S^h of M^h) on one
// group of G slots multiplied out, in FP64, into one dense block F
// (Nout x Kin); stored per chunk as the K-major operand [Re F; Im F].
void pack_tc(float *dst, const WidePass &wp, bool adjoint, const bf_plan_s &P, const bf_factors &f) {
    using cd = std::complex<double>;
    const int m = P.m, r = P.r, n0 = P.n0, G = wp.G, Kin = wp.Kin, Nout = wp.Nout;
    const UnitSource unit(wp, adjoint, P, f);
    const Stream &st = wp.st;
    auto S_at = [&](long long i) -> double {
        return f.dtype == BF_C64 ? (double)static_cast<const float *>(f.S)[i] : static_cast<const double *>(f.S)[i];
    };
    auto work = [&](int c0, int c1) {
        std::vector<cd> F, T;
        for (int c = c0; c < c1; ++c) {
            for (int g = 0; g < wp.ngroups; ++g) {
                int li = 0, rows;
                if (st.lev[0].kind == bfk::LEAF_IN) {
                    rows = G * r;
                    F.assign((size_t)rows * Kin, cd(0));
                    for (int j = 0; j < G; ++j)
                        for (int rr = 0; rr < r; ++rr)
                            for (int k = 0; k < n0; ++k)
                                F[(size_t)(j * r + rr) * Kin + j * n0 + k] = unit(st.lev[0], c, g, j, rr, k);
                    li = 1;
                } else {
                    rows = G * r;
                    F.assign((size_t)rows * Kin, cd(0));
                    for (int j = 0; j < G; ++j)
                        for (int kk = 0; kk < r; ++kk) {
                            double w = 1.0;
                            if (wp.load_kind == bfw::LD_GATHER) {
                                // M^h: slot ps of row node c holds logical block q = bitrev_h(ps), times S
                                const int q = host_bitrev(host_slot_of(wp, g, j), P.h);
                                w = adjoint ? S_at(((long long)q * m + c) * r + kk) : S_at(((long long)c * m + q) * r + kk);
                            }
                            F[(size_t)(j * r + kk) * Kin + j * r + kk] = w;
                        }
                }
                for (; li < st.nlev; ++li) {
                    const Level &lv = st.lev[li];
                    if (lv.kind == bfk::LEAF_OUT) {
                        T.assign((size_t)G * n0 * Kin, cd(0));
                        for (int j = 0; j < G; ++j)
                            for (int pt = 0; pt < n0; ++pt) {
                                cd *o = &T[(size_t)(j * n0 + pt) * Kin];
                                for (int kk = 0; kk < r; ++kk) {
                                    const cd b = unit(lv, c, g, j, pt, kk);
                                    const cd *x = &F[(size_t)(j * r + kk) * Kin];
                                    for (int k = 0; k < Kin; ++k) o[k] += b * x[k];
                                }
                            }
                        F.swap(T);
                        rows = G * n0;
                        continue;
                    }
                    // butterflies on slot pairs (j0, j1) differing in local bit lv.s
                    T.assign((size_t)2 * r * Kin, cd(0));
                    for (int u = 0; u < G / 2; ++u) {
                        const int j0 = host_insert0(u, lv.s), j1 = j0 | (1 << lv.s);
                        std::fill(T.begin(), T.end(), cd(0));
                        for (int rr = 0; rr < 2 * r; ++rr) {
                            cd *o = &T[(size_t)rr * Kin];
                            for (int k = 0; k < 2 * r; ++k) {
                                const cd b = unit(lv, c, g, u, rr, k);
                                const cd *x = &F[(size_t)((k < r ? j0 : j1) * r + k % r) * Kin];
                                for (int kx = 0; kx < Kin; ++kx) o[kx] += b * x[kx];
                            }
                        }
                        for (int rr = 0; rr < 2 * r; ++rr)
                            std::copy(&T[(size_t)rr * Kin], &T[(size_t)rr * Kin] + Kin,
                                      &F[(size_t)((rr < r ? j0 : j1) * r + rr % r) * Kin]);
                    }
                }
                float *o = dst + ((long long)c * wp.ngroups + g) * 2ll * Nout * Kin;
                for (int rr = 0; rr < Nout; ++rr)
                    for (int k = 0; k < Kin; ++k) {
                        const cd v = F[(size_t)rr * Kin + k];
                        o[bftc::boff(rr, k, 2 * Nout) >> 2] = (float)v.real();
                        o[bftc::boff(Nout + rr, k, 2 * Nout) >> 2] = (float)v.imag();
                    }
                (void)rows;
            }
        }
    };
    int nthreads = (int)std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
    nthreads = std::min(nthreads, m);
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t)
        pool.emplace_back(work, (int)((long long)m * t / nthreads), (int)((long long)m * (t + 1) / nthreads));
    for (auto &th : pool) th.join();
}

bf_status upload_wide(bf_plan_s &P, WidePass &wp, bool adjoint, const bf_factors &f, bool tc) {
    const size_t n = (size_t)P.m * wp.ngroups * wp.st.cta_len;
    std::vector<float2> host;
    try {
        host.resize(n);
    } catch (const std::bad_alloc &) {
        return BF_ERR_NOMEM;
    }
    if (tc) pack_tc(reinterpret_cast<float *>(host.data()), wp, adjoint, P, f);
    else pack_wide(host.data(), wp, adjoint, P, f);
    BF_CUDA(cudaMalloc(&wp.st.d, n * sizeof(float2)));
    P.device_bytes += n * sizeof(float2);
    BF_CUDA(cudaMemcpy(wp.st.d, host.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
    return BF_OK;
}

size_t wide_smem(const bf_plan_s &P, const WideCfg &c, int NR) {
    const int G = 1 << std::min(c.kmax, P.h);
    return bfw::wide_smem_bytes(c.stages, c.slot_len, G, P.W, NR);
}

// Largest RHS tile whose threads-per-unit fit the consumers and whose tile fits shared memory.
int wide_nr_max(const bf_plan_s &P, const WideCfg &c) {
    for (int NR : {64, 32, 16}) {
        bool ok = wide_smem(P, c, NR) <= (size_t)kMaxSmem;
        for (int rpu : {P.r, 2 * P.r, P.n0}) {
            const int rb = (rpu % 2 == 0) ? 2 : 1;
            if ((rpu / rb) * (NR / 4) > P.consumers) ok = false;
        }
        if (ok) return NR;
    }
    return 0;
}

// The dynamic shared memory attribute of a kernel is one value shared by every
// plan that launches it, so it is always set to the device's opt-in maximum
// (an upper bound; each launch still requests only what it uses).
template <int NR>
bf_status set_wide_attr(size_t bytes) {
    (void)bytes;
    BF_CUDA(cudaFuncSetAttribute(bfw::bf_wide_kernel<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    return BF_OK;
}

// RHS capacity of the workspaces: the tensor-core core pads to whole 128-RHS tiles.
long long ws_rhs(const bf_plan_s &P) {
    return P.tc ? (long long)(P.nrhs_max + bftc::NR - 1) / bftc::NR * bftc::NR : P.nrhs_max;
}

template <int NR>
cudaError_t launch_wide(const bf_plan_s &P, const WideDirection &D, const float *d_S, const float2 *in, long long ld_in,
                        float2 *out, long long ld_out, int nrhs, cudaStream_t s, Timing *tm) {
    const WideCfg &c = D.cfg;
    const size_t smem = wide_smem(P, c, NR);
    float2 *buf[2] = {P.d_wsA, P.d_ws};
    const int np = (int)D.pass.size();
    if (tm) cudaEventRecord(tm->a, s);
    for (int ps = 0; ps < np; ++ps) {
        const WidePass &wp = D.pass[ps];
        bfw::WideParams p;
        std::memset(&p, 0, sizeof(p));
        p.fac = wp.st.d;
        p.cta_len = wp.st.cta_len;
        p.in = ps == 0 ? in : buf[(ps - 1) & 1];
        p.ld_in = ps == 0 ? ld_in : P.R;
        p.out = ps == np - 1 ? out : buf[ps & 1];
        p.ld_out = ps == np - 1 ? ld_out : P.R;
        p.S = d_S;
        p.err = P.d_err;
        p.nlev = wp.st.nlev;
        p.load_kind = wp.load_kind;
        p.store_kind = wp.store_kind;
        p.m = P.m;
        p.r = P.r;
        p.n0 = P.n0;
        p.W = P.W;
        p.h = P.h;
        p.G = wp.G;
        p.a = wp.a;
        p.kb = wp.kb;
        p.ngroups = wp.ngroups;
        p.nrhs = nrhs;
        p.stages = c.stages;
        p.slot_len = c.slot_len;
        for (int i = 0; i < wp.st.nlev; ++i) p.lev[i] = wp.st.lev[i];
        const dim3 grid((nrhs + NR - 1) / NR, P.m * wp.ngroups);
        bfint::NvtxRange range(wp.down ? "bf_wide_kernel (merging pass)" : "bf_wide_kernel (splitting pass)");
        bfw::bf_wide_kernel<NR><<<grid, P.consumers + 32, smem, s>>>(p);
        if (tm && ps + 1 < np && !D.pass[ps + 1].down && wp.down) cudaEventRecord(tm->b, s);
    }
    if (tm) cudaEventRecord(tm->c, s);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        cudaGetLastError();
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Tensor map of nrhs column-major vectors (16-byte aligned, even ld) as a
// {2 N floats, nrhs rows} FP32 tensor read in tiles of 32 floats x W rows
// with the 128-byte swizzle; false if it cannot be made.
bool points_tmap(CUtensorMap *map, const float2 *in, long long N, long long ld, int nrhs, int W) {
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return false;
    const cuuint64_t dim[2] = {(cuuint64_t)(2 * N), (cuuint64_t)nrhs};
    const cuuint64_t stride[1] = {(cuuint64_t)ld * 8};
    const cuuint32_t box[2] = {32, (cuuint32_t)W};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2 *>(in), dim, stride, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// RHS per tile of a tensor-core apply of nrhs vectors: the fewest tiles of at
// most 128, evened out and rounded up to a multiple of 32 (one warp's lanes),
// so a call with fewer than 128 vectors moves only the columns it uses.
int tc_tile_width(int nrhs) {
    const int ntiles = (nrhs + bftc::NR - 1) / bftc::NR;
    const int per = (nrhs + ntiles - 1) / ntiles;
    return std::min(bftc::NR, (per + 31) / 32 * 32);
}

// Tensor-core multi-RHS core: one persistent launch (one CTA per SM) per
// pass; pass intermediates are W-RHS tiles, position-major and planar
// ([tile][position][re W | im W], W = tc_tile_width(nrhs)).  `in` / `out`
// must be 16-byte aligned with an even leading dimension.
cudaError_t launch_tc(const bf_plan_s &P, const WideDirection &D, const float2 *in, long long ld_in, float2 *out,
                      long long ld_out, int nrhs, cudaStream_t s, Timing *tm) {
    float2 *buf[2] = {P.d_wsA, P.d_ws};
    const int np = (int)D.pass.size();
    const int W = tc_tile_width(nrhs);
    const long long ntiles = (nrhs + W - 1) / W;
    if (tm) cudaEventRecord(tm->a, s);
    for (int ps = 0; ps < np; ++ps) {
        const WidePass &wp = D.pass[ps];
        bftc::TcParams p;
        std::memset(&p, 0, sizeof(p));
        p.fac = reinterpret_cast<const float *>(wp.st.d);
        p.fac16 = wp.d16;
        p.in = ps == 0 ? in : buf[(ps - 1) & 1];
        p.ld_in = ps == 0 ? ld_in : 0;
        p.out = ps == np - 1 ? out : buf[ps & 1];
        p.ld_out = ps == np - 1 ? ld_out : 0;
        p.R = P.R;
        p.err = P.d_err;
        p.load_kind = wp.load_kind;   // bfw and bftc load kinds share their numbering
        p.store_kind = wp.store_kind == bfw::ST_NONE ? bftc::ST_POINTS
                     : wp.store_kind == bfw::ST_LOGICAL ? bftc::ST_LOGICAL : bftc::ST_SLOTS;
        p.m = P.m;
        p.r = P.r;
        p.n0 = P.n0;
        p.h = P.h;
        p.a = wp.a;
        p.kb = wp.kb;
        p.G = wp.G;
        p.ngroups = wp.ngroups;
        p.Kin = wp.Kin;
        p.Nout = wp.Nout;
        p.nrhs = nrhs;
        p.W = W;
        p.split = P.tc_split;
        p.bf16 = P.tc_bf16;
        p.stall = P.inject_stall;
        if (p.load_kind == bftc::LD_POINTS && env_int("BF_TC_TMAP", 1) == 1)
            p.use_tmap = points_tmap(&p.tmap, p.in, P.N, p.ld_in, nrhs, W) ? 1 : 0;
        const long long items = ntiles * P.m * wp.ngroups;
        const int grid = (int)std::min<long long>(items, P.num_sms);
        bfint::NvtxRange range(wp.down ? "bf_tc_kernel (merging pass)" : "bf_tc_kernel (splitting pass)");
        bfint::tc_launch(p, grid, s);
        if (tm && ps + 1 < np && !D.pass[ps + 1].down && wp.down) cudaEventRecord(tm->b, s);
    }
    if (tm) cudaEventRecord(tm->c, s);
    return cudaGetLastError();
}

// Unit dimensions of every tensor-core pass; false if one does not fit the
// core (Kin and Nout multiples of 16, at most 64; r and n0 multiples of 8, as
// the epilogue stores runs of 8 outputs inside one r-block or leaf).
bool set_tc_dims(WideDirection &D, const bf_plan_s &P) {
    if (P.r % 8 != 0 || P.n0 % 8 != 0) return false;
    for (auto &wp : D.pass) {
        const int first = wp.st.lev[0].kind, last = wp.st.lev[wp.st.nlev - 1].kind;
        wp.Kin = wp.G * (first == bfk::LEAF_IN ? P.n0 : P.r);
        wp.Nout = wp.G * (last == bfk::LEAF_OUT ? P.n0 : P.r);
        wp.st.cta_len = (long long)wp.Nout * wp.Kin;   // complex entries per chunk
        for (int d : {wp.Kin, wp.Nout})
            if (d % 16 != 0 || d > bftc::kMaxDim) return false;
    }
    return true;
}

size_t plan_smem(const bf_plan_s &P, int T) { return bfk::smem_bytes(P.stages, P.slot_len, P.m, P.W, T); }

template <int T>
bf_status set_smem_attr(size_t bytes) {
    (void)bytes;   // shared by all plans: the opt-in maximum (see set_wide_attr)
    BF_CUDA(cudaFuncSetAttribute(bfk::bf_down_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    BF_CUDA(cudaFuncSetAttribute(bfk::bf_up_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
    return BF_OK;
}

void free_plan(bf_plan_s *P) {
    if (!P) return;
    for (Direction *d : {&P->fwd, &P->adj}) {
        cudaFree(d->down.d);
        cudaFree(d->up.d);
        cudaFree(d->d_S);
    }
    for (WideDirection *d : {&P->wfwd, &P->wadj, &P->tfwd, &P->tadj})
        for (auto &wp : d->pass) {
            cudaFree(wp.st.d);
            cudaFree(wp.d16);
        }
    cudaFree(P->d_wsA);
    cudaFree(P->d_ws);
    cudaFree(P->d_stage_in);
    cudaFree(P->d_stage_out);
    for (int g = 0; g < bf_plan_s::kGroups; ++g) {
        if (P->gstream[g]) cudaStreamDestroy(P->gstream[g]);
        if (P->gjoin[g]) cudaEventDestroy(P->gjoin[g]);
    }
    if (P->gfork) cudaEventDestroy(P->gfork);
    cudaFree(P->d_err);
    for (auto &t : P->timings) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
        cudaEventDestroy(t.c);
    }
    cudaGetLastError();
    delete P;
}

Params base_params(const bf_plan_s &P, const Stream &st) {
    Params p;
    std::memset(&p, 0, sizeof(p));
    p.fac = st.d;
    p.cta_len = st.cta_len;
    p.fac_elems = (long long)P.m * st.cta_len;
    p.s_elems = (long long)P.m * P.m * P.r;
    p.err = P.d_err;
    p.stall = P.inject_stall;
    p.nlev = st.nlev;
    for (int i = 0; i < st.nlev; ++i) p.lev[i] = st.lev[i];
    p.m = P.m;
    p.r = P.r;
    p.n0 = P.n0;
    p.W = P.W;
    p.stages = P.stages;
    p.slot_len = P.slot_len;
    return p;
}

template <int T>
cudaError_t launch_pair(const bf_plan_s &P, const Direction &D, const float2 *in, long long ld_in, float2 *out,
                        long long ld_out, int nrhs, cudaStream_t s, Timing *tm) {
    const dim3 grid((nrhs + T - 1) / T, P.m);
    const dim3 block(P.consumers + 32);
    const size_t smem = plan_smem(P, T);
    Params pd = base_params(P, D.down);
    pd.in = in;
    pd.ld_in = ld_in;
    pd.out = P.d_ws;
    pd.ld_out = P.R;
    pd.nrhs = nrhs;
    pd.in_elems = (long long)(nrhs - 1) * ld_in + P.N;
    pd.out_elems = P.R * ws_rhs(P);
    Params pu = base_params(P, D.up);
    pu.in = P.d_ws;
    pu.ld_in = P.R;
    pu.out = out;
    pu.ld_out = ld_out;
    pu.S = D.d_S;
    pu.nrhs = nrhs;
    pu.in_elems = P.R * ws_rhs(P);
    pu.out_elems = (long long)(nrhs - 1) * ld_out + P.N;
#ifdef BF_CHECKED
    // test hook of the checked build: state the output one element short, so the
    // kernel's last store falls outside and must be skipped and reported
    if (env_int("BF_CHECKED_SHRINK_OUT", 0) == 1) pu.out_elems -= 1;
#endif
    if (tm) cudaEventRecord(tm->a, s);
    {
        bfint::NvtxRange range("bf_down_kernel (leaf + merging levels)");
        bfk::bf_down_kernel<T><<<grid, block, smem, s>>>(pd);
    }
    if (tm) cudaEventRecord(tm->b, s);
    {
        bfint::NvtxRange range("bf_up_kernel (M^h + splitting levels + leaf)");
        bfk::bf_up_kernel<T><<<grid, block, smem, s>>>(pu);
    }
    if (tm) cudaEventRecord(tm->c, s);
    return cudaGetLastError();
}

int pick_T(const bf_plan_s &P, int nrhs) {
    int T = 1;
    for (int cand : {2, 4})
        if (nrhs >= cand && plan_smem(P, cand) <= (size_t)kMaxSmem) T = cand;
    return T;
}

Timing *next_timing(bf_plan_s &P) {
    if (!P.profiling) return nullptr;
    if (P.timing_used == P.timings.size()) {
        Timing t;
        if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess ||
            cudaEventCreate(&t.c) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        P.timings.push_back(t);
    }
    return &P.timings[P.timing_used++];
}

bool is_host_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

// True when the calling thread's current device is the one the plan was
// created on (its factors, workspaces and error word live there).
bool on_plan_device(const bf_plan_s &P) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return dev == P.device;
}

// The two host-pointer staging buffers (N x nrhs_max each), allocated on
// first use.  Both are installed together or not at all, so a failed second
// allocation never leaves a plan with one buffer and a null partner.
bf_status ensure_staging(bf_plan_s &P) {
    if (P.d_stage_in && P.d_stage_out) return BF_OK;
    const size_t bytes = (size_t)P.N * P.nrhs_max * sizeof(float2);
    float2 *a = nullptr, *b = nullptr;
    cudaError_t e = cudaMalloc(&a, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b, bytes);
    if (e != cudaSuccess) {
        cudaFree(a);
        cudaFree(b);
        return cuda_fail(e);
    }
    P.d_stage_in = a;
    P.d_stage_out = b;
    P.device_bytes += 2 * bytes;
    return BF_OK;
}

// Side streams and events of the overlapped host-buffer path.
bf_status ensure_groups(bf_plan_s &P) {
    if (P.gfork) return BF_OK;
    cudaEvent_t fork = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int g = 0; g < bf_plan_s::kGroups && e == cudaSuccess; ++g) {
        e = cudaStreamCreateWithFlags(&P.gstream[g], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.gjoin[g], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        for (int g = 0; g < bf_plan_s::kGroups; ++g) {
            if (P.gstream[g]) cudaStreamDestroy(P.gstream[g]);
            if (P.gjoin[g]) cudaEventDestroy(P.gjoin[g]);
            P.gstream[g] = nullptr;
            P.gjoin[g] = nullptr;
        }
        if (fork) cudaEventDestroy(fork);
        return cuda_fail(e);
    }
    P.gfork = fork;
    return BF_OK;
}

// The fused path with host buffers, its copies overlapping the kernels.  The
// m tree nodes split into G groups of consecutive nodes, each on a side
// stream forked from the caller's: the group's input points are copied in
// and its down-kernel CTAs run; after the join (the up half needs every
// node's segment), each group's up-kernel CTAs run and its output points are
// copied back on the same side stream, and the caller's stream joins them.
// Every node-dependent address in the kernels is linear in the node index
// (input and output points, factor chunk, level-h segment, the M^h gather and
// S row), so a group is the same kernel on pointers shifted by its first node;
// the checked build's extents shrink by the same offsets.  `src` / `dst` are
// the caller's host pointers (ld) or device pointers, as host_in / host_out say.
template <int T>
cudaError_t launch_pair_groups(const bf_plan_s &P, const Direction &D, const float2 *src, bool host_in, float2 *dst,
                               bool host_out, long long ld, int nrhs, cudaStream_t s) {
    const int G = (int)std::min<long long>(bf_plan_s::kGroups, P.m), per = P.m / G;
    const long long npts = P.N / P.m, nseg = (long long)P.m * P.r;   // points per node, segment length
    const dim3 grid((nrhs + T - 1) / T, per);
    const dim3 block(P.consumers + 32);
    const size_t smem = plan_smem(P, T);
    const float2 *din = host_in ? P.d_stage_in : src;
    const long long ld_in = host_in ? P.N : ld;
    float2 *dout = host_out ? P.d_stage_out : dst;
    const long long ld_out = host_out ? P.N : ld;
    cudaError_t e = cudaEventRecord(P.gfork, s);
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        const long long n0 = (long long)g * per;
        cudaStream_t gs = P.gstream[g];
        e = cudaStreamWaitEvent(gs, P.gfork, 0);
        if (e == cudaSuccess && host_in)
            e = cudaMemcpy2DAsync(P.d_stage_in + n0 * npts, P.N * 8, src + n0 * npts, ld * 8, per * npts * 8, nrhs,
                                  cudaMemcpyHostToDevice, gs);
        if (e != cudaSuccess) break;
        Params pd = base_params(P, D.down);
        pd.fac += n0 * pd.cta_len;
        pd.fac_elems -= n0 * pd.cta_len;
        pd.in = din + n0 * npts;
        pd.ld_in = ld_in;
        pd.out = P.d_ws + n0 * nseg;
        pd.ld_out = P.R;
        pd.nrhs = nrhs;
        pd.in_elems = (long long)(nrhs - 1) * ld_in + P.N - n0 * npts;
        pd.out_elems = P.R * ws_rhs(P) - n0 * nseg;
        bfk::bf_down_kernel<T><<<grid, block, smem, gs>>>(pd);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(P.gjoin[g], gs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, P.gjoin[g], 0);
    }
    if (e == cudaSuccess) e = cudaEventRecord(P.gfork, s);
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        const long long n0 = (long long)g * per;
        cudaStream_t gs = P.gstream[g];
        e = cudaStreamWaitEvent(gs, P.gfork, 0);
        if (e != cudaSuccess) break;
        Params pu = base_params(P, D.up);
        pu.fac += n0 * pu.cta_len;
        pu.fac_elems -= n0 * pu.cta_len;
        pu.in = P.d_ws + n0 * P.r;
        pu.ld_in = P.R;
        pu.S = D.d_S + n0 * nseg;
        pu.s_elems -= n0 * nseg;
        pu.out = dout + n0 * npts;
        pu.ld_out = ld_out;
        pu.nrhs = nrhs;
        pu.in_elems = P.R * ws_rhs(P) - n0 * P.r;
        pu.out_elems = (long long)(nrhs - 1) * ld_out + P.N - n0 * npts;
        bfk::bf_up_kernel<T><<<grid, block, smem, gs>>>(pu);
        e = cudaGetLastError();
        if (e == cudaSuccess && host_out)
            e = cudaMemcpy2DAsync(dst + n0 * npts, ld * 8, P.d_stage_out + n0 * npts, P.N * 8, per * npts * 8, nrhs,
                                  cudaMemcpyDeviceToHost, gs);
        if (e == cudaSuccess) e = cudaEventRecord(P.gjoin[g], gs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, P.gjoin[g], 0);
    }
    return e;
}

bf_status run(bf_plan P, const void *in, void *out, int nrhs, long long ld, cudaStream_t s, bool adjoint) {
    bfint::NvtxRange range(adjoint ? "bf_apply_adjoint" : "bf_apply");
    if (!P || !in || !out || nrhs < 0 || ld < P->N) return BF_ERR_INVALID;
    if (nrhs == 0) return BF_OK;
    const char *ib = static_cast<const char *>(in);
    const char *ob = static_cast<const char *>(out);
    const long long span = ((long long)(nrhs - 1) * ld + P->N) * 8;
    if (ib < ob + span && ob < ib + span) return BF_ERR_INVALID;
    if (!on_plan_device(*P)) return BF_ERR_INVALID;
    const Direction &D = adjoint ? P->adj : P->fwd;
    const bool host_in = is_host_pointer(in), host_out = is_host_pointer(out);
    if (host_in || host_out) {
        const bf_status st = ensure_staging(*P);
        if (st != BF_OK) return st;
    }
    for (int c0 = 0; c0 < nrhs; c0 += P->nrhs_max) {
        const int nc = std::min(P->nrhs_max, nrhs - c0);
        const float2 *src = static_cast<const float2 *>(in) + (long long)c0 * ld;
        float2 *dst = static_cast<float2 *>(out) + (long long)c0 * ld;
        long long ld_in = ld, ld_out = ld;
        const bool fused = !(P->tc && nc >= P->tc_min) && !(P->wide && nc >= P->wide_min);
        if (fused && (host_in || host_out) && !P->profiling && P->m >= 2) {   // copies overlap the kernels
            const bf_status st = ensure_groups(*P);
            if (st != BF_OK) return st;
            const int T = pick_T(*P, nc);
            const cudaError_t e =
                T == 4 ? launch_pair_groups<4>(*P, D, src, host_in, dst, host_out, ld, nc, s)
                : T == 2 ? launch_pair_groups<2>(*P, D, src, host_in, dst, host_out, ld, nc, s)
                         : launch_pair_groups<1>(*P, D, src, host_in, dst, host_out, ld, nc, s);
            if (e != cudaSuccess) return cuda_fail(e);
            continue;
        }
        if (host_in) {
            if (ld == P->N)   // contiguous columns: one plain copy
                BF_CUDA(cudaMemcpyAsync(P->d_stage_in, src, (size_t)nc * P->N * 8, cudaMemcpyHostToDevice, s));
            else
                BF_CUDA(cudaMemcpy2DAsync(P->d_stage_in, P->N * 8, src, ld * 8, P->N * 8, nc, cudaMemcpyHostToDevice,
                                          s));
            src = P->d_stage_in;
            ld_in = P->N;
        }
        float2 *kdst = host_out ? P->d_stage_out : dst;
        if (host_out) ld_out = P->N;
        Timing *tm = next_timing(*P);
        cudaError_t e;
        if (P->tc && nc >= P->tc_min) {
            // tensor-core multi-RHS core (RHS tiles of 32-128).  Its TMA row
            // copies and 16-byte stores need aligned vectors with an even leading
            // dimension; others go through the (aligned) staging buffers.
            auto aligned = [](const void *q, long long l) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0 && (l & 1) == 0; };
            if (!aligned(src, ld_in) || !aligned(kdst, ld_out)) {
                const bf_status st = ensure_staging(*P);
                if (st != BF_OK) return st;
                if (!aligned(src, ld_in)) {
                    BF_CUDA(cudaMemcpy2DAsync(P->d_stage_in, P->N * 8, src, ld_in * 8, P->N * 8, nc,
                                              cudaMemcpyDeviceToDevice, s));
                    src = P->d_stage_in;
                    ld_in = P->N;
                }
            }
            if (!aligned(kdst, ld_out)) {
                e = launch_tc(*P, adjoint ? P->tadj : P->tfwd, src, ld_in, P->d_stage_out, P->N, nc, s, tm);
                if (e == cudaSuccess)
                    e = cudaMemcpy2DAsync(kdst, ld_out * 8, P->d_stage_out, P->N * 8, P->N * 8, nc,
                                          cudaMemcpyDeviceToDevice, s);
            } else {
                e = launch_tc(*P, adjoint ? P->tadj : P->tfwd, src, ld_in, kdst, ld_out, nc, s, tm);
            }
        } else if (P->wide && nc >= P->wide_min) {
            // CUDA-core multi-RHS core: RHS tile = smallest of 16/32/64 covering nc, capped by the plan
            const WideDirection &WD = adjoint ? P->wadj : P->wfwd;
            const int NR = std::min(WD.cfg.nr_max, nc <= 16 ? 16 : nc <= 32 ? 32 : 64);
            e = NR == 64 ? launch_wide<64>(*P, WD, D.d_S, src, ld_in, kdst, ld_out, nc, s, tm)
              : NR == 32 ? launch_wide<32>(*P, WD, D.d_S, src, ld_in, kdst, ld_out, nc, s, tm)
                         : launch_wide<16>(*P, WD, D.d_S, src, ld_in, kdst, ld_out, nc, s, tm);
        } else {
            const int T = pick_T(*P, nc);
            e = T == 4 ? launch_pair<4>(*P, D, src, ld_in, kdst, ld_out, nc, s, tm)
              : T == 2 ? launch_pair<2>(*P, D, src, ld_in, kdst, ld_out, nc, s, tm)
                       : launch_pair<1>(*P, D, src, ld_in, kdst, ld_out, nc, s, tm);
        }
        if (e != cudaSuccess) return cuda_fail(e);
        if (host_out) {
            if (ld == P->N)
                BF_CUDA(cudaMemcpyAsync(dst, P->d_stage_out, (size_t)nc * P->N * 8, cudaMemcpyDeviceToHost, s));
            else
                BF_CUDA(cudaMemcpy2DAsync(dst, ld * 8, P->d_stage_out, P->N * 8, P->N * 8, nc, cudaMemcpyDeviceToHost,
                                          s));
        }
    }
    return BF_OK;
}

// ---------------------------------------------------------------------------
// Static scratch for bf_apply_static_scratch: the level-h vector lives in this
// file-scope device array instead of a cudaMalloc'd workspace.  Every GPU that
// loads the library holds it (16 MiB) until the process exits.
constexpr long long kStaticScratchEntries = 1LL << 21;   // complex64 entries
static __device__ __align__(256) float2 bf_static_scratch[kStaticScratchEntries];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
struct ScratchAddress {
    unsigned long long ctx_id = 0;   // context the address belongs to (0: none looked up yet)
    void *p = nullptr;
};
ScratchAddress g_scratch_address[kMaxDevices];

// Identity of the calling thread's current context (cuCtxGetCurrent +
// cuCtxGetId through the runtime's driver entry points); 0 if unavailable.
// A device reset destroys the primary context, and the one the runtime makes
// next has a new identity, so an address looked up before the reset is
// never reused after it.
unsigned long long current_context_id() {
    using GetCurrentFn = CUresult (*)(CUcontext *);
    using GetIdFn = CUresult (*)(CUcontext, unsigned long long *);
    static const std::pair<GetCurrentFn, GetIdFn> fns = [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess)
            a = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            b = nullptr;
        cudaGetLastError();
        return std::make_pair(reinterpret_cast<GetCurrentFn>(a), reinterpret_cast<GetIdFn>(b));
    }();
    if (!fns.first || !fns.second) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (fns.first(&ctx) != CUDA_SUCCESS || !ctx || fns.second(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of bf_static_scratch on the current device.  The host-side
// name of the array is only a stand-in; the address is looked up with the
// device current (cudaGetSymbolAddress, return code checked) the first time
// a device's context is seen, and cached per device together with that
// context's identity.  If the identity cannot be read, it is looked up on
// every call.
bf_status static_scratch_address(float2 **out) {
    int dev = 0;
    BF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return BF_ERR_UNSUPPORTED;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchAddress &c = g_scratch_address[dev];
    if (ctx == 0 || c.ctx_id != ctx || !c.p) {
        void *p = nullptr;
        BF_CUDA(cudaGetSymbolAddress(&p, bf_static_scratch));
        c.p = p;
        c.ctx_id = ctx;
    }
    *out = static_cast<float2 *>(c.p);
    return BF_OK;
}

template <int T>
cudaError_t launch_pair_static(const bf_plan_s &P, const Direction &D, const float2 *in, long long ld_in,
                               float2 *out, long long ld_out, int nrhs, float2 *ws, cudaStream_t s) {
    const dim3 grid((nrhs + T - 1) / T, P.m);
    const dim3 block(P.consumers + 32);
    const size_t smem = plan_smem(P, T);
    Params pd = base_params(P, D.down);
    pd.in = in;
    pd.ld_in = ld_in;
    pd.out = ws;
    pd.ld_out = P.R;
    pd.nrhs = nrhs;
    pd.in_elems = (long long)(nrhs - 1) * ld_in + P.N;
    pd.out_elems = kStaticScratchEntries;
    Params pu = base_params(P, D.up);
    pu.in = ws;
    pu.ld_in = P.R;
    pu.out = out;
    pu.ld_out = ld_out;
    pu.S = D.d_S;
    pu.nrhs = nrhs;
    pu.in_elems = kStaticScratchEntries;
    pu.out_elems = (long long)(nrhs - 1) * ld_out + P.N;
    bfk::bf_down_kernel<T><<<grid, block, smem, s>>>(pd);
    bfk::bf_up_kernel<T><<<grid, block, smem, s>>>(pu);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// Ring and path configuration of a plan.
struct PlanCfg {
    int consumers = 256;
    int slot_kb = 64;
    int stages = 3;
    size_t smem_limit = kMaxSmem;
    bool fused_only = false;   // no multi-RHS cores (grouped batches use the fused kernels)
    bool no_tc = false;        // no tensor-core core (routed batch operators use the CUDA-core one)
    int wide_min = 0;          // smallest batch for the CUDA-core core (0: BF_WIDE_MIN, default 8)
};

PlanCfg env_plan_cfg() {
    PlanCfg c;
    c.consumers = std::min(256, std::max(32, env_int("BF_CONSUMERS", 256) / 32 * 32));
    c.slot_kb = env_int("BF_SLOT_KB", 64);
    c.stages = std::max(2, env_int("BF_STAGES", 3));
    return c;
}

bf_status create_plan(bf_plan *plan, const bf_desc *desc, const bf_factors *f, cudaStream_t stream,
                      const PlanCfg &cfg) {
    if (!plan) return BF_ERR_INVALID;
    *plan = nullptr;
    if (!desc || !f) return BF_ERR_INVALID;
    const int L = desc->L, n0 = desc->leaf, r = desc->r;
    if (L < 0 || (L & 1) || n0 < 1 || r < 1 || desc->nrhs_max < 1) return BF_ERR_INVALID;
    if (f->dtype != BF_C64 && f->dtype != BF_C128) return BF_ERR_INVALID;
    if (!f->VL || !f->UL || !f->S) return BF_ERR_INVALID;
    if (L > 0 && (!f->H || !f->G)) return BF_ERR_INVALID;
    if (L > 24 || r > 32 || n0 > 64) return BF_ERR_UNSUPPORTED;
    for (int t = 0; t < L / 2; ++t)
        if (!f->H[t] || !f->G[t]) return BF_ERR_INVALID;
    bf_plan_s *P = new (std::nothrow) bf_plan_s();
    if (!P) return BF_ERR_NOMEM;
    P->L = L;
    P->n0 = n0;
    P->r = r;
    P->h = L / 2;
    P->m = 1 << P->h;
    P->W = std::max(n0, r);
    P->nrhs_max = desc->nrhs_max;
    P->N = (long long)n0 << L;
    P->R = (1LL << L) * r;
    if (cudaGetDevice(&P->device) != cudaSuccess) {
        delete P;
        return cuda_fail(cudaErrorInvalidDevice);
    }
    if ((long long)P->m * P->W > 8192) {
        delete P;
        return BF_ERR_UNSUPPORTED;
    }
    // Ring: `stages` slots of `slot_len` complex entries; one slot must hold a
    // whole 2r x 2r butterfly (4r^2) and a whole leaf (n0 r).
    // Defaults measured on GB300 at N = 2^20, r = 16: 256 consumers, 64 KB
    // slots and as many slots as fit (2 there) stream at the HBM copy rate.
    P->consumers = cfg.consumers;
    P->inject_stall = env_int("BF_INJECT_STALL", 0) == 1 ? 1 : 0;
    int slot_len = cfg.slot_kb * 128;
    const int slot_min = std::max(4 * r * r, n0 * r + 1);
    slot_len = std::max(slot_len, slot_min);
    P->slot_len = (slot_len + 1) & ~1;
    P->stages = std::max(2, cfg.stages);
    while (P->stages > 2 && plan_smem(*P, 1) > cfg.smem_limit) --P->stages;
    // Large node segments (m max(n0, r) near 8192) leave less room for the
    // ring: halve the slots while they still hold a whole unit.
    while (plan_smem(*P, 1) > cfg.smem_limit && P->slot_len / 2 >= slot_min) P->slot_len = ((P->slot_len / 2) + 1) & ~1;
    if (plan_smem(*P, 1) > cfg.smem_limit) {
        delete P;
        return BF_ERR_UNSUPPORTED;
    }
    bf_status st = BF_OK;
    auto fail = [&](bf_status e) {
        free_plan(P);
        return e;
    };
    if ((st = set_smem_attr<1>(plan_smem(*P, 1))) != BF_OK) return fail(st);
    if (plan_smem(*P, 2) <= (size_t)kMaxSmem && (st = set_smem_attr<2>(plan_smem(*P, 2))) != BF_OK) return fail(st);
    if (plan_smem(*P, 4) <= (size_t)kMaxSmem && (st = set_smem_attr<4>(plan_smem(*P, 4))) != BF_OK) return fail(st);
    make_levels(P->fwd.down, true, P->h, P->m, n0, r, P->slot_len);
    make_levels(P->fwd.up, false, P->h, P->m, n0, r, P->slot_len);
    make_levels(P->adj.down, true, P->h, P->m, n0, r, P->slot_len);
    make_levels(P->adj.up, false, P->h, P->m, n0, r, P->slot_len);
    if ((st = upload_stream(*P, P->fwd.down, FWD_DOWN, *f)) != BF_OK) return fail(st);
    if ((st = upload_stream(*P, P->fwd.up, FWD_UP, *f)) != BF_OK) return fail(st);
    if ((st = upload_stream(*P, P->adj.down, ADJ_DOWN, *f)) != BF_OK) return fail(st);
    if ((st = upload_stream(*P, P->adj.up, ADJ_UP, *f)) != BF_OK) return fail(st);
    if ((st = upload_S(*P, *f)) != BF_OK) return fail(st);
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            P->num_sms = 1;
        cudaGetLastError();
    }
    // Multi-RHS cores for batches.  CUDA-core: built when the plan may see
    // nrhs >= wide_min (8).  Tensor-core: built when nrhs_max >= tc_min (32)
    // and every pass's dense blocks fit the core; each call uses it for
    // batches of at least tc_min (measured on GB300 at N = 2^20, r = 16: from
    // 32 RHS on, 128-RHS work items beat the CUDA-core core even part-filled).
    P->wide_min = cfg.fused_only ? (1 << 30) : cfg.wide_min > 0 ? cfg.wide_min : env_int("BF_WIDE_MIN", 8);
    P->tc_min = cfg.fused_only ? (1 << 30) : env_int("BF_TC_MIN", 32);
    if (P->nrhs_max >= P->wide_min) {
        WideCfg c;
        c.tc = false;
        c.stages = std::max(2, env_int("BF_WIDE_STAGES", 2));
        c.kmax = std::max(1, env_int("BF_WIDE_KMAX", (P->h + 1) / 2));   // two passes per half
        int wl = env_int("BF_WIDE_SLOT_KB", 32) * 128;
        wl = std::max(wl, std::max(4 * r * r, n0 * r + 1));
        c.slot_len = (wl + 1) & ~1;
        c.nr_max = wide_nr_max(*P, c);
        if (c.nr_max > 0) {
            P->wide = true;
            for (int NR : {16, 32, 64}) {
                if (NR > c.nr_max) break;
                const size_t b = wide_smem(*P, c, NR);
                st = NR == 64 ? set_wide_attr<64>(b) : NR == 32 ? set_wide_attr<32>(b) : set_wide_attr<16>(b);
                if (st != BF_OK) return fail(st);
            }
            make_wide_passes(P->wfwd, *P, c);
            make_wide_passes(P->wadj, *P, c);
        }
    }
    if (P->nrhs_max >= std::max(P->tc_min, 1) && env_int("BF_TC", 1) == 1 && !cfg.no_tc) {
        // Groups of G = 4 slots (two levels per pass) when the dense blocks fit
        // (G max(n0, r) <= 64), else G = 2 or 1; BF_TC_KMAX caps the slot bits.
        int kb = 2;
        while (kb > 0 && (1 << kb) * std::max(n0, r) > bftc::kMaxDim) --kb;
        WideCfg c;
        c.tc = true;
        c.kmax = std::max(1, std::min(env_int("BF_TC_KMAX", kb), std::max(kb, 1)));
        c.slot_len = 1 << 30;   // unused: one dense block per chunk
        make_wide_passes(P->tfwd, *P, c);
        make_wide_passes(P->tadj, *P, c);
        const bool fits = (1 << std::min(c.kmax, std::max(P->h, 0))) * std::max(n0, r) <= bftc::kMaxDim;
        if (fits && set_tc_dims(P->tfwd, *P) && set_tc_dims(P->tadj, *P)) {
            P->tc = true;
            if (bfint::tc_prepare() != cudaSuccess)
                return fail(cuda_fail(cudaErrorInvalidValue));
        } else {
            P->tfwd.pass.clear();
            P->tadj.pass.clear();
        }
    }
    for (auto *D : {&P->wfwd, &P->wadj, &P->tfwd, &P->tadj}) {
        const bool adj = (D == &P->wadj || D == &P->tadj);
        for (auto &wp : D->pass)
            if ((st = upload_wide(*P, wp, adj, *f, D->cfg.tc)) != BF_OK) return fail(st);
    }
    if (P->wide || P->tc) {
        const size_t wsa = (size_t)P->R * ws_rhs(*P) * sizeof(float2);
        if (cudaMalloc(&P->d_wsA, wsa) != cudaSuccess) return fail(cuda_fail(cudaErrorMemoryAllocation));
        P->device_bytes += wsa;
    }
    const size_t ws = (size_t)P->R * ws_rhs(*P) * sizeof(float2);
    if (cudaMalloc(&P->d_ws, ws) != cudaSuccess) return fail(cuda_fail(cudaErrorMemoryAllocation));
    P->device_bytes += ws;
    if (cudaMalloc(&P->d_err, sizeof(unsigned)) != cudaSuccess) return fail(cuda_fail(cudaErrorMemoryAllocation));
    if (cudaMemsetAsync(P->d_err, 0, sizeof(unsigned), stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(cuda_fail(cudaErrorUnknown));
    *plan = P;
    return BF_OK;
}

}  // namespace

extern "C" {

bf_status bf_plan_create(bf_plan *plan, const bf_desc *desc, const bf_factors *f, cudaStream_t stream) {
    return create_plan(plan, desc, f, stream, env_plan_cfg());
}

bf_status bf_apply(bf_plan plan, const void *in, void *out, int nrhs, long long ld, cudaStream_t stream) {
    return run(plan, in, out, nrhs, ld, stream, false);
}

bf_status bf_apply_adjoint(bf_plan plan, const void *in, void *out, int nrhs, long long ld, cudaStream_t stream) {
    return run(plan, in, out, nrhs, ld, stream, true);
}

bf_status bf_plan_destroy(bf_plan plan) {
    if (!plan) return BF_OK;
    cudaDeviceSynchronize();
    free_plan(plan);
    return BF_OK;
}

bf_status bf_plan_check(bf_plan plan, cudaStream_t stream) {
    if (!plan) return BF_ERR_INVALID;
    unsigned h = 0;
    BF_CUDA(cudaMemcpyAsync(&h, plan->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    BF_CUDA(cudaStreamSynchronize(stream));
    if (h) {
        BF_CUDA(cudaMemsetAsync(plan->d_err, 0, sizeof(unsigned), stream));
        BF_CUDA(cudaStreamSynchronize(stream));
        return (h & bfk::kErrBounds) ? BF_ERR_INVALID : BF_ERR_TIMEOUT;   // bounds: checked builds only
    }
    return BF_OK;
}

size_t bf_plan_device_bytes(bf_plan plan) { return plan ? plan->device_bytes : 0; }

bf_status bf_plan_set_profiling(bf_plan plan, int enable) {
    if (!plan) return BF_ERR_INVALID;
    plan->profiling = enable != 0;
    return BF_OK;
}

bf_status bf_plan_kernel_times(bf_plan plan, int *down_launches, double *down_ms, int *up_launches, double *up_ms) {
    if (!plan || !down_launches || !down_ms || !up_launches || !up_ms) return BF_ERR_INVALID;
    BF_CUDA(cudaDeviceSynchronize());
    double d = 0, u = 0;
    for (size_t i = 0; i < plan->timing_used; ++i) {
        float a = 0, b = 0;
        BF_CUDA(cudaEventElapsedTime(&a, plan->timings[i].a, plan->timings[i].b));
        BF_CUDA(cudaEventElapsedTime(&b, plan->timings[i].b, plan->timings[i].c));
        d += a;
        u += b;
    }
    *down_launches = *up_launches = (int)plan->timing_used;
    *down_ms = d;
    *up_ms = u;
    plan->timing_used = 0;
    return BF_OK;
}

bf_status bf_apply_static_scratch(bf_plan plan, const void *in, void *out, int nrhs, long long ld, int adjoint,
                                  cudaStream_t stream) {
    bfint::NvtxRange range("bf_apply_static_scratch");
    bf_plan P = plan;
    if (!P || !in || !out || nrhs < 0 || ld < P->N) return BF_ERR_INVALID;
    if (P->R > kStaticScratchEntries) return BF_ERR_UNSUPPORTED;   // one vector's level-h data must fit
    if (nrhs == 0) return BF_OK;
    const char *ib = static_cast<const char *>(in);
    const char *ob = static_cast<const char *>(out);
    const long long span = ((long long)(nrhs - 1) * ld + P->N) * 8;
    if (ib < ob + span && ob < ib + span) return BF_ERR_INVALID;
    if (is_host_pointer(in) || is_host_pointer(out)) return BF_ERR_INVALID;   // staging would allocate
    if (!on_plan_device(*P)) return BF_ERR_INVALID;   // the scratch address is per device
    float2 *ws = nullptr;
    bf_status st = static_scratch_address(&ws);
    if (st != BF_OK) return st;
    const Direction &D = adjoint ? P->adj : P->fwd;
    const int per_pass = (int)std::min<long long>(kStaticScratchEntries / P->R, 1 << 30);
    for (int c0 = 0; c0 < nrhs; c0 += per_pass) {
        const int nc = std::min(per_pass, nrhs - c0);
        const float2 *src = static_cast<const float2 *>(in) + (long long)c0 * ld;
        float2 *dst = static_cast<float2 *>(out) + (long long)c0 * ld;
        const int T = pick_T(*P, nc);
        cudaError_t e = T == 4 ? launch_pair_static<4>(*P, D, src, ld, dst, ld, nc, ws, stream)
                      : T == 2 ? launch_pair_static<2>(*P, D, src, ld, dst, ld, nc, ws, stream)
                               : launch_pair_static<1>(*P, D, src, ld, dst, ld, nc, ws, stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return BF_OK;
}

const char *bf_status_string(bf_status s) {
    switch (s) {
        case BF_OK: return "BF_OK";
        case BF_ERR_INVALID: return "BF_ERR_INVALID: invalid argument";
        case BF_ERR_CUDA: return "BF_ERR_CUDA: a CUDA runtime call failed";
        case BF_ERR_NOMEM: return "BF_ERR_NOMEM: out of memory";
        case BF_ERR_UNSUPPORTED: return "BF_ERR_UNSUPPORTED: shape outside the library's compiled limits";
        case BF_ERR_TIMEOUT: return "BF_ERR_TIMEOUT: a kernel wait expired";
        case BF_ERR_CORRUPT: return "BF_ERR_CORRUPT: a factor file failed its checks";
    }
    return "unknown bf_status";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent operators (bf_batch_*): one internal fused-path plan
// per operator, all of them run by two grouped launches (every operator's
// down half, then every up half), optionally replayed from a CUDA graph.

struct bf_batch_s {
    int n = 0, T = 1, nitems = 0;
    std::vector<bf_plan> plans;
    Params *d_params = nullptr;           // [fwd down, fwd up, adj down, adj up] x n
    bfk::GroupItem *d_items = nullptr;    // (operator, node, RHS tile), largest operators first
    size_t smem = 0;                      // dynamic shared memory of the grouped launches
    std::vector<const void *> in;
    std::vector<void *> out;
    std::vector<int> nrhs;
    std::vector<long long> ld;
    cudaStream_t cap = nullptr;           // private stream for graph capture
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::vector<int> routed;              // operators on their own multi-RHS passes
    static constexpr int kSide = 8;       // side streams for the routed operators (4 measured the same)
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {};
};

namespace {

template <int T>
cudaError_t launch_grouped(const bf_batch_s &B, bool adjoint, cudaStream_t s) {
    const Params *pl = B.d_params + (adjoint ? 2 : 0) * B.n;
    bfk::bf_down_grouped<T><<<B.nitems, 256 + 32, B.smem, s>>>(pl, B.d_items);
    bfk::bf_up_grouped<T><<<B.nitems, 256 + 32, B.smem, s>>>(pl + B.n, B.d_items);
    return cudaGetLastError();
}

cudaError_t grouped_only(const bf_batch_s &B, bool adjoint, cudaStream_t s) {
    if (B.nitems == 0) return cudaSuccess;
    return B.T == 8   ? launch_grouped<8>(B, adjoint, s)
         : B.T == 4 ? launch_grouped<4>(B, adjoint, s)
         : B.T == 2 ? launch_grouped<2>(B, adjoint, s)
                    : launch_grouped<1>(B, adjoint, s);
}

// One routed operator: its plan's CUDA-core multi-RHS passes on its vectors.
cudaError_t launch_routed(const bf_batch_s &B, int o, bool adjoint, cudaStream_t s) {
    const bf_plan_s &P = *B.plans[o];
    const WideDirection &WD = adjoint ? P.wadj : P.wfwd;
    const Direction &D = adjoint ? P.adj : P.fwd;
    const int nc = B.nrhs[o];
    const float2 *in = static_cast<const float2 *>(B.in[o]);
    float2 *out = static_cast<float2 *>(B.out[o]);
    const int NR = std::min(WD.cfg.nr_max, nc <= 16 ? 16 : nc <= 32 ? 32 : 64);
    return NR == 64 ? launch_wide<64>(P, WD, D.d_S, in, B.ld[o], out, B.ld[o], nc, s, nullptr)
         : NR == 32 ? launch_wide<32>(P, WD, D.d_S, in, B.ld[o], out, B.ld[o], nc, s, nullptr)
                    : launch_wide<16>(P, WD, D.d_S, in, B.ld[o], out, B.ld[o], nc, s, nullptr);
}

// The whole batch on stream s: the routed operators' passes on the side
// streams (forked from s first, joined back at the end) beside the grouped
// launches on s.  Usable under stream capture.
cudaError_t grouped(const bf_batch_s &B, bool adjoint, cudaStream_t s) {
    if (B.routed.empty()) return grouped_only(B, adjoint, s);
    cudaError_t e = cudaEventRecord(B.fork, s);
    for (int k = 0; k < bf_batch_s::kSide && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(B.side[k], B.fork, 0);
    if (e == cudaSuccess) e = grouped_only(B, adjoint, s);
    for (size_t i = 0; i < B.routed.size() && e == cudaSuccess; ++i)
        e = launch_routed(B, B.routed[i], adjoint, B.side[i % bf_batch_s::kSide]);
    for (int k = 0; k < bf_batch_s::kSide && e == cudaSuccess; ++k) {
        e = cudaEventRecord(B.join[k], B.side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, B.join[k], 0);
    }
    return e;
}

template <int T>
bf_status set_grouped_attr(size_t bytes) {
    (void)bytes;   // shared by all batches: the maximum next to the static Params copy
    BF_CUDA(cudaFuncSetAttribute(bfk::bf_down_grouped<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMaxSmem - 1024));
    BF_CUDA(cudaFuncSetAttribute(bfk::bf_up_grouped<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMaxSmem - 1024));
    return BF_OK;
}

void free_batch(bf_batch_s *B) {
    if (!B) return;
    for (auto &e : B->exec)
        if (e) cudaGraphExecDestroy(e);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (int k = 0; k < bf_batch_s::kSide; ++k) {
        if (B->side[k]) cudaStreamDestroy(B->side[k]);
        if (B->join[k]) cudaEventDestroy(B->join[k]);
    }
    if (B->fork) cudaEventDestroy(B->fork);
    cudaFree(B->d_params);
    cudaFree(B->d_items);
    for (bf_plan p : B->plans) free_plan(p);
    cudaGetLastError();
    delete B;
}

}  // namespace

extern "C" {

bf_status bf_batch_create(bf_batch *out, int n, const bf_desc *descs, const bf_factors *factors,
                          const void *const *in, void *const *outv, const int *nrhs, const long long *ld,
                          const bf_batch_config *cfg, cudaStream_t stream) {
    if (!out) return BF_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || !descs || !factors || !in || !outv || !nrhs || !ld) return BF_ERR_INVALID;
    const int T = cfg && cfg->T ? cfg->T : 1;
    if (T != 1 && T != 2 && T != 4 && T != 8) return BF_ERR_INVALID;
    for (int o = 0; o < n; ++o) {
        if (!in[o] || !outv[o] || nrhs[o] < 1 || nrhs[o] > descs[o].nrhs_max) return BF_ERR_INVALID;
        if (ld[o] < ((long long)descs[o].leaf << descs[o].L)) return BF_ERR_INVALID;
        if (is_host_pointer(in[o]) || is_host_pointer(outv[o])) return BF_ERR_INVALID;
    }
    bf_batch_s *B = new (std::nothrow) bf_batch_s();
    if (!B) return BF_ERR_NOMEM;
    B->n = n;
    B->T = T;
    PlanCfg pc;
    pc.consumers = 256;
    pc.slot_kb = cfg && cfg->slot_kb ? cfg->slot_kb : 16;
    pc.stages = cfg && cfg->stages ? cfg->stages : 2;
    pc.fused_only = true;
    pc.smem_limit = kMaxSmem - 2048;   // the grouped kernels' Params copy is static shared memory
    const int route_rhs = cfg && cfg->route_min_rhs ? cfg->route_min_rhs : 8;
    const int route_L = cfg && cfg->route_min_L ? cfg->route_min_L : 6;
    std::vector<Params> host(4 * (size_t)n);
    std::vector<bfk::GroupItem> items;
    std::vector<std::pair<long long, int>> order;   // (work, operator)
    for (int o = 0; o < n; ++o) {
        bf_plan P = nullptr;
        const bool route = route_rhs > 0 && nrhs[o] >= route_rhs && descs[o].L >= route_L;
        bf_status st = BF_OK;
        if (route) {   // its own plan with the CUDA-core multi-RHS core (no tensor-core blocks)
            PlanCfg rc;
            rc.no_tc = true;
            rc.wide_min = route_rhs;
            st = create_plan(&P, &descs[o], &factors[o], stream, rc);
            if (st == BF_OK && !P->wide) {   // the core does not take this shape: back to the group
                free_plan(P);
                P = nullptr;
            }
        }
        if (!P && st == BF_OK) st = create_plan(&P, &descs[o], &factors[o], stream, pc);
        if (st != BF_OK) {
            free_batch(B);
            return st;
        }
        B->plans.push_back(P);
        B->in.push_back(in[o]);
        B->out.push_back(outv[o]);
        B->nrhs.push_back(nrhs[o]);
        B->ld.push_back(ld[o]);
        if (P->wide) {
            B->routed.push_back(o);
            continue;
        }
        if (plan_smem(*P, T) > pc.smem_limit) {
            free_batch(B);
            return BF_ERR_UNSUPPORTED;
        }
        B->smem = std::max(B->smem, plan_smem(*P, T));
        for (int dir = 0; dir < 2; ++dir) {
            const Direction &D = dir ? P->adj : P->fwd;
            Params pd = base_params(*P, D.down);
            pd.in = static_cast<const float2 *>(in[o]);
            pd.ld_in = ld[o];
            pd.out = P->d_ws;
            pd.ld_out = P->R;
            pd.nrhs = nrhs[o];
            pd.in_elems = (long long)(nrhs[o] - 1) * ld[o] + P->N;
            pd.out_elems = P->R * ws_rhs(*P);
            Params pu = base_params(*P, D.up);
            pu.in = P->d_ws;
            pu.ld_in = P->R;
            pu.out = static_cast<float2 *>(outv[o]);
            pu.ld_out = ld[o];
            pu.S = D.d_S;
            pu.nrhs = nrhs[o];
            pu.in_elems = P->R * ws_rhs(*P);
            pu.out_elems = (long long)(nrhs[o] - 1) * ld[o] + P->N;
            host[(size_t)(2 * dir) * n + o] = pd;
            host[(size_t)(2 * dir + 1) * n + o] = pu;
        }
        order.push_back({(long long)P->m * ((nrhs[o] + T - 1) / T) * (P->fwd.down.cta_len + P->fwd.up.cta_len), o});
    }
    if (!B->routed.empty()) {
        bool ok = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; k < bf_batch_s::kSide && ok; ++k)
            ok = cudaStreamCreateWithFlags(&B->side[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&B->join[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            free_batch(B);
            return cuda_fail(cudaErrorUnknown);
        }
    }
    std::sort(order.begin(), order.end(), [](auto &a, auto &b) { return a.first > b.first; });
    for (auto &w : order) {
        const bf_plan_s &P = *B->plans[w.second];
        for (int node = 0; node < P.m; ++node)
            for (int r0 = 0; r0 < nrhs[w.second]; r0 += T) items.push_back({w.second, node, r0, 0});
    }
    B->nitems = (int)items.size();
    bf_status st = BF_OK;
    st = T == 8   ? set_grouped_attr<8>(B->smem)
       : T == 4 ? set_grouped_attr<4>(B->smem)
       : T == 2 ? set_grouped_attr<2>(B->smem)
                : set_grouped_attr<1>(B->smem);
    if (st != BF_OK) {
        free_batch(B);
        return st;
    }
    if (cudaMalloc(&B->d_params, host.size() * sizeof(Params)) != cudaSuccess ||
        cudaMalloc(&B->d_items, items.size() * sizeof(bfk::GroupItem)) != cudaSuccess ||
        cudaMemcpy(B->d_params, host.data(), host.size() * sizeof(Params), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(B->d_items, items.data(), items.size() * sizeof(bfk::GroupItem), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        free_batch(B);
        return cuda_fail(cudaErrorMemoryAllocation);
    }
    *out = B;
    return BF_OK;
}

bf_status bf_batch_apply(bf_batch B, int adjoint, int mode, cudaStream_t stream) {
    bfint::NvtxRange range("bf_batch_apply");
    if (!B || mode < 0 || mode > 2) return BF_ERR_INVALID;
    const bool adj = adjoint != 0;
    if (mode == BF_BATCH_EACH) {   // one plan at a time: two launches per operator
        for (int o = 0; o < B->n; ++o) {
            bf_status st = run(B->plans[o], B->in[o], B->out[o], B->nrhs[o], B->ld[o], stream, adj);
            if (st != BF_OK) return st;
        }
        return BF_OK;
    }
    if (mode == BF_BATCH_GROUPED) {
        cudaError_t e = grouped(*B, adj, stream);
        return e == cudaSuccess ? BF_OK : cuda_fail(e);
    }
    // BF_BATCH_GRAPH: the two grouped launches captured once into a graph, then replayed.
    cudaGraphExec_t &ex = B->exec[adj ? 1 : 0];
    if (!ex) {
        if (!B->cap) BF_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        BF_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
        const cudaError_t e = grouped(*B, adj, B->cap);
        const cudaError_t e2 = cudaStreamEndCapture(B->cap, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(e != cudaSuccess ? e : e2);
        }
        const cudaError_t e3 = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e3 != cudaSuccess) {
            ex = nullptr;
            return cuda_fail(e3);
        }
    }
    BF_CUDA(cudaGraphLaunch(ex, stream));
    return BF_OK;
}

bf_status bf_batch_check(bf_batch B, cudaStream_t stream) {
    if (!B) return BF_ERR_INVALID;
    bf_status worst = BF_OK;
    for (bf_plan p : B->plans) {
        const bf_status st = bf_plan_check(p, stream);
        if (st != BF_OK) worst = st;
    }
    return worst;
}

int bf_batch_items(bf_batch B) { return B ? B->nitems : 0; }

// The tensor-core blocks of both directions split into the BF16 parts of the
// rung (split, bf16) (no parts kept for a TF32 rung), and the rung recorded.
// All new buffers are allocated before anything is released, so on
// BF_ERR_NOMEM the plan is unchanged; once they are installed the plan's rung
// is set to match them before any split runs, so a failure after that point
// can leave wrong values but never a rung that reads more parts than a buffer
// holds.  Synchronous: the splits run on the legacy default stream and are
// waited for.
static bf_status set_bf16_blocks(bf_plan_s &P, int split, int bf16) {
    const int parts = bf16 ? (split == 6 ? 3 : split == 3 ? 2 : 1) : 0;
    std::vector<WidePass *> todo;
    for (WideDirection *D : {&P.tfwd, &P.tadj})
        for (auto &wp : D->pass)
            if (wp.d16_parts != parts) todo.push_back(&wp);
    auto part_bytes = [&](const WidePass &wp) {
        return (size_t)P.m * wp.ngroups * 2 * wp.Nout * wp.Kin * sizeof(uint16_t);
    };
    std::vector<uint16_t *> fresh(todo.size(), nullptr);
    if (parts > 0)
        for (size_t i = 0; i < todo.size(); ++i)
            if (cudaMalloc(&fresh[i], part_bytes(*todo[i]) * parts) != cudaSuccess) {
                cudaGetLastError();
                for (uint16_t *q : fresh) cudaFree(q);
                return BF_ERR_NOMEM;
            }
    if (!todo.empty() && cudaDeviceSynchronize() != cudaSuccess)   // no launch reads the old parts
        return cuda_fail(cudaErrorUnknown);
    for (size_t i = 0; i < todo.size(); ++i) {
        WidePass &wp = *todo[i];
        cudaFree(wp.d16);
        P.device_bytes -= part_bytes(wp) * wp.d16_parts;
        wp.d16 = fresh[i];
        wp.d16_parts = parts;
        P.device_bytes += part_bytes(wp) * parts;
    }
    P.tc_split = split;
    P.tc_bf16 = bf16;
    if (parts == 0 || todo.empty()) return BF_OK;
    for (WidePass *w : todo) {
        WidePass &wp = *w;
        const long long nblocks = (long long)P.m * wp.ngroups;
        const long long chunks = nblocks * 2 * wp.Nout * wp.Kin / 8;
        const int grid = (int)std::min<long long>((chunks + 255) / 256, 8LL * P.num_sms);
        bftc::bf16_split_kernel<<<grid, 256>>>(reinterpret_cast<const float *>(wp.st.d),
                                               reinterpret_cast<uint4 *>(wp.d16), nblocks, 2 * wp.Nout, wp.Kin, parts);
        if (cudaGetLastError() != cudaSuccess) return cuda_fail(cudaErrorLaunchFailure);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail(cudaErrorUnknown);
    return BF_OK;
}

bf_status bf_plan_set_precision(bf_plan plan, int precision) {
    if (!plan) return BF_ERR_INVALID;
    int split, bf16;
    switch (precision) {
    case BF_PREC_FP32: split = 3; bf16 = 0; break;
    case BF_PREC_TF32: split = 1; bf16 = 0; break;
    case BF_PREC_BF16X3: split = 3; bf16 = 1; break;
    case BF_PREC_BF16: split = 1; bf16 = 1; break;
    case BF_PREC_BF16X6: split = 6; bf16 = 1; break;
    default: return BF_ERR_INVALID;
    }
    return set_bf16_blocks(*plan, split, bf16);
}

bf_status bf_batch_destroy(bf_batch B) {
    if (!B) return BF_OK;
    cudaDeviceSynchronize();
    free_batch(B);
    return BF_OK;
}

}  // extern "C"

namespace bfint {

template <int EPI>
cudaError_t tc_prepare_epi() {
    const cudaError_t e = cudaFuncSetAttribute(bftc::bf_tc_kernel<false, EPI>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bftc::Epi<EPI>::smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(bftc::bf_tc_kernel<true, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bftc::Epi<EPI>::smem);
}

cudaError_t tc_prepare() {
    const cudaError_t e = tc_prepare_epi<8>();
    return e != cudaSuccess ? e : tc_prepare_epi<16>();
}

// One tensor-core pass: 16 epilogue warps for tiles of up to 96 RHS, 8 for 128.
cudaError_t tc_launch(const bftc::TcParams &p, int grid, cudaStream_t s) {
    if (p.W <= 96) {
        if (p.bf16)
            bftc::bf_tc_kernel<true, 16><<<grid, bftc::Epi<16>::threads, bftc::Epi<16>::smem, s>>>(p);
        else
            bftc::bf_tc_kernel<false, 16><<<grid, bftc::Epi<16>::threads, bftc::Epi<16>::smem, s>>>(p);
    } else {
        if (p.bf16)
            bftc::bf_tc_kernel<true, 8><<<grid, bftc::Epi<8>::threads, bftc::Epi<8>::smem, s>>>(p);
        else
            bftc::bf_tc_kernel<false, 8><<<grid, bftc::Epi<8>::threads, bftc::Epi<8>::smem, s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t quad_tc_launch(const QuadTc &q, int num_sms, cudaStream_t s) {
    bftc::TcParams p;
    std::memset(&p, 0, sizeof(p));
    p.fac = q.fac;
    p.fac16 = q.fac16;
    p.in = q.in;
    p.out = q.out;
    p.R = q.R;
    p.err = q.err;
    p.load_kind = bftc::LD_QUAD;
    p.store_kind = bftc::ST_QUAD;
    p.m = 1;
    p.ngroups = 1;
    p.Kin = q.Kin;
    p.Nout = q.Nout;
    p.nrhs = q.nrhs;
    p.W = bftc::NR;   // the 2D CUDA-core edge levels read and write 128-wide planar tiles
    p.split = q.split;
    p.bf16 = q.bf16;
    p.stall = q.stall;
    p.q_ain = q.ain;
    p.q_bin = q.bin;
    p.q_sin = q.sin;
    p.q_aout = q.aout;
    p.q_bout = q.bout;
    p.q_sout = q.sout;
    p.q_bszi = q.bszi;
    p.q_bszo = q.bszo;
    p.q_nB = q.nB;
    p.q_ngroups = q.ngroups;
    p.q_parts = q.parts;
    p.q_chunks = q.chunks;
    const long long ntiles = (q.nrhs + bftc::NR - 1) / bftc::NR;
    const long long items = (long long)q.ngroups * q.parts * ntiles;
    const int grid = (int)std::min<long long>(items, num_sms);
    return tc_launch(p, grid, s);
}

cudaError_t bf16_split(const float *fac, uint16_t *out, long long nblocks, int rows, int Kin, int parts,
                       int num_sms) {
    const long long chunks = nblocks * rows * Kin / 8;
    const int grid = (int)std::min<long long>((chunks + 255) / 256, 8LL * num_sms);
    bftc::bf16_split_kernel<<<grid, 256>>>(fac, reinterpret_cast<uint4 *>(out), nblocks, rows, Kin, parts);
    return cudaGetLastError();
}

int tc_boff(int n, int k, int rows) { return bftc::boff(n, k, rows); }

}  // namespace bfint
