/*
 * Plain-C FP64 apply of a butterfly factorization and of its adjoint
 * (oracle, test infrastructure only; never linked into the product library).
 *
 *   u = U^L G^{L-1} ... G^h M^h (H^h)^* ... (H^{L-1})^* (V^L)^* g      (Eq. Kfactors)
 *
 * The same steps as oracle/apply.py, written as loops over the canonical
 * factor arrays (block layouts as in bfinputs/factors.py):
 *   leaf V   t[b r + k]                 = sum_p conj(V^L_b[p,k]) g[b n0 + p]         (Sec. 3.2.2)
 *   H level  t^l[(j s + 2i + d) r + k'] = sum_{c,k} conj(H^l_{2j+c,i}[k, d r + k'])
 *                                           * t^{l+1}[((2j+c) s/2 + i) r + k]        (mirror of Eq. RSh2)
 *   M^h      w[(i m + j) r + k]         = S_{i,j}[k] t[(j m + i) r + k]              (Eq. KeqUMV)
 *   G level  w^{l+1}[((2i+c) s/2 + j) r + k'] = sum_{d,k} G^l_{2i+c,j}[k', d r + k]
 *                                           * w^l[(i s + 2j + d) r + k]              (Eq. RSh2)
 *   leaf U   u[a n0 + p]                = sum_k U^L_a[p,k] w[a r + k]               (Eq. RFUh)
 * with s = 2^{L-l}.  The adjoint runs the conjugate transposes in reverse.
 *
 * Complex numbers are interleaved (re, im) doubles.  Vectors are column-major,
 * nrhs columns of N entries each.  Returns 0, or -1 on bad arguments / no memory.
 */
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cpx;

static inline cpx cmul(cpx a, cpx b) { cpx z = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; return z; }
static inline cpx cconj(cpx a) { cpx z = {a.re, -a.im}; return z; }
static inline void cacc(cpx *acc, cpx v) { acc->re += v.re; acc->im += v.im; }

static void forward_one(int L, int n0, int r, const cpx *VL, const cpx *const *H, const double *S,
                        const cpx *const *G, const cpx *UL, const cpx *g, cpx *u, cpx *x, cpx *y)
{
    const long nb = 1L << L;
    const int h = L / 2;
    const long m = 1L << h;
    long b;
    /* leaf V: t^L = (V^L)^* g */
#pragma omp parallel for schedule(static)
    for (b = 0; b < nb; ++b)
        for (int k = 0; k < r; ++k) {
            cpx acc = {0.0, 0.0};
            for (int p = 0; p < n0; ++p)
                cacc(&acc, cmul(cconj(VL[(b * n0 + p) * r + k]), g[b * n0 + p]));
            x[b * r + k] = acc;
        }
    /* H levels l = L-1 .. h */
    for (int l = L - 1; l >= h; --l) {
        const long nj = 1L << l, ni = 1L << (L - l - 1), s = 2 * ni;
        const cpx *Hl = H[l - h];
        long u_;
#pragma omp parallel for schedule(static)
        for (u_ = 0; u_ < nj * ni; ++u_) {
            const long j = u_ / ni, i = u_ % ni;
            for (int d = 0; d < 2; ++d)
                for (int kp = 0; kp < r; ++kp) {
                    cpx acc = {0.0, 0.0};
                    for (int c = 0; c < 2; ++c) {
                        const long blk = (2 * j + c) * ni + i;
                        for (int k = 0; k < r; ++k)
                            cacc(&acc, cmul(cconj(Hl[blk * 2L * r * r + (long)k * 2 * r + d * r + kp]), x[blk * r + k]));
                    }
                    y[(j * s + 2 * i + d) * r + kp] = acc;
                }
        }
        cpx *t = x; x = y; y = t;
    }
    /* M^h */
    long ij;
#pragma omp parallel for schedule(static)
    for (ij = 0; ij < m * m; ++ij) {
        const long i = ij / m, j = ij % m;
        for (int k = 0; k < r; ++k) {
            const double sk = S[(i * m + j) * r + k];
            const cpx v = x[(j * m + i) * r + k];
            cpx z = {sk * v.re, sk * v.im};
            y[(i * m + j) * r + k] = z;
        }
    }
    { cpx *t = x; x = y; y = t; }
    /* G levels l = h .. L-1 */
    for (int l = h; l < L; ++l) {
        const long ni = 1L << l, nj = 1L << (L - l - 1), s = 2 * nj;
        const cpx *Gl = G[l - h];
        long u_;
#pragma omp parallel for schedule(static)
        for (u_ = 0; u_ < ni * nj; ++u_) {
            const long i = u_ / nj, j = u_ % nj;
            for (int c = 0; c < 2; ++c) {
                const long blk = (2 * i + c) * nj + j;
                for (int kp = 0; kp < r; ++kp) {
                    cpx acc = {0.0, 0.0};
                    for (int d = 0; d < 2; ++d)
                        for (int k = 0; k < r; ++k)
                            cacc(&acc, cmul(Gl[blk * 2L * r * r + (long)kp * 2 * r + d * r + k], x[(i * s + 2 * j + d) * r + k]));
                    y[blk * r + kp] = acc;
                }
            }
        }
        cpx *t = x; x = y; y = t;
    }
    /* leaf U */
#pragma omp parallel for schedule(static)
    for (b = 0; b < nb; ++b)
        for (int p = 0; p < n0; ++p) {
            cpx acc = {0.0, 0.0};
            for (int k = 0; k < r; ++k)
                cacc(&acc, cmul(UL[(b * n0 + p) * r + k], x[b * r + k]));
            u[b * n0 + p] = acc;
        }
}

static void adjoint_one(int L, int n0, int r, const cpx *VL, const cpx *const *H, const double *S,
                        const cpx *const *G, const cpx *UL, const cpx *f, cpx *out, cpx *x, cpx *y)
{
    const long nb = 1L << L;
    const int h = L / 2;
    const long m = 1L << h;
    long b;
    /* (U^L)^* */
#pragma omp parallel for schedule(static)
    for (b = 0; b < nb; ++b)
        for (int k = 0; k < r; ++k) {
            cpx acc = {0.0, 0.0};
            for (int p = 0; p < n0; ++p)
                cacc(&acc, cmul(cconj(UL[(b * n0 + p) * r + k]), f[b * n0 + p]));
            x[b * r + k] = acc;
        }
    /* (G^l)^* for l = L-1 .. h */
    for (int l = L - 1; l >= h; --l) {
        const long ni = 1L << l, nj = 1L << (L - l - 1), s = 2 * nj;
        const cpx *Gl = G[l - h];
        long u_;
#pragma omp parallel for schedule(static)
        for (u_ = 0; u_ < ni * nj; ++u_) {
            const long i = u_ / nj, j = u_ % nj;
            for (int d = 0; d < 2; ++d)
                for (int k = 0; k < r; ++k) {
                    cpx acc = {0.0, 0.0};
                    for (int c = 0; c < 2; ++c) {
                        const long blk = (2 * i + c) * nj + j;
                        for (int kp = 0; kp < r; ++kp)
                            cacc(&acc, cmul(cconj(Gl[blk * 2L * r * r + (long)kp * 2 * r + d * r + k]), x[blk * r + kp]));
                    }
                    y[(i * s + 2 * j + d) * r + k] = acc;
                }
        }
        cpx *t = x; x = y; y = t;
    }
    /* (M^h)^* */
    long ij;
#pragma omp parallel for schedule(static)
    for (ij = 0; ij < m * m; ++ij) {
        const long i = ij / m, j = ij % m;
        for (int k = 0; k < r; ++k) {
            const double sk = S[(i * m + j) * r + k];
            const cpx v = x[(i * m + j) * r + k];
            cpx z = {sk * v.re, sk * v.im};
            y[(j * m + i) * r + k] = z;
        }
    }
    { cpx *t = x; x = y; y = t; }
    /* H^l for l = h .. L-1 */
    for (int l = h; l < L; ++l) {
        const long nj = 1L << l, ni = 1L << (L - l - 1), s = 2 * ni;
        const cpx *Hl = H[l - h];
        long u_;
#pragma omp parallel for schedule(static)
        for (u_ = 0; u_ < nj * ni; ++u_) {
            const long j = u_ / ni, i = u_ % ni;
            for (int c = 0; c < 2; ++c) {
                const long blk = (2 * j + c) * ni + i;
                for (int k = 0; k < r; ++k) {
                    cpx acc = {0.0, 0.0};
                    for (int d = 0; d < 2; ++d)
                        for (int kp = 0; kp < r; ++kp)
                            cacc(&acc, cmul(Hl[blk * 2L * r * r + (long)k * 2 * r + d * r + kp], x[(j * s + 2 * i + d) * r + kp]));
                    y[blk * r + k] = acc;
                }
            }
        }
        cpx *t = x; x = y; y = t;
    }
    /* V^L */
#pragma omp parallel for schedule(static)
    for (b = 0; b < nb; ++b)
        for (int p = 0; p < n0; ++p) {
            cpx acc = {0.0, 0.0};
            for (int k = 0; k < r; ++k)
                cacc(&acc, cmul(VL[(b * n0 + p) * r + k], x[b * r + k]));
            out[b * n0 + p] = acc;
        }
}

int oracle_bf_apply(int L, int n0, int r, const double *VL, const double *const *H,
                    const double *S, const double *const *G, const double *UL,
                    const double *in, double *out, long nrhs, int adjoint)
{
    if (L < 0 || (L & 1) || n0 < 1 || r < 1 || nrhs < 0 || !VL || !S || !UL || !in || !out)
        return -1;
    if (L > 0 && (!H || !G))
        return -1;
    const long N = (long)n0 << L, R = (1L << L) * r;
    cpx *x = (cpx *)malloc(sizeof(cpx) * (size_t)R);
    cpx *y = (cpx *)malloc(sizeof(cpx) * (size_t)R);
    if (!x || !y) { free(x); free(y); return -1; }
    for (long c = 0; c < nrhs; ++c) {
        const cpx *src = (const cpx *)in + c * N;
        cpx *dst = (cpx *)out + c * N;
        if (adjoint)
            adjoint_one(L, n0, r, (const cpx *)VL, (const cpx *const *)H, S, (const cpx *const *)G,
                        (const cpx *)UL, src, dst, x, y);
        else
            forward_one(L, n0, r, (const cpx *)VL, (const cpx *const *)H, S, (const cpx *const *)G,
                        (const cpx *)UL, src, dst, x, y);
    }
    free(x);
    free(y);
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
