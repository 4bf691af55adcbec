/*
 * FP64 direct-measurement polyspectrum oracle (plain C, OpenMP over m1).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code with the CUDA library.
 *
 * What it computes (Eq. bi_direct of the paper, over full spherical shells):
 *
 *   num[a][b][c] = sum over ordered (m1, m2, m3) with m1 in S_a, m2 in S_b,
 *                  m3 in S_c and m1 + m2 + m3 = 0 (mod N) of
 *                  Re[ D(m1) D(m2) D(m3) ]
 *   cnt[a][b][c] = number of such ordered triples (the triangle count
 *                  N_tri, the denominator of Eq. gen_Nspec3)
 *
 * where D is the unnormalised forward DFT of the real field (Eq.
 * DeltaFFTtoDelta).  Every component of m is reduced into [-N/2, N/2), the
 * frequency a length-N DFT resolves, and "m1+m2+m3 = 0 (mod N)" is the
 * discrete Kronecker delta of Sec. 2 (closure modulo the grid).
 *
 * Shell membership (the scalar reading of the bin-width rule of Eq.
 * gen_Nspec3): mode m belongs to bin b iff thr[b] <= |m|^2 < thr[b+1],
 * where thr[] are integer thresholds on |m|^2 supplied by the caller.
 *
 * The trispectrum routine is the p = 4 case of Eq. gen_Nspec3 (ordered
 * quadruples with m1+m2+m3+m4 = 0 mod N); it is O(|M|^3) and meant for tiny
 * grids only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int mx, my, mz; /* components in [-N/2, N/2) */
    int bin;
    int64_t idx;    /* flat index into the full N^3 spectrum (FFT order) */
} mode_t_;

/* Wrap an integer into [-N/2, N/2). */
static int wrap(int v, int N) {
    int r = v % N;
    if (r < 0) r += N;
    if (r >= N / 2 + (N & 1)) r -= N;
    return r;
}

/* Bin of an integer |m|^2, or -1 when it lies in no bin. */
static int bin_of(int64_t m2, int nbins, const int64_t *thr) {
    if (m2 < thr[0] || m2 >= thr[nbins]) return -1;
    /* thresholds are non-decreasing; find the b with thr[b] <= m2 < thr[b+1] */
    int lo = 0, hi = nbins - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (thr[mid] <= m2) lo = mid; else hi = mid - 1;
    }
    return (thr[lo] <= m2 && m2 < thr[lo + 1]) ? lo : -1;
}

static int64_t flat(int mx, int my, int mz, int N) {
    int ix = mx < 0 ? mx + N : mx;
    int iy = my < 0 ? my + N : my;
    int iz = mz < 0 ? mz + N : mz;
    return ((int64_t)ix * N + iy) * N + iz;
}

/* Enumerate the binned modes.  Returns the count; *out is malloc'd. */
static int64_t collect_modes(int N, int nbins, const int64_t *thr, mode_t_ **out) {
    int64_t cap = 1024, n = 0;
    mode_t_ *m = (mode_t_ *)malloc((size_t)cap * sizeof(mode_t_));
    int lo = -(N / 2), hi = N - N / 2; /* [-N/2, N/2) for even N */
    for (int x = lo; x < hi; ++x)
        for (int y = lo; y < hi; ++y)
            for (int z = lo; z < hi; ++z) {
                int64_t m2 = (int64_t)x * x + (int64_t)y * y + (int64_t)z * z;
                int b = bin_of(m2, nbins, thr);
                if (b < 0) continue;
                if (n == cap) {
                    cap *= 2;
                    m = (mode_t_ *)realloc(m, (size_t)cap * sizeof(mode_t_));
                }
                m[n].mx = x; m[n].my = y; m[n].mz = z; m[n].bin = b;
                m[n].idx = flat(x, y, z, N);
                ++n;
            }
    *out = m;
    return n;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Number of binned modes (|M|). */
int64_t oracle_count_modes(int N, int nbins, const int64_t *thr) {
    mode_t_ *m = NULL;
    int64_t n = collect_modes(N, nbins, thr, &m);
    free(m);
    return n;
}

/*
 * All-pairs direct bispectrum over ordered bin triples.
 *   re, im : full N^3 spectrum, C order [mx][my][mz] in FFT index order.
 *   num, num_im : nbins^3 doubles (ordered a, b, c), zeroed here.
 *   cnt    : nbins^3 int64 triangle counts, zeroed here.
 *   m1_start, m1_stride : process only m1 indices i with i % m1_stride ==
 *            m1_start (a bounded, unbiased sample for timing); pass 0, 1 for
 *            the full sum.
 * Returns the number of m1 modes processed.
 */
int64_t oracle_direct_bispectrum(int N, const double *re, const double *im, int nbins,
                                 const int64_t *thr, double *num, double *num_im,
                                 int64_t *cnt, int64_t m1_start, int64_t m1_stride) {
    mode_t_ *M = NULL;
    int64_t nm = collect_modes(N, nbins, thr, &M);
    const int64_t nb3 = (int64_t)nbins * nbins * nbins;
    memset(num, 0, (size_t)nb3 * sizeof(double));
    memset(num_im, 0, (size_t)nb3 * sizeof(double));
    memset(cnt, 0, (size_t)nb3 * sizeof(int64_t));
    /* bin lookup for every |m|^2 a wrapped mode can take */
    int64_t maxm2 = 3LL * (N / 2) * (N / 2) + 1;
    int *binsq = (int *)malloc((size_t)(maxm2 + 1) * sizeof(int));
    for (int64_t s = 0; s <= maxm2; ++s) binsq[s] = bin_of(s, nbins, thr);
    int64_t processed = 0;
    if (m1_stride < 1) m1_stride = 1;

#pragma omp parallel
    {
        double *ln = (double *)calloc((size_t)nb3, sizeof(double));
        double *li = (double *)calloc((size_t)nb3, sizeof(double));
        int64_t *lc = (int64_t *)calloc((size_t)nb3, sizeof(int64_t));
        int64_t myproc = 0;
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < nm; ++i) {
            if (i % m1_stride != m1_start) continue;
            ++myproc;
            const mode_t_ a = M[i];
            const double ar = re[a.idx], ai = im[a.idx];
            for (int64_t j = 0; j < nm; ++j) {
                const mode_t_ b = M[j];
                int x = wrap(-(a.mx + b.mx), N);
                int y = wrap(-(a.my + b.my), N);
                int z = wrap(-(a.mz + b.mz), N);
                int64_t m2 = (int64_t)x * x + (int64_t)y * y + (int64_t)z * z;
                int c = binsq[m2];
                if (c < 0) continue;
                int64_t k3 = flat(x, y, z, N);
                /* D1 D2 */
                double br = re[b.idx], bi = im[b.idx];
                double pr = ar * br - ai * bi;
                double pi = ar * bi + ai * br;
                /* (D1 D2) D3 */
                double cr = re[k3], ci = im[k3];
                int64_t o = ((int64_t)a.bin * nbins + b.bin) * nbins + c;
                ln[o] += pr * cr - pi * ci;
                li[o] += pr * ci + pi * cr;
                lc[o] += 1;
            }
        }
#pragma omp critical
        {
            for (int64_t o = 0; o < nb3; ++o) {
                num[o] += ln[o];
                num_im[o] += li[o];
                cnt[o] += lc[o];
            }
            processed += myproc;
        }
        free(ln); free(li); free(lc);
    }
    free(binsq);
    free(M);
    return processed;
}

/*
 * Direct sums for a list of requested (a, b, c) bin triples only: for each
 * triple, loop m1 in S_a and m2 in S_b and keep m3 = -(m1+m2) (mod N) when it
 * lies in S_c.  Cost sum_t |S_a||S_b|.
 *   abc : 3*ntrip bin indices; num, num_im, cnt : ntrip outputs.
 */
void oracle_direct_triplets(int N, const double *re, const double *im, int nbins,
                            const int64_t *thr, int ntrip, const int32_t *abc,
                            double *num, double *num_im, int64_t *cnt) {
    mode_t_ *M = NULL;
    int64_t nm = collect_modes(N, nbins, thr, &M);
    /* per-bin mode lists */
    int64_t *start = (int64_t *)calloc((size_t)nbins + 1, sizeof(int64_t));
    for (int64_t i = 0; i < nm; ++i) start[M[i].bin + 1]++;
    for (int b = 0; b < nbins; ++b) start[b + 1] += start[b];
    int64_t *fill = (int64_t *)malloc((size_t)nbins * sizeof(int64_t));
    memcpy(fill, start, (size_t)nbins * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)(nm ? nm : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < nm; ++i) order[fill[M[i].bin]++] = i;

    for (int t = 0; t < ntrip; ++t) {
        int A = abc[3 * t], B = abc[3 * t + 1], C = abc[3 * t + 2];
        double sr = 0.0, si = 0.0;
        int64_t sc = 0;
        if (A < 0 || B < 0 || C < 0 || A >= nbins || B >= nbins || C >= nbins) {
            num[t] = 0.0; num_im[t] = 0.0; cnt[t] = 0;
            continue;
        }
#pragma omp parallel for reduction(+ : sr, si, sc) schedule(dynamic, 16)
        for (int64_t p = start[A]; p < start[A + 1]; ++p) {
            const mode_t_ a = M[order[p]];
            const double ar = re[a.idx], ai = im[a.idx];
            for (int64_t q = start[B]; q < start[B + 1]; ++q) {
                const mode_t_ b = M[order[q]];
                int x = wrap(-(a.mx + b.mx), N);
                int y = wrap(-(a.my + b.my), N);
                int z = wrap(-(a.mz + b.mz), N);
                int64_t m2 = (int64_t)x * x + (int64_t)y * y + (int64_t)z * z;
                if (bin_of(m2, nbins, thr) != C) continue;
                int64_t k3 = flat(x, y, z, N);
                double br = re[b.idx], bi = im[b.idx];
                double pr = ar * br - ai * bi;
                double pi = ar * bi + ai * br;
                double cr = re[k3], ci = im[k3];
                sr += pr * cr - pi * ci;
                si += pr * ci + pi * cr;
                sc += 1;
            }
        }
        num[t] = sr; num_im[t] = si; cnt[t] = sc;
    }
    free(order); free(fill); free(start); free(M);
}

/* m1 + m2 = 0 (mod N) in every component. */
static int opposite(const mode_t_ *a, const mode_t_ *b, int N) {
    return wrap(a->mx + b->mx, N) == 0 && wrap(a->my + b->my, N) == 0 && wrap(a->mz + b->mz, N) == 0;
}

/*
 * All-triples direct trispectrum over ordered bin quadruples (tiny grids):
 * m4 = -(m1+m2+m3) (mod N).  num, num_im, cnt have nbins^4 entries.
 * connected != 0: leave out every quadruple in which some pair of modes sums
 * to zero (m1+m2, m1+m3 or m2+m3 = 0 mod N; with the closure these are all
 * three pairings).  Those are the only terms a Gaussian field's expectation
 * keeps (Wick pairings, the P x P parts); what remains is the connected part.
 */
void oracle_direct_trispectrum(int N, const double *re, const double *im, int nbins,
                               const int64_t *thr, double *num, double *num_im,
                               int64_t *cnt, int connected) {
    mode_t_ *M = NULL;
    int64_t nm = collect_modes(N, nbins, thr, &M);
    const int64_t nb4 = (int64_t)nbins * nbins * nbins * nbins;
    memset(num, 0, (size_t)nb4 * sizeof(double));
    memset(num_im, 0, (size_t)nb4 * sizeof(double));
    memset(cnt, 0, (size_t)nb4 * sizeof(int64_t));
#pragma omp parallel
    {
        double *ln = (double *)calloc((size_t)nb4, sizeof(double));
        double *li = (double *)calloc((size_t)nb4, sizeof(double));
        int64_t *lc = (int64_t *)calloc((size_t)nb4, sizeof(int64_t));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < nm; ++i) {
            const mode_t_ a = M[i];
            for (int64_t j = 0; j < nm; ++j) {
                const mode_t_ b = M[j];
                double pr = re[a.idx] * re[b.idx] - im[a.idx] * im[b.idx];
                double pi = re[a.idx] * im[b.idx] + im[a.idx] * re[b.idx];
                const int ab = connected && opposite(&a, &b, N);
                for (int64_t k = 0; k < nm; ++k) {
                    const mode_t_ c = M[k];
                    if (connected && (ab || opposite(&a, &c, N) || opposite(&b, &c, N))) continue;
                    int x = wrap(-(a.mx + b.mx + c.mx), N);
                    int y = wrap(-(a.my + b.my + c.my), N);
                    int z = wrap(-(a.mz + b.mz + c.mz), N);
                    int64_t m2 = (int64_t)x * x + (int64_t)y * y + (int64_t)z * z;
                    int d = bin_of(m2, nbins, thr);
                    if (d < 0) continue;
                    int64_t k4 = flat(x, y, z, N);
                    double qr = pr * re[c.idx] - pi * im[c.idx];
                    double qi = pr * im[c.idx] + pi * re[c.idx];
                    int64_t o = (((int64_t)a.bin * nbins + b.bin) * nbins + c.bin) * nbins + d;
                    ln[o] += qr * re[k4] - qi * im[k4];
                    li[o] += qr * im[k4] + qi * re[k4];
                    lc[o] += 1;
                }
            }
        }
#pragma omp critical
        {
            for (int64_t o = 0; o < nb4; ++o) {
                num[o] += ln[o];
                num_im[o] += li[o];
                cnt[o] += lc[o];
            }
        }
        free(ln); free(li); free(lc);
    }
    free(M);
}

/*
 * Diagonal-resolved trispectrum sums (ordered quadruples, tiny grids): as
 * oracle_direct_trispectrum, and the quadruple also goes by the bin D of its
 * diagonal q = m1 + m2 (wrapped into [-N/2, N/2) per component), dthr[ndiag+1]
 * integer thresholds on |q|^2; quadruples whose |q|^2 is in no diagonal bin
 * are left out.  Arrays [a][b][c][d][D].
 */
void oracle_direct_trispectrum_diag(int N, const double *re, const double *im, int nbins,
                                    const int64_t *thr, int ndiag, const int64_t *dthr, double *num,
                                    double *num_im, int64_t *cnt) {
    mode_t_ *M = NULL;
    int64_t nm = collect_modes(N, nbins, thr, &M);
    const int64_t n5 = (int64_t)nbins * nbins * nbins * nbins * ndiag;
    memset(num, 0, (size_t)n5 * sizeof(double));
    memset(num_im, 0, (size_t)n5 * sizeof(double));
    memset(cnt, 0, (size_t)n5 * sizeof(int64_t));
#pragma omp parallel
    {
        double *ln = (double *)calloc((size_t)n5, sizeof(double));
        double *li = (double *)calloc((size_t)n5, sizeof(double));
        int64_t *lc = (int64_t *)calloc((size_t)n5, sizeof(int64_t));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < nm; ++i) {
            const mode_t_ a = M[i];
            for (int64_t j = 0; j < nm; ++j) {
                const mode_t_ b = M[j];
                const int qx = wrap(a.mx + b.mx, N), qy = wrap(a.my + b.my, N), qz = wrap(a.mz + b.mz, N);
                const int D = bin_of((int64_t)qx * qx + (int64_t)qy * qy + (int64_t)qz * qz, ndiag, dthr);
                if (D < 0) continue;
                double pr = re[a.idx] * re[b.idx] - im[a.idx] * im[b.idx];
                double pi = re[a.idx] * im[b.idx] + im[a.idx] * re[b.idx];
                for (int64_t k = 0; k < nm; ++k) {
                    const mode_t_ c = M[k];
                    int x = wrap(-(a.mx + b.mx + c.mx), N);
                    int y = wrap(-(a.my + b.my + c.my), N);
                    int z = wrap(-(a.mz + b.mz + c.mz), N);
                    int64_t m2 = (int64_t)x * x + (int64_t)y * y + (int64_t)z * z;
                    int d = bin_of(m2, nbins, thr);
                    if (d < 0) continue;
                    int64_t k4 = flat(x, y, z, N);
                    double qr = pr * re[c.idx] - pi * im[c.idx];
                    double qi = pr * im[c.idx] + pi * re[c.idx];
                    int64_t o = ((((int64_t)a.bin * nbins + b.bin) * nbins + c.bin) * nbins + d) * ndiag + D;
                    ln[o] += qr * re[k4] - qi * im[k4];
                    li[o] += qr * im[k4] + qi * re[k4];
                    lc[o] += 1;
                }
            }
        }
#pragma omp critical
        {
            for (int64_t o = 0; o < n5; ++o) {
                num[o] += ln[o];
                num_im[o] += li[o];
                cnt[o] += lc[o];
            }
        }
        free(ln); free(li); free(lc);
    }
    free(M);
}

/*
 * Closure of bin triples (a, b, c): flag[t] = 1 when some ordered triple
 * m1 in S_a, m2 in S_b, m3 = -(m1+m2) (mod N) in S_c exists, i.e. when
 * N_tri > 0.  A witness search that stops at the first closed triple; the
 * caller may skip triples the triangle inequality already rules out.
 * Modes of each shell are visited from the largest |m| down, where closing
 * triangles of wide bin triples are found first.
 */
static int cmp_desc_m2(const void *x, const void *y) {
    const mode_t_ *a = (const mode_t_ *)x, *b = (const mode_t_ *)y;
    long long sa = (long long)a->mx * a->mx + (long long)a->my * a->my + (long long)a->mz * a->mz;
    long long sb = (long long)b->mx * b->mx + (long long)b->my * b->my + (long long)b->mz * b->mz;
    if (a->bin != b->bin) return a->bin - b->bin;
    return (sa < sb) - (sa > sb);
}

void oracle_closed_triplets(int N, int nbins, const int64_t *thr, int ntrip, const int32_t *abc,
                            int32_t *flag) {
    mode_t_ *M = NULL;
    int64_t nm = collect_modes(N, nbins, thr, &M);
    qsort(M, (size_t)nm, sizeof(mode_t_), cmp_desc_m2);
    int64_t *start = (int64_t *)calloc((size_t)nbins + 1, sizeof(int64_t));
    for (int64_t i = 0; i < nm; ++i) start[M[i].bin + 1]++;
    for (int b = 0; b < nbins; ++b) start[b + 1] += start[b];
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < ntrip; ++t) {
        int A = abc[3 * t], B = abc[3 * t + 1], C = abc[3 * t + 2];
        int found = 0;
        for (int64_t p = start[A]; p < start[A + 1] && !found; ++p) {
            const mode_t_ a = M[p];
            for (int64_t q = start[B]; q < start[B + 1]; ++q) {
                const mode_t_ b = M[q];
                int x = wrap(-(a.mx + b.mx), N);
                int y = wrap(-(a.my + b.my), N);
                int z = wrap(-(a.mz + b.mz), N);
                int64_t m2 = (int64_t)x * x + (int64_t)y * y + (int64_t)z * z;
                if (m2 >= thr[C] && m2 < thr[C + 1]) {
                    found = 1;
                    break;
                }
            }
        }
        flag[t] = found;
    }
    free(start);
    free(M);
}

/*
 * Separable models summed over each requested triplet's closed triangles:
 * for (a, b, c) = abc[3t..], out[t] = sum over ordered (m1, m2, m3) with
 * m1 in S_a, m2 in S_b, m3 = -(m1+m2) (mod N) in S_c of
 *   sum_k coef[k] w[terms[3k]][|m1|^2] w[terms[3k+1]][|m2|^2] w[terms[3k+2]][|m3|^2]
 * and cnt[t] the number of those triangles (the theory averaged over the
 * exact triangle set of a bin, as the paper's theory points are).
 *   w : nfunc tables of nw values at integer |m|^2.
 */
void oracle_triangle_sums(int N, int nbins, const int64_t *thr, int ntrip, const int32_t *abc, int nfunc,
                          int64_t nw, const double *w, int nterms, const int32_t *terms, const double *coef,
                          double *out, int64_t *cnt) {
    mode_t_ *M = NULL;
    int64_t nm = collect_modes(N, nbins, thr, &M);
    int64_t *start = (int64_t *)calloc((size_t)nbins + 1, sizeof(int64_t));
    for (int64_t i = 0; i < nm; ++i) start[M[i].bin + 1]++;
    for (int b = 0; b < nbins; ++b) start[b + 1] += start[b];
    int64_t *fill = (int64_t *)malloc((size_t)nbins * sizeof(int64_t));
    memcpy(fill, start, (size_t)nbins * sizeof(int64_t));
    int64_t *order = (int64_t *)malloc((size_t)(nm ? nm : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < nm; ++i) order[fill[M[i].bin]++] = i;
    (void)nfunc;
    for (int t = 0; t < ntrip; ++t) {
        int A = abc[3 * t], B = abc[3 * t + 1], C = abc[3 * t + 2];
        double s = 0.0;
        int64_t sc = 0;
#pragma omp parallel for reduction(+ : s, sc) schedule(dynamic, 16)
        for (int64_t p = start[A]; p < start[A + 1]; ++p) {
            const mode_t_ a = M[order[p]];
            const int64_t s1 = (int64_t)a.mx * a.mx + (int64_t)a.my * a.my + (int64_t)a.mz * a.mz;
            for (int64_t q = start[B]; q < start[B + 1]; ++q) {
                const mode_t_ b = M[order[q]];
                int x = wrap(-(a.mx + b.mx), N);
                int y = wrap(-(a.my + b.my), N);
                int z = wrap(-(a.mz + b.mz), N);
                int64_t s3 = (int64_t)x * x + (int64_t)y * y + (int64_t)z * z;
                if (bin_of(s3, nbins, thr) != C) continue;
                const int64_t s2 = (int64_t)b.mx * b.mx + (int64_t)b.my * b.my + (int64_t)b.mz * b.mz;
                double v = 0.0;
                for (int k = 0; k < nterms; ++k)
                    v += coef[k] * w[(int64_t)terms[3 * k] * nw + s1] * w[(int64_t)terms[3 * k + 1] * nw + s2] *
                         w[(int64_t)terms[3 * k + 2] * nw + s3];
                s += v;
                sc += 1;
            }
        }
        out[t] = s;
        cnt[t] = sc;
    }
    free(order); free(fill); free(start); free(M);
}
