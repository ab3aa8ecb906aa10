/*
 * Oracle for the linear-optics output distribution (TEST INFRASTRUCTURE ONLY).
 *
 * Plain, slow, obviously-correct FP64 CPU code.  Nothing in the product path
 * (the CUDA library and its Python binding) may link, load or call this file;
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.
 * It shares no code with the CUDA path.
 *
 * What it computes (Sec. II-A.1 "Essentials of linear optics"): for an input
 * Fock state s over m modes holding n photons and an m x m unitary U, the
 * amplitude of output Fock state t is
 *        <t|U|s> = Per(U[rows(t), cols(s)]) / sqrt(prod_j t_j! * prod_i s_i!)
 * where rows(t) lists output mode j t_j times and cols(s) lists input mode i
 * s_i times.  The permanent is evaluated output by output with Ryser's
 * inclusion-exclusion formula, using a Gray-code walk over column subsets:
 *        Per(A) = (-1)^n * sum_{S subset [n]} (-1)^{|S|} prod_i sum_{j in S} A_ij
 * Output states are produced by brute-force enumeration in descending
 * lexicographic order (first (n,0,...,0), last (0,...,0,n)); an output's index
 * is its position in that walk.
 *
 * Complex numbers are interleaved (re, im) doubles.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cplx;

static inline cplx cadd(cplx a, cplx b) { cplx r = {a.re + b.re, a.im + b.im}; return r; }
static inline cplx csub(cplx a, cplx b) { cplx r = {a.re - b.re, a.im - b.im}; return r; }
static inline cplx cmul(cplx a, cplx b) {
    cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return r;
}

/* Ryser permanent of an n x n complex matrix (row-major, interleaved). */
static cplx ryser(int n, const cplx *A) {
    cplx total = {0.0, 0.0};
    if (n == 0) { cplx one = {1.0, 0.0}; return one; }
    cplx rowsum[64];
    for (int i = 0; i < n; ++i) { rowsum[i].re = 0.0; rowsum[i].im = 0.0; }
    /* Gray code: subset g(k) = k ^ (k >> 1); step k toggles bit ctz(k). */
    uint64_t prev = 0;
    for (uint64_t k = 1; k < ((uint64_t)1 << n); ++k) {
        uint64_t g = k ^ (k >> 1);
        uint64_t diff = g ^ prev;
        int j = __builtin_ctzll(diff);
        int added = (g & diff) != 0;
        for (int i = 0; i < n; ++i)
            rowsum[i] = added ? cadd(rowsum[i], A[i * n + j]) : csub(rowsum[i], A[i * n + j]);
        prev = g;
        cplx prod = rowsum[0];
        for (int i = 1; i < n; ++i) prod = cmul(prod, rowsum[i]);
        int size = __builtin_popcountll(g);
        if (size & 1) total = csub(total, prod);
        else total = cadd(total, prod);
    }
    if (n & 1) { total.re = -total.re; total.im = -total.im; }
    return total;
}

void oracle_permanent(int n, const double *A, double *out) {
    cplx p = ryser(n, (const cplx *)A);
    out[0] = p.re;
    out[1] = p.im;
}

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/* Build the n x n submatrix U[rows(t), cols(s)] for output t. */
static void submatrix(int m, int n, const cplx *U, const int *s, const int *t, cplx *A) {
    int cols[64], rows[64];
    int nc = 0, nr = 0;
    for (int i = 0; i < m; ++i) for (int c = 0; c < s[i]; ++c) cols[nc++] = i;
    for (int j = 0; j < m; ++j) for (int c = 0; c < t[j]; ++c) rows[nr++] = j;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) A[a * n + b] = U[rows[a] * m + cols[b]];
}

/*
 * amps[k] = Per(U[rows(t_k), cols(s)]) / sqrt(prod t! prod s!) for the K
 * output states given in `outputs` (K x m ints).  U is m x m row-major,
 * U[j*m + i] = U_{j,i} (input mode i -> output mode j).
 */
void oracle_amplitudes(int m, int n, const double *U, const int *s, int64_t K,
                       const int *outputs, double *amps, int nthreads) {
    double sfact = 1.0;
    for (int i = 0; i < m; ++i) sfact *= factorial(s[i]);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < K; ++k) {
        cplx A[64 * 64 / 4];
        const int *t = outputs + k * m;
        submatrix(m, n, (const cplx *)U, s, t, A);
        cplx per = ryser(n, A);
        double tfact = 1.0;
        for (int j = 0; j < m; ++j) tfact *= factorial(t[j]);
        double norm = 1.0 / sqrt(tfact * sfact);
        amps[2 * k] = per.re * norm;
        amps[2 * k + 1] = per.im * norm;
    }
}

/*
 * Analytic gradient of L = sum_k c_k p(t_k) with respect to U, through the
 * permanent's minors: dPer(A)/dA_ab = Per(A without row a and column b).
 * Returned in the PyTorch convention dU = dL/dRe U + i dL/dIm U = 2 dL/d(conj U):
 *   dU_{j,i} = sum_k 2 c_k / (prod t! prod s!) * Per_k * conj(sum_{a: rows_a=j}
 *              sum_{b: cols_b=i} Per(minor_ab))
 */
void oracle_grad_U(int m, int n, const double *U, const int *s, int64_t K,
                   const int *outputs, const double *c, double *dU, int nthreads) {
    double sfact = 1.0;
    for (int i = 0; i < m; ++i) sfact *= factorial(s[i]);
    int cols[64];
    int nc = 0;
    for (int i = 0; i < m; ++i) for (int q = 0; q < s[i]; ++q) cols[nc++] = i;
    int nt = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    nt = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nt * m * m * 2, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t k = 0; k < K; ++k) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *mine = acc + (size_t)tid * m * m * 2;
        const int *t = outputs + k * m;
        int rows[64];
        int nr = 0;
        for (int j = 0; j < m; ++j) for (int q = 0; q < t[j]; ++q) rows[nr++] = j;
        cplx A[64 * 64 / 4], minor[64 * 64 / 4];
        submatrix(m, n, (const cplx *)U, s, t, A);
        cplx per = ryser(n, A);
        double tfact = 1.0;
        for (int j = 0; j < m; ++j) tfact *= factorial(t[j]);
        double w = 2.0 * c[k] / (tfact * sfact);
        for (int a = 0; a < n; ++a) {
            for (int b = 0; b < n; ++b) {
                int r = 0;
                for (int aa = 0; aa < n; ++aa) {
                    if (aa == a) continue;
                    int q = 0;
                    for (int bb = 0; bb < n; ++bb) {
                        if (bb == b) continue;
                        minor[r * (n - 1) + q] = A[aa * n + bb];
                        ++q;
                    }
                    ++r;
                }
                cplx pm = ryser(n - 1, minor);
                /* contribution w * per * conj(pm) to dU[rows[a], cols[b]] */
                cplx cpm = {pm.re, -pm.im};
                cplx v = cmul(per, cpm);
                double *d = mine + ((size_t)rows[a] * m + cols[b]) * 2;
                d[0] += w * v.re;
                d[1] += w * v.im;
            }
        }
    }
    memset(dU, 0, sizeof(double) * m * m * 2);
    for (int tid = 0; tid < nt; ++tid)
        for (int e = 0; e < m * m * 2; ++e) dU[e] += acc[(size_t)tid * m * m * 2 + e];
    free(acc);
}

/*
 * Brute-force walk over all compositions t of n photons into m modes in
 * descending lexicographic order.  The walk is a plain odometer: the state
 * after (n,0,...,0) is obtained by moving one photon out of the rightmost
 * non-last nonzero mode into the next mode and sweeping everything behind it
 * into that mode.  Positions listed in `wanted` (sorted ascending, -1 to stop)
 * are copied to `out` (count x m bytes).  Returns the total number of states.
 */
int64_t oracle_enumerate(int m, int n, int64_t count, const int64_t *wanted, uint8_t *out) {
    int t[64];
    for (int j = 0; j < m; ++j) t[j] = 0;
    t[0] = n;
    int64_t pos = 0, w = 0;
    for (;;) {
        while (w < count && wanted[w] == pos) {
            for (int j = 0; j < m; ++j) out[w * m + j] = (uint8_t)t[j];
            ++w;
        }
        ++pos;
        /* next composition in descending lex order */
        int i = m - 2;
        while (i >= 0 && t[i] == 0) --i;
        if (i < 0) break; /* (0,...,0,n) was the last one */
        t[i] -= 1;
        int rest = t[m - 1];
        t[m - 1] = 0;
        t[i + 1] += rest + 1;
    }
    return pos;
}
