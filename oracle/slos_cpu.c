/*
 * CPU SLOS recursion (TEST INFRASTRUCTURE: a timed CPU baseline, not a
 * parity reference).  Only tests/ and bench.py's CPU-baseline leg use it; it
 * shares no code with the CUDA library.  Its results are pinned against the
 * Ryser oracle (oracle.c) in tests/test_cpu_slos.py.
 *
 * What it computes (Sec. II-A.2/II-A.3, strong simulation photon by photon):
 * with the input photons in mode order c_1 <= ... <= c_n and a_0 = 1,
 *     a_k(t) = sum_{j : t_j > 0} U[j][c_k] a_{k-1}(t - e_j),   k = 1..n,
 *     p(t)   = |a_n(t)|^2 prod_j t_j! / prod_i s_i!
 * and, for L = sum_t g(t) p(t) with a given g (shared by the batch), the
 * reverse recursion in PyTorch's convention dZ = dL/dRe Z + i dL/dIm Z:
 *     G_n(t)       = 2 g(t) w(t) a_n(t)
 *     dU[j][c_k]  += conj(a_{k-1}(t - e_j)) G_k(t)
 *     G_{k-1}(t-e_j) += conj(U[j][c_k]) G_k(t)
 * Every layer is kept (no checkpointing).  FP64 throughout; OpenMP over the
 * instances of a batch, each instance walked sequentially.
 *
 * Fock states of k photons are listed in descending lexicographic order; the
 * position of t is  sum_{b=0}^{m-2} C(k+m-2-b-(t_0+...+t_b), m-1-b)
 * (the colex rank of its stars-and-bars string).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cx;

static int64_t choose(int a, int b) {
    if (b < 0 || a < 0 || b > a) return 0;
    int64_t r = 1;
    for (int i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r;
}

static int64_t ctab[128][64]; /* C(a, e), filled once */
static int ctab_ready = 0;

static void fill_ctab(void) {
    if (ctab_ready) return;
    for (int a = 0; a < 128; ++a)
        for (int e = 0; e < 64; ++e) ctab[a][e] = (e <= a) ? choose(a, e) : 0;
    ctab_ready = 1;
}

static int64_t position(const int *t, int m, int k) {
    int64_t r = 0;
    int cum = 0;
    for (int b = 0; b + 1 < m; ++b) {
        cum += t[b];
        const int a = k + m - 2 - b - cum, e = m - 1 - b;
        /* C(a, e) for a < e is 0; small arguments come from the table */
        if (a >= e) r += (a < 128 && e < 64) ? ctab[a][e] : choose(a, e);
    }
    return r;
}

/* next state in descending-lex order; returns 0 after the last one */
static int next_state(int *t, int m) {
    int i = m - 2;
    while (i >= 0 && t[i] == 0) --i;
    if (i < 0) return 0;
    int tail = 0;
    for (int q = i + 1; q < m; ++q) {
        tail += t[q];
        t[q] = 0;
    }
    t[i] -= 1;
    t[i + 1] = tail + 1;
    return 1;
}

/* Number of output states C(m+n-1, n). */
int64_t slos_cpu_dim(int m, int n) { return choose(m + n - 1, n); }

/* A plan: the input state and the transition tables of every layer, built
 * once and reused by every training pass (Sec. II-A.3). */
typedef struct {
    int m, n;
    int cols[64];
    int64_t F[65], off[66];
    int32_t *par[65]; /* par[k][c*m + j] = position of t - e_j in layer k-1, or -1 */
    double *w;        /* final layer: prod t_j! / prod s_i! */
} slos_cpu_plan;

void slos_cpu_plan_destroy(slos_cpu_plan *p) {
    if (!p) return;
    for (int k = 0; k <= p->n; ++k) free(p->par[k]);
    free(p->w);
    free(p);
}

slos_cpu_plan *slos_cpu_plan_create(int m, int n, const int *s) {
    if (m < 1 || m > 64 || n < 1 || n > 64) return NULL;
    fill_ctab();
    slos_cpu_plan *p = (slos_cpu_plan *)calloc(1, sizeof(slos_cpu_plan));
    if (!p) return NULL;
    p->m = m;
    p->n = n;
    int q = 0;
    double sfact = 1.0;
    for (int i = 0; i < m; ++i)
        for (int r = 0; r < s[i]; ++r) {
            if (q < 64) p->cols[q] = i;
            ++q;
            sfact *= (double)(r + 1);
        }
    if (q != n) {
        free(p);
        return NULL;
    }
    p->off[0] = 0;
    for (int k = 0; k <= n; ++k) {
        p->F[k] = choose(m + k - 1, k);
        p->off[k + 1] = p->off[k] + p->F[k];
    }
    p->w = (double *)malloc((size_t)p->F[n] * sizeof(double));
    if (!p->w) {
        slos_cpu_plan_destroy(p);
        return NULL;
    }
    int t[64];
    for (int k = 1; k <= n; ++k) {
        p->par[k] = (int32_t *)malloc((size_t)p->F[k] * m * sizeof(int32_t));
        if (!p->par[k]) {
            slos_cpu_plan_destroy(p);
            return NULL;
        }
        memset(t, 0, sizeof(t));
        t[0] = k;
        int64_t c = 0;
        do {
            /* parent t - e_j, ranked among the states of k - 1 photons */
            for (int j = 0; j < m; ++j) {
                if (t[j] > 0) {
                    t[j] -= 1;
                    p->par[k][c * m + j] = (int32_t)position(t, m, k - 1);
                    t[j] += 1;
                } else {
                    p->par[k][c * m + j] = -1;
                }
            }
            if (k == n) {
                double f = 1.0;
                for (int j = 0; j < m; ++j)
                    for (int r = 2; r <= t[j]; ++r) f *= (double)r;
                p->w[c] = f / sfact;
            }
            ++c;
        } while (next_state(t, m));
    }
    return p;
}

/*
 * Training pass for a batch: probabilities and dL/dU of L = sum_t g(t) p(t).
 *   B           instances; U: [B][m][m] complex (interleaved), U[b][j][i] = U_ji
 *   g           [K] doubles (shared by the batch), may be NULL (no backward)
 *   probs       [B][K] doubles out;  dU: [B][m][m] complex out (if g != NULL)
 * Returns 0, or -1 when memory runs out.
 */
int slos_cpu_plan_train(const slos_cpu_plan *P, int B, const double *U, const double *g, double *probs, double *dU,
                        int nthreads) {
    const int m = P->m, n = P->n;
    const int *cols = P->cols;
    const int64_t *F = P->F, *off = P->off;
    int32_t *const *par = P->par;
    const double *w = P->w;
    int fail = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        cx *a = (cx *)malloc((size_t)off[n + 1] * sizeof(cx));
        cx *G = (cx *)malloc((size_t)F[n] * sizeof(cx));
        cx *Gp = (cx *)malloc((size_t)F[n] * sizeof(cx));
        if (!a || !G || !Gp) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            fail = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int b = 0; b < B; ++b) {
            if (!a || !G || !Gp) continue;
            const cx *Ub = (const cx *)(U + (size_t)b * m * m * 2);
            a[0].re = 1.0;
            a[0].im = 0.0;
            for (int k = 1; k <= n; ++k) {
                const int col = cols[k - 1];
                const cx *prev = a + off[k - 1];
                cx *cur = a + off[k];
                for (int64_t c = 0; c < F[k]; ++c) {
                    double re = 0.0, im = 0.0;
                    const int32_t *pc = par[k] + c * m;
                    for (int j = 0; j < m; ++j) {
                        const int32_t p = pc[j];
                        if (p < 0) continue;
                        const cx x = Ub[j * m + col], y = prev[p];
                        re += x.re * y.re - x.im * y.im;
                        im += x.re * y.im + x.im * y.re;
                    }
                    cur[c].re = re;
                    cur[c].im = im;
                }
            }
            const cx *an = a + off[n];
            double *pb = probs + (size_t)b * F[n];
            for (int64_t c = 0; c < F[n]; ++c) pb[c] = w[c] * (an[c].re * an[c].re + an[c].im * an[c].im);
            if (!g) continue;
            cx *dUb = (cx *)(dU + (size_t)b * m * m * 2);
            memset(dUb, 0, sizeof(cx) * m * m);
            for (int64_t c = 0; c < F[n]; ++c) {
                const double sc = 2.0 * g[c] * w[c];
                G[c].re = sc * an[c].re;
                G[c].im = sc * an[c].im;
            }
            for (int k = n; k >= 1; --k) {
                const int col = cols[k - 1];
                const cx *prev = a + off[k - 1];
                memset(Gp, 0, sizeof(cx) * (size_t)F[k - 1]);
                for (int64_t c = 0; c < F[k]; ++c) {
                    const cx gk = G[c];
                    const int32_t *pc = par[k] + c * m;
                    for (int j = 0; j < m; ++j) {
                        const int32_t p = pc[j];
                        if (p < 0) continue;
                        const cx x = Ub[j * m + col], y = prev[p];
                        /* dU += conj(a_{k-1}) G_k ; G_{k-1} += conj(U) G_k */
                        dUb[j * m + col].re += y.re * gk.re + y.im * gk.im;
                        dUb[j * m + col].im += y.re * gk.im - y.im * gk.re;
                        Gp[p].re += x.re * gk.re + x.im * gk.im;
                        Gp[p].im += x.re * gk.im - x.im * gk.re;
                    }
                }
                cx *tmp = G;
                G = Gp;
                Gp = tmp;
            }
        }
        free(a);
        free(G);
        free(Gp);
    }
    return fail ? -1 : 0;
}

/* One-shot convenience: plan, train, destroy. */
int slos_cpu_train(int m, int n, const int *s, int B, const double *U, const double *g, double *probs, double *dU,
                   int nthreads) {
    slos_cpu_plan *p = slos_cpu_plan_create(m, n, s);
    if (!p) return -1;
    const int rc = slos_cpu_plan_train(p, B, U, g, probs, dU, nthreads);
    slos_cpu_plan_destroy(p);
    return rc;
}
