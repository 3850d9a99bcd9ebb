/*
 * FP64 reference transforms for the batched 1D complex-to-complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark use this file; the CUDA library never
 * links, includes or calls it, and it shares no code with the CUDA path.
 *
 * What is computed (the definition the paper's Eq. 1 factorises):
 *     X_k = sum_{j<n} x_j * exp(s * 2*pi*i * j*k / n),   s = -1 forward, +1 inverse,
 * unnormalised in both directions.
 *
 * Two independent routines:
 *   oracle_dft        the O(n^2) sum written out; the angle uses the exact integer
 *                     (j*k) mod n and the sum is compensated (Neumaier), so the only
 *                     rounding is that of cos/sin and of the final sum.
 *   oracle_fft_r2     recursive radix-2 decimation in time (Eq. 1 with K = 2 applied
 *                     recursively); each twiddle is cos/sin(2*pi*k/n) called
 *                     directly, never obtained by recurrence.
 *   oracle_fft_mixed  recursive decimation in time by the smallest prime factor p of n
 *                     (Eq. 1 with K = p, any n >= 1); a prime length is summed directly.
 *                     Every twiddle angle is reduced exactly in integers and read from
 *                     one table of cos/sin(2*pi*m/n).
 * Both take and return interleaved doubles: x[b][j][0] = Re, x[b][j][1] = Im.
 * Batches are split across POSIX threads (one transform per task).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------ */
/* direct O(n^2) DFT                                                   */
/* ------------------------------------------------------------------ */

/* Neumaier compensated accumulation of one real component. */
typedef struct {
    double sum, comp;
} acc_t;

static inline void acc_add(acc_t *a, double v) {
    double t = a->sum + v;
    if (fabs(a->sum) >= fabs(v))
        a->comp += (a->sum - t) + v;
    else
        a->comp += (v - t) + a->sum;
    a->sum = t;
}

/* table[m] = (cos(2*pi*m/n), sin(2*pi*m/n)) for m < n */
static double *unit_circle_table(int64_t n) {
    double *t = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!t) return NULL;
    for (int64_t m = 0; m < n; ++m) {
        double ang = ORACLE_TWO_PI * ((double)m / (double)n);
        t[2 * m] = cos(ang);
        t[2 * m + 1] = sin(ang);
    }
    return t;
}

static void dft_one(int64_t n, int sign, const double *x, double *X, const double *tab) {
    for (int64_t k = 0; k < n; ++k) {
        acc_t re = {0.0, 0.0}, im = {0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            int64_t m = (int64_t)(((__int128)j * k) % n); /* exact angle reduction */
            double c = tab[2 * m], s = sign * tab[2 * m + 1];
            double xr = x[2 * j], xi = x[2 * j + 1];
            /* (xr + i xi)(c + i s) */
            acc_add(&re, xr * c);
            acc_add(&re, -xi * s);
            acc_add(&im, xr * s);
            acc_add(&im, xi * c);
        }
        X[2 * k] = re.sum + re.comp;
        X[2 * k + 1] = im.sum + im.comp;
    }
}

/* ------------------------------------------------------------------ */
/* recursive radix-2 decimation in time                                */
/* ------------------------------------------------------------------ */

/*
 * out[0..n) <- DFT_n of the subsequence x[0], x[stride], x[2*stride], ...
 * Split into the even- and odd-indexed halves (the stride permutation with
 * K = 2), transform each half recursively, then combine with the twiddle
 * diagonal: X_k = E_k + w^k O_k, X_{k+n/2} = E_k - w^k O_k, w = exp(s*2*pi*i/n).
 * tab holds cos/sin(2*pi*m/ntop) for the top-level length ntop; at length n
 * the twiddle w^k is entry m = k*(ntop/n), i.e. the same angle 2*pi*k/n
 * (k/n and m/ntop are the same exactly representable fraction).
 */
static void r2_rec(int64_t n, int64_t ntop, int sign, const double *x, int64_t stride, double *out,
                   const double *tab) {
    if (n == 1) {
        out[0] = x[0];
        out[1] = x[1];
        return;
    }
    int64_t h = n / 2;
    r2_rec(h, ntop, sign, x, 2 * stride, out, tab);                  /* even samples */
    r2_rec(h, ntop, sign, x + 2 * stride, 2 * stride, out + 2 * h, tab); /* odd samples */
    int64_t step = ntop / n;
    for (int64_t k = 0; k < h; ++k) {
        double c = tab[2 * (k * step)], s = sign * tab[2 * (k * step) + 1];
        double er = out[2 * k], ei = out[2 * k + 1];
        double orr = out[2 * (k + h)], oi = out[2 * (k + h) + 1];
        double tr = orr * c - oi * s;
        double ti = orr * s + oi * c;
        out[2 * k] = er + tr;
        out[2 * k + 1] = ei + ti;
        out[2 * (k + h)] = er - tr;
        out[2 * (k + h) + 1] = ei - ti;
    }
}

/* ------------------------------------------------------------------ */
/* recursive mixed-radix decimation in time (smallest prime first)     */
/* ------------------------------------------------------------------ */

static int64_t smallest_prime_factor(int64_t n) {
    if (n % 2 == 0) return 2;
    for (int64_t f = 3; f * f <= n; f += 2)
        if (n % f == 0) return f;
    return n;
}

/*
 * out[0..n) <- DFT_n of x[0], x[stride], x[2*stride], ...
 * With p the smallest prime factor of n and m = n / p, the p decimated subsequences
 * x[r + p*j] (j < m) are transformed recursively into Y_r (the stride permutation and
 * I_p (x) DFT_m of Eq. 1), then
 *     X_k = sum_{r<p} w_n^{r*k} * Y_r[k mod m],   k < n,  w_n = exp(s*2*pi*i/n)
 * (the twiddle diagonal and DFT_p (x) I_m written as one sum). A prime n is summed
 * directly. tab holds cos/sin(2*pi*t/ntop) for t < ntop; the angle 2*pi*(r*k mod n)/n is
 * entry (r*k mod n) * (ntop/n), the same fraction in integers.
 */
static int mr_rec(int64_t n, int64_t ntop, int sign, const double *x, int64_t stride, double *out,
                  const double *tab) {
    if (n == 1) {
        out[0] = x[0];
        out[1] = x[1];
        return 0;
    }
    const int64_t p = smallest_prime_factor(n), m = n / p, step = ntop / n;
    double *y = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!y) return -3;
    if (p == n) { /* prime length: the sum over j itself */
        for (int64_t j = 0; j < n; ++j) {
            y[2 * j] = x[2 * j * stride];
            y[2 * j + 1] = x[2 * j * stride + 1];
        }
    } else {
        for (int64_t r = 0; r < p; ++r) {
            int rc = mr_rec(m, ntop, sign, x + 2 * r * stride, p * stride, y + 2 * r * m, tab);
            if (rc) {
                free(y);
                return rc;
            }
        }
    }
    /* prime n: Y_r is the single sample x_r (m = 1), so the same combination applies */
    for (int64_t k = 0; k < n; ++k) {
        acc_t re = {0.0, 0.0}, im = {0.0, 0.0};
        const int64_t km = k % m;
        for (int64_t r = 0; r < p; ++r) {
            const int64_t t = (int64_t)(((__int128)r * k) % n) * step;
            const double c = tab[2 * t], sn = sign * tab[2 * t + 1];
            const double yr = y[2 * (r * m + km)], yi = y[2 * (r * m + km) + 1];
            acc_add(&re, yr * c);
            acc_add(&re, -yi * sn);
            acc_add(&im, yr * sn);
            acc_add(&im, yi * c);
        }
        out[2 * k] = re.sum + re.comp;
        out[2 * k + 1] = im.sum + im.comp;
    }
    free(y);
    return 0;
}

/* cos/sin(2*pi*m/n) for m < n/2, each evaluated directly */
static double *half_circle_table(int64_t n) {
    int64_t h = n / 2 > 0 ? n / 2 : 1;
    double *t = (double *)malloc(sizeof(double) * 2 * (size_t)h);
    if (!t) return NULL;
    for (int64_t m = 0; m < h; ++m) {
        double ang = ORACLE_TWO_PI * ((double)m / (double)n);
        t[2 * m] = cos(ang);
        t[2 * m + 1] = sin(ang);
    }
    return t;
}

/* ------------------------------------------------------------------ */
/* batched drivers with a thread pool over transforms                  */
/* ------------------------------------------------------------------ */

typedef struct {
    int kind; /* 0 = direct DFT, 1 = radix-2, 2 = mixed radix */
    int64_t n, batch;
    int sign;
    const double *x;
    double *X;
    const double *tab;
    int64_t next;
    int err;
    pthread_mutex_t mu;
} job_t;

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t b = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (b >= J->batch) break;
        const double *x = J->x + 2 * J->n * b;
        double *X = J->X + 2 * J->n * b;
        if (J->kind == 0) {
            dft_one(J->n, J->sign, x, X, J->tab);
        } else if (J->kind == 1) {
            r2_rec(J->n, J->n, J->sign, x, 1, X, J->tab);
        } else if (mr_rec(J->n, J->n, J->sign, x, 1, X, J->tab) != 0) {
            pthread_mutex_lock(&J->mu);
            J->err = -3;
            pthread_mutex_unlock(&J->mu);
        }
    }
    return NULL;
}

static int run_batched(int kind, int64_t n, int64_t batch, int sign, const double *x, double *X,
                       int threads) {
    if (n < 1 || batch < 0 || (sign != 1 && sign != -1)) return -1;
    if (kind == 1 && (n & (n - 1)) != 0) return -2;
    if (batch == 0) return 0;
    double *tab = kind == 1 ? half_circle_table(n) : unit_circle_table(n);
    if (!tab) return -3;
    job_t J;
    J.kind = kind;
    J.n = n;
    J.batch = batch;
    J.sign = sign;
    J.x = x;
    J.X = X;
    J.tab = tab;
    J.next = 0;
    J.err = 0;
    pthread_mutex_init(&J.mu, NULL);
    if (threads < 1) threads = 1;
    if (threads > batch) threads = (int)batch;
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    int started = 0;
    for (int i = 1; tid && i < threads; ++i) {
        if (pthread_create(&tid[started], NULL, worker, &J) == 0) ++started;
    }
    worker(&J); /* the calling thread works too */
    for (int i = 0; i < started; ++i) pthread_join(tid[i], NULL);
    free(tid);
    pthread_mutex_destroy(&J.mu);
    free(tab);
    return J.err;
}

/* Direct O(n^2) DFT of `batch` transforms of length n (any n >= 1). Returns 0 on success. */
int oracle_dft(int64_t n, int64_t batch, int sign, const double *x, double *X, int threads) {
    return run_batched(0, n, batch, sign, x, X, threads);
}

/* Recursive radix-2 FFT of `batch` transforms of length n (a power of two). Returns 0 on success. */
int oracle_fft_r2(int64_t n, int64_t batch, int sign, const double *x, double *X, int threads) {
    return run_batched(1, n, batch, sign, x, X, threads);
}

/* Recursive mixed-radix FFT of `batch` transforms of length n (any n >= 1). Returns 0 on success. */
int oracle_fft_mixed(int64_t n, int64_t batch, int sign, const double *x, double *X, int threads) {
    return run_batched(2, n, batch, sign, x, X, threads);
}
