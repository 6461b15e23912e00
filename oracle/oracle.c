/*
 * oracle.c -- plain, untiled FP64 CPU evaluation of structured-mesh stencil loops.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library. It shares no code, header or constant with
 * the CUDA executor: it is the independent definition the executor is checked
 * against.
 *
 * What it computes (arXiv 1709.02125, Sec. 3): a parallel loop applies a kernel at
 * every point of an iteration range, reading datasets through stencils (relative
 * offsets) and writing datasets at the point itself; loops of a chain run one after
 * another in program order. Here every loop is evaluated over its whole range in
 * one sweep over full (untiled) arrays, the plain sequential meaning that the tiled
 * schedule of Sec. 3 / Sec. 4 must reproduce.
 *
 * Arrays are dense C-order arrays of the full extent including halos. A geometry is
 * six ints per array: extent e[0..2] (x, y, z; 1 for unused axes) and halo-low
 * h[0..2]; element (x, y, z) sits at ((z + h2) * e1 + (y + h1)) * e0 + (x + h0).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off (no FMA contraction, IEEE order).
 * Parallelism: the loop kernels split the (z, y) lines of the range over the threads
 * (both slow axes of a 3-D range, the y rows of a 2-D one); every point is computed
 * independently, so the results do not depend on the thread count. Reductions keep one
 * compensated partial per slowest-axis row (y in 2-D, z in 3-D) and fold the rows in
 * increasing order, which is also independent of the thread count.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

static inline size_t at(const int* g, int x, int y, int z)
{
    return ((size_t)(z + g[5]) * (size_t)g[1] + (size_t)(y + g[4])) * (size_t)g[0]
           + (size_t)(x + g[3]);
}

/* COPY (a loop whose kernel is dst = src at offset o). */
void or_copy(const int* lo, const int* hi, double* dst, const int* dg,
             const double* src, const int* sg, const int* o)
{
    int z, y;
#pragma omp parallel for collapse(2) schedule(static)
    for (z = lo[2]; z < hi[2]; ++z)
        for (y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x)
                dst[at(dg, x, y, z)] = src[at(sg, x + o[0], y + o[1], z + o[2])];
}

/*
 * LINCOMB: weighted sum of all stencil samples plus an optional bounded nonlinear
 * term. Samples x_0..x_{M-1} are taken input by input, point by point (any number
 * M >= 1 of them). Returns 0, -1 for M < 1, -2 if a sample buffer could not be
 * allocated.
 *   acc = c0*x0; acc = acc + cm*xm (m = 1..M-1);
 *   if alpha != 0: acc = acc + ((alpha*a)*b) / (1 + c*c), a = x0, b = x_{1 mod M},
 *   c = x_{2 mod M}.
 * src[j] / sg[6j..] / npts[j]: input j; offs: 3 ints per sample (x, y, z).
 * dst is never read at a non-zero offset, so the in-place sweep equals "all reads,
 * then all writes".
 */
int or_lincomb(const int* lo, const int* hi, double* dst, const int* dg, int nin,
               const double* const* src, const int* sg, const int* npts, const int* offs,
               const double* coef, double alpha)
{
    int M = 0;
    for (int j = 0; j < nin; ++j) M += npts[j];
    if (M < 1) return -1;
    int failed = 0;
#pragma omp parallel
    {
        /* the samples of one point; any count (one buffer per thread) */
        double* xs = (double*)malloc(sizeof(double) * (size_t)M);
        if (!xs) {
#pragma omp atomic write
            failed = 1;
        }
        int z, y;
#pragma omp for collapse(2) schedule(static)
        for (z = lo[2]; z < hi[2]; ++z)
            for (y = lo[1]; y < hi[1]; ++y) {
                if (!xs) continue;
                for (int x = lo[0]; x < hi[0]; ++x) {
                    int m = 0;
                    for (int j = 0; j < nin; ++j)
                        for (int k = 0; k < npts[j]; ++k, ++m) {
                            const int* o = offs + 3 * m;
                            xs[m] = src[j][at(sg + 6 * j, x + o[0], y + o[1], z + o[2])];
                        }
                    double acc = coef[0] * xs[0];
                    for (m = 1; m < M; ++m) acc = acc + coef[m] * xs[m];
                    if (alpha != 0.0) {
                        double a = xs[0], b = xs[1 % M], c = xs[2 % M];
                        acc = acc + ((alpha * a) * b) / (1.0 + c * c);
                    }
                    dst[at(dg, x, y, z)] = acc;
                }
            }
        free(xs);
    }
    return failed ? -2 : 0;
}

/*
 * Reduction value of one point: v = a (+ b), mode 0: v, 1: |v|, 2: v*v.
 * op 0 = sum, 1 = max, 2 = min over the range. A sum is accumulated with
 * Neumaier's compensated summation (error <= 2u|s| + O(n u^2) sum|v|, i.e. the
 * exactly rounded sum up to a couple of ulps), first per slowest-axis row (y in 2-D,
 * z in 3-D), then over the rows in increasing order, so the result is independent of
 * the thread count.
 * Returns the folded value; an empty range returns the identity (0, -inf, +inf).
 */
static inline void neumaier(double* s, double* c, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
    else                     *c += (v - t) + *s;
    *s = t;
}

double or_reduce(const int* lo, const int* hi, const double* a, const int* ag,
                 const double* b, const int* bg, int mode, int op)
{
    if (hi[2] <= lo[2] || hi[1] <= lo[1] || hi[0] <= lo[0])
        return op == 0 ? 0.0 : (op == 1 ? -INFINITY : INFINITY);
    /* slowest axis: z for a 3-D array (z extent > 1), y for a 2-D one */
    const int three = ag[2] > 1;
    const int r0 = three ? lo[2] : lo[1];
    const int nr = three ? hi[2] - lo[2] : hi[1] - lo[1];
    double* rs = (double*)malloc(sizeof(double) * (size_t)nr * 2);
    if (!rs) return NAN;
    int k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < nr; ++k) {
        double s = 0.0, c = 0.0;
        double m = op == 1 ? -INFINITY : INFINITY;
        const int z0 = three ? r0 + k : lo[2], z1 = three ? r0 + k + 1 : hi[2];
        const int y0 = three ? lo[1] : r0 + k, y1 = three ? hi[1] : r0 + k + 1;
        for (int z = z0; z < z1; ++z)
            for (int y = y0; y < y1; ++y)
                for (int x = lo[0]; x < hi[0]; ++x) {
                    double v = a[at(ag, x, y, z)];
                    if (b) v = v + b[at(bg, x, y, z)];
                    if (mode == 1) v = fabs(v);
                    else if (mode == 2) v = v * v;
                    if (op == 0) neumaier(&s, &c, v);
                    else if (op == 1) m = v > m ? v : m;
                    else m = v < m ? v : m;
                }
        rs[2 * k] = op == 0 ? s : m;
        rs[2 * k + 1] = c;
    }
    double s = 0.0, c = 0.0, m = op == 1 ? -INFINITY : INFINITY;
    for (k = 0; k < nr; ++k) {
        if (op == 0) { neumaier(&s, &c, rs[2 * k]); neumaier(&s, &c, rs[2 * k + 1]); }
        else if (op == 1) m = rs[2 * k] > m ? rs[2 * k] : m;
        else m = rs[2 * k] < m ? rs[2 * k] : m;
    }
    free(rs);
    return op == 0 ? s + c : m;
}

/* Threads the oracle runs with from now on (n >= 1), for timing it at one thread and at
 * all cores; results do not depend on it. */
void or_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Number of OpenMP threads the oracle runs with (for reporting). */
int or_threads(void)
{
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            n = omp_get_num_threads();
#endif
        }
    }
    return n;
}
