/*
 * oracle.c -- plain FP64 CPU reference for the second-order thin-disk force on
 * nested grids (Wang, Taam & Yen, "Self-gravitational force calculation of
 * infinitesimally thin gaseous disks on nested grids", Sec. 2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library and its binding) never calls it, and this file shares no code,
 * header, table or constant with the product path.
 *
 * What it computes (the definition, summed directly at O(N^4)):
 *   for every requested target cell centre (x_t, y_t) of level t,
 *     F_x = sum over levels s, over source cells c of level s that are not
 *           covered by level s+1, of
 *           Int_c (xb - x_t)/r^3 * [sig_c + dx_c (xb - x_c) + dy_c (yb - y_c)]
 *     F_y = same with (yb - y_t)/r^3,
 *   r = |(xb,yb) - (x_t,y_t)|, G = 1 (Sec. 2.1, Eq. for F^{x,0}+F^{x,x}+F^{x,y};
 *   the linear density within a cell is Eq. (eqnSigma), expanded about the
 *   source cell centre), and the potential of the same density,
 *     Phi = - sum over the same cells of Int_c [sig_c + ...] / r  (Sec. 2.1).
 * Each cell integral is evaluated exactly through antiderivatives evaluated at
 * the four cell corners (the double difference "g|^b_a|^d_c" of Sec. 2.1):
 *   Int u/r^3     = DD[ Kx0(u,v) ],  Kx0 = the kernel of Eq. (eqnCalK)
 *   Int v/r^3     = DD[ Kx0(v,u) ]   (x <-> y symmetry)
 *   Int u^2/r^3   = DD[ v ln(u + r) ]
 *   Int v^2/r^3   = DD[ u ln(v + r) ]
 *   Int u v/r^3   = DD[ -r ]
 * The last three are derived here by differentiation; the slope kernels
 * printed in Sec. 2.1 (K^{x,x}, K^{x,y}) do not differentiate back to the
 * slope integrands, so they are not used.
 *
 * Readings where the paper is silent (stated once, here and in the design notes):
 *  - N cells per side per level, level l cell size h0/2^l, one patch per level;
 *    level l's lower-left corner is level (l-1)'s corner plus off[l] cells of
 *    level l-1 (integer refinement ratio 2, Sec. 2.1 "positive integer").
 *  - Level l cells lying under the level l+1 patch are not part of Omega^l:
 *    they contribute no mass and receive no force (reported as 0).
 *  - Slopes: central difference (s[i+1]-s[i-1])/(2h) inside a patch,
 *    one-sided inward difference on the first and last cell of each row or
 *    column of every patch; before differencing, every covered cell takes the
 *    mean of its four children (recursively from the finest level).
 *  - Eq. (eqnCalK) with sgn(0) = 0, so the corner value at u = v = 0 is 0;
 *    no epsilon (Eq. eqnCalKepsilon) is added: lattice coordinates are exact.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_LEVELS 8

typedef struct {
    int n;          /* cells per side on every level */
    int levels;     /* number of levels, level 0 coarsest */
    double x0, y0;  /* lower-left corner of level 0 */
    double h0;      /* level-0 cell size */
    int off[ORACLE_MAX_LEVELS][2]; /* level l origin in level-(l-1) cells (x, y) */
} oracle_nest;

static double sgn(double x) { return (x > 0.0) - (x < 0.0); }

/* Eq. (eqnCalK):  Kx0(x,y) = -|sgn x| ln(y + sqrt(x^2+y^2)) - (1-|sgn x|) sgn(y) ln|y|.
 * For x != 0 the logarithm is evaluated through the identity
 * ln(y + sqrt(x^2+y^2)) = asinh(y/|x|) + ln|x|, which is the same function but
 * does not lose digits when y < 0 (y + sqrt(...) would cancel). */
static double kernel_x0(double x, double y)
{
    if (x != 0.0)
        return -(asinh(y / fabs(x)) + log(fabs(x)));
    if (y == 0.0)
        return 0.0; /* sgn(0) = 0 */
    return -sgn(y) * log(fabs(y));
}

/* Antiderivative of u^2/r^3:  d/du d/dv [ v ln(u + r) ] = u^2 / r^3.
 * For v != 0, ln(u + r) = asinh(u/|v|) + ln|v|; at v = 0 the value is 0
 * (v ln(...) -> 0). */
static double kernel_xx(double u, double v)
{
    if (v == 0.0)
        return 0.0;
    return v * (asinh(u / fabs(v)) + log(fabs(v)));
}

/* Antiderivative of u v / r^3:  d/du d/dv [ -r ] = u v / r^3. */
static double kernel_xy(double u, double v) { return -sqrt(u * u + v * v); }

/* The five corner antiderivatives at one corner (u, v) of a cell, relative
 * to the target point. */
static void corner_values(double u, double v, double k[5])
{
    k[0] = kernel_x0(u, v);  /* -> Int u/r^3   */
    k[1] = kernel_x0(v, u);  /* -> Int v/r^3   */
    k[2] = kernel_xx(u, v);  /* -> Int u^2/r^3 */
    k[3] = kernel_xx(v, u);  /* -> Int v^2/r^3 */
    k[4] = kernel_xy(u, v);  /* -> Int u v/r^3 */
}

/* Cell integrals over u in [a,b], v in [c,d] (target at the origin):
 * out = {Int u/r^3, Int v/r^3, Int u^2/r^3, Int v^2/r^3, Int uv/r^3},
 * each as the double difference g(b,d) - g(a,d) - g(b,c) + g(a,c). */
void oracle_cell_integrals(double a, double b, double c, double d, double *out)
{
    double kbd[5], kad[5], kbc[5], kac[5];
    corner_values(b, d, kbd);
    corner_values(a, d, kad);
    corner_values(b, c, kbc);
    corner_values(a, c, kac);
    for (int q = 0; q < 5; ++q)
        out[q] = kbd[q] - kad[q] - kbc[q] + kac[q];
}

/* ------------------------------------------------------------ potential */
/* The potential of the same linear density (G = 1):
 *   Phi(t) = - sum_c Int_c [sig_c + dx_c (xb - x_c) + dy_c (yb - y_c)] / r,
 * with the cell integrals (derived here by differentiation: each line's
 * antiderivative G has d/du d/dv G equal to the integrand)
 *   Int 1/r   = DD[ u ln(v + r) + v ln(u + r) ]
 *   Int u/r   = DD[ (v r + u^2 ln(v + r)) / 2 ]
 *   Int v/r   = DD[ (u r + v^2 ln(u + r)) / 2 ]
 * and ln(y + sqrt(x^2 + y^2)) written as asinh(y/|x|) + ln|x| for x != 0; a
 * term multiplied by the x that vanishes there is 0. */
static double log_r(double y, double x)  /* ln(y + sqrt(x^2 + y^2)), x != 0 */
{
    return asinh(y / fabs(x)) + log(fabs(x));
}

static void corner_values_potential(double u, double v, double k[3])
{
    const double r = sqrt(u * u + v * v);
    const double lu = u != 0.0 ? u * log_r(v, u) : 0.0;      /* u ln(v + r) */
    const double lv = v != 0.0 ? v * log_r(u, v) : 0.0;      /* v ln(u + r) */
    k[0] = lu + lv;                                          /* -> Int 1/r */
    k[1] = 0.5 * (v * r + (u != 0.0 ? u * lu : 0.0));        /* -> Int u/r */
    k[2] = 0.5 * (u * r + (v != 0.0 ? v * lv : 0.0));        /* -> Int v/r */
}

/* out = {Int 1/r, Int u/r, Int v/r} over u in [a,b], v in [c,d]. */
void oracle_cell_integrals_potential(double a, double b, double c, double d, double *out)
{
    double kbd[3], kad[3], kbc[3], kac[3];
    corner_values_potential(b, d, kbd);
    corner_values_potential(a, d, kad);
    corner_values_potential(b, c, kbc);
    corner_values_potential(a, c, kac);
    for (int q = 0; q < 3; ++q)
        out[q] = kbd[q] - kad[q] - kbc[q] + kac[q];
}

/* ---------------------------------------------------------------- geometry */

static double level_h(const oracle_nest *g, int l) { return ldexp(g->h0, -l); }

static void level_origin(const oracle_nest *g, int l, double *X, double *Y)
{
    double x = g->x0, y = g->y0;
    for (int k = 1; k <= l; ++k) {
        x += g->off[k][0] * level_h(g, k - 1);
        y += g->off[k][1] * level_h(g, k - 1);
    }
    *X = x;
    *Y = y;
}

/* Is cell (i, j) of level l under the level l+1 patch? */
static int covered(const oracle_nest *g, int l, int i, int j)
{
    if (l + 1 >= g->levels)
        return 0;
    int ox = g->off[l + 1][0], oy = g->off[l + 1][1], half = g->n / 2;
    return i >= ox && i < ox + half && j >= oy && j < oy + half;
}

int oracle_validate(const oracle_nest *g)
{
    if (g->n < 4 || (g->n & 1) || g->levels < 1 || g->levels > ORACLE_MAX_LEVELS || !(g->h0 > 0.0))
        return -1;
    for (int l = 1; l < g->levels; ++l)
        for (int a = 0; a < 2; ++a)
            if (g->off[l][a] < 0 || g->off[l][a] > g->n / 2)
                return -1;
    return 0;
}

/* ------------------------------------------------- density reconstruction */

/* sig[l], dsx[l], dsy[l]: caller-allocated n*n arrays (row-major [j][i]).
 * On return they hold the source fields of Eq. (eqnSigma): the cell value and
 * the x and y slopes per unit length, zero on covered cells. */
int oracle_prepare(const oracle_nest *g, const double *const *sigma_in,
                   double **sig, double **dsx, double **dsy)
{
    if (oracle_validate(g))
        return -1;
    const int n = g->n, L = g->levels;
    /* 1) copy, then fill covered cells with the mean of their children, finest first */
    for (int l = 0; l < L; ++l)
        memcpy(sig[l], sigma_in[l], sizeof(double) * (size_t)n * n);
    for (int l = L - 2; l >= 0; --l) {
        const int ox = g->off[l + 1][0], oy = g->off[l + 1][1];
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                if (!covered(g, l, i, j))
                    continue;
                const int ci = 2 * (i - ox), cj = 2 * (j - oy);
                const double *f = sig[l + 1];
                sig[l][(size_t)j * n + i] =
                    0.25 * (f[(size_t)cj * n + ci] + f[(size_t)cj * n + ci + 1] +
                            f[(size_t)(cj + 1) * n + ci] + f[(size_t)(cj + 1) * n + ci + 1]);
            }
    }
    /* 2) slopes per unit length, 3) remove covered cells from the sources */
    for (int l = 0; l < L; ++l) {
        const double h = level_h(g, l);
        const double *s = sig[l];
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double sx, sy;
                if (i == 0)
                    sx = (s[(size_t)j * n + 1] - s[(size_t)j * n]) / h;
                else if (i == n - 1)
                    sx = (s[(size_t)j * n + n - 1] - s[(size_t)j * n + n - 2]) / h;
                else
                    sx = (s[(size_t)j * n + i + 1] - s[(size_t)j * n + i - 1]) / (2.0 * h);
                if (j == 0)
                    sy = (s[(size_t)n + i] - s[i]) / h;
                else if (j == n - 1)
                    sy = (s[(size_t)(n - 1) * n + i] - s[(size_t)(n - 2) * n + i]) / h;
                else
                    sy = (s[(size_t)(j + 1) * n + i] - s[(size_t)(j - 1) * n + i]) / (2.0 * h);
                dsx[l][(size_t)j * n + i] = sx;
                dsy[l][(size_t)j * n + i] = sy;
            }
    }
    for (int l = 0; l < L; ++l)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                if (covered(g, l, i, j)) {
                    sig[l][(size_t)j * n + i] = 0.0;
                    dsx[l][(size_t)j * n + i] = 0.0;
                    dsy[l][(size_t)j * n + i] = 0.0;
                }
    return 0;
}

/* ------------------------------------------------------------ direct sum */

/* Force at one target point from the prepared source fields of one patch of
 * n x n cells of size h with lower-left corner (X, Y).  The corner
 * antiderivatives are evaluated on the patch's (n+1)^2 edge lattice one edge
 * row at a time, and every cell takes its double difference. */
static void sum_patch(int n, double X, double Y, double h, const double *sig, const double *dsx,
                      const double *dsy, double xt, double yt, double *row_lo, double *row_hi,
                      double *fx, double *fy)
{
    double ax = 0.0, ay = 0.0;
    for (int i = 0; i <= n; ++i)
        corner_values(X + i * h - xt, Y - yt, row_lo + 5 * i);
    for (int j = 0; j < n; ++j) {
        const double vlo = Y + j * h - yt;
        const double vhi = Y + (j + 1) * h - yt;
        for (int i = 0; i <= n; ++i)
            corner_values(X + i * h - xt, vhi, row_hi + 5 * i);
        const double vc = vlo + 0.5 * h; /* source cell centre, relative to the target */
        for (int i = 0; i < n; ++i) {
            const size_t c = (size_t)j * n + i;
            if (sig[c] == 0.0 && dsx[c] == 0.0 && dsy[c] == 0.0)
                continue; /* empty (or covered) cell: contributes exactly 0 */
            const double *kbd = row_hi + 5 * (i + 1), *kad = row_hi + 5 * i;
            const double *kbc = row_lo + 5 * (i + 1), *kac = row_lo + 5 * i;
            double I[5];
            for (int q = 0; q < 5; ++q)
                I[q] = kbd[q] - kad[q] - kbc[q] + kac[q];
            const double uc = X + (i + 0.5) * h - xt;
            /* F^{x,0} + F^{x,x} + F^{x,y}, slope weights about the source centre */
            ax += sig[c] * I[0] + dsx[c] * (I[2] - uc * I[0]) + dsy[c] * (I[4] - vc * I[0]);
            ay += sig[c] * I[1] + dsx[c] * (I[4] - uc * I[1]) + dsy[c] * (I[3] - vc * I[1]);
        }
        double *t = row_lo;
        row_lo = row_hi;
        row_hi = t;
    }
    *fx += ax;
    *fy += ay;
}

static void sum_level(const oracle_nest *g, int s, const double *sig, const double *dsx,
                      const double *dsy, double xt, double yt, double *row_lo, double *row_hi,
                      double *fx, double *fy)
{
    double X, Y;
    level_origin(g, s, &X, &Y);
    sum_patch(g->n, X, Y, level_h(g, s), sig, dsx, dsy, xt, yt, row_lo, row_hi, fx, fy);
}

/* Forces at nt targets (level tl[k], cell ti[k], tj[k]) from prepared fields.
 * Covered targets get 0.  nthreads <= 0 uses the OpenMP default. */
int oracle_force_targets(const oracle_nest *g, const double *const *sig, const double *const *dsx,
                         const double *const *dsy, long nt, const int *tl, const int *ti,
                         const int *tj, double *fx, double *fy, int nthreads)
{
    if (oracle_validate(g))
        return -1;
    const int n = g->n, L = g->levels;
    for (long k = 0; k < nt; ++k)
        if (tl[k] < 0 || tl[k] >= L || ti[k] < 0 || ti[k] >= n || tj[k] < 0 || tj[k] >= n)
            return -2;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int fail = 0;
#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * 10 * (size_t)(n + 1));
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (long k = 0; k < nt; ++k) {
            if (!buf)
                continue;
            double ax = 0.0, ay = 0.0;
            if (!covered(g, tl[k], ti[k], tj[k])) {
                double X, Y;
                level_origin(g, tl[k], &X, &Y);
                const double h = level_h(g, tl[k]);
                const double xt = X + (ti[k] + 0.5) * h, yt = Y + (tj[k] + 0.5) * h;
                for (int s = 0; s < L; ++s)
                    sum_level(g, s, sig[s], dsx[s], dsy[s], xt, yt, buf, buf + 5 * (size_t)(n + 1),
                              &ax, &ay);
            }
            fx[k] = ax;
            fy[k] = ay;
        }
        free(buf);
    }
    return fail ? -3 : 0;
}

/* Forces at the targets (ti[k], jt), k < nt, of one row jt of a single-level
 * grid (levels == 1), from prepared fields: the same direct sum over every
 * source cell as oracle_force_targets, evaluated for many targets of one row.
 * On one level every coordinate difference is a whole number of half cells:
 * a source corner lies (e - 1/2) h from a target centre along x, e = corner
 * column - target column, and the cell centre a h, a = cell column - target
 * column; along y likewise with the rows.  So for a source row j the cell
 * integrals depend on the target only through a, and they are evaluated once
 * per a in [-(n-1), n-1] (corner antiderivatives on the 2n corner offsets of
 * the row's two edges, then the double difference, in the order of sum_patch)
 * and read by every target of the row.  Each target sums the cells row by row,
 * column by column, as sum_patch does; differences are written (e - 1/2) h,
 * a h and (j - jt +- 1/2) h, which are the lattice positions themselves (exact
 * when h is a power of two, as for grids on [-1, 1] with n a power of two).
 * Returns 0, -1 for a descriptor with more than one level, -2 for a target
 * outside the grid, -3 when memory runs out. */
int oracle_force_row(const oracle_nest *g, const double *sig, const double *dsx, const double *dsy, int jt,
                     long nt, const int *ti, double *fx, double *fy, int nthreads)
{
    if (oracle_validate(g) || g->levels != 1)
        return -1;
    const int n = g->n;
    const double h = g->h0;
    if (jt < 0 || jt >= n)
        return -2;
    for (long k = 0; k < nt; ++k)
        if (ti[k] < 0 || ti[k] >= n)
            return -2;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const int E = 2 * n;  /* corner offsets e = -(n-1) .. n at index e + n - 1 */
    double *lo = (double *)malloc(sizeof(double) * 5 * (size_t)E);
    double *hi = (double *)malloc(sizeof(double) * 5 * (size_t)E);
    double *I = (double *)malloc(sizeof(double) * 5 * (size_t)(E - 1));  /* a + n - 1 */
    double *ax = (double *)calloc((size_t)(nt > 0 ? nt : 1), sizeof(double));
    double *ay = (double *)calloc((size_t)(nt > 0 ? nt : 1), sizeof(double));
    if (!lo || !hi || !I || !ax || !ay) {
        free(lo);
        free(hi);
        free(I);
        free(ax);
        free(ay);
        return -3;
    }
#pragma omp parallel
    {
#pragma omp for schedule(static)
        for (int x = 0; x < E; ++x)  /* lower edge of source row 0 */
            corner_values((x - n + 1 - 0.5) * h, (0 - jt - 0.5) * h, lo + 5 * (size_t)x);
        for (int j = 0; j < n; ++j) {
#pragma omp for schedule(static)
            for (int x = 0; x < E; ++x)  /* upper edge of source row j */
                corner_values((x - n + 1 - 0.5) * h, (j - jt + 0.5) * h, hi + 5 * (size_t)x);
#pragma omp for schedule(static)
            for (int x = 0; x < E - 1; ++x) {  /* cell offset a = x - (n - 1) */
                const double *kbd = hi + 5 * (size_t)(x + 1), *kad = hi + 5 * (size_t)x;
                const double *kbc = lo + 5 * (size_t)(x + 1), *kac = lo + 5 * (size_t)x;
                for (int q = 0; q < 5; ++q)
                    I[5 * (size_t)x + q] = kbd[q] - kad[q] - kbc[q] + kac[q];
            }
            const double vc = (j - jt) * h;
#pragma omp for schedule(static)
            for (long k = 0; k < nt; ++k) {
                double sx = ax[k], sy = ay[k];
                for (int i = 0; i < n; ++i) {
                    const size_t c = (size_t)j * n + i;
                    if (sig[c] == 0.0 && dsx[c] == 0.0 && dsy[c] == 0.0)
                        continue;
                    const int a = i - ti[k];
                    const double *Ia = I + 5 * (size_t)(a + n - 1);
                    const double uc = a * h;
                    sx += sig[c] * Ia[0] + dsx[c] * (Ia[2] - uc * Ia[0]) + dsy[c] * (Ia[4] - vc * Ia[0]);
                    sy += sig[c] * Ia[1] + dsx[c] * (Ia[4] - uc * Ia[1]) + dsy[c] * (Ia[3] - vc * Ia[1]);
                }
                ax[k] = sx;
                ay[k] = sy;
            }
#pragma omp single
            {
                double *t = lo;
                lo = hi;
                hi = t;
            }
        }
    }
    for (long k = 0; k < nt; ++k) {
        fx[k] = ax[k];
        fy[k] = ay[k];
    }
    free(lo);
    free(hi);
    free(I);
    free(ax);
    free(ay);
    return 0;
}

/* Potential at one target point from the prepared fields of one patch (the
 * same edge-lattice walk as sum_patch). */
static void sum_patch_potential(int n, double X, double Y, double h, const double *sig, const double *dsx,
                                const double *dsy, double xt, double yt, double *row_lo, double *row_hi,
                                double *phi)
{
    double acc = 0.0;
    for (int i = 0; i <= n; ++i)
        corner_values_potential(X + i * h - xt, Y - yt, row_lo + 3 * i);
    for (int j = 0; j < n; ++j) {
        const double vlo = Y + j * h - yt;
        const double vhi = Y + (j + 1) * h - yt;
        for (int i = 0; i <= n; ++i)
            corner_values_potential(X + i * h - xt, vhi, row_hi + 3 * i);
        const double vc = vlo + 0.5 * h;
        for (int i = 0; i < n; ++i) {
            const size_t c = (size_t)j * n + i;
            if (sig[c] == 0.0 && dsx[c] == 0.0 && dsy[c] == 0.0)
                continue;
            const double *kbd = row_hi + 3 * (i + 1), *kad = row_hi + 3 * i;
            const double *kbc = row_lo + 3 * (i + 1), *kac = row_lo + 3 * i;
            double J[3];
            for (int q = 0; q < 3; ++q)
                J[q] = kbd[q] - kad[q] - kbc[q] + kac[q];
            const double uc = X + (i + 0.5) * h - xt;
            acc -= sig[c] * J[0] + dsx[c] * (J[1] - uc * J[0]) + dsy[c] * (J[2] - vc * J[0]);
        }
        double *t = row_lo;
        row_lo = row_hi;
        row_hi = t;
    }
    *phi += acc;
}

static void sum_level_potential(const oracle_nest *g, int s, const double *sig, const double *dsx,
                                const double *dsy, double xt, double yt, double *row_lo, double *row_hi,
                                double *phi)
{
    double X, Y;
    level_origin(g, s, &X, &Y);
    sum_patch_potential(g->n, X, Y, level_h(g, s), sig, dsx, dsy, xt, yt, row_lo, row_hi, phi);
}

/* Potential at nt targets (level tl[k], cell ti[k], tj[k]) from prepared
 * fields.  Covered targets get 0.  nthreads <= 0 uses the OpenMP default. */
int oracle_potential_targets(const oracle_nest *g, const double *const *sig, const double *const *dsx,
                             const double *const *dsy, long nt, const int *tl, const int *ti,
                             const int *tj, double *phi, int nthreads)
{
    if (oracle_validate(g))
        return -1;
    const int n = g->n, L = g->levels;
    for (long k = 0; k < nt; ++k)
        if (tl[k] < 0 || tl[k] >= L || ti[k] < 0 || ti[k] >= n || tj[k] < 0 || tj[k] >= n)
            return -2;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int fail = 0;
#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * 6 * (size_t)(n + 1));
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (long k = 0; k < nt; ++k) {
            if (!buf)
                continue;
            double p = 0.0;
            if (!covered(g, tl[k], ti[k], tj[k])) {
                double X, Y;
                level_origin(g, tl[k], &X, &Y);
                const double h = level_h(g, tl[k]);
                const double xt = X + (ti[k] + 0.5) * h, yt = Y + (tj[k] + 0.5) * h;
                for (int s = 0; s < L; ++s)
                    sum_level_potential(g, s, sig[s], dsx[s], dsy[s], xt, yt, buf, buf + 3 * (size_t)(n + 1), &p);
            }
            phi[k] = p;
        }
        free(buf);
    }
    return fail ? -3 : 0;
}

/* ------------------------------------------------------------------ forests */
/* Several patches per level (Sec. 2.1: Omega^l_k, k = 1..K^l).  Every patch has
 * n x n cells of its level's size h0/2^l; patch p's lower-left corner is
 * (x0, y0) + org[p] cells of its level.  Readings (the paper allows any patch
 * extents; the patches here share n so that one transform size serves all):
 *  - patches are listed coarsest level first, level 0 first of all;
 *  - a patch of level l >= 1 starts on a cell edge of level l-1 (org even) and
 *    lies inside the union of the level l-1 patches; it may straddle several;
 *  - patches of one level do not overlap (they may share edges);
 *  - a cell of level l under a level l+1 patch is covered: no mass, no force
 *    (reported as 0), and for the slopes it takes the mean of its children;
 *  - slopes as for nests: central inside each patch, one-sided inward on the
 *    patch's first and last cell of every row and column (also where the
 *    patch touches another patch of its level). */
#define ORACLE_MAX_PATCHES 16

typedef struct {
    int n, patches;
    double x0, y0, h0;
    int level[ORACLE_MAX_PATCHES];
    int org[ORACLE_MAX_PATCHES][2];
} oracle_forest;

static double patch_h(const oracle_forest *f, int p) { return ldexp(f->h0, -f->level[p]); }

static void patch_origin(const oracle_forest *f, int p, double *X, double *Y)
{
    const double h = patch_h(f, p);
    *X = f->x0 + f->org[p][0] * h;
    *Y = f->y0 + f->org[p][1] * h;
}

/* The patch q of level(p)+1 that covers cell (i, j) of patch p, or -1; (fx, fy):
 * q's corner in p's cells. */
static int forest_child(const oracle_forest *f, int p, int i, int j, int *fx, int *fy)
{
    const int half = f->n / 2;
    for (int q = 0; q < f->patches; ++q) {
        if (f->level[q] != f->level[p] + 1)
            continue;
        const int cx = f->org[q][0] / 2 - f->org[p][0], cy = f->org[q][1] / 2 - f->org[p][1];
        if (i >= cx && i < cx + half && j >= cy && j < cy + half) {
            *fx = cx;
            *fy = cy;
            return q;
        }
    }
    return -1;
}

int oracle_forest_validate(const oracle_forest *f)
{
    const int n = f->n, K = f->patches;
    if (n < 4 || (n & 1) || K < 1 || K > ORACLE_MAX_PATCHES || !(f->h0 > 0.0) || f->level[0] != 0)
        return -1;
    for (int p = 1; p < K; ++p) {
        if (f->level[p] < f->level[p - 1] || f->level[p] > f->level[p - 1] + 1 || f->level[p] > 20)
            return -1;
        if (f->level[p] > 0 && ((f->org[p][0] & 1) || (f->org[p][1] & 1)))
            return -1;
    }
    for (int p = 0; p < K; ++p)
        for (int q = p + 1; q < K; ++q)
            if (f->level[p] == f->level[q] && abs(f->org[p][0] - f->org[q][0]) < n &&
                abs(f->org[p][1] - f->org[q][1]) < n)
                return -2; /* overlapping patches of one level */
    for (int p = 0; p < K; ++p) {
        if (f->level[p] == 0)
            continue;
        const int half = n / 2;
        for (int y = f->org[p][1] / 2; y < f->org[p][1] / 2 + half; ++y)
            for (int x = f->org[p][0] / 2; x < f->org[p][0] / 2 + half; ++x) {
                int inside = 0;
                for (int q = 0; q < K && !inside; ++q)
                    inside = f->level[q] == f->level[p] - 1 && x >= f->org[q][0] && x < f->org[q][0] + n &&
                             y >= f->org[q][1] && y < f->org[q][1] + n;
                if (!inside)
                    return -3; /* a patch outside the coarser level */
            }
    }
    return 0;
}

/* As oracle_prepare, per patch. */
int oracle_forest_prepare(const oracle_forest *f, const double *const *sigma_in, double **sig, double **dsx,
                          double **dsy)
{
    if (oracle_forest_validate(f))
        return -1;
    const int n = f->n, K = f->patches;
    for (int p = 0; p < K; ++p)
        memcpy(sig[p], sigma_in[p], sizeof(double) * (size_t)n * n);
    /* covered cells take the mean of their children, finest patches first */
    for (int p = K - 1; p >= 0; --p)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                int cx, cy;
                const int q = forest_child(f, p, i, j, &cx, &cy);
                if (q < 0)
                    continue;
                const int ci = 2 * (i - cx), cj = 2 * (j - cy);
                const double *c = sig[q];
                sig[p][(size_t)j * n + i] = 0.25 * (c[(size_t)cj * n + ci] + c[(size_t)cj * n + ci + 1] +
                                                    c[(size_t)(cj + 1) * n + ci] + c[(size_t)(cj + 1) * n + ci + 1]);
            }
    for (int p = 0; p < K; ++p) {
        const double h = patch_h(f, p);
        const double *v = sig[p];
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double sx, sy;
                if (i == 0)
                    sx = (v[(size_t)j * n + 1] - v[(size_t)j * n]) / h;
                else if (i == n - 1)
                    sx = (v[(size_t)j * n + n - 1] - v[(size_t)j * n + n - 2]) / h;
                else
                    sx = (v[(size_t)j * n + i + 1] - v[(size_t)j * n + i - 1]) / (2.0 * h);
                if (j == 0)
                    sy = (v[(size_t)n + i] - v[i]) / h;
                else if (j == n - 1)
                    sy = (v[(size_t)(n - 1) * n + i] - v[(size_t)(n - 2) * n + i]) / h;
                else
                    sy = (v[(size_t)(j + 1) * n + i] - v[(size_t)(j - 1) * n + i]) / (2.0 * h);
                dsx[p][(size_t)j * n + i] = sx;
                dsy[p][(size_t)j * n + i] = sy;
            }
    }
    for (int p = 0; p < K; ++p)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                int cx, cy;
                if (forest_child(f, p, i, j, &cx, &cy) >= 0) {
                    sig[p][(size_t)j * n + i] = 0.0;
                    dsx[p][(size_t)j * n + i] = 0.0;
                    dsy[p][(size_t)j * n + i] = 0.0;
                }
            }
    return 0;
}

/* Forces (want_phi = 0) or the potential (want_phi = 1, into fx) at nt targets
 * (patch tp[k], cell ti[k], tj[k]) from prepared fields; covered targets get 0. */
static int forest_targets(const oracle_forest *f, const double *const *sig, const double *const *dsx,
                          const double *const *dsy, long nt, const int *tp, const int *ti, const int *tj,
                          double *fx, double *fy, int nthreads, int want_phi)
{
    if (oracle_forest_validate(f))
        return -1;
    const int n = f->n, K = f->patches;
    for (long k = 0; k < nt; ++k)
        if (tp[k] < 0 || tp[k] >= K || ti[k] < 0 || ti[k] >= n || tj[k] < 0 || tj[k] >= n)
            return -2;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int fail = 0;
#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * 10 * (size_t)(n + 1));
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (long k = 0; k < nt; ++k) {
            if (!buf)
                continue;
            double ax = 0.0, ay = 0.0;
            int cx, cy;
            if (forest_child(f, tp[k], ti[k], tj[k], &cx, &cy) < 0) {
                double X, Y;
                patch_origin(f, tp[k], &X, &Y);
                const double h = patch_h(f, tp[k]);
                const double xt = X + (ti[k] + 0.5) * h, yt = Y + (tj[k] + 0.5) * h;
                for (int s = 0; s < K; ++s) {
                    double SX, SY;
                    patch_origin(f, s, &SX, &SY);
                    if (want_phi)
                        sum_patch_potential(n, SX, SY, patch_h(f, s), sig[s], dsx[s], dsy[s], xt, yt, buf,
                                            buf + 3 * (size_t)(n + 1), &ax);
                    else
                        sum_patch(n, SX, SY, patch_h(f, s), sig[s], dsx[s], dsy[s], xt, yt, buf,
                                  buf + 5 * (size_t)(n + 1), &ax, &ay);
                }
            }
            fx[k] = ax;
            if (!want_phi)
                fy[k] = ay;
        }
        free(buf);
    }
    return fail ? -3 : 0;
}

int oracle_forest_force_targets(const oracle_forest *f, const double *const *sig, const double *const *dsx,
                                const double *const *dsy, long nt, const int *tp, const int *ti, const int *tj,
                                double *fx, double *fy, int nthreads)
{
    return forest_targets(f, sig, dsx, dsy, nt, tp, ti, tj, fx, fy, nthreads, 0);
}

int oracle_forest_potential_targets(const oracle_forest *f, const double *const *sig, const double *const *dsx,
                                    const double *const *dsy, long nt, const int *tp, const int *ti,
                                    const int *tj, double *phi, int nthreads)
{
    return forest_targets(f, sig, dsx, dsy, nt, tp, ti, tj, phi, NULL, nthreads, 1);
}

/* Threads the OpenMP runtime would use (for reporting the CPU baseline). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------- generalized convolutions */

/* The one-dimensional generalized convolution forms of Sec. 2.2, written out
 * as the plain sums of Eqs. (eqnbmnn) and (eqnbnmn) over all index pairs for
 * which both sequences are defined (b has nb terms, c has nc terms, every
 * other term is 0).  out has nout terms, out[k] = a_k. */
void oracle_genconv_case2(const double *b, int nb, const double *c, int nc, int m, double *out,
                          int nout)
{
    for (int k = 0; k < nout; ++k) {
        double acc = 0.0; /* a_k = sum_j b_{m k - j} c_j */
        for (int j = 0; j < nc; ++j) {
            const int idx = m * k - j;
            if (idx >= 0 && idx < nb)
                acc += b[idx] * c[j];
        }
        out[k] = acc;
    }
}

void oracle_genconv_case3(const double *b, int nb, const double *c, int nc, int m, double *out,
                          int nout)
{
    for (int k = 0; k < nout; ++k) {
        double acc = 0.0; /* a_k = sum_j b_{k - m j} c_j */
        for (int j = 0; j < nc; ++j) {
            const int idx = k - m * j;
            if (idx >= 0 && idx < nb)
                acc += b[idx] * c[j];
        }
        out[k] = acc;
    }
}
