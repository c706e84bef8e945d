/*
 * sph_oracle.c -- plain, slow FP64 CPU oracle of one SPH timestep on the
 * rotating square patch (SPH-EXA mini-app, arXiv 1905.03344).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library,
 * its Python binding) may include, link or call this file.  It shares no code,
 * header, table or constant with the CUDA sources: every formula below is
 * written out again from the paper.  Where the paper only cites a formula or
 * prints it garbled, the reading taken is stated next to the function and
 * tagged R1..R18 (the same tags label the same readings in the CUDA sources).
 *
 * Build:  gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC  (see build.py)
 * -ffp-contract=off keeps every a*b+c as two rounded operations, so the
 * neighbour predicate below is evaluated exactly in the order written.
 *
 * What each function follows:
 *   orc_w, orc_gradw_fac ...... Eq. 2 (Wendland kernel, Sec. 3), 1/h^3 restored,
 *                               or the Sinc family of Sec. 3 (orc_set_kernel)
 *   orc_pair_in ............... neighbour predicate, symmetric union (R11)
 *   orc_neighbors_brute ....... O(N^2) definition of the neighbour set (Table 1
 *                               "Neighbour Discovery"; the tree walk is replaced
 *                               by the definition itself)
 *   orc_neighbors_grid ........ the same set from a uniform cell grid
 *   orc_density ............... standard density summation (Sec. 3 "vanilla
 *                               SPH", Table 1 "Standard" volume elements; R1)
 *   orc_eos ................... ideal gas (R9)
 *   orc_momentum_energy ....... momentum eq. [rosswog2009] + artificial
 *                               viscosity [monaghan1983], Sec. 3 (R4-R6); with
 *                               an Omega array, the grad-h form of the same
 *                               reference (R20)
 *   orc_dwdh, orc_omega ....... dW/dh and the grad-h factor Omega (R20)
 *   orc_courant ............... Courant condition, global time-step (Sec. 3,
 *                               Table 1 "Global"; R7)
 *   orc_step .................. Press (leapfrog) positions, Adams-Bashforth
 *                               energy (Sec. 3; R8), h adaptation (R10)
 *   orc_conserved ............. mass, momentum, L_z, kinetic and internal
 *                               energy (Sec. 4 stresses conservation laws)
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * (closed forms, brute force, invariants, convergence order); none is
 * "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Kernel: Eq. 2, W(v,h) = sigma_W / h^3 * (1 - v/2)^4 (2v + 1), 0 <= v <= 2, */
/* v = r/h, sigma_W = 21/(16 pi).  The printed form omits 1/h^3 (R2).         */
/* ------------------------------------------------------------------------ */
double orc_sigma_w(void) { return 21.0 / (16.0 * M_PI); }

/* ------------------------------------------------------------------------ */
/* Kernel family.  Sec. 3 gives the mini-app two kernels: Wendland (Eq. 2)    */
/* and the Sinc functions                                                    */
/*   W_n(v, h) = B_n / h^3 S_n(pi v / 2),  0 <= v <= 2,  S_n = sinc^n,          */
/*   sinc(x) = sin(x) / x,                                                   */
/* B_n the normalisation: int W d^3x = 1, i.e.                               */
/*   4 pi B_n int_0^2 v^2 S_n(pi v / 2) dv = 1,                               */
/* evaluated here by composite Simpson's rule.                               */
/* ------------------------------------------------------------------------ */
enum { ORC_WENDLAND = 0, ORC_SINC = 1 };
static int g_kernel = ORC_WENDLAND;
static int g_sinc_n = 6;
static double g_sinc_bn = 0.0;

static double sinc_of(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

static double ipow(double b, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; k++) r *= b;
    return r;
}

double orc_sinc_bn(int n)
{
    const int M = 200000; /* even number of Simpson intervals on [0, 2] */
    const double dv = 2.0 / M;
    double s = 0.0;
    for (int k = 0; k <= M; k++) {
        double v = k * dv;
        double f = v * v * ipow(sinc_of(0.5 * M_PI * v), n);
        double wgt = (k == 0 || k == M) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
        s += wgt * f;
    }
    s *= dv / 3.0;
    return 1.0 / (4.0 * M_PI * s);
}

/* kind 0: Wendland (Eq. 2); kind 1: Sinc with index n (n >= 2) */
int orc_set_kernel(int kind, int n)
{
    if (kind == ORC_WENDLAND) {
        g_kernel = ORC_WENDLAND;
        return 0;
    }
    if (kind == ORC_SINC && n >= 2 && n <= 16) {
        g_kernel = ORC_SINC;
        g_sinc_n = n;
        g_sinc_bn = orc_sinc_bn(n);
        return 0;
    }
    return -1;
}

double orc_kernel_bn(void) { return g_kernel == ORC_SINC ? g_sinc_bn : orc_sigma_w(); }

/* (sin x - x cos x) / x^3: by its Taylor series sum_{m>=1} (-1)^(m+1) 2m
 * x^(2m-2) / (2m+1)! below x = 1 (the direct form cancels there), directly
 * above */
static double sinc_slope(double x)
{
    if (x < 1.0) {
        double x2 = x * x, t = 0.0, pw = 1.0, fact = 6.0; /* (2m+1)! for m = 1 */
        for (int m = 1; m <= 10; m++) {
            double term = 2.0 * m * pw / fact;
            t += (m & 1) ? term : -term;
            pw *= x2;
            fact *= (2.0 * m + 2.0) * (2.0 * m + 3.0);
        }
        return t;
    }
    return (sin(x) - x * cos(x)) / (x * x * x);
}

static double w_sinc(double r, double h)
{
    double v = r / h;
    if (v >= 2.0) return 0.0;
    return g_sinc_bn / (h * h * h) * ipow(sinc_of(0.5 * M_PI * v), g_sinc_n);
}

/* dW/dr = B_n/h^3 n S^(n-1) sinc'(x) dx/dr with x = pi v/2, dx/dr = pi/(2h);
 * sinc'(x) = -(sin x - x cos x)/x^2 and r = 2 h x / pi, so with
 * grad_i W = -f (x_i - x_j):  f = B_n n pi^2 / (4 h^5) S^(n-1) (sin x - x cos x)/x^3 */
static double gradw_fac_sinc(double r, double h)
{
    double v = r / h;
    if (v >= 2.0) return 0.0;
    double x = 0.5 * M_PI * v;
    double h2 = h * h;
    return g_sinc_bn * g_sinc_n * M_PI * M_PI / (4.0 * h2 * h2 * h) * ipow(sinc_of(x), g_sinc_n - 1) *
           sinc_slope(x);
}

double orc_w(double r, double h)
{
    if (g_kernel == ORC_SINC) return w_sinc(r, h);
    double v = r / h;
    if (v >= 2.0) return 0.0;
    double q = 1.0 - 0.5 * v;
    return orc_sigma_w() / (h * h * h) * (q * q * q * q) * (2.0 * v + 1.0);
}

/* dW/dr = sigma_W/h^4 * d/dv[(1-v/2)^4 (2v+1)] = -5 sigma_W/h^4 * v (1-v/2)^3,
 * so grad_i W(r_ij, h) = dW/dr * (x_i - x_j)/r = -(5 sigma_W / h^5)(1-v/2)^3 (x_i - x_j).
 * Returns the scalar f >= 0 with grad_i W = -f * (x_i - x_j).                */
double orc_gradw_fac(double r, double h)
{
    if (g_kernel == ORC_SINC) return gradw_fac_sinc(r, h);
    double v = r / h;
    if (v >= 2.0) return 0.0;
    double q = 1.0 - 0.5 * v;
    double h2 = h * h;
    return 5.0 * orc_sigma_w() / (h2 * h2 * h) * (q * q * q);
}

/* dW/dh at fixed r.  W = K/h^3 F(v), v = r/h:  dW/dh = -K/h^4 (3 F + v F'(v)).
 * Wendland: F = (1 - v/2)^4 (2v + 1), F' = -5 v (1 - v/2)^3.
 * Sinc: F = S^n(x), x = pi v/2, v F' = n S^(n-1) x S'(x) = -n S^(n-1) x^2 g(x),
 * g = (sin x - x cos x)/x^3.                                                 */
double orc_dwdh(double r, double h)
{
    double v = r / h;
    if (v >= 2.0) return 0.0;
    double h4 = h * h * h * h;
    if (g_kernel == ORC_SINC) {
        double x = 0.5 * M_PI * v;
        double S = sinc_of(x);
        double F = ipow(S, g_sinc_n);
        double vF = -g_sinc_n * ipow(S, g_sinc_n - 1) * x * x * sinc_slope(x);
        return -g_sinc_bn / h4 * (3.0 * F + vF);
    }
    double q = 1.0 - 0.5 * v;
    double F = q * q * q * q * (2.0 * v + 1.0);
    double vF = -5.0 * v * v * q * q * q;
    return -orc_sigma_w() / h4 * (3.0 * F + vF);
}

/* ------------------------------------------------------------------------ */
/* Neighbour predicate (R11): j is a neighbour of i iff j != i and           */
/* r^2 < 4 h_i^2 or r^2 < 4 h_j^2, with the minimum image along periodic z.  */
/* The operation order below is the definition; the CUDA side must reach the */
/* same decision bit for bit.                                                */
/* ------------------------------------------------------------------------ */
static double pair_r2(double xi, double yi, double zi, double xj, double yj, double zj, double lz)
{
    double dx = xi - xj;
    double dy = yi - yj;
    double dz = zi - zj;
    if (dz > 0.5 * lz) dz -= lz;
    else if (dz < -0.5 * lz) dz += lz;
    return (dx * dx + dy * dy) + dz * dz;
}

/* bit 0: j in the symmetric set N(i); bit 1: r^2 < 4 h_i^2 (counts n_i, R10) */
int orc_pair_in(double xi, double yi, double zi, double hi,
                double xj, double yj, double zj, double hj, double lz)
{
    double r2 = pair_r2(xi, yi, zi, xj, yj, zj, lz);
    int own = r2 < (4.0 * hi) * hi;
    int other = r2 < (4.0 * hj) * hj;
    return (own || other) | (own << 1);
}

/* Brute force, O(N^2).  Two passes: with col == NULL only off[] and nown[] are
 * written and the total is returned; with col != NULL rows are filled in
 * ascending j.  Returns -1 if cap is exceeded.                              */
int64_t orc_neighbors_brute(int64_t n, const double* x, const double* y, const double* z,
                            const double* h, double lz, int64_t* off, int32_t* col,
                            int32_t* nown, int64_t cap, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    if (col == NULL) {
        int64_t* cnt = off + 1;
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; i++) {
            int64_t c = 0, o = 0;
            for (int64_t j = 0; j < n; j++) {
                if (j == i) continue;
                int f = orc_pair_in(x[i], y[i], z[i], h[i], x[j], y[j], z[j], h[j], lz);
                c += f & 1;
                o += (f >> 1) & 1;
            }
            cnt[i] = c;
            nown[i] = (int32_t)o;
        }
        off[0] = 0;
        for (int64_t i = 0; i < n; i++) off[i + 1] += off[i];
        return off[n];
    }
    if (off[n] > cap) return -1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        int64_t k = off[i];
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            if (orc_pair_in(x[i], y[i], z[i], h[i], x[j], y[j], z[j], h[j], lz) & 1)
                col[k++] = (int32_t)j;
        }
    }
    return off[n];
}

/* ------------------------------------------------------------------------ */
/* Uniform grid.  Cells of edge S = 2 h_max (1 + 1e-9) in x and y over the   */
/* bounding box; along periodic z, ncz = floor(lz / S) cells of edge lz/ncz  */
/* when ncz >= 3, else a single z cell.  Any pair within 2 h_max is then in  */
/* adjacent cells, and every candidate is decided by orc_pair_in.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double xmin, ymin, S, sz, lz;
    int64_t ncx, ncy, ncz;
    int64_t* start; /* ncell + 1, bucket offsets */
    int64_t* items; /* n, particle ids in ascending order per cell */
} grid_t;

static int64_t cell_of(const grid_t* g, double x, double y, double z, int64_t* cx, int64_t* cy, int64_t* cz)
{
    int64_t a = (int64_t)floor((x - g->xmin) / g->S);
    int64_t b = (int64_t)floor((y - g->ymin) / g->S);
    int64_t c = 0;
    if (g->ncz > 1) c = (int64_t)floor((z + 0.5 * g->lz) / g->sz);
    if (a < 0) a = 0;
    if (a >= g->ncx) a = g->ncx - 1;
    if (b < 0) b = 0;
    if (b >= g->ncy) b = g->ncy - 1;
    if (c < 0) c = 0;
    if (c >= g->ncz) c = g->ncz - 1;
    *cx = a; *cy = b; *cz = c;
    return (c * g->ncy + b) * g->ncx + a;
}

static int grid_build(grid_t* g, int64_t n, const double* x, const double* y, const double* z,
                      const double* h, double lz)
{
    double xmin = x[0], xmax = x[0], ymin = y[0], ymax = y[0], hmax = h[0];
    for (int64_t i = 1; i < n; i++) {
        if (x[i] < xmin) xmin = x[i];
        if (x[i] > xmax) xmax = x[i];
        if (y[i] < ymin) ymin = y[i];
        if (y[i] > ymax) ymax = y[i];
        if (h[i] > hmax) hmax = h[i];
    }
    g->xmin = xmin; g->ymin = ymin; g->lz = lz;
    g->S = 2.0 * hmax * (1.0 + 1e-9);
    g->ncx = (int64_t)floor((xmax - xmin) / g->S) + 1;
    g->ncy = (int64_t)floor((ymax - ymin) / g->S) + 1;
    g->ncz = (int64_t)floor(lz / g->S);
    if (g->ncz < 3) g->ncz = 1;
    g->sz = lz / (double)g->ncz;
    int64_t ncell = g->ncx * g->ncy * g->ncz;
    g->start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    g->items = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t* cid = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!g->start || !g->items || !cid) { free(cid); return -1; }
    for (int64_t i = 0; i < n; i++) {
        int64_t a, b, c;
        cid[i] = cell_of(g, x[i], y[i], z[i], &a, &b, &c);
        g->start[cid[i] + 1]++;
    }
    for (int64_t k = 0; k < ncell; k++) g->start[k + 1] += g->start[k];
    int64_t* fillp = (int64_t*)malloc((size_t)ncell * sizeof(int64_t) + 8);
    memcpy(fillp, g->start, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) g->items[fillp[cid[i]]++] = i;
    free(fillp);
    free(cid);
    return 0;
}

static void grid_free(grid_t* g) { free(g->start); free(g->items); }

static int cmp_i32(const void* a, const void* b)
{
    int32_t u = *(const int32_t*)a, v = *(const int32_t*)b;
    return (u > v) - (u < v);
}

/* Visits the (up to 27) distinct cells around particle i and applies fn. */
static int64_t grid_row(const grid_t* g, int64_t i, const double* x, const double* y, const double* z,
                        const double* h, int32_t* out, int64_t* n_own)
{
    int64_t cx, cy, cz;
    cell_of(g, x[i], y[i], z[i], &cx, &cy, &cz);
    int64_t cnt = 0, own = 0;
    int nzoff = g->ncz >= 3 ? 3 : 1;
    for (int oz = 0; oz < nzoff; oz++) {
        int64_t c3 = g->ncz >= 3 ? ((cz + oz - 1 + g->ncz) % g->ncz) : 0;
        for (int64_t b = cy - 1; b <= cy + 1; b++) {
            if (b < 0 || b >= g->ncy) continue;
            for (int64_t a = cx - 1; a <= cx + 1; a++) {
                if (a < 0 || a >= g->ncx) continue;
                int64_t cell = (c3 * g->ncy + b) * g->ncx + a;
                for (int64_t k = g->start[cell]; k < g->start[cell + 1]; k++) {
                    int64_t j = g->items[k];
                    if (j == i) continue;
                    int f = orc_pair_in(x[i], y[i], z[i], h[i], x[j], y[j], z[j], h[j], g->lz);
                    if (f & 1) {
                        if (out) out[cnt] = (int32_t)j;
                        cnt++;
                    }
                    own += (f >> 1) & 1;
                }
            }
        }
    }
    if (n_own) *n_own = own;
    return cnt;
}

int64_t orc_neighbors_grid(int64_t n, const double* x, const double* y, const double* z,
                           const double* h, double lz, int64_t* off, int32_t* col,
                           int32_t* nown, int64_t cap, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    if (n == 0) { off[0] = 0; return 0; }
    grid_t g;
    if (grid_build(&g, n, x, y, z, h, lz) != 0) return -2;
    if (col == NULL) {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; i++) {
            int64_t own;
            off[i + 1] = grid_row(&g, i, x, y, z, h, NULL, &own);
            nown[i] = (int32_t)own;
        }
        off[0] = 0;
        for (int64_t i = 0; i < n; i++) off[i + 1] += off[i];
        grid_free(&g);
        return off[n];
    }
    if (off[n] > cap) { grid_free(&g); return -1; }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        int64_t len = grid_row(&g, i, x, y, z, h, col + off[i], NULL);
        qsort(col + off[i], (size_t)len, sizeof(int32_t), cmp_i32);
    }
    grid_free(&g);
    return off[n];
}

/* ------------------------------------------------------------------------ */
/* Pair loops visit each unordered pair {i, j} once (j > i in row i) and add  */
/* the contribution to both particles, so pair forces are exactly opposite.  */
/* With nthreads > 1 each thread accumulates into private arrays that are     */
/* summed in thread order afterwards.                                         */
/* ------------------------------------------------------------------------ */
static int nthreads_eff(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* R1: rho_i = m_i W(0, h_i) + sum_{j in N(i)} m_j W(r_ij, h_i) */
void orc_density(int64_t n, const double* x, const double* y, const double* z, const double* m,
                 const double* h, double lz, const int64_t* off, const int32_t* col, double* rho,
                 int nthreads)
{
    int T = nthreads_eff(nthreads);
    double* acc = (double*)calloc((size_t)T * (size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel num_threads(T)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double* a = acc + (size_t)t * (size_t)n;
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; i++) {
            for (int64_t k = off[i]; k < off[i + 1]; k++) {
                int64_t j = col[k];
                if (j <= i) continue;
                double r = sqrt(pair_r2(x[i], y[i], z[i], x[j], y[j], z[j], lz));
                a[i] += m[j] * orc_w(r, h[i]);
                a[j] += m[i] * orc_w(r, h[j]);
            }
        }
    }
    for (int64_t i = 0; i < n; i++) {
        double s = m[i] * orc_w(0.0, h[i]);
        for (int t = 0; t < T; t++) s += acc[(size_t)t * (size_t)n + (size_t)i];
        rho[i] = s;
    }
    free(acc);
}

/* R20 (grad-h, [rosswog2009]):
 *   Omega_i = 1 - (dh_i/drho_i) sum_j m_j dW_ij(h_i)/dh_i,  dh/drho = -h/(3 rho)
 * (h proportional to rho^(-1/3), the relation behind the neighbour-number
 * rule R10); the sum runs over j in N(i) and j = i (the self term
 * dW(0, h)/dh = -3 W(0, h)/h).  rho from orc_density.                       */
void orc_omega(int64_t n, const double* x, const double* y, const double* z, const double* m,
               const double* h, const double* rho, double lz, const int64_t* off, const int32_t* col,
               double* omega, int nthreads)
{
    int T = nthreads_eff(nthreads);
    double* acc = (double*)calloc((size_t)T * (size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel num_threads(T)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double* a = acc + (size_t)t * (size_t)n;
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; i++) {
            for (int64_t k = off[i]; k < off[i + 1]; k++) {
                int64_t j = col[k];
                if (j <= i) continue;
                double r = sqrt(pair_r2(x[i], y[i], z[i], x[j], y[j], z[j], lz));
                a[i] += m[j] * orc_dwdh(r, h[i]);
                a[j] += m[i] * orc_dwdh(r, h[j]);
            }
        }
    }
    for (int64_t i = 0; i < n; i++) {
        double s = m[i] * orc_dwdh(0.0, h[i]);
        for (int t = 0; t < T; t++) s += acc[(size_t)t * (size_t)n + (size_t)i];
        omega[i] = 1.0 + h[i] / (3.0 * rho[i]) * s;
    }
    free(acc);
}

/* R9: ideal gas, P = (gamma - 1) rho u, c = sqrt(gamma P / rho) */
void orc_eos(int64_t n, const double* rho, const double* u, double gamma, double* P, double* c)
{
    for (int64_t i = 0; i < n; i++) {
        P[i] = (gamma - 1.0) * rho[i] * u[i];
        c[i] = sqrt(gamma * P[i] / rho[i]);
    }
}

/* R5: Monaghan artificial viscosity Pi_ij, zero unless the pair approaches.
 * mu = hbar (v_ij . x_ij) / (r^2 + eps hbar^2); Pi = (-alpha cbar mu + beta mu^2)/rhobar */
static double av_pi(double vdotr, double r2, double hi, double hj, double ci, double cj,
                    double rhoi, double rhoj, double alpha, double beta, double eps)
{
    if (!(vdotr < 0.0)) return 0.0;
    double hbar = 0.5 * (hi + hj);
    double cbar = 0.5 * (ci + cj);
    double rhobar = 0.5 * (rhoi + rhoj);
    double mu = hbar * vdotr / (r2 + eps * hbar * hbar);
    return (-alpha * cbar * mu + beta * mu * mu) / rhobar;
}

/* R4-R6.  With Wbar_ij = (W(r,h_i) + W(r,h_j))/2 and A = P/rho^2:
 *   a_i  = - sum_j m_j (A_i + A_j + Pi_ij) grad_i Wbar_ij
 *   du_i =   sum_j m_j (A_i + Pi_ij/2) v_ij . grad_i Wbar_ij
 * R20, when omega != NULL (grad-h form, each side's pressure term with its
 * own kernel, W_i = W(r, h_i), W_j = W(r, h_j)):
 *   a_i  = - sum_j m_j (A_i/Omega_i grad_i W_i + A_j/Omega_j grad_i W_j + Pi_ij grad_i Wbar_ij)
 *   du_i =   sum_j m_j (A_i/Omega_i v_ij . grad_i W_i + Pi_ij/2 v_ij . grad_i Wbar_ij)
 * Optional outputs sa, sdu (may be NULL) are per-particle condition scales:
 *   sa_i  = sum_j m_j |A_i + A_j + Pi_ij| |grad_i Wbar_ij|
 *   sdu_i = sum_j m_j |A_i + Pi_ij/2| |v_ij| |grad_i Wbar_ij|
 * i.e. the sums of the magnitudes of the terms, which bound any rounding error
 * of the sums (used by the tests to scale tolerances).                       */
void orc_momentum_energy(int64_t n, const double* x, const double* y, const double* z,
                         const double* vx, const double* vy, const double* vz, const double* m,
                         const double* h, const double* rho, const double* P, const double* c,
                         double lz, double alpha, double beta, double eps, const int64_t* off,
                         const int32_t* col, const double* omega, double* ax, double* ay, double* az,
                         double* du, double* sa, double* sdu, int nthreads)
{
    int T = nthreads_eff(nthreads);
    const int NF = 6;
    double* acc = (double*)calloc((size_t)T * (size_t)NF * (size_t)(n > 0 ? n : 1), sizeof(double));
#pragma omp parallel num_threads(T)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double* bx = acc + ((size_t)t * NF + 0) * (size_t)n;
        double* by = acc + ((size_t)t * NF + 1) * (size_t)n;
        double* bz = acc + ((size_t)t * NF + 2) * (size_t)n;
        double* bu = acc + ((size_t)t * NF + 3) * (size_t)n;
        double* ba = acc + ((size_t)t * NF + 4) * (size_t)n;
        double* bd = acc + ((size_t)t * NF + 5) * (size_t)n;
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; i++) {
            double Ai = P[i] / (rho[i] * rho[i]);
            for (int64_t k = off[i]; k < off[i + 1]; k++) {
                int64_t j = col[k];
                if (j <= i) continue;
                double Aj = P[j] / (rho[j] * rho[j]);
                double dx = x[i] - x[j];
                double dy = y[i] - y[j];
                double dz = z[i] - z[j];
                if (dz > 0.5 * lz) dz -= lz;
                else if (dz < -0.5 * lz) dz += lz;
                double r2 = (dx * dx + dy * dy) + dz * dz;
                double r = sqrt(r2);
                double vxij = vx[i] - vx[j], vyij = vy[i] - vy[j], vzij = vz[i] - vz[j];
                double vdotr = vxij * dx + vyij * dy + vzij * dz;
                double vn = sqrt(vxij * vxij + vyij * vyij + vzij * vzij);
                if (!omega) {
                    /* grad_i Wbar_ij = -(f(h_i) + f(h_j))/2 * x_ij ; grad_j Wbar_ji = -grad_i Wbar_ij */
                    double f = 0.5 * (orc_gradw_fac(r, h[i]) + orc_gradw_fac(r, h[j]));
                    double gx = -f * dx, gy = -f * dy, gz = -f * dz;
                    double Pi = av_pi(vdotr, r2, h[i], h[j], c[i], c[j], rho[i], rho[j], alpha, beta, eps);
                    double s = Ai + Aj + Pi;
                    /* particle i */
                    bx[i] -= m[j] * s * gx;
                    by[i] -= m[j] * s * gy;
                    bz[i] -= m[j] * s * gz;
                    bu[i] += m[j] * (Ai + 0.5 * Pi) * (vxij * gx + vyij * gy + vzij * gz);
                    /* particle j: grad_j Wbar_ji = -g, v_ji = -v_ij */
                    bx[j] -= m[i] * s * (-gx);
                    by[j] -= m[i] * s * (-gy);
                    bz[j] -= m[i] * s * (-gz);
                    bu[j] += m[i] * (Aj + 0.5 * Pi) * ((-vxij) * (-gx) + (-vyij) * (-gy) + (-vzij) * (-gz));
                    double gn = f * r;
                    ba[i] += m[j] * fabs(s) * gn;
                    ba[j] += m[i] * fabs(s) * gn;
                    bd[i] += m[j] * fabs(Ai + 0.5 * Pi) * vn * gn;
                    bd[j] += m[i] * fabs(Aj + 0.5 * Pi) * vn * gn;
                } else {
                    /* R20: grad_i W(r, h) = -f(h) x_ij for each side's own kernel,
                     * grad_i Wbar_ij = -(f_i + f_j)/2 x_ij; the pair force is a
                     * multiple k of x_ij: a_i -= m_j k x_ij, a_j += m_i k x_ij   */
                    double fi = orc_gradw_fac(r, h[i]), fj = orc_gradw_fac(r, h[j]);
                    double f = 0.5 * (fi + fj);
                    double Pi = av_pi(vdotr, r2, h[i], h[j], c[i], c[j], rho[i], rho[j], alpha, beta, eps);
                    double Bi = Ai / omega[i], Bj = Aj / omega[j];
                    double kf = -(Bi * fi + Bj * fj + Pi * f);
                    double ei = -(Bi * fi + 0.5 * Pi * f);
                    double ej = -(Bj * fj + 0.5 * Pi * f);
                    bx[i] -= m[j] * kf * dx;
                    by[i] -= m[j] * kf * dy;
                    bz[i] -= m[j] * kf * dz;
                    bu[i] += m[j] * ei * vdotr;
                    bx[j] += m[i] * kf * dx;
                    by[j] += m[i] * kf * dy;
                    bz[j] += m[i] * kf * dz;
                    bu[j] += m[i] * ej * vdotr;
                    double sk = (fabs(Bi * fi) + fabs(Bj * fj) + fabs(Pi * f)) * r;
                    ba[i] += m[j] * sk;
                    ba[j] += m[i] * sk;
                    bd[i] += m[j] * (fabs(Bi * fi) + fabs(0.5 * Pi * f)) * r * vn;
                    bd[j] += m[i] * (fabs(Bj * fj) + fabs(0.5 * Pi * f)) * r * vn;
                }
            }
        }
    }
    for (int64_t i = 0; i < n; i++) {
        double sx = 0, sy = 0, sz = 0, su = 0, s1 = 0, s2 = 0;
        for (int t = 0; t < T; t++) {
            sx += acc[((size_t)t * NF + 0) * (size_t)n + (size_t)i];
            sy += acc[((size_t)t * NF + 1) * (size_t)n + (size_t)i];
            sz += acc[((size_t)t * NF + 2) * (size_t)n + (size_t)i];
            su += acc[((size_t)t * NF + 3) * (size_t)n + (size_t)i];
            s1 += acc[((size_t)t * NF + 4) * (size_t)n + (size_t)i];
            s2 += acc[((size_t)t * NF + 5) * (size_t)n + (size_t)i];
        }
        ax[i] = sx; ay[i] = sy; az[i] = sz; du[i] = su;
        if (sa) sa[i] = s1;
        if (sdu) sdu[i] = s2;
    }
    free(acc);
}

/* R7: dt = C * min_i h_i / c_i  (global time-step) */
double orc_courant(int64_t n, const double* h, const double* c, double courant)
{
    double mn = INFINITY;
    for (int64_t i = 0; i < n; i++) {
        double t = h[i] / c[i];
        if (t < mn) mn = t;
    }
    return courant * mn;
}

/* Neumaier compensated sum, used for the conserved quantities. */
typedef struct { double s, c; } ksum_t;
static void ks_add(ksum_t* k, double v)
{
    double t = k->s + v;
    if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
    else k->c += (v - t) + k->s;
    k->s = t;
}

/* out = { M, Px, Py, Pz, Lz, Ekin, Eint } with M = sum m, P = sum m v,
 * Lz = sum m (x v_y - y v_x), Ekin = sum m |v|^2 / 2, Eint = sum m u.       */
void orc_conserved(int64_t n, const double* x, const double* y, const double* vx,
                   const double* vy, const double* vz, const double* m, const double* u,
                   double* out)
{
    ksum_t k[7];
    memset(k, 0, sizeof(k));
    for (int64_t i = 0; i < n; i++) {
        ks_add(&k[0], m[i]);
        ks_add(&k[1], m[i] * vx[i]);
        ks_add(&k[2], m[i] * vy[i]);
        ks_add(&k[3], m[i] * vz[i]);
        ks_add(&k[4], m[i] * (x[i] * vy[i] - y[i] * vx[i]));
        ks_add(&k[5], 0.5 * m[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]));
        ks_add(&k[6], m[i] * u[i]);
    }
    for (int q = 0; q < 7; q++) out[q] = k[q].s + k[q].c;
}

/* ------------------------------------------------------------------------ */
/* One timestep (Sec. 3): neighbours -> density -> EOS -> momentum/energy ->  */
/* Courant dt -> Press/leapfrog positions, Adams-Bashforth energy -> h.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double gamma, n_target, courant, dt_growth, av_alpha, av_beta, av_eps, lz;
    double dt_fixed; /* > 0: use this dt instead of the Courant condition */
    int32_t adapt_h;
    int32_t use_grid; /* 0 brute force, 1 grid, -1 grid when n > 5000 */
    int32_t grad_h;   /* 1: the grad-h momentum and energy form (R20) */
    int32_t pad;
} orc_params;

typedef struct {
    int64_t n;
    double *x, *y, *z, *vx, *vy, *vz, *m, *h, *u, *du_prev;
    double *axp, *ayp, *azp; /* a_{n-1}, the previous step's acceleration */
    /* outputs of the last step (values at t_n, before the update) */
    double *rho, *P, *c, *ax, *ay, *az, *du;
    int32_t* nown;
    int64_t nnz;
    double dt, dt_prev;
    int64_t step;
} orc_state;

/* R8: v_{n+1/2} = v_{n-1/2} + a_n (dt_n + dt_{n-1})/2 (dt_{-1} := 0, v_{-1/2} := v_0);
 *     x_{n+1} = x_n + v_{n+1/2} dt_n, z wrapped into [-lz/2, lz/2);
 *     u_{n+1} = u_n + dt_n [(1 + r/2) du_n - (r/2) du_{n-1}], r = dt_n/dt_{n-1}
 *     (Euler on step 0).
 *     The viscosity and du_n use the time-centred velocity
 *     vhat_n = v_{n-1/2} + a_{n-1} dt_{n-1}/2 (a_{-1} := 0), which is O(dt^2)
 *     accurate at t_n; with v_{n-1/2} itself the energy update would only be
 *     first order.
 * R10: h_i <- h_i (1 + (N_t/n_i)^(1/3)) / 2 with this step's n_i; n_i = 0 doubles h.
 * Returns 0, or -1 on allocation failure.                                   */
int orc_step(const orc_params* prm, orc_state* s, int nthreads)
{
    int64_t n = s->n;
    if (n == 0) { s->step++; return 0; }
    int64_t* off = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!off) return -1;
    int grid = prm->use_grid < 0 ? (n > 5000) : prm->use_grid;
    int64_t nnz;
    if (grid) nnz = orc_neighbors_grid(n, s->x, s->y, s->z, s->h, prm->lz, off, NULL, s->nown, 0, nthreads);
    else nnz = orc_neighbors_brute(n, s->x, s->y, s->z, s->h, prm->lz, off, NULL, s->nown, 0, nthreads);
    if (nnz < 0) { free(off); return -1; }
    int32_t* col = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!col) { free(off); return -1; }
    if (grid) orc_neighbors_grid(n, s->x, s->y, s->z, s->h, prm->lz, off, col, s->nown, nnz, nthreads);
    else orc_neighbors_brute(n, s->x, s->y, s->z, s->h, prm->lz, off, col, s->nown, nnz, nthreads);
    s->nnz = nnz;

    orc_density(n, s->x, s->y, s->z, s->m, s->h, prm->lz, off, col, s->rho, nthreads);
    orc_eos(n, s->rho, s->u, prm->gamma, s->P, s->c);
    double* vh = (double*)malloc((size_t)n * 3 * sizeof(double));
    if (!vh) { free(col); free(off); return -1; }
    double half = s->step > 0 ? 0.5 * s->dt_prev : 0.0;
    for (int64_t i = 0; i < n; i++) {
        vh[i] = s->vx[i] + s->axp[i] * half;
        vh[n + i] = s->vy[i] + s->ayp[i] * half;
        vh[2 * n + i] = s->vz[i] + s->azp[i] * half;
    }
    double* om = NULL;
    if (prm->grad_h) {
        om = (double*)malloc((size_t)n * sizeof(double));
        if (!om) { free(vh); free(col); free(off); return -1; }
        orc_omega(n, s->x, s->y, s->z, s->m, s->h, s->rho, prm->lz, off, col, om, nthreads);
    }
    orc_momentum_energy(n, s->x, s->y, s->z, vh, vh + n, vh + 2 * n, s->m, s->h, s->rho, s->P,
                        s->c, prm->lz, prm->av_alpha, prm->av_beta, prm->av_eps, off, col, om, s->ax,
                        s->ay, s->az, s->du, NULL, NULL, nthreads);
    free(om);
    free(vh);
    free(col);
    free(off);

    double dt;
    if (prm->dt_fixed > 0.0) {
        dt = prm->dt_fixed;
    } else {
        dt = orc_courant(n, s->h, s->c, prm->courant);
        if (s->step > 0 && prm->dt_growth * s->dt_prev < dt) dt = prm->dt_growth * s->dt_prev;
    }
    double dtm1 = s->step > 0 ? s->dt_prev : 0.0;
    double kick = 0.5 * (dt + dtm1);
    double r = s->step > 0 ? dt / s->dt_prev : 0.0;
    for (int64_t i = 0; i < n; i++) {
        s->vx[i] += s->ax[i] * kick;
        s->vy[i] += s->ay[i] * kick;
        s->vz[i] += s->az[i] * kick;
        s->x[i] += s->vx[i] * dt;
        s->y[i] += s->vy[i] * dt;
        s->z[i] += s->vz[i] * dt;
        if (s->z[i] >= 0.5 * prm->lz) s->z[i] -= prm->lz;
        else if (s->z[i] < -0.5 * prm->lz) s->z[i] += prm->lz;
        if (s->step > 0)
            s->u[i] += dt * ((1.0 + 0.5 * r) * s->du[i] - 0.5 * r * s->du_prev[i]);
        else
            s->u[i] += dt * s->du[i];
        s->du_prev[i] = s->du[i];
        s->axp[i] = s->ax[i];
        s->ayp[i] = s->ay[i];
        s->azp[i] = s->az[i];
        if (prm->adapt_h) {
            if (s->nown[i] == 0) s->h[i] *= 2.0;
            else s->h[i] *= 0.5 * (1.0 + cbrt(prm->n_target / (double)s->nown[i]));
        }
    }
    s->dt = dt;
    s->dt_prev = dt;
    s->step++;
    return 0;
}
