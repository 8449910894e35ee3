/*
 * ib_oracle.c -- plain FP64 CPU oracle of the immersed-boundary projection
 * method (Ong & Miura, arXiv 1807.10504).
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the product path.  Written for
 * clarity, not speed: every routine is the definition (or the algorithm's
 * steps in the paper's order) with no blocking, fusion or reordering.  Built
 * with -O3 -ffp-contract=off so that no multiply-add is contracted.  The
 * OpenMP pragmas mark loops whose iterations touch disjoint outputs (cells
 * of one colour, faces, markers); a build with -fopenmp runs them on all host
 * cores for the timed CPU baseline with results identical bit for bit (no
 * sum changes its order); without -fopenmp they are ignored.
 *
 * Parity status: every routine here is pinned by a CPU test against a closed
 * form, an invariant or a brute-force computation (tests/test_oracle_*.py),
 * except the choice of reading where the paper is silent; those readings are
 * listed at the routine that makes them.
 */
#include "ib_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define XF(i, j) ((size_t)(j) * (size_t)(nx + 1) + (size_t)(i))
#define YF(i, j) ((size_t)(j) * (size_t)(nx) + (size_t)(i))
#define CC(i, j) ((size_t)(j) * (size_t)(nx) + (size_t)(i))

/* ------------------------------------------------------------------------ */
/* Section 2.2, Eq. (cherby).  The paper writes phi with a 1/(4 ds) factor and
 * Eq. (delta) with 1/(dx dy); counting both would normalise twice, so phi is
 * taken in grid units: phi(r) = (1 + cos(pi r / 2)) / 4 for |r| < 2.
 * kernel 1 is the 4-point kernel of Peskin (2002), cited in Section 2.2, which
 * also has a zero first moment.                                              */
double or_phi(int kernel, double r)
{
    double a = fabs(r);
    if (a >= 2.0) return 0.0;
    if (kernel == 0) return 0.25 * (1.0 + cos(M_PI * r / 2.0));
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
}

/* Section 3.2, Eq. (new_hea): H(r) = integral of phi from -2 to r (grid units),
 * = 1/2 + r/4 + sin(pi r / 2)/(2 pi).  The printed closed form is garbled and
 * its region-II value 0.409 contradicts the integral; this is the integral. */
double or_heaviside_profile(double r)
{
    if (r <= -2.0) return 0.0;
    if (r >= 2.0) return 1.0;
    return 0.5 + r / 4.0 + sin(M_PI * r / 2.0) / (2.0 * M_PI);
}

/* ------------------------------------------------------------------------ */
/* Section 2.2 Eq. (indicator): psi = psi_1 + (psi_2 - psi_1) I, fluid 1 the
 * ambient (H = 0), fluid 2 the drop (H = 1).  Section 2.1: the face density is
 * the average of the two adjacent cells (arithmetic mean); beta = 1/rho_face;
 * wall faces carry beta = 0 (homogeneous Neumann for p).                     */
void or_coeffs(int nx, int ny, double rho_g, double rho_l, double mu_g,
               double mu_l, const double *H, double *rho, double *mu,
               double *bx, double *by)
{
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            rho[CC(i, j)] = rho_g + (rho_l - rho_g) * H[CC(i, j)];
            mu[CC(i, j)] = mu_g + (mu_l - mu_g) * H[CC(i, j)];
        }
    for (int j = 0; j < ny; j++)
        for (int i = 0; i <= nx; i++)
            bx[XF(i, j)] = (i == 0 || i == nx)
                               ? 0.0
                               : 1.0 / (0.5 * (rho[CC(i - 1, j)] + rho[CC(i, j)]));
    for (int j = 0; j <= ny; j++)
        for (int i = 0; i < nx; i++)
            by[YF(i, j)] = (j == 0 || j == ny)
                               ? 0.0
                               : 1.0 / (0.5 * (rho[CC(i, j - 1)] + rho[CC(i, j)]));
}

/* ------------------------------------------------------------------------ */
/* Section 2.1 Eq. (ps), second-order central differences in flux form:
 * (A p)_ij = [bx_{i+1,j}(p_{i+1,j}-p_ij) - bx_ij(p_ij-p_{i-1,j})
 *           + by_{i,j+1}(p_{i,j+1}-p_ij) - by_ij(p_ij-p_{i,j-1})] / h^2.
 * Wall faces have no outside neighbour and contribute nothing.              */
void or_apply_A(int nx, int ny, double h, const double *bx, const double *by,
                const double *p, double *out)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double c = p[CC(i, j)];
            double s = 0.0;
            if (i + 1 < nx) s += bx[XF(i + 1, j)] * (p[CC(i + 1, j)] - c);
            if (i > 0) s -= bx[XF(i, j)] * (c - p[CC(i - 1, j)]);
            if (j + 1 < ny) s += by[YF(i, j + 1)] * (p[CC(i, j + 1)] - c);
            if (j > 0) s -= by[YF(i, j)] * (c - p[CC(i, j - 1)]);
            out[CC(i, j)] = s / (h * h);
        }
}

void or_residual(int nx, int ny, double h, const double *bx, const double *by,
                 const double *b, const double *p, double *r)
{
    or_apply_A(nx, ny, h, bx, by, p, r);
    #pragma omp parallel for schedule(static)
    for (size_t k = 0; k < (size_t)nx * ny; k++) r[k] = b[k] - r[k];
}

/* Red-black Gauss-Seidel for A p = b: red cells ((i+j) even) first, then
 * black; each cell takes the value that zeroes its own residual,
 * p_ij = (sum_f beta_f p_nb - h^2 b_ij) / sum_f beta_f.                      */
void or_rbgs(int nx, int ny, double h, const double *bx, const double *by,
             const double *b, double *p, int nsweeps)
{
    for (int s = 0; s < nsweeps; s++)
        for (int color = 0; color < 2; color++)
            #pragma omp parallel for schedule(static)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    if (((i + j) & 1) != color) continue;
                    double num = 0.0, den = 0.0;
                    if (i + 1 < nx) { num += bx[XF(i + 1, j)] * p[CC(i + 1, j)]; den += bx[XF(i + 1, j)]; }
                    if (i > 0)      { num += bx[XF(i, j)] * p[CC(i - 1, j)];     den += bx[XF(i, j)]; }
                    if (j + 1 < ny) { num += by[YF(i, j + 1)] * p[CC(i, j + 1)]; den += by[YF(i, j + 1)]; }
                    if (j > 0)      { num += by[YF(i, j)] * p[CC(i, j - 1)];     den += by[YF(i, j)]; }
                    if (den != 0.0) p[CC(i, j)] = (num - h * h * b[CC(i, j)]) / den;
                }
}

/* Cell-centred restriction: average of the four children.                  */
void or_restrict(int nx, int ny, const double *r, double *rc)
{
    int nxc = nx / 2, nyc = ny / 2;
    #pragma omp parallel for schedule(static)
    for (int J = 0; J < nyc; J++)
        for (int I = 0; I < nxc; I++)
            rc[(size_t)J * nxc + I] =
                0.25 * (r[CC(2 * I, 2 * J)] + r[CC(2 * I + 1, 2 * J)] +
                        r[CC(2 * I, 2 * J + 1)] + r[CC(2 * I + 1, 2 * J + 1)]);
}

/* Coarse face coefficient = mean of the two fine faces that make it up.     */
void or_coarsen_beta(int nx, int ny, const double *bx, const double *by,
                     double *bxc, double *byc)
{
    int nxc = nx / 2, nyc = ny / 2;
    for (int J = 0; J < nyc; J++)
        for (int I = 0; I <= nxc; I++)
            bxc[(size_t)J * (nxc + 1) + I] =
                0.5 * (bx[XF(2 * I, 2 * J)] + bx[XF(2 * I, 2 * J + 1)]);
    for (int J = 0; J <= nyc; J++)
        for (int I = 0; I < nxc; I++)
            byc[(size_t)J * nxc + I] =
                0.5 * (by[YF(2 * I, 2 * J)] + by[YF(2 * I + 1, 2 * J)]);
}

/* Cell-centred bilinear prolongation (weights 9, 3, 3, 1 over 16), added to
 * the fine iterate.  Outside the coarse grid the nearest coarse value is used
 * (zero normal gradient at the walls).                                       */
void or_prolong_add(int nxc, int nyc, const double *ec, double *ef)
{
    int nx = 2 * nxc, ny = 2 * nyc;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int I = i / 2, J = j / 2;
            int I2 = I + ((i & 1) ? 1 : -1), J2 = J + ((j & 1) ? 1 : -1);
            if (I2 < 0) I2 = 0;
            if (I2 > nxc - 1) I2 = nxc - 1;
            if (J2 < 0) J2 = 0;
            if (J2 > nyc - 1) J2 = nyc - 1;
            double c00 = ec[(size_t)J * nxc + I], c10 = ec[(size_t)J * nxc + I2];
            double c01 = ec[(size_t)J2 * nxc + I], c11 = ec[(size_t)J2 * nxc + I2];
            ef[CC(i, j)] += (9.0 * c00 + 3.0 * c10 + 3.0 * c01 + c11) / 16.0;
        }
}

/* Levels halve both sides while both are even and the level has more than
 * 16 cells.                                                                 */
int or_mg_levels(int nx, int ny, int *nxs, int *nys, int maxlev)
{
    int L = 0;
    nxs[L] = nx; nys[L] = ny; L++;
    while (L < maxlev && nx % 2 == 0 && ny % 2 == 0 && nx * ny > 16) {
        nx /= 2; ny /= 2;
        nxs[L] = nx; nys[L] = ny; L++;
    }
    return L;
}

/* Dense matrix of A (column k = A e_k) plus s * 1 1^T with s = A_00, which
 * removes the constant null space: A' e = r gives A e = r - mean(r).        */
static double *dense_matrix(int nx, int ny, double h, const double *bx,
                            const double *by)
{
    int n = nx * ny;
    double *M = (double *)calloc((size_t)n * n, sizeof(double));
    double *ek = (double *)calloc((size_t)n, sizeof(double));
    double *col = (double *)calloc((size_t)n, sizeof(double));
    for (int k = 0; k < n; k++) {
        ek[k] = 1.0;
        or_apply_A(nx, ny, h, bx, by, ek, col);
        ek[k] = 0.0;
        for (int r = 0; r < n; r++) M[(size_t)r * n + k] = col[r];
    }
    double s = M[0];
    for (size_t k = 0; k < (size_t)n * n; k++) M[k] += s;
    free(ek); free(col);
    return M;
}

/* Gaussian elimination with partial pivoting; x = M^{-1} b; M destroyed.  */
static int gauss_solve(int n, double *M, const double *b, double *x)
{
    double *rhs = (double *)malloc((size_t)n * sizeof(double));
    memcpy(rhs, b, (size_t)n * sizeof(double));
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(M[(size_t)r * n + c]) > fabs(M[(size_t)piv * n + c])) piv = r;
        if (M[(size_t)piv * n + c] == 0.0) { free(rhs); return -1; }
        if (piv != c) {
            for (int k = 0; k < n; k++) {
                double t = M[(size_t)c * n + k];
                M[(size_t)c * n + k] = M[(size_t)piv * n + k];
                M[(size_t)piv * n + k] = t;
            }
            double t = rhs[c]; rhs[c] = rhs[piv]; rhs[piv] = t;
        }
        for (int r = c + 1; r < n; r++) {
            double f = M[(size_t)r * n + c] / M[(size_t)c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; k++) M[(size_t)r * n + k] -= f * M[(size_t)c * n + k];
            rhs[r] -= f * rhs[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = rhs[r];
        for (int k = r + 1; k < n; k++) s -= M[(size_t)r * n + k] * x[k];
        x[r] = s / M[(size_t)r * n + r];
    }
    free(rhs);
    return 0;
}

static double mean_of(size_t n, const double *a)
{
    double s = 0.0;
    for (size_t k = 0; k < n; k++) s += a[k];
    return s / (double)n;
}

static double norm2_of(size_t n, const double *a)
{
    double s = 0.0;
    for (size_t k = 0; k < n; k++) s += a[k] * a[k];
    return sqrt(s);
}

/* Exact solution of A p = b - mean(b) with mean(p) = 0, by a dense solve.   */
int or_dense_solve(int nx, int ny, double h, const double *bx,
                   const double *by, const double *b, double *p)
{
    size_t n = (size_t)nx * ny;
    double *M = dense_matrix(nx, ny, h, bx, by);
    double *b0 = (double *)malloc(n * sizeof(double));
    double mb = mean_of(n, b);
    for (size_t k = 0; k < n; k++) b0[k] = b[k] - mb;
    int st = gauss_solve((int)n, M, b0, p);
    double mp = mean_of(n, p);
    for (size_t k = 0; k < n; k++) p[k] -= mp;
    free(M); free(b0);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Multigrid (Section 2.1 names multigrid and nothing more; this is the
 * V(nu1,nu2) cycle with the smoother, transfers and coarse solve above).    */
typedef struct {
    int nx, ny;
    double h;
    double *bx, *by, *e, *r, *t;
    float *bxf, *byf, *ef, *rf, *tf;
} olev;

static void coarse_solve_d(olev *L)
{
    int n = L->nx * L->ny;
    double *M = dense_matrix(L->nx, L->ny, L->h, L->bx, L->by);
    gauss_solve(n, M, L->r, L->e);
    free(M);
}

static void vcycle_d(olev *L, int l, int nl, int nu1, int nu2)
{
    if (l == nl - 1) { coarse_solve_d(&L[l]); return; }
    olev *f = &L[l], *c = &L[l + 1];
    or_rbgs(f->nx, f->ny, f->h, f->bx, f->by, f->r, f->e, nu1);
    or_residual(f->nx, f->ny, f->h, f->bx, f->by, f->r, f->e, f->t);
    or_restrict(f->nx, f->ny, f->t, c->r);
    memset(c->e, 0, (size_t)c->nx * c->ny * sizeof(double));
    vcycle_d(L, l + 1, nl, nu1, nu2);
    or_prolong_add(c->nx, c->ny, c->e, f->e);
    or_rbgs(f->nx, f->ny, f->h, f->bx, f->by, f->r, f->e, nu2);
}

/* FP32 copies of the same steps, for the mixed-precision inner cycle.       */
static void apply_A_f(int nx, int ny, float h, const float *bx, const float *by,
                      const float *p, float *out)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            float c = p[CC(i, j)];
            float s = 0.0f;
            if (i + 1 < nx) s += bx[XF(i + 1, j)] * (p[CC(i + 1, j)] - c);
            if (i > 0) s -= bx[XF(i, j)] * (c - p[CC(i - 1, j)]);
            if (j + 1 < ny) s += by[YF(i, j + 1)] * (p[CC(i, j + 1)] - c);
            if (j > 0) s -= by[YF(i, j)] * (c - p[CC(i, j - 1)]);
            out[CC(i, j)] = s / (h * h);
        }
}

static void rbgs_f(int nx, int ny, float h, const float *bx, const float *by,
                   const float *b, float *p, int nsweeps)
{
    for (int s = 0; s < nsweeps; s++)
        for (int color = 0; color < 2; color++)
            #pragma omp parallel for schedule(static)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    if (((i + j) & 1) != color) continue;
                    float num = 0.0f, den = 0.0f;
                    if (i + 1 < nx) { num += bx[XF(i + 1, j)] * p[CC(i + 1, j)]; den += bx[XF(i + 1, j)]; }
                    if (i > 0)      { num += bx[XF(i, j)] * p[CC(i - 1, j)];     den += bx[XF(i, j)]; }
                    if (j + 1 < ny) { num += by[YF(i, j + 1)] * p[CC(i, j + 1)]; den += by[YF(i, j + 1)]; }
                    if (j > 0)      { num += by[YF(i, j)] * p[CC(i, j - 1)];     den += by[YF(i, j)]; }
                    if (den != 0.0f) p[CC(i, j)] = (num - h * h * b[CC(i, j)]) / den;
                }
}

static void coarse_solve_f(olev *L)
{
    /* The FP32 cycle's coarsest solve stays FP64 (it is tiny and its
     * stability needs it): FP64 matrix, FP32 right-hand side and result.    */
    int n = L->nx * L->ny;
    double *M = dense_matrix(L->nx, L->ny, L->h, L->bx, L->by);
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *e = (double *)malloc((size_t)n * sizeof(double));
    for (int k = 0; k < n; k++) r[k] = (double)L->rf[k];
    gauss_solve(n, M, r, e);
    for (int k = 0; k < n; k++) L->ef[k] = (float)e[k];
    free(M); free(r); free(e);
}

static void vcycle_f(olev *L, int l, int nl, int nu1, int nu2)
{
    if (l == nl - 1) { coarse_solve_f(&L[l]); return; }
    olev *f = &L[l], *c = &L[l + 1];
    int nx = f->nx, ny = f->ny;
    float h = (float)f->h;
    rbgs_f(nx, ny, h, f->bxf, f->byf, f->rf, f->ef, nu1);
    apply_A_f(nx, ny, h, f->bxf, f->byf, f->ef, f->tf);
    #pragma omp parallel for schedule(static)
    for (size_t k = 0; k < (size_t)nx * ny; k++) f->tf[k] = f->rf[k] - f->tf[k];
    #pragma omp parallel for schedule(static)
    for (int J = 0; J < c->ny; J++)
        for (int I = 0; I < c->nx; I++)
            c->rf[(size_t)J * c->nx + I] =
                0.25f * (f->tf[CC(2 * I, 2 * J)] + f->tf[CC(2 * I + 1, 2 * J)] +
                         f->tf[CC(2 * I, 2 * J + 1)] + f->tf[CC(2 * I + 1, 2 * J + 1)]);
    memset(c->ef, 0, (size_t)c->nx * c->ny * sizeof(float));
    vcycle_f(L, l + 1, nl, nu1, nu2);
    int nxc = c->nx, nyc = c->ny;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int I = i / 2, J = j / 2;
            int I2 = I + ((i & 1) ? 1 : -1), J2 = J + ((j & 1) ? 1 : -1);
            if (I2 < 0) I2 = 0;
            if (I2 > nxc - 1) I2 = nxc - 1;
            if (J2 < 0) J2 = 0;
            if (J2 > nyc - 1) J2 = nyc - 1;
            float c00 = c->ef[(size_t)J * nxc + I], c10 = c->ef[(size_t)J * nxc + I2];
            float c01 = c->ef[(size_t)J2 * nxc + I], c11 = c->ef[(size_t)J2 * nxc + I2];
            f->ef[CC(i, j)] += (9.0f * c00 + 3.0f * c10 + 3.0f * c01 + c11) / 16.0f;
        }
    rbgs_f(nx, ny, h, f->bxf, f->byf, f->rf, f->ef, nu2);
}

/* Solve A p = b - mean(b) to ||b0 - A p||_2 <= tol ||b0||_2, then remove the
 * mean of p.  precision 0: FP64 V-cycles on p.  precision 1: FP64 defect
 * correction, p += V32(b0 - A p), with the inner cycle in FP32.  precision 2:
 * the same with two FP32 V-cycles on the defect equation per FP64 residual
 * (the second starts from the first's correction).  *cycles counts V-cycles
 * (FP32 ones in the mixed modes); the cap is tested before each outer step,
 * so it may be passed by one; hist (max_cycles + 2 entries) gets the relative
 * residual after each cycle, NaN where none is formed.
 * Returns 0 converged, 3 cycle cap reached, 4 non-finite residual.          */
int or_mg_solve(int nx, int ny, double h, const double *bx, const double *by,
                const double *b, double *p, int precision, double tol,
                int max_cycles, int nu1, int nu2, int *cycles, double *relres,
                double *hist)
{
    int nxs[32], nys[32];
    int nl = or_mg_levels(nx, ny, nxs, nys, 32);
    olev L[32];
    size_t n0 = (size_t)nx * ny;
    for (int l = 0; l < nl; l++) {
        size_t n = (size_t)nxs[l] * nys[l];
        L[l].nx = nxs[l]; L[l].ny = nys[l];
        L[l].h = l == 0 ? h : 2.0 * L[l - 1].h;
        L[l].bx = (double *)malloc((size_t)(nxs[l] + 1) * nys[l] * sizeof(double));
        L[l].by = (double *)malloc((size_t)nxs[l] * (nys[l] + 1) * sizeof(double));
        L[l].e = (double *)calloc(n, sizeof(double));
        L[l].r = (double *)calloc(n, sizeof(double));
        L[l].t = (double *)calloc(n, sizeof(double));
        L[l].bxf = (float *)malloc((size_t)(nxs[l] + 1) * nys[l] * sizeof(float));
        L[l].byf = (float *)malloc((size_t)nxs[l] * (nys[l] + 1) * sizeof(float));
        L[l].ef = (float *)calloc(n, sizeof(float));
        L[l].rf = (float *)calloc(n, sizeof(float));
        L[l].tf = (float *)calloc(n, sizeof(float));
        if (l == 0) {
            memcpy(L[l].bx, bx, (size_t)(nx + 1) * ny * sizeof(double));
            memcpy(L[l].by, by, (size_t)nx * (ny + 1) * sizeof(double));
        } else {
            or_coarsen_beta(nxs[l - 1], nys[l - 1], L[l - 1].bx, L[l - 1].by,
                            L[l].bx, L[l].by);
        }
        for (size_t k = 0; k < (size_t)(nxs[l] + 1) * nys[l]; k++) L[l].bxf[k] = (float)L[l].bx[k];
        for (size_t k = 0; k < (size_t)nxs[l] * (nys[l] + 1); k++) L[l].byf[k] = (float)L[l].by[k];
    }
    double *b0 = (double *)malloc(n0 * sizeof(double));
    double *res = (double *)malloc(n0 * sizeof(double));
    double mb = mean_of(n0, b);
    for (size_t k = 0; k < n0; k++) b0[k] = b[k] - mb;
    double nb = norm2_of(n0, b0);
    int c = 0, status = 0;
    double rr = 0.0;
    if (nb == 0.0) {
        memset(p, 0, n0 * sizeof(double));
    } else {
        or_residual(nx, ny, h, bx, by, b0, p, res);
        rr = norm2_of(n0, res) / nb;
        if (hist) hist[0] = rr;
        while (rr > tol && c < max_cycles && isfinite(rr)) {
            if (precision == 0) {
                memcpy(L[0].e, p, n0 * sizeof(double));
                memcpy(L[0].r, b0, n0 * sizeof(double));
                vcycle_d(L, 0, nl, nu1, nu2);
                memcpy(p, L[0].e, n0 * sizeof(double));
            } else {
                int inner = precision == 2 ? 2 : 1;
                for (size_t k = 0; k < n0; k++) { L[0].rf[k] = (float)res[k]; L[0].ef[k] = 0.0f; }
                for (int q = 0; q < inner; q++) vcycle_f(L, 0, nl, nu1, nu2);
                for (size_t k = 0; k < n0; k++) p[k] += (double)L[0].ef[k];
                c += inner - 1;
            }
            c++;
            or_residual(nx, ny, h, bx, by, b0, p, res);
            rr = norm2_of(n0, res) / nb;
            if (hist) {
                if (precision == 2) hist[c - 1] = NAN;  /* no residual between inner cycles */
                hist[c] = rr;
            }
        }
        double mp = mean_of(n0, p);
        for (size_t k = 0; k < n0; k++) p[k] -= mp;
        if (!isfinite(rr)) status = 4;
        else if (rr > tol) status = 3;
    }
    if (cycles) *cycles = c;
    if (relres) *relres = rr;
    for (int l = 0; l < nl; l++) {
        free(L[l].bx); free(L[l].by); free(L[l].e); free(L[l].r); free(L[l].t);
        free(L[l].bxf); free(L[l].byf); free(L[l].ef); free(L[l].rf); free(L[l].tf);
    }
    free(b0); free(res);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Section 2.1 Eq. (ps) with the force moved into the projection (Section 3.2,
 * Eq. (ns2_new)): u^{n+1} = u* + dt beta (-grad p + F), so div u^{n+1} = 0
 * requires div(beta grad p) = div(u*)/dt + div(beta F).                     */
void or_rhs(int nx, int ny, double h, double dt, const double *us,
            const double *vs, const double *Fx, const double *Fy,
            const double *bx, const double *by, double *b)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double divu = (us[XF(i + 1, j)] - us[XF(i, j)] + vs[YF(i, j + 1)] - vs[YF(i, j)]) / h;
            double divf = (bx[XF(i + 1, j)] * Fx[XF(i + 1, j)] - bx[XF(i, j)] * Fx[XF(i, j)] +
                           by[YF(i, j + 1)] * Fy[YF(i, j + 1)] - by[YF(i, j)] * Fy[YF(i, j)]) / h;
            b[CC(i, j)] = divu / dt + divf;
        }
}

void or_correct(int nx, int ny, double h, double dt, const double *us,
                const double *vs, const double *p, const double *Fx,
                const double *Fy, const double *bx, const double *by,
                double *u, double *v)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i <= nx; i++) {
            if (i == 0 || i == nx) { u[XF(i, j)] = 0.0; continue; }
            double gp = (p[CC(i, j)] - p[CC(i - 1, j)]) / h;
            u[XF(i, j)] = us[XF(i, j)] + dt * (bx[XF(i, j)] * (Fx[XF(i, j)] - gp));
        }
    #pragma omp parallel for schedule(static)
    for (int j = 0; j <= ny; j++)
        for (int i = 0; i < nx; i++) {
            if (j == 0 || j == ny) { v[YF(i, j)] = 0.0; continue; }
            double gp = (p[CC(i, j)] - p[CC(i, j - 1)]) / h;
            v[YF(i, j)] = vs[YF(i, j)] + dt * (by[YF(i, j)] * (Fy[YF(i, j)] - gp));
        }
}

void or_divergence(int nx, int ny, double h, const double *u, const double *v,
                   double *div)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++)
            div[CC(i, j)] = (u[XF(i + 1, j)] - u[XF(i, j)] + v[YF(i, j + 1)] - v[YF(i, j)]) / h;
}

/* ------------------------------------------------------------------------ */
/* Section 2.1, Eqs. (ad_bf) and (cr_ni) on the u- and v-control volumes,
 * divided by the control-volume area h^2:
 *   rho (u* - u)/dt = -(3/2 A^n - 1/2 A^{n-1}) + D^n   (Euler when no A^{n-1})
 * A = flux-form advection with cell densities on the normal faces and node
 * (four-cell) averages on the tangential faces; D = div(mu grad u) with cell
 * viscosities on the normal faces and node averages on the tangential faces;
 * no-slip walls by a reflected ghost value.  The viscous term is explicit
 * (the Crank-Nicolson variant is not part of this path).  rho on the face is
 * the two-cell average.  gx, gy is a uniform body acceleration.              */
void or_predictor(int nx, int ny, double h, double dt, const double *rho,
                  const double *mu, const double *u, const double *v,
                  const double *au_prev, const double *av_prev, int have_prev,
                  double gx, double gy, double *us, double *vs, double *au,
                  double *av)
{
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i <= nx; i++) {
            size_t k = XF(i, j);
            if (i == 0 || i == nx) { us[k] = 0.0; au[k] = 0.0; continue; }
            double uc = u[k], uE = u[XF(i + 1, j)], uW = u[XF(i - 1, j)];
            double uN = (j + 1 < ny) ? u[XF(i, j + 1)] : -uc;
            double uS = (j > 0) ? u[XF(i, j - 1)] : -uc;
            double aE = 0.5 * (uE + uc), aW = 0.5 * (uc + uW);
            double fE = rho[CC(i, j)] * aE * aE;
            double fW = rho[CC(i - 1, j)] * aW * aW;
            double gN = 0.0, gS = 0.0, muN, muS;
            if (j + 1 < ny) {
                double rN = 0.25 * (rho[CC(i - 1, j)] + rho[CC(i, j)] + rho[CC(i - 1, j + 1)] + rho[CC(i, j + 1)]);
                double vN = 0.5 * (v[YF(i - 1, j + 1)] + v[YF(i, j + 1)]);
                gN = rN * vN * (0.5 * (uc + uN));
                muN = 0.25 * (mu[CC(i - 1, j)] + mu[CC(i, j)] + mu[CC(i - 1, j + 1)] + mu[CC(i, j + 1)]);
            } else {
                muN = 0.5 * (mu[CC(i - 1, j)] + mu[CC(i, j)]);
            }
            if (j > 0) {
                double rS = 0.25 * (rho[CC(i - 1, j - 1)] + rho[CC(i, j - 1)] + rho[CC(i - 1, j)] + rho[CC(i, j)]);
                double vS = 0.5 * (v[YF(i - 1, j)] + v[YF(i, j)]);
                gS = rS * vS * (0.5 * (uc + uS));
                muS = 0.25 * (mu[CC(i - 1, j - 1)] + mu[CC(i, j - 1)] + mu[CC(i - 1, j)] + mu[CC(i, j)]);
            } else {
                muS = 0.5 * (mu[CC(i - 1, j)] + mu[CC(i, j)]);
            }
            double adv = (fE - fW) / h + (gN - gS) / h;
            double vis = (mu[CC(i, j)] * (uE - uc) - mu[CC(i - 1, j)] * (uc - uW) +
                          muN * (uN - uc) - muS * (uc - uS)) / (h * h);
            double rf = 0.5 * (rho[CC(i - 1, j)] + rho[CC(i, j)]);
            double ae = have_prev ? 1.5 * adv - 0.5 * au_prev[k] : adv;
            us[k] = uc + dt * ((vis - ae) / rf + gx);
            au[k] = adv;
        }
    #pragma omp parallel for schedule(static)
    for (int j = 0; j <= ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t k = YF(i, j);
            if (j == 0 || j == ny) { vs[k] = 0.0; av[k] = 0.0; continue; }
            double vc = v[k], vN = v[YF(i, j + 1)], vS = v[YF(i, j - 1)];
            double vE = (i + 1 < nx) ? v[YF(i + 1, j)] : -vc;
            double vW = (i > 0) ? v[YF(i - 1, j)] : -vc;
            double aN = 0.5 * (vN + vc), aS = 0.5 * (vc + vS);
            double fN = rho[CC(i, j)] * aN * aN;
            double fS = rho[CC(i, j - 1)] * aS * aS;
            double gE = 0.0, gW = 0.0, muE, muW;
            if (i + 1 < nx) {
                double rE = 0.25 * (rho[CC(i, j - 1)] + rho[CC(i + 1, j - 1)] + rho[CC(i, j)] + rho[CC(i + 1, j)]);
                double uE = 0.5 * (u[XF(i + 1, j - 1)] + u[XF(i + 1, j)]);
                gE = rE * uE * (0.5 * (vc + vE));
                muE = 0.25 * (mu[CC(i, j - 1)] + mu[CC(i + 1, j - 1)] + mu[CC(i, j)] + mu[CC(i + 1, j)]);
            } else {
                muE = 0.5 * (mu[CC(i, j - 1)] + mu[CC(i, j)]);
            }
            if (i > 0) {
                double rW = 0.25 * (rho[CC(i - 1, j - 1)] + rho[CC(i, j - 1)] + rho[CC(i - 1, j)] + rho[CC(i, j)]);
                double uW = 0.5 * (u[XF(i, j - 1)] + u[XF(i, j)]);
                gW = rW * uW * (0.5 * (vc + vW));
                muW = 0.25 * (mu[CC(i - 1, j - 1)] + mu[CC(i, j - 1)] + mu[CC(i - 1, j)] + mu[CC(i, j)]);
            } else {
                muW = 0.5 * (mu[CC(i, j - 1)] + mu[CC(i, j)]);
            }
            double adv = (fN - fS) / h + (gE - gW) / h;
            double vis = (mu[CC(i, j)] * (vN - vc) - mu[CC(i, j - 1)] * (vc - vS) +
                          muE * (vE - vc) - muW * (vc - vW)) / (h * h);
            double rf = 0.5 * (rho[CC(i, j - 1)] + rho[CC(i, j)]);
            double ae = have_prev ? 1.5 * adv - 0.5 * av_prev[k] : adv;
            vs[k] = vc + dt * ((vis - ae) / rf + gy);
            av[k] = adv;
        }
}

/* ------------------------------------------------------------------------ */
/* Marker-to-cell key: floor((Y-y0)/h) * nx + floor((X-x0)/h), clamped.      */
void or_cell_keys(int M, const double *X, const double *Y, double x0,
                  double y0, double h, int nx, int ny, uint32_t *key)
{
    for (int m = 0; m < M; m++) {
        int kx = (int)floor((X[m] - x0) / h);
        int ky = (int)floor((Y[m] - y0) / h);
        if (kx < 0) kx = 0;
        if (kx > nx - 1) kx = nx - 1;
        if (ky < 0) ky = 0;
        if (ky > ny - 1) ky = ny - 1;
        key[m] = (uint32_t)ky * (uint32_t)nx + (uint32_t)kx;
    }
}

static const uint32_t *sort_keys_ptr;
static int cmp_key_id(const void *a, const void *b)
{
    uint32_t ia = *(const uint32_t *)a, ib = *(const uint32_t *)b;
    uint32_t ka = sort_keys_ptr[ia], kb = sort_keys_ptr[ib];
    if (ka != kb) return ka < kb ? -1 : 1;
    return ia < ib ? -1 : (ia > ib ? 1 : 0);
}

/* Marker ids ordered by (key, id).                                          */
void or_marker_sort(int M, const uint32_t *key, uint32_t *order)
{
    for (int m = 0; m < M; m++) order[m] = (uint32_t)m;
    sort_keys_ptr = key;
    qsort(order, (size_t)M, sizeof(uint32_t), cmp_key_id);
}

/* ------------------------------------------------------------------------ */
/* Section 2.2 Eq. (jump_condu): U(X) = sum_faces u phi(rx) phi(ry), where
 * (rx, ry) is the face position minus the marker position in grid units;
 * the dx dy of the sum cancels the 1/(dx dy) of Eq. (delta).  Faces outside
 * the arrays contribute nothing.                                             */
void or_interp(int kernel, int nx, int ny, double h, double x0, double y0,
               const double *u, const double *v, int M, const double *X,
               const double *Y, double *U, double *V)
{
    #pragma omp parallel for schedule(static)
    for (int m = 0; m < M; m++) {
        double sx = (X[m] - x0) / h, sy = (Y[m] - y0) / h - 0.5;
        int i0 = (int)floor(sx) - 1, j0 = (int)floor(sy) - 1;
        double acc = 0.0;
        for (int b = 0; b < 4; b++)
            for (int a = 0; a < 4; a++) {
                int i = i0 + a, j = j0 + b;
                if (i < 0 || i > nx || j < 0 || j > ny - 1) continue;
                acc += u[XF(i, j)] * (or_phi(kernel, (double)i - sx) * or_phi(kernel, (double)j - sy));
            }
        U[m] = acc;
        sx = (X[m] - x0) / h - 0.5; sy = (Y[m] - y0) / h;
        i0 = (int)floor(sx) - 1; j0 = (int)floor(sy) - 1;
        acc = 0.0;
        for (int b = 0; b < 4; b++)
            for (int a = 0; a < 4; a++) {
                int i = i0 + a, j = j0 + b;
                if (i < 0 || i > nx - 1 || j < 0 || j > ny) continue;
                acc += v[YF(i, j)] * (or_phi(kernel, (double)i - sx) * or_phi(kernel, (double)j - sy));
            }
        V[m] = acc;
    }
}

/* Section 3.1 Eq. (delta_vec): F(x) = sum_m f_m delta(x - X_m) ds_m with
 * f_m = fmag_m n_m, delta = phi phi / h^2.  Summed in ascending marker id.
 * Wall faces are left at zero.                                               */
void or_spread_conv(int kernel, int nx, int ny, double h, double x0,
                    double y0, int M, const double *X, const double *Y,
                    const double *fmag, const double *nxm, const double *nym,
                    const double *ds, double *Fx, double *Fy)
{
    memset(Fx, 0, (size_t)(nx + 1) * ny * sizeof(double));
    memset(Fy, 0, (size_t)nx * (ny + 1) * sizeof(double));
    double ih2 = 1.0 / (h * h);
    for (int m = 0; m < M; m++) {
        double cx = fmag[m] * nxm[m] * ds[m] * ih2;
        double cy = fmag[m] * nym[m] * ds[m] * ih2;
        double sx = (X[m] - x0) / h, sy = (Y[m] - y0) / h - 0.5;
        int i0 = (int)floor(sx) - 1, j0 = (int)floor(sy) - 1;
        for (int b = 0; b < 4; b++)
            for (int a = 0; a < 4; a++) {
                int i = i0 + a, j = j0 + b;
                if (i < 1 || i > nx - 1 || j < 0 || j > ny - 1) continue;
                Fx[XF(i, j)] += cx * (or_phi(kernel, (double)i - sx) * or_phi(kernel, (double)j - sy));
            }
        sx = (X[m] - x0) / h - 0.5; sy = (Y[m] - y0) / h;
        i0 = (int)floor(sx) - 1; j0 = (int)floor(sy) - 1;
        for (int b = 0; b < 4; b++)
            for (int a = 0; a < 4; a++) {
                int i = i0 + a, j = j0 + b;
                if (i < 0 || i > nx - 1 || j < 1 || j > ny - 1) continue;
                Fy[YF(i, j)] += cy * (or_phi(kernel, (double)i - sx) * or_phi(kernel, (double)j - sy));
            }
    }
}

/* ------------------------------------------------------------------------ */
/* Predecessor and successor of every marker along its closed polyline.     */
static void links(int M, int ndrops, const int32_t *ds_, int *prev, int *next)
{
    for (int d = 0; d < ndrops; d++) {
        int s = ds_[d], e = ds_[d + 1];
        for (int m = s; m < e; m++) {
            prev[m] = (m == s) ? e - 1 : m - 1;
            next[m] = (m == e - 1) ? s : m + 1;
        }
    }
    (void)M;
}

/* Section 4 Eq. (ten_f): curvature = change of the unit tangent over the
 * local arc length.  Tangents are those of the two segments meeting at the
 * marker, ds_m = (|X_m - X_{m-1}| + |X_{m+1} - X_m|)/2, and the sign is that
 * of the turn (positive for a convex drop traversed counter-clockwise; the
 * printed formula is unsigned).  The inward normal at a marker is the unit
 * bisector of the two segments' left normals.                               */
void or_curvature(int M, const double *X, const double *Y, int ndrops,
                  const int32_t *drop_start, double *kappa, double *nxm,
                  double *nym, double *ds)
{
    int *prv = (int *)malloc((size_t)M * sizeof(int)), *nxt = (int *)malloc((size_t)M * sizeof(int));
    links(M, ndrops, drop_start, prv, nxt);
    for (int m = 0; m < M; m++) {
        int pm = prv[m], nm = nxt[m];
        double ax = X[m] - X[pm], ay = Y[m] - Y[pm];
        double bx = X[nm] - X[m], by = Y[nm] - Y[m];
        double la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
        double tax = ax / la, tay = ay / la, tbx = bx / lb, tby = by / lb;
        double dsm = 0.5 * (la + lb);
        double dx = tbx - tax, dy = tby - tay;
        double cr = tax * tby - tay * tbx;
        double k = sqrt(dx * dx + dy * dy) / dsm;
        kappa[m] = cr >= 0.0 ? k : -k;
        double nx_ = -tay - tby, ny_ = tax + tbx;
        double ln = sqrt(nx_ * nx_ + ny_ * ny_);
        nxm[m] = nx_ / ln;
        nym[m] = ny_ / ln;
        ds[m] = dsm;
    }
    free(prv); free(nxt);
}

/* ------------------------------------------------------------------------ */
/* Crossing-number test of a point against every segment of every drop.      */
static int inside_point(double px, double py, int M, const double *X,
                        const double *Y, const int *nxt)
{
    int cnt = 0;
    for (int m = 0; m < M; m++) {
        int nm = nxt[m];
        double ax = X[m], ay = Y[m], bx = X[nm], by = Y[nm];
        if ((ay > py) != (by > py)) {
            double xc = ax + (py - ay) * (bx - ax) / (by - ay);
            if (xc > px) cnt++;
        }
    }
    return cnt & 1;
}

double or_inside_cell(int i, int j, double h, double x0, double y0, int M,
                      const double *X, const double *Y, int ndrops,
                      const int32_t *drop_start)
{
    int *prv = (int *)malloc((size_t)M * sizeof(int)), *nxt = (int *)malloc((size_t)M * sizeof(int));
    links(M, ndrops, drop_start, prv, nxt);
    int r = inside_point(x0 + ((double)i + 0.5) * h, y0 + ((double)j + 0.5) * h, M, X, Y, nxt);
    free(prv); free(nxt);
    return r;
}

/* The same crossing-number test for every cell centre, row by row: the
 * crossings of a row's centre line are computed once, and a cell is inside
 * when an odd number of them lie strictly to the right of its centre.       */
static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void or_inside(int nx, int ny, double h, double x0, double y0, int M,
               const double *X, const double *Y, int ndrops,
               const int32_t *drop_start, double *chi)
{
    int *prv = (int *)malloc((size_t)M * sizeof(int)), *nxt = (int *)malloc((size_t)M * sizeof(int));
    double *xs = (double *)malloc((size_t)(M + 1) * sizeof(double));
    links(M, ndrops, drop_start, prv, nxt);
    for (int j = 0; j < ny; j++) {
        double py = y0 + ((double)j + 0.5) * h;
        int nc = 0;
        for (int m = 0; m < M; m++) {
            double ax = X[m], ay = Y[m], bx = X[nxt[m]], by = Y[nxt[m]];
            if ((ay > py) != (by > py)) xs[nc++] = ax + (py - ay) * (bx - ax) / (by - ay);
        }
        qsort(xs, (size_t)nc, sizeof(double), cmp_double);
        int k = 0; /* crossings <= the current centre */
        for (int i = 0; i < nx; i++) {
            double px = x0 + ((double)i + 0.5) * h;
            while (k < nc && !(xs[k] > px)) k++;
            chi[CC(i, j)] = (double)((nc - k) & 1);
        }
    }
    free(prv); free(nxt); free(xs);
}

/* Area of the part of polygon (px,py)[n] inside the unit square [0,1]^2, by
 * Sutherland-Hodgman clipping against x>=0, x<=1, y>=0, y<=1 and the
 * shoelace formula.                                                          */
static double clip_area_unit(int n, const double *px, const double *py)
{
    double ax[16], ay[16], bx[16], by[16];
    int na = n;
    for (int k = 0; k < n; k++) { ax[k] = px[k]; ay[k] = py[k]; }
    for (int side = 0; side < 4; side++) {
        int nb = 0;
        for (int k = 0; k < na; k++) {
            double sx = ax[k], sy = ay[k];
            double ex = ax[(k + 1) % na], ey = ay[(k + 1) % na];
            double ds_, de;
            switch (side) {
            case 0: ds_ = sx; de = ex; break;             /* x >= 0 */
            case 1: ds_ = 1.0 - sx; de = 1.0 - ex; break; /* x <= 1 */
            case 2: ds_ = sy; de = ey; break;             /* y >= 0 */
            default: ds_ = 1.0 - sy; de = 1.0 - ey; break;/* y <= 1 */
            }
            int sin_ = ds_ >= 0.0, ein = de >= 0.0;
            if (sin_ && ein) { bx[nb] = ex; by[nb] = ey; nb++; }
            else if (sin_ && !ein) {
                double t = ds_ / (ds_ - de);
                bx[nb] = sx + t * (ex - sx); by[nb] = sy + t * (ey - sy); nb++;
            } else if (!sin_ && ein) {
                double t = ds_ / (ds_ - de);
                bx[nb] = sx + t * (ex - sx); by[nb] = sy + t * (ey - sy); nb++;
                bx[nb] = ex; by[nb] = ey; nb++;
            }
        }
        na = nb;
        for (int k = 0; k < na; k++) { ax[k] = bx[k]; ay[k] = by[k]; }
        if (na == 0) return 0.0;
    }
    double a = 0.0;
    for (int k = 0; k < na; k++) {
        int k1 = (k + 1) % na;
        a += ax[k] * ay[k1] - ax[k1] * ay[k];
    }
    return 0.5 * a;
}

/* Section 3.2, Fig. (pp_hf), (pp_df): the polygon about segment (m, m+1) is
 * the quadrilateral between the offsets r = -2.5 and r = +2.5 grid cells
 * along the marker normals n_m, n_{m+1} (inward positive); it is split into
 * five strips of width one cell, [k-2.5, k-1.5] for k = 0..4 (regions I..V),
 * each with the constant H = or_heaviside_profile(k - 2), the integral of the
 * kernel to the strip centre.  Adjacent polygons share the normal edge at
 * their common marker, so along a smooth interface they tile the band with
 * neither gap nor overlap.  H_ij = sum of (area of cell ∩ strip) * H_strip
 * over all strips (areas in units of the cell area), plus the cell area
 * covered by no strip times chi_ij (1 if the cell centre lies inside a drop).
 * Vertices are placed in grid units: (X - x0)/h + r n.                      */
static void strip_quad(int m, int nm, int k, const double *X, const double *Y,
                       const double *nxm, const double *nym, double x0,
                       double y0, double h, double *qx, double *qy)
{
    double a = (double)k - 2.5, b = (double)k - 1.5;
    double gxa = (X[m] - x0) / h, gya = (Y[m] - y0) / h;
    double gxb = (X[nm] - x0) / h, gyb = (Y[nm] - y0) / h;
    qx[0] = gxa + a * nxm[m];  qy[0] = gya + a * nym[m];
    qx[1] = gxb + a * nxm[nm]; qy[1] = gyb + a * nym[nm];
    qx[2] = gxb + b * nxm[nm]; qy[2] = gyb + b * nym[nm];
    qx[3] = gxa + b * nxm[m];  qy[3] = gya + b * nym[m];
}

static void marker_normals(int M, const double *X, const double *Y, int ndrops,
                           const int32_t *drop_start, double *nxm, double *nym)
{
    double *kap = (double *)malloc((size_t)M * sizeof(double));
    double *dsm = (double *)malloc((size_t)M * sizeof(double));
    or_curvature(M, X, Y, ndrops, drop_start, kap, nxm, nym, dsm);
    free(kap); free(dsm);
}

double or_heaviside_cell(int i, int j, double h, double x0, double y0, int M,
                         const double *X, const double *Y, int ndrops,
                         const int32_t *drop_start, double chi)
{
    double *nxm = (double *)malloc((size_t)M * sizeof(double));
    double *nym = (double *)malloc((size_t)M * sizeof(double));
    marker_normals(M, X, Y, ndrops, drop_start, nxm, nym);
    int *prv = (int *)malloc((size_t)M * sizeof(int)), *nxt = (int *)malloc((size_t)M * sizeof(int));
    links(M, ndrops, drop_start, prv, nxt);
    double acc = 0.0, cov = 0.0;
    for (int m = 0; m < M; m++) {
        int nm = nxt[m];
        for (int k = 0; k < 5; k++) {
            double qx[4], qy[4];
            strip_quad(m, nm, k, X, Y, nxm, nym, x0, y0, h, qx, qy);
            for (int t = 0; t < 4; t++) { qx[t] -= (double)i; qy[t] -= (double)j; }
            double A = clip_area_unit(4, qx, qy);
            acc += A * or_heaviside_profile((double)k - 2.0);
            cov += A;
        }
    }
    free(nxm); free(nym); free(prv); free(nxt);
    double unc = 1.0 - cov;
    if (unc < 0.0) unc = 0.0;
    return acc + unc * chi;
}

void or_heaviside(int nx, int ny, double h, double x0, double y0, int M,
                  const double *X, const double *Y, int ndrops,
                  const int32_t *drop_start, double *H)
{
    size_t n = (size_t)nx * ny;
    double *chi = (double *)malloc(n * sizeof(double));
    double *acc = (double *)calloc(n, sizeof(double));
    double *cov = (double *)calloc(n, sizeof(double));
    double *nxm = (double *)malloc((size_t)M * sizeof(double));
    double *nym = (double *)malloc((size_t)M * sizeof(double));
    or_inside(nx, ny, h, x0, y0, M, X, Y, ndrops, drop_start, chi);
    marker_normals(M, X, Y, ndrops, drop_start, nxm, nym);
    int *prv = (int *)malloc((size_t)M * sizeof(int)), *nxt = (int *)malloc((size_t)M * sizeof(int));
    links(M, ndrops, drop_start, prv, nxt);
    for (int m = 0; m < M; m++) {
        int nm = nxt[m];
        for (int k = 0; k < 5; k++) {
            double qx[4], qy[4];
            strip_quad(m, nm, k, X, Y, nxm, nym, x0, y0, h, qx, qy);
            double mnx = qx[0], mxx = qx[0], mny = qy[0], mxy = qy[0];
            for (int t = 1; t < 4; t++) {
                if (qx[t] < mnx) mnx = qx[t];
                if (qx[t] > mxx) mxx = qx[t];
                if (qy[t] < mny) mny = qy[t];
                if (qy[t] > mxy) mxy = qy[t];
            }
            int i0 = (int)floor(mnx), i1 = (int)floor(mxx);
            int j0 = (int)floor(mny), j1 = (int)floor(mxy);
            if (i0 < 0) i0 = 0;
            if (j0 < 0) j0 = 0;
            if (i1 > nx - 1) i1 = nx - 1;
            if (j1 > ny - 1) j1 = ny - 1;
            double Hk = or_heaviside_profile((double)k - 2.0);
            for (int j = j0; j <= j1; j++)
                for (int i = i0; i <= i1; i++) {
                    double lx[4], ly[4];
                    for (int t = 0; t < 4; t++) { lx[t] = qx[t] - (double)i; ly[t] = qy[t] - (double)j; }
                    double A = clip_area_unit(4, lx, ly);
                    acc[CC(i, j)] += A * Hk;
                    cov[CC(i, j)] += A;
                }
        }
    }
    for (size_t c = 0; c < n; c++) {
        double unc = 1.0 - cov[c];
        if (unc < 0.0) unc = 0.0;
        H[c] = acc[c] + unc * chi[c];
    }
    free(chi); free(acc); free(cov); free(nxm); free(nym); free(prv); free(nxt);
}

/* Section 3.2 Eq. (delta_hea_xy), with the 1/h that turns the difference of
 * H into a force density: F_x(i-1/2,j) = f_face (H_ij - H_{i-1,j}) / h.  The
 * face value f_face = sigma kappa is taken from the nearest segment (closest
 * point clamped to the segment; ties to the lower segment id), linearly
 * interpolated between that segment's two markers.  Faces with a zero
 * difference carry no force; wall faces none.                                */
static double face_fmag(double qx, double qy, int M, const double *X,
                        const double *Y, const int *nxt, double x0, double y0,
                        double h, const double *fmag)
{
    double best = INFINITY, fb = 0.0;
    for (int m = 0; m < M; m++) {
        int nm = nxt[m];
        double ax = (X[m] - x0) / h, ay = (Y[m] - y0) / h;
        double bx = (X[nm] - x0) / h, by = (Y[nm] - y0) / h;
        double ex = bx - ax, ey = by - ay;
        double t = ((qx - ax) * ex + (qy - ay) * ey) / (ex * ex + ey * ey);
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
        double dx = ax + t * ex - qx, dy = ay + t * ey - qy;
        double d2 = dx * dx + dy * dy;
        if (d2 < best) { best = d2; fb = (1.0 - t) * fmag[m] + t * fmag[nm]; }
    }
    return fb;
}

void or_spread_irrot(int nx, int ny, double h, double x0, double y0, int M,
                     const double *X, const double *Y, int ndrops,
                     const int32_t *drop_start, const double *fmag,
                     const double *H, double *Fx, double *Fy)
{
    int *prv = (int *)malloc((size_t)M * sizeof(int)), *nxt = (int *)malloc((size_t)M * sizeof(int));
    links(M, ndrops, drop_start, prv, nxt);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i <= nx; i++) {
            double F = 0.0;
            if (i > 0 && i < nx) {
                double dH = H[CC(i, j)] - H[CC(i - 1, j)];
                if (dH != 0.0)
                    F = face_fmag((double)i, (double)j + 0.5, M, X, Y, nxt, x0, y0, h,
                                  fmag) * dH / h;
            }
            Fx[XF(i, j)] = F;
        }
    #pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j <= ny; j++)
        for (int i = 0; i < nx; i++) {
            double F = 0.0;
            if (j > 0 && j < ny) {
                double dH = H[CC(i, j)] - H[CC(i, j - 1)];
                if (dH != 0.0)
                    F = face_fmag((double)i + 0.5, (double)j, M, X, Y, nxt, x0, y0, h,
                                  fmag) * dH / h;
            }
            Fy[YF(i, j)] = F;
        }
    free(prv); free(nxt);
}

/* ------------------------------------------------------------------------ */
/* Section 4.  Periodic cubic B-spline with uniform knots t_k = k tau
 * (spacing tau = L/g, g = round(L / (1.5 h)) spans, L the polyline length),
 * basis by the Cox-de Boor recursion of Eq. (bspline); marker parameters are
 * the cumulative chord lengths; the least-squares fit of Eq. (bspline_ls) is
 * solved for x and y by the normal equations with a dense Cholesky
 * factorisation.  The markers are then placed at equal arc length along the
 * fitted curve (arc length by 8-point Gauss-Legendre per span; each target
 * parameter by 12 Newton steps on the partial arc length, kept in its span),
 * the first at parameter 0.                                                   */
static void bspl_basis(double s, double tau, int g, int *idx, double *w,
                       double *dw)
{
    int q = (int)floor(s / tau);
    if (q > g - 1) q = g - 1;
    if (q < 0) q = 0;
    /* N[d][r] = B_{q-d+r, d}(s), r = 0..d (Cox-de Boor, knots t_k = k tau). */
    double N[4][4];
    N[0][0] = 1.0;
    for (int d = 1; d <= 3; d++)
        for (int r = 0; r <= d; r++) {
            int k = q - d + r;
            double tk = k * tau, tkd = (k + d) * tau, tk1 = (k + 1) * tau, tkd1 = (k + d + 1) * tau;
            double left = (r >= 1) ? (s - tk) / (tkd - tk) * N[d - 1][r - 1] : 0.0;
            double right = (r <= d - 1) ? (tkd1 - s) / (tkd1 - tk1) * N[d - 1][r] : 0.0;
            N[d][r] = left + right;
        }
    for (int r = 0; r <= 3; r++) {
        int k = q - 3 + r;
        idx[r] = ((k % g) + g) % g;
        w[r] = N[3][r];
        /* d/ds B_{k,3} = 3/(t_{k+3}-t_k) B_{k,2} - 3/(t_{k+4}-t_{k+1}) B_{k+1,2} */
        double a = (r >= 1) ? N[2][r - 1] : 0.0;
        double b = (r <= 2) ? N[2][r] : 0.0;
        dw[r] = 3.0 / (3.0 * tau) * a - 3.0 / (3.0 * tau) * b;
    }
}

static const double GL8X[8] = {-0.9602898564975363, -0.7966664774136267,
                               -0.5255324099163290, -0.1834346424956498,
                               0.1834346424956498,  0.5255324099163290,
                               0.7966664774136267,  0.9602898564975363};
static const double GL8W[8] = {0.1012285362903763, 0.2223810344533745,
                               0.3137066458778873, 0.3626837833783620,
                               0.3626837833783620, 0.3137066458778873,
                               0.2223810344533745, 0.1012285362903763};

static double bspl_speed(double s, double tau, int g, const double *cx,
                         const double *cy)
{
    int idx[4];
    double w[4], dw[4], dx = 0.0, dy = 0.0;
    bspl_basis(s, tau, g, idx, w, dw);
    for (int r = 0; r < 4; r++) { dx += cx[idx[r]] * dw[r]; dy += cy[idx[r]] * dw[r]; }
    return sqrt(dx * dx + dy * dy);
}

static double gl_len(double a, double b, double tau, int g, const double *cx,
                     const double *cy)
{
    double mid = 0.5 * (a + b), half = 0.5 * (b - a), s = 0.0;
    for (int k = 0; k < 8; k++) s += GL8W[k] * bspl_speed(mid + half * GL8X[k], tau, g, cx, cy);
    return s * half;
}

static int cholesky_solve(int n, double *A, double *b)
{
    for (int c = 0; c < n; c++) {
        double s = A[(size_t)c * n + c];
        for (int k = 0; k < c; k++) s -= A[(size_t)c * n + k] * A[(size_t)c * n + k];
        if (!(s > 0.0)) return -1;
        double d = sqrt(s);
        A[(size_t)c * n + c] = d;
        for (int r = c + 1; r < n; r++) {
            double t = A[(size_t)r * n + c];
            for (int k = 0; k < c; k++) t -= A[(size_t)r * n + k] * A[(size_t)c * n + k];
            A[(size_t)r * n + c] = t / d;
        }
    }
    for (int r = 0; r < n; r++) {
        double s = b[r];
        for (int k = 0; k < r; k++) s -= A[(size_t)r * n + k] * b[k];
        b[r] = s / A[(size_t)r * n + r];
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < n; k++) s -= A[(size_t)k * n + r] * b[k];
        b[r] = s / A[(size_t)r * n + r];
    }
    return 0;
}

int or_bspline_relocate(int M, const double *X, const double *Y, int ndrops,
                        const int32_t *drop_start, double h, double *Xo,
                        double *Yo)
{
    for (int d = 0; d < ndrops; d++) {
        int s0 = drop_start[d], n = drop_start[d + 1] - s0;
        double *sp = (double *)malloc((size_t)n * sizeof(double));
        double L = 0.0;
        for (int m = 0; m < n; m++) {
            int a = s0 + m, b = s0 + (m + 1) % n;
            sp[m] = L;
            double dx = X[b] - X[a], dy = Y[b] - Y[a];
            L += sqrt(dx * dx + dy * dy);
        }
        int g = (int)floor(L / (1.5 * h) + 0.5);
        if (g < 4) g = 4;
        if (g > n) g = n;
        if (g < 1) g = 1;
        double tau = L / g;
        double *G = (double *)calloc((size_t)g * g, sizeof(double));
        double *cx = (double *)calloc((size_t)g, sizeof(double));
        double *cy = (double *)calloc((size_t)g, sizeof(double));
        for (int m = 0; m < n; m++) {
            int idx[4];
            double w[4], dw[4];
            bspl_basis(sp[m], tau, g, idx, w, dw);
            for (int a = 0; a < 4; a++) {
                cx[idx[a]] += w[a] * X[s0 + m];
                cy[idx[a]] += w[a] * Y[s0 + m];
                for (int b = 0; b < 4; b++) G[(size_t)idx[a] * g + idx[b]] += w[a] * w[b];
            }
        }
        double *G2 = (double *)malloc((size_t)g * g * sizeof(double));
        memcpy(G2, G, (size_t)g * g * sizeof(double));
        int st = cholesky_solve(g, G, cx);
        if (st == 0) st = cholesky_solve(g, G2, cy);
        if (st != 0) { free(sp); free(G); free(G2); free(cx); free(cy); return -1; }
        double *cum = (double *)malloc((size_t)(g + 1) * sizeof(double));
        cum[0] = 0.0;
        for (int q = 0; q < g; q++) cum[q + 1] = cum[q] + gl_len(q * tau, (q + 1) * tau, tau, g, cx, cy);
        double Lp = cum[g];
        int q = 0;
        for (int m = 0; m < n; m++) {
            double target = Lp * (double)m / (double)n;
            while (q + 1 < g && cum[q + 1] <= target) q++;
            double a = q * tau, b = (q + 1) * tau;
            double seg = cum[q + 1] - cum[q];
            double s = a + tau * (target - cum[q]) / seg;
            for (int it = 0; it < 12; it++) {
                double f = cum[q] + gl_len(a, s, tau, g, cx, cy) - target;
                double sp_ = bspl_speed(s, tau, g, cx, cy);
                s -= f / sp_;
                if (s < a) s = a;
                if (s > b) s = b;
            }
            int idx[4];
            double w[4], dw[4], px = 0.0, py = 0.0;
            bspl_basis(s, tau, g, idx, w, dw);
            for (int r = 0; r < 4; r++) { px += cx[idx[r]] * w[r]; py += cy[idx[r]] * w[r]; }
            Xo[s0 + m] = px;
            Yo[s0 + m] = py;
        }
        free(sp); free(G); free(G2); free(cx); free(cy); free(cum);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Section 2.5 (conservation of mass): the area a drop's markers enclose
 * (planar: the shoelace sum in marker order; axisymmetric: the volume of
 * revolution 2 pi sum (z2 - z1)(r1^2 + r1 r2 + r2^2) / 6 over the right
 * half of the meridian, markers 0 .. n/2, the axis edge adding nothing).   */
double or_drop_measure(int n, const double *X, const double *Y, int axisym)
{
    double a = 0.0;
    if (!axisym) {
        for (int k = 0; k < n; k++) {
            int q = (k + 1 == n) ? 0 : k + 1;
            a += X[k] * Y[q] - X[q] * Y[k];
        }
        return 0.5 * a;
    }
    for (int k = 0; k < n / 2; k++) {
        double r1 = X[k], z1 = Y[k], r2 = X[k + 1], z2 = Y[k + 1];
        a += (z2 - z1) * (r1 * r1 + r1 * r2 + r2 * r2) / 6.0;
    }
    return 2.0 * 3.14159265358979323846 * a;
}

/* Section 2.5: where |A_n - A_o| > tol A_o, every marker of the drop moves
 * by one offset eps along its inward unit normal (the normals of the
 * uncorrected markers, as in or_curvature), eps found by bisection on
 * [-h, h] (moving inward shrinks the drop) until the bracket is below
 * 1e-13 h or 80 halvings: eps = the bracket's midpoint.  A0 per drop;
 * eps_out (per drop, may be NULL) gets 0 where no correction was needed.
 * Returns the number of drops corrected.                                  */
int or_mass_correct(int M, const double *X, const double *Y, int ndrops,
                    const int32_t *drop_start, const double *A0, int axisym, double tol,
                    double h, double *Xo, double *Yo, double *eps_out)
{
    double *kap = (double *)malloc((size_t)M * sizeof(double));
    double *nxm = (double *)malloc((size_t)M * sizeof(double));
    double *nym = (double *)malloc((size_t)M * sizeof(double));
    double *dsm = (double *)malloc((size_t)M * sizeof(double));
    or_curvature(M, X, Y, ndrops, drop_start, kap, nxm, nym, dsm);
    memcpy(Xo, X, (size_t)M * sizeof(double));
    memcpy(Yo, Y, (size_t)M * sizeof(double));
    int corrected = 0;
    for (int d = 0; d < ndrops; d++) {
        int s = drop_start[d], n = drop_start[d + 1] - s;
        double A = or_drop_measure(n, X + s, Y + s, axisym);
        if (eps_out) eps_out[d] = 0.0;
        if (!(fabs(A - A0[d]) > tol * A0[d])) continue;
        double lo = -h, hi = h;
        for (int it = 0; it < 80 && hi - lo > 1e-13 * h; it++) {
            double mid = 0.5 * (lo + hi);
            for (int k = 0; k < n; k++) {
                Xo[s + k] = X[s + k] + mid * nxm[s + k];
                Yo[s + k] = Y[s + k] + mid * nym[s + k];
            }
            if (or_drop_measure(n, Xo + s, Yo + s, axisym) > A0[d]) lo = mid; else hi = mid;
        }
        double eps = 0.5 * (lo + hi);
        for (int k = 0; k < n; k++) {
            Xo[s + k] = X[s + k] + eps * nxm[s + k];
            Yo[s + k] = Y[s + k] + eps * nym[s + k];
        }
        if (eps_out) eps_out[d] = eps;
        corrected++;
    }
    free(kap); free(nxm); free(nym); free(dsm);
    return corrected;
}

/* ------------------------------------------------------------------------ */
/* Crank-Nicolson viscous step (Section 2.1: Crank-Nicolson for the viscous
 * term).  With u_e the explicit predictor of this step computed with half
 * the viscosity (AB2 advection, half of D(u^n), body force), the
 * intermediate velocity solves
 *     u* - (dt / (2 rho_f)) D(u*) = u_e
 * per component, D the discrete div(mu grad) of or_predictor (cell mu on the
 * normal faces, node averages on the tangential ones, the reflected ghost of
 * a no-slip wall moving with axial velocity wb; axisymmetric: fluxes times
 * their face radius over the volume radius and -mu_f u / r^2 on the radial
 * component).  Solved by nsweeps red-black Gauss-Seidel sweeps in place on
 * each component's interior faces, red = (i + j) even first, u then v;
 * boundary faces keep their values.                                        */
static void cn_coeffs_u(int nx, int ny, double h, const double *mu, int axisym, int i, int j,
                        double c[4], double *extra)
{
    /* c = {E, W, N, S} with D(u) = sum c_k (u_k - u) - extra u; a wall
     * neighbour (ghost -u) gives c_k = 0 and extra += 2 c */
    double r0 = axisym ? i * h : 1.0, rE = axisym ? (i + 0.5) * h : 1.0,
           rW = axisym ? (i - 0.5) * h : 1.0;
    double s = 1.0 / (r0 * h * h);
    double muN = (j + 1 < ny) ? 0.25 * (mu[CC(i - 1, j)] + mu[CC(i, j)] + mu[CC(i - 1, j + 1)] + mu[CC(i, j + 1)])
                              : 0.5 * (mu[CC(i - 1, j)] + mu[CC(i, j)]);
    double muS = (j > 0) ? 0.25 * (mu[CC(i - 1, j - 1)] + mu[CC(i, j - 1)] + mu[CC(i - 1, j)] + mu[CC(i, j)])
                         : 0.5 * (mu[CC(i - 1, j)] + mu[CC(i, j)]);
    c[0] = rE * mu[CC(i, j)] * s;
    c[1] = rW * mu[CC(i - 1, j)] * s;
    double cN = r0 * muN * s, cS = r0 * muS * s;
    *extra = 0.0;
    if (j + 1 < ny) c[2] = cN; else { c[2] = 0.0; *extra += 2.0 * cN; }
    if (j > 0) c[3] = cS; else { c[3] = 0.0; *extra += 2.0 * cS; }
    if (axisym) *extra += 0.5 * (mu[CC(i - 1, j)] + mu[CC(i, j)]) / (r0 * r0);
}

static void cn_coeffs_v(int nx, int ny, double h, const double *mu, int axisym, int i, int j,
                        double c[4], double *extra, double *wall)
{
    /* c = {E, W, N, S}; *wall: the coefficient of the moving-wall ghost
     * 2 wb - v at the outer wall (E side of the last column): D gets
     * cE (2 wb - 2 v), i.e. extra += 2 cE and a source 2 cE wb            */
    double r0 = axisym ? (i + 0.5) * h : 1.0, rE = axisym ? (i + 1) * h : 1.0,
           rW = axisym ? i * h : 1.0;
    double s = 1.0 / (r0 * h * h);
    double muE = (i + 1 < nx) ? 0.25 * (mu[CC(i, j - 1)] + mu[CC(i + 1, j - 1)] + mu[CC(i, j)] + mu[CC(i + 1, j)])
                              : 0.5 * (mu[CC(i, j - 1)] + mu[CC(i, j)]);
    double muW = (i > 0) ? 0.25 * (mu[CC(i - 1, j - 1)] + mu[CC(i, j - 1)] + mu[CC(i - 1, j)] + mu[CC(i, j)])
                         : 0.5 * (mu[CC(i, j - 1)] + mu[CC(i, j)]);
    c[2] = r0 * mu[CC(i, j)] * s;
    c[3] = r0 * mu[CC(i, j - 1)] * s;
    double cE = rE * muE * s, cW = rW * muW * s;
    *extra = 0.0;
    *wall = 0.0;
    if (i + 1 < nx) c[0] = cE; else { c[0] = 0.0; *extra += 2.0 * cE; *wall = 2.0 * cE; }
    if (i > 0) c[1] = cW;
    else if (axisym) c[1] = 0.0;            /* the axis: zero area (rW = 0) */
    else { c[1] = 0.0; *extra += 2.0 * cW; } /* planar left wall */
}

void or_cn_solve(int nx, int ny, double h, double dt, const double *rho, const double *mu,
                 int axisym, double wb, int nsweeps, double *us, double *vs)
{
    double *ue = (double *)malloc((size_t)(nx + 1) * ny * sizeof(double));
    double *ve = (double *)malloc((size_t)nx * (ny + 1) * sizeof(double));
    memcpy(ue, us, (size_t)(nx + 1) * ny * sizeof(double));
    memcpy(ve, vs, (size_t)nx * (ny + 1) * sizeof(double));
    for (int sw = 0; sw < nsweeps; sw++) {
        for (int color = 0; color < 2; color++)
            for (int j = 0; j < ny; j++)
                for (int i = 1; i < nx; i++) {
                    if (((i + j) & 1) != color) continue;
                    double c[4], ex;
                    cn_coeffs_u(nx, ny, h, mu, axisym, i, j, c, &ex);
                    double tau = dt / (2.0 * 0.5 * (rho[CC(i - 1, j)] + rho[CC(i, j)]));
                    double nb = c[0] * us[XF(i + 1, j)] + c[1] * us[XF(i - 1, j)];
                    if (j + 1 < ny) nb += c[2] * us[XF(i, j + 1)];
                    if (j > 0) nb += c[3] * us[XF(i, j - 1)];
                    us[XF(i, j)] = (ue[XF(i, j)] + tau * nb) /
                                   (1.0 + tau * (c[0] + c[1] + c[2] + c[3] + ex));
                }
        for (int color = 0; color < 2; color++)
            for (int j = 1; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    if (((i + j) & 1) != color) continue;
                    double c[4], ex, wall;
                    cn_coeffs_v(nx, ny, h, mu, axisym, i, j, c, &ex, &wall);
                    double tau = dt / (2.0 * 0.5 * (rho[CC(i, j - 1)] + rho[CC(i, j)]));
                    double nb = c[2] * vs[YF(i, j + 1)] + c[3] * vs[YF(i, j - 1)] + wall * wb;
                    if (i + 1 < nx) nb += c[0] * vs[YF(i + 1, j)];
                    if (i > 0) nb += c[1] * vs[YF(i - 1, j)];
                    vs[YF(i, j)] = (ve[YF(i, j)] + tau * nb) /
                                   (1.0 + tau * (c[0] + c[1] + c[2] + c[3] + ex));
                }
    }
    free(ue); free(ve);
}
