/*
 * ib_oracle.h -- plain, slow, FP64 CPU oracle for the immersed-boundary
 * projection method of Ong & Miura (arXiv 1807.10504).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no header, helper or table with the CUDA
 * library, and it includes nothing from it.
 *
 * Conventions (shared by definition with the method, not by code):
 *   - uniform cell size h in x and y; domain [x0, x0 + nx h] x [y0, y0 + ny h];
 *   - cell (i,j), index j*nx + i, centre (x0 + (i+1/2)h, y0 + (j+1/2)h);
 *   - x-face (i,j), i = 0..nx, index j*(nx+1) + i, centre (x0 + i h, y0 + (j+1/2)h);
 *   - y-face (i,j), j = 0..ny, index j*nx + i,     centre (x0 + (i+1/2)h, y0 + j h);
 *   - wall faces (i = 0, nx for x; j = 0, ny for y) carry beta = 0, u = 0, F = 0;
 *   - markers: closed counter-clockwise polylines, drop d owns markers
 *     [drop_start[d], drop_start[d+1]); the successor of the last marker of a
 *     drop is its first marker.
 */
#ifndef IB_ORACLE_H
#define IB_ORACLE_H
#include <stdint.h>

/* Section 2.2, Eq. (cherby) in grid units, and the Peskin 4-point kernel.  */
double or_phi(int kernel, double r);
/* Section 3.2, Eq. (new_hea): integral of the cosine kernel from -2 to r.  */
double or_heaviside_profile(double r);

/* Section 2.2 Eq. (indicator) and Section 2.1 (face-averaged density).     */
void or_coeffs(int nx, int ny, double rho_g, double rho_l, double mu_g,
               double mu_l, const double *H, double *rho, double *mu,
               double *bx, double *by);

/* Section 2.1 Eq. (ps): the variable-coefficient 5-point operator.          */
void or_apply_A(int nx, int ny, double h, const double *bx, const double *by,
                const double *p, double *out);
void or_residual(int nx, int ny, double h, const double *bx, const double *by,
                 const double *b, const double *p, double *r);
void or_rbgs(int nx, int ny, double h, const double *bx, const double *by,
             const double *b, double *p, int nsweeps);
void or_restrict(int nx, int ny, const double *r, double *rc);
void or_coarsen_beta(int nx, int ny, const double *bx, const double *by,
                     double *bxc, double *byc);
void or_prolong_add(int nxc, int nyc, const double *ec, double *ef);
int  or_mg_levels(int nx, int ny, int *nxs, int *nys, int maxlev);
int  or_dense_solve(int nx, int ny, double h, const double *bx,
                    const double *by, const double *b, double *p);
int  or_mg_solve(int nx, int ny, double h, const double *bx, const double *by,
                 const double *b, double *p, int precision, double tol,
                 int max_cycles, int nu1, int nu2, int *cycles,
                 double *relres, double *hist);

/* Section 2.1 Eqs. (ps), (ns2_new) and Section 3.2 (force in projection).  */
void or_rhs(int nx, int ny, double h, double dt, const double *us,
            const double *vs, const double *Fx, const double *Fy,
            const double *bx, const double *by, double *b);
void or_correct(int nx, int ny, double h, double dt, const double *us,
                const double *vs, const double *p, const double *Fx,
                const double *Fy, const double *bx, const double *by,
                double *u, double *v);
void or_divergence(int nx, int ny, double h, const double *u, const double *v,
                   double *div);
/* Section 2.1 Eqs. (ad_bf), (cr_ni): explicit AB2 advection + viscous.     */
void or_predictor(int nx, int ny, double h, double dt, const double *rho,
                  const double *mu, const double *u, const double *v,
                  const double *au_prev, const double *av_prev, int have_prev,
                  double gx, double gy, double *us, double *vs, double *au,
                  double *av);

/* Marker-to-cell binning and the stable (key, id) order.                   */
void or_cell_keys(int M, const double *X, const double *Y, double x0,
                  double y0, double h, int nx, int ny, uint32_t *key);
void or_marker_sort(int M, const uint32_t *key, uint32_t *order);

/* Section 2.2 Eq. (jump_condu).                                             */
void or_interp(int kernel, int nx, int ny, double h, double x0, double y0,
               const double *u, const double *v, int M, const double *X,
               const double *Y, double *U, double *V);
/* Section 3.1 Eq. (delta_vec): conventional spreading.                     */
void or_spread_conv(int kernel, int nx, int ny, double h, double x0,
                    double y0, int M, const double *X, const double *Y,
                    const double *fmag, const double *nxm, const double *nym,
                    const double *ds, double *Fx, double *Fy);
/* Section 4 Eq. (ten_f): discrete signed curvature, normals, arc weights.  */
void or_curvature(int M, const double *X, const double *Y, int ndrops,
                  const int32_t *drop_start, double *kappa, double *nxm,
                  double *nym, double *ds);
/* Section 3.2: polygon discrete Heaviside and Eq. (delta_hea_xy).          */
void or_inside(int nx, int ny, double h, double x0, double y0, int M,
               const double *X, const double *Y, int ndrops,
               const int32_t *drop_start, double *chi);
double or_inside_cell(int i, int j, double h, double x0, double y0, int M,
                      const double *X, const double *Y, int ndrops,
                      const int32_t *drop_start);
void or_heaviside(int nx, int ny, double h, double x0, double y0, int M,
                  const double *X, const double *Y, int ndrops,
                  const int32_t *drop_start, double *H);
double or_heaviside_cell(int i, int j, double h, double x0, double y0, int M,
                         const double *X, const double *Y, int ndrops,
                         const int32_t *drop_start, double chi);
void or_spread_irrot(int nx, int ny, double h, double x0, double y0, int M,
                     const double *X, const double *Y, int ndrops,
                     const int32_t *drop_start, const double *fmag,
                     const double *H, double *Fx, double *Fy);
/* Section 4 Eqs. (bspline), (bcurve), (bspline_ls): LS relocation.         */
int or_bspline_relocate(int M, const double *X, const double *Y, int ndrops,
                        const int32_t *drop_start, double h, double *Xo,
                        double *Yo);

/* Section 2.1 Crank-Nicolson viscous step: nsweeps red-black sweeps on
 * u* - dt / (2 rho_f) D(u*) = u_e, (us, vs) = u_e on entry.               */
void or_cn_solve(int nx, int ny, double h, double dt, const double *rho, const double *mu,
                 int axisym, double wb, int nsweeps, double *us, double *vs);
/* Section 2.5: enclosed area (planar) or volume of revolution (axisymmetric)
 * of one drop, and the bisection correction of every drop's measure.      */
double or_drop_measure(int n, const double *X, const double *Y, int axisym);
int or_mass_correct(int M, const double *X, const double *Y, int ndrops,
                    const int32_t *drop_start, const double *A0, int axisym, double tol,
                    double h, double *Xo, double *Yo, double *eps_out);

/* ---- axisymmetric (r, z) form, ib_oracle_axi.c (x = r from the axis) ---- */
void or_apply_A_axi(int nx, int ny, double h, const double *bx, const double *by,
                    const double *p, double *out);
void or_axi_weights(int nx, int ny, double h, const double *bx, const double *by,
                    double *bxa, double *bya);
void or_divergence_axi(int nx, int ny, double h, const double *u, const double *v,
                       double *d);
void or_rhs_axi(int nx, int ny, double h, double dt, const double *us, const double *vs,
                const double *Fx, const double *Fy, const double *bx, const double *by,
                double *b);
void or_predictor_axi(int nx, int ny, double h, double dt, const double *rho,
                      const double *mu, const double *u, const double *v,
                      const double *au_prev, const double *av_prev, int have_prev,
                      double gx, double gy, double wb, double *us, double *vs, double *au,
                      double *av);
void or_curvature_axi(int M, const double *X, const double *Y, int ndrops,
                      const int32_t *drop_start, double *kappa, double *nxm, double *nym,
                      double *ds);
void or_spread_conv_axi(int kernel, int nx, int ny, double h, int M, const double *X,
                        const double *Y, const double *fmag, const double *nxm,
                        const double *nym, const double *ds, double *Fx, double *Fy);
void or_interp_axi(int kernel, int nx, int ny, double h, const double *u, const double *v,
                   int M, const double *X, const double *Y, double *U, double *V);
void or_drop_com_axi(int M, const double *X, const double *Y, const int32_t *drop_start,
                     int d, double *volume, double *zc);

#endif
