/*
 * ib_oracle_axi.c -- plain FP64 CPU oracle of the axisymmetric (r, z) form of
 * the immersed-boundary projection method (Ong & Miura, arXiv 1807.10504,
 * Section 2.1: "the same discretization schemes are adopted ... in the
 * axisymmetric cylindrical coordinate system"; Section 4 Eq. (curv_ax);
 * Section 2.4 Eqs. (fictitious), (fic_1), (fic_2)).
 *
 * TEST INFRASTRUCTURE ONLY (see ib_oracle.c).  Grid: x = r from the axis
 * (r = 0 at the left edge), y = z; cell (i, j) centred at r_i = (i + 1/2) h,
 * x-face i at r = i h (face 0 is the axis, where u = 0).  Every operator is
 * the finite-volume balance of a ring-shaped control volume (volume r h^2
 * per radian, face areas r_face h), written out directly.  An interface is
 * the closed meridian curve of the drop including its mirror image at r < 0
 * (the markers of the right half and their reflections), so that the planar
 * Heaviside and strip geometry of ib_oracle.c apply to it unchanged.
 *
 * Readings where the paper is silent are stated at each routine.
 */
#include "ib_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define XF(i, j) ((size_t)(j) * (size_t)(nx + 1) + (size_t)(i))
#define YF(i, j) ((size_t)(j) * (size_t)nx + (size_t)(i))
#define CC(i, j) ((size_t)(j) * (size_t)nx + (size_t)(i))

static double rc(int i, double h) { return (i + 0.5) * h; }  /* cell centre radius */
static double rf(int i, double h) { return i * h; }          /* x-face radius */

/* ------------------------------------------------------------------------ */
/* (1/r) d/dr (r beta dp/dr) + d/dz (beta dp/dz) on cell (i, j): the net flux
 * of beta grad p through the four faces of the ring control volume (areas
 * r_face h, r_i h), divided by its volume r_i h^2.  Wall faces carry beta = 0;
 * the axis face has zero area.                                             */
void or_apply_A_axi(int nx, int ny, double h, const double *bx, const double *by,
                    const double *p, double *out)
{
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double c = p[CC(i, j)], s = 0.0;
            if (i + 1 < nx) s += rf(i + 1, h) * bx[XF(i + 1, j)] * (p[CC(i + 1, j)] - c);
            if (i > 0) s -= rf(i, h) * bx[XF(i, j)] * (c - p[CC(i - 1, j)]);
            if (j + 1 < ny) s += rc(i, h) * by[YF(i, j + 1)] * (p[CC(i, j + 1)] - c);
            if (j > 0) s -= rc(i, h) * by[YF(i, j)] * (c - p[CC(i, j - 1)]);
            out[CC(i, j)] = s / (rc(i, h) * h * h);
        }
}

/* The same operator multiplied by r_i: A~ p = r_i (A_axi p), a symmetric
 * 5-point operator with face coefficients beta~_x = r_face beta_x and
 * beta~_y = r_i beta_y, which the planar multigrid solves unchanged for the
 * right-hand side r_i b.  Writes the weighted coefficients.                */
void or_axi_weights(int nx, int ny, double h, const double *bx, const double *by,
                    double *bxa, double *bya)
{
    for (int j = 0; j < ny; j++)
        for (int i = 0; i <= nx; i++) bxa[XF(i, j)] = rf(i, h) * bx[XF(i, j)];
    for (int j = 0; j <= ny; j++)
        for (int i = 0; i < nx; i++) bya[YF(i, j)] = rc(i, h) * by[YF(i, j)];
}

/* Discrete divergence (1/r) d(r u)/dr + dv/dz of a face field.             */
void or_divergence_axi(int nx, int ny, double h, const double *u, const double *v,
                       double *d)
{
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++)
            d[CC(i, j)] = (rf(i + 1, h) * u[XF(i + 1, j)] - rf(i, h) * u[XF(i, j)]) / (rc(i, h) * h) +
                          (v[YF(i, j + 1)] - v[YF(i, j)]) / h;
}

/* Pressure right-hand side, Section 2.1 Eq. (ps) with the force in the
 * projection: b = div(u* / dt + beta F) in the axisymmetric divergence.      */
void or_rhs_axi(int nx, int ny, double h, double dt, const double *us, const double *vs,
                const double *Fx, const double *Fy, const double *bx, const double *by,
                double *b)
{
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double qE = us[XF(i + 1, j)] / dt + bx[XF(i + 1, j)] * Fx[XF(i + 1, j)];
            double qW = us[XF(i, j)] / dt + bx[XF(i, j)] * Fx[XF(i, j)];
            double qN = vs[YF(i, j + 1)] / dt + by[YF(i, j + 1)] * Fy[YF(i, j + 1)];
            double qS = vs[YF(i, j)] / dt + by[YF(i, j)] * Fy[YF(i, j)];
            b[CC(i, j)] = (rf(i + 1, h) * qE - rf(i, h) * qW) / (rc(i, h) * h) + (qN - qS) / h;
        }
}

/* ------------------------------------------------------------------------ */
/* Section 2.1 Eqs. (ad_bf) and (cr_ni) on the ring control volumes of the u-
 * (radial) and v- (axial) components, divided by the volume: the planar
 * fluxes of or_predictor, each multiplied by the radius of its face, over
 * r_cv h^2.  The radial component's diffusion of a vector adds -mu u / r^2
 * (mu the two-cell face average), the term that makes div(mu grad u) the
 * vector operator in cylindrical coordinates (reading: the paper's
 * div(mu grad u) form, no swirl).  u = 0 on the axis and the outer wall;
 * the boundaries z = 0, Lz and the outer wall r = R move axially with
 * velocity wb (0: fixed walls; in the drop's frame of Section 2.4 the
 * ambient fluid streams past with wb): v = wb on the z boundary faces, and
 * the reflected ghost value of a no-slip wall moving at wb is 2 wb - v
 * (u's ghost -u at z = 0, Lz); (gx, gy) a uniform body acceleration (gx = 0
 * on a symmetric problem).                                                 */
void or_predictor_axi(int nx, int ny, double h, double dt, const double *rho,
                      const double *mu, const double *u, const double *v,
                      const double *au_prev, const double *av_prev, int have_prev,
                      double gx, double gy, double wb, double *us, double *vs, double *au,
                      double *av)
{
    for (int j = 0; j < ny; j++)
        for (int i = 0; i <= nx; i++) {
            size_t k = XF(i, j);
            if (i == 0 || i == nx) { us[k] = 0.0; au[k] = 0.0; continue; }
            double r0 = rf(i, h), rE = rc(i, h), rW = rc(i - 1, h);
            double uc = u[k], uE = u[XF(i + 1, j)], uW = u[XF(i - 1, j)];
            double uN = (j + 1 < ny) ? u[XF(i, j + 1)] : -uc;
            double uS = (j > 0) ? u[XF(i, j - 1)] : -uc;
            double aE = 0.5 * (uE + uc), aW = 0.5 * (uc + uW);
            double fE = rE * rho[CC(i, j)] * aE * aE;
            double fW = rW * rho[CC(i - 1, j)] * aW * aW;
            double gN = 0.0, gS = 0.0, muN, muS;
            if (j + 1 < ny) {
                double rN = 0.25 * (rho[CC(i - 1, j)] + rho[CC(i, j)] + rho[CC(i - 1, j + 1)] + rho[CC(i, j + 1)]);
                double vN = 0.5 * (v[YF(i - 1, j + 1)] + v[YF(i, j + 1)]);
                gN = r0 * rN * vN * (0.5 * (uc + uN));
                muN = 0.25 * (mu[CC(i - 1, j)] + mu[CC(i, j)] + mu[CC(i - 1, j + 1)] + mu[CC(i, j + 1)]);
            } else {
                muN = 0.5 * (mu[CC(i - 1, j)] + mu[CC(i, j)]);
            }
            if (j > 0) {
                double rS = 0.25 * (rho[CC(i - 1, j - 1)] + rho[CC(i, j - 1)] + rho[CC(i - 1, j)] + rho[CC(i, j)]);
                double vS = 0.5 * (v[YF(i - 1, j)] + v[YF(i, j)]);
                gS = r0 * rS * vS * (0.5 * (uc + uS));
                muS = 0.25 * (mu[CC(i - 1, j - 1)] + mu[CC(i, j - 1)] + mu[CC(i - 1, j)] + mu[CC(i, j)]);
            } else {
                muS = 0.5 * (mu[CC(i - 1, j)] + mu[CC(i, j)]);
            }
            double adv = ((fE - fW) + (gN - gS)) / (r0 * h);
            double muf = 0.5 * (mu[CC(i - 1, j)] + mu[CC(i, j)]);
            double vis = (rE * mu[CC(i, j)] * (uE - uc) - rW * mu[CC(i - 1, j)] * (uc - uW) +
                          r0 * muN * (uN - uc) - r0 * muS * (uc - uS)) / (r0 * h * h) -
                         muf * uc / (r0 * r0);
            double rhof = 0.5 * (rho[CC(i - 1, j)] + rho[CC(i, j)]);
            double ae = have_prev ? 1.5 * adv - 0.5 * au_prev[k] : adv;
            us[k] = uc + dt * ((vis - ae) / rhof + gx);
            au[k] = adv;
        }
    for (int j = 0; j <= ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t k = YF(i, j);
            if (j == 0 || j == ny) { vs[k] = wb; av[k] = 0.0; continue; }
            double r0 = rc(i, h), rE = rf(i + 1, h), rW = rf(i, h);
            double vc = v[k], vN = v[YF(i, j + 1)], vS = v[YF(i, j - 1)];
            double vE = (i + 1 < nx) ? v[YF(i + 1, j)] : 2.0 * wb - vc;
            double vW = (i > 0) ? v[YF(i - 1, j)] : vc;  /* symmetric across the axis */
            double aN = 0.5 * (vN + vc), aS = 0.5 * (vc + vS);
            double fN = r0 * rho[CC(i, j)] * aN * aN;
            double fS = r0 * rho[CC(i, j - 1)] * aS * aS;
            double gE = 0.0, gW = 0.0, muE, muW;
            if (i + 1 < nx) {
                double rhE = 0.25 * (rho[CC(i, j - 1)] + rho[CC(i + 1, j - 1)] + rho[CC(i, j)] + rho[CC(i + 1, j)]);
                double uE = 0.5 * (u[XF(i + 1, j - 1)] + u[XF(i + 1, j)]);
                gE = rE * rhE * uE * (0.5 * (vc + vE));
                muE = 0.25 * (mu[CC(i, j - 1)] + mu[CC(i + 1, j - 1)] + mu[CC(i, j)] + mu[CC(i + 1, j)]);
            } else {
                muE = 0.5 * (mu[CC(i, j - 1)] + mu[CC(i, j)]);
            }
            if (i > 0) {
                double rhW = 0.25 * (rho[CC(i - 1, j - 1)] + rho[CC(i, j - 1)] + rho[CC(i - 1, j)] + rho[CC(i, j)]);
                double uW = 0.5 * (u[XF(i, j - 1)] + u[XF(i, j)]);
                gW = rW * rhW * uW * (0.5 * (vc + vW));
                muW = 0.25 * (mu[CC(i - 1, j - 1)] + mu[CC(i, j - 1)] + mu[CC(i - 1, j)] + mu[CC(i, j)]);
            } else {
                muW = 0.5 * (mu[CC(i, j - 1)] + mu[CC(i, j)]);  /* multiplied by r = 0 below */
            }
            double adv = ((fN - fS) + (gE - gW)) / (r0 * h);
            double vis = (r0 * mu[CC(i, j)] * (vN - vc) - r0 * mu[CC(i, j - 1)] * (vc - vS) +
                          rE * muE * (vE - vc) - rW * muW * (vc - vW)) / (r0 * h * h);
            double rhof = 0.5 * (rho[CC(i, j - 1)] + rho[CC(i, j)]);
            double ae = have_prev ? 1.5 * adv - 0.5 * av_prev[k] : adv;
            vs[k] = vc + dt * ((vis - ae) / rhof + gy);
            av[k] = adv;
        }
}

/* ------------------------------------------------------------------------ */
/* Section 4 Eq. (curv_ax): total curvature of the surface of revolution =
 * the meridian curvature (the planar discrete curvature of or_curvature,
 * positive for a convex drop traversed counter-clockwise) + the azimuthal
 * curvature -n_r / r, n the inward unit normal (for a sphere of radius R
 * both are 1/R).  On the axis (|r| <= 1e-9 ds) the azimuthal term takes its
 * limit, the meridian curvature.                                           */
void or_curvature_axi(int M, const double *X, const double *Y, int ndrops,
                      const int32_t *drop_start, double *kappa, double *nxm, double *nym,
                      double *ds)
{
    or_curvature(M, X, Y, ndrops, drop_start, kappa, nxm, nym, ds);
    for (int m = 0; m < M; m++) {
        double kaz = fabs(X[m]) <= 1e-9 * ds[m] ? kappa[m] : -nxm[m] / X[m];
        kappa[m] += kaz;
    }
}

/* Conventional spreading (Section 3.1 Eq. (delta_vec)) of the ring force: a
 * marker at radius |r_m| carries sigma kappa n ds over its ring 2 pi |r_m|;
 * spread onto the ring of the face at radius r_f it is the planar weight
 * times |r_m| / r_f.  Every marker of the closed curve (both halves)
 * contributes; the axis face (r = 0) and the walls carry no force.        */
void or_spread_conv_axi(int kernel, int nx, int ny, double h, int M, const double *X,
                        const double *Y, const double *fmag, const double *nxm,
                        const double *nym, const double *ds, double *Fx, double *Fy)
{
    memset(Fx, 0, (size_t)(nx + 1) * ny * sizeof(double));
    memset(Fy, 0, (size_t)nx * (ny + 1) * sizeof(double));
    for (int j = 0; j < ny; j++)
        for (int i = 1; i < nx; i++) {
            double acc = 0.0;
            for (int m = 0; m < M; m++) {
                double rx = i - X[m] / h, ry = (j + 0.5) - Y[m] / h;
                double w = or_phi(kernel, rx) * or_phi(kernel, ry);
                if (w == 0.0) continue;
                acc += fmag[m] * nxm[m] * ds[m] * fabs(X[m]) / rf(i, h) * w / (h * h);
            }
            Fx[XF(i, j)] = acc;
        }
    for (int j = 1; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double acc = 0.0;
            for (int m = 0; m < M; m++) {
                double rx = (i + 0.5) - X[m] / h, ry = j - Y[m] / h;
                double w = or_phi(kernel, rx) * or_phi(kernel, ry);
                if (w == 0.0) continue;
                acc += fmag[m] * nym[m] * ds[m] * fabs(X[m]) / rc(i, h) * w / (h * h);
            }
            Fy[YF(i, j)] = acc;
        }
}

/* Velocity at the markers (Section 2.2 Eq. (jump_condu)) with the field
 * continued across the axis by symmetry: u(-r) = -u(r) on x-faces, v(-r) =
 * v(r) on y-faces (x-face -i mirrors face i, cell -1-i mirrors cell i).    */
void or_interp_axi(int kernel, int nx, int ny, double h, const double *u, const double *v,
                   int M, const double *X, const double *Y, double *U, double *V)
{
    for (int m = 0; m < M; m++) {
        double sx = X[m] / h, sy = Y[m] / h - 0.5, acc = 0.0;
        for (int j = (int)floor(sy) - 1; j <= (int)floor(sy) + 2; j++)
            for (int i = (int)floor(sx) - 1; i <= (int)floor(sx) + 2; i++) {
                if (j < 0 || j >= ny) continue;
                int ii = i < 0 ? -i : i;
                if (ii > nx) continue;
                double val = (i < 0 ? -1.0 : 1.0) * u[XF(ii, j)];
                acc += val * or_phi(kernel, i - sx) * or_phi(kernel, j - sy);
            }
        U[m] = acc;
        sx = X[m] / h - 0.5;
        sy = Y[m] / h;
        acc = 0.0;
        for (int j = (int)floor(sy) - 1; j <= (int)floor(sy) + 2; j++)
            for (int i = (int)floor(sx) - 1; i <= (int)floor(sx) + 2; i++) {
                if (j < 0 || j > ny) continue;
                int ii = i < 0 ? -1 - i : i;
                if (ii >= nx) continue;
                acc += v[YF(ii, j)] * or_phi(kernel, i - sx) * or_phi(kernel, j - sy);
            }
        V[m] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Volume of revolution and centre of mass (z) of drop d: the polygon of its
 * markers clipped to r >= 0, by Green's theorem per straight edge,
 *   int int r dA   = sum (z2 - z1) (r1^2 + r1 r2 + r2^2) / 6,
 *   int int r z dA = sum (z2 - z1) (r1^2 (3 z1 + z2) + 2 r1 r2 (z1 + z2)
 *                                    + r2^2 (z1 + 3 z2)) / 24,
 * (counter-clockwise traversal); volume = 2 pi int int r dA.  Used by the
 * non-inertial frame (Section 2.4 Eqs. (fic_1), (fic_2)).                  */
void or_drop_com_axi(int M, const double *X, const double *Y, const int32_t *drop_start,
                     int d, double *volume, double *zc)
{
    int s = drop_start[d], e = drop_start[d + 1], n = e - s;
    double *px = (double *)malloc((size_t)(2 * n + 2) * sizeof(double));
    double *py = (double *)malloc((size_t)(2 * n + 2) * sizeof(double));
    int q = 0;
    for (int k = 0; k < n; k++) {  /* Sutherland-Hodgman against r >= 0 */
        double ax = X[s + k], ay = Y[s + k];
        double bx = X[s + (k + 1) % n], by = Y[s + (k + 1) % n];
        int ain = ax >= 0.0, bin = bx >= 0.0;
        if (ain) { px[q] = ax; py[q] = ay; q++; }
        if (ain != bin) {
            double t = ax / (ax - bx);
            px[q] = 0.0; py[q] = ay + t * (by - ay); q++;
        }
    }
    double I1 = 0.0, I2 = 0.0;
    for (int k = 0; k < q; k++) {
        double r1 = px[k], z1 = py[k], r2 = px[(k + 1) % q], z2 = py[(k + 1) % q];
        I1 += (z2 - z1) * (r1 * r1 + r1 * r2 + r2 * r2) / 6.0;
        I2 += (z2 - z1) * (r1 * r1 * (3.0 * z1 + z2) + 2.0 * r1 * r2 * (z1 + z2) +
                           r2 * r2 * (z1 + 3.0 * z2)) / 24.0;
    }
    free(px); free(py);
    /* Green: int int r dA = oint (r^2 / 2) dz, counter-clockwise traversal */
    *volume = 2.0 * 3.14159265358979323846 * I1;
    *zc = I1 != 0.0 ? I2 / I1 : 0.0;
}
