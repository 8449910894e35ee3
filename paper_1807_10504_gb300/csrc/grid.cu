// Face/cell kernels of one time step: properties and face coefficients
// (Section 2.2 Eq. (indicator), Section 2.1), the pressure right-hand side
// and velocity correction with the force in the projection (Section 2.1
// Eq. (ps), Section 3.2 Eq. (ns2_new)), and the AB2 advection + explicit
// viscous predictor (Section 2.1 Eqs. (ad_bf), (cr_ni)).
//
// All kernels are single-pass, one thread per cell or face, coalesced along
// x; they are HBM-bound and small next to the multigrid solve.
#include "ib_internal.cuh"

namespace ibk {
namespace {

constexpr int kT = 256;

__global__ void k_cells_props(int n, double rho_g, double drho, double mu_g,
                              double dmu, const double *__restrict__ H,
                              double *__restrict__ rho, double *__restrict__ mu)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double hk = H[k];
    rho[k] = rho_g + drho * hk;
    mu[k] = mu_g + dmu * hk;
}

// beta on x-faces then y-faces in one index space.
__global__ void k_face_beta(int nx, int ny, const double *__restrict__ rho,
                            double *__restrict__ bx, double *__restrict__ by)
{
    // one row of x-faces (j < ny) and of y-faces (j <= ny) per blockIdx.y
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (j < ny && i <= nx) {
        const long k = (long)j * (nx + 1) + i;
        bx[k] = (i == 0 || i == nx)
                    ? 0.0
                    : recip_nr(0.5 * (rho[(long)j * nx + i - 1] + rho[(long)j * nx + i]));
    }
    if (i < nx) {
        const long k = (long)j * nx + i;
        by[k] = (j == 0 || j == ny)
                    ? 0.0
                    : recip_nr(0.5 * (rho[(long)(j - 1) * nx + i] + rho[(long)j * nx + i]));
    }
}

__global__ void k_rhs(int nx, int ny, double ih, double idt,
                      const double *__restrict__ us, const double *__restrict__ vs,
                      const double *__restrict__ Fx, const double *__restrict__ Fy,
                      const double *__restrict__ bx, const double *__restrict__ by,
                      double *__restrict__ b)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    long xw = (long)j * (nx + 1) + i, ys = (long)j * nx + i, yn = ys + nx;
    double divu = (us[xw + 1] - us[xw] + vs[yn] - vs[ys]) * ih;
    double divf = (bx[xw + 1] * Fx[xw + 1] - bx[xw] * Fx[xw] + by[yn] * Fy[yn] -
                   by[ys] * Fy[ys]) * ih;
    b[ys] = divu * idt + divf;
}

__global__ void k_correct(int nx, int ny, double ih, double dt,
                          const double *__restrict__ us, const double *__restrict__ vs,
                          const double *__restrict__ p, const double *__restrict__ Fx,
                          const double *__restrict__ Fy, const double *__restrict__ bx,
                          const double *__restrict__ by, double *__restrict__ u,
                          double *__restrict__ v)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long nxf = (long)(nx + 1) * ny;
    if (k < nxf) {
        int j = (int)(k / (nx + 1)), i = (int)(k - (long)j * (nx + 1));
        if (i == 0 || i == nx) { u[k] = 0.0; return; }
        double gp = (p[(long)j * nx + i] - p[(long)j * nx + i - 1]) * ih;
        u[k] = us[k] + dt * (bx[k] * (Fx[k] - gp));
        return;
    }
    k -= nxf;
    if (k >= (long)nx * (ny + 1)) return;
    int j = (int)(k / nx), i = (int)(k - (long)j * nx);
    if (j == 0 || j == ny) { v[k] = 0.0; return; }
    double gp = (p[(long)j * nx + i] - p[(long)(j - 1) * nx + i]) * ih;
    v[k] = vs[k] + dt * (by[k] * (Fy[k] - gp));
}

// Tiled predictor: a 32 x 8 block of cells stages rho, mu, u and v with a
// one-cell ring in shared memory, forms the node averages of rho and mu once
// per node (four cells inside, the two wall cells on a wall), then every
// flux that two faces share once per tile: per cell the advective flux
// rho a^2 and the viscous flux mu du of each component, per node the
// advective flux rho_n a_v a_u (one product for both components, zero
// through a wall) and the viscous flux mu_n du of each component (the
// reflected ghost folded in at a wall node).  Each thread then updates the x-face left of and the y-face
// below its cell (and the wall face on the far side for the last column /
// row) from differences of those fluxes, in the order of the per-face
// formula, so each face gets the same value as if it formed them itself.
// The advective fluxes are kept without their power-of-two factors (the
// 1/2 of each face average, the 1/4 of the node density): 4 rho a^2 per
// cell, 16 rho_n a_v a_u per node, the factors folded into 1/h of the
// difference; the node viscosity is kept as 4 mu_n, its 1/4 folded into the
// viscous difference.  Scaling by a power of two is exact, so every rounding
// is as in the per-face formula (fewer FP64 multiplications, the same
// values), except that the node product is formed in one order for both
// components.
constexpr int PX = 32, PY = 8;
__global__ void __launch_bounds__(PX * PY)
k_predictor(int nx, int ny, double ih, double ih2, double dt,
            const double *__restrict__ rho, const double *__restrict__ mu,
            const double *__restrict__ u, const double *__restrict__ v,
            const double *__restrict__ aup, const double *__restrict__ avp,
            int have_prev, double gx, double gy, const double *__restrict__ bx,
            const double *__restrict__ by, double *__restrict__ us,
            double *__restrict__ vs, double *__restrict__ au, double *__restrict__ av)
{
    constexpr int W = PX + 2, Hh = PY + 2;  // staged window: cells / faces i0-1 .. i0+PX
    __shared__ double sr[Hh][W], sm[Hh][W], su[Hh][W + 1], sv[Hh + 1][W];
    __shared__ double nm4[PY + 1][PX + 1];  // 4 mu_n
    // shared fluxes: x-momentum at cells i0-1 .. i0+PX-1 (fx, vx) and nodes
    // (i0 .. i0+PX-1, j0 .. j0+PY) (gx, wx); y-momentum at cells j0-1 ..
    // j0+PY-1 (fy, vy) and nodes (i0 .. i0+PX, j0 .. j0+PY-1) (gy, wy)
    __shared__ double fx[PY][PX + 1], vx[PY][PX + 1], gxn[PY + 1][PX], wxn[PY + 1][PX];
    __shared__ double fy[PY + 1][PX], vy[PY + 1][PX], gyn[PY][PX + 1], wyn[PY][PX + 1];
    const int i0 = blockIdx.x * PX, j0 = blockIdx.y * PY;
    const int t = threadIdx.y * PX + threadIdx.x;
    const long nxf = nx + 1;
    // staging; out-of-domain entries are never used by a face that is updated
    for (int k = t; k < Hh * (W + 1); k += PX * PY) {
        const int r = k / (W + 1), c = k - r * (W + 1), gi = i0 - 1 + c, gj = j0 - 1 + r;
        const bool inj = gj >= 0 && gj < ny;
        if (c < W) {
            const bool in = inj && gi >= 0 && gi < nx;
            const long o = (long)gj * nx + gi;
            sr[r][c] = in ? rho[o] : 0.0;
            sm[r][c] = in ? mu[o] : 0.0;
        }
        su[r][c] = (inj && gi >= 0 && gi <= nx) ? u[(long)gj * nxf + gi] : 0.0;
    }
    for (int k = t; k < (Hh + 1) * W; k += PX * PY) {
        const int r = k / W, c = k - r * W, gi = i0 - 1 + c, gj = j0 - 1 + r;
        sv[r][c] = (gi >= 0 && gi < nx && gj >= 0 && gj <= ny) ? v[(long)gj * nx + gi] : 0.0;
    }
    __syncthreads();
    // node (I, J) = corner of cells (I-1, J-1), (I, J-1), (I-1, J), (I, J);
    // window index of cell (gi, gj) is (gj - j0 + 1, gi - i0 + 1).  The
    // advective node flux 16 rho_n a_v a_u, between u(I, J-1) and u(I, J)
    // (window (r, c+1), (r+1, c+1)) and between v(I-1, J) and v(I, J)
    // (window (r+1, c), (r+1, c+1)), serves the x-momentum (zero on the
    // walls J = 0, ny) and the y-momentum (zero on the walls I = 0, nx)
    for (int k = t; k < (PY + 1) * (PX + 1); k += PX * PY) {
        const int r = k / (PX + 1), c = k - r * (PX + 1), I = i0 + c, J = j0 + r;
        if (I > nx || J > ny) continue;
        const double *r0 = &sr[r][c], *r1 = &sr[r + 1][c];  // rows J-1, J; columns I-1, I
        const double *m0 = &sm[r][c], *m1 = &sm[r + 1][c];
        const bool wx = I == 0 || I == nx, wy = J == 0 || J == ny;
        const double rn4 = r0[0] + r0[1] + r1[0] + r1[1];  // 4 rho_n
        if (!wx && !wy) nm4[r][c] = m0[0] + m0[1] + m1[0] + m1[1];
        else if (wy && !wx) nm4[r][c] = J == 0 ? 2.0 * (m1[0] + m1[1]) : 2.0 * (m0[0] + m0[1]);
        else if (wx && !wy) nm4[r][c] = I == 0 ? 2.0 * (m0[1] + m1[1]) : 2.0 * (m0[0] + m1[0]);
        else nm4[r][c] = 0.0;  // corner: never used
        const double g = rn4 * (sv[r + 1][c] + sv[r + 1][c + 1]) * (su[r][c + 1] + su[r + 1][c + 1]);
        if (c < PX) gxn[r][c] = wy ? 0.0 : g;
        if (r < PY) gyn[r][c] = wx ? 0.0 : g;
    }
    __syncthreads();
    // cell fluxes: x-momentum of cell (i0-1+c, j0+r), window (r+1, c)
    for (int k = t; k < PY * (PX + 1); k += PX * PY) {
        const int r = k / (PX + 1), c = k - r * (PX + 1);
        const double a = su[r + 1][c + 1] + su[r + 1][c];  // 2 a
        fx[r][c] = sr[r + 1][c] * a * a;                   // 4 rho a^2
        vx[r][c] = sm[r + 1][c] * (su[r + 1][c + 1] - su[r + 1][c]);
    }
    // y-momentum of cell (i0+c, j0-1+r), window (r, c+1)
    for (int k = t; k < (PY + 1) * PX; k += PX * PY) {
        const int r = k / PX, c = k - r * PX;
        const double a = sv[r + 1][c + 1] + sv[r][c + 1];  // 2 a
        fy[r][c] = sr[r][c + 1] * a * a;                   // 4 rho a^2
        vy[r][c] = sm[r][c + 1] * (sv[r + 1][c + 1] - sv[r][c + 1]);
    }
    // viscous node fluxes (times 4) of the x-momentum at node (I, J) =
    // (i0+c, j0+r): between u(I, J-1) (window (r, c+1)) and u(I, J) (window
    // (r+1, c+1))
    for (int k = t; k < (PY + 1) * PX; k += PX * PY) {
        const int r = k / PX, c = k - r * PX, I = i0 + c, J = j0 + r;
        if (I > nx || J > ny) continue;
        const double ub = su[r][c + 1], ut = su[r + 1][c + 1];
        const double uT = J < ny ? ut : -ub, uB = J > 0 ? ub : -ut;
        wxn[r][c] = nm4[r][c] * (uT - uB);
    }
    // of the y-momentum at node (I, J) = (i0+c, j0+r): between v(I-1, J)
    // (window (r+1, c)) and v(I, J) (window (r+1, c+1))
    for (int k = t; k < PY * (PX + 1); k += PX * PY) {
        const int r = k / (PX + 1), c = k - r * (PX + 1), I = i0 + c, J = j0 + r;
        if (I > nx || J > ny) continue;
        const double vl = sv[r + 1][c], vr = sv[r + 1][c + 1];
        const double vR = I < nx ? vr : -vl, vL = I > 0 ? vl : -vr;
        wyn[r][c] = nm4[r][c] * (vR - vL);
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y, i = i0 + tx, j = j0 + ty;
    if (i >= nx || j >= ny) return;
    const int R = ty + 1, C = tx + 1;  // window index of cell (i, j)
    const double ih4 = 0.25 * ih, ih16 = 0.0625 * ih;  // the folded factors
    // x-face (i, j), left of cell (i, j)
    {
        const long k = (long)j * nxf + i;
        if (i == 0) {
            us[k] = 0.0; au[k] = 0.0;
        } else {
            const double uc = su[R][C];
            const double adv = (fx[ty][tx + 1] - fx[ty][tx]) * ih4 + (gxn[ty + 1][tx] - gxn[ty][tx]) * ih16;
            // (vx E - vx W + wx N - wx S) / h^2 with wx = wxn / 4 (exact)
            const double vis = fma(-0.25, wxn[ty][tx], fma(0.25, wxn[ty + 1][tx], vx[ty][tx + 1] - vx[ty][tx])) * ih2;
            // 1 / rho_face: the face coefficient beta when given (the same
            // reciprocal of the same rho), else formed here
            const double irf = bx ? bx[k] : recip_nr(0.5 * (sr[R][C - 1] + sr[R][C]));
            const double ae = have_prev ? 1.5 * adv - 0.5 * aup[k] : adv;
            us[k] = uc + dt * ((vis - ae) * irf + gx);
            au[k] = adv;
        }
        if (i == nx - 1) { us[k + 1] = 0.0; au[k + 1] = 0.0; }  // right wall face
    }
    // y-face (i, j), below cell (i, j)
    {
        const long k = (long)j * nx + i;
        if (j == 0) {
            vs[k] = 0.0; av[k] = 0.0;
        } else {
            const double vc = sv[R][C];
            const double adv = (fy[ty + 1][tx] - fy[ty][tx]) * ih4 + (gyn[ty][tx + 1] - gyn[ty][tx]) * ih16;
            const double vis = fma(-0.25, wyn[ty][tx], fma(0.25, wyn[ty][tx + 1], vy[ty + 1][tx] - vy[ty][tx])) * ih2;
            const double irf = by ? by[k] : recip_nr(0.5 * (sr[R - 1][C] + sr[R][C]));
            const double ae = have_prev ? 1.5 * adv - 0.5 * avp[k] : adv;
            vs[k] = vc + dt * ((vis - ae) * irf + gy);
            av[k] = adv;
        }
        if (j == ny - 1) { vs[k + nx] = 0.0; av[k + nx] = 0.0; }  // top wall face
    }
}

// Crank-Nicolson viscous step (Section 2.1): one red-black colour of a
// Gauss-Seidel sweep on u* - dt / (2 rho_f) D(u*) = u_e for both components
// at once (they do not couple), in place, boundary faces fixed.  D is the
// predictor's div(mu grad): cell mu on normal faces, node averages on
// tangential ones, a no-slip wall by the reflected ghost (moving with the
// frame's axial velocity wb at the axisymmetric outer wall); axisymmetric:
// fluxes times their face radius over the volume radius and -mu_f u / r^2
// on the radial component, zero flux through the axis.
__global__ void k_cn_sweep(int nx, int ny, double h, double dt, const double *__restrict__ rho,
                           const double *__restrict__ mu, int axisym,
                           const double *__restrict__ frame, int color,
                           const double *__restrict__ ue, const double *__restrict__ ve,
                           double *__restrict__ us, double *__restrict__ vs)
{
    const long nxf = nx + 1;
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long nu = nxf * ny;
    auto M = [&](int i, int j) { return mu[(long)j * nx + i]; };
    if (k < nu) {
        const int j = (int)(k / nxf), i = (int)(k - (long)j * nxf);
        if (i == 0 || i == nx || ((i + j) & 1) != color) return;
        const double r0 = axisym ? i * h : 1.0, rE = axisym ? (i + 0.5) * h : 1.0,
                     rW = axisym ? (i - 0.5) * h : 1.0;
        const double s = 1.0 / (r0 * h * h);
        const double muN = (j + 1 < ny) ? 0.25 * (M(i - 1, j) + M(i, j) + M(i - 1, j + 1) + M(i, j + 1))
                                        : 0.5 * (M(i - 1, j) + M(i, j));
        const double muS = (j > 0) ? 0.25 * (M(i - 1, j - 1) + M(i, j - 1) + M(i - 1, j) + M(i, j))
                                   : 0.5 * (M(i - 1, j) + M(i, j));
        const double cE = rE * M(i, j) * s, cW = rW * M(i - 1, j) * s;
        const double cN = r0 * muN * s, cS = r0 * muS * s;
        double ex = 0.0, nb = cE * us[k + 1] + cW * us[k - 1], cs = cE + cW;
        if (j + 1 < ny) { nb += cN * us[k + nxf]; cs += cN; } else ex += 2.0 * cN;
        if (j > 0) { nb += cS * us[k - nxf]; cs += cS; } else ex += 2.0 * cS;
        if (axisym) ex += 0.5 * (M(i - 1, j) + M(i, j)) / (r0 * r0);
        const double tau = dt / (2.0 * (0.5 * (rho[(long)j * nx + i - 1] + rho[(long)j * nx + i])));
        us[k] = (ue[k] + tau * nb) / (1.0 + tau * (cs + ex));
        return;
    }
    k -= nu;
    if (k >= (long)nx * (ny + 1)) return;
    const int j = (int)(k / nx), i = (int)(k - (long)j * nx);
    if (j == 0 || j == ny || ((i + j) & 1) != color) return;
    const double r0 = axisym ? (i + 0.5) * h : 1.0, rE = axisym ? (i + 1) * h : 1.0,
                 rW = axisym ? i * h : 1.0;
    const double s = 1.0 / (r0 * h * h);
    const double muE = (i + 1 < nx) ? 0.25 * (M(i, j - 1) + M(i + 1, j - 1) + M(i, j) + M(i + 1, j))
                                    : 0.5 * (M(i, j - 1) + M(i, j));
    const double muW = (i > 0) ? 0.25 * (M(i - 1, j - 1) + M(i, j - 1) + M(i - 1, j) + M(i, j))
                               : 0.5 * (M(i, j - 1) + M(i, j));
    const double cN = r0 * M(i, j) * s, cS = r0 * M(i, j - 1) * s;
    const double cE = rE * muE * s, cW = rW * muW * s;
    const double wb = frame ? frame[kFrWb] : 0.0;
    double ex = 0.0, nb = cN * vs[k + nx] + cS * vs[k - nx], cs = cN + cS;
    if (i + 1 < nx) { nb += cE * vs[k + 1]; cs += cE; } else { ex += 2.0 * cE; nb += 2.0 * cE * wb; }
    if (i > 0) { nb += cW * vs[k - 1]; cs += cW; }
    else if (!axisym) ex += 2.0 * cW;
    const double tau = dt / (2.0 * (0.5 * (rho[(long)(j - 1) * nx + i] + rho[(long)j * nx + i])));
    vs[k] = (ve[k] + tau * nb) / (1.0 + tau * (cs + ex));
}

// Indicator function of Section 2.2 Eq. (ind_psn), div grad I = div G:
// the right-hand side div G of the face field G (the spread delta vector),
// r_i times the axisymmetric divergence in that form; unit coefficients with
// the walls at zero (r_face for the axisymmetric form).
__global__ void k_div_faces(int nx, int ny, double h, int axisym, const double *__restrict__ Gx,
                            const double *__restrict__ Gy, double *__restrict__ b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    const long xw = (long)j * (nx + 1) + i, ys = (long)j * nx + i, yn = ys + nx;
    if (!axisym) {
        b[ys] = (Gx[xw + 1] - Gx[xw] + Gy[yn] - Gy[ys]) / h;
        return;
    }
    const double ri = (i + 0.5) * h;
    b[ys] = ri * (((i + 1) * h * Gx[xw + 1] - i * h * Gx[xw]) / (ri * h) + (Gy[yn] - Gy[ys]) / h);
}

__global__ void k_unit_beta(int nx, int ny, double h, int axisym, double *__restrict__ bx,
                            double *__restrict__ by)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (j < ny && i <= nx) bx[(long)j * (nx + 1) + i] = (i == 0 || i == nx) ? 0.0 : (axisym ? i * h : 1.0);
    if (i < nx) by[(long)j * nx + i] = (j == 0 || j == ny) ? 0.0 : (axisym ? (i + 0.5) * h : 1.0);
}

// I = clamp(sol - mean over the cells along the walls (the axis column is not
// a wall), 0, 1); the mean in a fixed order (bottom row, top row, then the
// right column and, planar, the left column, each in index order) by one
// thread into *ref, then the shift by a grid of threads.
__global__ void k_wall_mean(int nx, int ny, int axisym, const double *__restrict__ sol,
                            double *__restrict__ ref)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    long cnt = 0;
    for (int i = 0; i < nx; i++) { s += sol[i]; cnt++; }
    for (int i = 0; i < nx; i++) { s += sol[(long)(ny - 1) * nx + i]; cnt++; }
    for (int j = 1; j < ny - 1; j++) { s += sol[(long)j * nx + nx - 1]; cnt++; }
    if (!axisym)
        for (int j = 1; j < ny - 1; j++) { s += sol[(long)j * nx]; cnt++; }
    *ref = s / (double)cnt;
}

__global__ void k_shift_clip(long n, const double *__restrict__ sol, const double *__restrict__ ref,
                             double *__restrict__ I)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) I[k] = fmin(fmax(sol[k] - *ref, 0.0), 1.0);
}

// Initial guess of the pressure solve extrapolated in time: p <- 2 p - q,
// q <- the old p (p^n and p^(n-1) in, p0 = 2 p^n - p^(n-1) and p^n out).
__global__ void k_extrapolate(long n, double *__restrict__ p, double *__restrict__ q)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double t = p[k];
    p[k] = 2.0 * t - q[k];
    q[k] = t;
}

__global__ void k_fill(long n, double a, double *__restrict__ y)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) y[k] = a;
}

__global__ void k_scale(long n, double a, const double *__restrict__ x, double *__restrict__ y)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) y[k] = a * x[k];
}

}  // namespace

void launch_cn_solve(int nx, int ny, double h, double dt, const double *rho, const double *mu,
                     int axisym, const double *frame, int nsweeps, const double *ue,
                     const double *ve, double *us, double *vs, cudaStream_t s)
{
    const long nf = (long)(nx + 1) * ny + (long)nx * (ny + 1);
    for (int sw = 0; sw < nsweeps; sw++)
        for (int c = 0; c < 2; c++) {
            note_launch();
            k_cn_sweep<<<cdiv(nf, kT), kT, 0, s>>>(nx, ny, h, dt, rho, mu, axisym, frame, c, ue, ve,
                                                   us, vs);
        }
}

void launch_div_faces(int nx, int ny, double h, int axisym, const double *Gx, const double *Gy,
                      double *b, cudaStream_t s)
{
    note_launch();
    k_div_faces<<<dim3(cdiv(nx, 128), ny), 128, 0, s>>>(nx, ny, h, axisym, Gx, Gy, b);
}

void launch_unit_beta(int nx, int ny, double h, int axisym, double *bx, double *by, cudaStream_t s)
{
    note_launch();
    k_unit_beta<<<dim3(cdiv(nx + 1, 128), ny + 1), 128, 0, s>>>(nx, ny, h, axisym, bx, by);
}

void launch_indicator_finish(int nx, int ny, int axisym, const double *sol, double *ref, double *I,
                             cudaStream_t s)
{
    note_launch();
    k_wall_mean<<<1, 32, 0, s>>>(nx, ny, axisym, sol, ref);
    const long n = (long)nx * ny;
    note_launch();
    k_shift_clip<<<cdiv(n, kT), kT, 0, s>>>(n, sol, ref, I);
}

void launch_extrapolate(long n, double *p, double *q, cudaStream_t s)
{
    note_launch();
    k_extrapolate<<<cdiv(n, kT), kT, 0, s>>>(n, p, q);
}

void launch_fill(long n, double a, double *y, cudaStream_t s)
{
    note_launch();
    k_fill<<<cdiv(n, kT), kT, 0, s>>>(n, a, y);
}

void launch_scale(long n, double a, const double *x, double *y, cudaStream_t s)
{
    note_launch();
    k_scale<<<cdiv(n, kT), kT, 0, s>>>(n, a, x, y);
}

void launch_coeffs(int nx, int ny, double rho_g, double rho_l, double mu_g,
                   double mu_l, const double *H, double *rho, double *mu,
                   double *bx, double *by, cudaStream_t s)
{
    long n = (long)nx * ny;
    note_launch();
    k_cells_props<<<cdiv(n, kT), kT, 0, s>>>((int)n, rho_g, rho_l - rho_g, mu_g,
                                             mu_l - mu_g, H, rho, mu);
    dim3 gb(cdiv(nx + 1, 128), ny + 1);
    note_launch();
    k_face_beta<<<gb, 128, 0, s>>>(nx, ny, rho, bx, by);
}

void launch_rhs(int nx, int ny, double h, double dt, const double *us,
                const double *vs, const double *Fx, const double *Fy,
                const double *bx, const double *by, double *b, cudaStream_t s)
{
    dim3 g(cdiv(nx, 128), ny);
    note_launch();
    k_rhs<<<g, 128, 0, s>>>(nx, ny, 1.0 / h, 1.0 / dt, us, vs, Fx, Fy, bx, by, b);
}

void launch_correct(int nx, int ny, double h, double dt, const double *us,
                    const double *vs, const double *p, const double *Fx,
                    const double *Fy, const double *bx, const double *by,
                    double *u, double *v, cudaStream_t s)
{
    long nf = (long)(nx + 1) * ny + (long)nx * (ny + 1);
    note_launch();
    k_correct<<<cdiv(nf, kT), kT, 0, s>>>(nx, ny, 1.0 / h, dt, us, vs, p, Fx, Fy,
                                          bx, by, u, v);
}

void launch_predictor(int nx, int ny, double h, double dt, const double *rho,
                      const double *mu, const double *u, const double *v,
                      const double *au_prev, const double *av_prev,
                      int have_prev, double gx, double gy, const double *bx,
                      const double *by, double *us, double *vs, double *au, double *av,
                      cudaStream_t s)
{
    dim3 g(cdiv(nx, PX), cdiv(ny, PY)), b(PX, PY);
    note_launch();
    k_predictor<<<g, b, 0, s>>>(nx, ny, 1.0 / h, 1.0 / (h * h), dt, rho, mu, u, v, au_prev,
                                av_prev, have_prev, gx, gy, bx, by, us, vs, au, av);
}

}  // namespace ibk
