// Axisymmetric (r, z) form of the time step (Section 2.1: the planar
// discretisation carried over to the cylindrical coordinate system; Section 4
// Eq. (curv_ax)).  Grid: x = r from the axis (r = 0 at the left edge),
// y = z; cell (i, j) centred at r = (i + 1/2) h, x-face i at r = i h (face 0
// is the axis, where u = 0).  Operators are finite-volume balances of ring
// control volumes (volume r h^2 per radian, face areas r_face h).
//
// The pressure equation (1/r) d/dr (r beta dp/dr) + d/dz (beta dp/dz) = b is
// solved as r times itself: the planar 5-point operator with coefficients
// r_face beta and right-hand side r_i b, which the multigrid handles
// unchanged (the axis face has zero weight).
//
// Markers: a drop is its full closed meridian curve (right half and mirror
// image at r < 0), kept mirror-symmetric.  The marker kernels run unchanged
// on a planar grid widened by G ghost columns at r < 0 (origin -G h); the
// velocity field is continued into the ghost columns by symmetry (u odd, w
// even) before interpolation, and the Heaviside and face forces computed on
// the wide grid are folded back onto the real cells and faces (the
// conventional ring force divided by the face radius).
#include <math.h>

#include "ib_internal.cuh"

namespace ibk {
namespace {

constexpr int kT = 256;

// Tiled predictor in ring control volumes: the planar kernel's staging and
// node averages; every flux carries the radius of its face and each balance
// is divided by the radius of its control volume; the radial component adds
// -mu_face u / r^2 (vector diffusion).  With a frame record (non-inertial
// frame, see k_axi_frame) the axial body acceleration adds its S and the
// boundaries z = 0, Lz and the outer wall move axially with its wb: v = wb
// on the z boundary faces, the outer wall's reflected ghost is 2 wb - v.
constexpr int PX = 32, PY = 8;
__global__ void __launch_bounds__(PX * PY)
k_predictor_axi(int nx, int ny, double h, double dt, const double *__restrict__ rho,
                const double *__restrict__ mu, const double *__restrict__ u,
                const double *__restrict__ v, const double *__restrict__ aup,
                const double *__restrict__ avp, int have_prev, double gx, double gy,
                const double *__restrict__ frame, const double *__restrict__ bx,
                const double *__restrict__ by, double *__restrict__ us,
                double *__restrict__ vs, double *__restrict__ au, double *__restrict__ av)
{
    constexpr int W = PX + 2, Hh = PY + 2;
    const double gz = gy + (frame ? frame[kFrS] : 0.0), wb = frame ? frame[kFrWb] : 0.0;
    __shared__ double sr[Hh][W], sm[Hh][W], su[Hh][W + 1], sv[Hh + 1][W];
    __shared__ double nr[PY + 1][PX + 1], nm[PY + 1][PX + 1];
    // fluxes two faces share, with their radius (as the planar predictor):
    // radial momentum at cells i0-1 .. i0+PX-1 and nodes (i0 .. i0+PX-1,
    // j0 .. j0+PY); axial momentum at cells j0-1 .. j0+PY-1 and nodes
    // (i0 .. i0+PX, j0 .. j0+PY-1)
    __shared__ double fx[PY][PX + 1], vx[PY][PX + 1], gxn[PY + 1][PX], wxn[PY + 1][PX];
    __shared__ double fy[PY + 1][PX], vy[PY + 1][PX], gyn[PY][PX + 1], wyn[PY][PX + 1];
    const int i0 = blockIdx.x * PX, j0 = blockIdx.y * PY;
    const int t = threadIdx.y * PX + threadIdx.x;
    const long nxf = nx + 1;
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
    for (int k = t; k < (PY + 1) * (PX + 1); k += PX * PY) {
        const int r = k / (PX + 1), c = k - r * (PX + 1), I = i0 + c, J = j0 + r;
        if (I > nx || J > ny) continue;
        const double *r0 = &sr[r][c], *r1 = &sr[r + 1][c];
        const double *m0 = &sm[r][c], *m1 = &sm[r + 1][c];
        const bool wx = I == 0 || I == nx, wy = J == 0 || J == ny;
        nr[r][c] = 0.25 * (r0[0] + r0[1] + r1[0] + r1[1]);
        if (!wx && !wy) nm[r][c] = 0.25 * (m0[0] + m0[1] + m1[0] + m1[1]);
        else if (wy && !wx) nm[r][c] = J == 0 ? 0.5 * (m1[0] + m1[1]) : 0.5 * (m0[0] + m0[1]);
        else if (wx && !wy) nm[r][c] = I == 0 ? 0.5 * (m0[1] + m1[1]) : 0.5 * (m0[0] + m1[0]);
        else nm[r][c] = 0.0;
    }
    __syncthreads();
    // radial momentum of cell (i0-1+c, j0+r) at its outer radius (gi + 1/2) h
    for (int k = t; k < PY * (PX + 1); k += PX * PY) {
        const int r = k / (PX + 1), c = k - r * (PX + 1), gi = i0 - 1 + c;
        const double rc = (gi + 0.5) * h, a = 0.5 * (su[r + 1][c + 1] + su[r + 1][c]);
        fx[r][c] = rc * sr[r + 1][c] * a * a;
        vx[r][c] = rc * sm[r + 1][c] * (su[r + 1][c + 1] - su[r + 1][c]);
    }
    // axial momentum of cell (i0+c, j0-1+r) at the column's radius (gi + 1/2) h
    for (int k = t; k < (PY + 1) * PX; k += PX * PY) {
        const int r = k / PX, c = k - r * PX, gi = i0 + c;
        const double rc = (gi + 0.5) * h, a = 0.5 * (sv[r + 1][c + 1] + sv[r][c + 1]);
        fy[r][c] = rc * sr[r][c + 1] * a * a;
        vy[r][c] = rc * sm[r][c + 1] * (sv[r + 1][c + 1] - sv[r][c + 1]);
    }
    // radial momentum at node (I, J) = (i0+c, j0+r), radius I h: between
    // u(I, J-1) and u(I, J); reflected ghost at the bottom and top walls
    for (int k = t; k < (PY + 1) * PX; k += PX * PY) {
        const int r = k / PX, c = k - r * PX, I = i0 + c, J = j0 + r;
        if (I > nx || J > ny) continue;
        const double rn = I * h, ub = su[r][c + 1], ut = su[r + 1][c + 1];
        gxn[r][c] = (J > 0 && J < ny)
                        ? rn * nr[r][c] * (0.5 * (sv[r + 1][c] + sv[r + 1][c + 1])) * (0.5 * (ub + ut))
                        : 0.0;
        const double uT = J < ny ? ut : -ub, uB = J > 0 ? ub : -ut;
        wxn[r][c] = rn * nm[r][c] * (uT - uB);
    }
    // axial momentum at node (I, J), radius I h: between v(I-1, J) and
    // v(I, J); at the outer wall the ghost 2 wb - v, at the axis v itself
    for (int k = t; k < PY * (PX + 1); k += PX * PY) {
        const int r = k / (PX + 1), c = k - r * (PX + 1), I = i0 + c, J = j0 + r;
        if (I > nx || J > ny) continue;
        const double rn = I * h, vl = sv[r + 1][c], vr = sv[r + 1][c + 1];
        gyn[r][c] = (I > 0 && I < nx)
                        ? rn * nr[r][c] * (0.5 * (su[r][c + 1] + su[r + 1][c + 1])) * (0.5 * (vl + vr))
                        : 0.0;
        const double vR = I < nx ? vr : 2.0 * wb - vl, vL = I > 0 ? vl : vr;
        wyn[r][c] = rn * nm[r][c] * (vR - vL);
    }
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y, i = i0 + tx, j = j0 + ty;
    if (i >= nx || j >= ny) return;
    const int R = ty + 1, C = tx + 1;
    const double h2 = h * h;
    // radial face (i, j) at r = i h, control volume [r_(i-1), r_i]
    {
        const long k = (long)j * nxf + i;
        if (i == 0) {
            us[k] = 0.0; au[k] = 0.0;
        } else {
            const double r0 = i * h;
            const double uc = su[R][C];
            const double adv = ((fx[ty][tx + 1] - fx[ty][tx]) + (gxn[ty + 1][tx] - gxn[ty][tx])) / (r0 * h);
            const double muf = 0.5 * (sm[R][C - 1] + sm[R][C]);
            const double vis = (vx[ty][tx + 1] - vx[ty][tx] + wxn[ty + 1][tx] - wxn[ty][tx]) / (r0 * h2) -
                               muf * uc / (r0 * r0);
            // 1 / rho_face: the plain face coefficient beta when given
            const double irf = bx ? bx[k] : 1.0 / (0.5 * (sr[R][C - 1] + sr[R][C]));
            const double ae = have_prev ? 1.5 * adv - 0.5 * aup[k] : adv;
            us[k] = uc + dt * ((vis - ae) * irf + gx);
            au[k] = adv;
        }
        if (i == nx - 1) { us[k + 1] = 0.0; au[k + 1] = 0.0; }
    }
    // axial face (i, j) at r = (i + 1/2) h, control volume [i h, (i + 1) h]
    {
        const long k = (long)j * nx + i;
        if (j == 0) {
            vs[k] = wb; av[k] = 0.0;
        } else {
            const double r0 = (i + 0.5) * h;
            const double vc = sv[R][C];
            const double adv = ((fy[ty + 1][tx] - fy[ty][tx]) + (gyn[ty][tx + 1] - gyn[ty][tx])) / (r0 * h);
            const double vis = (vy[ty + 1][tx] - vy[ty][tx] + wyn[ty][tx + 1] - wyn[ty][tx]) / (r0 * h2);
            const double irf = by ? by[k] : 1.0 / (0.5 * (sr[R - 1][C] + sr[R][C]));
            const double ae = have_prev ? 1.5 * adv - 0.5 * avp[k] : adv;
            vs[k] = vc + dt * ((vis - ae) * irf + gz);
            av[k] = adv;
        }
        if (j == ny - 1) { vs[k + nx] = wb; av[k + nx] = 0.0; }
    }
}

// r_i b with b = div(u*/dt + beta F) in the axisymmetric divergence: the
// right-hand side of the r-weighted pressure equation.
__global__ void k_rhs_axi(int nx, int ny, double h, double idt, const double *__restrict__ us,
                          const double *__restrict__ vs, const double *__restrict__ Fx,
                          const double *__restrict__ Fy, const double *__restrict__ bx,
                          const double *__restrict__ by, double *__restrict__ b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    const long xw = (long)j * (nx + 1) + i, ys = (long)j * nx + i, yn = ys + nx;
    const double qE = us[xw + 1] * idt + bx[xw + 1] * Fx[xw + 1];
    const double qW = us[xw] * idt + bx[xw] * Fx[xw];
    const double qN = vs[yn] * idt + by[yn] * Fy[yn];
    const double qS = vs[ys] * idt + by[ys] * Fy[ys];
    const double ri = (i + 0.5) * h;
    const double bb = ((i + 1) * h * qE - i * h * qW) / (ri * h) + (qN - qS) / h;
    b[ys] = ri * bb;
}

// Coefficients of the r-weighted pressure operator: r_face beta_x, r_i beta_y.
__global__ void k_axi_weights(int nx, int ny, double h, const double *__restrict__ bx,
                              const double *__restrict__ by, double *__restrict__ bxa,
                              double *__restrict__ bya)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (j < ny && i <= nx) {
        const long k = (long)j * (nx + 1) + i;
        bxa[k] = (i * h) * bx[k];
    }
    if (i < nx) {
        const long k = (long)j * nx + i;
        bya[k] = ((i + 0.5) * h) * by[k];
    }
}

// Velocity on the wide marker grid (G ghost columns at r < 0): u odd and w
// even across the axis (x-face -i mirrors face i, cell -1-i mirrors cell i).
__global__ void k_axi_extend(int nx, int ny, int G, const double *__restrict__ u,
                             const double *__restrict__ v, double *__restrict__ uw,
                             double *__restrict__ vw)
{
    const int iw = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    const int nw = nx + G;
    if (j < ny && iw <= nw) {
        const int i = iw - G;
        const double val = i >= 0 ? u[(long)j * (nx + 1) + i] : -u[(long)j * (nx + 1) - i];
        uw[(long)j * (nw + 1) + iw] = val;
    }
    if (iw < nw) {
        const int i = iw - G;
        vw[(long)j * nw + iw] = v[(long)j * nx + (i >= 0 ? i : -1 - i)];
    }
}

// Real cells and faces from the wide grid: H, and the face forces (divided
// by the face radius for the ring-weighted conventional force); the axis and
// the outer wall carry no radial force.
__global__ void k_axi_fold(int nx, int ny, int G, double h, int ring, const double *__restrict__ Hw,
                           const double *__restrict__ Fxw, const double *__restrict__ Fyw,
                           double *__restrict__ H, double *__restrict__ Fx, double *__restrict__ Fy)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    const int nw = nx + G;
    if (Hw && j < ny && i < nx) H[(long)j * nx + i] = Hw[(long)j * nw + i + G];
    if (!Fxw) return;
    if (j < ny && i <= nx) {
        double f = 0.0;
        if (i > 0 && i < nx) {
            f = Fxw[(long)j * (nw + 1) + i + G];
            if (ring) f /= i * h;
        }
        Fx[(long)j * (nx + 1) + i] = f;
    }
    if (i < nx) {
        double f = Fyw[(long)j * nw + i + G];
        if (ring) f /= (i + 0.5) * h;
        Fy[(long)j * nx + i] = f;
    }
}

// Section 4 Eq. (curv_ax): the planar (meridian) curvature of k_geometry plus
// the azimuthal -n_r / r (its limit, the meridian curvature, on the axis);
// force magnitude sigma kappa.
__global__ void k_axi_curvature(int M, double sigma, const double *__restrict__ X,
                                const double *__restrict__ nxm, const double *__restrict__ ds,
                                double *__restrict__ kappa, double *__restrict__ fmag)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double x = X[m], k = kappa[m];
    const double kaz = fabs(x) <= 1e-9 * ds[m] ? k : -nxm[m] / x;
    const double kk = k + kaz;
    kappa[m] = kk;
    fmag[m] = sigma * kk;
}

// Ring magnitude of the conventional spreading: fmag |r| (the force per unit
// length of the marker's ring, up to the 2 pi shared with the face rings).
__global__ void k_axi_ring(int M, const double *__restrict__ fmag, const double *__restrict__ X,
                           double *__restrict__ fr)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) fr[m] = fmag[m] * fabs(X[m]);
}

// Mirror symmetry of each drop's meridian curve: marker k of a drop of n
// pairs with (n - k) mod n; each pair becomes its symmetric mean (one thread
// per pair, k = 0 .. n/2; markers 0 and n/2 land on the axis).
__global__ void k_axi_symmetrise(int ndrops, const int32_t *__restrict__ drop_start,
                                 double *__restrict__ X, double *__restrict__ Y)
{
    const int d = blockIdx.y;
    if (d >= ndrops) return;
    const int s = drop_start[d], n = drop_start[d + 1] - s;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n / 2) return;
    const int p = (n - k) % n;
    const double xk = X[s + k], xp = X[s + p], yk = Y[s + k], yp = Y[s + p];
    const double x = 0.5 * (xk - xp), y = 0.5 * (yk + yp);
    X[s + k] = x;
    Y[s + k] = y;
    if (p != k) {
        X[s + p] = 0.5 * (xp - xk);
        Y[s + p] = y;
    }
}

// Prescribed axial velocity wb of the z boundary faces (frame record).
__global__ void k_axi_zbc(int nx, int ny, const double *__restrict__ frame, double *__restrict__ v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const double wb = frame[kFrWb];
    v[i] = wb;
    v[(long)ny * nx + i] = wb;
}

// Volume-weighted axial centre of drop d: the right half of its meridian
// (markers 0 .. n/2, from the bottom axis point to the top one) closed along
// the axis, by Green's theorem per straight edge,
//   int int r dA = sum (z2 - z1)(r1^2 + r1 r2 + r2^2) / 6,
//   int int r z dA = sum (z2 - z1)(r1^2 (3 z1 + z2) + 2 r1 r2 (z1 + z2)
//                                  + r2^2 (z1 + 3 z2)) / 24,
// (the axis edge adds nothing).  One block of kFrT threads: thread t sums
// edges t, t + kFrT, ... and the partial sums meet in a fixed tree, so the
// result is the same on every run; the constant factors are applied once.
constexpr int kFrT = 256;
__device__ double drop_zc(const double *X, const double *Y, int s, int n)
{
    __shared__ double a1[kFrT], a2[kFrT];
    double I1 = 0.0, I2 = 0.0;
    for (int k = threadIdx.x; k < n / 2; k += kFrT) {
        const double r1 = X[s + k], z1 = Y[s + k], r2 = X[s + k + 1], z2 = Y[s + k + 1];
        I1 += (z2 - z1) * (r1 * r1 + r1 * r2 + r2 * r2);
        I2 += (z2 - z1) * (r1 * r1 * (3.0 * z1 + z2) + 2.0 * r1 * r2 * (z1 + z2) +
                           r2 * r2 * (z1 + 3.0 * z2));
    }
    a1[threadIdx.x] = I1;
    a2[threadIdx.x] = I2;
    __syncthreads();
    for (int o = kFrT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            a1[threadIdx.x] += a1[threadIdx.x + o];
            a2[threadIdx.x] += a2[threadIdx.x + o];
        }
        __syncthreads();
    }
    const double J1 = a1[0] / 6.0, J2 = a2[0] / 24.0;
    return J1 != 0.0 ? J2 / J1 : 0.0;
}

// Non-inertial frame following drop 0 (Section 2.4 Eqs. (fictitious),
// (fic_1), (fic_2), read as a restoring law on the drop's centre of mass):
// after a step that applied acceleration S to all fluid, the frame velocity
// Vf changes by -S dt and the next step's S = (c1 (COM_o - COM_n) -
// c2 (COM_n - COM_(n-1))) / dt^2; the ambient fluid at rest in the
// laboratory streams past the frame with wb = -Vf.  init: COM_o = COM_(n-1)
// = the current centre, S = Vf = wb = 0.  One block.
__global__ void __launch_bounds__(kFrT)
k_axi_frame(const double *__restrict__ X, const double *__restrict__ Y,
            const int32_t *__restrict__ drop_start, double dt, double c1, double c2, int init,
            double *__restrict__ frame)
{
    const int s = drop_start[0], n = drop_start[1] - s;
    const double com = drop_zc(X, Y, s, n);
    if (threadIdx.x != 0) return;
    if (init) {
        frame[kFrCom0] = com; frame[kFrComPrev] = com; frame[kFrCom] = com;
        frame[kFrS] = 0.0; frame[kFrVf] = 0.0; frame[kFrWb] = 0.0;
        return;
    }
    const double vf = frame[kFrVf] - frame[kFrS] * dt;
    const double S = (c1 * (frame[kFrCom0] - com) - c2 * (com - frame[kFrComPrev])) / (dt * dt);
    frame[kFrVf] = vf;
    frame[kFrS] = S;
    frame[kFrComPrev] = com;
    frame[kFrCom] = com;
    frame[kFrWb] = -vf;
}

}  // namespace

void launch_predictor_axi(int nx, int ny, double h, double dt, const double *rho,
                          const double *mu, const double *u, const double *v,
                          const double *au_prev, const double *av_prev, int have_prev,
                          double gx, double gy, const double *frame, const double *bx,
                          const double *by, double *us, double *vs, double *au, double *av,
                          cudaStream_t s)
{
    dim3 g(cdiv(nx, PX), cdiv(ny, PY)), b(PX, PY);
    note_launch();
    k_predictor_axi<<<g, b, 0, s>>>(nx, ny, h, dt, rho, mu, u, v, au_prev, av_prev, have_prev, gx,
                                    gy, frame, bx, by, us, vs, au, av);
}

void launch_axi_zbc(int nx, int ny, const double *frame, double *v, cudaStream_t s)
{
    note_launch();
    k_axi_zbc<<<cdiv(nx, 128), 128, 0, s>>>(nx, ny, frame, v);
}

void launch_axi_frame(const Markers &mk, double dt, double c1, double c2, int init, double *frame,
                      cudaStream_t s)
{
    note_launch();
    k_axi_frame<<<1, kFrT, 0, s>>>(mk.X, mk.Y, mk.drop_start, dt, c1, c2, init, frame);
}

void launch_rhs_axi(int nx, int ny, double h, double dt, const double *us, const double *vs,
                    const double *Fx, const double *Fy, const double *bx, const double *by,
                    double *b, cudaStream_t s)
{
    dim3 g(cdiv(nx, 128), ny);
    note_launch();
    k_rhs_axi<<<g, 128, 0, s>>>(nx, ny, h, 1.0 / dt, us, vs, Fx, Fy, bx, by, b);
}

void launch_axi_weights(int nx, int ny, double h, const double *bx, const double *by,
                        double *bxa, double *bya, cudaStream_t s)
{
    dim3 g(cdiv(nx + 1, 128), ny + 1);
    note_launch();
    k_axi_weights<<<g, 128, 0, s>>>(nx, ny, h, bx, by, bxa, bya);
}

void launch_axi_extend(int nx, int ny, int G, const double *u, const double *v, double *uw,
                       double *vw, cudaStream_t s)
{
    dim3 g(cdiv(nx + G + 1, 128), ny + 1);
    note_launch();
    k_axi_extend<<<g, 128, 0, s>>>(nx, ny, G, u, v, uw, vw);
}

void launch_axi_fold(int nx, int ny, int G, double h, int ring, const double *Hw, const double *Fxw,
                     const double *Fyw, double *H, double *Fx, double *Fy, cudaStream_t s)
{
    dim3 g(cdiv(nx + 1, 128), ny + 1);
    note_launch();
    k_axi_fold<<<g, 128, 0, s>>>(nx, ny, G, h, ring, Hw, Fxw, Fyw, H, Fx, Fy);
}

void launch_axi_curvature(Markers &mk, double sigma, cudaStream_t s)
{
    note_launch();
    k_axi_curvature<<<cdiv(mk.M, kT), kT, 0, s>>>(mk.M, sigma, mk.X, mk.nxm, mk.ds, mk.kappa,
                                                  mk.fmag);
}

void launch_axi_ring(const Markers &mk, const double *fmag, double *fr, cudaStream_t s)
{
    note_launch();
    k_axi_ring<<<cdiv(mk.M, kT), kT, 0, s>>>(mk.M, fmag, mk.X, fr);
}

void launch_axi_symmetrise(Markers &mk, cudaStream_t s)
{
    dim3 g(cdiv(mk.max_drop / 2 + 1, kT), mk.ndrops);
    note_launch();
    k_axi_symmetrise<<<g, kT, 0, s>>>(mk.ndrops, mk.drop_start, mk.X, mk.Y);
}

}  // namespace ibk
