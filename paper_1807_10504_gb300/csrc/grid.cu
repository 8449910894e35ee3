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
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long nxf = (long)(nx + 1) * ny;
    if (k < nxf) {
        int j = (int)(k / (nx + 1)), i = (int)(k - (long)j * (nx + 1));
        bx[k] = (i == 0 || i == nx)
                    ? 0.0
                    : 1.0 / (0.5 * (rho[(long)j * nx + i - 1] + rho[(long)j * nx + i]));
        return;
    }
    k -= nxf;
    if (k >= (long)nx * (ny + 1)) return;
    int j = (int)(k / nx), i = (int)(k - (long)j * nx);
    by[k] = (j == 0 || j == ny)
                ? 0.0
                : 1.0 / (0.5 * (rho[(long)(j - 1) * nx + i] + rho[(long)j * nx + i]));
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

// Predictor for u (x-faces) and v (y-faces) in one index space.  Node
// averages use the four surrounding cells (two at a wall); no-slip walls by
// the reflected ghost value.
__global__ void k_predictor(int nx, int ny, double ih, double ih2, double dt,
                            const double *__restrict__ rho, const double *__restrict__ mu,
                            const double *__restrict__ u, const double *__restrict__ v,
                            const double *__restrict__ aup, const double *__restrict__ avp,
                            int have_prev, double gx, double gy, double *__restrict__ us,
                            double *__restrict__ vs, double *__restrict__ au,
                            double *__restrict__ av)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long nxf = (long)(nx + 1) * ny;
#define RC(i, j) rho[(long)(j) * nx + (i)]
#define MC(i, j) mu[(long)(j) * nx + (i)]
#define UF(i, j) u[(long)(j) * (nx + 1) + (i)]
#define VF(i, j) v[(long)(j) * nx + (i)]
    if (k < nxf) {
        int j = (int)(k / (nx + 1)), i = (int)(k - (long)j * (nx + 1));
        if (i == 0 || i == nx) { us[k] = 0.0; au[k] = 0.0; return; }
        double uc = u[k], uE = UF(i + 1, j), uW = UF(i - 1, j);
        double uN = (j + 1 < ny) ? UF(i, j + 1) : -uc;
        double uS = (j > 0) ? UF(i, j - 1) : -uc;
        double aE = 0.5 * (uE + uc), aW = 0.5 * (uc + uW);
        double fE = RC(i, j) * aE * aE, fW = RC(i - 1, j) * aW * aW;
        double gN = 0.0, gS = 0.0, muN, muS;
        if (j + 1 < ny) {
            double rN = 0.25 * (RC(i - 1, j) + RC(i, j) + RC(i - 1, j + 1) + RC(i, j + 1));
            double vN = 0.5 * (VF(i - 1, j + 1) + VF(i, j + 1));
            gN = rN * vN * (0.5 * (uc + uN));
            muN = 0.25 * (MC(i - 1, j) + MC(i, j) + MC(i - 1, j + 1) + MC(i, j + 1));
        } else {
            muN = 0.5 * (MC(i - 1, j) + MC(i, j));
        }
        if (j > 0) {
            double rS = 0.25 * (RC(i - 1, j - 1) + RC(i, j - 1) + RC(i - 1, j) + RC(i, j));
            double vS = 0.5 * (VF(i - 1, j) + VF(i, j));
            gS = rS * vS * (0.5 * (uc + uS));
            muS = 0.25 * (MC(i - 1, j - 1) + MC(i, j - 1) + MC(i - 1, j) + MC(i, j));
        } else {
            muS = 0.5 * (MC(i - 1, j) + MC(i, j));
        }
        double adv = (fE - fW) * ih + (gN - gS) * ih;
        double vis = (MC(i, j) * (uE - uc) - MC(i - 1, j) * (uc - uW) + muN * (uN - uc) -
                      muS * (uc - uS)) * ih2;
        double rf = 0.5 * (RC(i - 1, j) + RC(i, j));
        double ae = have_prev ? 1.5 * adv - 0.5 * aup[k] : adv;
        us[k] = uc + dt * ((vis - ae) / rf + gx);
        au[k] = adv;
        return;
    }
    k -= nxf;
    if (k >= (long)nx * (ny + 1)) return;
    int j = (int)(k / nx), i = (int)(k - (long)j * nx);
    if (j == 0 || j == ny) { vs[k] = 0.0; av[k] = 0.0; return; }
    double vc = v[k], vN = VF(i, j + 1), vS = VF(i, j - 1);
    double vE = (i + 1 < nx) ? VF(i + 1, j) : -vc;
    double vW = (i > 0) ? VF(i - 1, j) : -vc;
    double aN = 0.5 * (vN + vc), aS = 0.5 * (vc + vS);
    double fN = RC(i, j) * aN * aN, fS = RC(i, j - 1) * aS * aS;
    double gE = 0.0, gW = 0.0, muE, muW;
    if (i + 1 < nx) {
        double rE = 0.25 * (RC(i, j - 1) + RC(i + 1, j - 1) + RC(i, j) + RC(i + 1, j));
        double uE = 0.5 * (UF(i + 1, j - 1) + UF(i + 1, j));
        gE = rE * uE * (0.5 * (vc + vE));
        muE = 0.25 * (MC(i, j - 1) + MC(i + 1, j - 1) + MC(i, j) + MC(i + 1, j));
    } else {
        muE = 0.5 * (MC(i, j - 1) + MC(i, j));
    }
    if (i > 0) {
        double rW = 0.25 * (RC(i - 1, j - 1) + RC(i, j - 1) + RC(i - 1, j) + RC(i, j));
        double uW = 0.5 * (UF(i, j - 1) + UF(i, j));
        gW = rW * uW * (0.5 * (vc + vW));
        muW = 0.25 * (MC(i - 1, j - 1) + MC(i, j - 1) + MC(i - 1, j) + MC(i, j));
    } else {
        muW = 0.5 * (MC(i, j - 1) + MC(i, j));
    }
    double adv = (fN - fS) * ih + (gE - gW) * ih;
    double vis = (MC(i, j) * (vN - vc) - MC(i, j - 1) * (vc - vS) + muE * (vE - vc) -
                  muW * (vc - vW)) * ih2;
    double rf = 0.5 * (RC(i, j - 1) + RC(i, j));
    double ae = have_prev ? 1.5 * adv - 0.5 * avp[k] : adv;
    vs[k] = vc + dt * ((vis - ae) / rf + gy);
    av[k] = adv;
#undef RC
#undef MC
#undef UF
#undef VF
}

}  // namespace

void launch_coeffs(int nx, int ny, double rho_g, double rho_l, double mu_g,
                   double mu_l, const double *H, double *rho, double *mu,
                   double *bx, double *by, cudaStream_t s)
{
    long n = (long)nx * ny;
    note_launch();
    k_cells_props<<<cdiv(n, kT), kT, 0, s>>>((int)n, rho_g, rho_l - rho_g, mu_g,
                                             mu_l - mu_g, H, rho, mu);
    long nf = (long)(nx + 1) * ny + (long)nx * (ny + 1);
    note_launch();
    k_face_beta<<<cdiv(nf, kT), kT, 0, s>>>(nx, ny, rho, bx, by);
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
                      int have_prev, double gx, double gy, double *us,
                      double *vs, double *au, double *av, cudaStream_t s)
{
    long nf = (long)(nx + 1) * ny + (long)nx * (ny + 1);
    note_launch();
    k_predictor<<<cdiv(nf, kT), kT, 0, s>>>(nx, ny, 1.0 / h, 1.0 / (h * h), dt, rho,
                                            mu, u, v, au_prev, av_prev, have_prev,
                                            gx, gy, us, vs, au, av);
}

}  // namespace ibk
