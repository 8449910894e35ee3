// Lagrangian marker kernels of the method (Sections 2.2, 3 and 4):
//   binning + deterministic (key, id) order, velocity interpolation
//   (Eq. (jump_condu)), conventional spreading (Eq. (delta_vec)) as a gather
//   over markers sorted by cell, the polygon discrete Heaviside and the
//   irrotational face force (Eqs. (delta_hea), (delta_hea_xy)), discrete
//   curvature (Eq. (ten_f)) and least-squares B-spline relocation
//   (Eqs. (bspline), (bcurve), (bspline_ls)).
//
// This translation unit is compiled without multiply-add contraction so that
// integer decisions taken from floating point (cell keys, inside/outside
// crossings, nearest segment) follow the same IEEE operations as a plain
// reading of the definitions.  No floating-point atomics: every sum has a
// fixed order.  All marker work is O(markers x stencil) and small next to the
// pressure solve; the band kernels touch only 8x8-cell blocks that have a
// marker within kSearch cells.
#include <math.h>

#include "ib_internal.cuh"

namespace ibk {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ double phi(int kernel, double r)
{
    double a = fabs(r);
    if (a >= 2.0) return 0.0;
    if (kernel == 0) return 0.25 * (1.0 + cospi(0.5 * r));
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
}

// Integer key with the order of the doubles (non-NaN; -0 treated as +0), so
// that the many exact comparisons of the inside test run on the integer pipe.
__device__ __forceinline__ unsigned long long okey(double d)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(d + 0.0);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

__device__ __forceinline__ void nbrs(int m, const int32_t *drop_of,
                                     const int32_t *drop_start, int *pm, int *nm)
{
    int d = drop_of[m], s = drop_start[d], e = drop_start[d + 1];
    *pm = (m == s) ? e - 1 : m - 1;
    *nm = (m == e - 1) ? s : m + 1;
}

// ------------------------------------------------------------ validation
__global__ void k_validate(int M, const double *__restrict__ X, const double *__restrict__ Y,
                           double xlo, double xhi, double ylo, double yhi,
                           uint32_t *__restrict__ flags)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double x = X[m], y = Y[m];
    if (!(x >= xlo && x <= xhi && y >= ylo && y <= yhi)) atomicOr(&flags[0], 1u);
}

// ------------------------------------------------------------ geometry
__global__ void k_geometry(int M, const double *__restrict__ X, const double *__restrict__ Y,
                           const int32_t *__restrict__ drop_of,
                           const int32_t *__restrict__ drop_start, double sigma, double x0,
                           double y0, double h, double *__restrict__ kappa,
                           double *__restrict__ nxm, double *__restrict__ nym,
                           double *__restrict__ ds, double *__restrict__ fmag,
                           double *__restrict__ gx, double *__restrict__ gy,
                           float *__restrict__ gxf, float *__restrict__ gyf,
                           unsigned long long *__restrict__ ykey)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    ykey[m] = okey(Y[m]);
    {
        double a = (X[m] - x0) / h, b = (Y[m] - y0) / h;
        gx[m] = a; gy[m] = b;
        gxf[m] = d2f_rn(a); gyf[m] = d2f_rn(b);
    }
    int pm, nm;
    nbrs(m, drop_of, drop_start, &pm, &nm);
    double ax = X[m] - X[pm], ay = Y[m] - Y[pm];
    double bx = X[nm] - X[m], by = Y[nm] - Y[m];
    double la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
    double tax = ax / la, tay = ay / la, tbx = bx / lb, tby = by / lb;
    double dsm = 0.5 * (la + lb);
    double dx = tbx - tax, dy = tby - tay;
    double cr = tax * tby - tay * tbx;
    double k = sqrt(dx * dx + dy * dy) / dsm;
    k = cr >= 0.0 ? k : -k;
    double nx_ = -tay - tby, ny_ = tax + tbx;
    double ln = sqrt(nx_ * nx_ + ny_ * ny_);
    kappa[m] = k;
    nxm[m] = nx_ / ln;
    nym[m] = ny_ / ln;
    ds[m] = dsm;
    fmag[m] = sigma * k;
}

// Half-plane {x : n.x - c >= 0} on the left of the directed line P -> Q, with
// n the unit left normal (a zero vector, which constrains nothing, if P = Q).
__device__ __forceinline__ void left_of(double px, double py, double qx, double qy, double *l)
{
    const double dx = qx - px, dy = qy - py, len = sqrt(dx * dx + dy * dy);
    const double il = recip_any(len);
    const double nx_ = -dy * il, ny_ = dx * il;
    l[0] = nx_; l[1] = ny_; l[2] = nx_ * px + ny_ * py;
}

// Segment geometry of (m, next m): the strip corners at offsets -2.5 .. 2.5
// cells along both marker normals (grid units), the strip and slab boxes
// rounded outward to FP32 so that an FP32 test against a cell never rejects
// a strip that touches it, the eight bounding half-planes and whether all
// five strips are convex.

__global__ void k_segments(int M, const int32_t *__restrict__ next, const double *__restrict__ gx,
                           const double *__restrict__ gy, const double *__restrict__ nxm,
                           const double *__restrict__ nym, float4 *__restrict__ sbox,
                           double *__restrict__ sv, float4 *__restrict__ sb5,
                           double *__restrict__ sl, float4 *__restrict__ slf,
                           uint8_t *__restrict__ scvx, double *__restrict__ sinv)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    int nm = next[m];
    const double gxa = gx[m], gya = gy[m], gxb = gx[nm], gyb = gy[nm];
    {
        const double ex = gxb - gxa, ey = gyb - gya;  // 1 / |segment|^2 (grid units)
        sinv[m] = recip_any(ex * ex + ey * ey);
    }
    const double nax = nxm[m], nay = nym[m], nbx = nxm[nm], nby = nym[nm];
    // corner o (offset o - 2.5 cells) on the normal at m: (2o, 2o+1); at next m: 12 + (2o, 2o+1)
    double *v = sv + (long)m * 24;
    double ax[6], ay[6], bx[6], by[6];
    for (int o = 0; o < 6; o++) {
        const double a = (double)o - 2.5;
        ax[o] = gxa + a * nax; ay[o] = gya + a * nay;
        bx[o] = gxb + a * nbx; by[o] = gyb + a * nby;
        v[2 * o] = ax[o]; v[2 * o + 1] = ay[o];
        v[12 + 2 * o] = bx[o]; v[12 + 2 * o + 1] = by[o];
    }
    // minima and maxima of the (finite) corners compared on their bit
    // patterns, in integer instructions (ordered like the values)
    auto kb = [](double d) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(d);
        return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
    };
    auto dmin = [&](double a, double b) { return kb(a) <= kb(b) ? a : b; };
    auto dmax = [&](double a, double b) { return kb(a) >= kb(b) ? a : b; };
    float fx0 = INFINITY, fx1 = -INFINITY, fy0 = INFINITY, fy1 = -INFINITY;
    for (int k = 0; k < 5; k++) {
        double x0 = dmin(dmin(ax[k], ax[k + 1]), dmin(bx[k], bx[k + 1]));
        double x1 = dmax(dmax(ax[k], ax[k + 1]), dmax(bx[k], bx[k + 1]));
        double y0 = dmin(dmin(ay[k], ay[k + 1]), dmin(by[k], by[k + 1]));
        double y1 = dmax(dmax(ay[k], ay[k + 1]), dmax(by[k], by[k + 1]));
        float4 f = make_float4(__double2float_rd(x0) - 1e-3f, __double2float_ru(x1) + 1e-3f,
                               __double2float_rd(y0) - 1e-3f, __double2float_ru(y1) + 1e-3f);
        sb5[(long)m * 5 + k] = f;
        fx0 = fminf(fx0, f.x); fx1 = fmaxf(fx1, f.y); fy0 = fminf(fy0, f.z); fy1 = fmaxf(fy1, f.w);
    }
    sbox[m] = make_float4(fx0, fx1, fy0, fy1);
    // half-planes of the slab (the quadrilaterals are counter-clockwise):
    // 0: normal edge at m (A5 -> A0), 1: normal edge at next m (B0 -> B5),
    // 2 + o: offset line o (A_o -> B_o), inside = larger offsets
    double L[8][3];
    left_of(ax[5], ay[5], ax[0], ay[0], L[0]);
    left_of(bx[0], by[0], bx[5], by[5], L[1]);
    for (int o = 0; o < 6; o++) left_of(ax[o], ay[o], bx[o], by[o], L[2 + o]);
    // FP64 record (kSegLine doubles): per line a, b, c, 1/a, 1/b (0 where
    // the component vanishes), then the reciprocals of the determinants
    // a_i b_j - b_i a_j of the two normal edges and of each normal edge with
    // each offset line, which the per-cell area formula would otherwise
    // recompute for every cell the segment meets.
    double *d = sl + (long)m * kSegLine;
    auto rcp = [](double v) { return recip_any(v); };
    for (int q = 0; q < 8; q++) {
        d[5 * q + 0] = L[q][0]; d[5 * q + 1] = L[q][1]; d[5 * q + 2] = L[q][2];
        d[5 * q + 3] = rcp(L[q][0]); d[5 * q + 4] = rcp(L[q][1]);
        // |n| in FP32: left_of normalised n (to a few units of 1e-16), so
        // (float)|n| is 1.0f, or 0.0f for the zero vector of a degenerate line
        const bool nz = ((__double_as_longlong(L[q][0]) | __double_as_longlong(L[q][1])) &
                         0x7fffffffffffffffLL) != 0;
        slf[(long)m * 8 + q] = make_float4(d2f_rn(L[q][0]), d2f_rn(L[q][1]), d2f_rn(L[q][2]),
                                           nz ? 1.0f : 0.0f);
    }
    d[40] = rcp(L[0][0] * L[1][1] - L[0][1] * L[1][0]);
    for (int o = 0; o < 6; o++) {
        d[41 + 2 * o] = rcp(L[0][0] * L[2 + o][1] - L[0][1] * L[2 + o][0]);
        d[42 + 2 * o] = rcp(L[1][0] * L[2 + o][1] - L[1][1] * L[2 + o][0]);
    }
    // The strips are the intersections of those half-planes only when every
    // strip quadrilateral (A_k, B_k, B_k+1, A_k+1) is strictly convex; a
    // radius of curvature below about 2.5 cells folds the inner strips.
    // Segments that fail either test use quadrilateral clipping.
    bool cvx = true;
    for (int k = 0; k < 5; k++) {
        const double qx[4] = {ax[k], bx[k], bx[k + 1], ax[k + 1]}, qy[4] = {ay[k], by[k], by[k + 1], ay[k + 1]};
        for (int c = 0; c < 4; c++) {
            const int c1 = (c + 1) & 3, c2 = (c + 2) & 3;
            const double cr = (qx[c1] - qx[c]) * (qy[c2] - qy[c1]) - (qy[c1] - qy[c]) * (qx[c2] - qx[c1]);
            // cr > 1e-6 on the bit patterns (a negative cr has a negative one)
            cvx = cvx && __double_as_longlong(cr) > __double_as_longlong(1e-6);
        }
    }
    // The half-plane path also wants every line at least 0.001 rad away from
    // the grid axes (or exactly on one): a line nearly parallel to a cell edge
    // meets it at an ill-conditioned point, which the area formula would use
    // twice (once per boundary piece); quadrilateral clipping has no such
    // sensitivity and takes those segments.
    const long long k3 = __double_as_longlong(1e-3);
    for (int q = 0; q < 8; q++) {
        // |a| == 0 or |a| >= 1e-3, likewise b, on the bit patterns of |a|, |b|
        const long long aa = __double_as_longlong(L[q][0]) & 0x7fffffffffffffffLL,
                        bb = __double_as_longlong(L[q][1]) & 0x7fffffffffffffffLL;
        cvx = cvx && (aa == 0 || aa >= k3) && (bb == 0 || bb >= k3);
    }
    scvx[m] = cvx ? 1 : 0;
}

// One warp per drop: the range of its marker Y.
__global__ void k_drop_yrange(int ndrops, const int32_t *__restrict__ drop_start,
                              const double *__restrict__ Y, double2 *__restrict__ dyr,
                              ulonglong2 *__restrict__ dyk)
{
    int d = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (d >= ndrops) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int m = drop_start[d] + lane; m < drop_start[d + 1]; m += 32) {
        lo = fmin(lo, Y[m]);
        hi = fmax(hi, Y[m]);
    }
    for (int o = 16; o; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
        dyr[d] = make_double2(lo, hi);
        dyk[d] = make_ulonglong2(okey(lo), okey(hi));
    }
}

// ------------------------------------------------------------ binning
__global__ void k_keys(int M, const double *__restrict__ X, const double *__restrict__ Y,
                       double x0, double y0, double h, int nx, int ny, int bnx,
                       uint32_t *__restrict__ key, uint32_t *__restrict__ count,
                       uint32_t *__restrict__ bcount)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    int kx = (int)floor((X[m] - x0) / h), ky = (int)floor((Y[m] - y0) / h);
    kx = min(max(kx, 0), nx - 1);
    ky = min(max(ky, 0), ny - 1);
    uint32_t k = (uint32_t)ky * (uint32_t)nx + (uint32_t)kx;
    key[m] = k;
    atomicAdd(&count[k], 1u);
    atomicAdd(&bcount[(ky / kBlk) * bnx + kx / kBlk], 1u);
}

constexpr int kScanItems = 8;
constexpr int kScanChunk = kT * kScanItems;

__device__ uint32_t block_excl_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t sh[kT];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kT; o <<= 1) {
        uint32_t t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0u;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t incl = sh[threadIdx.x];
    if (total) *total = sh[kT - 1];
    __syncthreads();
    return incl - v;
}

__global__ void k_scan_partial(long n, const uint32_t *__restrict__ a, uint32_t *__restrict__ part)
{
    long base = (long)blockIdx.x * kScanChunk;
    uint32_t s = 0;
    for (int k = 0; k < kScanItems; k++) {
        long q = base + (long)threadIdx.x * kScanItems + k;
        if (q < n) s += a[q];
    }
    uint32_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_scan_parts(int nparts, uint32_t *__restrict__ part)
{
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nparts; base += kT) {
        int q = base + threadIdx.x;
        uint32_t v = q < nparts ? part[q] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan(v, &tot);
        if (q < nparts) part[q] = ex + carry;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

__global__ void k_scan_final(long n, const uint32_t *__restrict__ a,
                             const uint32_t *__restrict__ part, uint32_t *__restrict__ out,
                             uint32_t total_M)
{
    long base = (long)blockIdx.x * kScanChunk + (long)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
    for (int k = 0; k < kScanItems; k++) {
        long q = base + k;
        v[k] = q < n ? a[q] : 0u;
        s += v[k];
    }
    uint32_t ex = block_excl_scan(s, nullptr) + part[blockIdx.x];
    for (int k = 0; k < kScanItems; k++) {
        long q = base + k;
        if (q < n) out[q] = ex;
        ex += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = total_M;
}

__global__ void k_place(int M, const uint32_t *__restrict__ key,
                        const uint32_t *__restrict__ cell_start, uint32_t *__restrict__ count,
                        uint32_t *__restrict__ tmp_ids)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    uint32_t k = key[m];
    uint32_t slot = cell_start[k] + atomicSub(&count[k], 1u) - 1u;
    tmp_ids[slot] = (uint32_t)m;
}

// Deterministic rank inside the cell: ids ascending.
__global__ void k_rerank(int M, const uint32_t *__restrict__ key,
                         const uint32_t *__restrict__ cell_start,
                         const uint32_t *__restrict__ tmp_ids, uint32_t *__restrict__ ids)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    uint32_t k = key[m], s = cell_start[k], e = cell_start[k + 1], r = 0;
    for (uint32_t t = s; t < e; t++) r += tmp_ids[t] < (uint32_t)m ? 1u : 0u;
    ids[s + r] = (uint32_t)m;
}

__global__ void k_block_active(int bnx, int bny, const uint32_t *__restrict__ bcount,
                               uint32_t *__restrict__ active)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= bnx * bny) return;
    int bi = b % bnx, bj = b / bnx;
    uint32_t any = 0;
    for (int dj = -1; dj <= 1; dj++)
        for (int di = -1; di <= 1; di++) {
            int ii = bi + di, jj = bj + dj;
            if (ii >= 0 && ii < bnx && jj >= 0 && jj < bny) any |= bcount[jj * bnx + ii];
        }
    active[b] = any ? 1u : 0u;
}

// ------------------------------------------------------------ interpolation
__global__ void k_interp(int M, int kernel, int nx, int ny, double h, double x0, double y0,
                         const double *__restrict__ u, const double *__restrict__ v,
                         double *__restrict__ X, double *__restrict__ Y,
                         double *__restrict__ U, double *__restrict__ V, double dt_move)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double Xm = X[m], Ym = Y[m];
    // the kernel is a product phi(dx) phi(dy): its 4 + 4 factors once per
    // component (the same values the 4 x 4 products use)
    double px[4], py[4];
    double sx = (Xm - x0) / h, sy = (Ym - y0) / h - 0.5;
    int i0 = (int)floor(sx) - 1, j0 = (int)floor(sy) - 1;
    for (int a = 0; a < 4; a++) {
        px[a] = phi(kernel, (double)(i0 + a) - sx);
        py[a] = phi(kernel, (double)(j0 + a) - sy);
    }
    double acc = 0.0;
    for (int b = 0; b < 4; b++)
        for (int a = 0; a < 4; a++) {
            int i = i0 + a, j = j0 + b;
            if (i < 0 || i > nx || j < 0 || j > ny - 1) continue;
            acc += u[(long)j * (nx + 1) + i] * (px[a] * py[b]);
        }
    double Um = acc;
    sx = (Xm - x0) / h - 0.5;
    sy = (Ym - y0) / h;
    i0 = (int)floor(sx) - 1;
    j0 = (int)floor(sy) - 1;
    for (int a = 0; a < 4; a++) {
        px[a] = phi(kernel, (double)(i0 + a) - sx);
        py[a] = phi(kernel, (double)(j0 + a) - sy);
    }
    acc = 0.0;
    for (int b = 0; b < 4; b++)
        for (int a = 0; a < 4; a++) {
            int i = i0 + a, j = j0 + b;
            if (i < 0 || i > nx - 1 || j < 0 || j > ny) continue;
            acc += v[(long)j * nx + i] * (px[a] * py[b]);
        }
    double Vm = acc;
    if (U) U[m] = Um;
    if (V) V[m] = Vm;
    if (dt_move != 0.0) {
        X[m] = Xm + dt_move * Um;
        Y[m] = Ym + dt_move * Vm;
    }
}

// ------------------------------------------------------------ conventional spread
// One thread per face; markers of the 4 x 5 (x-faces) or 5 x 4 (y-faces)
// cells that can reach the face, visited row by row in (cell, id) order.
__global__ void k_spread_conv(int kernel, int nx, int ny, double h, double x0, double y0,
                              int bnx, const uint32_t *__restrict__ bactive,
                              const uint32_t *__restrict__ cell_start,
                              const uint32_t *__restrict__ ids, const double *__restrict__ X,
                              const double *__restrict__ Y, const double *__restrict__ fmag,
                              const double *__restrict__ nxm, const double *__restrict__ nym,
                              const double *__restrict__ ds, double *__restrict__ Fx,
                              double *__restrict__ Fy)
{
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long nxf = (long)(nx + 1) * ny;
    const double ih2 = 1.0 / (h * h);
    bool isx = k < nxf;
    int i, j;
    if (isx) {
        j = (int)(k / (nx + 1));
        i = (int)(k - (long)j * (nx + 1));
        if (i == 0 || i == nx) return;
    } else {
        k -= nxf;
        if (k >= (long)nx * (ny + 1)) return;
        j = (int)(k / nx);
        i = (int)(k - (long)j * nx);
        if (j == 0 || j == ny) return;
    }
    int ci = min(i, nx - 1), cj = min(j, ny - 1);
    if (!bactive[(cj / kBlk) * bnx + ci / kBlk]) return;
    int ia = isx ? i - 2 : i - 2, ib = isx ? i + 1 : i + 2;
    int ja = isx ? j - 2 : j - 2, jb = isx ? j + 2 : j + 1;
    ia = max(ia, 0); ib = min(ib, nx - 1); ja = max(ja, 0); jb = min(jb, ny - 1);
    double acc = 0.0;
    for (int jj = ja; jj <= jb; jj++) {
        uint32_t s = cell_start[(long)jj * nx + ia], e = cell_start[(long)jj * nx + ib + 1];
        for (uint32_t t = s; t < e; t++) {
            int m = (int)ids[t];
            double sx, sy, c;
            if (isx) {
                sx = (X[m] - x0) / h; sy = (Y[m] - y0) / h - 0.5;
                c = fmag[m] * nxm[m] * ds[m] * ih2;
            } else {
                sx = (X[m] - x0) / h - 0.5; sy = (Y[m] - y0) / h;
                c = fmag[m] * nym[m] * ds[m] * ih2;
            }
            double rx = (double)i - sx, ry = (double)j - sy;
            if (fabs(rx) >= 2.0 || fabs(ry) >= 2.0) continue;
            acc += c * (phi(kernel, rx) * phi(kernel, ry));
        }
    }
    if (isx) Fx[k] = acc; else Fy[k] = acc;
}

// ------------------------------------------------------------ inside / outside
// Order-preserving key of the centre x of every column, x0 + (i + 0.5) h,
// formed once per context (the grid does not move; the same FP64 operations
// as the crossing test would use per cell).
__global__ void k_colkeys(int nx, double h, double x0, unsigned long long *__restrict__ ck)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nx) ck[i] = okey(x0 + ((double)i + 0.5) * h);
}

// One CTA per row: crossings of the row's centre line with every segment,
// sorted, then a crossing count per cell centre (the centres' keys from
// k_colkeys).  Writes H = chi.
__global__ void __launch_bounds__(kT)
k_rows_inside(int ndrops, int nx, double h, double x0, double y0, const double *__restrict__ X,
              const double *__restrict__ Y, const unsigned long long *__restrict__ ykey,
              const unsigned long long *__restrict__ colkey,
              const int32_t *__restrict__ next, const int32_t *__restrict__ drop_start,
              const ulonglong2 *__restrict__ dyk, double *__restrict__ H,
              uint32_t *__restrict__ flags)
{
    __shared__ unsigned long long xs[kMaxCross], srt[kMaxCross];
    __shared__ int nc;
    const int j = blockIdx.x;
    const double py = y0 + ((double)j + 0.5) * h;
    const unsigned long long kp = okey(py);
    if (threadIdx.x == 0) nc = 0;
    __syncthreads();
    // a drop entirely above (py < min Y) or not above (py >= max Y) the line
    // has no segment with one end above it and the other not
    for (int d = 0; d < ndrops; d++) {
        const ulonglong2 r = dyk[d];
        if (kp < r.x || kp >= r.y) continue;
        for (int m = drop_start[d] + threadIdx.x; m < drop_start[d + 1]; m += kT) {
            const int nm = next[m];
            if ((ykey[m] > kp) != (ykey[nm] > kp)) {
                double ax = X[m], ay = Y[m], bx = X[nm], by = Y[nm];
                double xc = ax + (py - ay) * (bx - ax) / (by - ay);
                int q = atomicAdd(&nc, 1);
                if (q < kMaxCross) xs[q] = okey(xc);
            }
        }
    }
    __syncthreads();
    int n = nc;
    if (n > kMaxCross) {
        if (threadIdx.x == 0) atomicOr(&flags[1], 1u);
        n = kMaxCross;
    }
    for (int q = threadIdx.x; q < n; q += kT) {
        unsigned long long v = xs[q];
        int r = 0;
        for (int t = 0; t < n; t++) r += (xs[t] < v || (xs[t] == v && t < q)) ? 1 : 0;
        srt[r] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nx; i += kT) {
        const unsigned long long kx = colkey[i];  // okey(x0 + (i + 0.5) h)
        int lo = 0, hi = n;  // first index with srt > px
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (srt[mid] > kx) hi = mid; else lo = mid + 1;
        }
        H[(long)j * nx + i] = ((n - lo) & 1) ? 1.0 : 0.0;
    }
}

// ------------------------------------------------------------ band candidates
// Segments (start-marker ids) whose start marker lies within kSearch cells of
// an 8x8 block, gathered row by row and sorted ascending.
__device__ int gather_candidates(int bi, int bj, int nx, int ny,
                                 const uint32_t *__restrict__ cell_start,
                                 const uint32_t *__restrict__ ids, uint32_t *cand,
                                 uint32_t *tmp, uint32_t *flags)
{
    constexpr int kRows = kBlk + 2 * kSearch;  // at most 22 rows: one warp
    __shared__ uint32_t rowoff[kRows + 1], rowsrc[kRows];
    __shared__ int total;
    const int ia = max(bi * kBlk - kSearch, 0), ib = min(bi * kBlk + kBlk - 1 + kSearch, nx - 1);
    const int ja = max(bj * kBlk - kSearch, 0), jb = min(bj * kBlk + kBlk - 1 + kSearch, ny - 1);
    const int nrows = jb - ja + 1;
    if (threadIdx.x < 32) {  // per row: first id and count, then an exclusive warp scan
        const int r = threadIdx.x;
        uint32_t src = 0, cnt = 0;
        if (r < nrows) {
            const long base = (long)(ja + r) * nx;
            src = cell_start[base + ia];
            cnt = cell_start[base + ib + 1] - src;
        }
        uint32_t inc = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (r >= o) inc += v;
        }
        if (r < nrows) { rowoff[r] = inc - cnt; rowsrc[r] = src; }
        if (r == 31) { rowoff[nrows] = inc; total = (int)inc; }
    }
    __syncthreads();
    int n = total;
    if (n > kMaxCand) {
        if (threadIdx.x == 0) atomicOr(&flags[1], 1u);
        n = kMaxCand;
    }
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        int r = 0;
        while (r + 1 < nrows && rowoff[r + 1] <= (uint32_t)q) r++;
        tmp[q] = ids[rowsrc[r] + (uint32_t)q - rowoff[r]];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        uint32_t v = tmp[q];
        int r = 0;
        for (int t = 0; t < n; t++) r += tmp[t] < v ? 1 : 0;
        cand[r] = v;
    }
    __syncthreads();
    return n;
}

// Area of the part of a polygon inside the unit square (Sutherland-Hodgman
// against x >= 0, x <= 1, y >= 0, y <= 1, then the shoelace formula).
__device__ double clip_area_unit(const double *px, const double *py)
{
    double ax[12], ay[12], bx[12], by[12];
    int na = 4;
    for (int k = 0; k < 4; k++) { ax[k] = px[k]; ay[k] = py[k]; }
    for (int side = 0; side < 4; side++) {
        int nb = 0;
        for (int k = 0; k < na; k++) {
            int k1 = (k + 1 == na) ? 0 : k + 1;
            double sx = ax[k], sy = ay[k], ex = ax[k1], ey = ay[k1];
            double ds_, de;
            if (side == 0) { ds_ = sx; de = ex; }
            else if (side == 1) { ds_ = 1.0 - sx; de = 1.0 - ex; }
            else if (side == 2) { ds_ = sy; de = ey; }
            else { ds_ = 1.0 - sy; de = 1.0 - ey; }
            bool sin_ = ds_ >= 0.0, ein = de >= 0.0;
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
        int k1 = (k + 1 == na) ? 0 : k + 1;
        a += ax[k] * ay[k1] - ax[k1] * ay[k];
    }
    return 0.5 * a;
}

__device__ __forceinline__ double strip_value(int k)
{
    // integral of the cosine kernel from -2 to the strip centre r = k - 2
    double r = (double)k - 2.0;
    if (r <= -2.0) return 0.0;
    if (r >= 2.0) return 1.0;
    return 0.5 + r / 4.0 + sin(M_PI * r / 2.0) / (2.0 * M_PI);
}

constexpr int kBT = kBlk * kBlk;  // one thread per cell of the block


// Position of the unit cell [i, i+1] x [j, j+1] against a half-plane
// n.x - c >= 0 evaluated in FP32 with a margin far above the FP32 error:
// -1 entirely outside, +1 entirely inside, 0 cut (or too close to tell).
__device__ __forceinline__ int cell_side(float4 l, float fi, float fj)
{
    const float base = l.x * fi + l.y * fj - l.z;
    const float hi = base + fmaxf(l.x, 0.0f) + fmaxf(l.y, 0.0f);
    const float lo = base + fminf(l.x, 0.0f) + fminf(l.y, 0.0f);
    const float m = 1e-2f * l.w;
    return hi < -m ? -1 : (lo > m ? 1 : 0);
}

// The band Heaviside runs in three launches so that the FP64 clipping, whose
// cost varies from cell to cell, is spread evenly over the GPU:
//  k_band_pairs (one CTA per active 8x8 block): every cell counts the
//    candidate segments whose slab (the four outer half-planes) may meet it,
//    tested in FP32; the block takes a range of the global pair list and
//    writes its (cell, segment) pairs, per cell in ascending segment order;
//  k_band_area (flat over the pair list): the areas of cell and strips;
//  k_band_sum (one CTA per active block): every cell sums its pairs in order,
//    H = sum A_k H_k + max(0, 1 - sum A_k) chi.
// Pair ranges are claimed with an atomic counter, so their place in the list
// varies from run to run, but each cell's pairs and their order do not: H is
// deterministic.
constexpr int kPairT = 256, kPairSub = kPairT / kBT;  // 4 threads per cell
// Pairs of non-convex strips (quadrilateral clipping, long serial FP64 work)
// are listed for the first kClipBlocks blocks of k_band_area, 32 pairs a
// block, and marked in the segment id's top bit.
constexpr int kClipBlocks = 32, kClipCap = kClipBlocks * 32;
constexpr uint32_t kClipFlag = 0x80000000u;
constexpr int kStage = 256;  // candidates whose slab tests are staged in shared memory
__global__ void __launch_bounds__(kPairT)
k_band_pairs(int nx, int ny, int bnx, const uint32_t *__restrict__ bactive,
             const uint32_t *__restrict__ cell_start, const uint32_t *__restrict__ ids,
             const float4 *__restrict__ slf, const uint8_t *__restrict__ scvx,
             const float4 *__restrict__ sbox, uint32_t cap, uint32_t *__restrict__ npairs,
             uint32_t *__restrict__ pseg, uint32_t *__restrict__ pcell, uint2 *__restrict__ crange,
             uint32_t *__restrict__ clip_list,
             uint32_t *__restrict__ flags)
{
    __shared__ uint32_t cand[kMaxCand], tmp[kMaxCand];
    __shared__ float4 s_box[kStage], s_l[4][kStage];
    __shared__ uint8_t s_cvx[kStage];
    __shared__ uint32_t cnt[kPairT], wsum[kPairT / 32 + 1];
    __shared__ uint32_t base;
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (!bactive[bj * bnx + bi]) return;
    const int n = gather_candidates(bi, bj, nx, ny, cell_start, ids, cand, tmp, flags);
    const int ns = min(n, kStage);
    for (int q = threadIdx.x; q < ns; q += kPairT) {
        const uint32_t m = cand[q];
        s_box[q] = sbox[m];
        s_l[0][q] = slf[(long)m * 8 + 0];
        s_l[1][q] = slf[(long)m * 8 + 1];
        s_l[2][q] = slf[(long)m * 8 + 2];
        s_l[3][q] = slf[(long)m * 8 + 7];
        s_cvx[q] = scvx[m];
    }
    __syncthreads();
    const int t = threadIdx.x, cl = t / kPairSub, sub = t - cl * kPairSub;
    const int i = bi * kBlk + (cl % kBlk), j = bj * kBlk + (cl / kBlk);
    const bool live = i < nx && j < ny;
    const float fi = (float)i, fj = (float)j;
    auto meets = [&](int q) {
        const uint32_t m = cand[q];
        const bool st = q < kStage;
        const float4 b = st ? s_box[q] : sbox[m];
        if (b.x > fi + 1.0f || b.y < fi || b.z > fj + 1.0f || b.w < fj) return false;
        if (!(st ? s_cvx[q] : scvx[m])) return true;
        const float4 *L = slf + (long)m * 8;
        return cell_side(st ? s_l[0][q] : L[0], fi, fj) >= 0 &&
               cell_side(st ? s_l[1][q] : L[1], fi, fj) >= 0 &&
               cell_side(st ? s_l[2][q] : L[2], fi, fj) >= 0 &&
               cell_side(st ? s_l[3][q] : L[7], fi, fj) <= 0;
    };
    // this thread's contiguous share of the (ascending) candidate list; its
    // test results are kept as bits in tmp (free after the gathering: four
    // words a thread, word w of thread t at tmp[w * kPairT + t]) for the
    // second pass, when the block has at most 4 x 128 candidates
    const int q0 = (n * sub) / kPairSub, q1 = (n * (sub + 1)) / kPairSub;
    static_assert(kMaxCand >= 4 * kPairT, "four words of tmp per thread");
    const bool keep = n <= kPairSub * 128;
    uint32_t c = 0;
    if (live) {
        uint32_t word = 0;
        for (int q = q0; q < q1; q++) {
            const bool mt = meets(q);
            c += mt ? 1u : 0u;
            if (keep) {
                const int b = q - q0;
                word |= (mt ? 1u : 0u) << (b & 31);
                if ((b & 31) == 31 || q + 1 == q1) { tmp[(b >> 5) * kPairT + t] = word; word = 0; }
            }
        }
    }
    // exclusive scan over threads (cell-major, then share): warp scans, then
    // the warp totals
    const int lane = t & 31, warp = t >> 5;
    uint32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (t == 0) {
        uint32_t acc = 0;
        for (int w = 0; w < kPairT / 32; w++) { const uint32_t v = wsum[w]; wsum[w] = acc; acc += v; }
        wsum[kPairT / 32] = acc;
        const uint32_t b0 = atomicAdd(npairs, acc);
        if (b0 > cap || acc > cap - b0) {
            atomicOr(&flags[1], 1u);
            base = 0xffffffffu;
        } else {
            base = b0;
        }
    }
    __syncthreads();
    const uint32_t excl = wsum[warp] + incl - c;
    cnt[t] = excl;
    __syncthreads();
    if (!live) return;
    const long cidx = (long)j * nx + i;
    if (base == 0xffffffffu) {
        if (sub == 0) crange[cidx] = make_uint2(0u, 0u);
        return;
    }
    if (sub == 0) {
        const uint32_t end = (cl + 1 < kBT) ? cnt[t + kPairSub] : wsum[kPairT / 32];
        crange[cidx] = make_uint2(base + excl, end - excl);
    }
    uint32_t o = base + excl;
    for (int q = q0; q < q1; q++)
        if (keep ? ((tmp[((q - q0) >> 5) * kPairT + t] >> ((q - q0) & 31)) & 1u) : meets(q)) {
            uint32_t seg = cand[q];
            // a pair of a non-convex strip goes to the clip list of
            // k_band_area (while it has room), marked in the id's top bit
            if (!(q < kStage ? s_cvx[q] : scvx[seg])) {
                const uint32_t at = atomicAdd(npairs + 1, 1u);
                if (at < kClipCap) { clip_list[at] = o; seg |= kClipFlag; }
            }
            pseg[o] = seg;
            pcell[o] = (uint32_t)cidx;
            o++;
        }
}

// A bounding line of a strip in the cell's local frame (the cell is the unit
// square [0,1]^2): f(x, y) = a x + b y - c >= 0 inside, (a, b) a unit vector,
// with the reciprocals of a and b (0 where they vanish); on = false makes the
// slot constrain nothing.
struct CellLine {
    double a, b, c, ra, rb;
    bool on;
};

// l: a, b, c, 1/a, 1/b of the line in grid coordinates.
__device__ __forceinline__ CellLine cell_line(const double *l, double di, double dj, bool on)
{
    CellLine L;
    L.a = on ? l[0] : 0.0;
    L.b = on ? l[1] : 0.0;
    L.c = on ? l[2] - l[0] * di - l[1] * dj : -1.0;
    L.ra = on ? l[3] : 0.0;
    L.rb = on ? l[4] : 0.0;
    L.on = on;
    return L;
}

// Comparisons and selections of doubles on their bit patterns, in integer
// instructions: this part issues FP64 compares and min/max on its reduced
// FP64 pipe.  A double's 64-bit key, flipped below zero, orders like the
// number (finite values and infinities; -0 and +0 adjacent), so the maxima
// and minima below select exactly what fmax / fmin would.
__device__ __forceinline__ long long dkey(double x)
{
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool dpos(double x)  // x > 0
{
    return __double_as_longlong(x) > 0;
}
__device__ __forceinline__ bool dneg(double x)  // x < 0
{
    const long long b = __double_as_longlong(x);
    return b < 0 && b != (long long)0x8000000000000000ULL;
}
__device__ __forceinline__ bool dzero(double x)  // x == 0
{
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) == 0;
}
// fmax(x, 0): x if it is positive (finite or +inf), else 0 (also for a NaN,
// as fmax gives for the empty interval -inf - (-inf))
__device__ __forceinline__ double dmax0(double x)
{
    const long long b = __double_as_longlong(x);
    return (b > 0 && b <= 0x7ff0000000000000LL) ? x : 0.0;
}

// Narrow [lo, hi] to the s with alpha + beta s >= 0 (rbeta = 1 / beta).
__device__ __forceinline__ void narrow(double alpha, double beta, double rbeta, double &lo, double &hi)
{
    const double q = -alpha * rbeta;
    if (dpos(beta)) { if (dkey(q) > dkey(lo)) lo = q; }
    else if (dneg(beta)) { if (dkey(q) < dkey(hi)) hi = q; }
    else if (dneg(alpha)) hi = -INFINITY;
}

// Areas of the unit square cut by half-planes, by Green's theorem: area =
// 1/2 of the boundary integral of x dy - y dx.  On the square's bottom and
// left edges the integrand vanishes; the right edge contributes the length
// of its part inside every half-plane, and so does the top edge; a line,
// traversed with its inside on the left from P(s0) to P(s1), P(s) =
// c (a, b) + s (b, -a), contributes (s1 - s0) cross(P(0), (b, -a)) =
// -(s1 - s0) c.  Each piece is an interval cut down by the other
// constraints.  The result equals clipping the square by the half-planes in
// turn and taking the shoelace area, up to rounding.
//
// A cell meets the two normal edges of a segment and one offset line at a
// time: the pieces' intervals under the normal edges alone are formed once
// (RailCut, which also gives the area a0 of the cell between the normal
// edges) and each cutting offset line only narrows them further.

// A line lying on the top or right edge with the square on its inner side
// traces the same boundary as that edge: its own piece is not counted.
__device__ __forceinline__ bool on_edge(const CellLine &L)
{
    return (dzero(L.a) && dneg(L.b) && dzero(L.b - L.c)) || (dzero(L.b) && dneg(L.a) && dzero(L.a - L.c));
}

// Interval of line L's own piece inside the unit square.
__device__ __forceinline__ void square_piece(const CellLine &L, double &lo, double &hi)
{
    const double px = L.c * L.a, py = L.c * L.b;
    lo = -INFINITY; hi = INFINITY;
    narrow(px, L.b, L.rb, lo, hi);              // x >= 0
    narrow(1.0 - px, -L.b, -L.rb, lo, hi);      // x <= 1
    narrow(py, -L.a, -L.ra, lo, hi);            // y >= 0
    narrow(1.0 - py, L.a, L.ra, lo, hi);        // y <= 1
}

// Narrow line J's piece by half-plane I (rIJ = 1 / (a_I b_J - b_I a_J)).
__device__ __forceinline__ void cross_narrow(const CellLine &I, const CellLine &J, double rIJ,
                                             double &lo, double &hi)
{
    const double px = J.c * J.a, py = J.c * J.b;
    narrow(I.a * px + I.b * py - I.c, I.a * J.b - I.b * J.a, rIJ, lo, hi);
}

struct RailCut {
    double Rlo, Rhi, Tlo, Thi;  // right edge (y) and top edge (x) inside both normal edges
    double Plo[2], Phi[2];      // normal-edge pieces (s)
    bool piece[2];              // normal edge j cuts the cell and has a piece of its own
};

// L[0], L[1]: the normal edges (on = cuts the cell); r01 = 1 / D_01.
__device__ __forceinline__ void rail_cut(const CellLine *L, double r01, RailCut &rc)
{
    rc.Rlo = 0.0; rc.Rhi = 1.0; rc.Tlo = 0.0; rc.Thi = 1.0;
#pragma unroll
    for (int j = 0; j < 2; j++) {
        narrow(L[j].a - L[j].c, L[j].b, L[j].rb, rc.Rlo, rc.Rhi);  // x = 1
        narrow(L[j].b - L[j].c, L[j].a, L[j].ra, rc.Tlo, rc.Thi);  // y = 1
    }
#pragma unroll
    for (int j = 0; j < 2; j++) {
        rc.piece[j] = L[j].on && !on_edge(L[j]);
        rc.Plo[j] = 0.0; rc.Phi[j] = 0.0;
        if (!rc.piece[j]) continue;
        square_piece(L[j], rc.Plo[j], rc.Phi[j]);
        if (L[1 - j].on) cross_narrow(L[1 - j], L[j], j == 1 ? r01 : -r01, rc.Plo[j], rc.Phi[j]);
    }
}

// Area of the cell between the normal edges (no offset line).
__device__ __forceinline__ double rail_area(const CellLine *L, const RailCut &rc)
{
    double acc = dmax0(rc.Rhi - rc.Rlo);
    acc += dmax0(rc.Thi - rc.Tlo);
#pragma unroll
    for (int j = 0; j < 2; j++)
        if (rc.piece[j]) acc -= L[j].c * dmax0(rc.Phi[j] - rc.Plo[j]);
    return 0.5 * acc;
}

// Area of the cell between the normal edges and inside offset line O;
// r0O, r1O = 1 / D_0O, 1 / D_1O.
__device__ __forceinline__ double rail_line_area(const CellLine *L, const RailCut &rc,
                                                 const CellLine &O, double r0O, double r1O)
{
    double lo = rc.Rlo, hi = rc.Rhi, acc;
    narrow(O.a - O.c, O.b, O.rb, lo, hi);
    acc = dmax0(hi - lo);
    lo = rc.Tlo; hi = rc.Thi;
    narrow(O.b - O.c, O.a, O.ra, lo, hi);
    acc += dmax0(hi - lo);
#pragma unroll
    for (int j = 0; j < 2; j++) {
        if (!rc.piece[j]) continue;
        lo = rc.Plo[j]; hi = rc.Phi[j];
        cross_narrow(O, L[j], j == 0 ? -r0O : -r1O, lo, hi);  // D_Oj = -D_jO
        acc -= L[j].c * dmax0(hi - lo);
    }
    if (!on_edge(O)) {
        square_piece(O, lo, hi);
#pragma unroll
        for (int i = 0; i < 2; i++)
            if (L[i].on) cross_narrow(L[i], O, i == 0 ? r0O : r1O, lo, hi);
        acc -= O.c * dmax0(hi - lo);
    }
    return 0.5 * acc;
}

// Area of cell (ci, cj) inside each of the five strips of segment m, weighted
// sum and total.  Convex, well-conditioned strips: P is the cell square cut by the slab's normal
// edges that cross it (area a0), S_o = area(P on the inner side of offset line
// o) for o = 0..5 (a0 or 0 when the FP32 test finds the line clear of the
// cell, else rail_line_area in FP64, the cut lines in ascending o), and strip
// k has area S_k - S_k+1.  Other
// segments (folded strips, lines within 0.001 rad of a grid axis): each
// quadrilateral is clipped against the cell (Sutherland-Hodgman).
__device__ __forceinline__ void pair_area(uint32_t m, int ci, int cj, const double *__restrict__ sl,
                                          const float4 *__restrict__ slf,
                                          const uint8_t *__restrict__ scvx,
                                          const double *__restrict__ sv,
                                          const float4 *__restrict__ sb5, const double *Hk,
                                          double &acc, double &cov)
{
    const float gi = (float)ci, gj = (float)cj;
    const double di = (double)ci, dj = (double)cj;
    acc = 0.0;
    cov = 0.0;
    if (!scvx[m]) {
        const double *v = sv + (long)m * 24;
        for (int k = 0; k < 5; k++) {
            const float4 b = sb5[(long)m * 5 + k];
            if (b.x > gi + 1.0f || b.y < gi || b.z > gj + 1.0f || b.w < gj) continue;
            double qx[4], qy[4];
            qx[0] = v[2 * k] - di;            qy[0] = v[2 * k + 1] - dj;
            qx[1] = v[12 + 2 * k] - di;       qy[1] = v[12 + 2 * k + 1] - dj;
            qx[2] = v[12 + 2 * k + 2] - di;   qy[2] = v[12 + 2 * k + 3] - dj;
            qx[3] = v[2 * k + 2] - di;        qy[3] = v[2 * k + 3] - dj;
            const double A = clip_area_unit(qx, qy);
            acc += A * Hk[k];
            cov += A;
        }
        return;
    }
    const float4 *Lf = slf + (long)m * 8;
    const double *Ld = sl + (long)m * kSegLine;
    int side[8];
#pragma unroll
    for (int q = 0; q < 8; q++) side[q] = cell_side(Lf[q], gi, gj);
    // the normal edges; one that does not cut the cell constrains nothing
    CellLine L[2];
#pragma unroll
    for (int q = 0; q < 2; q++) L[q] = cell_line(Ld + 5 * q, di, dj, side[q] == 0);
    RailCut rc;
    rail_cut(L, Ld[40], rc);
    const double a0 = (side[0] == 0 || side[1] == 0) ? rail_area(L, rc) : 1.0;
    // lines clear of the cell first; then the cut ones, lowest first: step
    // k of the loop takes the k-th cut line of every lane's pair, so the
    // FP64 area runs on converged warps whichever lines the pairs cut
    double S[6];
    unsigned cut = 0;
#pragma unroll
    for (int o = 0; o < 6; o++) {
        S[o] = side[2 + o] > 0 ? a0 : 0.0;
        if (side[2 + o] == 0) cut |= 1u << o;
    }
    while (cut) {
        const int o = __ffs(cut) - 1;
        cut &= cut - 1;
        const CellLine O = cell_line(Ld + 5 * (2 + o), di, dj, true);
        const double v = rail_line_area(L, rc, O, Ld[41 + 2 * o], Ld[42 + 2 * o]);
#pragma unroll
        for (int r = 0; r < 6; r++)
            if (r == o) S[r] = v;
    }
#pragma unroll
    for (int k = 0; k < 5; k++) {
        const double A = S[k] - S[k + 1];
        acc += A * Hk[k];
        cov += A;
    }
}

// The first kClipBlocks blocks take the listed pairs of non-convex strips,
// a group of 8 lanes per pair, lane k < 5 clipping strip k's quadrilateral;
// lane 0 sums the strips in order, as one thread would.  Being dispatched
// first, their long FP64 chains overlap the rest.  The other blocks take one
// pair per thread (flat over the list), skipping the listed ones.
__global__ void __launch_bounds__(256)
k_band_area(int nx, const uint32_t *__restrict__ npairs, uint32_t cap,
            const uint32_t *__restrict__ pseg, const uint32_t *__restrict__ pcell,
            const uint32_t *__restrict__ clip_list,
            const double *__restrict__ sl, const float4 *__restrict__ slf,
            const uint8_t *__restrict__ scvx, const double *__restrict__ sv,
            const float4 *__restrict__ sb5, double *__restrict__ pacc, double *__restrict__ pcov)
{
    const uint32_t total = min(*npairs, cap);
    double Hk[5];
    for (int k = 0; k < 5; k++) Hk[k] = strip_value(k);
    if (blockIdx.x < kClipBlocks) {
        const uint32_t nc = min(npairs[1], (uint32_t)kClipCap);
        const uint32_t idx = blockIdx.x * 32 + threadIdx.x / 8;
        const int k = threadIdx.x % 8;
        // every lane reaches the shuffles below; a group past the list's end
        // (the same for its 8 lanes) only does no work
        const bool live = idx < nc;
        const uint32_t p = live ? clip_list[idx] : 0u;
        const uint32_t m = live ? (pseg[p] & ~kClipFlag) : 0u, cell = live ? pcell[p] : 0u;
        const int cj = (int)(cell / (uint32_t)nx), ci = (int)(cell - (uint32_t)cj * (uint32_t)nx);
        const float gi = (float)ci, gj = (float)cj;
        const double di = (double)ci, dj = (double)cj;
        double A = 0.0;
        bool hit = false;
        if (live && k < 5) {
            const float4 bb = sb5[(long)m * 5 + k];
            hit = !(bb.x > gi + 1.0f || bb.y < gi || bb.z > gj + 1.0f || bb.w < gj);
            if (hit) {
                const double *v = sv + (long)m * 24;
                double qx[4], qy[4];
                qx[0] = v[2 * k] - di;            qy[0] = v[2 * k + 1] - dj;
                qx[1] = v[12 + 2 * k] - di;       qy[1] = v[12 + 2 * k + 1] - dj;
                qx[2] = v[12 + 2 * k + 2] - di;   qy[2] = v[12 + 2 * k + 3] - dj;
                qx[3] = v[2 * k + 2] - di;        qy[3] = v[2 * k + 3] - dj;
                A = clip_area_unit(qx, qy);
            }
        }
        double acc = 0.0, cov = 0.0;
        const int g0 = (threadIdx.x & 31) & ~7;  // the group's first lane
#pragma unroll
        for (int s = 0; s < 5; s++) {
            const double As = __shfl_sync(0xffffffffu, A, g0 + s);
            const bool hs = __shfl_sync(0xffffffffu, hit, g0 + s);
            if (hs) { acc += As * Hk[s]; cov += As; }
        }
        if (live && k == 0) { pacc[p] = acc; pcov[p] = cov; }
        return;
    }
    const uint32_t stride = (gridDim.x - kClipBlocks) * blockDim.x;
    for (uint32_t p = (blockIdx.x - kClipBlocks) * blockDim.x + threadIdx.x; p < total; p += stride) {
        const uint32_t seg = pseg[p];
        if (seg & kClipFlag) continue;
        const uint32_t cell = pcell[p];
        const int cj = (int)(cell / (uint32_t)nx), ci = (int)(cell - (uint32_t)cj * (uint32_t)nx);
        double acc, cov;
        pair_area(seg, ci, cj, sl, slf, scvx, sv, sb5, Hk, acc, cov);
        pacc[p] = acc;
        pcov[p] = cov;
    }
}

__global__ void __launch_bounds__(kBT)
k_band_sum(int nx, int ny, int bnx, const uint32_t *__restrict__ bactive,
           const uint2 *__restrict__ crange, const double *__restrict__ pacc,
           const double *__restrict__ pcov, double *__restrict__ H)
{
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (!bactive[bj * bnx + bi]) return;
    const int i = bi * kBlk + (threadIdx.x % kBlk), j = bj * kBlk + (threadIdx.x / kBlk);
    if (i >= nx || j >= ny) return;
    const long cidx = (long)j * nx + i;
    const uint2 r = crange[cidx];
    double acc = 0.0, cov = 0.0;
    for (uint32_t p = r.x; p < r.x + r.y; p++) { acc += pacc[p]; cov += pcov[p]; }
    double unc = 1.0 - cov;
    if (unc < 0.0) unc = 0.0;
    H[cidx] = acc + unc * H[cidx];
}

// Irrotational face force F = f_face (H_ij - H_nb) / h on the x-face left of
// and the y-face below every cell of an active block; f_face from the nearest
// segment (closest point clamped to the segment, ties to the lower id),
// linear in the segment parameter between its two markers.  One thread per
// face: the block's 128 faces are tested for dH != 0, the faces with work
// are packed into a list (so the FP64 part runs on full warps), and each of
// those screens the block's candidates (staged in shared memory in FP32),
// lists the survivors in ascending id and then evaluates them exactly in
// FP64 in that order: step k of the evaluation takes the k-th survivor of
// every face at once, so the FP64 instructions run on converged warps (a
// face with more than kNear survivors evaluates them in a pass of its own).
constexpr int kIrrT = 2 * kBT;  // one thread per face of the block
constexpr int kNear = 8;        // survivors listed per face
__global__ void __launch_bounds__(kIrrT)
k_spread_irrot(int nx, int ny, double ih, int bnx, const uint32_t *__restrict__ bactive,
               const uint32_t *__restrict__ cell_start, const uint32_t *__restrict__ ids,
               const int32_t *__restrict__ next, const double *__restrict__ gx,
               const double *__restrict__ gy, const double *__restrict__ sinv,
               const float *__restrict__ gxf, const float *__restrict__ gyf,
               const double *__restrict__ fmag, const double *__restrict__ H,
               double *__restrict__ Fx, double *__restrict__ Fy, uint32_t *__restrict__ flags)
{
    __shared__ uint32_t cand[kMaxCand], tmp[kMaxCand];
    __shared__ float4 seg[kMaxCand];   // FP32 candidate segments: start, direction
    __shared__ float seg_il[kMaxCand]; // 1 / |direction|^2
    __shared__ uint8_t work[kIrrT];     // faces with dH != 0, packed
    __shared__ double wdH[kIrrT];
    __shared__ uint16_t near_q[kNear][kIrrT];  // survivors of the FP32 screen, per face
    __shared__ int nwork;
    const int bi = blockIdx.x, bj = blockIdx.y;
    if (!bactive[bj * bnx + bi]) return;
    const int n = gather_candidates(bi, bj, nx, ny, cell_start, ids, cand, tmp, flags);
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int m = (int)cand[q], nm = next[m];
        const float ax = gxf[m], ay = gyf[m], ex = gxf[nm] - ax, ey = gyf[nm] - ay;
        seg[q] = make_float4(ax, ay, ex, ey);
        seg_il[q] = 1.0f / (ex * ex + ey * ey);
    }
    if (threadIdx.x == 0) nwork = 0;
    __syncthreads();
    // face f: dir = f / 64 (0: x-face left of the cell, 1: y-face below), cell f % 64
    auto face = [&](int f, int &dir, int &i, int &j) {
        dir = f / kBT;
        const int c = f - dir * kBT;
        i = bi * kBlk + (c % kBlk);
        j = bj * kBlk + (c / kBlk);
    };
    {
        const int f = threadIdx.x;
        int dir, i, j;
        face(f, dir, i, j);
        if (i < nx && j < ny && !(dir == 0 && i == 0) && !(dir == 1 && j == 0)) {
            const double dH = dir == 0 ? H[(long)j * nx + i] - H[(long)j * nx + i - 1]
                                       : H[(long)j * nx + i] - H[(long)(j - 1) * nx + i];
            if (dH != 0.0) {
                const int w = atomicAdd(&nwork, 1);
                work[w] = (uint8_t)f;
                wdH[w] = dH;
            } else if (dir == 0) {
                Fx[(long)j * (nx + 1) + i] = 0.0;
            } else {
                Fy[(long)j * nx + i] = 0.0;
            }
        }
    }
    __syncthreads();
    if ((int)threadIdx.x >= nwork) return;
    int dir, i, j;
    face(work[threadIdx.x], dir, i, j);
    const double dH = wdH[threadIdx.x];
    const double qx = dir == 0 ? (double)i : (double)i + 0.5;
    const double qy = dir == 0 ? (double)j + 0.5 : (double)j;
    // FP32 screen: for faces within the band (distance below ~4 cells) and
    // coordinates below 2^12 cells the FP32 squared distances carry an error
    // below 2e-3 (grid units), so the exact nearest segment is among those
    // within best + 0.01 of the FP32 minimum.
    const float fqx = d2f_rn(qx), fqy = d2f_rn(qy);
    auto d2f = [&](int q) {
        const float4 sg = seg[q];
        float t = ((fqx - sg.x) * sg.z + (fqy - sg.y) * sg.w) * seg_il[q];
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        const float dx = sg.x + t * sg.z - fqx, dy = sg.y + t * sg.w - fqy;
        return dx * dx + dy * dy;
    };
    float best32 = INFINITY;
    for (int q = 0; q < n; q++) best32 = fminf(best32, d2f(q));
    const float lim = best32 + 0.01f;
    static_assert(kMaxCand <= 65536, "candidate index in 16 bits");
    int cnt = 0;
    for (int q = 0; q < n; q++)
        if (!(d2f(q) > lim)) {
            if (cnt < kNear) near_q[cnt][threadIdx.x] = (uint16_t)q;
            cnt++;
        }
    double best = INFINITY, fb = 0.0;
    auto eval = [&](int q) {
        const int m = (int)cand[q], nm = next[m];
        const double ax = gx[m], ay = gy[m];
        const double ex = gx[nm] - ax, ey = gy[nm] - ay;
        double t = ((qx - ax) * ex + (qy - ay) * ey) * sinv[m];
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
        const double dx = ax + t * ex - qx, dy = ay + t * ey - qy;
        const double d2 = dx * dx + dy * dy;
        if (d2 < best) { best = d2; fb = (1.0 - t) * fmag[m] + t * fmag[nm]; }
    };
    if (cnt <= kNear) {
        for (int k = 0; k < cnt; k++) eval(near_q[k][threadIdx.x]);
    } else {
        for (int q = 0; q < n; q++)
            if (!(d2f(q) > lim)) eval(q);
    }
    const double F = fb * dH * ih;
    if (dir == 0) Fx[(long)j * (nx + 1) + i] = F;
    else Fy[(long)j * nx + i] = F;
}

// ------------------------------------------------------------ B-spline
// Section 4: relocation along a periodic cubic B-spline fitted to each drop
// by least squares.  Same steps as the definition: chord-length parameters,
// g = round(L / 1.5h) spans (4 <= g <= n), normal equations accumulated in
// ascending marker order, Cholesky in the matrix's envelope (band of 3 plus
// the last three rows, which is where the cyclic wrap fills in), arc length
// by 8-point Gauss-Legendre per span, 12 Newton steps per new marker.  Two
// kernels: the fit (one CTA per drop) and the placement of the new markers
// (one thread per marker over the whole grid).
// The basis follows the same arithmetic as a serial program: the span of a
// parameter is floor(s / tau) and the weights come from the Cox-de Boor
// recursion on knots t_k = k tau, so that relocated markers agree with it to
// rounding of the same operations.
__device__ __forceinline__ int bspl_span(double s, double tau, int g)
{
    int q = (int)floor(s / tau);
    if (q > g - 1) q = g - 1;
    if (q < 0) q = 0;
    return q;
}

__device__ void bspl_basis(double s, double tau, int g, int *idx, double *w, double *dw)
{
    const int q = bspl_span(s, tau, g);
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
        double a = (r >= 1) ? N[2][r - 1] : 0.0;
        double b = (r <= 2) ? N[2][r] : 0.0;
        dw[r] = 3.0 / (3.0 * tau) * a - 3.0 / (3.0 * tau) * b;
    }
}

__constant__ double cGLX[8] = {-0.9602898564975363, -0.7966664774136267,
                               -0.5255324099163290, -0.1834346424956498,
                               0.1834346424956498,  0.5255324099163290,
                               0.7966664774136267,  0.9602898564975363};
__constant__ double cGLW[8] = {0.1012285362903763, 0.2223810344533745,
                               0.3137066458778873, 0.3626837833783620,
                               0.3626837833783620, 0.3137066458778873,
                               0.2223810344533745, 0.1012285362903763};

// The same basis in closed form.  The knots t_k = k tau are uniform, so on
// span q (u = s / tau - q in [0, 1]) the four cubic B-splines that do not
// vanish, of control points q-3 .. q, are the uniform ones:
// (1-u)^3/6, (3u^3 - 6u^2 + 4)/6, (-3u^3 + 3u^2 + 3u + 1)/6, u^3/6, and their
// derivatives in s are these polynomials' derivatives over tau.  The
// recursion above gives the same functions with about eight times the FP64
// operations (a dozen divisions); the Newton placement evaluates the speed
// ~100 times per marker, so it uses this form (the values agree to
// rounding).  The span is floor(s / tau) clamped to [0, g-1], found from
// s (1/tau): at a knot either neighbouring span gives the same value and
// first derivative (the curve is C^2).
struct SpanU {
    int i0, i1, i2, i3;  // control points q-3 .. q (cyclic)
    double u;
};
__device__ __forceinline__ SpanU bspl_span_u(double s, double itau, int g)
{
    const double x = s * itau;
    int q = (int)floor(x);
    q = q > g - 1 ? g - 1 : (q < 0 ? 0 : q);
    SpanU r;
    r.u = x - (double)q;
    const int k = q - 3;  // >= -3, and q <= g - 1
    r.i0 = k < 0 ? k + g : k;
    r.i1 = k + 1 < 0 ? k + 1 + g : k + 1;
    r.i2 = k + 2 < 0 ? k + 2 + g : k + 2;
    r.i3 = q;
    return r;
}

__device__ double bspl_speed(double s, double tau, int g, const double *cx, const double *cy)
{
    const double itau = 1.0 / tau;
    const SpanU p = bspl_span_u(s, itau, g);
    const double u = p.u, v = 1.0 - u;
    // twice the derivatives in u: -(1-u)^2, 3u^2 - 4u, -3u^2 + 2u + 1, u^2
    const double d0 = -v * v, d1 = u * (3.0 * u - 4.0), d2 = fma(u, 2.0 - 3.0 * u, 1.0), d3 = u * u;
    const double dx = d0 * cx[p.i0] + d1 * cx[p.i1] + d2 * cx[p.i2] + d3 * cx[p.i3];
    const double dy = d0 * cy[p.i0] + d1 * cy[p.i1] + d2 * cy[p.i2] + d3 * cy[p.i3];
    return 0.5 * itau * sqrt(dx * dx + dy * dy);
}

// The curve's point at s (closed form, as bspl_speed).
__device__ void bspl_point(double s, double tau, int g, const double *cx, const double *cy,
                           double &px, double &py)
{
    const SpanU p = bspl_span_u(s, 1.0 / tau, g);
    const double u = p.u, v = 1.0 - u, u2 = u * u, u3 = u2 * u;
    const double b0 = v * v * v, b1 = fma(3.0, u3, fma(-6.0, u2, 4.0));
    const double b2 = fma(-3.0, u3, fma(3.0, u2, fma(3.0, u, 1.0))), b3 = u3;
    const double s6 = 1.0 / 6.0;
    px = s6 * (b0 * cx[p.i0] + b1 * cx[p.i1] + b2 * cx[p.i2] + b3 * cx[p.i3]);
    py = s6 * (b0 * cy[p.i0] + b1 * cy[p.i1] + b2 * cy[p.i2] + b3 * cy[p.i3]);
}

__device__ double gl_len(double a, double b, double tau, int g, const double *cx, const double *cy)
{
    double mid = 0.5 * (a + b), half = 0.5 * (b - a), s = 0.0;
    for (int k = 0; k < 8; k++) s += cGLW[k] * bspl_speed(mid + half * cGLX[k], tau, g, cx, cy);
    return s * half;
}

struct Env {
    // L (lower Cholesky factor) in its envelope: band rows r in [3, g-3) keep
    // columns r-3..r, the other rows are dense.
    int g;
    double *band, *dense;
    __device__ bool is_band(int r) const { return r >= 3 && r < g - 3; }
    __device__ int dense_row(int r) const { return r < 3 ? r : 3 + (r - (g - 3)); }
    __device__ int first(int r) const { return is_band(r) ? r - 3 : 0; }
    __device__ double get(int r, int c) const {
        if (is_band(r)) return (c >= r - 3 && c <= r) ? band[r * 4 + (c - r + 3)] : 0.0;
        return dense[(long)dense_row(r) * g + c];
    }
    __device__ void set(int r, int c, double v) {
        if (is_band(r)) band[r * 4 + (c - r + 3)] = v;
        else dense[(long)dense_row(r) * g + c] = v;
    }
};

// G[r][c] of the cyclic band matrix stored as Gc[i*4 + d] = G[i][(i+d) mod g].
__device__ double gval(const double *Gc, int g, int r, int c)
{
    int d1 = ((c - r) % g + g) % g, d2 = ((r - c) % g + g) % g;
    if (d1 <= 3) return Gc[r * 4 + d1];
    if (d2 <= 3) return Gc[c * 4 + d2];
    return 0.0;
}

// Cholesky factorisation in the envelope by warp 0 (lane t of 32), each
// entry by the sums of a dense Cholesky in ascending order: per column c,
// lane 0 takes the diagonal while lanes 1..6 take the envelope rows below it
// (c+1..c+3 and the dense last three rows), whose sums need only earlier
// columns; they are then scaled by the diagonal's reciprocal, which is kept
// in rinv[c] for the substitutions.  The columns are a serial chain of FP64
// latencies on this part (a division costs about 1.5 k cycles there), so
// the reciprocal comes from rsqrt_nr (FP32 seed, two Newton steps), the
// diagonal is s times it, and the entries multiply by it.  Returns -1 (in every lane) if not positive
// definite.
__device__ int env_factor(Env &L, const double *Gc, int g, int t, double *rinv)
{
    for (int c = 0; c < g; c++) {
        // envelope row of lane t (t >= 1): the (t-1)-th of the ascending walk
        int r = -1;
        if (t >= 1 && t <= 6) {
            int k = 0;
            for (int q = c + 1; q < g; q = (q == c + 3 && q + 1 < g - 3) ? g - 3 : q + 1) {
                if (L.is_band(q) && q - 3 > c) continue;
                if (++k == t) { r = q; break; }
            }
        }
        double acc = 0.0;
        if (c >= g - 3 && c > 32) {
            // the last columns: the diagonal and the (dense) rows below have
            // sums over all earlier columns; the warp takes them in strided
            // partial sums and a shuffle tree (the same total in every lane)
            double pd = 0.0, p1 = 0.0, p2 = 0.0;
            for (int k = t; k < c; k += 32) {
                const double lc = L.get(c, k);
                pd += lc * lc;
                if (c + 1 < g) p1 += L.get(c + 1, k) * lc;
                if (c + 2 < g) p2 += L.get(c + 2, k) * lc;
            }
            for (int o = 16; o; o >>= 1) {
                pd += __shfl_xor_sync(0xffffffffu, pd, o);
                p1 += __shfl_xor_sync(0xffffffffu, p1, o);
                p2 += __shfl_xor_sync(0xffffffffu, p2, o);
            }
            // rows c + 1, c + 2 are the walk's first two: lanes 1 and 2
            if (t == 0) acc = gval(Gc, g, c, c) - pd;
            else if (r == c + 1) acc = gval(Gc, g, r, c) - p1;
            else if (r == c + 2) acc = gval(Gc, g, r, c) - p2;
        } else {
            // lane 0 the diagonal (its row is c), lanes 1..6 the rows below:
            // one code path, so the same FP64 warp instructions serve all
            // (on this part they cost the same for one lane as for 32)
            const int rr = t == 0 ? c : r;
            if (rr >= 0) {
                acc = gval(Gc, g, rr, c);
                for (int k = max(L.first(rr), L.first(c)); k < c; k++) acc -= L.get(rr, k) * L.get(c, k);
            }
        }
        const double s = __shfl_sync(0xffffffffu, acc, 0);
        if (!(s > 0.0)) return -1;
        // the diagonal d = sqrt(s) and its reciprocal from one reciprocal
        // square root (a shorter chain than a square root and a reciprocal)
        const bool fast = s > 1e-30 && s < 1e30;
        const double rd = fast ? rsqrt_nr(s) : 1.0 / sqrt(s);
        const double d = fast ? s * rd : sqrt(s);
        if (t == 0) { L.set(c, c, d); rinv[c] = rd; }
        else if (r >= 0) L.set(r, c, acc * rd);
        __syncwarp();
    }
    return 0;
}

// L L^T x = b for the two right-hand sides bx, by (in place) by warp 0
// (lane t): every lane runs the serial substitution, lane 0 stores each
// entry; the long sums of the dense last rows go to the whole warp (strided
// partial sums and a shuffle tree); scaling by the diagonal's reciprocals
// rinv (no division on the serial chain).
__device__ void env_subst(const Env &L, int g, const double *rinv, double *bx, double *by, int t)
{
    // Even lanes take the x right-hand side, odd lanes the y one, so that
    // one warp instruction advances both: on this part an FP64 warp
    // instruction occupies the FP64 unit as long for one lane as for 32, and
    // the passes are chains of them.  Each lane keeps its side's latest
    // three entries (and, backwards, the dense last rows') in registers;
    // lanes 0 and 1 store them for the long sums and the other pass, after
    // one warp barrier a row (every lane has read the row's right-hand side).
    double *b = (t & 1) ? by : bx;
    double x1 = 0.0, x2 = 0.0, x3 = 0.0;  // rows r-1, r-2, r-3
    for (int r = 0; r < g; r++) {
        double s = b[r];
        const int k0 = L.first(r);
        if (r - k0 > 3) {
            // a dense last row: all earlier entries, from shared memory
            __syncwarp();
            if (r - k0 > 32) {
                double ps = 0.0, pu = 0.0;
                for (int k = k0 + t; k < r; k += 32) { const double l = L.get(r, k); ps += l * bx[k]; pu += l * by[k]; }
                for (int o = 16; o; o >>= 1) {
                    ps += __shfl_xor_sync(0xffffffffu, ps, o);
                    pu += __shfl_xor_sync(0xffffffffu, pu, o);
                }
                s -= (t & 1) ? pu : ps;
            } else {
                for (int k = k0; k < r; k++) s -= L.get(r, k) * b[k];
            }
        } else {
            for (int k = k0; k < r; k++) {  // ascending k, the last (at most) three rows
                const int back = r - k;
                s -= L.get(r, k) * (back == 1 ? x1 : (back == 2 ? x2 : x3));
            }
        }
        s *= rinv[r];
        __syncwarp();
        if (t < 2) b[r] = s;
        x3 = x2; x2 = x1; x1 = s;
    }
    __syncwarp();
    double f1 = 0.0, f2 = 0.0, f3 = 0.0;  // rows r+1, r+2, r+3
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;  // rows g-3, g-2, g-1
    for (int r = g - 1; r >= 0; r--) {
        double s = b[r];
        for (int k = r + 1; k < g; k = (k == r + 3 && k + 1 < g - 3) ? g - 3 : k + 1) {
            if (L.is_band(k) && k - 3 > r) continue;
            double xv;
            if (k - r <= 3) {
                const int back = k - r;
                xv = back == 1 ? f1 : (back == 2 ? f2 : f3);
            } else {  // k >= g - 3
                const int q = k - (g - 3);
                xv = q == 0 ? t0 : (q == 1 ? t1 : t2);
            }
            s -= L.get(k, r) * xv;
        }
        s *= rinv[r];
        __syncwarp();
        if (t < 2) b[r] = s;
        f3 = f2; f2 = f1; f1 = s;
        if (r == g - 1) t2 = s;
        else if (r == g - 2) t1 = s;
        else if (r == g - 3) t0 = s;
    }
}

// Per-drop fit results: at offset 3 * s0 + d of fit (s0 the drop's first
// marker, n its markers, g <= n) the control points cx[g], cy[g] and the
// cumulative arc length at the knots cum[g + 1]; par[4d .. 4d+3] = (g, tau,
// total arc length, failed).
__device__ __forceinline__ long fit_base(int s0, int d) { return 3L * s0 + d; }

__global__ void __launch_bounds__(kT)
k_reloc_fit(const double *__restrict__ X, const double *__restrict__ Y,
            const int32_t *__restrict__ drop_start, double h, int maxn,
            double *__restrict__ fit, double *__restrict__ par, double *__restrict__ wts,
            uint32_t *__restrict__ flags)
{
    extern __shared__ double sm[];
    const int d = blockIdx.x, s0 = drop_start[d], n = drop_start[d + 1] - s0;
    // shared layout: sp[n+1], qs[maxg+1] and span[maxn] (ints), Gc[4g],
    // cx[g], cy[g], band[4g], dense[6g], cum[g+1]
    const int maxg = maxn;
    double *sp = sm;
    int *qs = (int *)(sp + maxn + 1);
    int *span = qs + (maxg + 1);
    double *Gc = (double *)(qs + 2 * (maxg + 1));
    double *cx = Gc + 4 * maxg, *cy = cx + maxg, *band = cy + maxg, *dense = band + 4 * maxg;
    double *cum = dense + 6 * maxg;
    __shared__ int g_s, bad;
    __shared__ double tau_s;
    // chord lengths in parallel (cx as scratch), their running sum in marker
    // order by one thread
    for (int m = threadIdx.x; m < n; m += kT) {
        const int a = s0 + m, b = s0 + (m + 1 == n ? 0 : m + 1);
        const double dx = X[b] - X[a], dy = Y[b] - Y[a];
        cx[m] = sqrt(dx * dx + dy * dy);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double L = 0.0;
        for (int m = 0; m < n; m++) {
            sp[m] = L;
            L += cx[m];
        }
        int g = (int)floor(L / (1.5 * h) + 0.5);
        if (g < 4) g = 4;
        if (g > n) g = n;
        g_s = g;
        tau_s = L / g;
        bad = 0;
    }
    __syncthreads();
    const int g = g_s;
    const double tau = tau_s;
    // each marker's span and basis weights once (wts, 4 per marker); the
    // first marker of every span (parameters ascend with m): qs[k] is the
    // first marker of span >= k, n if none
    for (int m = threadIdx.x; m < n; m += kT) {
        int idx[4];
        double w[4], dw[4];
        bspl_basis(sp[m], tau, g, idx, w, dw);
        span[m] = bspl_span(sp[m], tau, g);
        for (int r = 0; r < 4; r++) wts[4L * (s0 + m) + r] = w[r];
    }
    __syncthreads();
    for (int m = threadIdx.x; m < n; m += kT) {
        const int lo = m == 0 ? 0 : span[m - 1] + 1;
        for (int k = lo; k <= span[m]; k++) qs[k] = m;
    }
    for (int k = span[n - 1] + 1 + threadIdx.x; k <= g; k += kT) qs[k] = n;
    __syncthreads();
    // normal equations: entry (i, i+d) and rhs i, markers of spans i..i+3 in
    // ascending marker order
    for (int e = threadIdx.x; e < 5 * g; e += kT) {
        int i = e / 5, dd = e % 5;  // dd 0..3: G[i][(i+dd)%g]; dd 4: rhs row i
        int sp4[4];
        for (int t = 0; t < 4; t++) sp4[t] = (i + t) % g;
        for (int a = 1; a < 4; a++)
            for (int b = a; b > 0 && sp4[b] < sp4[b - 1]; b--) { int tt = sp4[b]; sp4[b] = sp4[b - 1]; sp4[b - 1] = tt; }
        int jcol = (i + (dd < 4 ? dd : 0)) % g;
        double acc = 0.0, accy = 0.0;
        for (int t = 0; t < 4; t++) {
            if (t > 0 && sp4[t] == sp4[t - 1]) continue;
            for (int m = qs[sp4[t]]; m < qs[sp4[t] + 1]; m++) {
                const double *w = wts + 4L * (s0 + m);
                int a = -1, b = -1;
                for (int r = 0; r < 4; r++) {
                    const int k = span[m] - 3 + r, id = ((k % g) + g) % g;
                    if (id == i) a = r;
                    if (id == jcol) b = r;
                }
                if (a < 0) continue;
                if (dd < 4) { if (b >= 0) acc += w[a] * w[b]; }
                else { acc += w[a] * X[s0 + m]; accy += w[a] * Y[s0 + m]; }
            }
        }
        if (dd < 4) Gc[i * 4 + dd] = acc;
        else { cx[i] = acc; cy[i] = accy; }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        Env L{g, band, dense};
        // cum holds the diagonal's reciprocals until the arc lengths below
        const int f = env_factor(L, Gc, g, threadIdx.x, cum);  // the same in every lane
        if (f != 0) {
            if (threadIdx.x == 0) bad = 1;
        } else {
            env_subst(L, g, cum, cx, cy, threadIdx.x);
        }
    }
    __syncthreads();
    double *out = fit + fit_base(s0, d);
    if (bad) {
        if (threadIdx.x == 0) {
            atomicOr(&flags[2], 1u);
            par[4 * d] = (double)g; par[4 * d + 1] = tau; par[4 * d + 2] = 0.0; par[4 * d + 3] = 1.0;
        }
        return;
    }
    for (int q = threadIdx.x; q < g; q += kT) cum[q + 1] = gl_len(q * tau, (q + 1) * tau, tau, g, cx, cy);
    __syncthreads();
    if (threadIdx.x == 0) {
        cum[0] = 0.0;
        for (int q = 0; q < g; q++) cum[q + 1] = cum[q] + cum[q + 1];
        par[4 * d] = (double)g; par[4 * d + 1] = tau; par[4 * d + 2] = cum[g]; par[4 * d + 3] = 0.0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < g; q += kT) { out[q] = cx[q]; out[n + q] = cy[q]; }
    for (int q = threadIdx.x; q <= g; q += kT) out[2 * n + q] = cum[q];
}

// New marker m of its drop at arc length L m / n along the fitted curve: the
// span by bisection of the knot arc lengths, then 12 Newton steps on the
// partial arc length, kept in the span.  With LN = 8 lanes per marker (few
// markers: the FP64 latency of one thread's steps dominates), lane k
// evaluates the k-th Gauss-Legendre term of the partial arc length and lane
// 0 also the speed at s; every lane then sums the eight terms in order, so
// all lanes carry the same s.  With LN = 1 (many markers: FP64 throughput
// dominates) one thread does all.  A drop whose fit failed keeps its markers.
constexpr int kPlaceT = 64;
template <int LN>
__global__ void __launch_bounds__(kPlaceT)
k_reloc_place(int M, const double *__restrict__ X, const double *__restrict__ Y,
              const int32_t *__restrict__ drop_of, const int32_t *__restrict__ drop_start,
              const double *__restrict__ fit, const double *__restrict__ par,
              double *__restrict__ Xo, double *__restrict__ Yo)
{
    const int lane = LN == 8 ? (threadIdx.x & 7) : 0, tid = blockIdx.x * kPlaceT + threadIdx.x;
    const int j = LN == 8 ? tid >> 3 : tid;
    const unsigned grp = 0xffu << (threadIdx.x & 24);  // the eight lanes of this marker
    if (j >= M) return;  // whole groups leave together (groups of LN lanes)
    const int d = drop_of[j], s0 = drop_start[d], n = drop_start[d + 1] - s0, m = j - s0;
    if (par[4 * d + 3] != 0.0) {
        if (lane == 0) { Xo[j] = X[j]; Yo[j] = Y[j]; }
        return;
    }
    const int g = (int)par[4 * d];
    const double tau = par[4 * d + 1], Lp = par[4 * d + 2];
    const double *cx = fit + fit_base(s0, d), *cy = cx + n, *cum = cx + 2 * n;
    const double target = Lp * (double)m / (double)n;
    int lo = 0, hi = g - 1;  // largest q <= g-1 with cum[q] <= target
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cum[mid] <= target) lo = mid; else hi = mid - 1;
    }
    const int q = lo;
    const double a = q * tau, b = (q + 1) * tau;
    const double seg = cum[q + 1] - cum[q];
    double s = a + tau * (target - cum[q]) / seg;
    for (int it = 0; it < 12; it++) {
        if constexpr (LN == 1) {
            const double f = cum[q] + gl_len(a, s, tau, g, cx, cy) - target;
            const double sp_ = bspl_speed(s, tau, g, cx, cy);
            s -= f / sp_;
            if (s < a) s = a;
            if (s > b) s = b;
            continue;
        }
        // cum[q] + gl_len(a, s) - target, the Gauss-Legendre sum as gl_len
        const double mid = 0.5 * (a + s), half = 0.5 * (s - a);
        const double term = cGLW[lane] * bspl_speed(mid + half * cGLX[lane], tau, g, cx, cy);
        const double sp_ = lane == 0 ? bspl_speed(s, tau, g, cx, cy) : 0.0;
        double sum = 0.0;
        for (int k = 0; k < 8; k++) sum += __shfl_sync(grp, term, k, 8);
        const double f = cum[q] + sum * half - target;
        s -= f / __shfl_sync(grp, sp_, 0, 8);
        if (s < a) s = a;
        if (s > b) s = b;
    }
    if (lane != 0) return;
    double px, py;
    bspl_point(s, tau, g, cx, cy, px, py);
    Xo[j] = px;
    Yo[j] = py;
}

}  // namespace

// --------------------------------------------------------------------- host
static size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

cudaError_t markers_alloc(Markers &mk, int M, int ndrops, int nx, int ny, double h,
                          double x0, double y0, const int32_t *drop_start_host)
{
    mk.M = M; mk.ndrops = ndrops; mk.nx = nx; mk.ny = ny; mk.h = h; mk.x0 = x0; mk.y0 = y0;
    mk.bnx = (nx + kBlk - 1) / kBlk;
    mk.bny = (ny + kBlk - 1) / kBlk;
    mk.drop_start_h.assign(drop_start_host, drop_start_host + ndrops + 1);
    mk.max_drop = 0;
    for (int d = 0; d < ndrops; d++)
        mk.max_drop = std::max(mk.max_drop, drop_start_host[d + 1] - drop_start_host[d]);
    size_t ncell = (size_t)nx * ny, nb = (size_t)mk.bnx * mk.bny;
    size_t nparts = (ncell + kScanChunk - 1) / kScanChunk;
    // (cell, segment) pairs of the band: about (5 + 1) x (segment length + 1)
    // per segment; 64 per segment covers segments up to ~9 cells long.
    const size_t pair_cap = (size_t)M * 64 + 4096;
    mk.pair_cap = (uint32_t)pair_cap;
    size_t bytes = al(M * 8) * 13 + al(M * 4) * 2 + al(M * 16) + al(ndrops * 16) * 2 + al((3 * (size_t)M + ndrops) * 8) + al((size_t)ndrops * 32) + al((size_t)M * 32) +
                   al((size_t)M * 24 * 8) + al((size_t)M * kSegLine * 8) + al((size_t)M * 8 * 16) + al((size_t)M * 5 * 16) + al(M * 8) + al(M) + al(M * 8) +
                   al(64) + al(pair_cap * 4) * 2 + al(pair_cap * 8) * 2 + al(ncell * 8) +
                   al((ndrops + 1) * 4) + al(M * 4) * 5 + al(ncell * 4) +
                   al((ncell + 1) * 4) + al(nparts * 4) + al(nb * 4) * 2 + al(64) +
                   al((size_t)nx * 8) + al((size_t)kClipCap * 4);
    cudaError_t e = cudaMalloc(&mk.mem, bytes);
    if (e != cudaSuccess) { mk.mem = nullptr; return e; }
    char *q = (char *)mk.mem;
    auto take = [&](size_t b) { char *r = q; q += al(b); return (void *)r; };
    mk.X = (double *)take(M * 8); mk.Y = (double *)take(M * 8);
    mk.kappa = (double *)take(M * 8); mk.nxm = (double *)take(M * 8); mk.nym = (double *)take(M * 8);
    mk.ds = (double *)take(M * 8); mk.fmag = (double *)take(M * 8);
    mk.U = (double *)take(M * 8); mk.V = (double *)take(M * 8);
    mk.Xn = (double *)take(M * 8); mk.Yn = (double *)take(M * 8);
    mk.gx = (double *)take(M * 8); mk.gy = (double *)take(M * 8);
    mk.gxf = (float *)take(M * 4); mk.gyf = (float *)take(M * 4);
    mk.sbox = (float4 *)take(M * 16);
    mk.dyr = (double2 *)take(ndrops * 16);
    mk.dyk = (ulonglong2 *)take(ndrops * 16);
    mk.rfit = (double *)take((3 * (size_t)M + ndrops) * 8);
    mk.rpar = (double *)take((size_t)ndrops * 32);
    mk.rwts = (double *)take((size_t)M * 32);
    mk.sv = (double *)take((size_t)M * 24 * 8);
    mk.sl = (double *)take((size_t)M * kSegLine * 8);
    mk.slf = (float4 *)take((size_t)M * 8 * 16);
    mk.sb5 = (float4 *)take((size_t)M * 5 * 16);
    mk.scvx = (uint8_t *)take(M);
    mk.sinv = (double *)take(M * 8);
    mk.npairs = (uint32_t *)take(64);
    mk.pseg = (uint32_t *)take(pair_cap * 4); mk.pcell = (uint32_t *)take(pair_cap * 4);
    mk.pacc = (double *)take(pair_cap * 8); mk.pcov = (double *)take(pair_cap * 8);
    mk.crange = (uint2 *)take(ncell * 8);
    mk.ykey = (unsigned long long *)take(M * 8);
    mk.drop_start = (int32_t *)take((ndrops + 1) * 4);
    mk.drop_of = (int32_t *)take(M * 4);
    mk.next = (int32_t *)take(M * 4);
    mk.key = (uint32_t *)take(M * 4); mk.tmp_ids = (uint32_t *)take(M * 4); mk.ids = (uint32_t *)take(M * 4);
    mk.cell_count = (uint32_t *)take(ncell * 4);
    mk.cell_start = (uint32_t *)take((ncell + 1) * 4);
    mk.scan_part = (uint32_t *)take(nparts * 4);
    mk.bcount = (uint32_t *)take(nb * 4); mk.bactive = (uint32_t *)take(nb * 4);
    mk.flags = (uint32_t *)take(64);
    mk.colkey = (unsigned long long *)take((size_t)nx * 8);
    mk.clip_list = (uint32_t *)take((size_t)kClipCap * 4);
    std::vector<int32_t> dof(M), nxt(M);
    for (int d = 0; d < ndrops; d++)
        for (int m = drop_start_host[d]; m < drop_start_host[d + 1]; m++) {
            dof[m] = d;
            nxt[m] = (m + 1 == drop_start_host[d + 1]) ? drop_start_host[d] : m + 1;
        }
    e = cudaMemset(mk.mem, 0, bytes);
    if (e == cudaSuccess) {
        // the column keys of the scanline fill (the grid does not move); the
        // copies below, on the same legacy stream, follow the kernel
        k_colkeys<<<cdiv(nx, kT), kT>>>(nx, h, x0, mk.colkey);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(mk.drop_start, drop_start_host, (ndrops + 1) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && M > 0) e = cudaMemcpy(mk.drop_of, dof.data(), M * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && M > 0) e = cudaMemcpy(mk.next, nxt.data(), M * 4, cudaMemcpyHostToDevice);
    return e;
}

void markers_free(Markers &mk)
{
    if (mk.mem) cudaFree(mk.mem);
    mk.mem = nullptr;
}

void launch_validate(Markers &mk, cudaStream_t s)
{
    double m3 = 3.0 * mk.h;
    note_launch();
    k_validate<<<cdiv(mk.M, kT), kT, 0, s>>>(mk.M, mk.X, mk.Y, mk.x0 + m3, mk.x0 + mk.nx * mk.h - m3,
                                            mk.y0 + m3, mk.y0 + mk.ny * mk.h - m3, mk.flags);
}

void launch_geometry(Markers &mk, double sigma, cudaStream_t s)
{
    note_launch();
    k_geometry<<<cdiv(mk.M, kT), kT, 0, s>>>(mk.M, mk.X, mk.Y, mk.drop_of, mk.drop_start, sigma,
                                            mk.x0, mk.y0, mk.h, mk.kappa, mk.nxm, mk.nym, mk.ds,
                                            mk.fmag, mk.gx, mk.gy, mk.gxf, mk.gyf, mk.ykey);
    note_launch();
    k_segments<<<cdiv(mk.M, 32), 32, 0, s>>>(  // FP64-heavy: spread over all SMs
        mk.M, mk.next, mk.gx, mk.gy, mk.nxm, mk.nym, mk.sbox,
                                            mk.sv, mk.sb5, mk.sl, mk.slf, mk.scvx, mk.sinv);
    note_launch();
    k_drop_yrange<<<cdiv((long)mk.ndrops * 32, kT), kT, 0, s>>>(mk.ndrops, mk.drop_start, mk.Y,
                                                               mk.dyr, mk.dyk);
}

void launch_sort(Markers &mk, cudaStream_t s)
{
    long ncell = (long)mk.nx * mk.ny;
    cudaMemsetAsync(mk.cell_count, 0, ncell * 4, s);
    cudaMemsetAsync(mk.bcount, 0, (size_t)mk.bnx * mk.bny * 4, s);
    note_launch();
    k_keys<<<cdiv(mk.M, kT), kT, 0, s>>>(mk.M, mk.X, mk.Y, mk.x0, mk.y0, mk.h, mk.nx, mk.ny,
                                        mk.bnx, mk.key, mk.cell_count, mk.bcount);
    int nparts = (int)cdiv(ncell, kScanChunk);
    note_launch();
    k_scan_partial<<<nparts, kT, 0, s>>>(ncell, mk.cell_count, mk.scan_part);
    note_launch();
    k_scan_parts<<<1, kT, 0, s>>>(nparts, mk.scan_part);
    note_launch();
    k_scan_final<<<nparts, kT, 0, s>>>(ncell, mk.cell_count, mk.scan_part, mk.cell_start,
                                       (uint32_t)mk.M);
    note_launch();
    k_place<<<cdiv(mk.M, kT), kT, 0, s>>>(mk.M, mk.key, mk.cell_start, mk.cell_count, mk.tmp_ids);
    note_launch();
    k_rerank<<<cdiv(mk.M, kT), kT, 0, s>>>(mk.M, mk.key, mk.cell_start, mk.tmp_ids, mk.ids);
    int nb = mk.bnx * mk.bny;
    note_launch();
    k_block_active<<<cdiv(nb, kT), kT, 0, s>>>(mk.bnx, mk.bny, mk.bcount, mk.bactive);
}

void launch_interp(const Markers &mk, int kernel, const double *u, const double *v,
                   double *U, double *V, double dt_move, cudaStream_t s)
{
    note_launch();
    k_interp<<<cdiv(mk.M, 128), 128, 0, s>>>(mk.M, kernel, mk.nx, mk.ny, mk.h, mk.x0, mk.y0, u, v,
                                            mk.X, mk.Y, U, V, dt_move);
}

void launch_spread_conv(const Markers &mk, int kernel, const double *fmag, double *Fx,
                        double *Fy, cudaStream_t s)
{
    long nf = (long)(mk.nx + 1) * mk.ny + (long)mk.nx * (mk.ny + 1);
    cudaMemsetAsync(Fx, 0, (size_t)(mk.nx + 1) * mk.ny * 8, s);
    cudaMemsetAsync(Fy, 0, (size_t)mk.nx * (mk.ny + 1) * 8, s);
    note_launch();
    k_spread_conv<<<cdiv(nf, kT), kT, 0, s>>>(kernel, mk.nx, mk.ny, mk.h, mk.x0, mk.y0, mk.bnx,
                                             mk.bactive, mk.cell_start, mk.ids, mk.X, mk.Y,
                                             fmag, mk.nxm, mk.nym, mk.ds, Fx, Fy);
}

// Grid of the strip-area kernel: kClipBlocks clip blocks, then 8 CTAs of
// 256 threads per SM for the flat pair loop (grid-stride).
int band_area_grid()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return kClipBlocks + 8 * sms;
}

// Strip areas of the current band pair list (idempotent: pacc, pcov only).
void launch_band_area(const Markers &mk, cudaStream_t s)
{
    note_launch();
    k_band_area<<<band_area_grid(), 256, 0, s>>>(mk.nx, mk.npairs, mk.pair_cap, mk.pseg, mk.pcell,
                                                 mk.clip_list, mk.sl, mk.slf, mk.scvx, mk.sv, mk.sb5, mk.pacc,
                                                 mk.pcov);
}

void launch_heaviside(const Markers &mk, double *H, cudaStream_t s, cudaStream_t side,
                      cudaEvent_t ev_fork, cudaEvent_t ev_join)
{
    // the scanline fill of the rows inside the drops needs neither the
    // sort nor the segment records: with a side stream it runs next to the
    // band kernels, joining before the band sum that reads its H
    cudaStream_t sr = s;
    if (side) {
        cudaEventRecord(ev_fork, s);
        cudaStreamWaitEvent(side, ev_fork, 0);
        sr = side;
    }
    note_launch();
    k_rows_inside<<<mk.ny, kT, 0, sr>>>(mk.ndrops, mk.nx, mk.h, mk.x0, mk.y0, mk.X, mk.Y, mk.ykey,
                                        mk.colkey, mk.next, mk.drop_start, mk.dyk, H, mk.flags);
    if (side) cudaEventRecord(ev_join, side);
    dim3 g(mk.bnx, mk.bny);
    cudaMemsetAsync(mk.npairs, 0, 2 * sizeof(uint32_t), s);  // pairs, listed clip pairs
    note_launch();
    k_band_pairs<<<g, kPairT, 0, s>>>(mk.nx, mk.ny, mk.bnx, mk.bactive, mk.cell_start, mk.ids, mk.slf,
                                   mk.scvx, mk.sbox, mk.pair_cap, mk.npairs, mk.pseg, mk.pcell,
                                   mk.crange, mk.clip_list, mk.flags);
    launch_band_area(mk, s);
    if (side) cudaStreamWaitEvent(s, ev_join, 0);
    note_launch();
    k_band_sum<<<g, kBT, 0, s>>>(mk.nx, mk.ny, mk.bnx, mk.bactive, mk.crange, mk.pacc, mk.pcov, H);
}

void launch_spread_irrot(const Markers &mk, const double *fmag, const double *H, double *Fx,
                         double *Fy, cudaStream_t s)
{
    cudaMemsetAsync(Fx, 0, (size_t)(mk.nx + 1) * mk.ny * 8, s);
    cudaMemsetAsync(Fy, 0, (size_t)mk.nx * (mk.ny + 1) * 8, s);
    dim3 g(mk.bnx, mk.bny);
    note_launch();
    k_spread_irrot<<<g, kIrrT, 0, s>>>(mk.nx, mk.ny, 1.0 / mk.h, mk.bnx, mk.bactive, mk.cell_start,
                                       mk.ids, mk.next, mk.gx, mk.gy, mk.sinv, mk.gxf, mk.gyf, fmag,
                                       H, Fx, Fy, mk.flags);
}

size_t relocate_smem(int maxn)
{
    return (size_t)(maxn + 1) * 8 + (size_t)2 * (maxn + 1) * 4 + (size_t)4 * maxn * 8 +
           (size_t)2 * maxn * 8 + (size_t)4 * maxn * 8 + (size_t)6 * maxn * 8 + (size_t)(maxn + 1) * 8 + 64;
}

// ------------------------------------------------------------ measure correction
// Section 2.5 (conservation of mass).  The measure of drop markers shifted by
// e along the normals: planar, the enclosed area by the shoelace sum in
// marker order; axisymmetric, the volume of revolution 2 pi sum (z2 - z1)
// (r1^2 + r1 r2 + r2^2) / 6 over the right half of the meridian (markers
// 0 .. n/2).  Serial in marker order (one thread per drop), so that the
// bisection below takes each decision on the same sum as a serial program.
// nx == NULL: the markers as they are.
__device__ double drop_measure(int n, const double *X, const double *Y, const double *nx,
                               const double *ny, double e, int axisym)
{
    auto px = [&](int k) { return nx ? X[k] + e * nx[k] : X[k]; };
    auto py = [&](int k) { return nx ? Y[k] + e * ny[k] : Y[k]; };
    double a = 0.0;
    if (!axisym) {
        for (int k = 0; k < n; k++) {
            const int q = (k + 1 == n) ? 0 : k + 1;
            a += px(k) * py(q) - px(q) * py(k);
        }
        return 0.5 * a;
    }
    for (int k = 0; k < n / 2; k++) {
        const double r1 = px(k), z1 = py(k), r2 = px(k + 1), z2 = py(k + 1);
        a += (z2 - z1) * (r1 * r1 + r1 * r2 + r2 * r2) / 6.0;
    }
    return 2.0 * 3.14159265358979323846 * a;
}

// Initial measure of every drop (one thread per drop).
__global__ void k_drop_measure(int ndrops, const int32_t *__restrict__ drop_start,
                               const double *__restrict__ X, const double *__restrict__ Y,
                               int axisym, double *__restrict__ A)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndrops) return;
    const int s = drop_start[d], n = drop_start[d + 1] - s;
    A[d] = drop_measure(n, X + s, Y + s, nullptr, nullptr, 0.0, axisym);
}

// Where |A - A0| > tol A0, one offset eps along the inward unit normals (of
// the uncorrected markers) restores the measure: bisection on [-h, h] until
// the bracket is below 1e-13 h or 80 halvings, eps its midpoint.  One thread
// per drop; eps (may be NULL) gets 0 where nothing moved.
__global__ void k_mass_correct(int ndrops, const int32_t *__restrict__ drop_start,
                               const double *__restrict__ A0, int axisym, double tol, double h,
                               const double *__restrict__ nxm, const double *__restrict__ nym,
                               double *__restrict__ X, double *__restrict__ Y,
                               double *__restrict__ eps_out)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndrops) return;
    const int s = drop_start[d], n = drop_start[d + 1] - s;
    const double a0 = A0[d];
    const double A = drop_measure(n, X + s, Y + s, nullptr, nullptr, 0.0, axisym);
    if (eps_out) eps_out[d] = 0.0;
    if (!(fabs(A - a0) > tol * a0)) return;
    double lo = -h, hi = h;
    for (int it = 0; it < 80 && hi - lo > 1e-13 * h; it++) {
        const double mid = 0.5 * (lo + hi);
        if (drop_measure(n, X + s, Y + s, nxm + s, nym + s, mid, axisym) > a0) lo = mid;
        else hi = mid;
    }
    const double eps = 0.5 * (lo + hi);
    for (int k = 0; k < n; k++) {
        X[s + k] = X[s + k] + eps * nxm[s + k];
        Y[s + k] = Y[s + k] + eps * nym[s + k];
    }
    if (eps_out) eps_out[d] = eps;
}

void launch_drop_measure(const Markers &mk, int axisym, double *A, cudaStream_t s)
{
    note_launch();
    k_drop_measure<<<cdiv(mk.ndrops, 128), 128, 0, s>>>(mk.ndrops, mk.drop_start, mk.X, mk.Y,
                                                        axisym, A);
}

void launch_mass_correct(Markers &mk, const double *A0, int axisym, double tol, double *eps,
                         cudaStream_t s)
{
    note_launch();
    k_mass_correct<<<cdiv(mk.ndrops, 128), 128, 0, s>>>(mk.ndrops, mk.drop_start, A0, axisym, tol,
                                                        mk.h, mk.nxm, mk.nym, mk.X, mk.Y, eps);
}

void launch_relocate(Markers &mk, cudaStream_t s)
{
    size_t sm = relocate_smem(mk.max_drop);
    raise_smem_limit((const void *)k_reloc_fit, (int)sm);
    note_launch();
    k_reloc_fit<<<mk.ndrops, kT, sm, s>>>(mk.X, mk.Y, mk.drop_start, mk.h, mk.max_drop, mk.rfit,
                                          mk.rpar, mk.rwts, mk.flags);
    note_launch();
    if (mk.M < 4096)
        k_reloc_place<8><<<cdiv(8 * mk.M, kPlaceT), kPlaceT, 0, s>>>(mk.M, mk.X, mk.Y, mk.drop_of,
                                                                     mk.drop_start, mk.rfit, mk.rpar,
                                                                     mk.Xn, mk.Yn);
    else
        k_reloc_place<1><<<cdiv(mk.M, kPlaceT), kPlaceT, 0, s>>>(mk.M, mk.X, mk.Y, mk.drop_of,
                                                                 mk.drop_start, mk.rfit, mk.rpar,
                                                                 mk.Xn, mk.Yn);
    cudaMemcpyAsync(mk.X, mk.Xn, (size_t)mk.M * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(mk.Y, mk.Yn, (size_t)mk.M * 8, cudaMemcpyDeviceToDevice, s);
}

}  // namespace ibk
