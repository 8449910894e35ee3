// Multigrid for the variable-coefficient pressure equation of Section 2.1
// Eq. (ps), div(beta grad p) = b, on the cell-centred MAC grid.  The paper
// names multigrid and nothing more; this is the V(nu1, nu2) cycle with a
// red-black Gauss-Seidel smoother, residual + four-child averaging
// restriction, bilinear (9,3,3,1)/16 prolongation, coarse face coefficients
// = mean of the two fine faces, and an exact solve of the coarsest level
// with the constant null space removed by A + s 1 1^T (s = A_00), applied as
// a product with the inverse of that matrix (formed once per coefficient set
// by Gauss-Jordan elimination in FP64).
//
// GB300 mapping:
//  * sweeps are tiled (two sweeps per launch on shrinking rings of a 4-cell
//    halo; the FP64 sweep on a pre-scaled stencil, four weights and h^2 b /
//    diag per cell; a single FP64 sweep per launch on a 2-cell halo for other
//    sweep counts) and out of place: a launch reads the iterate from one
//    buffer and writes its tiles to the other, since blocks read their
//    neighbours' tiles as halo.
//  * the V(2,2) cycle fuses the residual and restriction into the
//    pre-smoothing launch and the prolongation into the post-smoothing
//    launch, so a level costs two launches (FP32 and FP64).
//  * kernels of the cycle use programmatic dependent launch: the next grid is
//    scheduled while the previous one drains and waits (griddepcontrol) for
//    its results.
//  * levels with <= 1024 cells (FP64) / <= 4096 cells (FP32) run as one
//    single-CTA kernel (the whole lower V-cycle and the coarsest solve) with
//    its data in shared memory, since launches dominate there.
//  * norms are deterministic two-stage reductions (fixed per-thread order,
//    fixed tree, last-block fold) with no floating-point atomics.
//  * the FP32 instantiations of the same kernels form the inner cycle of the
//    defect-correction solve; the residual, the update and the coarsest
//    solve stay FP64.
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

#include "ib_internal.cuh"

namespace ibk {
namespace {

constexpr int TW = 64, TH = 16, TT = 256;
constexpr int kRedT = 256;

// Programmatic dependent launch: kernels of the V-cycle are launched with
// programmatic stream serialisation, so the next grid is scheduled while the
// previous one drains.  Each such kernel first waits until the grid before
// it has completed and its writes are visible (griddepcontrol.wait), then
// lets the next grid launch (griddepcontrol.launch_dependents); nothing is
// read or written before the wait.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}

// ------------------------------------------------------------------ sweeps
template <typename T>
__global__ void __launch_bounds__(TT)
k_rbgs_sweep(int nx, int ny, T h2, const T *__restrict__ bx, const T *__restrict__ by,
             const T *__restrict__ invd, const T *__restrict__ b, const T *__restrict__ pin,
             T *__restrict__ p)
{
    pdl_enter();
    __shared__ T ps[TH + 4][TW + 4];
    const int gi0 = blockIdx.x * TW - 2, gj0 = blockIdx.y * TH - 2;
    const long nxf = nx + 1;
    for (int k = threadIdx.x; k < (TH + 4) * (TW + 4); k += TT) {
        int r = k / (TW + 4), c = k - r * (TW + 4);
        int gi = gi0 + c, gj = gj0 + r;
        ps[r][c] = (gi >= 0 && gi < nx && gj >= 0 && gj < ny) ? pin[(long)gj * nx + gi] : T(0);
    }
    __syncthreads();
    // red cells ((i+j) even) of the tile and its one-cell ring
    constexpr int RW = (TW + 2) / 2;
    for (int k = threadIdx.x; k < (TH + 2) * RW; k += TT) {
        int r = 1 + k / RW, cc = k - (r - 1) * RW;
        int gj = gj0 + r;
        int c = 1 + 2 * cc + ((gi0 + 1 + gj) & 1);
        int gi = gi0 + c;
        if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) continue;
        long kc = (long)gj * nx + gi, kx = (long)gj * nxf + gi;
        T s = bx[kx + 1] * ps[r][c + 1];
        s = fma(bx[kx], ps[r][c - 1], s);
        s = fma(by[kc + nx], ps[r + 1][c], s);
        s = fma(by[kc], ps[r - 1][c], s);
        T id = invd ? invd[kc]
                    : T(1) / ((gi + 1 < nx ? bx[kx + 1] : T(0)) + (gi > 0 ? bx[kx] : T(0)) +
                              (gj + 1 < ny ? by[kc + nx] : T(0)) + (gj > 0 ? by[kc] : T(0)));
        ps[r][c] = (s - h2 * b[kc]) * id;
    }
    __syncthreads();
    constexpr int BW = TW / 2;
    for (int k = threadIdx.x; k < TH * BW; k += TT) {
        int r = 2 + k / BW, cc = k - (r - 2) * BW;
        int gj = gj0 + r;
        int c = 2 + 2 * cc + ((gi0 + gj + 1) & 1);
        int gi = gi0 + c;
        if (gi >= nx || gj >= ny) continue;
        long kc = (long)gj * nx + gi, kx = (long)gj * nxf + gi;
        T s = bx[kx + 1] * ps[r][c + 1];
        s = fma(bx[kx], ps[r][c - 1], s);
        s = fma(by[kc + nx], ps[r + 1][c], s);
        s = fma(by[kc], ps[r - 1][c], s);
        T id = invd ? invd[kc]
                    : T(1) / ((gi + 1 < nx ? bx[kx + 1] : T(0)) + (gi > 0 ? bx[kx] : T(0)) +
                              (gj + 1 < ny ? by[kc + nx] : T(0)) + (gj > 0 ? by[kc] : T(0)));
        ps[r][c] = (s - h2 * b[kc]) * id;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < TH * TW; k += TT) {
        int r = 2 + k / TW, c = 2 + (k - (r - 2) * TW);
        int gi = gi0 + c, gj = gj0 + r;
        if (gi < nx && gj < ny) p[(long)gj * nx + gi] = ps[r][c];
    }
}

// The FP64 sweep on the pre-scaled stencil: p_c <- sum_f w_{c,f} p_nb(f) - bt_c
// with w_{c,f} = beta_f / diag_c and bt_c = h^2 b_c / diag_c, the update of
// k_rbgs_sweep ((sum_f beta_f p_nb - h^2 b_c) / diag_c) in four FP64 FMAs
// instead of six.  This part issues FP64 at 1/70 of its FP32 rate, so the
// six-operation sweep is bound by the FP64 pipe before HBM; the weights cost
// 8 more bytes per cell (w 32 B + bt 8 B in place of beta_x, beta_y, 1/diag
// and b) and move the bound back towards memory.  Same tiling as
// k_rbgs_sweep: red on the tile and its one-cell ring, then black on the
// tile, from a shared-memory copy of the iterate with a 2-cell halo.
__global__ void __launch_bounds__(TT)
k_rbgs_sweep_w(int nx, int ny, const double2 *__restrict__ w, const double *__restrict__ bt,
               const double *__restrict__ pin, double *__restrict__ p)
{
    pdl_enter();
    __shared__ double ps[TH + 4][TW + 4];
    const int gi0 = blockIdx.x * TW - 2, gj0 = blockIdx.y * TH - 2;
    for (int k = threadIdx.x; k < (TH + 4) * (TW + 4); k += TT) {
        int r = k / (TW + 4), c = k - r * (TW + 4);
        int gi = gi0 + c, gj = gj0 + r;
        ps[r][c] = (gi >= 0 && gi < nx && gj >= 0 && gj < ny) ? pin[(long)gj * nx + gi] : 0.0;
    }
    __syncthreads();
    constexpr int RW = (TW + 2) / 2;
    for (int k = threadIdx.x; k < (TH + 2) * RW; k += TT) {
        const int r = 1 + k / RW, cc = k - (r - 1) * RW;
        const int gj = gj0 + r;
        const int c = 1 + 2 * cc + ((gi0 + 1 + gj) & 1);
        const int gi = gi0 + c;
        if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) continue;
        const long kc = (long)gj * nx + gi;
        const double2 we = w[2 * kc], sn = w[2 * kc + 1];
        double s = fma(we.x, ps[r][c - 1], -bt[kc]);
        s = fma(we.y, ps[r][c + 1], s);
        s = fma(sn.x, ps[r - 1][c], s);
        ps[r][c] = fma(sn.y, ps[r + 1][c], s);
    }
    __syncthreads();
    constexpr int BW = TW / 2;
    for (int k = threadIdx.x; k < TH * BW; k += TT) {
        const int r = 2 + k / BW, cc = k - (r - 2) * BW;
        const int gj = gj0 + r;
        const int c = 2 + 2 * cc + ((gi0 + gj + 1) & 1);
        const int gi = gi0 + c;
        if (gi >= nx || gj >= ny) continue;
        const long kc = (long)gj * nx + gi;
        const double2 we = w[2 * kc], sn = w[2 * kc + 1];
        double s = fma(we.x, ps[r][c - 1], -bt[kc]);
        s = fma(we.y, ps[r][c + 1], s);
        s = fma(sn.x, ps[r - 1][c], s);
        ps[r][c] = fma(sn.y, ps[r + 1][c], s);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < TH * TW; k += TT) {
        int r = 2 + k / TW, c = 2 + (k - (r - 2) * TW);
        int gi = gi0 + c, gj = gj0 + r;
        if (gi < nx && gj < ny) p[(long)gj * nx + gi] = ps[r][c];
    }
}

constexpr int FW = 64, FH = 16, FT = 256;

// Test hook (ib_debug_stall_staging): when nonzero, every TMA-staged smoother
// block also waits, after its copies have landed, on a barrier phase that
// nothing completes, so that its bounded wait runs out and the time-out
// path (fault word, IB_ECUDA from the solve) can be tested without a fault.
__device__ int g_stall_staging = 0;

// Asynchronous global -> shared copies (both addresses aligned to the size);
// src-size 0 writes zeros without reading.
__device__ __forceinline__ void cp_async16(void *d, const void *src, bool v)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(d)),
                 "l"(src), "r"(v ? 16 : 0));
}
__device__ __forceinline__ void cp_async4(void *d, const void *src, bool v)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(d)),
                 "l"(src), "r"(v ? 4 : 0));
}

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// Global timer (nanoseconds).
__device__ __forceinline__ unsigned long long gtimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Limits of the smoother's staging waits: the first wait for the tile's
// copies (they take microseconds; the limit only has to outlast a context
// switch), and the drain after a time-out, which must see the copies land
// before the block leaves (its shared memory is their destination).
constexpr unsigned long long kStageWaitNs = 50000000ull;   // 50 ms
constexpr unsigned long long kDrainNs = 500000000ull;      // 0.5 s

// Wait for phase `parity` of a shared-memory barrier: true once it has
// completed, false when limit_ns of global time (or, should the timer stall,
// 2^26 polls) have passed first.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          unsigned long long limit_ns)
{
    const unsigned long long t0 = gtimer_ns();
    for (int it = 0; it < (1 << 26); it++) {
        unsigned done;
        asm volatile("{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, P;\n}\n"
                     : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
        if (done) return true;
        if (gtimer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// One 2-D tensor copy global -> shared completing on `bar`; the box (set in
// the map) lands densely, row-major, at dst; cells outside the array read 0.
__device__ __forceinline__ void tma_load2(void *dst, const CUtensorMap *map, int x, int y,
                                          unsigned long long *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];\n"
                 ::"r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar)) : "memory");
}

// Two red-black sweeps in one launch (FP32 inner cycle), staged in shared
// memory; the sweeps run from shared memory on shrinking rings (red, black,
// red, black) so that the tile's result equals two global sweeps.  MODE 0:
// the sweeps alone (halo 4).  MODE 1: the sweeps, then the residual b - A p
// of the tile's cells averaged over 2x2 children into the coarse right-hand
// side (coarse correction set to zero); the last black phase also covers the
// tile's one-cell ring so that the residual sees final neighbours (halo 5).
// MODE 2: p + P e_c (the bilinear prolongation of the coarse correction) is
// formed while staging, then the sweeps (halo 4); with p64 (the finest level
// of a defect-correction cycle) the result is added to the FP64 iterate
// instead of being stored.  Each mode equals the separate kernels in turn.
// Staging: with TMA (widths that are a multiple of 4), one thread issues
// tensor copies of the iterate, right-hand side, 1/diag and beta_y windows
// (zero outside the grid) onto one barrier while all threads copy the x-face
// rows (rows of nx + 1 faces are not 16-byte aligned, so no tensor map
// describes them) with 16-byte asynchronous copies; otherwise every array
// goes through asynchronous copies.  A barrier wait that times out (50 ms)
// makes the block skip its tile: it waits up to 0.5 s more for its copies to
// land and raises the fault word to 1 (landed) or 3 (not landed); misaligned
// shared memory raises it to 2.
// The iterate is read from pin and the tile written to p (a different
// buffer): blocks read their neighbours' tiles as halo, so an in-place update
// would let a block see values another block has already smoothed.
template <int MODE, bool TMA>
__global__ void __launch_bounds__(FT)
k_smooth2_f32(int nx, int ny, float h2, float ih2, const float *__restrict__ bx,
              const float *__restrict__ by, const float *__restrict__ invd,
              const float *__restrict__ b, const float *__restrict__ pin, float *__restrict__ p,
              float *__restrict__ rc, float *__restrict__ ecz, const float *__restrict__ ecp,
              double *__restrict__ p64, const __grid_constant__ TileMaps tm)
{
    constexpr int HA = MODE == 1 ? 5 : 4;   // rows of halo
    constexpr int XO = MODE == 1 ? 8 : 4;   // columns of halo (a multiple of 4: 16-byte rows)
    constexpr int PW = FW + 2 * XO, PH = FH + 2 * HA;
    __shared__ __align__(128) float ps[PH][PW];
    __shared__ __align__(128) float bs[PH][PW];
    __shared__ __align__(128) float ds[PH][PW];
    __shared__ __align__(128) float ys[PH + 1][PW];
    // x-faces: row r holds the faces gi0 .. gi0 + PW from column xoff[r] on
    // (the 16-byte-aligned copy of a row of (nx + 1) faces starts up to three
    // faces early)
    __shared__ __align__(16) float xs[PH][PW + 8];
    __shared__ int xoff[PH];
    __shared__ __align__(8) unsigned long long bar, stall_bar;
    const int gi0 = blockIdx.x * FW - XO, gj0 = blockIdx.y * FH - HA;
    const long nxf = nx + 1;
    const int nxc = nx / 2, nyc = ny / 2;
    // P e_c at fine cell (gi, gj) (MODE 2)
    auto cor = [&](int gi, int gj) {
        const int I = gi >> 1, J = gj >> 1;
        const int I2 = min(max(I + ((gi & 1) ? 1 : -1), 0), nxc - 1);
        const int J2 = min(max(J + ((gj & 1) ? 1 : -1), 0), nyc - 1);
        const float c00 = ecp[(long)J * nxc + I], c10 = ecp[(long)J * nxc + I2];
        const float c01 = ecp[(long)J2 * nxc + I], c11 = ecp[(long)J2 * nxc + I2];
        return (9.0f * c00 + 3.0f * c10 + 3.0f * c01 + c11) * 0.0625f;
    };
    auto pro = [&](int gi, int gj) { return pin[(long)gj * nx + gi] + cor(gi, gj); };
    // x-faces of the window rows by asynchronous copies: 16-byte copies of
    // whole in-range chunks, single faces (zero beyond the walls) at the ends
    auto load_xfaces = [&]() {
        constexpr int NC = (PW + 1 + 3 + 3) / 4;  // 16-byte chunks per x-face row, worst alignment
        const long nbx = nxf * ny;
        for (int k = threadIdx.x; k < PH * NC; k += FT) {
            const int r = k / NC, q = k - r * NC, gj = gj0 + r;
            if (gj < 0 || gj >= ny) {
                cp_async16(&xs[r][4 * q], bx, false);
                if (q == 0) xoff[r] = 0;
                continue;
            }
            const long start = (long)gj * nxf + gi0, a0 = start & ~3L;
            if (q == 0) xoff[r] = (int)(start - a0);
            const long e0 = a0 + 4 * q;
            const int c0 = (int)(e0 - start);  // window column of face e0
            if (e0 >= 0 && e0 + 4 <= nbx && gi0 + c0 >= 0 && gi0 + c0 + 3 <= nx) {
                cp_async16(&xs[r][4 * q], bx + e0, true);
            } else {
                for (int t = 0; t < 4; t++) {
                    const int gi = gi0 + c0 + t;
                    const bool ok = gi >= 0 && gi <= nx;
                    cp_async4(&xs[r][4 * q + t], ok ? bx + e0 + t : bx, ok);
                }
            }
        }
    };
    if constexpr (TMA) {
        // tensor copies land on 128-byte boundaries (checked, not assumed)
        if (((smem_addr(&ps[0][0]) | smem_addr(&bs[0][0]) | smem_addr(&ds[0][0]) |
              smem_addr(&ys[0][0])) & 127u) != 0) {
            if (threadIdx.x == 0) atomicMax(tm.fault, 2);
            return;
        }
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bar)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&stall_bar)));
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
        }
        __syncthreads();  // the barrier is initialised before any thread waits on it
        // the coefficients (1/diag, beta_y, beta_x) are built before the
        // solve and not written during it: their copies start before the
        // wait for the previous grid, overlapping its tail; the iterate and
        // right-hand side it writes follow the wait
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;\n" ::);
            constexpr unsigned kBytes = (3 * PH + PH + 1) * PW * 4;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                         ::"r"(smem_addr(&bar)), "r"(kBytes));
            tma_load2(&ds[0][0], &tm.d, gi0, gj0, &bar);
            tma_load2(&ys[0][0], &tm.y, gi0, gj0, &bar);
        }
        load_xfaces();
        pdl_enter();
        if (threadIdx.x == 0) {
            tma_load2(&ps[0][0], &tm.p, gi0, gj0, &bar);
            tma_load2(&bs[0][0], &tm.b, gi0, gj0, &bar);
        }
        // the prolongation of the coarse correction overlaps the copies
        constexpr int NPRO = MODE == 2 ? (PH * PW + FT - 1) / FT : 1;
        float pc[NPRO];
        if constexpr (MODE == 2) {
#pragma unroll
            for (int i = 0; i < NPRO; i++) {
                const int k = threadIdx.x + i * FT, r = k / PW, c = k - r * PW;
                const int gi = gi0 + c, gj = gj0 + r;
                pc[i] = (k < PH * PW && gi >= 0 && gi < nx && gj >= 0 && gj < ny) ? cor(gi, gj) : 0.0f;
            }
        }
        asm volatile("cp.async.wait_all;\n" ::);
        bool ok = mbar_wait(&bar, 0, kStageWaitNs);
        if (ok && g_stall_staging) ok = mbar_wait(&stall_bar, 0, kStageWaitNs);
        // one outcome for the whole block (each thread's wait is bounded)
        if (__syncthreads_or(!ok)) {
            // skip the tile; the copies must land before the block leaves
            const bool landed = mbar_wait(&bar, 0, kDrainNs);
            if (threadIdx.x == 0) atomicMax(tm.fault, landed ? 1 : 3);
            return;
        }
        if constexpr (MODE == 2) {
#pragma unroll
            for (int i = 0; i < NPRO; i++) {
                const int k = threadIdx.x + i * FT, r = k / PW, c = k - r * PW;
                if (k < PH * PW) ps[r][c] += pc[i];
            }
        }
        __syncthreads();
    } else {
        pdl_enter();
        // rows of a multiple of 4 cells: every 4-cell chunk of the window
        // (gi0 and the window width are multiples of 4) lies wholly inside or
        // wholly outside the grid
        const bool vec = (nx & 3) == 0;
        if (vec) {
            constexpr int V = PW / 4;  // float4 per row
            for (int k = threadIdx.x; k < (PH + 1) * V; k += FT) {
                const int r = k / V, c4 = k - r * V, gj = gj0 + r, gc = gi0 + 4 * c4;
                const bool inx = gc >= 0 && gc + 4 <= nx;
                const long o = (long)gj * nx + gc;
                if (r < PH) {
                    const bool in = inx && gj >= 0 && gj < ny;
                    if (MODE == 2) {
                        for (int q = 0; q < 4; q++) ps[r][4 * c4 + q] = in ? pro(gi0 + 4 * c4 + q, gj) : 0.0f;
                    } else {
                        cp_async16(&ps[r][4 * c4], in ? pin + o : pin, in);
                    }
                    cp_async16(&bs[r][4 * c4], in ? b + o : b, in);
                    cp_async16(&ds[r][4 * c4], in ? invd + o : invd, in);
                }
                const bool iny = inx && gj >= 0 && gj <= ny;
                cp_async16(&ys[r][4 * c4], iny ? by + o : by, iny);
            }
        } else {
            for (int k = threadIdx.x; k < (PH + 1) * PW; k += FT) {
                const int r = k / PW, c = k - r * PW, gi = gi0 + c, gj = gj0 + r;
                const long o = (long)gj * nx + gi;
                if (r < PH) {
                    const bool in = gi >= 0 && gi < nx && gj >= 0 && gj < ny;
                    ps[r][c] = in ? (MODE == 2 ? pro(gi, gj) : pin[o]) : 0.0f;
                    bs[r][c] = in ? b[o] : 0.0f;
                    ds[r][c] = in ? invd[o] : 0.0f;
                }
                ys[r][c] = (gi >= 0 && gi < nx && gj >= 0 && gj <= ny) ? by[o] : 0.0f;
            }
        }
        if (vec) {
            load_xfaces();
        } else {
            for (int k = threadIdx.x; k < PH * (PW + 1); k += FT) {
                const int r = k / (PW + 1), c = k - r * (PW + 1), gi = gi0 + c, gj = gj0 + r;
                const bool in = gi >= 0 && gi <= nx && gj >= 0 && gj < ny;
                cp_async4(&xs[r][c], in ? bx + (long)gj * nxf + gi : bx, in);
                if (c == 0) xoff[r] = 0;
            }
        }
        asm volatile("cp.async.wait_all;\n" ::);
        __syncthreads();
    }
    // ring q: local rows [HA - q, HA + FH + q), columns [XO - q, XO + FW + q)
    constexpr int Q0 = HA - 1;  // outermost ring updated
#pragma unroll
    for (int ph = 0; ph < 4; ph++) {
        const int q = Q0 - ph, color = ph & 1;
        const int w = FW + 2 * q, hgt = FH + 2 * q, hw = w / 2;
        for (int k = threadIdx.x; k < hgt * hw; k += FT) {
            const int rr = k / hw, cc = k - rr * hw;
            const int r = HA - q + rr, gj = gj0 + r;
            const int c = XO - q + 2 * cc + ((gi0 + XO - q + gj + color) & 1);
            const int gi = gi0 + c;
            if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) continue;
            const int xc = c + xoff[r];
            float sm = xs[r][xc + 1] * ps[r][c + 1];
            sm = fmaf(xs[r][xc], ps[r][c - 1], sm);
            sm = fmaf(ys[r + 1][c], ps[r + 1][c], sm);
            sm = fmaf(ys[r][c], ps[r - 1][c], sm);
            ps[r][c] = (sm - h2 * bs[r][c]) * ds[r][c];
        }
        __syncthreads();
    }
    if (MODE == 1) {
        // one coarse cell per thread: FW/2 x FH/2 = 32 x 8
        const int I = blockIdx.x * (FW / 2) + (threadIdx.x % (FW / 2));
        const int J = blockIdx.y * (FH / 2) + (threadIdx.x / (FW / 2));
        if (I < nxc && J < nyc) {
            auto res = [&](int gi, int gj) {
                const int r = gj - gj0, c = gi - gi0;
                const float cc = ps[r][c];
                const float pE = gi + 1 < nx ? ps[r][c + 1] : cc, pW = gi > 0 ? ps[r][c - 1] : cc;
                const float pN = gj + 1 < ny ? ps[r + 1][c] : cc, pS = gj > 0 ? ps[r - 1][c] : cc;
                const int xc = c + xoff[r];
                float s = xs[r][xc + 1] * (pE - cc);
                s -= xs[r][xc] * (cc - pW);
                s += ys[r + 1][c] * (pN - cc);
                s -= ys[r][c] * (cc - pS);
                return bs[r][c] - s * ih2;
            };
            const int i = 2 * I, j = 2 * J;
            const float r00 = res(i, j), r10 = res(i + 1, j), r01 = res(i, j + 1), r11 = res(i + 1, j + 1);
            rc[(long)J * nxc + I] = 0.25f * (r00 + r10 + r01 + r11);
            ecz[(long)J * nxc + I] = 0.0f;
        }
    }
    for (int k = threadIdx.x; k < FH * FW; k += FT) {
        const int r = HA + k / FW, c = XO + (k - (k / FW) * FW);
        const int gi = gi0 + c, gj = gj0 + r;
        if (gi < nx && gj < ny) {
            if (MODE == 2 && p64) p64[(long)gj * nx + gi] += f2d(ps[r][c]);
            else p[(long)gj * nx + gi] = ps[r][c];
        }
    }
}

// The TMA-staged form of k_smooth2_f32 (widths a multiple of 4), written for
// few instructions per cell: the profile of the general kernel at 2048^2
// showed it issue-bound (~360 thread instructions a cell, 72 % issue
// active, DRAM 30 %, memory instructions an eighth of them), its index
// arithmetic and per-cell global loads outweighing the eight FMAs of two
// sweeps.  Here a cell's operands sit at fixed offsets from its flat shared
// index (west/east faces, south/north faces, the four neighbours, b and
// 1/diag), its colour parity comes from one per-tile sum, and tiles whose
// window lies inside the grid skip the bounds tests.
// MODE 2 takes the coarse correction from a shared copy of its window
// (14 x 38 coarse cells, loaded while the tensor copies are in flight) and
// prolongs it one 2 x 2 block of fine cells per thread step (nine coarse
// values for four fine ones); the FP64 iterate of a defect-correction cycle
// is read into registers before the sweeps.  The arithmetic of every value
// (the order of its FMAs) is that of k_smooth2_f32, so results agree bit for
// bit.  All five operand windows come by tensor copies, beta_x from the
// level's padded-row copy (the packed rows of nx + 1 values have no 16-byte
// stride); the bounded barrier waits and the fault word are as there.
template <int MODE>
__global__ void __launch_bounds__(FT, MODE == 1 ? 5 : 6)  // as many CTAs as shared memory holds
k_smooth2t_f32(int nx, int ny, float h2, float ih2, float *__restrict__ p, float *__restrict__ rc,
               float *__restrict__ ecz, const float *__restrict__ ecp, double *__restrict__ p64,
               const __grid_constant__ TileMaps tm)
{
    constexpr int HA = MODE == 1 ? 5 : 4;   // rows of halo
    constexpr int XO = MODE == 1 ? 8 : 4;   // columns of halo (a multiple of 4: 16-byte rows)
    constexpr int PW = FW + 2 * XO, PH = FH + 2 * HA;
    constexpr int CWW = FW / 2 + 6, CHH = FH / 2 + 6;  // coarse window (MODE 2): 38 x 14
    __shared__ __align__(128) float ps[PH * PW];
    __shared__ __align__(128) float bs[PH * PW];
    __shared__ __align__(128) float ds[PH * PW];
    __shared__ __align__(128) float ys[(PH + 1) * PW];
    // x-faces: row r holds faces gi0 .. gi0 + PW - 1, the west face of each
    // window cell (no updated cell needs the east face of the window's last
    // column), so one offset addresses all five windows
    __shared__ __align__(128) float xs[PH * PW];
    __shared__ float cs[MODE == 2 ? CHH * CWW : 1];
    __shared__ __align__(8) unsigned long long bar, stall_bar;
    const int gi0 = blockIdx.x * FW - XO, gj0 = blockIdx.y * FH - HA;
    const int nxc = nx / 2, nyc = ny / 2;
    const int tid = threadIdx.x;
    if (((smem_addr(ps) | smem_addr(bs) | smem_addr(ds) | smem_addr(ys) | smem_addr(xs)) & 127u) != 0) {
        if (tid == 0) atomicMax(tm.fault, 2);
        return;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&bar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&stall_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    __syncthreads();  // the barrier is initialised before any thread waits on it
    // the coefficients (1/diag, beta_y, beta_x) are built before the solve
    // and not written during it: their copies start before the wait for the
    // previous grid; the iterate and right-hand side follow the wait.  gi0
    // is a multiple of 4: every copy starts on a 16-byte boundary.
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::);
        constexpr unsigned kBytes = (4 * PH + PH + 1) * PW * 4;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                     ::"r"(smem_addr(&bar)), "r"(kBytes));
        tma_load2(ds, &tm.d, gi0, gj0, &bar);
        tma_load2(ys, &tm.y, gi0, gj0, &bar);
        tma_load2(xs, &tm.x, gi0, gj0, &bar);
    }
    pdl_enter();
    if (tid == 0) {
        tma_load2(ps, &tm.p, gi0, gj0, &bar);
        tma_load2(bs, &tm.b, gi0, gj0, &bar);
    }
    const int cI0 = blockIdx.x * (FW / 2) - 3, cJ0 = blockIdx.y * (FH / 2) - 3;
    const int lane = tid & 31, warp = tid >> 5;
    // the coarse window inside the coarse grid (then so are the neighbours
    // of all its prolonged blocks): no range tests
    const bool cin = cI0 >= 0 && cI0 + CWW <= nxc && cJ0 >= 0 && cJ0 + CHH <= nyc;
    if constexpr (MODE == 2) {
        // the coarse correction's window, while the tensor copies fly
        static_assert(CWW > 32 && CWW <= 64, "a window row is one or two loads a lane");
        if (cin) {
            for (int j = warp; j < CHH; j += FT / 32) {
                const float *src = ecp + (long)(cJ0 + j) * nxc + cI0;
                cs[j * CWW + lane] = src[lane];
                if (lane < CWW - 32) cs[j * CWW + 32 + lane] = src[32 + lane];
            }
        } else {
            for (int k = tid; k < CHH * CWW; k += FT) {
                const int j = k / CWW, i = k - j * CWW, gI = cI0 + i, gJ = cJ0 + j;
                cs[k] = (gI >= 0 && gI < nxc && gJ >= 0 && gJ < nyc) ? ecp[(long)gJ * nxc + gI] : 0.0f;
            }
        }
    }
    // the tile's cells all inside the grid: no range tests on the global
    // iterate (thread k of the block takes column k % FW of rows k / FW + 4 j)
    const bool whole = (blockIdx.x + 1) * FW <= nx && (blockIdx.y + 1) * FH <= ny;
    const int tcol = tid % FW, trow = tid / FW;
    constexpr int RS = FT / FW;  // rows a pass of the block covers
    // the FP64 iterate of the tile (defect correction), read ahead
    double v64[MODE == 2 ? (FW * FH) / FT : 1];
    if constexpr (MODE == 2) {
        if (p64) {
            const long g0 = (long)(blockIdx.y * FH + trow) * nx + blockIdx.x * FW + tcol;
#pragma unroll
            for (int j = 0; j < (FW * FH) / FT; j++) {
                const int gi = blockIdx.x * FW + tcol, gj = blockIdx.y * FH + trow + RS * j;
                v64[j] = (whole || (gi < nx && gj < ny)) ? p64[g0 + (long)RS * j * nx] : 0.0;
            }
        }
    }
    // the first warp waits for the tensor copies (a bounded wait) and the
    // block barrier of the outcome passes the copied data on to the others;
    // the other warps issue nothing while they wait there
    bool ok = true;
    if (warp == 0) {
        ok = mbar_wait(&bar, 0, kStageWaitNs);
        if (ok && g_stall_staging) ok = mbar_wait(&stall_bar, 0, kStageWaitNs);
    }
    // one outcome for the whole block
    if (__syncthreads_or(!ok)) {
        // skip the tile; the copies must land before the block leaves
        const bool landed = mbar_wait(&bar, 0, kDrainNs);
        if (tid == 0) atomicMax(tm.fault, landed ? 1 : 3);
        return;
    }
    const bool interior = gi0 >= 0 && gi0 + PW <= nx && gj0 >= 0 && gj0 + PH <= ny;
    if constexpr (MODE == 2) {
        // p += P e_c, one 2 x 2 block of fine cells (coarse cell (I, J)) per
        // step: (9 c00 + 3 c10 + 3 c01 + c11) / 16 with the neighbours on the
        // cell's side, clamped at the walls (zero gradient)
        constexpr int BW = PW / 2, BH = PH / 2;
        // cin: no range tests, no clamps, the nine values at fixed offsets
        static_assert(CWW == BW + 2 && CHH == BH + 2, "coarse window = blocks + neighbours");
        if (cin) {
            // block (bj, bi); sx = 1 takes the east children first
            auto block = [&](int bj, int bi, int sx) {
                const float *c0 = cs + bj * CWW + bi;  // the block's south-west neighbour
                const float cSW = c0[0], cS = c0[1], cSE = c0[2];
                const float cW = c0[CWW], c = c0[CWW + 1], cE = c0[CWW + 2];
                const float cNW = c0[2 * CWW], cN = c0[2 * CWW + 1], cNE = c0[2 * CWW + 2];
                const float v00 = (9.0f * c + 3.0f * cW + 3.0f * cS + cSW) * 0.0625f;
                const float v10 = (9.0f * c + 3.0f * cE + 3.0f * cS + cSE) * 0.0625f;
                const float v01 = (9.0f * c + 3.0f * cW + 3.0f * cN + cNW) * 0.0625f;
                const float v11 = (9.0f * c + 3.0f * cE + 3.0f * cN + cNE) * 0.0625f;
                float *q0 = ps + (2 * bj) * PW + 2 * bi;
                q0[sx] += sx ? v10 : v00;
                q0[1 - sx] += sx ? v00 : v10;
                q0[PW + sx] += sx ? v11 : v01;
                q0[PW + 1 - sx] += sx ? v01 : v11;
            };
            // blocks 0-31 of a block row: a warp each, lanes 16-31 east
            // children first (even words for lanes 0-15, odd for 16-31: no
            // bank conflicts); blocks 32 on to the warps with fewer rows
            static_assert(BW >= 32 && (BW - 32) * BH <= FT - 32 * (BH % (FT / 32)), "block split");
            for (int bj = warp; bj < BH; bj += FT / 32) block(bj, lane, lane >> 4);
            const int k = tid - 32 * (BH % (FT / 32));
            if (k >= 0 && k < (BW - 32) * BH) block(k / (BW - 32), 32 + k % (BW - 32), 0);
        } else
        for (int kb = tid; kb < BW * BH; kb += FT) {
            const int bj = kb / BW, bi = kb - bj * BW;
            const int I = cI0 + 1 + bi, J = cJ0 + 1 + bj;
            if (I < 0 || I >= nxc || J < 0 || J >= nyc) continue;
            const int iW = max(I - 1, 0) - cI0, iC = I - cI0, iE = min(I + 1, nxc - 1) - cI0;
            const int jS = (max(J - 1, 0) - cJ0) * CWW, jC = (J - cJ0) * CWW,
                      jN = (min(J + 1, nyc - 1) - cJ0) * CWW;
            const float c = cs[jC + iC];
            const float cW = cs[jC + iW], cE = cs[jC + iE], cS = cs[jS + iC], cN = cs[jN + iC];
            const float cSW = cs[jS + iW], cSE = cs[jS + iE], cNW = cs[jN + iW], cNE = cs[jN + iE];
            float *q0 = ps + (2 * bj) * PW + 2 * bi;
            q0[0] += (9.0f * c + 3.0f * cW + 3.0f * cS + cSW) * 0.0625f;
            q0[1] += (9.0f * c + 3.0f * cE + 3.0f * cS + cSE) * 0.0625f;
            q0[PW] += (9.0f * c + 3.0f * cW + 3.0f * cN + cNW) * 0.0625f;
            q0[PW + 1] += (9.0f * c + 3.0f * cE + 3.0f * cN + cNE) * 0.0625f;
        }
        __syncthreads();
    }
    // ring q: local rows [HA - q, HA + FH + q), columns [XO - q, XO + FW + q);
    // its cells of one colour: hq (even) rows of hw = FW/2 + q.  The first
    // FW/2 cells of each row go in warp-sized chunks of 16 cells from each of
    // two adjacent rows: same-colour cells of a row are two words apart and
    // the two rows' parities differ (the pitch is even), so a chunk's 32
    // lanes meet all 32 shared-memory banks once.  The last q cells of each
    // row are dealt out flat.
    constexpr int Q0 = HA - 1;  // outermost ring updated
    static_assert(PW % 2 == 0 && FW == 64, "bank pattern of the chunks");
    const int par0 = gi0 + gj0 + XO + HA;
    // one red-black update of the cell at shared offset o
    auto relax = [&](int o) {
        float sm = xs[o + 1] * ps[o + 1];
        sm = fmaf(xs[o], ps[o - 1], sm);
        sm = fmaf(ys[o + PW], ps[o + PW], sm);
        sm = fmaf(ys[o], ps[o - PW], sm);
        ps[o] = (sm - h2 * bs[o]) * ds[o];
    };
    // outside an interior tile, cells beyond the walls are not updated
    auto inside = [&](int r, int c) {
        const int gi = gi0 + c, gj = gj0 + r;
        return gi >= 0 && gi < nx && gj >= 0 && gj < ny;
    };
    constexpr int NW = FT / 32;  // warps; NW is even, so a warp's chunks keep one half
    static_assert(NW % 2 == 0 && (FH + 2 * Q0) * Q0 <= FT, "chunk halves; one pass for the rest");
    const int rr0 = 2 * (warp >> 1) + (lane >> 4);  // row of the warp's first chunk
    const int cc0 = 16 * (warp & 1) + (lane & 15);
    // the four phases, with (CHECK) or without the wall tests
    auto sweeps = [&](auto check) {
        constexpr bool CHECK = decltype(check)::value;
#pragma unroll
        for (int ph = 0; ph < 4; ph++) {
            const int q = Q0 - ph, color = ph & 1;
            const int hq = FH + 2 * q;
            // chunks g = warp + NW t: row pair g >> 1, half g & 1; lanes 0-15
            // the pair's first row, 16-31 its second.  Along t the row
            // advances by NW, the column and parity stay; the trip count is
            // a constant, and chunks with (t + 1) NW <= hq exist for every
            // warp.  (gi + gj + color) even: column XO - q + 2 cc + parity
            const int c = XO - q + 2 * cc0 + ((par0 - 2 * q + rr0 + color) & 1);
            const int r0 = HA - q + rr0, o0 = r0 * PW + c;
            constexpr int NT = (FH + 2 * Q0 + NW - 1) / NW;  // enough for the largest ring
#pragma unroll
            for (int t = 0; t < NT; t++) {
                if (t * NW >= hq) break;  // constant after unrolling
                if ((t + 1) * NW <= hq || warp + t * NW < hq)
                    if (!CHECK || inside(r0 + t * NW, c)) relax(o0 + t * NW * PW);
            }
            // the last q cells of each row (hq * q <= FT), first to the
            // warps with one chunk fewer (from warp hq % NW on)
            const int k = (tid + FT - 32 * (hq % NW)) % FT;
            if (k < hq * q) {
                const int rr = k / q, cc = FW / 2 + (k - rr * q);
                const int cq = XO - q + 2 * cc + ((par0 - 2 * q + rr + color) & 1);
                const int r = HA - q + rr;
                if (!CHECK || inside(r, cq)) relax(r * PW + cq);
            }
            __syncthreads();
        }
    };
    if (interior) sweeps(std::false_type{});
    else sweeps(std::true_type{});
    if (MODE == 1) {
        // one coarse cell per thread: FW/2 x FH/2 = 32 x 8, a warp per
        // coarse row.  Lanes 16-31 take the two children of a row in the
        // other order, so that each step's reads of a warp fall on even
        // words (lanes 0-15) and odd words (16-31): no bank conflicts.  The
        // four residuals are summed in the fixed order all the same.
        static_assert(FW / 2 == 32, "a warp per coarse row");
        const int ti = tid % (FW / 2), tj = tid / (FW / 2);
        const int I = blockIdx.x * (FW / 2) + ti, J = blockIdx.y * (FH / 2) + tj;
        const int sx = lane >> 4;  // 1: east child first
        if (I < nxc && J < nyc) {
            auto res = [&](int gi, int gj) {
                const int r = gj - gj0, c = gi - gi0, o = r * PW + c;
                const float cc = ps[o];
                float pE, pW, pN, pS;
                if (interior) {  // every neighbour is in the grid
                    pE = ps[o + 1]; pW = ps[o - 1]; pN = ps[o + PW]; pS = ps[o - PW];
                } else {
                    pE = gi + 1 < nx ? ps[o + 1] : cc; pW = gi > 0 ? ps[o - 1] : cc;
                    pN = gj + 1 < ny ? ps[o + PW] : cc; pS = gj > 0 ? ps[o - PW] : cc;
                }
                float sv = xs[o + 1] * (pE - cc);
                sv -= xs[o] * (cc - pW);
                sv += ys[o + PW] * (pN - cc);
                sv -= ys[o] * (cc - pS);
                return bs[o] - sv * ih2;
            };
            const int i = 2 * I, j = 2 * J;
            const float ra = res(i + sx, j), rb = res(i + 1 - sx, j);
            const float rcN = res(i + sx, j + 1), rdN = res(i + 1 - sx, j + 1);
            const float r00 = sx ? rb : ra, r10 = sx ? ra : rb;
            const float r01 = sx ? rdN : rcN, r11 = sx ? rcN : rdN;
            rc[(long)J * nxc + I] = 0.25f * (r00 + r10 + r01 + r11);
            ecz[(long)J * nxc + I] = 0.0f;
        }
    }
    {
        const long g0 = (long)(blockIdx.y * FH + trow) * nx + blockIdx.x * FW + tcol;
#pragma unroll
        for (int j = 0; j < (FW * FH) / FT; j++) {
            const int gi = blockIdx.x * FW + tcol, gj = blockIdx.y * FH + trow + RS * j;
            if (whole || (gi < nx && gj < ny)) {
                const float v = ps[(HA + trow + RS * j) * PW + XO + tcol];
                const long g = g0 + (long)RS * j * nx;
                if (MODE == 2 && p64) p64[g] = v64[MODE == 2 ? j : 0] + f2d(v);
                else p[g] = v;
            }
        }
    }
}

template <typename T>
__device__ __forceinline__ T flux_sum(int nx, int ny, int i, int j, const T *bx,
                                      const T *by, const T *p)
{
    // sum_f beta_f (p_nb - p_c) in the order E, W, N, S; wall faces have beta = 0
    long kc = (long)j * nx + i, kx = (long)j * (nx + 1) + i;
    T c = p[kc];
    T pE = (i + 1 < nx) ? p[kc + 1] : c, pW = (i > 0) ? p[kc - 1] : c;
    T pN = (j + 1 < ny) ? p[kc + nx] : c, pS = (j > 0) ? p[kc - nx] : c;
    T s = bx[kx + 1] * (pE - c);
    s -= bx[kx] * (c - pW);
    s += by[kc + nx] * (pN - c);
    s -= by[kc] * (c - pS);
    return s;
}

// Two FP64 red-black sweeps in one launch on the pre-scaled stencil of
// k_rbgs_sweep_w (p_c <- sum_f w_f p_nb - bt_c, four FMAs a cell in the same
// order), on a DW x DH tile: the iterate's window (halo HA) is staged in
// shared memory and the sweeps run on shrinking rings (red, black, red,
// black), each cell reading its weights and right-hand side from global
// memory (L1 / L2), so the tile's result equals two global sweeps.
// MODE 1: then the residual of the tile's cells averaged over 2x2 children
// into the coarse right-hand side rc, its pre-scaled copy btc = h_c^2 rc /
// diag_c (when btc is given) and a zero coarse correction.  The residual is
// taken from the last black half-sweep instead of b - A p: a relaxed cell
// satisfies its own equation, so after that half-sweep every black cell's
// residual is zero (to rounding) and a red cell's is -(1/h^2) sum_f beta_f
// delta_f, the deltas being the changes of its four black neighbours in that
// half-sweep (the residual identity of red-black Gauss-Seidel; four FP64
// operations for two cells instead of ten a cell).  The last black phase
// covers the tile's one-cell ring (halo 5), stores the tile's black cells
// and keeps their deltas in shared memory in place of the values.
// MODE 2: p + P e_c (bilinear prolongation of the coarse correction) formed
// while staging, then the sweeps (halo 4).
// The FP64 pipe bounds these kernels on this part (its instruction rate, not
// HBM), so the design counts FP64 instructions: fused sweeps, the residual
// identity, prolongation in FMAs; tiles of 32 x 16 spread the small levels
// over more SMs.
template <int MODE, int DW, int DH>
__global__ void __launch_bounds__(256)
k_smooth2_f64(int nx, int ny, double ih2, const double2 *__restrict__ w,
              const double *__restrict__ bt, const double *__restrict__ bx,
              const double *__restrict__ by, const double *__restrict__ pin,
              double *__restrict__ p, double *__restrict__ rc, double *__restrict__ ecz,
              double h2c, const double *__restrict__ invdc, double *__restrict__ btc,
              const double *__restrict__ ecp)
{
    constexpr int NT = 256;
    constexpr int HA = MODE == 1 ? 5 : 4;
    constexpr int PW = DW + 2 * HA, PH = DH + 2 * HA;
    __shared__ double ps[PH][PW];
    const int gi0 = blockIdx.x * DW - HA, gj0 = blockIdx.y * DH - HA;
    const int nxc = nx / 2, nyc = ny / 2;
    pdl_enter();
    for (int k = threadIdx.x; k < PH * PW; k += NT) {
        const int r = k / PW, c = k - r * PW, gi = gi0 + c, gj = gj0 + r;
        double v = 0.0;
        if (gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
            v = pin[(long)gj * nx + gi];
            if (MODE == 2) {
                // (9 c00 + 3 c10 + 3 c01 + c11) / 16 in three FMAs and an add
                const int I = gi >> 1, J = gj >> 1;
                const int I2 = min(max(I + ((gi & 1) ? 1 : -1), 0), nxc - 1);
                const int J2 = min(max(J + ((gj & 1) ? 1 : -1), 0), nyc - 1);
                const double c00 = ecp[(long)J * nxc + I], c10 = ecp[(long)J * nxc + I2];
                const double c01 = ecp[(long)J2 * nxc + I], c11 = ecp[(long)J2 * nxc + I2];
                v = fma(fma(9.0, c00, fma(3.0, c10 + c01, c11)), 0.0625, v);
            }
        }
        ps[r][c] = v;
    }
    __syncthreads();
    // ring q: local rows [HA - q, HA + DH + q), columns [HA - q, HA + DW + q)
#pragma unroll
    for (int ph = 0; ph < 4; ph++) {
        const int q = HA - 1 - ph, color = ph & 1;
        const int wq = DW + 2 * q, hq = DH + 2 * q, hw = wq / 2;
        for (int k = threadIdx.x; k < hq * hw; k += NT) {
            const int rr = k / hw, cc = k - rr * hw;
            const int r = HA - q + rr, gj = gj0 + r;
            const int c = HA - q + 2 * cc + ((gi0 + HA - q + gj + color) & 1);
            const int gi = gi0 + c;
            if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) continue;
            const long kc = (long)gj * nx + gi;
            const double2 we = w[2 * kc], sn = w[2 * kc + 1];
            double sm = fma(we.x, ps[r][c - 1], -bt[kc]);
            sm = fma(we.y, ps[r][c + 1], sm);
            sm = fma(sn.x, ps[r - 1][c], sm);
            sm = fma(sn.y, ps[r + 1][c], sm);
            if (MODE == 1 && ph == 3) {
                // last black half-sweep: tile cells go out now, every black
                // cell of the ring keeps its change for the residual
                if (r >= HA && r < HA + DH && c >= HA && c < HA + DW) p[kc] = sm;
                ps[r][c] = sm - ps[r][c];
            } else {
                ps[r][c] = sm;
            }
        }
        __syncthreads();
    }
    if (MODE == 1) {
        const long nxf = nx + 1;
        // -(1/h^2) sum_f beta_f delta_f of a red cell (its neighbours are black)
        auto sbd = [&](int gi, int gj) {
            const int r = gj - gj0, c = gi - gi0;
            const long kc = (long)gj * nx + gi, kx = (long)gj * nxf + gi;
            double sf = bx[kx + 1] * ps[r][c + 1];
            sf = fma(bx[kx], ps[r][c - 1], sf);
            sf = fma(by[kc + nx], ps[r + 1][c], sf);
            return fma(by[kc], ps[r - 1][c], sf);
        };
        const double kr = -0.25 * ih2;
        for (int k = threadIdx.x; k < (DW / 2) * (DH / 2); k += NT) {
            const int I = blockIdx.x * (DW / 2) + (k % (DW / 2));
            const int J = blockIdx.y * (DH / 2) + (k / (DW / 2));
            if (I >= nxc || J >= nyc) continue;
            // children (2I, 2J) and (2I+1, 2J+1) are red, the other two black
            const double rv = (sbd(2 * I, 2 * J) + sbd(2 * I + 1, 2 * J + 1)) * kr;
            const long kcc = (long)J * nxc + I;
            rc[kcc] = rv;
            ecz[kcc] = 0.0;
            if (btc) btc[kcc] = rv * h2c * invdc[kcc];
        }
    }
    for (int k = threadIdx.x; k < DH * DW; k += NT) {
        const int r = HA + k / DW, c = HA + (k % DW);
        const int gi = gi0 + c, gj = gj0 + r;
        // MODE 1 stored its black cells in the last phase
        if (gi < nx && gj < ny && (MODE != 1 || ((gi + gj) & 1) == 0)) p[(long)gj * nx + gi] = ps[r][c];
    }
}

// Coarse residual = average of the four children's b - A p; zeroes the coarse
// correction.  With btc, also the coarse right-hand side of the pre-scaled
// FP64 sweep, h_c^2 rc / diag_c.
template <typename T>
__global__ void k_restrict_residual(int nx, int ny, T ih2, const T *__restrict__ bx,
                                    const T *__restrict__ by, const T *__restrict__ b,
                                    const T *__restrict__ p, T *__restrict__ rc,
                                    T *__restrict__ ec, T h2c, const T *__restrict__ invdc,
                                    T *__restrict__ btc)
{
    pdl_enter();
    int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
    int nxc = nx / 2;
    if (I >= nxc) return;
    int i = 2 * I, j = 2 * J;
    T r00 = b[(long)j * nx + i] - flux_sum(nx, ny, i, j, bx, by, p) * ih2;
    T r10 = b[(long)j * nx + i + 1] - flux_sum(nx, ny, i + 1, j, bx, by, p) * ih2;
    T r01 = b[(long)(j + 1) * nx + i] - flux_sum(nx, ny, i, j + 1, bx, by, p) * ih2;
    T r11 = b[(long)(j + 1) * nx + i + 1] - flux_sum(nx, ny, i + 1, j + 1, bx, by, p) * ih2;
    long kc = (long)J * nxc + I;
    const T rv = T(0.25) * (r00 + r10 + r01 + r11);
    rc[kc] = rv;
    if (ec) ec[kc] = T(0);
    if (btc) btc[kc] = rv * h2c * invdc[kc];
}

template <typename T>
__global__ void k_prolong_add(int nxc, int nyc, const T *__restrict__ ec, T *__restrict__ ef)
{
    pdl_enter();
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    int nx = 2 * nxc;
    if (i >= nx) return;
    int I = i >> 1, J = j >> 1;
    int I2 = min(max(I + ((i & 1) ? 1 : -1), 0), nxc - 1);
    int J2 = min(max(J + ((j & 1) ? 1 : -1), 0), nyc - 1);
    T c00 = ec[(long)J * nxc + I], c10 = ec[(long)J * nxc + I2];
    T c01 = ec[(long)J2 * nxc + I], c11 = ec[(long)J2 * nxc + I2];
    ef[(long)j * nx + i] += (T(9) * c00 + T(3) * c10 + T(3) * c01 + c11) * T(0.0625);
}

template <typename T>
__global__ void k_residual(int nx, int ny, T ih2, const T *__restrict__ bx,
                           const T *__restrict__ by, const T *__restrict__ b,
                           const T *__restrict__ p, T *__restrict__ r)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    r[(long)j * nx + i] = b[(long)j * nx + i] - flux_sum(nx, ny, i, j, bx, by, p) * ih2;
}

template <typename T>
__global__ void k_invdiag(int nx, int ny, const double *__restrict__ bx,
                          const double *__restrict__ by, T *__restrict__ invd)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    long kc = (long)j * nx + i, kx = (long)j * (nx + 1) + i;
    double d = bx[kx + 1] + bx[kx] + by[kc + nx] + by[kc];
    invd[kc] = (T)(d > 0.0 ? 1.0 / d : 0.0);
}

__global__ void k_coarsen_beta(int nx, int ny, const double *__restrict__ bx,
                               const double *__restrict__ by, double *__restrict__ bxc,
                               double *__restrict__ byc)
{
    int nxc = nx / 2, nyc = ny / 2;
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long nxfc = (long)(nxc + 1) * nyc;
    if (k < nxfc) {
        int J = (int)(k / (nxc + 1)), I = (int)(k - (long)J * (nxc + 1));
        bxc[k] = 0.5 * (bx[(long)(2 * J) * (nx + 1) + 2 * I] + bx[(long)(2 * J + 1) * (nx + 1) + 2 * I]);
        return;
    }
    k -= nxfc;
    if (k >= (long)nxc * (nyc + 1)) return;
    int J = (int)(k / nxc), I = (int)(k - (long)J * nxc);
    byc[k] = 0.5 * (by[(long)(2 * J) * nx + 2 * I] + by[(long)(2 * J) * nx + 2 * I + 1]);
}

// Row pitch of the padded FP32 x-face copy: nx + 1 faces rounded up to a
// multiple of 4 values (16 bytes).
__host__ __device__ constexpr int xface_pitch(int nx) { return (nx + 4) & ~3; }

// Coefficients of one level in one pass, one thread per cell: the cell's
// west and south faces (and the east / north wall faces of the last column /
// row) from the finer level (mean of the two fine faces; at level 0 the
// caller's faces with the walls set to zero), their FP32 copies (the x-faces
// twice: packed and in padded rows), and the FP64 and FP32 inverse
// diagonals (the cell's four faces, recomputed locally).
__device__ __forceinline__ void level_coeffs_cell(int nx, int ny, int level0, int i, int j,
                                                  const double *__restrict__ fbx,
                                                  const double *__restrict__ fby,
                                                  double *__restrict__ bx, double *__restrict__ by,
                                                  float *__restrict__ bxf, float *__restrict__ byf,
                                                  float *__restrict__ bxp,
                                                  double *__restrict__ invd, float *__restrict__ invdf,
                                                  double *__restrict__ w4)
{
    const int fnx = 2 * nx;  // finer level width (unused at level 0)
    auto xface = [&](int I, int J) -> double {   // coefficient of x-face (I, J)
        if (I == 0 || I == nx) return 0.0;
        if (level0) return fbx[(long)J * (nx + 1) + I];
        return 0.5 * (fbx[(long)(2 * J) * (fnx + 1) + 2 * I] + fbx[(long)(2 * J + 1) * (fnx + 1) + 2 * I]);
    };
    auto yface = [&](int I, int J) -> double {
        if (J == 0 || J == ny) return 0.0;
        if (level0) return fby[(long)J * nx + I];
        return 0.5 * (fby[(long)(2 * J) * fnx + 2 * I] + fby[(long)(2 * J) * fnx + 2 * I + 1]);
    };
    const double w = xface(i, j), e = xface(i + 1, j), s = yface(i, j), n = yface(i, j + 1);
    const long kx = (long)j * (nx + 1) + i, kc = (long)j * nx + i;
    // FP32 copies by d2f_rn: (float) on integer instructions
    const float wf = d2f_rn(w);
    bx[kx] = w; bxf[kx] = wf;
    by[kc] = s; byf[kc] = d2f_rn(s);
    if (i == nx - 1) { bx[kx + 1] = e; bxf[kx + 1] = d2f_rn(e); }
    if (j == ny - 1) { by[kc + nx] = n; byf[kc + nx] = d2f_rn(n); }
    const int xp = xface_pitch(nx);
    float *rowp = bxp + (long)j * xp;
    rowp[i] = wf;
    if (i == nx - 1) {
        rowp[nx] = d2f_rn(e);
        for (int t = nx + 1; t < xp; t++) rowp[t] = 0.0f;  // padding
    }
    const double d = e + w + n + s;
    const double id = d > 0.0 ? recip_nr(d) : 0.0;
    invd[kc] = id;
    invdf[kc] = d2f_rn(id);
    if (w4) {
        reinterpret_cast<double2 *>(w4)[2 * kc] = make_double2(w * id, e * id);
        reinterpret_cast<double2 *>(w4)[2 * kc + 1] = make_double2(s * id, n * id);
    }
}

// The FP64 sweep weights w_f = beta_f / diag of every level from its faces
// and inverse diagonal (the products level_coeffs_cell forms when given w4),
// one thread per cell over all levels.
struct LevelWArgs {
    int nl;
    long start[17];  // first flat index of each level
    int nx[16];
    const double *bx[16], *by[16], *invd[16];
    double *w4[16];
};

__global__ void k_level_w(LevelWArgs a)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.start[a.nl]) return;
    int l = 0;
    while (t >= a.start[l + 1]) l++;
    const int nx = a.nx[l];
    const long kc = t - a.start[l];
    const int j = (int)(kc / nx), i = (int)(kc - (long)j * nx);
    const long kx = (long)j * (nx + 1) + i;
    const double id = a.invd[l][kc];
    const double w = a.bx[l][kx], e = a.bx[l][kx + 1], s = a.by[l][kc], n = a.by[l][kc + nx];
    reinterpret_cast<double2 *>(a.w4[l])[2 * kc] = make_double2(w * id, e * id);
    reinterpret_cast<double2 *>(a.w4[l])[2 * kc + 1] = make_double2(s * id, n * id);
}

__global__ void k_level_coeffs(int nx, int ny, int level0, const double *__restrict__ fbx,
                               const double *__restrict__ fby, double *__restrict__ bx,
                               double *__restrict__ by, float *__restrict__ bxf,
                               float *__restrict__ byf, float *__restrict__ bxp,
                               double *__restrict__ invd, float *__restrict__ invdf,
                               double *__restrict__ w4)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= nx) return;
    level_coeffs_cell(nx, ny, level0, i, j, fbx, fby, bx, by, bxf, byf, bxp, invd, invdf, w4);
}

// The small levels (from `first` on) in one CTA, level after level; a level
// reads the faces the previous one wrote (same block: visible after the
// barrier).
struct LevelCoeffArgs {
    int first, nl;
    int nx[16], ny[16];
    double *bx[16], *by[16], *invd[16], *w4[16];
    float *bxf[16], *byf[16], *bxp[16], *invdf[16];
};

__global__ void __launch_bounds__(1024) k_level_coeffs_small(LevelCoeffArgs a)
{
    for (int l = a.first; l < a.nl; l++) {
        const int nx = a.nx[l], ny = a.ny[l];
        for (int k = threadIdx.x; k < nx * ny; k += blockDim.x) {
            const int j = k / nx, i = k - j * nx;
            level_coeffs_cell(nx, ny, l == 0, i, j, a.bx[l - 1], a.by[l - 1], a.bx[l], a.by[l], a.bxf[l],
                              a.byf[l], a.bxp[l], a.invd[l], a.invdf[l], a.w4[l]);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ coarsest solve
// Dense A' = A + s 1 1^T (s = A_00, removes the constant null space), then its
// inverse, stored transposed (Ainv^T) so that the per-cycle solve x = A'^-1 r
// is one coalesced matrix-vector product.  A is negative semi-definite with
// the constants as null space and s < 0, so A' is negative definite and
// Gauss-Jordan elimination needs no pivoting: in place, column by column,
// row c is scaled by 1 / A'_cc and eliminated from every other row, the
// eliminated column becoming the inverse's (n^3 multiply-adds, all on one
// SM's FP64 pipe: the size of the coarsest level decides its cost).  One
// CTA; A' lives in shared memory when n^2 + n doubles fit in 96 KB, else in
// the scratch `Ag`.
__global__ void __launch_bounds__(1024)
k_coarse_inv(int nx, int ny, double h, const double *__restrict__ bx,
             const double *__restrict__ by, double *__restrict__ Ag, double *__restrict__ AinvT,
             int in_smem)
{
    extern __shared__ __align__(16) double cinv_sm[];
    __shared__ double colc[kMaxCoarsest];
    __shared__ double invp;
    const int n = nx * ny;
    const double hh = h * h;
    double *A = in_smem ? cinv_sm : Ag;
    for (int k = threadIdx.x; k < n * n; k += blockDim.x) A[k] = 0.0;
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        int i = c % nx, j = c / nx;
        long kx = (long)j * (nx + 1) + i, kc = c;
        double d = 0.0;
        if (i + 1 < nx) { d += bx[kx + 1] * (0.0 - 1.0); A[(c + 1) * n + c] = bx[kx + 1] * (1.0 - 0.0) / hh; }
        if (i > 0) { d -= bx[kx] * (1.0 - 0.0); A[(c - 1) * n + c] = -bx[kx] * (0.0 - 1.0) / hh; }
        if (j + 1 < ny) { d += by[kc + nx] * (0.0 - 1.0); A[(c + nx) * n + c] = by[kc + nx] * (1.0 - 0.0) / hh; }
        if (j > 0) { d -= by[kc] * (1.0 - 0.0); A[(c - nx) * n + c] = -by[kc] * (0.0 - 1.0) / hh; }
        A[c * n + c] = d / hh;
    }
    __syncthreads();
    __shared__ double s0;
    if (threadIdx.x == 0) s0 = A[0];
    __syncthreads();
    for (int k = threadIdx.x; k < n * n; k += blockDim.x) A[k] += s0;
    __syncthreads();
    for (int c = 0; c < n; c++) {
        if (threadIdx.x == 0) invp = 1.0 / A[c * n + c];
        __syncthreads();
        const double ip = invp;
        for (int r = threadIdx.x; r < n; r += blockDim.x) colc[r] = A[r * n + c];
        __syncthreads();
        // row c scaled (its pivot entry becomes 1 / pivot)
        for (int k = threadIdx.x; k < n; k += blockDim.x) A[c * n + k] = (k == c) ? ip : A[c * n + k] * ip;
        __syncthreads();
        // every other row: subtract its column-c multiple of row c; the
        // eliminated entry becomes -A'_rc / pivot
        for (int k = threadIdx.x; k < n * n; k += blockDim.x) {
            const int r = k / n, q = k - r * n;
            if (r == c) continue;
            A[k] = (q == c) ? -colc[r] * ip : A[k] - colc[r] * A[c * n + q];
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < n * n; k += blockDim.x) {
        const int r = k / n, q = k - r * n;
        AinvT[q * n + r] = A[k];
    }
}

// ------------------------------------------------------------ tail kernel
constexpr int kMaxLv = 16;
template <typename T>
struct TailArgs {
    int lt, nl;
    int nx[kMaxLv], ny[kMaxLv];
    T h2[kMaxLv], ih2[kMaxLv];
    T *e[kMaxLv], *r[kMaxLv];
    const T *bx[kMaxLv], *by[kMaxLv], *invd[kMaxLv];
    const double *ainvT;   // coarsest inverse, transposed
    int nu1, nu2;
    // shared-memory layout (tail_prepare): element offset of each level's
    // arrays, byte offset of the coarsest inverse (-1: read from ainvT)
    int off[kMaxLv];
    int inv_off;
};

// Shared-memory layout of the tail levels.  A level above the coarsest (even
// nx, ny) is split by colour: cell (i, j) of colour c = (i + j) & 1 sits at
// slot j * nx/2 + i/2 of colour c's block, and block c starts at
// c * (n/2 + kTailPad).  A colour phase then reads every array at
// consecutive slots from consecutive threads, free of bank conflicts (row-
// major storage would read every other word).  Each level holds e, r, 1/diag
// and the beta of each cell's east and north face (the west and south faces
// are the east and north faces of the neighbours, held by the other colour),
// one array after the other.  The coarsest level (odd sizes allowed, solved
// directly) keeps row-major e and r only.  The coarsest level's inverse
// (FP64, 8-byte aligned) follows when it takes at most 64 KB; otherwise the
// solve reads it from global memory.
constexpr int kTailPad = 16;
constexpr size_t kTailInvMax = 64 * 1024;
__host__ __device__ inline size_t tail_level_elems(int nx, int ny, bool coarsest)
{
    const size_t n = (size_t)nx * ny;
    return coarsest ? 2 * n : 5 * (n + 2 * kTailPad);
}

__host__ __device__ inline size_t tail_inv_bytes(int nco)
{
    const size_t b = (size_t)nco * nco * sizeof(double);
    return b <= kTailInvMax ? b : 0;
}

// Fills a.off / a.inv_off; returns the dynamic shared memory of the launch.
template <typename T>
size_t tail_prepare(TailArgs<T> &a)
{
    size_t n = 0;
    for (int l = a.lt; l < a.nl; l++) {
        a.off[l] = (int)n;
        n += tail_level_elems(a.nx[l], a.ny[l], l == a.nl - 1);
    }
    const size_t lv = (n * sizeof(T) + 7) & ~(size_t)7;
    const size_t inv = tail_inv_bytes(a.nx[a.nl - 1] * a.ny[a.nl - 1]);
    a.inv_off = inv ? (int)lv : -1;
    return lv + inv;
}

// One element (4 or 8 bytes) global -> shared by an asynchronous copy.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *d, const T *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(d)),
                 "l"(src), "n"(sizeof(T)));
}

// Copy n elements global -> shared: 16-byte copies while both addresses are
// 16-byte aligned (the element count rounded down to whole 16-byte chunks),
// single elements for the rest.
template <typename T>
__device__ __forceinline__ void stage_array(T *d, const T *src, int n, int tid, int nthr)
{
    constexpr int V = 16 / sizeof(T);
    int done = 0;
    if ((((uintptr_t)d | (uintptr_t)src) & 15) == 0) {
        const int nv = n / V;
        for (int k = tid; k < nv; k += nthr)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n"
                         ::"r"((unsigned)__cvta_generic_to_shared(d + V * k)), "l"(src + V * k));
        done = nv * V;
    }
    for (int k = done + tid; k < n; k += nthr) cp_async_elem(d + k, src + k);
}

// A split level's arrays (pointers into the kernel's shared memory).
template <typename T>
struct TailLv {
    T *e, *r, *iv, *cx, *cy;
};

template <typename T>
__device__ __forceinline__ TailLv<T> tail_lv(const TailArgs<T> &g, T *sm, int l)
{
    const int s = g.nx[l] * g.ny[l] + 2 * kTailPad;
    T *b = sm + g.off[l];
    return {b, b + s, b + 2 * s, b + 3 * s, b + 4 * s};
}

// Work of one level by a group of NT threads (thread index t): the whole
// block (NT = 1024), warps 0-3 (128, named barrier 1) or warp 0 (32), chosen
// by the level's size so that barriers are not wider than the work.
template <int NT>
__device__ __forceinline__ void gsync()
{
    if constexpr (NT == 1024) __syncthreads();
    else if constexpr (NT == 128) asm volatile("bar.sync 1, 128;\n" ::: "memory");
    else __syncwarp();
}

// Walk of the slots q = t, t + NT, ... of a w-wide grid as (row, column)
// without a division per step.
struct Walk {
    int a, b, da, db, w;
    __device__ Walk(int t, int NT, int w_) : w(w_)
    {
        a = t / w; b = t - a * w; da = NT / w; db = NT - da * w;
    }
    __device__ void next()
    {
        a += da; b += db;
        if (b >= w) { b -= w; a++; }
    }
};

// Red-black Gauss-Seidel on a split level: colour phases first .. 2 nsw - 1
// (phase 2s + c sweeps colour c of sweep s).  Same arithmetic, in the same
// order, as the row-major update (beta_E p_E + beta_W p_W + beta_N p_N +
// beta_S p_S - h^2 r) / diag, with p = 0 beyond the walls.
// Two consecutive values of a row (8 or 16 bytes, aligned: nx is even).
template <typename T> struct Pair;
template <> struct Pair<float> { using V = float2; };
template <> struct Pair<double> { using V = double2; };

// One colour phase on a split level with nx a multiple of 4: each thread
// updates the cells of slots m, m + 1 (m even) of one row with paired
// shared-memory loads.  In row j the cells of colour c are i = 2m + o,
// o = (j + c) & 1; their west / east neighbours are the other colour's slots
// m - 1 + o and m + o of the same row.
template <typename T, int NT>
__device__ __forceinline__ void tail_phase2(const TailArgs<T> &g, const TailLv<T> &v, int l, int c, int t)
{
    using P2 = typename Pair<T>::V;
    const int nx = g.nx[l], ny = g.ny[l], hx = nx / 2, bl = hx * ny + kTailPad, hp = hx / 2;
    const int oc = c * bl, ob = bl - oc;
    const T h2 = g.h2[l];
    auto ld2 = [](const T *a, int k) { return *reinterpret_cast<const P2 *>(a + k); };
    Walk w(t, NT, hp);
    for (int q = t; q < hp * ny; q += NT, w.next()) {
        const int j = w.a, m = 2 * w.b, o = (j + c) & 1, k = j * hx + m;
        const P2 eo = ld2(v.e, ob + k), xo = ld2(v.cx, ob + k);
        T pW0, pE0, pW1, pE1, bW0, bW1;
        if (o == 0) {
            pW0 = m > 0 ? v.e[ob + k - 1] : T(0);
            bW0 = m > 0 ? v.cx[ob + k - 1] : T(0);
            pE0 = eo.x; pW1 = eo.x; pE1 = eo.y; bW1 = xo.x;
        } else {
            pW0 = eo.x; pE0 = eo.y; pW1 = eo.y;
            pE1 = m + 2 < hx ? v.e[ob + k + 2] : T(0);
            bW0 = xo.x; bW1 = xo.y;
        }
        P2 eN, eS, yS;
        if (j + 1 < ny) eN = ld2(v.e, ob + k + hx); else eN.x = eN.y = T(0);
        if (j > 0) { eS = ld2(v.e, ob + k - hx); yS = ld2(v.cy, ob + k - hx); }
        else { eS.x = eS.y = T(0); yS.x = yS.y = T(0); }
        const P2 xc = ld2(v.cx, oc + k), yc = ld2(v.cy, oc + k), rc = ld2(v.r, oc + k), dc = ld2(v.iv, oc + k);
        T s0 = xc.x * pE0;
        s0 = fma(bW0, pW0, s0);
        s0 = fma(yc.x, eN.x, s0);
        s0 = fma(yS.x, eS.x, s0);
        T s1 = xc.y * pE1;
        s1 = fma(bW1, pW1, s1);
        s1 = fma(yc.y, eN.y, s1);
        s1 = fma(yS.y, eS.y, s1);
        P2 out;
        out.x = (s0 - h2 * rc.x) * dc.x;
        out.y = (s1 - h2 * rc.y) * dc.y;
        *reinterpret_cast<P2 *>(v.e + oc + k) = out;
    }
}

template <typename T, int NT>
__device__ __forceinline__ void tail_smooth(const TailArgs<T> &g, T *sm, int l, int nsw, int first, int t)
{
    const int nx = g.nx[l], ny = g.ny[l], hx = nx / 2, nh = hx * ny, bl = nh + kTailPad;
    const TailLv<T> v = tail_lv(g, sm, l);
    const T h2 = g.h2[l];
    if ((nx & 3) == 0) {
        for (int ph = first; ph < 2 * nsw; ph++) {
            tail_phase2<T, NT>(g, v, l, ph & 1, t);
            gsync<NT>();
        }
        return;
    }
    for (int ph = first; ph < 2 * nsw; ph++) {
        const int c = ph & 1, oc = c * bl, ob = bl - oc;
        Walk w(t, NT, hx);
        for (int q = t; q < nh; q += NT, w.next()) {
            const int j = w.a, m = w.b, o = (j + c) & 1, i = 2 * m + o, k = j * hx + m;
            const T pE = (i + 1 < nx) ? v.e[ob + k + o] : T(0);
            const T pW = (i > 0) ? v.e[ob + k - 1 + o] : T(0);
            const T bW = (i > 0) ? v.cx[ob + k - 1 + o] : T(0);
            const T pN = (j + 1 < ny) ? v.e[ob + k + hx] : T(0);
            const T pS = (j > 0) ? v.e[ob + k - hx] : T(0);
            const T bS = (j > 0) ? v.cy[ob + k - hx] : T(0);
            T s = v.cx[oc + k] * pE;
            s = fma(bW, pW, s);
            s = fma(v.cy[oc + k], pN, s);
            s = fma(bS, pS, s);
            v.e[oc + k] = (s - h2 * v.r[oc + k]) * v.iv[oc + k];
        }
        gsync<NT>();
    }
}

// Coarse residual of a split level l: the average of the four children's
// b - A p, with A p in the order E, W, N, S as flux_sum.  The coarse
// correction starts at zero; with fold, the red cells of a split coarse level
// get the result of the first red sweep from that zero start,
// (0 - h_c^2 r_c) / diag_c, so its smoothing starts with the black phase.
template <typename T, int NT>
__device__ __forceinline__ void tail_restrict(const TailArgs<T> &g, T *sm, int l, int fold, int t)
{
    const int nx = g.nx[l], ny = g.ny[l], hx = nx / 2, bl = hx * ny + kTailPad;
    const int nxc = nx / 2, nyc = ny / 2, nc = nxc * nyc;
    const bool cnat = l + 1 == g.nl - 1;
    const int hxc = nxc / 2, blc = nc / 2 + kTailPad;
    const TailLv<T> v = tail_lv(g, sm, l);
    const T ih2 = g.ih2[l], h2c = g.h2[l + 1];
    T *ec = sm + g.off[l + 1];
    T *rc = cnat ? ec + nc : ec + nc + 2 * kTailPad;
    const T *ivc = ec + 2 * (nc + 2 * kTailPad);  // split coarse level only
    auto res = [&](int i, int j) {
        const int c = (i + j) & 1, oc = c * bl, ob = bl - oc, o = i & 1, k = j * hx + (i >> 1);
        const T pc = v.e[oc + k];
        const T pE = (i + 1 < nx) ? v.e[ob + k + o] : pc;
        const T pW = (i > 0) ? v.e[ob + k - 1 + o] : pc;
        const T bW = (i > 0) ? v.cx[ob + k - 1 + o] : T(0);
        const T pN = (j + 1 < ny) ? v.e[ob + k + hx] : pc;
        const T pS = (j > 0) ? v.e[ob + k - hx] : pc;
        const T bS = (j > 0) ? v.cy[ob + k - hx] : T(0);
        T s = v.cx[oc + k] * (pE - pc);
        s -= bW * (pc - pW);
        s += v.cy[oc + k] * (pN - pc);
        s -= bS * (pc - pS);
        return v.r[oc + k] - s * ih2;
    };
    Walk w(t, NT, nxc);
    for (int k = t; k < nc; k += NT, w.next()) {
        const int J = w.a, I = w.b, i = 2 * I, j = 2 * J;
        T acc = res(i, j);
        acc += res(i + 1, j);
        acc += res(i, j + 1);
        acc += res(i + 1, j + 1);
        const T rv = T(0.25) * acc;
        if (cnat) {
            rc[k] = rv;
            ec[k] = T(0);
        } else {
            const int cc = (I + J) & 1, kc = cc * blc + J * hxc + (I >> 1);
            rc[kc] = rv;
            ec[kc] = (fold && cc == 0) ? (T(0) - h2c * rv) * ivc[kc] : T(0);
        }
    }
    gsync<NT>();
}

// e_l += P e_{l+1} (bilinear, weights 9/16, 3/16, 3/16, 1/16).  With
// black_only, the red cells are left out: the red phase that follows
// overwrites them without reading them.
template <typename T, int NT>
__device__ __forceinline__ void tail_prolong(const TailArgs<T> &g, T *sm, int l, int black_only, int t)
{
    const int nx = g.nx[l], ny = g.ny[l], hx = nx / 2, nh = hx * ny, bl = nh + kTailPad;
    const int nxc = nx / 2, nyc = ny / 2, hxc = nxc / 2, blc = nxc * nyc / 2 + kTailPad;
    const bool cnat = l + 1 == g.nl - 1;
    const T *ec = sm + g.off[l + 1];
    T *ef = sm + g.off[l];
    auto at = [&](int I, int J) {
        return cnat ? ec[J * nxc + I] : ec[((I + J) & 1) * blc + J * hxc + (I >> 1)];
    };
    for (int c = black_only ? 1 : 0; c < 2; c++) {
        Walk w(t, NT, hx);
        for (int q = t; q < nh; q += NT, w.next()) {
            const int j = w.a, m = w.b, i = 2 * m + ((j + c) & 1);
            const int I = m, J = j >> 1;
            const int I2 = min(max(I + ((i & 1) ? 1 : -1), 0), nxc - 1);
            const int J2 = min(max(J + ((j & 1) ? 1 : -1), 0), nyc - 1);
            const T c00 = at(I, J), c10 = at(I2, J), c01 = at(I, J2), c11 = at(I2, J2);
            ef[c * bl + j * hx + m] += (T(9) * c00 + T(3) * c10 + T(3) * c01 + c11) * T(0.0625);
        }
    }
    gsync<NT>();
}

template <typename T, int NT>
__device__ __forceinline__ void tail_down(const TailArgs<T> &g, T *sm, int l0, int l1, int t)
{
    for (int l = l0; l < l1; l++) {
        tail_smooth<T, NT>(g, sm, l, g.nu1, (l > g.lt && g.nu1 > 0) ? 1 : 0, t);
        tail_restrict<T, NT>(g, sm, l, g.nu1 > 0, t);
    }
}

template <typename T, int NT>
__device__ __forceinline__ void tail_up(const TailArgs<T> &g, T *sm, int l0, int l1, int t)
{
    for (int l = l1 - 1; l >= l0; l--) {
        tail_prolong<T, NT>(g, sm, l, g.nu2 > 0, t);
        tail_smooth<T, NT>(g, sm, l, g.nu2, 0, t);
    }
}

// The lower V-cycle (levels lt..L-1) in one CTA: the coefficients, the
// level-lt iterate and right-hand side and the coarsest inverse are loaded
// into shared memory (into the colour-split layout: pairs of row neighbours
// are loaded together and stored to their two colours), the cycle runs
// there, and the level-lt iterate is copied back.  Levels of at least 512
// cells use the whole block, those of at least 128 cells warps 0-3, the rest
// and the coarsest solve warp 0.
template <typename T>
__global__ void __launch_bounds__(1024) k_tail(const __grid_constant__ TailArgs<T> g)
{
    using P2 = typename Pair<T>::V;
    extern __shared__ __align__(16) unsigned char tail_sm[];
    __shared__ double xs[kMaxCoarsest];
    T *sm = reinterpret_cast<T *>(tail_sm);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int L = g.nl, lc = L - 1, nco = g.nx[lc] * g.ny[lc];
    const double *ainv = g.inv_off >= 0 ? reinterpret_cast<const double *>(tail_sm + g.inv_off) : g.ainvT;
    // the coefficients and the coarsest inverse are built before the solve
    // and not written during it: they are staged before the wait for the
    // previous grid (overlapping its tail); the level-lt iterate and
    // right-hand side it writes after the wait
    if (g.inv_off >= 0)
        stage_array(reinterpret_cast<double *>(tail_sm + g.inv_off), g.ainvT, nco * nco, tid, nthr);
    // pairs of row neighbours of all split levels, numbered level by level;
    // a batch of kStage pairs per thread has all its loads in flight before
    // its stores
    constexpr int kStage = sizeof(T) == 4 ? 4 : 2;
    int npairs = 0;
    for (int l = g.lt; l < lc; l++) npairs += g.nx[l] * g.ny[l] / 2;
    for (int base = 0; base < npairs; base += kStage * nthr) {
        P2 d[kStage], yn[kStage];
        T x0[kStage], x1[kStage];
        int s0[kStage], s1[kStage], lv[kStage];
#pragma unroll
        for (int u = 0; u < kStage; u++) {
            int q = base + u * nthr + tid, l = g.lt;
            lv[u] = -1;
            if (q >= npairs) continue;
            while (q >= g.nx[l] * g.ny[l] / 2) { q -= g.nx[l] * g.ny[l] / 2; l++; }
            // cells (i, j), (i + 1, j): colours c and 1 - c, slot m of both
            const int nx = g.nx[l], hx = nx / 2, bl = nx * g.ny[l] / 2 + kTailPad;
            const int j = q / hx, m = q - j * hx, i = 2 * m, k = j * nx + i, c = j & 1;
            lv[u] = l;
            s0[u] = c * bl + j * hx + m;
            s1[u] = (1 - c) * bl + j * hx + m;
            d[u] = __ldg(reinterpret_cast<const P2 *>(g.invd[l] + k));
            yn[u] = __ldg(reinterpret_cast<const P2 *>(g.by[l] + k + nx));
            x0[u] = __ldg(g.bx[l] + (long)j * (nx + 1) + i + 1);
            x1[u] = __ldg(g.bx[l] + (long)j * (nx + 1) + i + 2);
        }
#pragma unroll
        for (int u = 0; u < kStage; u++) {
            const int l = lv[u];
            if (l < 0) continue;
            const TailLv<T> v = tail_lv(g, sm, l);
            v.iv[s0[u]] = d[u].x; v.iv[s1[u]] = d[u].y;
            v.cy[s0[u]] = yn[u].x; v.cy[s1[u]] = yn[u].y;
            v.cx[s0[u]] = x0[u]; v.cx[s1[u]] = x1[u];
        }
    }
    pdl_enter();
    if (g.lt == lc) {
        stage_array(sm + g.off[lc], g.e[lc], nco, tid, nthr);
        stage_array(sm + g.off[lc] + nco, g.r[lc], nco, tid, nthr);
    } else {
        // the level-lt iterate and right-hand side, pairs of row neighbours
        const int nx = g.nx[g.lt], hx = nx / 2, n = nx * g.ny[g.lt], bl = n / 2 + kTailPad;
        const TailLv<T> v = tail_lv(g, sm, g.lt);
        Walk w(tid, nthr, hx);
        for (int q = tid; q < n / 2; q += nthr, w.next()) {
            const int j = w.a, m = w.b, k = j * nx + 2 * m, c = j & 1;
            const P2 ev = *reinterpret_cast<const P2 *>(g.e[g.lt] + k);
            const P2 rv = *reinterpret_cast<const P2 *>(g.r[g.lt] + k);
            const int s0 = c * bl + j * hx + m, s1 = (1 - c) * bl + j * hx + m;
            v.e[s0] = ev.x; v.e[s1] = ev.y;
            v.r[s0] = rv.x; v.r[s1] = rv.y;
        }
    }
    asm volatile("cp.async.wait_all;\n" ::);
    __syncthreads();
    int lb = g.lt;  // first level of warps 0-3
    while (lb < lc && g.nx[lb] * g.ny[lb] >= 512) lb++;
    int lw = lb;    // first level of warp 0
    while (lw < lc && g.nx[lw] * g.ny[lw] >= 128) lw++;
    tail_down<T, 1024>(g, sm, g.lt, lb, tid);
    if (tid < 128) {
        tail_down<T, 128>(g, sm, lb, lw, tid);
        if (tid < 32) {
            tail_down<T, 32>(g, sm, lw, lc, tid);
            // coarsest: x = A'^{-1} r, one row of the inverse per lane
            T *ecs = sm + g.off[lc];
            const T *rcs = ecs + nco;
            for (int k = tid; k < nco; k += 32) xs[k] = (double)rcs[k];
            __syncwarp();
            for (int k = tid; k < nco; k += 32) {
                double acc = 0.0;
                for (int q = 0; q < nco; q++) acc += ainv[q * nco + k] * xs[q];
                ecs[k] = (T)acc;
            }
            __syncwarp();
            tail_up<T, 32>(g, sm, lw, lc, tid);
        }
        gsync<128>();
        tail_up<T, 128>(g, sm, lb, lw, tid);
    }
    __syncthreads();
    tail_up<T, 1024>(g, sm, g.lt, lb, tid);
    const int nx0 = g.nx[g.lt], n0 = nx0 * g.ny[g.lt];
    T *eo = g.e[g.lt];
    if (g.lt == lc) {
        for (int k = tid; k < n0; k += nthr) eo[k] = sm[g.off[lc] + k];
    } else {
        const int hx = nx0 / 2, bl = n0 / 2 + kTailPad;
        const T *es = sm + g.off[g.lt];
        Walk w(tid, nthr, hx);
        for (int q = tid; q < n0 / 2; q += nthr, w.next()) {
            const int j = w.a, m = w.b, c = j & 1;
            P2 o;
            o.x = es[c * bl + j * hx + m];
            o.y = es[(1 - c) * bl + j * hx + m];
            *reinterpret_cast<P2 *>(eo + j * nx0 + 2 * m) = o;
        }
    }
}

// --------------------------------------------------------------- reductions
// Deterministic sum: each block folds a fixed strided slice in a fixed order
// and a fixed tree; the last block to finish folds the block partials.
// Returns true in the one thread that wrote the total.
template <typename F>
__device__ bool block_fold_and_finish(double v, double *part, unsigned *count,
                                      double *out)
{
    __shared__ double sh[kRedT];
    __shared__ bool last;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kRedT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sh[0];
        __threadfence();
        unsigned t = atomicAdd(count, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += kRedT) s += ((volatile double *)part)[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kRedT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *out = sh[0];
        *count = 0u;
        return true;
    }
    return false;
}

// Convergence test of the device-side solve loop (one thread, after the
// residual norm res[2] is final): updates the cycle count and relative
// residual and sets the WHILE condition.
__device__ void solve_check(SolveCtl *ctl, const double *res, cudaGraphConditionalHandle hnd,
                            int first, int inc)
{
    const double nb = sqrt(res[1]);
    if (first) { ctl->cycles = 0; ctl->zero_p = nb == 0.0 ? 1 : 0; }
    else ctl->cycles += inc;
    const double rr = nb == 0.0 ? 0.0 : sqrt(res[2]) / nb;
    ctl->rr = rr;
    const unsigned go = (nb != 0.0 && rr > ctl->tol && ctl->cycles < ctl->max_cycles && isfinite(rr)) ? 1u : 0u;
    cudaGraphSetConditional(hnd, go);
}

struct NoOp {};

__global__ void __launch_bounds__(kRedT)
k_sum(long n, const double *__restrict__ a, double *part, unsigned *count, double *out)
{
    double s = 0.0;
    for (long k = (long)blockIdx.x * kRedT + threadIdx.x; k < n; k += (long)gridDim.x * kRedT)
        s += a[k];
    block_fold_and_finish<NoOp>(s, part, count, out);
}

// r0 = b - sum/n; accumulates sum r0^2.  With bt, also the right-hand side
// of the pre-scaled FP64 sweep, h^2 r0 / diag.
__global__ void __launch_bounds__(kRedT)
k_sub_mean(long n, const double *__restrict__ b, const double *__restrict__ sum,
           double *__restrict__ r0, double h2, const double *__restrict__ invd,
           double *__restrict__ bt, double *part, unsigned *count, double *out)
{
    // the mean once per block (one FP64 division, the same value everywhere)
    __shared__ double mb;
    if (threadIdx.x == 0) mb = *sum / (double)n;
    __syncthreads();
    const double m = mb;
    double s = 0.0;
    for (long k = (long)blockIdx.x * kRedT + threadIdx.x; k < n; k += (long)gridDim.x * kRedT) {
        double v = b[k] - m;
        r0[k] = v;
        if (bt) bt[k] = v * h2 * invd[k];
        s += v * v;
    }
    block_fold_and_finish<NoOp>(s, part, count, out);
}

__global__ void k_apply_mean(long n, double *__restrict__ p, const double *__restrict__ sum,
                             double *__restrict__ dst)
{
    __shared__ double mb;  // the mean once per block
    if (threadIdx.x == 0) mb = *sum / (double)n;
    __syncthreads();
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[k] = p[k] - mb;
}

// sum (b0 - A p)^2 over the fine grid, FP64, into res[2].  With rf != NULL
// also writes the FP32 residual and zeroes the FP32 correction for the inner
// cycle.  check = 1 (first) or 2 (after `inc` cycles): the block that
// finishes the sum also runs the convergence test of the graph's solve loop.
__global__ void __launch_bounds__(kRedT)
k_resnorm(int nx, int ny, double ih2, const double *__restrict__ bx,
          const double *__restrict__ by, const double *__restrict__ b0,
          const double *__restrict__ p, float *__restrict__ rf, float *__restrict__ ef,
          double *part, unsigned *count, double *res, SolveCtl *ctl,
          cudaGraphConditionalHandle hnd, int check, int inc)
{
    pdl_enter();
    // an equal contiguous share of the cells per block (the grid is one
    // wave of resident blocks), consecutive cells on consecutive threads
    const long n = (long)nx * ny;
    const long per = (n + gridDim.x - 1) / gridDim.x;
    const long ke = min(n, (long)blockIdx.x * per + per);
    long k = (long)blockIdx.x * per + threadIdx.x;
    int j = (int)(k / nx), i = (int)(k - (long)j * nx);
    double s = 0.0;
    for (; k < ke; k += kRedT) {
        const double r = b0[k] - flux_sum(nx, ny, i, j, bx, by, p) * ih2;
        s += r * r;
        if (rf) { rf[k] = d2f_rn(r); ef[k] = 0.0f; }
        for (i += kRedT; i >= nx; i -= nx) j++;
    }
    if (block_fold_and_finish<NoOp>(s, part, count, res + 2) && check)
        solve_check(ctl, res, hnd, check == 1, inc);
}

__global__ void k_add_f32(long n, const float *__restrict__ e, double *__restrict__ p)
{
    pdl_enter();
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] += f2d(e[k]);
}

__global__ void k_finalize(long n, const double *__restrict__ e0, const double *__restrict__ sum,
                           const SolveCtl *__restrict__ ctl, double *__restrict__ p)
{
    __shared__ double mb;  // the mean once per block
    if (threadIdx.x == 0) mb = *sum / (double)n;
    __syncthreads();
    long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = ctl->zero_p ? 0.0 : e0[k] - mb;
}

// The other buffer of a level's iterate (sweeps read one and write the other).
template <typename T>
T *other(LevelT<T> &a, T *cur) { return cur == a.e ? a.e2 : a.e; }

// One fused FP32 smoother launch of MODE on level v: reads the iterate from
// pin (one of the level's two buffers) and writes p; stages by TMA where the
// level has tensor maps.
template <int MODE>
void launch_smooth2(const Level &v, const LevelT<float> &a, const float *pin, float *p,
                    float *rc, float *ecz, const float *ecp, cudaStream_t s,
                    double *p64 = nullptr)
{
    dim3 g2(cdiv(v.nx, FW), cdiv(v.ny, FH));
    const float h2 = (float)(v.h * v.h), ih2 = MODE == 1 ? (float)(1.0 / (v.h * v.h)) : 0.0f;
    TileMaps tm;
    memset(&tm, 0, sizeof(tm));
    note_launch();
    if (v.tma && (pin == a.e || pin == a.e2)) {
        const LevelTma &w = v.tm[MODE == 1 ? 1 : 0];
        tm.p = pin == a.e ? w.e : w.e2;
        tm.b = w.r;
        tm.d = w.invd;
        tm.y = w.by;
        tm.fault = v.fault;
        tm.x = w.bxp;
        launch_pdl(k_smooth2t_f32<MODE>, g2, FT, 0, s, v.nx, v.ny, h2, ih2, p, rc, ecz, ecp, p64, tm);
    } else {
        launch_pdl(k_smooth2_f32<MODE, false>, g2, FT, 0, s, v.nx, v.ny, h2, ih2, a.bx, a.by,
                   a.invd, a.r, pin, p, rc, ecz, ecp, p64, tm);
    }
}

// One fused FP64 smoother launch of MODE on level v (pin -> p): 64 x 32 tiles
// from 512^2 cells up, 32 x 16 below (more tiles, so more SMs share the FP64
// work of a small level).
template <int MODE>
void launch_smooth2_f64(const Level &v, const LevelT<double> &a, const double *pin, double *p,
                        double *rc, double *ecz, double h2c, const double *invdc, double *btc,
                        const double *ecp, cudaStream_t s)
{
    const double ih2 = 1.0 / (v.h * v.h);
    note_launch();
    if ((long)v.nx * v.ny >= (1L << 18)) {
        dim3 g(cdiv(v.nx, 64), cdiv(v.ny, 32));
        launch_pdl(k_smooth2_f64<MODE, 64, 32>, g, 256, 0, s, v.nx, v.ny, ih2, (const double2 *)a.w,
                   (const double *)a.bt, (const double *)a.bx, (const double *)a.by, pin, p, rc,
                   ecz, h2c, invdc, btc, ecp);
    } else {
        dim3 g(cdiv(v.nx, 32), cdiv(v.ny, 16));
        launch_pdl(k_smooth2_f64<MODE, 32, 16>, g, 256, 0, s, v.nx, v.ny, ih2, (const double2 *)a.w,
                   (const double *)a.bt, (const double *)a.bx, (const double *)a.by, pin, p, rc,
                   ecz, h2c, invdc, btc, ecp);
    }
}

// nsw sweeps on one level, reading the iterate from cur and leaving it in the
// returned buffer: FP32 in fused pairs, FP64 one sweep per launch (the FP64
// sweep is bound by the FP64 pipe, where fusing only adds halo work).
template <typename T>
T *smooth(const Level &v, LevelT<T> &a, T *cur, int nsw, bool fine, cudaStream_t s)
{
    const T h2 = (T)(v.h * v.h);
    int k = 0;
    if constexpr (sizeof(T) == 4) {
        for (; k + 2 <= nsw; k += 2) {
            const bool pr = fine && prof_on(kProfSweep32);
            if (pr) prof_mark(s, true);
            T *nxt = other(a, cur);
            launch_smooth2<0>(v, a, cur, nxt, nullptr, nullptr, nullptr, s);
            cur = nxt;
            if (pr) prof_mark(s, false);
        }
    }
    dim3 g(cdiv(v.nx, TW), cdiv(v.ny, TH));
    for (; k < nsw; k++) {
        const bool pr = fine && sizeof(T) == 8 && prof_on(kProfSweep64);
        if (pr) prof_mark(s, true);
        note_launch();
        T *nxt = other(a, cur);
        if constexpr (sizeof(T) == 8)
            launch_pdl(k_rbgs_sweep_w, g, TT, 0, s, v.nx, v.ny, (const double2 *)a.w,
                       (const double *)a.bt, (const double *)cur, nxt);
        else
            launch_pdl(k_rbgs_sweep<T>, g, TT, 0, s, v.nx, v.ny, h2, a.bx, a.by, a.invd, a.r,
                       (const T *)cur, nxt);
        cur = nxt;
        if (pr) prof_mark(s, false);
    }
    return cur;
}

// One V(nu1, nu2) cycle on the level-0 data of precision T.  Every level's
// iterate moves between its two buffers (cur[l]); the coarse corrections
// start in the canonical buffer, which the restriction zeroes, and level 0
// ends in its canonical buffer (copied back when the sweep count is odd).
// Cycles with nu1 = nu2 = 2 use the fused kernels (sweeps + residual +
// restriction going down, prolongation + sweeps going up; FP32 and FP64
// alike, other sweep counts one launch per sweep); given add64 (the
// FP64 iterate of the defect correction), such a cycle adds its level-0
// result to it in the last smoother and returns true (the FP32 level-0
// iterate is then not stored).
template <typename T>
bool vcycle(MG &mg, int nu1, int nu2, cudaStream_t s, double *add64 = nullptr)
{
    auto lvT = [&](int l) -> LevelT<T> & {
        if constexpr (sizeof(T) == 8) return mg.lv[l].d; else return mg.lv[l].f;
    };
    const int L = mg.L, lt = sizeof(T) == 8 ? mg.tail : mg.tail_f;
    constexpr bool f32 = sizeof(T) == 4;
    const bool fused = nu1 == 2 && nu2 == 2;
    T *cur[kMaxLv];
    for (int l = 0; l < L; l++) cur[l] = lvT(l).e;
    for (int l = 0; l < lt; l++) {
        Level &v = mg.lv[l];
        LevelT<T> &a = lvT(l), &c = lvT(l + 1);
        if (fused) {
            const bool pr = l == 0 && prof_on(f32 ? kProfSweep32 : kProfSweep64);
            if (pr) prof_mark(s, true);
            T *nxt = other(a, cur[l]);
            if constexpr (f32) {
                launch_smooth2<1>(v, a, cur[l], nxt, c.r, c.e, nullptr, s);
            } else {
                // the next level's pre-scaled right-hand side where it is swept
                // by the fused kernels (above the tail)
                const double hc = mg.lv[l + 1].h;
                launch_smooth2_f64<1>(v, a, cur[l], nxt, c.r, c.e, hc * hc, c.invd,
                                      l + 1 < lt ? c.bt : nullptr, nullptr, s);
            }
            if (pr) prof_mark(s, false);
            cur[l] = nxt;
        } else {
            cur[l] = smooth<T>(v, a, cur[l], nu1, l == 0, s);
            dim3 gr(cdiv(v.nx / 2, 128), v.ny / 2);
            note_launch();
            // the next level's pre-scaled right-hand side where it is swept by
            // k_rbgs_sweep_w (FP64, above the tail)
            const bool wt = sizeof(T) == 8 && l + 1 < lt;
            const double hc = mg.lv[l + 1].h;
            launch_pdl(k_restrict_residual<T>, gr, 128, 0, s, v.nx, v.ny, (T)(1.0 / (v.h * v.h)),
                       a.bx, a.by, a.r, (const T *)cur[l], c.r, c.e, (T)(hc * hc),
                       (const T *)c.invd, wt ? c.bt : (T *)nullptr);
        }
        cur[l + 1] = c.e;
    }
    TailArgs<T> ta;
    ta.lt = lt;
    ta.nl = L;
    for (int l = lt; l < L; l++) {
        Level &v = mg.lv[l];
        LevelT<T> &a = lvT(l);
        ta.nx[l] = v.nx; ta.ny[l] = v.ny;
        ta.h2[l] = (T)(v.h * v.h); ta.ih2[l] = (T)(1.0 / (v.h * v.h));
        ta.e[l] = a.e; ta.r[l] = a.r; ta.bx[l] = a.bx; ta.by[l] = a.by; ta.invd[l] = a.invd;
    }
    ta.e[lt] = cur[lt];
    ta.ainvT = mg.lu + (size_t)mg.lv[mg.L - 1].nx * mg.lv[mg.L - 1].ny * mg.lv[mg.L - 1].nx * mg.lv[mg.L - 1].ny;
    ta.nu1 = nu1;
    ta.nu2 = nu2;
    note_launch();
    const size_t smem = tail_prepare(ta);
    launch_pdl(k_tail<T>, 1, 1024, smem, s, ta);
    for (int l = lt - 1; l >= 0; l--) {
        Level &v = mg.lv[l];
        LevelT<T> &a = lvT(l);
        if (fused) {
            const bool pr = l == 0 && (prof_on(f32 ? kProfSweep32 : kProfSweep64) ||
                                       (f32 && add64 && prof_on(kProfProlong32)));
            if (pr) prof_mark(s, true);
            if constexpr (f32) {
                if (l == 0 && add64) {
                    launch_smooth2<2>(v, a, cur[0], nullptr, nullptr, nullptr, cur[1], s, add64);
                    if (pr) prof_mark(s, false);
                    return true;
                }
            }
            T *nxt = other(a, cur[l]);
            if constexpr (f32)
                launch_smooth2<2>(v, a, cur[l], nxt, nullptr, nullptr, cur[l + 1], s);
            else
                launch_smooth2_f64<2>(v, a, cur[l], nxt, nullptr, nullptr, 0.0, nullptr, nullptr,
                                      cur[l + 1], s);
            if (pr) prof_mark(s, false);
            cur[l] = nxt;
        } else {
            dim3 gp(cdiv(v.nx, 128), v.ny);
            note_launch();
            launch_pdl(k_prolong_add<T>, gp, 128, 0, s, v.nx / 2, v.ny / 2, (const T *)cur[l + 1],
                       cur[l]);
            cur[l] = smooth<T>(v, a, cur[l], nu2, l == 0, s);
        }
    }
    if (cur[0] != lvT(0).e)
        cudaMemcpyAsync(lvT(0).e, cur[0], (size_t)mg.lv[0].nx * mg.lv[0].ny * sizeof(T),
                        cudaMemcpyDeviceToDevice, s);
    return false;
}

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// ------------------------------------------------------------------- host
namespace {
std::atomic<unsigned long long> g_launches{0};
constexpr int kProfMax = 16384;
struct Prof {
    int kind = -1;
    int n = 0;
    bool open = false;
    std::vector<cudaEvent_t> ev;
} g_prof;
}  // namespace

void note_launch(int n) { g_launches += (unsigned long long)(long long)n; }

const char *fault_message(int code)
{
    switch (code) {
    case 1: return "a smoother's staging wait timed out (50 ms); its tile was skipped";
    case 2: return "a smoother's shared-memory tiles are misaligned";
    case 3: return "a smoother's staging copies did not land within 0.5 s";
    default: return "a smoother reported an unknown fault";
    }
}

cudaError_t set_stall_staging(int on)
{
    const int v = on ? 1 : 0;
    return cudaMemcpyToSymbol(g_stall_staging, &v, sizeof(int));
}
unsigned long long launch_count() { return g_launches.load(); }
bool prof_on(int kind) { return g_prof.kind == kind && g_prof.n < kProfMax; }
static bool prof_active() { return g_prof.kind >= 0 && g_prof.kind < kProfPre; }
bool profiling_active() { return prof_active(); }

void raise_smem_limit(const void *kernel, int bytes)
{
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> set;
    std::lock_guard<std::mutex> lock(mu);
    for (auto &e : set)
        if (e.first == kernel) {
            if (bytes > e.second) {
                cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
                e.second = bytes;
            }
            return;
        }
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    set.emplace_back(kernel, bytes);
}
void prof_mark(cudaStream_t s, bool start)
{
    if (start) {
        cudaEventRecord(g_prof.ev[2 * g_prof.n], s);
        g_prof.open = true;
    } else if (g_prof.open) {
        cudaEventRecord(g_prof.ev[2 * g_prof.n + 1], s);
        g_prof.n++;
        g_prof.open = false;
    }
}

bool prof_begin(int kind)
{
    if (g_prof.ev.empty()) {
        g_prof.ev.resize(2 * kProfMax);
        for (auto &e : g_prof.ev)
            if (cudaEventCreate(&e) != cudaSuccess) return false;
    }
    g_prof.kind = kind;
    g_prof.n = 0;
    g_prof.open = false;
    return true;
}

bool prof_end(double *total_ms, int *launches)
{
    double t = 0.0;
    for (int k = 0; k < g_prof.n; k++) {
        if (cudaEventSynchronize(g_prof.ev[2 * k + 1]) != cudaSuccess) return false;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, g_prof.ev[2 * k], g_prof.ev[2 * k + 1]) != cudaSuccess)
            return false;
        t += ms;
    }
    if (total_ms) *total_ms = t;
    if (launches) *launches = g_prof.n;
    g_prof.kind = -1;
    g_prof.n = 0;
    return true;
}

bool mg_levels(int nx, int ny, std::vector<int> &nxs, std::vector<int> &nys)
{
    nxs.assign(1, nx);
    nys.assign(1, ny);
    while ((int)nxs.size() < kMaxLv && nx % 2 == 0 && ny % 2 == 0 && (long)nx * ny > 16) {
        nx /= 2; ny /= 2;
        nxs.push_back(nx); nys.push_back(ny);
    }
    return (long)nx * ny <= kMaxCoarsest;
}

// The CUDA driver API's tensor-map encoder, looked up once through the
// runtime (no link against the driver library); null where the installed
// driver lacks it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return (PFN_cuTensorMapEncodeTiled_v12000)f;
    }();
    return fn;
}

// 2-D map of a row-major FP32 array of w x hgt values with a bw x bh box
// (no swizzle, zero fill outside the array).
static bool map2d(CUtensorMap *m, const float *base, int w, int hgt, int bw, int bh)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || w < bw || hgt < bh || (w & 3) != 0 || ((uintptr_t)base & 15) != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)hgt};
    const cuuint64_t strides[1] = {(cuuint64_t)w * 4};
    const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh}, es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of a level's FP32 smoother operands for both window shapes
// (FW + 2 XO) x (FH + 2 HA) with (XO, HA) = (4, 4) and (8, 5); beta_y windows
// have one more row; beta_x windows come from the padded rows.  Needs rows
// of a multiple of 4 values (16-byte strides).
static bool encode_level_maps(Level &v)
{
    const LevelT<float> &a = v.f;
    for (int k = 0; k < 2; k++) {
        const int bw = FW + 2 * (k ? 8 : 4), bh = FH + 2 * (k ? 5 : 4);
        LevelTma &w = v.tm[k];
        if (!map2d(&w.e, a.e, v.nx, v.ny, bw, bh) || !map2d(&w.e2, a.e2, v.nx, v.ny, bw, bh) ||
            !map2d(&w.r, a.r, v.nx, v.ny, bw, bh) || !map2d(&w.invd, a.invd, v.nx, v.ny, bw, bh) ||
            !map2d(&w.by, a.by, v.nx, v.ny + 1, bw, bh + 1) ||
            !map2d(&w.bxp, a.bxp, xface_pitch(v.nx), v.ny, bw, bh))
            return false;
    }
    return true;
}

// Blocks of the reduction kernels (residual norm, sums): as many as are
// resident at once on the device (one wave: each block's share of the cells
// is then done in one go), at most 8 per SM of 152.
static int resident_red_blocks()
{
    static int nb = 0;
    if (nb == 0) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_resnorm, kRedT, 0) != cudaSuccess ||
            sms <= 0 || per <= 0) {
            cudaGetLastError();
            return 8 * 152;
        }
        nb = std::min(per * sms, 8 * 152);
    }
    return nb;
}

size_t mg_layout(MG &mg, int nx, int ny, double h, char *base)
{
    int nxs[16], nys[16], L = 0;
    nxs[0] = nx; nys[0] = ny; L = 1;
    while (L < kMaxLv && nx % 2 == 0 && ny % 2 == 0 && (long)nx * ny > 16) {
        nx /= 2; ny /= 2;
        nxs[L] = nx; nys[L] = ny; L++;
    }
    const long nc = (long)nxs[L - 1] * nys[L - 1];
    mg.red_blocks = resident_red_blocks();
    char *q = base;
    size_t off = 0;
    auto take = [&](size_t b) -> void * {
        void *r = base ? (void *)(q + off) : nullptr;
        off += al(b);
        return r;
    };
    mg.L = L;
    for (int l = 0; l < L; l++) {
        Level &v = mg.lv[l];
        v.nx = nxs[l]; v.ny = nys[l]; v.h = h * (double)(1 << l);
        size_t n = (size_t)v.nx * v.ny, fx = (size_t)(v.nx + 1) * v.ny, fy = (size_t)v.nx * (v.ny + 1);
        v.d.e = (double *)take(n * 8); v.d.e2 = (double *)take(n * 8);
        v.d.r = (double *)take(n * 8); v.d.invd = (double *)take(n * 8);
        v.d.bx = (double *)take(fx * 8); v.d.by = (double *)take(fy * 8);
        v.d.w = (double *)take(n * 32); v.d.bt = (double *)take(n * 8);
        v.f.e = (float *)take(n * 4); v.f.e2 = (float *)take(n * 4);
        v.f.r = (float *)take(n * 4); v.f.invd = (float *)take(n * 4);
        v.f.bx = (float *)take(fx * 4); v.f.by = (float *)take(fy * 4);
        v.f.bxp = (float *)take((size_t)xface_pitch(v.nx) * v.ny * 4);
    }
    mg.lu = (double *)take((size_t)nc * nc * 8 * 2);  // A' and its transposed inverse
    mg.piv = (int *)take((size_t)nc * 4);
    mg.red = (double *)take((size_t)(mg.red_blocks + 16) * 8);
    mg.red_count = (unsigned *)take(64);
    mg.ctl = (SolveCtl *)take(sizeof(SolveCtl));
    for (int l = 0; l < L; l++) {
        Level &v = mg.lv[l];
        v.fault = base ? &mg.ctl->fault : nullptr;
        v.tma = base && encode_level_maps(v);
    }
    int t = 0;
    while (t < L && (long)nxs[t] * nys[t] > kTailCells) t++;
    mg.tail = std::min(t, L - 1);
    t = 0;
    while (t < L && (long)nxs[t] * nys[t] > kTailCellsF32) t++;
    mg.tail_f = std::min(t, L - 1);
    return off;
}

cudaError_t mg_alloc(MG &mg, int nx, int ny, double h)
{
    const size_t bytes = mg_layout(mg, nx, ny, h, nullptr);
    cudaError_t e = cudaMalloc(&mg.mem, bytes);
    if (e != cudaSuccess) { mg.mem = nullptr; return e; }
    mg_layout(mg, nx, ny, h, (char *)mg.mem);
    mg.bytes = bytes;
    e = cudaMallocHost((void **)&mg.red_host, 16 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&mg.ctl_host, sizeof(SolveCtl));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&mg.cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&mg.cap_body, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemset(mg.mem, 0, bytes);
    return e;
}

void mg_free(MG &mg)
{
    for (auto &g : mg.graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    mg.graphs.clear();
    if (mg.cap) cudaStreamDestroy(mg.cap);
    if (mg.cap_body) cudaStreamDestroy(mg.cap_body);
    mg.cap = mg.cap_body = nullptr;
    if (mg.ctl_host) cudaFreeHost(mg.ctl_host);
    mg.ctl_host = nullptr;
    if (mg.mem) cudaFree(mg.mem);
    if (mg.red_host) cudaFreeHost(mg.red_host);
    mg.mem = nullptr;
    mg.red_host = nullptr;
    mg.L = 0;
}

// One launch of one kernel of the cycle on the hierarchy's current data, for
// kernel timing: op 0 FP32 two-sweep smoother, 1 FP64 sweep, 3 FP32 sweeps +
// restriction, 4 FP32 prolongation + sweeps (+ the FP64 update at level 0),
// 7 FP64 sweeps + restriction, 8 FP64 prolongation + sweeps, all at
// `level`; 5 FP32 tail, 6 FP64 residual norm of the mixed solve (level 0).  Returns the cells of the level, or -1 if the op does not exist
// there.  Writes only solve scratch (second iterate buffers, coarse
// right-hand sides and corrections, the level-0 FP64 iterate copy, FP32
// residual, norm partials).
long mg_bench_op(MG &mg, int op, int level, cudaStream_t s)
{
    if (level < 0 || level >= mg.L) return -1;
    Level &v = mg.lv[level];
    const long cells = (long)v.nx * v.ny;
    switch (op) {
    case 0: smooth<float>(v, v.f, v.f.e, 2, false, s); return cells;
    case 1: ensure_fp64_w(mg, s); smooth<double>(v, v.d, v.d.e, 1, false, s); return cells;
    case 3:
        if (level >= mg.tail_f) return -1;
        launch_smooth2<1>(v, v.f, v.f.e, v.f.e2, mg.lv[level + 1].f.r, mg.lv[level + 1].f.e2,
                          nullptr, s);
        return cells;
    case 4:  // at level 0 with the FP64 update, as in the defect-correction cycle
        if (level >= mg.tail_f) return -1;
        launch_smooth2<2>(v, v.f, v.f.e, v.f.e2, nullptr, nullptr, mg.lv[level + 1].f.e, s,
                          level == 0 ? v.d.e : nullptr);
        return cells;
    case 5: {
        const int lt = mg.tail_f, L = mg.L;
        TailArgs<float> ta;
        ta.lt = lt;
        ta.nl = L;
        for (int l = lt; l < L; l++) {
            Level &w = mg.lv[l];
            ta.nx[l] = w.nx; ta.ny[l] = w.ny;
            ta.h2[l] = (float)(w.h * w.h); ta.ih2[l] = (float)(1.0 / (w.h * w.h));
            ta.e[l] = w.f.e2; ta.r[l] = w.f.r; ta.bx[l] = w.f.bx; ta.by[l] = w.f.by; ta.invd[l] = w.f.invd;
        }
        const long nc = (long)mg.lv[L - 1].nx * mg.lv[L - 1].ny;
        ta.ainvT = mg.lu + nc * nc;
        ta.nu1 = 2;
        ta.nu2 = 2;
        note_launch();
        const size_t smem = tail_prepare(ta);
        launch_pdl(k_tail<float>, 1, 1024, smem, s, ta);
        return (long)mg.lv[lt].nx * mg.lv[lt].ny;
    }
    case 7:
    case 8: {  // the fused FP64 smoothers (7: sweeps + restriction, 8: prolongation + sweeps)
        if (level >= mg.tail) return -1;
        ensure_fp64_w(mg, s);
        Level &c = mg.lv[level + 1];
        if (op == 7)
            launch_smooth2_f64<1>(v, v.d, v.d.e, v.d.e2, c.d.r, c.d.e2, c.h * c.h, c.d.invd,
                                  level + 1 < mg.tail ? c.d.bt : nullptr, nullptr, s);
        else
            launch_smooth2_f64<2>(v, v.d, v.d.e, v.d.e2, nullptr, nullptr, 0.0, nullptr, nullptr,
                                  c.d.e, s);
        return cells;
    }
    case 6: {
        Level &v0 = mg.lv[0];
        note_launch();
        launch_pdl(k_resnorm, mg.red_blocks, kRedT, 0, s, v0.nx, v0.ny, 1.0 / (v0.h * v0.h), v0.d.bx,
                   v0.d.by, (const double *)v0.d.r, (const double *)v0.d.e, v0.f.r, v0.f.e,
                   mg.red + 8, mg.red_count, mg.red, (SolveCtl *)nullptr,
                   (cudaGraphConditionalHandle)0, 0, 0);
        return (long)v0.nx * v0.ny;
    }
    default: return -1;
    }
}

void ensure_fp64_w(MG &mg, cudaStream_t s)
{
    if (mg.fp64_w) return;
    LevelWArgs a;
    a.nl = mg.L;
    a.start[0] = 0;
    for (int l = 0; l < mg.L; l++) {
        Level &v = mg.lv[l];
        a.nx[l] = v.nx;
        a.bx[l] = v.d.bx; a.by[l] = v.d.by; a.invd[l] = v.d.invd; a.w4[l] = v.d.w;
        a.start[l + 1] = a.start[l] + (long)v.nx * v.ny;
    }
    note_launch();
    k_level_w<<<(unsigned)cdiv(a.start[mg.L], 256), 256, 0, s>>>(a);
    mg.fp64_w = true;
}

void mg_build(MG &mg, const double *bx, const double *by, cudaStream_t s, bool with_w)
{
    const int L = mg.L;
    mg.fp64_w = with_w;
    // levels above 1024 cells one launch each (their FP64 work spread over
    // the SMs), the rest in one CTA
    int lsmall = 1;
    while (lsmall < L && (long)mg.lv[lsmall].nx * mg.lv[lsmall].ny > 1024) lsmall++;
    for (int l = 0; l < lsmall; l++) {
        Level &v = mg.lv[l];
        const double *fbx = l == 0 ? bx : mg.lv[l - 1].d.bx, *fby = l == 0 ? by : mg.lv[l - 1].d.by;
        dim3 g(cdiv(v.nx, 128), v.ny);
        note_launch();
        k_level_coeffs<<<g, 128, 0, s>>>(v.nx, v.ny, l == 0, fbx, fby, v.d.bx, v.d.by, v.f.bx, v.f.by,
                                         v.f.bxp, v.d.invd, v.f.invd, with_w ? v.d.w : nullptr);
    }
    if (lsmall < L) {
        LevelCoeffArgs a;
        a.first = lsmall;
        a.nl = L;
        for (int l = 0; l < L; l++) {
            Level &v = mg.lv[l];
            a.nx[l] = v.nx; a.ny[l] = v.ny;
            a.bx[l] = v.d.bx; a.by[l] = v.d.by; a.invd[l] = v.d.invd; a.w4[l] = with_w ? v.d.w : nullptr;
            a.bxf[l] = v.f.bx; a.byf[l] = v.f.by; a.bxp[l] = v.f.bxp; a.invdf[l] = v.f.invd;
        }
        note_launch();
        k_level_coeffs_small<<<1, 1024, 0, s>>>(a);
    }
    {
        // shared memory of the single-CTA tail (set here, outside any capture)
        size_t e = 0;
        size_t ef = 0;
        for (int l = mg.tail; l < L; l++) e += tail_level_elems(mg.lv[l].nx, mg.lv[l].ny, l == L - 1);
        for (int l = mg.tail_f; l < L; l++) ef += tail_level_elems(mg.lv[l].nx, mg.lv[l].ny, l == L - 1);
        const size_t inv = tail_inv_bytes(mg.lv[L - 1].nx * mg.lv[L - 1].ny);
        raise_smem_limit((const void *)k_tail<double>, (int)(((e * 8 + 7) & ~(size_t)7) + inv));
        raise_smem_limit((const void *)k_tail<float>, (int)(((ef * 4 + 7) & ~(size_t)7) + inv));
    }
    Level &vc = mg.lv[L - 1];
    note_launch();
    const size_t nc2 = (size_t)vc.nx * vc.ny * vc.nx * vc.ny;
    const size_t cbytes = nc2 * sizeof(double);
    const int in_smem = cbytes <= 96 * 1024;
    if (in_smem) raise_smem_limit((const void *)k_coarse_inv, (int)cbytes);
    k_coarse_inv<<<1, 1024, in_smem ? cbytes : 0, s>>>(vc.nx, vc.ny, vc.h, vc.d.bx, vc.d.by, mg.lu,
                                                       mg.lu + nc2, in_smem);
}

// Host-driven solve: one launch per kernel and a host read of the residual
// after every cycle.  Used when per-kernel event timing is active (events
// cannot time kernels inside a graph) and as the reference for the graph
// solve below.
ib_status mg_run_direct(MG &mg, const double *rhs, double *p, int precision, double tol,
                        int max_cycles, int nu1, int nu2, int *cycles, double *relres,
                        cudaStream_t s, std::string &err)
{
    if (precision == 0) ensure_fp64_w(mg, s);
    Level &v0 = mg.lv[0];
    const long n = (long)v0.nx * v0.ny;
    const int RB = mg.red_blocks;
    double *part = mg.red + 8;
    double *res = mg.red;  // res[0] sum b, res[1] |b0|^2, res[2] |r|^2, res[3] sum p
    double *e0 = v0.d.e, *b0 = v0.d.r;
    const double ih2 = 1.0 / (v0.h * v0.h);
    cudaMemsetAsync(&mg.ctl->fault, 0, sizeof(int), s);  // fault word of this solve
    cudaMemcpyAsync(e0, p, n * 8, cudaMemcpyDeviceToDevice, s);
    note_launch();
    k_sum<<<RB, kRedT, 0, s>>>(n, rhs, part, mg.red_count, res + 0);
    note_launch();
    k_sub_mean<<<RB, kRedT, 0, s>>>(n, rhs, res + 0, b0, v0.h * v0.h, v0.d.invd,
                                    precision ? nullptr : v0.d.bt, part, mg.red_count, res + 1);
    auto resnorm = [&]() {
        const bool pr = prof_on(kProfResnorm);
        if (pr) prof_mark(s, true);
        note_launch();
        k_resnorm<<<RB, kRedT, 0, s>>>(v0.nx, v0.ny, ih2, v0.d.bx, v0.d.by, b0, e0,
                                       precision ? v0.f.r : nullptr,
                                       precision ? v0.f.e : nullptr, part, mg.red_count,
                                       res, nullptr, (cudaGraphConditionalHandle)0, 0, 0);
        if (pr) prof_mark(s, false);
        cudaMemcpyAsync(mg.red_host, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
        return cudaStreamSynchronize(s);
    };
    cudaError_t ce = resnorm();
    if (ce != cudaSuccess) { err = cudaGetErrorString(ce); return IB_ECUDA; }
    double nb = sqrt(mg.red_host[1]);
    int c = 0;
    double rr = 0.0;
    ib_status st = IB_OK;
    if (nb == 0.0) {
        cudaMemsetAsync(p, 0, n * 8, s);
        ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) { err = cudaGetErrorString(ce); return IB_ECUDA; }
    } else {
        rr = sqrt(mg.red_host[2]) / nb;
        while (rr > tol && c < max_cycles && isfinite(rr)) {
            if (precision == 0) {
                vcycle<double>(mg, nu1, nu2, s);
            } else {
                const int inner = precision == 2 ? 2 : 1;
                bool added = false;
                for (int q = 0; q < inner; q++)
                    added = vcycle<float>(mg, nu1, nu2, s, q == inner - 1 ? e0 : nullptr);
                if (!added) {
                    note_launch();
                    k_add_f32<<<cdiv(n, 256), 256, 0, s>>>(n, v0.f.e, e0);
                }
                c += inner - 1;
            }
            c++;
            ce = resnorm();
            if (ce != cudaSuccess) { err = cudaGetErrorString(ce); return IB_ECUDA; }
            rr = sqrt(mg.red_host[2]) / nb;
        }
        note_launch();
        k_sum<<<RB, kRedT, 0, s>>>(n, e0, part, mg.red_count, res + 3);
        note_launch();
        k_apply_mean<<<cdiv(n, 256), 256, 0, s>>>(n, e0, res + 3, p);
        int fault = 0;  // pageable landing (the no-allocation solve has no pinned control block)
        ce = cudaMemcpyAsync(&fault, &mg.ctl->fault, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) { err = cudaGetErrorString(ce); return IB_ECUDA; }
        if (fault) { err = fault_message(fault); return IB_ECUDA; }
        if (!isfinite(rr)) { st = IB_ENAN; err = "non-finite residual"; }
        else if (rr > tol) { st = IB_ENOTCONV; err = "cycle cap reached above tolerance"; }
    }
    if (cycles) *cycles = c;
    if (relres) *relres = rr;
    return st;
}

// The same solve as one CUDA graph: prologue (copy-in, mean removal, initial
// residual, convergence test), a device-side WHILE node whose body is one
// cycle + FP64 residual + convergence test, and an epilogue (mean removal,
// control block to the host).  One graph launch and one host synchronisation
// per solve; the loop is bounded by max_cycles on the device.
static cudaError_t build_solve_graph(MG &mg, SolveGraph &sg)
{
    Level &v0 = mg.lv[0];
    const long n = (long)v0.nx * v0.ny;
    const int RB = mg.red_blocks;
    double *part = mg.red + 8, *res = mg.red;
    double *e0 = v0.d.e, *b0 = v0.d.r;
    const double ih2 = 1.0 / (v0.h * v0.h);
    cudaStream_t c = mg.cap, cb = mg.cap_body;
    const unsigned long long k0 = launch_count();
    cudaError_t e = cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(&mg.ctl->fault, 0, sizeof(int), c);  // fault word of this solve
    if (sg.p != e0) cudaMemcpyAsync(e0, sg.p, n * 8, cudaMemcpyDeviceToDevice, c);
    note_launch();
    k_sum<<<RB, kRedT, 0, c>>>(n, sg.rhs, part, mg.red_count, res + 0);
    note_launch();
    k_sub_mean<<<RB, kRedT, 0, c>>>(n, sg.rhs, res + 0, b0, v0.h * v0.h, v0.d.invd,
                                    sg.precision ? nullptr : v0.d.bt, part, mg.red_count, res + 1);
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t *deps;
    const cudaGraphEdgeData *ed;
    size_t nd;
    cudaGraphConditionalHandle hnd = 0;
    unsigned long long kb0 = 0, kb1 = 0;
    // residual norm + convergence test (check 1: before the loop, 2: in its body)
    auto resnorm = [&](cudaStream_t st, int check) {
        note_launch();
        launch_pdl(k_resnorm, RB, kRedT, 0, st, v0.nx, v0.ny, ih2, v0.d.bx, v0.d.by, b0, e0,
                   sg.precision ? v0.f.r : nullptr, sg.precision ? v0.f.e : nullptr, part,
                   mg.red_count, res, mg.ctl, hnd, check, sg.precision == 2 ? 2 : 1);
    };
    e = cudaStreamGetCaptureInfo(c, &cs, nullptr, &g, &deps, &ed, &nd);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hnd, g, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        resnorm(c, 1);
        e = cudaStreamGetCaptureInfo(c, &cs, nullptr, &g, &deps, &ed, &nd);
    }
    cudaGraphNode_t wnode;
    cudaGraphNodeParams cp = {};
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = hnd;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, g, deps, ed, nd, &cp);
    }
    if (e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(c, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        kb0 = launch_count();
        e = cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            if (sg.precision == 0) {
                vcycle<double>(mg, sg.nu1, sg.nu2, cb);
            } else {
                const int inner = sg.precision == 2 ? 2 : 1;
                bool added = false;
                for (int q = 0; q < inner; q++)
                    added = vcycle<float>(mg, sg.nu1, sg.nu2, cb, q == inner - 1 ? e0 : nullptr);
                if (!added) {
                    note_launch();
                    launch_pdl(k_add_f32, cdiv(n, 256), 256, 0, cb, n, v0.f.e, e0);
                }
            }
            resnorm(cb, 2);
            e = cudaStreamEndCapture(cb, &body);
        }
        kb1 = launch_count();
    }
    if (e == cudaSuccess) {
        note_launch();
        k_sum<<<RB, kRedT, 0, c>>>(n, e0, part, mg.red_count, res + 3);
        note_launch();
        k_finalize<<<cdiv(n, 256), 256, 0, c>>>(n, e0, res + 3, mg.ctl, sg.p);
        cudaMemcpyAsync(mg.ctl_host, mg.ctl, sizeof(SolveCtl), cudaMemcpyDeviceToHost, c);
    }
    cudaGraph_t full = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c, &full);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&sg.exec, full, 0);
    if (full) cudaGraphDestroy(full);
    const unsigned long long kall = launch_count() - k0;
    sg.body_kernels = kb1 - kb0;
    sg.outer_kernels = kall - sg.body_kernels;
    note_launch(-(int)kall);  // capture issues no kernel; executions are counted per launch
    cudaGetLastError();
    return e;
}

static bool prof_active();

ib_status mg_run_launch(MG &mg, const double *rhs, double *p, int precision, double tol,
                        int max_cycles, int nu1, int nu2, int *cycles, double *relres,
                        cudaStream_t s, std::string &err, MgPending &pend)
{
    pend.pending = false;
    if (!mg.use_graphs || prof_active())
        return mg_run_direct(mg, rhs, p, precision, tol, max_cycles, nu1, nu2, cycles, relres, s, err);
    if (precision == 0) ensure_fp64_w(mg, s);  // before the graph, which reads them
    SolveGraph *sg = nullptr;
    for (auto &g : mg.graphs)
        if (g.rhs == rhs && g.p == p && g.precision == precision && g.nu1 == nu1 && g.nu2 == nu2)
            sg = &g;
    if (!sg) {
        if (mg.graphs.size() >= 8) {
            cudaGraphExecDestroy(mg.graphs.front().exec);
            mg.graphs.erase(mg.graphs.begin());
        }
        SolveGraph ng;
        ng.rhs = rhs; ng.p = p; ng.precision = precision; ng.nu1 = nu1; ng.nu2 = nu2;
        cudaError_t e = build_solve_graph(mg, ng);
        if (e != cudaSuccess) {
            if (ng.exec) cudaGraphExecDestroy(ng.exec);
            // graphs unavailable: keep solving with direct launches
            mg.use_graphs = false;
            return mg_run_direct(mg, rhs, p, precision, tol, max_cycles, nu1, nu2, cycles, relres, s, err);
        }
        mg.graphs.push_back(ng);
        sg = &mg.graphs.back();
    }
    mg.ctl_host->tol = tol;
    mg.ctl_host->max_cycles = max_cycles;
    cudaError_t e = cudaMemcpyAsync(mg.ctl, mg.ctl_host, 2 * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(sg->exec, s);
    if (e != cudaSuccess) { err = cudaGetErrorString(e); return IB_ECUDA; }
    pend.pending = true;
    pend.tol = tol;
    pend.outer_kernels = sg->outer_kernels;
    pend.body_kernels = sg->body_kernels;
    return IB_OK;
}

ib_status mg_run_finish(MG &mg, const MgPending &pend, int *cycles, double *relres, std::string &err)
{
    if (mg.ctl_host->fault) { err = fault_message(mg.ctl_host->fault); return IB_ECUDA; }
    const int c = mg.ctl_host->cycles;
    const double rr = mg.ctl_host->rr;
    note_launch((int)(pend.outer_kernels + (unsigned long long)c * pend.body_kernels));
    if (cycles) *cycles = c;
    if (relres) *relres = rr;
    if (mg.ctl_host->zero_p) return IB_OK;
    if (!isfinite(rr)) { err = "non-finite residual"; return IB_ENAN; }
    if (rr > pend.tol) { err = "cycle cap reached above tolerance"; return IB_ENOTCONV; }
    return IB_OK;
}

ib_status mg_run(MG &mg, const double *rhs, double *p, int precision, double tol,
                 int max_cycles, int nu1, int nu2, int *cycles, double *relres,
                 cudaStream_t s, std::string &err)
{
    MgPending pend;
    const ib_status st = mg_run_launch(mg, rhs, p, precision, tol, max_cycles, nu1, nu2, cycles,
                                       relres, s, err, pend);
    if (!pend.pending) return st;
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { err = cudaGetErrorString(e); return IB_ECUDA; }
    return mg_run_finish(mg, pend, cycles, relres, err);
}

// Context-free launches used by the verification entry points.
void launch_rbgs(int nx, int ny, double h, const double *bx, const double *by,
                 const double *invd, const double *b, const double *pin, double *p,
                 cudaStream_t s)
{
    dim3 g(cdiv(nx, TW), cdiv(ny, TH));
    note_launch();
    k_rbgs_sweep<double><<<g, TT, 0, s>>>(nx, ny, h * h, bx, by, invd, b, pin, p);
}

void launch_invdiag(int nx, int ny, const double *bx, const double *by,
                    double *invd, cudaStream_t s)
{
    dim3 g(cdiv(nx, 128), ny);
    note_launch();
    k_invdiag<double><<<g, 128, 0, s>>>(nx, ny, bx, by, invd);
}

void launch_restrict_residual(int nx, int ny, double h, const double *bx,
                              const double *by, const double *b, const double *p,
                              double *rc, double *ec, cudaStream_t s)
{
    dim3 gr(cdiv(nx / 2, 128), ny / 2);
    note_launch();
    k_restrict_residual<double><<<gr, 128, 0, s>>>(nx, ny, 1.0 / (h * h), bx, by, b, p, rc, ec, 0.0,
                                                   nullptr, nullptr);
}

void launch_prolong_add(int nxc, int nyc, const double *ec, double *ef, cudaStream_t s)
{
    dim3 gp(cdiv(2 * nxc, 128), 2 * nyc);
    note_launch();
    k_prolong_add<double><<<gp, 128, 0, s>>>(nxc, nyc, ec, ef);
}

void launch_coarsen_beta(int nx, int ny, const double *bx, const double *by,
                         double *bxc, double *byc, cudaStream_t s)
{
    long nfc = (long)(nx / 2 + 1) * (ny / 2) + (long)(nx / 2) * (ny / 2 + 1);
    note_launch();
    k_coarsen_beta<<<cdiv(nfc, 256), 256, 0, s>>>(nx, ny, bx, by, bxc, byc);
}

void launch_residual(int nx, int ny, double h, const double *bx, const double *by,
                     const double *b, const double *p, double *r, cudaStream_t s)
{
    dim3 g(cdiv(nx, 128), ny);
    note_launch();
    k_residual<double><<<g, 128, 0, s>>>(nx, ny, 1.0 / (h * h), bx, by, b, p, r);
}

}  // namespace ibk
