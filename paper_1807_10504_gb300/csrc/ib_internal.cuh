// Internal declarations shared by the CUDA translation units of the library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ib.h"

namespace ibk {

constexpr int kTailCells = 1024;     // levels with at most this many cells run in one CTA (FP64)
constexpr int kTailCellsF32 = 4096;  // the same for the FP32 cycle (its levels fit shared memory)
constexpr int kMaxCoarsest = 1024;   // dense LU limit of the coarsest level
constexpr int kBlk = 8;              // marker-activity block edge (cells)
constexpr int kSearch = 7;           // marker search radius (cells) around a cell or face
constexpr int kMaxCand = 1024;       // candidate segments per activity block
constexpr int kSegLine = 56;        // doubles per segment of the FP64 strip-line record
constexpr int kMaxCross = 2048;      // interface crossings per grid row

inline unsigned cdiv(long a, long b) { return (unsigned)((a + b - 1) / b); }

// Conversions between double and float on integer instructions, for values
// in the FP32 normal range: this part runs FP64 conversions on its reduced
// FP64 pipe, at the rate of its FP64 arithmetic.  d2f_trunc keeps the top 23
// mantissa bits (truncation, relative error below 2^-23); f2d_exact is exact.
__device__ __forceinline__ float d2f_trunc(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned e = ((hi >> 20) & 0x7ffu) - 896u;  // FP64 bias 1023 -> FP32 bias 127
    return __uint_as_float((hi & 0x80000000u) | (e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
__device__ __forceinline__ double f2d_exact(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = ((u >> 23) & 0xffu) + 896u, m = u & 0x7fffffu;
    const unsigned hi = (u & 0x80000000u) | (e << 20) | (m >> 3);
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | ((unsigned long long)(m & 7u) << 29)));
}

// (float)x, round to nearest even, on integer instructions where x is zero
// or within the FP32 normal range (the hardware conversion elsewhere: FP32
// subnormals, overflow, infinities, NaN); the result is the conversion's.
__device__ __forceinline__ float d2f_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e >= 897u && e <= 1150u) {
        unsigned r = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu;  // the 29 dropped bits
        r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
        return __uint_as_float((hi & 0x80000000u) | r);
    }
    if ((b & 0x7fffffffffffffffULL) == 0) return __uint_as_float(hi & 0x80000000u);
    return (float)x;
}
// (double)f, exact, on integer instructions for zero and FP32 normals (the
// hardware conversion for subnormals, infinities and NaN).
__device__ __forceinline__ double f2d(float f)
{
    const unsigned u = __float_as_uint(f), e = (u >> 23) & 0xffu;
    if (e - 1u < 254u) return f2d_exact(f);
    if ((u & 0x7fffffffu) == 0) return __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32));
    return (double)f;
}

// 1/sqrt(x) for x in the FP32 normal range: the FP32 estimate (rsqrtf) of
// x's leading bits refined by two Newton steps y <- y (3/2 - x y^2 / 2) in
// FP64 (relative error 2^-22 -> 2^-43 -> below FP64 rounding); a short chain
// of dependent operations, for serial code where FP64 latency counts.
__device__ __forceinline__ double rsqrt_nr(double x)
{
    double y = f2d_exact(rsqrtf(d2f_trunc(x)));
    const double hx = -0.5 * x;
    y = y * fma(hx, y * y, 1.5);
    return y * fma(hx, y * y, 1.5);
}

// 1/x for x of either sign within the FP32 normal range (about 1e-37 < |x|
// < 1e37): the FP32 reciprocal (__frcp_rn) of x's leading bits refined by two
// Newton-Raphson steps r <- r + r (1 - x r) in FP64; each step squares the
// relative error (2^-22 -> 2^-44 -> below the FP64 rounding), so the result
// is within one unit in the last place of 1.0 / x at a fraction of the FP64
// division's cost on this part, with no FP64 conversion.
__device__ __forceinline__ double recip_nr(double x)
{
    double r = f2d_exact(__frcp_rn(d2f_trunc(x)));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// 1/x for any nonzero finite x of either sign (0 for x = 0): recip_nr where
// |x| lies well inside the FP32 normal range, the FP64 division elsewhere.
__device__ __forceinline__ double recip_any(double x)
{
    // the tests on |x|'s bit pattern (ordered like the value), in integer
    // instructions
    const unsigned long long a = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    if (a == 0) return 0.0;
    const unsigned long long lo = (unsigned long long)__double_as_longlong(1e-30),
                             hi = (unsigned long long)__double_as_longlong(1e30);
    return (a > lo && a < hi) ? recip_nr(x) : 1.0 / x;
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes` (one
// host call the first time a larger value is needed, none afterwards, so
// that launches recorded into a CUDA graph make no such call).
void raise_smem_limit(const void *kernel, int bytes);

// Process-wide count of kernel launches issued by this library.
// True while per-kernel event timing is active (no graph replays then).
bool profiling_active();
void note_launch(int n = 1);
unsigned long long launch_count();

// The message of a smoother fault word (1 staging time-out, 2 misaligned
// tiles, 3 copies not landed), and the staging-stall test hook.
const char *fault_message(int code);
cudaError_t set_stall_staging(int on);

// Optional CUDA-event timing of one kernel class, on the stream it runs on.
// Per-launch kinds (0-3) time single kernels (one launch per kernel: no
// graph replay meanwhile); phase kinds (4-6) time the parts of ns_step on the
// context stream around their graphs.
enum ProfKind {
    kProfSweep64 = 0, kProfSweep32 = 1, kProfResnorm = 2, kProfProlong32 = 3,
    kProfPre = 4, kProfSolve = 5, kProfPost = 6
};
bool prof_on(int kind);
void prof_mark(cudaStream_t s, bool start);
bool prof_begin(int kind);
bool prof_end(double *total_ms, int *launches);

// ---------------------------------------------------------------- grid ops
void launch_coeffs(int nx, int ny, double rho_g, double rho_l, double mu_g,
                   double mu_l, const double *H, double *rho, double *mu,
                   double *bx, double *by, cudaStream_t s);
void launch_rhs(int nx, int ny, double h, double dt, const double *us,
                const double *vs, const double *Fx, const double *Fy,
                const double *bx, const double *by, double *b, cudaStream_t s);
void launch_correct(int nx, int ny, double h, double dt, const double *us,
                    const double *vs, const double *p, const double *Fx,
                    const double *Fy, const double *bx, const double *by,
                    double *u, double *v, cudaStream_t s);
// bx, by: the face coefficients 1 / rho_face of the same rho (k_face_beta),
// or NULL to form the reciprocals in the kernel
void launch_predictor(int nx, int ny, double h, double dt, const double *rho,
                      const double *mu, const double *u, const double *v,
                      const double *au_prev, const double *av_prev,
                      int have_prev, double gx, double gy, const double *bx,
                      const double *by, double *us, double *vs, double *au, double *av,
                      cudaStream_t s);

// Crank-Nicolson viscous solve: nsweeps red-black sweeps of
// u* - dt / (2 rho_f) D(u*) = u_e on both components; (us, vs) hold the
// starting iterate (u_e itself) and receive u*.
void launch_cn_solve(int nx, int ny, double h, double dt, const double *rho, const double *mu,
                     int axisym, const double *frame, int nsweeps, const double *ue,
                     const double *ve, double *us, double *vs, cudaStream_t s);
void launch_scale(long n, double a, const double *x, double *y, cudaStream_t s);
void launch_fill(long n, double a, double *y, cudaStream_t s);
void launch_extrapolate(long n, double *p, double *q, cudaStream_t s);
// Indicator function (Section 2.2 Eq. (ind_psn)): right-hand side div G, the
// unit (or r-weighted) coefficients, and the shift to zero along the walls
// with clipping to [0, 1].
void launch_div_faces(int nx, int ny, double h, int axisym, const double *Gx, const double *Gy,
                      double *b, cudaStream_t s);
void launch_unit_beta(int nx, int ny, double h, int axisym, double *bx, double *by, cudaStream_t s);
void launch_indicator_finish(int nx, int ny, int axisym, const double *sol, double *ref, double *I,
                             cudaStream_t s);

// ------------------------------------------------------------ axisymmetric
// Record of the non-inertial frame (device doubles): reference, previous and
// current centre of mass of drop 0, the next step's acceleration S, the frame
// velocity Vf and the boundary velocity wb = -Vf.
enum FrameSlot { kFrCom0 = 0, kFrComPrev = 1, kFrCom = 2, kFrS = 3, kFrVf = 4, kFrWb = 5, kFrSlots = 8 };
void launch_predictor_axi(int nx, int ny, double h, double dt, const double *rho,
                          const double *mu, const double *u, const double *v,
                          const double *au_prev, const double *av_prev, int have_prev,
                          double gx, double gy, const double *frame, const double *bx,
                          const double *by, double *us, double *vs, double *au, double *av,
                          cudaStream_t s);
void launch_axi_zbc(int nx, int ny, const double *frame, double *v, cudaStream_t s);
void launch_rhs_axi(int nx, int ny, double h, double dt, const double *us, const double *vs,
                    const double *Fx, const double *Fy, const double *bx, const double *by,
                    double *b, cudaStream_t s);
void launch_axi_weights(int nx, int ny, double h, const double *bx, const double *by,
                        double *bxa, double *bya, cudaStream_t s);
void launch_axi_extend(int nx, int ny, int G, const double *u, const double *v, double *uw,
                       double *vw, cudaStream_t s);
void launch_axi_fold(int nx, int ny, int G, double h, int ring, const double *Hw, const double *Fxw,
                     const double *Fyw, double *H, double *Fx, double *Fy, cudaStream_t s);

// ---------------------------------------------------------------- multigrid
template <typename T>
struct LevelT {
    T *e = nullptr, *r = nullptr, *bx = nullptr, *by = nullptr, *invd = nullptr;
    T *e2 = nullptr;  // second iterate buffer: sweeps read one and write the other
    // FP64 levels only: the pre-scaled stencil of the sweep, 4 weights per
    // cell (W, E, S, N) = beta_f / diag, and the right-hand side h^2 b / diag
    T *w = nullptr, *bt = nullptr;
    // FP32 levels only: the x-face coefficients again, rows at a pitch of
    // (nx + 1) rounded up to 4 values (zero padded), for tensor copies, whose
    // row strides are multiples of 16 bytes
    T *bxp = nullptr;
};

// Tensor maps (TMA descriptors) of one fused FP32 smoother launch: windows of
// the iterate read, the right-hand side, 1/diag, beta_y and beta_x (padded
// rows), and the word that a timed-out staging wait sets.
struct TileMaps {
    CUtensorMap p, b, d, y, x;
    int *fault;
};

// A level's FP32 smoother maps for one window shape (both iterate buffers).
struct LevelTma {
    CUtensorMap e, e2, r, invd, by, bxp;
};

struct Level {
    int nx = 0, ny = 0;
    double h = 0;
    LevelT<double> d;
    LevelT<float> f;
    bool tma = false;  // tm[] valid: the FP32 smoother stages by TMA on this level
    LevelTma tm[2];    // [0] 72 x 24 windows (halo 4), [1] 80 x 26 windows (halo 5)
    int *fault = nullptr;
};

struct SolveCtl {
    double tol;
    int max_cycles;
    int cycles;
    double rr;
    int zero_p;
    int fault;  // set by a kernel whose bounded wait timed out
};

struct SolveGraph {
    const double *rhs = nullptr;
    double *p = nullptr;
    int precision = 0, nu1 = 0, nu2 = 0;
    cudaGraphExec_t exec = nullptr;
    unsigned long long outer_kernels = 0, body_kernels = 0;
};

struct MG {
    Level lv[16];
    int L = 0;                    // number of levels in lv
    std::vector<SolveGraph> graphs;  // instantiated solves, keyed by pointers and settings
    cudaStream_t cap = nullptr, cap_body = nullptr;
    SolveCtl *ctl = nullptr, *ctl_host = nullptr;
    bool use_graphs = true;
    int tail = 0;                 // first level handled by the single-CTA tail kernel (FP64)
    int tail_f = 0;               // the same for the FP32 cycle
    double *lu = nullptr;         // coarsest dense LU (n x n), FP64
    int *piv = nullptr;           // coarsest row permutation
    double *red = nullptr;        // reduction partials + results (device)
    unsigned *red_count = nullptr;
    double *red_host = nullptr;   // pinned mirror of the results
    int red_blocks = 0;
    // the FP64 sweep weights (LevelT<double>::w) match the coefficients: the
    // build leaves them out (only FP64 cycles read them), ensure_fp64_w forms
    // them before one
    bool fp64_w = false;
    void *mem = nullptr;          // one allocation for all of the above
    size_t bytes = 0;
};

bool mg_levels(int nx, int ny, std::vector<int> &nxs, std::vector<int> &nys);
// Places the hierarchy (levels, coarsest LU, reduction partials, control
// block) at `base` (or only measures it when base is NULL); returns its bytes.
// Allocates nothing.
size_t mg_layout(MG &mg, int nx, int ny, double h, char *base);
cudaError_t mg_alloc(MG &mg, int nx, int ny, double h);
void mg_free(MG &mg);
// One launch of one cycle kernel on the hierarchy's current data, for timing.
long mg_bench_op(MG &mg, int op, int level, cudaStream_t s);
// Copy level-0 coefficients (walls forced to 0) and build the hierarchy; the
// FP64 sweep weights too with with_w (for a solver that runs FP64 cycles).
void mg_build(MG &mg, const double *bx, const double *by, cudaStream_t s, bool with_w = false);
// The FP64 sweep weights of every level, if the last build left them out.
void ensure_fp64_w(MG &mg, cudaStream_t s);
// Runs the solve on level-0 arrays of the hierarchy; p is read/written in place.
ib_status mg_run(MG &mg, const double *rhs, double *p, int precision, double tol,
                 int max_cycles, int nu1, int nu2, int *cycles, double *relres,
                 cudaStream_t s, std::string &err);
// The same in two parts, so that work queued after the solve need not wait
// for the host: mg_run_launch queues the solve graph and returns with
// pend.pending set (or, where it solves with direct launches, finishes and
// returns the status with pend.pending clear); once the stream has been
// synchronised, mg_run_finish reads the solve's status.
struct MgPending {
    bool pending = false;
    double tol = 0;
    unsigned long long outer_kernels = 0, body_kernels = 0;
};
ib_status mg_run_launch(MG &mg, const double *rhs, double *p, int precision, double tol,
                        int max_cycles, int nu1, int nu2, int *cycles, double *relres,
                        cudaStream_t s, std::string &err, MgPending &pend);
ib_status mg_run_finish(MG &mg, const MgPending &pend, int *cycles, double *relres, std::string &err);

// The same solve with one launch per kernel and a host read of the residual
// after each cycle (no graph objects, no allocation of its own).
ib_status mg_run_direct(MG &mg, const double *rhs, double *p, int precision, double tol,
                        int max_cycles, int nu1, int nu2, int *cycles, double *relres,
                        cudaStream_t s, std::string &err);

void launch_rbgs(int nx, int ny, double h, const double *bx, const double *by,
                 const double *invd, const double *b, const double *pin, double *p,
                 cudaStream_t s);
void launch_invdiag(int nx, int ny, const double *bx, const double *by,
                    double *invd, cudaStream_t s);
void launch_restrict_residual(int nx, int ny, double h, const double *bx,
                              const double *by, const double *b, const double *p,
                              double *rc, double *ec, cudaStream_t s);
void launch_prolong_add(int nxc, int nyc, const double *ec, double *ef,
                        cudaStream_t s);
void launch_coarsen_beta(int nx, int ny, const double *bx, const double *by,
                         double *bxc, double *byc, cudaStream_t s);
void launch_residual(int nx, int ny, double h, const double *bx,
                     const double *by, const double *b, const double *p,
                     double *r, cudaStream_t s);

// ---------------------------------------------------------------- markers
struct Markers {
    int M = 0, ndrops = 0, nx = 0, ny = 0, bnx = 0, bny = 0;
    double h = 0, x0 = 0, y0 = 0;
    double *X = nullptr, *Y = nullptr, *kappa = nullptr, *nxm = nullptr,
           *nym = nullptr, *ds = nullptr, *fmag = nullptr, *U = nullptr,
           *V = nullptr, *Xn = nullptr, *Yn = nullptr;
    double *gx = nullptr, *gy = nullptr;   // marker positions in grid units
    float *gxf = nullptr, *gyf = nullptr;  // the same rounded to FP32 (screening only)
    float4 *sbox = nullptr;                // slab box of segment (m, next m), grid units
    double2 *dyr = nullptr;                // per-drop [min Y, max Y]
    unsigned long long *ykey = nullptr;    // order-preserving integer key of each Y
    ulonglong2 *dyk = nullptr;             // keys of the per-drop Y range
    unsigned long long *colkey = nullptr;  // order-preserving key of each column's centre x
    double *sv = nullptr;                  // per segment: 12 strip corner points (24 doubles)
    double *sl = nullptr;                  // per segment: 8 half-planes (a, b, c, 1/a, 1/b) + determinant reciprocals, FP64
    float4 *slf = nullptr;                 // the same in FP32 (nx, ny, c, |n|)
    uint8_t *scvx = nullptr;               // per segment: 1 = half-plane path (strips convex, lines well conditioned)
    double *sinv = nullptr;                // per segment: 1 / |segment|^2 in grid units
    double *rfit = nullptr;                // relocation: per-drop control points and knot arc lengths
    double *rpar = nullptr;                // relocation: per drop (g, tau, arc length, failed)
    double *rwts = nullptr;                // relocation: per marker, its four basis weights
    uint32_t pair_cap = 0;                 // capacity of the band (cell, segment) pair list
    uint32_t *npairs = nullptr;            // pairs claimed by the last band pass
    uint32_t *pseg = nullptr, *pcell = nullptr;  // pair list: segment (top bit: listed for clipping), cell index
    uint32_t *clip_list = nullptr;         // pairs of non-convex strips (the second word of npairs counts them)
    double *pacc = nullptr, *pcov = nullptr;     // per pair: sum A_k H_k, sum A_k
    uint2 *crange = nullptr;               // per cell of an active block: (first pair, count)
    float4 *sb5 = nullptr;                 // per segment: FP32 outward box of each of 5 strips
    int32_t *drop_start = nullptr, *drop_of = nullptr, *next = nullptr;
    uint32_t *key = nullptr, *tmp_ids = nullptr, *ids = nullptr,
             *cell_count = nullptr, *cell_start = nullptr, *scan_part = nullptr,
             *bcount = nullptr, *bactive = nullptr, *flags = nullptr;
    std::vector<int32_t> drop_start_h;
    int max_drop = 0;
    void *mem = nullptr;
};

cudaError_t markers_alloc(Markers &mk, int M, int ndrops, int nx, int ny,
                          double h, double x0, double y0,
                          const int32_t *drop_start_host);
void markers_free(Markers &mk);
// flags[0]: bad marker (outside / too near a wall); flags[1]: candidate,
// crossing or band pair list overflow; flags[2]: B-spline system not positive definite.
void launch_validate(Markers &mk, cudaStream_t s);
void launch_geometry(Markers &mk, double sigma, cudaStream_t s);
void launch_sort(Markers &mk, cudaStream_t s);
void launch_interp(const Markers &mk, int kernel, const double *u,
                   const double *v, double *U, double *V, double dt_move,
                   cudaStream_t s);
void launch_spread_conv(const Markers &mk, int kernel, const double *fmag,
                        double *Fx, double *Fy, cudaStream_t s);
void launch_heaviside(const Markers &mk, double *H, cudaStream_t s, cudaStream_t side = nullptr,
                      cudaEvent_t ev_fork = nullptr, cudaEvent_t ev_join = nullptr);
void launch_band_area(const Markers &mk, cudaStream_t s);
void launch_spread_irrot(const Markers &mk, const double *fmag, const double *H,
                         double *Fx, double *Fy, cudaStream_t s);
void launch_relocate(Markers &mk, cudaStream_t s);
void launch_drop_measure(const Markers &mk, int axisym, double *A, cudaStream_t s);
void launch_mass_correct(Markers &mk, const double *A0, int axisym, double tol, double *eps,
                         cudaStream_t s);
void launch_axi_curvature(Markers &mk, double sigma, cudaStream_t s);
void launch_axi_ring(const Markers &mk, const double *fmag, double *fr, cudaStream_t s);
void launch_axi_symmetrise(Markers &mk, cudaStream_t s);
void launch_axi_frame(const Markers &mk, double dt, double c1, double c2, int init, double *frame,
                      cudaStream_t s);

// ---------------------------------------------------------------- CNN
struct Cnn;
Cnn *cnn_new(int c1, int c2, unsigned long long seed, cudaStream_t s, cudaError_t *err);
void cnn_free(Cnn *n);
cudaError_t cnn_pack(Cnn &n, cudaStream_t s);
cudaError_t cnn_workspace(Cnn &n, int B, int N);
void cnn_forward(Cnn &n, int B, int N, double h, const double *rhs, const double *rho,
                 const double *p, cudaStream_t s);
void cnn_backward(Cnn &n, int B, int N, cudaStream_t s);
void cnn_adam(Cnn &n, float lr, cudaStream_t s);
void cnn_output(Cnn &n, int B, int N, double h, double *p0, cudaStream_t s);
cudaError_t cnn_infer_levels(Cnn &n, int B, int N, double h, const double *rhs, const double *rho,
                             double *p0, int levels, cudaStream_t s);
void cnn_set_scale(Cnn &n, double c);
void cnn_set_tc(Cnn &n, int on);
cudaError_t cnn_take_fault(int *f);
cudaError_t cnn_fit_scale(Cnn &n, int B, int N, double h, const double *rhs, const double *p,
                          double *c, cudaStream_t s);
cudaError_t cnn_train_loop(Cnn &n, int ns, int N, double h, const double *rhs, const double *rho,
                           const double *p, int steps, int batch, float lr0, unsigned long long seed,
                           float *losses_host, cudaStream_t s);
double cnn_get_scale(const Cnn &n);
const void *cnn_workspace_ptr(const Cnn &n);  // current activation workspace (moves when it grows)
const void *cnn_cbuf_ptr(const Cnn &n);       // current coarse-grid buffer
size_t cnn_nparam(const Cnn &n);
float *cnn_weights(Cnn &n);
float *cnn_grads(Cnn &n);
float *cnn_lsum(Cnn &n);
int cnn_steps(const Cnn &n);
void cnn_reset_adam(Cnn &n);

}  // namespace ibk
