/*
 * ib.h -- C ABI of the GB300 (sm_103a) immersed-boundary projection library:
 * the per-time-step variable-density projection of Ong & Miura's one-fluid
 * immersed-boundary method (arXiv 1807.10504) and the marker kernels it
 * consumes.
 *
 * Layout (all arrays row-major, x fastest, no padding):
 *   cells   (i,j)  i = 0..nx-1, j = 0..ny-1   index j*nx + i
 *   x-faces (i,j)  i = 0..nx,   j = 0..ny-1   index j*(nx+1) + i   (u, Fx, beta_x)
 *   y-faces (i,j)  i = 0..nx-1, j = 0..ny     index j*nx + i       (v, Fy, beta_y)
 *   cell (i,j) has centre (x0 + (i+1/2)h, y0 + (j+1/2)h); cells are square.
 *   Wall faces (i = 0, nx of u; j = 0, ny of v) are no-slip walls: u, v,
 *   beta and F there are zero on output and ignored on input.
 *   Markers: ndrops closed counter-clockwise polylines; drop d owns markers
 *   drop_start[d] .. drop_start[d+1]-1, the last joined to the first.
 *
 * Pointers: "device" arrays are caller-owned CUDA device memory (borrowed for
 * the duration of the call, never freed or retained); "host" arrays are plain
 * host memory.  Every call is ordered on the stream given to ib_init (or
 * passed explicitly); calls that return results to the host synchronise
 * that stream.  No call aborts, traps or prints: each returns an ib_status
 * and, for context calls, ib_last_error() gives a one-line message.
 * Numbers are IEEE binary64 unless stated.
 */
#ifndef IB_H
#define IB_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IB_OK = 0,
    IB_EINVAL = 1,   /* bad argument: sizes, null pointer, unsupported grid */
    IB_ENOMEM = 2,   /* device allocation failed */
    IB_ENOTCONV = 3, /* pressure solve hit max_cycles above tol (result kept) */
    IB_ENAN = 4,     /* non-finite residual */
    IB_EMARKER = 5,  /* marker outside the domain, closer than 3 cells to a
                        wall, or a drop not counter-clockwise */
    IB_ECUDA = 6     /* a CUDA runtime call failed */
} ib_status;

typedef struct ib_config {
    int32_t nx, ny;           /* cells; multigrid halves both while even, down to <= 16 cells */
    double h, x0, y0;         /* cell size and lower-left corner */
    double rho_g, rho_l;      /* ambient (H = 0) and drop (H = 1) density */
    double mu_g, mu_l;        /* ambient and drop dynamic viscosity */
    double sigma;             /* surface tension coefficient */
    double gx, gy;            /* uniform body acceleration */
    int32_t kernel;           /* 0: cosine kernel, Sec. 2.2 Eq. (cherby); 1: Peskin 4-point */
    int32_t spread;           /* 0: conventional, Sec. 3.1 Eq. (delta_vec);
                                 1: irrotational, Sec. 3.2 Eq. (delta_hea_xy) */
    int32_t precision;        /* 0: FP64 multigrid; 1: FP32 V-cycles inside FP64
                                 defect correction (residual, coarsest solve FP64),
                                 one V-cycle per FP64 residual; 2: the same with
                                 two V-cycles per FP64 residual */
    double tol;               /* relative residual ||b - A p||_2 / ||b||_2 */
    int32_t max_cycles;       /* V-cycles per solve (tested before each outer
                                 step: precision 2 may pass it by one) */
    int32_t nu1, nu2;         /* pre/post red-black Gauss-Seidel sweeps */
    int32_t relocate_every;   /* B-spline relocation period in steps, 0 = never */
    int32_t axisym;           /* 1: axisymmetric (r, z), Sec. 2.1 and Sec. 4 Eq. (curv_ax):
                                 x = r with the axis at x0 = 0, y = z; each drop is
                                 its full closed meridian curve (right half and its
                                 mirror image, an even number of markers, marker k
                                 and n - k mirror images, 0 and n/2 on the axis);
                                 gx must be 0.  0: planar */
    int32_t frame;            /* axisymmetric only.  1: non-inertial frame following drop 0,
                                 Sec. 2.4 Eqs. (fictitious), (fic_1), (fic_2): every step
                                 all fluid gets the axial acceleration S = (c1 (COM_o - COM_n)
                                 - c2 (COM_n - COM_(n-1))) / dt^2 (COM: drop 0's
                                 volume-weighted axial centre, COM_o its value at
                                 ib_init), the frame velocity Vf changes by -S dt, and
                                 the ambient fluid enters at z = 0, leaves at z = Lz
                                 and slides along the outer wall with axial velocity
                                 -Vf (a laboratory at rest seen from the frame).
                                 0: fixed walls */
    double c1, c2;            /* the constants of Eq. (fictitious) (the paper: 0.1, 0.1) */
    int32_t mass_every;       /* Sec. 2.5: every mass_every steps (after the first), each
                                 drop whose enclosed area (planar) or volume of revolution
                                 (axisymmetric) differs from its value at ib_init by more
                                 than mass_tol (relative) is offset along its inward
                                 normals by the bisection root that restores it (the
                                 paper: every 20 steps, 1e-6).  0: never */
    double mass_tol;
    int32_t viscous;          /* 0: explicit viscous term; 1: Crank-Nicolson (Sec. 2.1):
                                 the explicit predictor with half the viscosity, then
                                 u* - dt / (2 rho_f) D(u*) = that, per component, by
                                 cn_sweeps red-black Gauss-Seidel sweeps (the system's
                                 off-diagonal / diagonal ratio is at most 2s / (1 + 2s),
                                 s = nu dt / h^2, and a sweep contracts the error by
                                 about its square: 20 sweeps reach ~1e-12 for s <= 0.5;
                                 larger steps need more) */
    int32_t cn_sweeps;
    int32_t indicator;        /* density and viscosity from 0: the polygon Heaviside H;
                                 1: the indicator I of Sec. 2.2 Eq. (ind_psn),
                                 div grad I = div(delta vector), the conventional
                                 spreading of the inward normals times the arc weights
                                 (ring-weighted, r-weighted equation, in axisymmetric
                                 form); Neumann walls, I = 0 on average along the walls
                                 (not the axis), clipped to [0, 1]; solved by the FP64
                                 multigrid to 1e-12 from the previous step's I */
} ib_config;

typedef struct ib_ctx ib_ctx;

/* ---------------------------------------------------------------------- */
/* Context: owns every device buffer it allocates (fields, markers, cell
 * lists, the multigrid hierarchy).  `stream` is a cudaStream_t (0 = legacy
 * default stream).  X, Y, drop_start are HOST arrays of nmarkers and
 * ndrops+1 entries, copied in.  Fields start at zero.
 * Errors: IB_EINVAL (sizes, grid that cannot coarsen to <= 1024 coarsest
 * cells, more than 2^20 markers), IB_EMARKER, IB_ENOMEM, IB_ECUDA; on error
 * *out is NULL and nothing stays allocated.  Levels halve while both sides
 * are even and the level has more than 16 cells; the coarsest level's dense
 * inverse is rebuilt with the coefficients (every time step) at O(n^3) in
 * one CTA, so grid sides with a large odd factor (200 = 8 x 25 ends at
 * 25 x 25: tens of ms a step) are slow; sides of the form 2^k times a small
 * odd number coarsen to a few cells.                                        */
ib_status ib_init(ib_ctx **out, const ib_config *cfg, const double *X,
                  const double *Y, const int32_t *drop_start, int32_t ndrops,
                  void *stream);
void ib_destroy(ib_ctx *ctx);
const char *ib_last_error(const ib_ctx *ctx); /* never NULL */

/* Replace / read the marker positions (nmarkers entries each).  where = 0:
 * host pointers, 1: device pointers.  Set validates the positions
 * (IB_EMARKER) and keeps the drop structure given to ib_init.             */
ib_status ib_set_markers(ib_ctx *ctx, const double *X, const double *Y, int where);
ib_status ib_get_markers(ib_ctx *ctx, double *X, double *Y, int where);
int32_t ib_num_markers(const ib_ctx *ctx);

/* Named fields of the context, copied to/from `dst`/`src` (where = 0 host,
 * 1 device).  which: 0 u, 1 v, 2 p, 3 H, 4 rho, 5 beta_x, 6 beta_y, 7 Fx,
 * 8 Fy, 9 rhs b, 10 mu, 11 u*, 12 v*.  Sizes follow the layout above.    */
ib_status ib_get_field(ib_ctx *ctx, int which, double *dst, int where);
ib_status ib_set_field(ib_ctx *ctx, int which, const double *src, int where);

/* Section 4 Eq. (ten_f): signed discrete curvature at each marker (positive
 * for a convex counter-clockwise drop), unit inward normal and arc weight
 * ds_m = (|X_m - X_{m-1}| + |X_{m+1} - X_m|)/2.  Device outputs, nmarkers
 * each; any may be NULL.                                                   */
ib_status ib_marker_geometry(ib_ctx *ctx, double *kappa, double *nx,
                             double *ny, double *ds);

/* Marker-to-cell binning: key = floor((Y-y0)/h)*nx + floor((X-x0)/h) and the
 * marker ids ordered by (key, id); device outputs (uint32, nmarkers each;
 * either may be NULL) and cell_start (uint32, nx*ny+1, may be NULL).
 * Planar contexts only (IB_EINVAL in axisymmetric mode, whose binning grid
 * carries ghost columns).                                                  */
ib_status ib_marker_sort(ib_ctx *ctx, uint32_t *keys_sorted,
                         uint32_t *ids_sorted, uint32_t *cell_start);

/* Section 2.2 Eq. (jump_condu): U(X_m) = sum over faces u phi(rx) phi(ry)
 * with the configured kernel; u, v device face arrays, U, V device
 * marker arrays (nmarkers).                                                */
ib_status ib_interp(ib_ctx *ctx, const double *u, const double *v, double *U,
                    double *V);

/* Surface-tension spreading onto faces.  mode 0: conventional, Sec. 3.1 Eq.
 * (delta_vec), F = sum_m fmag_m n_m ds_m phi phi / h^2, a deterministic
 * gather over markers sorted by cell.  mode 1: irrotational, Sec. 3.2 Eqs.
 * (delta_hea), (delta_hea_xy): H from the five-strip polygons about every
 * segment, F = f_face (H_ij - H_{i-1,j}) / h with f_face from the nearest
 * segment.  fmag: device per-marker force magnitude, or NULL for sigma *
 * kappa.  Fx, Fy device face arrays; H device cell array or NULL (mode 1
 * only; mode 0 leaves H untouched).  Also stores Fx, Fy (and H) in the
 * context.                                                                 */
ib_status ib_spread(ib_ctx *ctx, int mode, const double *fmag, double *Fx,
                    double *Fy, double *H);

/* Section 3.2 polygon discrete Heaviside alone (device cell array).        */
ib_status ib_heaviside(ib_ctx *ctx, double *H);

/* Section 4 Eqs. (bspline), (bcurve), (bspline_ls): least-squares periodic
 * cubic B-spline through each drop's markers (knot spacing ~1.5 h, chord
 * length parameters) and re-placement of the same number of markers at equal
 * arc length.  Updates the context's markers.  IB_EINVAL if a drop's normal
 * equations are not positive definite.                                     */
ib_status ib_relocate(ib_ctx *ctx);

/* Section 2.1 Eq. (ps): load the face coefficients beta_x, beta_y (device
 * face arrays) the solver will use and build the coarse hierarchy
 * (coarse face = mean of its two fine faces, FP32 copies, inverse
 * diagonals, dense LU of the coarsest level).                              */
ib_status mg_setup(ib_ctx *ctx, const double *bx, const double *by);

/* Solve div(beta grad p) = rhs - mean(rhs) with the coefficients of the last
 * mg_setup (or ns_step) to ||b - A p||_2 <= tol ||b||_2 by V(nu1,nu2)
 * cycles (precision 0) or FP64 defect correction around FP32 V-cycles, one
 * (precision 1) or two (precision 2, the second starting from the first's
 * correction) per FP64 residual; *cycles_out counts V-cycles.  The residual,
 * its norm, the update of p and the coarsest solve stay FP64.  p (device
 * cell array) is the initial guess on entry and
 * the mean-zero solution on exit; rhs (device) is not modified.  cycles_out,
 * relres_out are host pointers (may be NULL).  Returns IB_ENOTCONV when the
 * cap is reached (p holds the last iterate) and IB_ENAN on a non-finite
 * residual.  IB_ECUDA also reports a smoother fault (ib_last_error names it):
 * a block whose wait for its staged tile ran out (50 ms) skips the tile and
 * waits up to 0.5 s more for its copies to land; the solve's result is then
 * not to be trusted, but the context stays usable and the next solve starts
 * with a clear fault word.                                                 */
ib_status mg_solve(ib_ctx *ctx, const double *rhs, double *p, int precision,
                   double tol, int max_cycles, int *cycles_out,
                   double *relres_out);

/* One or more time steps of Section 2.1's fractional step with the force in
 * the projection (Sec. 3.2 Eq. (ns2_new)): [B-spline relocation every
 * relocate_every steps, Sec. 2.5 measure correction every mass_every],
 * curvature, Heaviside (or the indicator), rho/mu/beta (Eq. (indicator)),
 * AB2 advection + viscous predictor (Eqs. (ad_bf), (cr_ni); explicit or
 * Crank-Nicolson), spreading, rhs, pressure solve, correction,
 * interpolation and marker advection X += dt U.  warm: the pressure solve's
 * initial guess, 0 zero, 1 the previous step's pressure, 2 the attached
 * network's estimate (square grid, side a multiple of 4), 3 the previous
 * two steps' pressures extrapolated in time, 2 p^n - p^(n-1) (p^n until two
 * exist).  The last step's cycles and residual are returned by
 * ib_last_solve.  A step queues the launches after the pressure solve
 * without waiting for the solve to end; the solve's status is read with the
 * step's marker flags, so a step whose solve returns IB_ENOTCONV (or reports
 * a smoother fault, IB_ECUDA) has still corrected the velocity with the last
 * iterate and moved the markers.  The solve's status comes first when the
 * marker flags also report an error; nsteps > 1 stops after that step.     */
ib_status ns_step(ib_ctx *ctx, double dt, int nsteps, int warm);

/* One time step as ns_step(ctx, dt, 1, warm) with host buffers (pinned
 * memory lets the copies run asynchronously): X_in, Y_in (M doubles each,
 * or both NULL) replace the markers first, after the same host checks as
 * ib_set_markers; p_out (nx*ny doubles, row-major), X_out, Y_out (M each;
 * either may be NULL, X_out and Y_out together) receive the step's pressure
 * and markers.  The copies are queued on the context's stream around the
 * step, which synchronises with the host once at its end; the buffers are
 * the caller's and must stay valid until the call returns.  Errors as
 * ns_step; IB_EINVAL for an unpaired marker buffer.                       */
ib_status ns_step_io(ib_ctx *ctx, double dt, int warm, const double *X_in, const double *Y_in,
                     double *p_out, double *X_out, double *Y_out);
/* Non-inertial frame (cfg.frame = 1): out[0] drop 0's axial centre of mass,
 * out[1] the acceleration S of the next step, out[2] the frame velocity Vf
 * (the drop's velocity in the laboratory, up to its small drift in the
 * frame), out[3] the boundary velocity -Vf; host array, synchronises.
 * IB_EINVAL without a frame.                                               */
ib_status ib_frame_state(ib_ctx *ctx, double *out);
/* Section 2.5 measure correction of the current markers against the drops'
 * measures at ib_init (tolerance cfg.mass_tol, or 1e-6 if it is 0); eps
 * (host, ndrops, may be NULL) receives each drop's normal offset (0 where
 * none was needed).  Synchronises.                                          */
ib_status ib_mass_correct(ib_ctx *ctx, double *eps);
ib_status ib_last_solve(const ib_ctx *ctx, int *cycles, double *relres);

/* ---------------------------------------------------------------------- */
/* Learned warm start (no counterpart in the paper; the network only moves
 * the starting point of the multigrid solve, which still runs to the same
 * residual tolerance).  A 3-level encoder/decoder CNN, channels c1 = 16 and
 * c2 = 32 (the only supported widths), BF16 weights and activations with
 * FP32 accumulation on the tensor cores, FP32 master weights and Adam state.
 * Input of a sample: rhs b and cell density rho (device FP64 N x N, N a
 * multiple of 4, cell size h; B samples stored back to back); features
 * ((b - mean b)/s, (1/rho)/max(1/rho)) with s = rms(b - mean b); target
 * p / (s h^2 c) with a mean-removed squared-error loss; output
 * p0 = s h^2 c (y - mean y).  c is the network's pressure scale
 * (cnn_set_scale, default 1), set from the training data.
 * Parameters are a flat FP32 host array, layer by layer (c1a, c1b, c2a, c2b,
 * c3a, c3b, c4, c5, c6), each weights [cout][3][3][cin] then bias [cout].
 * Calls run on `stream`; cnn_train_step, cnn_grad synchronise it when they
 * return the loss (host float, may be NULL).                               */
typedef struct ib_cnn ib_cnn;
ib_status cnn_init(ib_cnn **out, int32_t c1, int32_t c2, uint64_t seed, void *stream);
void cnn_destroy(ib_cnn *net);
int64_t cnn_num_params(const ib_cnn *net);
ib_status cnn_get_params(ib_cnn *net, float *host, int64_t n);
ib_status cnn_set_params(ib_cnn *net, const float *host, int64_t n);  /* resets Adam */
/* Loss and parameter gradients (host, cnn_num_params floats) without update. */
ib_status cnn_grad(ib_cnn *net, int32_t B, int32_t N, double h, const double *rhs,
                   const double *rho, const double *p, float *loss,
                   float *grads_host, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on a batch.            */
ib_status cnn_train_step(ib_cnn *net, int32_t B, int32_t N, double h,
                         const double *rhs, const double *rho, const double *p,
                         float lr, float *loss, void *stream);
/* The pressure scale c from training data (device FP64, B samples of
 * N x N, cell size h): the median over the samples of
 * rms(p - mean p) / (rms(b - mean b) h^2), samples with a constant b
 * skipped, the mean of the two middle values for an even count.  Sets the
 * network's scale and returns it in *c_out (host, may be NULL); synchronises.
 * IB_EINVAL if no sample has a varying b.                                  */
ib_status cnn_fit_scale(ib_cnn *net, int32_t B, int32_t N, double h, const double *rhs,
                        const double *p, double *c_out, void *stream);
/* Training run: cnn_fit_scale on all nsamples samples, then `steps` Adam
 * steps, each on `batch` samples drawn with replacement by a SplitMix64
 * stream of `seed` and gathered on the device, the learning rate
 * lr0 * 0.1^(k / steps) at step k (a tenfold decay over the run).  losses
 * (host, `steps` floats) receives each step's batch loss; one
 * synchronisation at the end.                                              */
ib_status cnn_train(ib_cnn *net, int32_t nsamples, int32_t N, double h, const double *rhs,
                    const double *rho, const double *p, int32_t steps, int32_t batch,
                    float lr0, uint64_t seed, float *losses, void *stream);
/* p0 (device FP64, B x N x N) = network estimate of the pressure.  With
 * cnn_set_coarsen(net, k), k > 0, rhs and rho are first averaged over
 * 2^k x 2^k blocks, the network runs on that grid (cell size h 2^k) and its
 * estimate is interpolated back to N x N (cell-centred bilinear, zero
 * gradient at the walls, once per halving); N must then be a multiple of
 * 4 * 2^k.  The same setting applies to ns_step(..., warm = 2).
 * IB_EINVAL for bad sizes, IB_ENOMEM if the scratch cannot be allocated.  */
ib_status cnn_infer(ib_cnn *net, int32_t B, int32_t N, double h, const double *rhs,
                    const double *rho, double *p0, void *stream);
ib_status cnn_set_coarsen(ib_cnn *net, int32_t levels);   /* 0 .. 6 */
/* Convolution path of the forward pass: 0 the warp-level mma.sync kernel
 * for every layer; 1 (default) the fifth-generation tensor cores
 * (tcgen05.mma, FP32 accumulators in tensor memory) for the layer shapes
 * where they measured faster (16 -> 32 channels) when the width is a
 * multiple of 128, the warp-level kernel elsewhere; 2 tcgen05 for every
 * layer whose width is a multiple of 128.  The paths accumulate in the same
 * order and agree bit for bit.  The backward pass always uses the
 * warp-level kernel.
 * cnn_grad and cnn_train return IB_ECUDA if a tensor-core completion wait
 * ran out (50 ms).                                                         */
ib_status cnn_set_tensor_path(ib_cnn *net, int32_t mode);
ib_status cnn_set_scale(ib_cnn *net, double c);
double cnn_get_scale(const ib_cnn *net);
/* Attach (or detach with NULL) a network used by ns_step(..., warm = 2); the
 * context does not own it.                                                 */
ib_status ib_attach_cnn(ib_ctx *ctx, ib_cnn *net);

/* Measurement hooks.  ib_launch_count: kernels launched by this library in
 * this process so far.  ib_profile_begin(kind) starts CUDA-event timing, on
 * the launching stream, of every launch of one kernel class (0: fine-level
 * FP64 smoother launch (one sweep, or two fused in V(2,2)), 1: fine-level
 * FP32 smoother launch, 2: fine-level FP64 residual norm, 3: the fine-level
 * FP32 prolongation + post-smoothing launch that also adds the cycle's
 * result to the FP64 iterate (defect correction), alone), or of one part of
 * every ns_step on the context stream (4: the launches before the pressure
 * solve, side streams joined; 5: the warm start and the pressure solve; 6:
 * the launches after it).  Kinds 0-3 launch one kernel at a time (no CUDA
 * graph replay while they are active); kinds 4-6 leave the graphs on.
 * ib_profile_end synchronises on the recorded events and
 * returns their summed duration (ms) and count.  Timing is process-wide and
 * not thread-safe; at most 16384 launches are recorded.                    */
unsigned long long ib_launch_count(void);
/* FP64 FMA throughput of the current device (TFLOP/s, an FMA counted as two
 * operations): three timed launches of independent FMA chains on every SM,
 * CUDA events on `stream` (synchronises it).  The peak against which FP64-
 * bound kernels are stated.                                                */
ib_status ib_probe_fp64(void *stream, double *tflops);
/* Solve with the captured CUDA graph (default, enable = 1) or with one launch
 * per kernel and a host residual check per cycle (enable = 0); results are
 * the same.  Kernels inside the graph's device-side loop cannot be timed
 * one by one by events or kernel profilers, hence the switch.             */
ib_status ib_use_graphs(ib_ctx *ctx, int enable);
/* Test hook for the failure path above: with enable = 1, every TMA-staged
 * FP32 smoother block (precision 1 and 2 solves, levels whose width is a
 * multiple of 4), after its copies have landed, also waits on a barrier
 * phase that nothing completes, so that its bounded wait runs out and the
 * solve returns IB_ECUDA; enable = 0 restores normal operation.  Process-wide
 * (a device variable of the current device); IB_ECUDA if it cannot be set. */
ib_status ib_debug_stall_staging(int enable);
ib_status ib_profile_begin(int kind);
ib_status ib_profile_end(double *total_ms, int *launches);
/* Kernel timing on the context's current data: `reps` back-to-back launches
 * of one kernel between two CUDA events on the context stream (after one
 * untimed launch); *us_per_launch = their mean duration, *units = the work
 * units of one launch.  which (at multigrid level `level`, 0 = finest):
 * 0 FP32 two-sweep smoother, 1 FP64 sweep, 3 FP32 sweeps + residual +
 * restriction, 4 FP32 prolongation + sweeps (at level 0 with the FP64
 * update of the defect correction, as in the solve) (units = cells of the
 * level); 7 FP64 two sweeps + residual + restriction, 8 FP64 prolongation +
 * two sweeps (the fused V(2,2) kernels of the FP64 solve; cells of the
 * level); 5 the FP32 single-CTA lower cycle (cells of its first level), 6 the
 * FP64 residual norm of the mixed solve (cells); 2 band strip areas of the
 * last Heaviside pass (units = (cell, segment) pairs; level ignored); 9 the
 * predictor on the current fields, 10 the irrotational face force (planar
 * contexts) from the last step's H and marker forces (both into scratch
 * the call allocates and frees; units = faces, (nx + 1) ny + nx (ny + 1)).  Only
 * solve scratch is overwritten (second iterate buffers, coarse right-hand
 * sides, the solver's level-0 FP64 iterate copy, FP32 residual, norm
 * partials) and the strip areas are recomputed: the
 * context's state is unchanged.  Needs a prior solve (or, for 2, Heaviside
 * pass); IB_EINVAL if the kernel does not run at that level.              */
ib_status ib_bench_kernel(ib_ctx *ctx, int which, int level, int reps, double *us_per_launch,
                          double *units);

/* Checkpoint: every field, the AB2 history, markers and the step counter,
 * written to / read from a binary file at `path` (host I/O, synchronises).
 * ib_load requires a context with the same nx, ny and marker count.       */
ib_status ib_save(ib_ctx *ctx, const char *path);
ib_status ib_load(ib_ctx *ctx, const char *path);

/* ---------------------------------------------------------------------- */
/* Pressure solve that allocates nothing (the paper has no counterpart; it
 * serves callers that cannot allocate device memory: code running under a
 * memory manager that owns all device memory, such as a framework's caching
 * allocator or a fixed-budget embedded deployment, and latency-critical loops
 * that cannot afford cudaMalloc's implicit device synchronisation).
 *
 * Same solve as mg_setup + mg_solve with the host-driven cycle loop, on the
 * coefficients bx, by (device face arrays, walls ignored), right-hand side
 * rhs and initial guess / mean-zero solution p (device cell arrays) of an
 * nx x ny grid with cell size h, launched on `stream`.  Its scratch (the
 * multigrid hierarchy, coarsest LU, reduction partials) is one file-scope
 * device array of IB_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading
 * the library holds until the process exits; grids above
 * IB_NOALLOC_MAX_CELLS cells (or whose hierarchy does not fit) return
 * IB_EINVAL.  No cudaMalloc, cudaFree or other allocating call is made.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All
 * calls share the array and its contents persist between calls, so calls
 * that overlap on the GPU (other streams, other host threads) race; the call
 * is not thread-safe.  precision 0, 1 or 2 as in mg_solve.  Status codes as
 * mg_solve; mg_solve_noalloc_error() returns the last call's message (empty
 * after a success; stored in the library, so it shares the one-caller-at-a-
 * time rule of the scratch array).                                         */
#define IB_NOALLOC_SCRATCH_BYTES (16u << 20)
#define IB_NOALLOC_MAX_CELLS 65536
ib_status mg_solve_noalloc(int32_t nx, int32_t ny, double h, const double *bx,
                           const double *by, const double *rhs, double *p,
                           int precision, double tol, int max_cycles, int nu1,
                           int nu2, int *cycles_out, double *relres_out,
                           void *stream);
const char *mg_solve_noalloc_error(void); /* never NULL */

/* ---------------------------------------------------------------------- */
/* Context-free grid operators (device arrays, launched on `stream`, no
 * allocation).  Each is one step of the path, exposed for verification.
 * Errors: IB_EINVAL for bad sizes or NULL pointers, IB_ECUDA on launch
 * failure.                                                                 */

/* Section 2.2 Eq. (indicator) and Section 2.1: rho, mu from H; beta on
 * faces = 1 / (two-cell average of rho), walls 0.                          */
ib_status ib_op_coeffs(int32_t nx, int32_t ny, double rho_g, double rho_l,
                       double mu_g, double mu_l, const double *H, double *rho,
                       double *mu, double *bx, double *by, void *stream);
/* Section 2.1 Eq. (ps): r = b - A p (A the 5-point flux-form operator).    */
ib_status ib_op_residual(int32_t nx, int32_t ny, double h, const double *bx,
                         const double *by, const double *b, const double *p,
                         double *r, void *stream);
/* nsweeps red-black Gauss-Seidel sweeps on A p = b (red = (i+j) even first). */
ib_status ib_op_rbgs(int32_t nx, int32_t ny, double h, const double *bx,
                     const double *by, const double *b, double *p,
                     int32_t nsweeps, void *stream);
/* rc = average of the four children of r - A p (nx, ny even).            */
ib_status ib_op_restrict_residual(int32_t nx, int32_t ny, double h,
                                  const double *bx, const double *by,
                                  const double *b, const double *p, double *rc,
                                  void *stream);
/* ef += bilinear prolongation (9,3,3,1)/16 of ec (nxc x nyc).             */
ib_status ib_op_prolong_add(int32_t nxc, int32_t nyc, const double *ec,
                            double *ef, void *stream);
/* Coarse faces = mean of the two fine faces (nx, ny even).                 */
ib_status ib_op_coarsen_beta(int32_t nx, int32_t ny, const double *bx,
                             const double *by, double *bxc, double *byc,
                             void *stream);
/* Section 2.1 Eq. (ps) and Sec. 3.2 Eq. (ns2_new):
 * b = div(u*)/dt + div(beta F).                                            */
ib_status ib_op_rhs(int32_t nx, int32_t ny, double h, double dt,
                    const double *us, const double *vs, const double *Fx,
                    const double *Fy, const double *bx, const double *by,
                    double *b, void *stream);
/* u = u* + dt beta (F - grad p) on interior faces, walls 0.               */
ib_status ib_op_correct(int32_t nx, int32_t ny, double h, double dt,
                        const double *us, const double *vs, const double *p,
                        const double *Fx, const double *Fy, const double *bx,
                        const double *by, double *u, double *v, void *stream);
/* Section 2.1 Eqs. (ad_bf), (cr_ni): u* = u + dt((D - (3/2 A - 1/2 A_prev))
 * / rho_face + g), Euler when have_prev = 0; au, av receive A (face
 * arrays).                                                                 */
ib_status ib_op_predictor(int32_t nx, int32_t ny, double h, double dt,
                          const double *rho, const double *mu, const double *u,
                          const double *v, const double *au_prev,
                          const double *av_prev, int32_t have_prev, double gx,
                          double gy, double *us, double *vs, double *au,
                          double *av, void *stream);

/* Axisymmetric (r, z) forms (Section 2.1 in cylindrical coordinates; x = r
 * from the axis, cell i at r = (i + 1/2) h, x-face i at r = i h).
 * Predictor: the same AB2 + viscous update on ring control volumes (fluxes
 * times their face radius over the volume radius; the radial component adds
 * -mu u / r^2), u = 0 on the axis and walls, gy the axial body acceleration;
 * frame: NULL (fixed walls) or device doubles whose slot 3 is an extra axial
 * acceleration S and slot 5 the axial velocity wb of the z boundaries and
 * the outer wall (the non-inertial frame's record).
 * Right-hand side: r_i div(u* / dt + beta F) with the axisymmetric
 * divergence (the right-hand side of the r-weighted pressure equation).
 * Weights: bxa = r_face bx, bya = r_i by (its coefficients).               */
ib_status ib_op_predictor_axi(int32_t nx, int32_t ny, double h, double dt,
                              const double *rho, const double *mu,
                              const double *u, const double *v,
                              const double *au_prev, const double *av_prev,
                              int32_t have_prev, double gy, const double *frame,
                              double *us, double *vs, double *au, double *av,
                              void *stream);
ib_status ib_op_rhs_axi(int32_t nx, int32_t ny, double h, double dt,
                        const double *us, const double *vs, const double *Fx,
                        const double *Fy, const double *bx, const double *by,
                        double *b, void *stream);
/* Crank-Nicolson viscous solve (Section 2.1): nsweeps red-black sweeps on
 * u* - dt / (2 rho_f) D(u*) = u_e for both components (planar, or
 * axisymmetric with fixed outer wall), starting from u_e; boundary faces keep
 * u_e's values.  ue, ve: inputs; us, vs: outputs (device face arrays).     */
ib_status ib_op_cn_solve(int32_t nx, int32_t ny, double h, double dt,
                         const double *rho, const double *mu, int32_t axisym,
                         int32_t nsweeps, const double *ue, const double *ve,
                         double *us, double *vs, void *stream);
ib_status ib_op_axi_weights(int32_t nx, int32_t ny, double h, const double *bx,
                            const double *by, double *bxa, double *bya,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif
