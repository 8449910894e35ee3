// C ABI of the library (declared in include/ib.h): the context that owns the
// fields, markers and multigrid hierarchy, the composed time step, and the
// context-free verification entry points.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ib_internal.cuh"

// A recorded phase of a time step: its launches as a CUDA graph, keyed by
// the time step and the step's options.
struct StepGraph {
    double dt = 0.0;
    int key = 0;
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;
};

struct ib_ctx {
    ib_config cfg;
    cudaStream_t s = nullptr;
    std::string err;
    ibk::MG mg;
    ibk::Markers mk;
    double *u = nullptr, *v = nullptr, *us = nullptr, *vs = nullptr, *au = nullptr,
           *av = nullptr, *p = nullptr, *H = nullptr, *rho = nullptr, *mu = nullptr,
           *bx = nullptr, *by = nullptr, *Fx = nullptr, *Fy = nullptr, *b = nullptr;
    void *fmem = nullptr;
    int step = 0;
    int have_prev = 0;
    int last_cycles = 0;
    double last_relres = 0.0;
    bool mg_ready = false;
    uint32_t *flags_host = nullptr;
    struct ib_cnn *cnn = nullptr;   // attached warm-start network (not owned)
    // axisymmetric mode: ghost columns G of the marker grid (origin -G h), the
    // velocity continued onto it, the Heaviside and forces computed on it, the
    // r-weighted pressure coefficients and the ring force magnitudes
    int G = 0;
    double *uw = nullptr, *vw = nullptr, *Hw = nullptr, *Fxw = nullptr, *Fyw = nullptr,
           *bxa = nullptr, *bya = nullptr, *fr = nullptr;
    double *frame = nullptr;   // non-inertial frame record (kFrSlots doubles)
    double *ue = nullptr, *ve = nullptr, *mh = nullptr;  // Crank-Nicolson: u_e and mu / 2
    double *pprev = nullptr;   // the previous step's pressure (warm start 3)
    bool have_pprev = false;
    // indicator function (Eq. (ind_psn)): unit coefficients, the solution
    // carried between steps, the wall mean
    double *ibx = nullptr, *iby = nullptr, *isol = nullptr, *iref = nullptr, *ione = nullptr;
    void *imem = nullptr;
    // side stream of a step: the multigrid hierarchy is built there while the
    // predictor, spreading and right-hand side run on s
    cudaStream_t s2 = nullptr, s3 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join3 = nullptr;
    cudaEvent_t ev_sort_fork = nullptr, ev_sort_join = nullptr;  // the marker sort on s2
    cudaEvent_t ev_rows_fork = nullptr, ev_rows_join = nullptr;  // the rows inside on s3
    cudaEvent_t ev_force_fork = nullptr;  // the face force on s3, after the Heaviside
    // recorded step phases (see run_recorded) and their capture stream
    std::vector<StepGraph> sgraphs;
    cudaStream_t cap = nullptr;
    bool step_graphs_off = false;
    double *A0 = nullptr;      // per drop: measure at ib_init (Section 2.5), then eps scratch
    void *dmem = nullptr;
    void *amem = nullptr;
};

// An inference of the network recorded as a CUDA graph, keyed by every value
// the launches bake in (pointers, sizes, the output scale and the workspace
// it was recorded against).
struct CnnGraph {
    int B = 0, N = 0, coarsen = 0;
    double h = 0, scale = 0;
    const double *rhs = nullptr, *rho = nullptr;
    double *p0 = nullptr;
    const void *amem = nullptr, *cbuf = nullptr;
    cudaGraphExec_t exec = nullptr;   // null: seen once, not recorded yet
    unsigned long long kernels = 0;
};

struct ib_cnn {
    ibk::Cnn *n = nullptr;
    int coarsen = 0;   // inference grid = solve grid / 2^coarsen
    std::string err;
    std::vector<CnnGraph> graphs;
    cudaStream_t cap = nullptr;   // private stream the graphs are recorded on
    bool no_graphs = false;
};

namespace {

using namespace ibk;

ib_status fail(ib_ctx *c, ib_status st, const std::string &msg)
{
    if (c) c->err = msg;
    return st;
}

// One inference of the network (cnn_infer_levels) on stream s.  A call whose
// key was seen before replays a CUDA graph of the same launches (recorded on
// the handle's private stream on the second call, once the first has sized
// the workspace), so the ~30 small launches of a coarse-grid inference cost
// one launch; the first call of a key, and every call if recording fails,
// runs the launches directly.
cudaError_t cnn_run(ib_cnn *h, int B, int N, double hs, const double *rhs, const double *rho,
                    double *p0, cudaStream_t s)
{
    Cnn &n = *h->n;
    const double scale = cnn_get_scale(n);
    CnnGraph *g = nullptr;
    for (auto &q : h->graphs)
        if (q.B == B && q.N == N && q.coarsen == h->coarsen && q.h == hs && q.scale == scale &&
            q.rhs == rhs && q.rho == rho && q.p0 == p0)
            g = &q;
    if (g && (g->amem != cnn_workspace_ptr(n) || g->cbuf != cnn_cbuf_ptr(n))) {
        // the workspace moved since: forget the recording
        if (g->exec) cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
        g->amem = cnn_workspace_ptr(n);
        g->cbuf = cnn_cbuf_ptr(n);
    }
    if (!h->no_graphs && g && !g->exec) {
        cudaError_t e = h->cap ? cudaSuccess : cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
        const unsigned long long k0 = launch_count();
        if (e == cudaSuccess) e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t ei = cnn_infer_levels(n, B, N, hs, rhs, rho, p0, h->coarsen, h->cap);
            cudaGraph_t gr = nullptr;
            e = cudaStreamEndCapture(h->cap, &gr);
            if (e == cudaSuccess) e = ei;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, gr, 0);
            if (gr) cudaGraphDestroy(gr);
        }
        g->kernels = launch_count() - k0;
        note_launch(-(int)g->kernels);  // recording issues no kernel
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (g->exec) cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
            h->no_graphs = true;
        }
    }
    if (!h->no_graphs && g && g->exec) {
        note_launch((int)g->kernels);
        return cudaGraphLaunch(g->exec, s);
    }
    cudaError_t e = cnn_infer_levels(n, B, N, hs, rhs, rho, p0, h->coarsen, s);
    if (e == cudaSuccess && !g && !h->no_graphs) {
        if (h->graphs.size() >= 8) {
            if (h->graphs.front().exec) cudaGraphExecDestroy(h->graphs.front().exec);
            h->graphs.erase(h->graphs.begin());
        }
        CnnGraph q;
        q.B = B; q.N = N; q.coarsen = h->coarsen; q.h = hs; q.scale = scale;
        q.rhs = rhs; q.rho = rho; q.p0 = p0;
        q.amem = cnn_workspace_ptr(n);
        q.cbuf = cnn_cbuf_ptr(n);
        h->graphs.push_back(q);
    }
    return e;
}

ib_status cuda_check(ib_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return IB_OK;
    return fail(c, IB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

ib_status launch_check(ib_ctx *c, const char *what)
{
    return cuda_check(c, cudaGetLastError(), what);
}

size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

// Orientation and wall distance of host marker arrays.
// Ghost columns of the axisymmetric marker grid: the mirror half of the
// widest drop plus 8 cells, a multiple of 8, at most nx; 0 if it does not fit.
int axi_ghost(const ib_config &g, const double *X, int M)
{
    double w = 0.0;
    for (int m = 0; m < M; m++) w = fmax(w, fabs(X[m]));
    const long G = ((long)ceil(w / g.h) + 8 + 7) / 8 * 8;
    return G <= g.nx ? (int)G : 0;
}

ib_status check_markers_host(ib_ctx *c, const ib_config &g, const double *X, const double *Y,
                             const int32_t *ds, int nd)
{
    const double m3 = 3.0 * g.h;
    const double xlo = g.axisym ? -c->G * g.h : g.x0;  // the axisymmetric marker grid's left edge
    for (int d = 0; d < nd; d++) {
        int s = ds[d], e = ds[d + 1];
        if (e - s < 3) return fail(c, IB_EINVAL, "a drop needs at least 3 markers");
        if (g.axisym) {
            const int n = e - s;
            if (n % 2) return fail(c, IB_EMARKER, "an axisymmetric drop needs an even marker count");
            for (int k = 0; k <= n / 2; k++) {
                const int p = (n - k) % n;
                if (X[s + k] != -X[s + p] || Y[s + k] != Y[s + p])
                    return fail(c, IB_EMARKER, "an axisymmetric drop must be a mirror-symmetric "
                                               "meridian curve (marker k mirrors n - k)");
            }
        }
        double a = 0.0;
        for (int m = s; m < e; m++) {
            int n = (m + 1 == e) ? s : m + 1;
            if (!(X[m] >= xlo + m3 && X[m] <= g.x0 + g.nx * g.h - m3 && Y[m] >= g.y0 + m3 &&
                  Y[m] <= g.y0 + g.ny * g.h - m3))
                return fail(c, IB_EMARKER, "marker outside the domain or within 3 cells of a wall");
            a += X[m] * Y[n] - X[n] * Y[m];
        }
        if (!(a > 0.0)) return fail(c, IB_EMARKER, "drop markers are not counter-clockwise");
    }
    return IB_OK;
}

// Marker geometry (curvature, normals, arc weights, force magnitude), with
// the azimuthal curvature added in axisymmetric mode.
void geometry(ib_ctx *c)
{
    launch_geometry(c->mk, c->cfg.sigma, c->s);
    if (c->cfg.axisym) launch_axi_curvature(c->mk, c->cfg.sigma, c->s);
}

// Heaviside onto the real cells (through the wide grid in axisymmetric mode).
void heaviside_into(ib_ctx *c, double *H)
{
    if (!c->cfg.axisym) {
        launch_heaviside(c->mk, H, c->s, c->s3, c->ev_rows_fork, c->ev_rows_join);
        return;
    }
    launch_heaviside(c->mk, c->Hw, c->s, c->s3, c->ev_rows_fork, c->ev_rows_join);
    launch_axi_fold(c->cfg.nx, c->cfg.ny, c->G, c->cfg.h, 0, c->Hw, nullptr, nullptr, H, nullptr,
                    nullptr, c->s);
}

// Face force of one spreading mode onto the real faces, after geometry,
// sorting and (mode 1) the Heaviside H of the real cells.  Axisymmetric:
// conventional spreading of the ring magnitudes sigma kappa |r| on the wide
// grid, folded with division by the face radius; irrotational spreading on
// the wide grid's Heaviside (set by heaviside_into), folded.
void force_into(ib_ctx *c, int mode, const double *fmag, const double *H, double *Fx, double *Fy,
                cudaStream_t s)
{
    const ib_config &g = c->cfg;
    if (!g.axisym) {
        if (mode == 0) launch_spread_conv(c->mk, g.kernel, fmag, Fx, Fy, s);
        else launch_spread_irrot(c->mk, fmag, H, Fx, Fy, s);
        return;
    }
    if (mode == 0) {
        launch_axi_ring(c->mk, fmag, c->fr, s);
        launch_spread_conv(c->mk, g.kernel, c->fr, c->Fxw, c->Fyw, s);
    } else {
        launch_spread_irrot(c->mk, fmag, c->Hw, c->Fxw, c->Fyw, s);
    }
    launch_axi_fold(g.nx, g.ny, c->G, g.h, mode == 0, nullptr, c->Fxw, c->Fyw, nullptr, Fx, Fy, s);
}

// Indicator function of Section 2.2 Eq. (ind_psn) into I (after geometry and
// sorting): the conventional spreading of the unit normals (ring-weighted in
// axisymmetric mode) into Fx, Fy (scratch here), its divergence into b,
// the FP64 multigrid on unit (r-weighted) coefficients to 1e-12 from the
// previous step's solution, the wall mean removed and [0, 1] clipping.  The
// hierarchy is rebuilt with the pressure coefficients afterwards.
ib_status indicator_into(ib_ctx *c, double *I)
{
    const ib_config &g = c->cfg;
    force_into(c, 0, c->ione, nullptr, c->Fx, c->Fy, c->s);
    launch_div_faces(g.nx, g.ny, g.h, g.axisym, c->Fx, c->Fy, c->b, c->s);
    mg_build(c->mg, c->ibx, c->iby, c->s);
    int cyc = 0;
    double rr = 0.0;
    ib_status st = mg_run(c->mg, c->b, c->isol, 0, 1e-12, 300, g.nu1, g.nu2, &cyc, &rr, c->s, c->err);
    if (st != IB_OK) return st;
    launch_indicator_finish(g.nx, g.ny, g.axisym, c->isol, c->iref, I, c->s);
    return IB_OK;
}

// Section 2.5 measure correction: normals of the current markers, then the
// per-drop bisection offset (re-symmetrised in axisymmetric mode).
void mass_correct(ib_ctx *c, double *eps)
{
    const ib_config &g = c->cfg;
    launch_geometry(c->mk, g.sigma, c->s);
    launch_mass_correct(c->mk, c->A0, g.axisym, g.mass_tol > 0 ? g.mass_tol : 1e-6, eps, c->s);
    if (g.axisym) launch_axi_symmetrise(c->mk, c->s);
}

// Velocity at the markers (and optional advection), continued across the
// axis in axisymmetric mode; the curve is re-symmetrised after a move.
void interp_into(ib_ctx *c, const double *u, const double *v, double *U, double *V, double dt_move)
{
    const ib_config &g = c->cfg;
    if (!g.axisym) {
        launch_interp(c->mk, g.kernel, u, v, U, V, dt_move, c->s);
        return;
    }
    launch_axi_extend(g.nx, g.ny, c->G, u, v, c->uw, c->vw, c->s);
    launch_interp(c->mk, g.kernel, c->uw, c->vw, U, V, dt_move, c->s);
    if (dt_move != 0.0) launch_axi_symmetrise(c->mk, c->s);
}

ib_status read_flags(ib_ctx *c)
{
    cudaError_t e = cudaMemcpyAsync(c->flags_host, c->mk.flags, 3 * sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return cuda_check(c, e, "flags");
    ib_status st = IB_OK;
    if (c->flags_host[0]) st = fail(c, IB_EMARKER, "a marker left the domain or came within 3 cells of a wall");
    else if (c->flags_host[1]) st = fail(c, IB_EINVAL, "too many interface segments near a cell block or row");
    else if (c->flags_host[2]) st = fail(c, IB_EINVAL, "B-spline normal equations not positive definite");
    cudaMemsetAsync(c->mk.flags, 0, 3 * sizeof(uint32_t), c->s);
    return st;
}

double *field_ptr(ib_ctx *c, int which, size_t *n)
{
    const size_t nc = (size_t)c->cfg.nx * c->cfg.ny, fx = (size_t)(c->cfg.nx + 1) * c->cfg.ny,
                 fy = (size_t)c->cfg.nx * (c->cfg.ny + 1);
    switch (which) {
    case 0: *n = fx; return c->u;
    case 1: *n = fy; return c->v;
    case 2: *n = nc; return c->p;
    case 3: *n = nc; return c->H;
    case 4: *n = nc; return c->rho;
    case 5: *n = fx; return c->bx;
    case 6: *n = fy; return c->by;
    case 7: *n = fx; return c->Fx;
    case 8: *n = fy; return c->Fy;
    case 9: *n = nc; return c->b;
    case 10: *n = nc; return c->mu;
    case 11: *n = fx; return c->us;
    case 12: *n = fy; return c->vs;
    default: *n = 0; return nullptr;
    }
}

ib_status spread_into(ib_ctx *c, int mode, const double *fmag, double *Fx, double *Fy, double *H)
{
    Markers &mk = c->mk;
    geometry(c);
    launch_sort(mk, c->s);
    const double *f = fmag ? fmag : mk.fmag;
    double *Hd = H ? H : c->H;
    if (mode == 1) heaviside_into(c, Hd);
    force_into(c, mode, f, Hd, Fx, Fy, c->s);
    return launch_check(c, "spread");
}

// The launches of one time step before the pressure solve, on c->s: marker
// upkeep (relocation, measure correction), geometry, binning, Heaviside (or
// the indicator), properties and face coefficients; then, with the side
// stream, the multigrid hierarchy and the face force next to the predictor
// (and the Crank-Nicolson solve); the right-hand side; p = 0 for a cold start.
ib_status step_pre(ib_ctx *c, double dt, bool reloc, bool mass, int warm)
{
    const ib_config &g = c->cfg;
    Markers &mk = c->mk;
    if (reloc) {
        launch_relocate(mk, c->s);
        if (g.axisym) launch_axi_symmetrise(mk, c->s);
    }
    if (mass) mass_correct(c, nullptr);
    // the marker sort (integer work on the positions) on s2 next to the
    // curvature and segment records; both read only X, Y and write disjoint
    // arrays; they join before the band pairs, which need both
    cudaEventRecord(c->ev_sort_fork, c->s);
    cudaStreamWaitEvent(c->s2, c->ev_sort_fork, 0);
    launch_sort(mk, c->s2);
    cudaEventRecord(c->ev_sort_join, c->s2);
    geometry(c);
    cudaStreamWaitEvent(c->s, c->ev_sort_join, 0);
    heaviside_into(c, c->H);
    // the face force needs the geometry, the sort and H only: on s3 from
    // here, next to the properties, the hierarchy and the predictor (after
    // the indicator instead, which uses Fx, Fy as scratch)
    const bool early_force = !g.indicator;
    if (early_force) {
        cudaEventRecord(c->ev_force_fork, c->s);
        cudaStreamWaitEvent(c->s3, c->ev_force_fork, 0);
        force_into(c, g.spread, mk.fmag, c->H, c->Fx, c->Fy, c->s3);
        cudaEventRecord(c->ev_join3, c->s3);
    }
    const double *prop = c->H;
    if (g.indicator) {
        ib_status is = indicator_into(c, c->mh);
        if (is != IB_OK) return is;
        prop = c->mh;
    }
    launch_coeffs(g.nx, g.ny, g.rho_g, g.rho_l, g.mu_g, g.mu_l, prop, c->rho, c->mu, c->bx, c->by,
                  c->s);
    // explicit viscous term, or Crank-Nicolson: the explicit predictor with
    // half the viscosity, then the implicit half
    const double *mup = c->mu;
    if (g.viscous) {
        launch_scale((long)g.nx * g.ny, 0.5, c->mu, c->mh, c->s);
        mup = c->mh;
    }
    // on two side streams, overlapping the predictor: the hierarchy of the
    // pressure coefficients (the r-weighted operator r_face beta in
    // axisymmetric form), and (with the indicator) the face force; neither
    // depends on the other or on the predictor
    if (g.axisym) launch_axi_weights(g.nx, g.ny, g.h, c->bx, c->by, c->bxa, c->bya, c->s);
    cudaEventRecord(c->ev_fork, c->s);
    cudaStreamWaitEvent(c->s2, c->ev_fork, 0);
    mg_build(c->mg, g.axisym ? c->bxa : c->bx, g.axisym ? c->bya : c->by, c->s2, g.precision == 0);
    cudaEventRecord(c->ev_join, c->s2);
    if (!early_force) {
        cudaStreamWaitEvent(c->s3, c->ev_fork, 0);
        force_into(c, g.spread, mk.fmag, c->H, c->Fx, c->Fy, c->s3);
        cudaEventRecord(c->ev_join3, c->s3);
    }
    if (g.axisym)
        launch_predictor_axi(g.nx, g.ny, g.h, dt, c->rho, mup, c->u, c->v, c->au, c->av, c->have_prev,
                             0.0, g.gy, g.frame ? c->frame : nullptr, c->bx, c->by, c->us, c->vs,
                             c->au, c->av, c->s);
    else
        launch_predictor(g.nx, g.ny, g.h, dt, c->rho, mup, c->u, c->v, c->au, c->av, c->have_prev,
                         g.gx, g.gy, c->bx, c->by, c->us, c->vs, c->au, c->av, c->s);
    if (g.viscous) {
        cudaMemcpyAsync(c->ue, c->us, (size_t)(g.nx + 1) * g.ny * 8, cudaMemcpyDeviceToDevice, c->s);
        cudaMemcpyAsync(c->ve, c->vs, (size_t)g.nx * (g.ny + 1) * 8, cudaMemcpyDeviceToDevice, c->s);
        launch_cn_solve(g.nx, g.ny, g.h, dt, c->rho, c->mu, g.axisym, g.frame ? c->frame : nullptr,
                        g.cn_sweeps, c->ue, c->ve, c->us, c->vs, c->s);
    }
    c->mg_ready = true;
    cudaStreamWaitEvent(c->s, c->ev_join, 0);   // the hierarchy is complete
    cudaStreamWaitEvent(c->s, c->ev_join3, 0);  // and the force
    if (g.axisym)
        launch_rhs_axi(g.nx, g.ny, g.h, dt, c->us, c->vs, c->Fx, c->Fy, c->bx, c->by, c->b, c->s);
    else
        launch_rhs(g.nx, g.ny, g.h, dt, c->us, c->vs, c->Fx, c->Fy, c->bx, c->by, c->b, c->s);
    if (warm == 0) cudaMemsetAsync(c->p, 0, (size_t)g.nx * g.ny * 8, c->s);
    return launch_check(c, "step");
}

// The launches after the pressure solve: velocity correction, the frame's
// boundary velocity, marker advection (re-symmetrised), the frame update and
// the marker check.
ib_status step_post(ib_ctx *c, double dt)
{
    const ib_config &g = c->cfg;
    Markers &mk = c->mk;
    launch_correct(g.nx, g.ny, g.h, dt, c->us, c->vs, c->p, c->Fx, c->Fy, c->bx, c->by, c->u, c->v,
                   c->s);
    if (g.frame) launch_axi_zbc(g.nx, g.ny, c->frame, c->v, c->s);
    interp_into(c, c->u, c->v, mk.U, mk.V, dt);
    if (g.frame) launch_axi_frame(mk, dt, g.c1, g.c2, 0, c->frame, c->s);
    launch_validate(mk, c->s);
    return launch_check(c, "step");
}

// Runs fn's launches on c->s through a CUDA graph recorded the first time
// (dt, key) is seen: recorded on the private stream c->cap (c->s points at
// it meanwhile), then replayed on c->s.  Direct launches while graphs are
// off or per-kernel timing is active, and for good if recording fails.
template <typename F>
ib_status run_recorded(ib_ctx *c, double dt, int key, F fn)
{
    if (!c->mg.use_graphs || profiling_active() || c->step_graphs_off) return fn();
    StepGraph *sg = nullptr;
    for (auto &q : c->sgraphs)
        if (q.dt == dt && q.key == key) sg = &q;
    if (!sg) {
        if (c->sgraphs.size() >= 16) {
            cudaGraphExecDestroy(c->sgraphs.front().exec);
            c->sgraphs.erase(c->sgraphs.begin());
        }
        cudaStream_t user = c->s;
        c->s = c->cap;
        const unsigned long long k0 = launch_count();
        cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
        ib_status st = IB_OK;
        cudaGraph_t gr = nullptr;
        if (e == cudaSuccess) {
            st = fn();
            e = cudaStreamEndCapture(c->cap, &gr);
        }
        c->s = user;
        StepGraph q;
        q.dt = dt;
        q.key = key;
        q.kernels = launch_count() - k0;
        note_launch(-(int)q.kernels);  // recording launches nothing
        // per-node priorities: the side streams' launches (hierarchy, face
        // force) keep their higher priority inside the replayed graph, so
        // their blocks take free SM slots ahead of the predictor's
        if (e == cudaSuccess && st == IB_OK)
            e = cudaGraphInstantiate(&q.exec, gr, cudaGraphInstantiateFlagUseNodePriority);
        if (gr) cudaGraphDestroy(gr);
        if (e != cudaSuccess || st != IB_OK || !q.exec) {
            cudaGetLastError();
            c->err.clear();
            c->step_graphs_off = true;
            return fn();
        }
        c->sgraphs.push_back(q);
        sg = &c->sgraphs.back();
    }
    note_launch((int)sg->kernels);
    return cuda_check(c, cudaGraphLaunch(sg->exec, c->s), "step graph");
}

}  // namespace

extern "C" {

const char *ib_last_error(const ib_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : "null context";
}

void ib_destroy(ib_ctx *c)
{
    if (!c) return;
    if (c->s) cudaStreamSynchronize(c->s);
    else cudaDeviceSynchronize();
    mg_free(c->mg);
    markers_free(c->mk);
    if (c->fmem) cudaFree(c->fmem);
    if (c->amem) cudaFree(c->amem);
    if (c->dmem) cudaFree(c->dmem);
    if (c->imem) cudaFree(c->imem);
    for (auto &q : c->sgraphs)
        if (q.exec) cudaGraphExecDestroy(q.exec);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_join3) cudaEventDestroy(c->ev_join3);
    if (c->ev_sort_fork) cudaEventDestroy(c->ev_sort_fork);
    if (c->ev_sort_join) cudaEventDestroy(c->ev_sort_join);
    if (c->ev_rows_fork) cudaEventDestroy(c->ev_rows_fork);
    if (c->ev_rows_join) cudaEventDestroy(c->ev_rows_join);
    if (c->ev_force_fork) cudaEventDestroy(c->ev_force_fork);
    if (c->s2) cudaStreamDestroy(c->s2);
    if (c->s3) cudaStreamDestroy(c->s3);
    if (c->flags_host) cudaFreeHost(c->flags_host);
    delete c;
}

ib_status ib_init(ib_ctx **out, const ib_config *cfg, const double *X, const double *Y,
                  const int32_t *drop_start, int32_t ndrops, void *stream)
{
    if (!out) return IB_EINVAL;
    *out = nullptr;
    if (!cfg || !X || !Y || !drop_start || ndrops < 1) return IB_EINVAL;
    const ib_config &g = *cfg;
    if (g.nx < 2 || g.ny < 2 || (long)g.nx * g.ny > (1L << 28) || !(g.h > 0) || g.nu1 < 0 ||
        g.nu2 < 0 || g.max_cycles < 0 || !(g.tol >= 0) || g.kernel < 0 || g.kernel > 1 ||
        g.spread < 0 || g.spread > 1 || g.precision < 0 || g.precision > 2 || g.axisym < 0 ||
        g.axisym > 1 || (g.axisym && (g.x0 != 0.0 || g.gx != 0.0)) || g.frame < 0 || g.frame > 1 ||
        (g.frame && (!g.axisym || !(g.c1 >= 0) || !(g.c2 >= 0))) || g.mass_every < 0 ||
        !(g.mass_tol >= 0) || g.viscous < 0 || g.viscous > 1 || (g.viscous && g.cn_sweeps < 1) ||
        g.indicator < 0 || g.indicator > 1)
        return IB_EINVAL;
    std::vector<int> nxs, nys;
    if (!mg_levels(g.nx, g.ny, nxs, nys)) return IB_EINVAL;
    if (drop_start[0] != 0) return IB_EINVAL;
    for (int d = 0; d < ndrops; d++)
        if (drop_start[d + 1] - drop_start[d] < 3) return IB_EINVAL;
    const int M = drop_start[ndrops];
    if (M > (1 << 20)) return IB_EINVAL;
    ib_ctx *c = new ib_ctx();
    c->cfg = g;
    c->s = (cudaStream_t)stream;
    if (g.axisym) {
        c->G = axi_ghost(g, X, M);
        if (!c->G) { delete c; return IB_EMARKER; }
    }
    ib_status st = check_markers_host(c, g, X, Y, drop_start, ndrops);
    if (st != IB_OK) { delete c; return st; }
    const size_t nc = (size_t)g.nx * g.ny, fx = (size_t)(g.nx + 1) * g.ny, fy = (size_t)g.nx * (g.ny + 1);
    size_t bytes = al(fx * 8) * 6 + al(fy * 8) * 6 + al(nc * 8) * 7;
    if (cudaMalloc(&c->fmem, bytes) != cudaSuccess) { c->fmem = nullptr; ib_destroy(c); return IB_ENOMEM; }
    char *q = (char *)c->fmem;
    auto take = [&](size_t b) { char *r = q; q += al(b); return (double *)r; };
    c->u = take(fx * 8); c->us = take(fx * 8); c->au = take(fx * 8);
    c->bx = take(fx * 8); c->Fx = take(fx * 8);
    c->ue = take(fx * 8);
    c->v = take(fy * 8); c->vs = take(fy * 8); c->av = take(fy * 8);
    c->by = take(fy * 8); c->Fy = take(fy * 8);
    c->ve = take(fy * 8);
    c->p = take(nc * 8); c->H = take(nc * 8); c->rho = take(nc * 8); c->mu = take(nc * 8);
    c->b = take(nc * 8); c->mh = take(nc * 8); c->pprev = take(nc * 8);
    cudaError_t e = cudaMemset(c->fmem, 0, bytes);
    if (e == cudaSuccess) e = mg_alloc(c->mg, g.nx, g.ny, g.h);
    if (e == cudaSuccess && g.axisym) {
        const long nw = g.nx + c->G;
        const size_t wx = (size_t)(nw + 1) * g.ny, wy = (size_t)nw * (g.ny + 1), wc = (size_t)nw * g.ny;
        const size_t ab = 2 * al(wx * 8) + 2 * al(wy * 8) + al(wc * 8) + al(fx * 8) + al(fy * 8) +
                          al((size_t)M * 8) + al(kFrSlots * 8);
        e = cudaMalloc(&c->amem, ab);
        if (e == cudaSuccess) {
            char *a = (char *)c->amem;
            auto tk = [&](size_t b) { char *r = a; a += al(b); return (double *)r; };
            c->uw = tk(wx * 8); c->Fxw = tk(wx * 8);
            c->vw = tk(wy * 8); c->Fyw = tk(wy * 8);
            c->Hw = tk(wc * 8);
            c->bxa = tk(fx * 8); c->bya = tk(fy * 8);
            c->fr = tk((size_t)M * 8);
            c->frame = tk(kFrSlots * 8);
            e = cudaMemset(c->amem, 0, ab);
        } else {
            c->amem = nullptr;
        }
    }
    if (e == cudaSuccess)
        e = g.axisym ? markers_alloc(c->mk, M, ndrops, g.nx + c->G, g.ny, g.h, -c->G * g.h, g.y0, drop_start)
                     : markers_alloc(c->mk, M, ndrops, g.nx, g.ny, g.h, g.x0, g.y0, drop_start);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->flags_host, 64);
    if (e == cudaSuccess) e = cudaMemcpy(c->mk.X, X, (size_t)M * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->mk.Y, Y, (size_t)M * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && g.frame) {
        launch_axi_frame(c->mk, 1.0, g.c1, g.c2, 1, c->frame, c->s);
        e = cudaStreamSynchronize(c->s);
    }
    if (e == cudaSuccess && g.indicator) {
        const size_t ib = al(fx * 8) + al(fy * 8) + al(nc * 8) + al(8) + al((size_t)M * 8);
        e = cudaMalloc(&c->imem, ib);
        if (e == cudaSuccess) {
            char *a = (char *)c->imem;
            c->ibx = (double *)a; a += al(fx * 8);
            c->iby = (double *)a; a += al(fy * 8);
            c->isol = (double *)a; a += al(nc * 8);
            c->iref = (double *)a; a += al(8);
            c->ione = (double *)a;
            e = cudaMemset(c->imem, 0, ib);
            if (e == cudaSuccess) {
                launch_unit_beta(g.nx, g.ny, g.h, g.axisym, c->ibx, c->iby, c->s);
                launch_fill(M, 1.0, c->ione, c->s);
                e = cudaStreamSynchronize(c->s);
            }
        } else {
            c->imem = nullptr;
        }
    }
    if (e == cudaSuccess) {
        // highest priority: the side stream's small kernels (single-CTA
        // coefficient and coarse-inverse builds) take free SM slots ahead of
        // the predictor's blocks instead of waiting for its grid to drain
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        e = cudaStreamCreateWithPriority(&c->s2, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->s3, cudaStreamNonBlocking, hi);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join3, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_sort_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_sort_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_rows_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_rows_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_force_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&c->dmem, 2 * al((size_t)ndrops * 8));
    if (e == cudaSuccess) {
        c->A0 = (double *)c->dmem;
        launch_drop_measure(c->mk, g.axisym, c->A0, c->s);
        e = cudaStreamSynchronize(c->s);
    } else {
        c->dmem = nullptr;
    }
    if (e != cudaSuccess) {
        ib_status r = (e == cudaErrorMemoryAllocation) ? IB_ENOMEM : IB_ECUDA;
        ib_destroy(c);
        return r;
    }
    *out = c;
    return IB_OK;
}

int32_t ib_num_markers(const ib_ctx *c) { return c ? c->mk.M : 0; }

ib_status ib_set_markers(ib_ctx *c, const double *X, const double *Y, int where)
{
    if (!c || !X || !Y) return IB_EINVAL;
    const int M = c->mk.M;
    if (where == 0) {
        ib_status st = check_markers_host(c, c->cfg, X, Y, c->mk.drop_start_h.data(), c->mk.ndrops);
        if (st != IB_OK) return st;
    }
    cudaMemcpyKind k = where ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(c->mk.X, X, (size_t)M * 8, k, c->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->mk.Y, Y, (size_t)M * 8, k, c->s);
    if (e != cudaSuccess) return cuda_check(c, e, "set markers");
    if (where) {
        launch_validate(c->mk, c->s);
        return read_flags(c);
    }
    return IB_OK;
}

ib_status ib_get_markers(ib_ctx *c, double *X, double *Y, int where)
{
    if (!c || !X || !Y) return IB_EINVAL;
    cudaMemcpyKind k = where ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaMemcpyAsync(X, c->mk.X, (size_t)c->mk.M * 8, k, c->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Y, c->mk.Y, (size_t)c->mk.M * 8, k, c->s);
    if (e == cudaSuccess && !where) e = cudaStreamSynchronize(c->s);
    return cuda_check(c, e, "get markers");
}

ib_status ib_get_field(ib_ctx *c, int which, double *dst, int where)
{
    if (!c || !dst) return IB_EINVAL;
    size_t n;
    double *f = field_ptr(c, which, &n);
    if (!f) return fail(c, IB_EINVAL, "unknown field");
    cudaError_t e = cudaMemcpyAsync(dst, f, n * 8, where ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess && !where) e = cudaStreamSynchronize(c->s);
    return cuda_check(c, e, "get field");
}

ib_status ib_set_field(ib_ctx *c, int which, const double *src, int where)
{
    if (!c || !src) return IB_EINVAL;
    size_t n;
    double *f = field_ptr(c, which, &n);
    if (!f) return fail(c, IB_EINVAL, "unknown field");
    cudaError_t e = cudaMemcpyAsync(f, src, n * 8, where ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->s);
    if (which == 5 || which == 6) c->mg_ready = false;
    return cuda_check(c, e, "set field");
}

ib_status ib_marker_geometry(ib_ctx *c, double *kappa, double *nx, double *ny, double *ds)
{
    if (!c) return IB_EINVAL;
    geometry(c);
    const size_t b = (size_t)c->mk.M * 8;
    cudaError_t e = cudaSuccess;
    if (kappa && e == cudaSuccess) e = cudaMemcpyAsync(kappa, c->mk.kappa, b, cudaMemcpyDeviceToDevice, c->s);
    if (nx && e == cudaSuccess) e = cudaMemcpyAsync(nx, c->mk.nxm, b, cudaMemcpyDeviceToDevice, c->s);
    if (ny && e == cudaSuccess) e = cudaMemcpyAsync(ny, c->mk.nym, b, cudaMemcpyDeviceToDevice, c->s);
    if (ds && e == cudaSuccess) e = cudaMemcpyAsync(ds, c->mk.ds, b, cudaMemcpyDeviceToDevice, c->s);
    if (e != cudaSuccess) return cuda_check(c, e, "geometry");
    return launch_check(c, "geometry");
}

__global__ void k_gather_keys(int M, const uint32_t *key, const uint32_t *ids, uint32_t *out)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < M) out[k] = key[ids[k]];
}

ib_status ib_marker_sort(ib_ctx *c, uint32_t *keys_sorted, uint32_t *ids_sorted, uint32_t *cell_start)
{
    if (!c) return IB_EINVAL;
    if (c->cfg.axisym) return fail(c, IB_EINVAL, "marker binning is exposed for planar contexts only");
    Markers &mk = c->mk;
    launch_sort(mk, c->s);
    if (keys_sorted) { note_launch(); k_gather_keys<<<cdiv(mk.M, 256), 256, 0, c->s>>>(mk.M, mk.key, mk.ids, keys_sorted);
    }
    cudaError_t e = cudaSuccess;
    if (ids_sorted) e = cudaMemcpyAsync(ids_sorted, mk.ids, (size_t)mk.M * 4, cudaMemcpyDeviceToDevice, c->s);
    if (cell_start && e == cudaSuccess)
        e = cudaMemcpyAsync(cell_start, mk.cell_start, ((size_t)mk.nx * mk.ny + 1) * 4,
                            cudaMemcpyDeviceToDevice, c->s);
    if (e != cudaSuccess) return cuda_check(c, e, "sort");
    return launch_check(c, "sort");
}

ib_status ib_interp(ib_ctx *c, const double *u, const double *v, double *U, double *V)
{
    if (!c || !u || !v || !U || !V) return IB_EINVAL;
    interp_into(c, u, v, U, V, 0.0);
    return launch_check(c, "interp");
}

ib_status ib_spread(ib_ctx *c, int mode, const double *fmag, double *Fx, double *Fy, double *H)
{
    if (!c || !Fx || !Fy || mode < 0 || mode > 1) return IB_EINVAL;
    ib_status st = spread_into(c, mode, fmag, c->Fx, c->Fy, H ? H : nullptr);
    if (st != IB_OK) return st;
    st = read_flags(c);
    if (st != IB_OK) return st;
    const size_t fx = (size_t)(c->cfg.nx + 1) * c->cfg.ny, fy = (size_t)c->cfg.nx * (c->cfg.ny + 1);
    cudaError_t e = cudaMemcpyAsync(Fx, c->Fx, fx * 8, cudaMemcpyDeviceToDevice, c->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Fy, c->Fy, fy * 8, cudaMemcpyDeviceToDevice, c->s);
    if (e == cudaSuccess && H && mode == 1)
        e = cudaMemcpyAsync(c->H, H, (size_t)c->cfg.nx * c->cfg.ny * 8, cudaMemcpyDeviceToDevice, c->s);
    return cuda_check(c, e, "spread copy");
}

ib_status ib_heaviside(ib_ctx *c, double *H)
{
    if (!c || !H) return IB_EINVAL;
    geometry(c);
    launch_sort(c->mk, c->s);
    heaviside_into(c, H);
    ib_status st = launch_check(c, "heaviside");
    if (st != IB_OK) return st;
    return read_flags(c);
}

ib_status ib_relocate(ib_ctx *c)
{
    if (!c) return IB_EINVAL;
    launch_relocate(c->mk, c->s);
    if (c->cfg.axisym) launch_axi_symmetrise(c->mk, c->s);
    ib_status st = launch_check(c, "relocate");
    if (st != IB_OK) return st;
    return read_flags(c);
}

ib_status mg_setup(ib_ctx *c, const double *bx, const double *by)
{
    if (!c || !bx || !by) return IB_EINVAL;
    mg_build(c->mg, bx, by, c->s);
    c->mg_ready = true;
    return launch_check(c, "mg_setup");
}

ib_status mg_solve(ib_ctx *c, const double *rhs, double *p, int precision, double tol,
                   int max_cycles, int *cycles_out, double *relres_out)
{
    if (!c || !rhs || !p || precision < 0 || precision > 2 || max_cycles < 0 || !(tol >= 0))
        return IB_EINVAL;
    if (!c->mg_ready) return fail(c, IB_EINVAL, "mg_setup (or ns_step) has not loaded coefficients");
    int cyc = 0;
    double rr = 0.0;
    ib_status st = mg_run(c->mg, rhs, p, precision, tol, max_cycles, c->cfg.nu1, c->cfg.nu2,
                          &cyc, &rr, c->s, c->err);
    if (cycles_out) *cycles_out = cyc;
    if (relres_out) *relres_out = rr;
    return st;
}

}  // extern "C"

namespace {

ib_status step_args(ib_ctx *c, double dt, int nsteps, int warm)
{
    if (!c || !(dt > 0) || nsteps < 0 || warm < 0 || warm > 3) return IB_EINVAL;
    if (warm == 2 && c->cfg.axisym)
        return fail(c, IB_EINVAL, "the network warm start is trained for the planar equation");
    if (warm == 2 && (!c->cnn || c->cfg.nx != c->cfg.ny || c->cfg.nx % (4 << c->cnn->coarsen) != 0))
        return fail(c, IB_EINVAL, "warm start 2 needs an attached network and a square grid "
                                  "(side a multiple of 4 * 2^coarsen)");
    return IB_OK;
}

// One time step; before_flags enqueues work on c->s ahead of the step's
// final host synchronisation (the marker flags read).
template <typename F>
ib_status step_one(ib_ctx *c, double dt, int warm, F before_flags)
{
    const ib_config &g = c->cfg;
    const bool reloc = g.relocate_every > 0 && c->step % g.relocate_every == 0;
    const bool mass = g.mass_every > 0 && c->step > 0 && c->step % g.mass_every == 0;
    // the launches before the pressure solve replay a recorded graph once
    // the step's shape has been seen (not with the indicator's inner solve
    // or the network, which synchronise with the host)
    const bool rec = c->have_prev && !g.indicator && warm != 2;
    const int key = (reloc ? 1 : 0) | (mass ? 2 : 0) | (warm == 0 ? 4 : 0);
    const bool t_pre = prof_on(kProfPre), t_solve = prof_on(kProfSolve), t_post = prof_on(kProfPost);
    if (t_pre) prof_mark(c->s, true);
    ib_status st = rec ? run_recorded(c, dt, key, [&] { return step_pre(c, dt, reloc, mass, warm); })
                       : step_pre(c, dt, reloc, mass, warm);
    // the step rebuilt the hierarchy, with the FP64 sweep weights only for an
    // FP64 solver (a replayed graph runs no host code)
    c->mg.fp64_w = g.precision == 0;
    if (t_pre) prof_mark(c->s, false);
    if (st != IB_OK) return st;
    if (t_solve) prof_mark(c->s, true);
    if (warm == 2) {
        cudaError_t ce = cnn_run(c->cnn, 1, g.nx, g.h, c->b, c->rho, c->p, c->s);
        if (ce != cudaSuccess) return cuda_check(c, ce, "network warm start");
    }
    if (warm == 3) {
        // p0 = 2 p^n - p^(n-1) once two pressures are known, else p^n
        const long n = (long)g.nx * g.ny;
        if (c->have_pprev) launch_extrapolate(n, c->p, c->pprev, c->s);
        else cudaMemcpyAsync(c->pprev, c->p, (size_t)n * 8, cudaMemcpyDeviceToDevice, c->s);
        c->have_pprev = true;
    } else {
        c->have_pprev = false;
    }
    // the solve is queued without waiting for it: the launches after it
    // follow at once, and its status is read at the step's one
    // synchronisation (the flags read)
    MgPending pend;
    st = mg_run_launch(c->mg, c->b, c->p, g.precision, g.tol, g.max_cycles, g.nu1, g.nu2,
                       &c->last_cycles, &c->last_relres, c->s, c->err, pend);
    if (t_solve) prof_mark(c->s, false);
    if (st != IB_OK && st != IB_ENOTCONV) return st;
    if (t_post) prof_mark(c->s, true);
    const ib_status sp = rec ? run_recorded(c, dt, 64, [&] { return step_post(c, dt); })
                             : step_post(c, dt);
    if (t_post) prof_mark(c->s, false);
    if (sp != IB_OK) return sp;
    c->have_prev = 1;
    c->step++;
    before_flags();
    ib_status fs = read_flags(c);
    if (pend.pending) {
        // a failed solve is reported ahead of the flags (its message wins)
        const ib_status ss = mg_run_finish(c->mg, pend, &c->last_cycles, &c->last_relres, c->err);
        if (ss != IB_OK && ss != IB_ENOTCONV) return ss;
        st = ss;
    }
    if (fs != IB_OK) return fs;
    return st;
}

}  // namespace

extern "C" {

ib_status ns_step(ib_ctx *c, double dt, int nsteps, int warm)
{
    ib_status st = step_args(c, dt, nsteps, warm);
    if (st != IB_OK) return st;
    for (int it = 0; it < nsteps; it++) {
        st = step_one(c, dt, warm, [] {});
        if (st != IB_OK) return st;
    }
    return IB_OK;
}

ib_status ns_step_io(ib_ctx *c, double dt, int warm, const double *X_in, const double *Y_in,
                     double *p_out, double *X_out, double *Y_out)
{
    ib_status st = step_args(c, dt, 1, warm);
    if (st != IB_OK) return st;
    if ((X_in == nullptr) != (Y_in == nullptr) || (X_out == nullptr) != (Y_out == nullptr))
        return fail(c, IB_EINVAL, "marker buffers come in pairs (X and Y)");
    const size_t mb = (size_t)c->mk.M * 8;
    if (X_in) {
        st = check_markers_host(c, c->cfg, X_in, Y_in, c->mk.drop_start_h.data(), c->mk.ndrops);
        if (st != IB_OK) return st;
        cudaError_t e = cudaMemcpyAsync(c->mk.X, X_in, mb, cudaMemcpyHostToDevice, c->s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->mk.Y, Y_in, mb, cudaMemcpyHostToDevice, c->s);
        if (e != cudaSuccess) return cuda_check(c, e, "markers in");
    }
    cudaError_t ce = cudaSuccess;
    st = step_one(c, dt, warm, [&] {
        const size_t pb = (size_t)c->cfg.nx * c->cfg.ny * 8;
        if (p_out) ce = cudaMemcpyAsync(p_out, c->p, pb, cudaMemcpyDeviceToHost, c->s);
        if (X_out && ce == cudaSuccess) ce = cudaMemcpyAsync(X_out, c->mk.X, mb, cudaMemcpyDeviceToHost, c->s);
        if (Y_out && ce == cudaSuccess) ce = cudaMemcpyAsync(Y_out, c->mk.Y, mb, cudaMemcpyDeviceToHost, c->s);
    });
    if (ce != cudaSuccess) return cuda_check(c, ce, "results out");
    return st;
}

unsigned long long ib_launch_count(void) { return launch_count(); }

ib_status ib_use_graphs(ib_ctx *c, int enable)
{
    if (!c) return IB_EINVAL;
    c->mg.use_graphs = enable != 0;
    return IB_OK;
}

ib_status ib_debug_stall_staging(int enable)
{
    return set_stall_staging(enable) == cudaSuccess ? IB_OK : IB_ECUDA;
}

ib_status ib_profile_begin(int kind)
{
    if (kind < 0 || kind > 6) return IB_EINVAL;
    return prof_begin(kind) ? IB_OK : IB_ECUDA;
}

ib_status ib_profile_end(double *total_ms, int *launches)
{
    return prof_end(total_ms, launches) ? IB_OK : IB_ECUDA;
}

ib_status ib_bench_kernel(ib_ctx *c, int which, int level, int reps, double *us_per_launch,
                          double *units)
{
    if (!c || which < 0 || which > 10 || reps < 1 || !us_per_launch) return IB_EINVAL;
    if (which != 2 && !c->mg_ready) return fail(c, IB_EINVAL, "no multigrid hierarchy yet");
    if (which == 10 && c->cfg.axisym)
        return fail(c, IB_EINVAL, "the face-force timing is planar only");
    const ib_config &g = c->cfg;
    const long nfx = (long)(g.nx + 1) * g.ny, nfy = (long)g.nx * (g.ny + 1);
    double u = which >= 9 ? (double)(nfx + nfy) : 0.0;
    // the predictor and face-force timings write into scratch, not the state
    double *scr = nullptr;
    if (which >= 9) {
        cudaError_t e = cudaMalloc(&scr, (size_t)(nfx + nfy) * 2 * 8);
        if (e != cudaSuccess) return fail(c, IB_ENOMEM, "timing scratch");
    }
    if (which == 2) {
        uint32_t np = 0;
        cudaError_t e = cudaMemcpyAsync(&np, c->mk.npairs, 4, cudaMemcpyDeviceToHost, c->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
        if (e != cudaSuccess) return cuda_check(c, e, "pair count");
        u = (double)std::min(np, c->mk.pair_cap);
    }
    auto one = [&]() -> bool {
        if (which == 2) { launch_band_area(c->mk, c->s); return true; }
        if (which == 9) {
            double *us = scr, *vs = scr + nfx, *au = scr + nfx + nfy, *av = au + nfx;
            if (g.axisym)
                launch_predictor_axi(g.nx, g.ny, g.h, 1e-6, c->rho, c->mu, c->u, c->v, c->au, c->av,
                                     c->have_prev, 0.0, g.gy, g.frame ? c->frame : nullptr, c->bx,
                                     c->by, us, vs, au, av, c->s);
            else
                launch_predictor(g.nx, g.ny, g.h, 1e-6, c->rho, c->mu, c->u, c->v, c->au, c->av,
                                 c->have_prev, g.gx, g.gy, c->bx, c->by, us, vs, au, av, c->s);
            return true;
        }
        if (which == 10) {
            launch_spread_irrot(c->mk, c->mk.fmag, c->H, scr, scr + nfx, c->s);
            return true;
        }
        const long cells = mg_bench_op(c->mg, which, level, c->s);
        if (cells < 0) return false;
        u = (double)cells;
        return true;
    };
    if (!one()) {
        if (scr) cudaFree(scr);
        return fail(c, IB_EINVAL, "no such kernel at this level");  // warm-up
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->s);
    for (int r = 0; r < reps; r++) one();
    cudaEventRecord(e1, c->s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (scr) cudaFree(scr);
    if (e != cudaSuccess) return cuda_check(c, e, "kernel timing");
    *us_per_launch = 1e3 * ms / reps;
    if (units) *units = u;
    return IB_OK;
}

ib_status ib_mass_correct(ib_ctx *c, double *eps)
{
    if (!c) return IB_EINVAL;
    mass_correct(c, eps ? c->A0 + al((size_t)c->mk.ndrops * 8) / 8 : nullptr);
    ib_status st = launch_check(c, "mass correction");
    if (st != IB_OK || !eps) return st;
    cudaError_t e = cudaMemcpyAsync(eps, c->A0 + al((size_t)c->mk.ndrops * 8) / 8,
                                    (size_t)c->mk.ndrops * 8, cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    return cuda_check(c, e, "mass correction");
}

ib_status ib_frame_state(ib_ctx *c, double *out)
{
    if (!c || !out) return IB_EINVAL;
    if (!c->cfg.frame) return fail(c, IB_EINVAL, "no non-inertial frame");
    double f[kFrSlots];
    cudaError_t e = cudaMemcpyAsync(f, c->frame, sizeof(f), cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return cuda_check(c, e, "frame state");
    out[0] = f[kFrCom]; out[1] = f[kFrS]; out[2] = f[kFrVf]; out[3] = f[kFrWb];
    return IB_OK;
}

ib_status ib_last_solve(const ib_ctx *c, int *cycles, double *relres)
{
    if (!c) return IB_EINVAL;
    if (cycles) *cycles = c->last_cycles;
    if (relres) *relres = c->last_relres;
    return IB_OK;
}

// ------------------------------------------------------------- CNN warm start
ib_status cnn_init(ib_cnn **out, int32_t c1, int32_t c2, uint64_t seed, void *stream)
{
    if (!out) return IB_EINVAL;
    *out = nullptr;
    if (c1 != 16 || c2 != 32) return IB_EINVAL;
    cudaError_t e = cudaSuccess;
    ibk::Cnn *n = ibk::cnn_new(c1, c2, seed, (cudaStream_t)stream, &e);
    if (!n) return e == cudaErrorMemoryAllocation ? IB_ENOMEM : IB_ECUDA;
    e = ibk::cnn_pack(*n, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) { ibk::cnn_free(n); return IB_ECUDA; }
    ib_cnn *h = new ib_cnn();
    h->n = n;
    *out = h;
    return IB_OK;
}

void cnn_destroy(ib_cnn *h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    for (auto &g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (h->cap) cudaStreamDestroy(h->cap);
    ibk::cnn_free(h->n);
    delete h;
}

int64_t cnn_num_params(const ib_cnn *h) { return h ? (int64_t)ibk::cnn_nparam(*h->n) : 0; }

ib_status cnn_get_params(ib_cnn *h, float *host, int64_t n)
{
    if (!h || !host || n != (int64_t)ibk::cnn_nparam(*h->n)) return IB_EINVAL;
    cudaError_t e = cudaMemcpy(host, ibk::cnn_weights(*h->n), (size_t)n * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? IB_OK : IB_ECUDA;
}

ib_status cnn_set_params(ib_cnn *h, const float *host, int64_t n)
{
    if (!h || !host || n != (int64_t)ibk::cnn_nparam(*h->n)) return IB_EINVAL;
    cudaError_t e = cudaMemcpy(ibk::cnn_weights(*h->n), host, (size_t)n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = ibk::cnn_pack(*h->n, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    ibk::cnn_reset_adam(*h->n);
    return e == cudaSuccess ? IB_OK : IB_ECUDA;
}

static ib_status cnn_fb(ib_cnn *h, int32_t B, int32_t N, double hs, const double *rhs,
                        const double *rho, const double *p, float *loss, cudaStream_t s)
{
    if (!h || B < 1 || N < 4 || N % 4 || !(hs > 0) || !rhs || !rho || !p) return IB_EINVAL;
    cudaError_t e = ibk::cnn_workspace(*h->n, B, N);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? IB_ENOMEM : IB_ECUDA;
    ibk::cnn_forward(*h->n, B, N, hs, rhs, rho, p, s);
    ibk::cnn_backward(*h->n, B, N, s);
    if (loss) {
        std::vector<float> ls(B);
        e = cudaMemcpyAsync(ls.data(), ibk::cnn_lsum(*h->n), B * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        float t = 0.0f;
        for (float v : ls) t += v;
        *loss = t;
        int f = 0;
        if (e == cudaSuccess) e = ibk::cnn_take_fault(&f);
        if (e == cudaSuccess && f) return IB_ECUDA;  // a tensor-core completion wait ran out
    }
    return cudaGetLastError() == cudaSuccess && e == cudaSuccess ? IB_OK : IB_ECUDA;
}

ib_status cnn_grad(ib_cnn *h, int32_t B, int32_t N, double hs, const double *rhs,
                   const double *rho, const double *p, float *loss, float *grads_host,
                   void *stream)
{
    ib_status st = cnn_fb(h, B, N, hs, rhs, rho, p, loss, (cudaStream_t)stream);
    if (st != IB_OK || !grads_host) return st;
    cudaError_t e = cudaMemcpy(grads_host, ibk::cnn_grads(*h->n), ibk::cnn_nparam(*h->n) * 4,
                               cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? IB_OK : IB_ECUDA;
}

ib_status cnn_train_step(ib_cnn *h, int32_t B, int32_t N, double hs, const double *rhs,
                         const double *rho, const double *p, float lr, float *loss,
                         void *stream)
{
    ib_status st = cnn_fb(h, B, N, hs, rhs, rho, p, loss, (cudaStream_t)stream);
    if (st != IB_OK) return st;
    ibk::cnn_adam(*h->n, lr, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ECUDA;
}

ib_status cnn_fit_scale(ib_cnn *h, int32_t B, int32_t N, double hs, const double *rhs,
                        const double *p, double *c_out, void *stream)
{
    if (!h || B < 1 || N < 1 || !(hs > 0) || !rhs || !p) return IB_EINVAL;
    double c = 0.0;
    cudaError_t e = ibk::cnn_fit_scale(*h->n, B, N, hs, rhs, p, &c, (cudaStream_t)stream);
    if (e == cudaErrorInvalidValue) return IB_EINVAL;
    if (e == cudaErrorMemoryAllocation) return IB_ENOMEM;
    if (e != cudaSuccess) return IB_ECUDA;
    if (c_out) *c_out = c;
    return IB_OK;
}

ib_status cnn_train(ib_cnn *h, int32_t nsamples, int32_t N, double hs, const double *rhs,
                    const double *rho, const double *p, int32_t steps, int32_t batch, float lr0,
                    uint64_t seed, float *losses, void *stream)
{
    if (!h || nsamples < 1 || N < 4 || N % 4 || !(hs > 0) || !rhs || !rho || !p || steps < 1 ||
        batch < 1 || !(lr0 > 0.0f) || !losses)
        return IB_EINVAL;
    cudaError_t e = ibk::cnn_train_loop(*h->n, nsamples, N, hs, rhs, rho, p, steps, batch, lr0,
                                        seed, losses, (cudaStream_t)stream);
    if (e == cudaErrorInvalidValue) return IB_EINVAL;
    if (e == cudaErrorMemoryAllocation) return IB_ENOMEM;
    return e == cudaSuccess ? IB_OK : IB_ECUDA;
}

ib_status cnn_infer(ib_cnn *h, int32_t B, int32_t N, double hs, const double *rhs,
                    const double *rho, double *p0, void *stream)
{
    if (!h || B < 1 || N < 4 || N % (4 << h->coarsen) || !(hs > 0) || !rhs || !rho || !p0)
        return IB_EINVAL;
    cudaError_t e = cnn_run(h, B, N, hs, rhs, rho, p0, (cudaStream_t)stream);
    if (e == cudaErrorMemoryAllocation) return IB_ENOMEM;
    return e == cudaSuccess ? IB_OK : IB_ECUDA;
}

ib_status cnn_set_coarsen(ib_cnn *h, int32_t levels)
{
    if (!h || levels < 0 || levels > 6) return IB_EINVAL;
    h->coarsen = levels;
    return IB_OK;
}

ib_status cnn_set_tensor_path(ib_cnn *h, int32_t mode)
{
    if (!h || mode < 0 || mode > 2) return IB_EINVAL;
    ibk::cnn_set_tc(*h->n, mode);
    // recorded inference graphs hold the other path's launches
    cudaDeviceSynchronize();
    for (auto &g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
    return IB_OK;
}

ib_status cnn_set_scale(ib_cnn *h, double c)
{
    if (!h || !(c > 0)) return IB_EINVAL;
    ibk::cnn_set_scale(*h->n, c);
    return IB_OK;
}

double cnn_get_scale(const ib_cnn *h) { return h ? ibk::cnn_get_scale(*h->n) : 0.0; }

ib_status ib_attach_cnn(ib_ctx *c, ib_cnn *h)
{
    if (!c) return IB_EINVAL;
    c->cnn = h;
    return IB_OK;
}

// ------------------------------------------------------------- checkpoint
static const uint64_t kMagic = 0x31303531304249ULL;  // "IB01501"

ib_status ib_save(ib_ctx *c, const char *path)
{
    if (!c || !path) return IB_EINVAL;
    const size_t nc = (size_t)c->cfg.nx * c->cfg.ny, fx = (size_t)(c->cfg.nx + 1) * c->cfg.ny,
                 fy = (size_t)c->cfg.nx * (c->cfg.ny + 1), M = c->mk.M;
    std::vector<double> buf(3 * fx + 3 * fy + nc + 2 * M);
    double *q = buf.data();
    struct { double *d; size_t n; } parts[] = {{c->u, fx}, {c->au, fx}, {c->us, fx}, {c->v, fy},
                                               {c->av, fy}, {c->vs, fy}, {c->p, nc},
                                               {c->mk.X, M}, {c->mk.Y, M}};
    for (auto &pt : parts) {
        cudaError_t e = cudaMemcpyAsync(q, pt.d, pt.n * 8, cudaMemcpyDeviceToHost, c->s);
        if (e != cudaSuccess) return cuda_check(c, e, "save");
        q += pt.n;
    }
    cudaError_t e = cudaStreamSynchronize(c->s);
    if (e != cudaSuccess) return cuda_check(c, e, "save");
    FILE *f = fopen(path, "wb");
    if (!f) return fail(c, IB_EINVAL, "cannot open checkpoint for writing");
    int64_t hdr[6] = {(int64_t)kMagic, c->cfg.nx, c->cfg.ny, (int64_t)M, c->step, c->have_prev};
    bool ok = fwrite(hdr, sizeof(hdr), 1, f) == 1 && fwrite(buf.data(), 8, buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? IB_OK : fail(c, IB_EINVAL, "checkpoint write failed");
}

ib_status ib_load(ib_ctx *c, const char *path)
{
    if (!c || !path) return IB_EINVAL;
    const size_t nc = (size_t)c->cfg.nx * c->cfg.ny, fx = (size_t)(c->cfg.nx + 1) * c->cfg.ny,
                 fy = (size_t)c->cfg.nx * (c->cfg.ny + 1), M = c->mk.M;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(c, IB_EINVAL, "cannot open checkpoint");
    int64_t hdr[6];
    std::vector<double> buf(3 * fx + 3 * fy + nc + 2 * M);
    bool ok = fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == (int64_t)kMagic &&
              hdr[1] == c->cfg.nx && hdr[2] == c->cfg.ny && hdr[3] == (int64_t)M &&
              fread(buf.data(), 8, buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return fail(c, IB_EINVAL, "checkpoint does not match this context");
    const double *q = buf.data();
    struct { double *d; size_t n; } parts[] = {{c->u, fx}, {c->au, fx}, {c->us, fx}, {c->v, fy},
                                               {c->av, fy}, {c->vs, fy}, {c->p, nc},
                                               {c->mk.X, M}, {c->mk.Y, M}};
    for (auto &pt : parts) {
        cudaError_t e = cudaMemcpyAsync(pt.d, q, pt.n * 8, cudaMemcpyHostToDevice, c->s);
        if (e != cudaSuccess) return cuda_check(c, e, "load");
        q += pt.n;
    }
    c->step = (int)hdr[4];
    c->have_prev = (int)hdr[5];
    return cuda_check(c, cudaStreamSynchronize(c->s), "load");
}

// ------------------------------------------------------------- context-free ops
#define OPCHK(cond) do { if (!(cond)) return IB_EINVAL; } while (0)
static ib_status op_done()
{
    return cudaGetLastError() == cudaSuccess ? IB_OK : IB_ECUDA;
}

ib_status ib_op_coeffs(int32_t nx, int32_t ny, double rho_g, double rho_l, double mu_g,
                       double mu_l, const double *H, double *rho, double *mu, double *bx,
                       double *by, void *stream)
{
    OPCHK(nx > 0 && ny > 0 && H && rho && mu && bx && by);
    launch_coeffs(nx, ny, rho_g, rho_l, mu_g, mu_l, H, rho, mu, bx, by, (cudaStream_t)stream);
    return op_done();
}

ib_status ib_op_residual(int32_t nx, int32_t ny, double h, const double *bx, const double *by,
                         const double *b, const double *p, double *r, void *stream)
{
    OPCHK(nx > 0 && ny > 0 && h > 0 && bx && by && b && p && r);
    launch_residual(nx, ny, h, bx, by, b, p, r, (cudaStream_t)stream);
    return op_done();
}

ib_status ib_op_rbgs(int32_t nx, int32_t ny, double h, const double *bx, const double *by,
                     const double *b, double *p, int32_t nsweeps, void *stream)
{
    OPCHK(nx > 0 && ny > 0 && h > 0 && bx && by && b && p && nsweeps >= 0);
    // sweeps alternate between p and a scratch copy (a sweep reads its
    // neighbours' halo, so it must not write the buffer it reads)
    double *tmp = nullptr;
    const size_t bytes = (size_t)nx * ny * 8;
    if (nsweeps > 0 && cudaMalloc(&tmp, bytes) != cudaSuccess) return IB_ENOMEM;
    double *cur = p;
    for (int k = 0; k < nsweeps; k++) {
        double *nxt = cur == p ? tmp : p;
        launch_rbgs(nx, ny, h, bx, by, nullptr, b, cur, nxt, (cudaStream_t)stream);
        cur = nxt;
    }
    if (cur != p) cudaMemcpyAsync(p, cur, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (tmp) {
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaFree(tmp);
    }
    return op_done();
}

ib_status ib_op_restrict_residual(int32_t nx, int32_t ny, double h, const double *bx,
                                  const double *by, const double *b, const double *p,
                                  double *rc, void *stream)
{
    OPCHK(nx > 1 && ny > 1 && nx % 2 == 0 && ny % 2 == 0 && h > 0 && bx && by && b && p && rc);
    launch_restrict_residual(nx, ny, h, bx, by, b, p, rc, nullptr, (cudaStream_t)stream);
    return op_done();
}

ib_status ib_op_prolong_add(int32_t nxc, int32_t nyc, const double *ec, double *ef, void *stream)
{
    OPCHK(nxc > 0 && nyc > 0 && ec && ef);
    launch_prolong_add(nxc, nyc, ec, ef, (cudaStream_t)stream);
    return op_done();
}

ib_status ib_op_coarsen_beta(int32_t nx, int32_t ny, const double *bx, const double *by,
                             double *bxc, double *byc, void *stream)
{
    OPCHK(nx > 1 && ny > 1 && nx % 2 == 0 && ny % 2 == 0 && bx && by && bxc && byc);
    launch_coarsen_beta(nx, ny, bx, by, bxc, byc, (cudaStream_t)stream);
    return op_done();
}

ib_status ib_op_rhs(int32_t nx, int32_t ny, double h, double dt, const double *us,
                    const double *vs, const double *Fx, const double *Fy, const double *bx,
                    const double *by, double *b, void *stream)
{
    OPCHK(nx > 0 && ny > 0 && h > 0 && dt > 0 && us && vs && Fx && Fy && bx && by && b);
    launch_rhs(nx, ny, h, dt, us, vs, Fx, Fy, bx, by, b, (cudaStream_t)stream);
    return op_done();
}

ib_status ib_op_correct(int32_t nx, int32_t ny, double h, double dt, const double *us,
                        const double *vs, const double *p, const double *Fx, const double *Fy,
                        const double *bx, const double *by, double *u, double *v, void *stream)
{
    OPCHK(nx > 0 && ny > 0 && h > 0 && us && vs && p && Fx && Fy && bx && by && u && v);
    launch_correct(nx, ny, h, dt, us, vs, p, Fx, Fy, bx, by, u, v, (cudaStream_t)stream);
    return op_done();
}

ib_status ib_op_predictor(int32_t nx, int32_t ny, double h, double dt, const double *rho,
                          const double *mu, const double *u, const double *v,
                          const double *au_prev, const double *av_prev, int32_t have_prev,
                          double gx, double gy, double *us, double *vs, double *au, double *av,
                          void *stream)
{
    OPCHK(nx > 0 && ny > 0 && h > 0 && rho && mu && u && v && us && vs && au && av);
    OPCHK(!have_prev || (au_prev && av_prev));
    launch_predictor(nx, ny, h, dt, rho, mu, u, v, au_prev, av_prev, have_prev, gx, gy, nullptr,
                     nullptr, us, vs,
                     au, av, (cudaStream_t)stream);
    return op_done();
}

ib_status ib_op_predictor_axi(int32_t nx, int32_t ny, double h, double dt, const double *rho,
                              const double *mu, const double *u, const double *v,
                              const double *au_prev, const double *av_prev, int32_t have_prev,
                              double gy, const double *frame, double *us, double *vs, double *au,
                              double *av, void *stream)
{
    OPCHK(nx > 0 && ny > 0 && h > 0 && rho && mu && u && v && us && vs && au && av);
    OPCHK(!have_prev || (au_prev && av_prev));
    launch_predictor_axi(nx, ny, h, dt, rho, mu, u, v, au_prev, av_prev, have_prev, 0.0, gy, frame,
                         nullptr, nullptr, us, vs, au, av, (cudaStream_t)stream);
    return op_done();
}

ib_status ib_op_rhs_axi(int32_t nx, int32_t ny, double h, double dt, const double *us,
                        const double *vs, const double *Fx, const double *Fy, const double *bx,
                        const double *by, double *b, void *stream)
{
    OPCHK(nx > 0 && ny > 0 && h > 0 && dt > 0 && us && vs && Fx && Fy && bx && by && b);
    launch_rhs_axi(nx, ny, h, dt, us, vs, Fx, Fy, bx, by, b, (cudaStream_t)stream);
    return op_done();
}

ib_status ib_op_cn_solve(int32_t nx, int32_t ny, double h, double dt, const double *rho,
                         const double *mu, int32_t axisym, int32_t nsweeps, const double *ue,
                         const double *ve, double *us, double *vs, void *stream)
{
    OPCHK(nx > 0 && ny > 0 && h > 0 && dt > 0 && nsweeps >= 0 && rho && mu && ue && ve && us && vs);
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemcpyAsync(us, ue, (size_t)(nx + 1) * ny * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(vs, ve, (size_t)nx * (ny + 1) * 8, cudaMemcpyDeviceToDevice, s);
    launch_cn_solve(nx, ny, h, dt, rho, mu, axisym ? 1 : 0, nullptr, nsweeps, ue, ve, us, vs, s);
    return op_done();
}

ib_status ib_op_axi_weights(int32_t nx, int32_t ny, double h, const double *bx, const double *by,
                            double *bxa, double *bya, void *stream)
{
    OPCHK(nx > 0 && ny > 0 && h > 0 && bx && by && bxa && bya);
    launch_axi_weights(nx, ny, h, bx, by, bxa, bya, (cudaStream_t)stream);
    return op_done();
}

}  // extern "C"
