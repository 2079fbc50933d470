/*
 * ebvisc.h -- C-ABI of the GB300 (sm_103a) embedded-boundary viscoplastic
 * flow library.
 *
 * The library advances the incompressible flow of a generalised Newtonian
 * (Bingham / Herschel-Bulkley) fluid around an embedded boundary (EB) on a
 * single uniform grid with the two-stage Runge-Kutta projection method of
 * Sverdrup, Almgren & Nikiforakis, "An embedded boundary approach for efficient
 * simulations of viscoplastic fluids in three dimensions" (arXiv:1905.07392),
 * Algorithm 1.  All arithmetic runs in CUDA kernels; the host only launches
 * kernels and reads back convergence scalars.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Cells are cubes of side h; the box is lo + [0, n[d] h].  Cell arrays hold
 *    n0*n1*n2 values, x fastest, no ghost cells.  Vector cell fields hold the
 *    three components one after another (SoA, 3*n0*n1*n2).  Face arrays with
 *    normal d hold (n[d]+1) entries along d: x-faces (n0+1)*n1*n2, y-faces
 *    n0*(n1+1)*n2, z-faces n0*n1*(n2+1); a "face triple" is the three arrays
 *    concatenated in that order.  Nodal arrays (pressure) hold
 *    (n0+1)*(n1+1)*(n2+1) values, x fastest.
 *  - Field pointers are DEVICE pointers unless a name says _host.  The caller
 *    owns them; the library never frees or keeps them past the call.
 *  - The library owns its context: geometry, multigrid hierarchy and work
 *    fields, allocated by ebv_create / ebv_build_geometry only.  Stepping
 *    calls allocate nothing.
 *  - Work is queued on the context's CUDA stream.  Calls that return host
 *    values (stats, drag, dt) synchronise that stream; the solvers read one
 *    residual scalar per iteration.
 *  - Errors: every call returns an ebv_status; ebv_last_error gives a text.
 *    There is no CPU fallback: without a CUDA device ebv_create fails with
 *    EBV_ERR_CUDA.  Covered cells (volume fraction 0) read as 0 on output.
 */
#ifndef EBVISC_H
#define EBVISC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ebv_ctx ebv_ctx;

typedef enum {
    EBV_OK = 0,
    EBV_ERR_INVALID = -1,        /* bad argument, size or state */
    EBV_ERR_CUDA = -2,           /* a CUDA call failed (text in ebv_last_error) */
    EBV_ERR_NOT_CONVERGED = -3,  /* a linear solve hit max_iters above tol */
    EBV_ERR_TIMEOUT = -4,        /* a bounded wait inside a kernel gave up (ebv_set_spin_limit);
                                    the kernel let its copies in flight land and returned, the
                                    context stays usable */
    EBV_ERR_NAN = -5,            /* a residual became NaN or Inf */
    EBV_ERR_GEOMETRY = -6,       /* geometry missing or unsupported */
    EBV_ERR_TOO_LARGE = -7,      /* beyond the fixed working storage of ebv_drag_noalloc */
    EBV_ERR_OOM = -8,            /* a device allocation failed for lack of memory (or past the
                                    budget of ebv_set_alloc_limit); nothing is left allocated */
    EBV_ERR_CUDA_PENDING = -9    /* a CUDA error of earlier work was pending on entry; it is
                                    left in place for its owner (ebv_drag_noalloc) */
} ebv_status;

/* Box side types, sides ordered x-, x+, y-, y+, z-, z+. */
enum { EBV_INFLOW = 0, EBV_OUTFLOW = 1, EBV_SLIP = 2, EBV_NOSLIP = 3 };
/* Rheology (paper Table "Generalised Newtonian fluid models"). */
enum { EBV_NEWTONIAN = 0, EBV_BINGHAM = 1, EBV_HERSCHEL_BULKLEY = 2, EBV_POWER_LAW = 3,
       EBV_SOUZA_MENDES_DUTRA = 4 };
/* Precision forms; every one converges each linear solve to ebv_params.tol.
 * EBV_FP64: conjugate gradients and multigrid in FP64.  EBV_FP32_REFINE:
 * every linear solve is FP64 iterative refinement (FP64 operator, residual
 * and solution) around corrections solved by FP32 conjugate gradients with an
 * FP32 multigrid preconditioner whose cell-centred V-cycle stores its face
 * coefficients in BF16; geometry and every field FP64.  EBV_FP32_MIXED: the
 * same, and the strain rate and apparent viscosity of fluid cells away from
 * the EB (neither cut nor next to a cut cell, all six neighbours fluid) are
 * formed in FP32 from FP64 velocity differences, the near-wall ones in FP64
 * (results within about 1e-7 of FP64 rather than 1e-10; the adjoint
 * differentiates the FP64 formula). */
enum { EBV_FP64 = 0, EBV_FP32_REFINE = 1, EBV_FP32_MIXED = 2 };

typedef struct {
    int n[3];        /* cells per direction; each even down to the multigrid bottom */
    double lo[3];    /* low corner of the box */
    double h;        /* cell size */
    int bc[6];       /* EBV_INFLOW / OUTFLOW / SLIP / NOSLIP per side */
    double u_in[3];  /* inflow velocity (used on EBV_INFLOW sides) */
} ebv_grid;

typedef struct {
    double rho;       /* density */
    double mu;        /* plastic viscosity (Bingham) or consistency kappa (HB, power law) */
    double tau0;      /* yield stress */
    double m;         /* Papanastasiou parameter 1/epsilon; also floors ||gamma|| at 1/m for n < 1 */
    double n_flow;    /* flow index n (HB, power law, SMD) */
    double eta0;      /* zero-shear viscosity (Souza Mendes-Dutra) */
    int model;        /* EBV_NEWTONIAN ... */
    double cfl;       /* C_CFL of Eq. cfl:dt */
    double bi_cfl;    /* Bingham number in the viscous limit, Eq. cfl:viscous:new */
    double tol;       /* relative residual of every linear solve */
    int max_iters;    /* Krylov iterations per solve */
    double delta_min; /* lower bound (cell units) of the wall distance in the implicit EB flux:
                         a cell centre behind the EB plane counts as this close to the wall
                         (0.01 in the bindings; larger values under-enforce no-slip in small
                         cut cells and raise the drag) */
    int precision;    /* EBV_FP64, EBV_FP32_REFINE or EBV_FP32_MIXED */
    int advect;       /* 1: Algorithm 1 as printed; 0: creeping flow, the convective term C = 0
                         (the paper's evaluation runs at Re = 1e-3, Sec. "Cylinder moving through
                         Bingham fluid"); the adjoint (ebv_adjoint_step) follows either */
} ebv_params;

typedef struct {
    double dt;          /* time step used */
    double drag;        /* z-force on the body at the end of the step (Eq. drag-force) */
    double yield_frac;  /* fluid volume fraction with ||tau|| <= (1 + 1e-3) tau0 */
    int iters[10];      /* Krylov iterations: MAC, visc x3, nodal (predictor); same (corrector) */
    double res[10];     /* final relative residuals, same order */
    double div_rel;     /* largest relative divergence the step's four projections leave: the
                           cell-centred ones' ||D u^F|| / ||D u~^F|| and the nodal ones' relative
                           residual (the projection is approximate) */
    float ms[8];        /* GPU time of the step's phases (ebv_advance only; 0 from the graph
                           forms): time step, predictor derived quantities (Algorithm 2),
                           predictor viscous solves, predictor projection, the same three for
                           the corrector, drag.  The phases are also NVTX ranges. */
} ebv_step_stats;

/* Implicit function of the body: > 0 in the fluid, <= 0 in the body. */
typedef double (*ebv_implicit_fn)(const double x[3], void *user);

/* Create a context on the current CUDA device, queueing work on `stream`
 * (a cudaStream_t, NULL for the legacy default stream).  Allocates the work
 * fields and multigrid hierarchy.  EBV_ERR_INVALID if a size is not
 * coarsenable (see ebv_grid.n) or a parameter is out of range. */
ebv_status ebv_create(const ebv_grid *grid, const ebv_params *params, void *stream,
                      ebv_ctx **out);
/* Replace the parameters (rheology, tolerances, precision); no allocation. */
ebv_status ebv_set_params(ebv_ctx *ctx, const ebv_params *params);

/* EB geometry from an implicit function (paper Sec. "Embedded boundaries"):
 * planar cut per cell, face apertures, volume fraction, EB area, unit normal
 * into the fluid and EB centroid.  Evaluated on the host (the callback is a
 * host function), uploaded once; builds the geometry-only solver data. */
ebv_status ebv_build_geometry(ebv_ctx *ctx, ebv_implicit_fn fn, void *user);
/* The same for a sphere of centre c and radius r (fluid outside). */
ebv_status ebv_build_geometry_sphere(ebv_ctx *ctx, const double c[3], double r);
/* The same for a half-space n.x > d (tests of planar cuts). */
ebv_status ebv_build_geometry_plane(ebv_ctx *ctx, const double nrm[3], double d);
/* Bodies for the device-side geometry builders: the fluid is outside every
 * body (their union is the EB).  q holds, per kind:
 *   EBV_BODY_SPHERE    centre x, y, z and radius;
 *   EBV_BODY_BOX       low corner x, y, z and high corner x, y, z (axis-aligned);
 *   EBV_BODY_CYLINDER  axis (0, 1 or 2), the centre's two other coordinates in
 *                      axis order after it ((axis+1) % 3, (axis+2) % 3), radius
 *                      (infinite along the axis). */
enum { EBV_BODY_SPHERE = 0, EBV_BODY_BOX = 1, EBV_BODY_CYLINDER = 2 };
typedef struct {
    int kind;
    double q[6];
} ebv_body;
/* The geometry of ebv_build_geometry for n spheres (c_r: n rows cx, cy, cz,
 * r in host memory), computed on the device (the same planar-cut steps, run
 * by GPU threads per node, edge, face and cell) -- the fast path for large
 * grids.  Agrees with the host builder to rounding.  n in [1, 16]. */
ebv_status ebv_build_geometry_spheres(ebv_ctx *ctx, int n, const double *c_r);
/* The same for any union of up to 16 bodies (host array), e.g. the paper's
 * sphere-and-cube body (Sec. "Non-trivial particle shape") or its cylinder
 * (Sec. "Cylinder moving through Bingham fluid"). */
ebv_status ebv_build_geometry_bodies(ebv_ctx *ctx, int n, const ebv_body *bodies);
/* Copy the geometry out (device pointers, any may be NULL):
 * alpha, area (cells), ax/ay/az (faces), nrm/bcen (3 x cells; bcen relative
 * to the cell centre in units of h), flag (cells: 0 covered, 1 regular, 2 cut). */
ebv_status ebv_get_geometry(ebv_ctx *ctx, double *alpha, double *ax, double *ay, double *az,
                            double *area, double *nrm, double *bcen, unsigned char *flag);

/* Resumable state (checkpoint / restart of a run of Algorithm 1).
 * ebv_save_state writes the grid, the parameters, the geometry and the
 * fields u (3 x cells) and p (nodes) -- device pointers, unchanged -- to the
 * file at `path` (host byte order; a file of this library version).
 * ebv_load_state reads such a file into a context created on the same grid:
 * it replaces the parameters and the geometry (and rebuilds the solver data
 * from them, allocating as a geometry build does) and writes u and p (device).
 * Steps taken from a loaded state are bit for bit those the saving run would
 * have taken.  EBV_ERR_INVALID for an unreadable or foreign file or another
 * grid; EBV_ERR_GEOMETRY if no geometry was built (save). */
ebv_status ebv_save_state(ebv_ctx *ctx, const double *u, const double *p, const char *path);
ebv_status ebv_load_state(ebv_ctx *ctx, double *u, double *p, const char *path);

/* Fused strain rate and apparent viscosity (paper Sec. "Strain rate tensor and
 * apparent viscosity", Table of rheologies): central differences, one-sided
 * quadratic differences next to covered cells; ||gamma|| = sqrt(tr(g g^T)/2).
 * u: 3 x cells; eta: cells; srate: cells or NULL. */
ebv_status ebv_update_viscosity(ebv_ctx *ctx, const double *u, double *eta, double *srate);

/* Flow diagnostics of the paper's cylinder and sphere studies (Sec. "Cylinder
 * moving through Bingham fluid"): per cell the flow topology parameter of
 * Eq. ryovar, lambda = (||g||^2 - |w|^2) / (||g||^2 + |w|^2) with w = curl u
 * (-1 rigid rotation, 0 shear, 1 extension; 0 where both vanish), and the
 * relative deviation from the yield stress, stress_dev = eta ||g|| / tau0 - 1
 * (negative where unyielded; 0 when tau0 = 0).  Gradients as in
 * ebv_update_viscosity.  u: 3 x cells; lambda, stress_dev: cells (device). */
ebv_status ebv_flow_diagnostics(ebv_ctx *ctx, const double *u, double *lambda, double *stress_dev);

/* Derived quantities of Algorithm 2 for a velocity u: convective term C,
 * apparent viscosity eta and explicit viscous term V (3 x cells, cells,
 * 3 x cells).  Runs the cell-centred projection internally; iters/res of that
 * solve are written when the pointers are not NULL (host). */
ebv_status ebv_derived(ebv_ctx *ctx, const double *u, double *C, double *eta, double *V,
                       int *iters, double *res);

/* Slope-limited, upwinded normal face velocities of u (Algorithm 2, lines
 * 2-3), written as a face triple. */
ebv_status ebv_face_states(ebv_ctx *ctx, const double *u, double *uf);
/* Cell-centred projection (Eq. helmholtz and the Poisson equation after it):
 * uf (face triple) is made discretely divergence free in place; phi (cells)
 * receives the potential. */
ebv_status ebv_solve_mac(ebv_ctx *ctx, double *uf, double *phi, int *iters, double *res);
/* Semi-implicit viscous update (Eq. implicit-viscous) for the three
 * components: (rho - dt div(eta grad)) ut = psi with the EB no-slip wall.
 * eta: cells; psi, ut: 3 x cells.  stats->iters[1..3], res[1..3] if stats. */
ebv_status ebv_solve_viscous(ebv_ctx *ctx, const double *eta, const double *psi, double dt,
                             double *ut, ebv_step_stats *stats);
/* Nodal projection (paper Sec. "Incompressibility constraint"): adds
 * (dt/rho) grad p to ut, solves div((dt/rho) grad p_new) = div ut for nodal
 * p_new, and writes ut -= (dt/rho) grad p_new.  ut: 3 x cells (in/out);
 * p: nodes (in: old pressure, out: new).  stats->iters[4], res[4] if stats. */
ebv_status ebv_solve_projection(ebv_ctx *ctx, double *ut, double *p, double dt,
                                ebv_step_stats *stats);
/* Time step of Eqs. cfl:dt .. cfl:viscous:new for velocity u and force f
 * (3 x cells or NULL); result on the host. */
ebv_status ebv_timestep(ebv_ctx *ctx, const double *u, const double *f, double *dt_host);
/* One step of Algorithm 1 in place: u (3 x cells), p (nodes).  dt <= 0 takes
 * the CFL step.  f: body force 3 x cells or NULL.  stats (host) or NULL. */
ebv_status ebv_advance(ebv_ctx *ctx, double *u, double *p, double dt, const double *f,
                       ebv_step_stats *stats);
/* `steps` steps of Algorithm 1 in place, as ebv_advance, from one captured
 * CUDA graph per (u, p, dt, f): every solver loop of the step is a
 * conditional WHILE node whose condition a device kernel sets, so each step
 * is one graph launch with no host synchronisation inside it.  The graph is
 * captured on the first call (and again when u, p, dt, f, the parameters or
 * the geometry change); the call synchronises once at the end.  A failed
 * solve in any step gives EBV_ERR_NAN / EBV_ERR_NOT_CONVERGED (the failing
 * solve slot is named in ebv_last_error); the steps after it still ran.
 * stats (host, or NULL): the last step's iterations, residuals, dt, drag. */
ebv_status ebv_advance_graph(ebv_ctx *ctx, double *u, double *p, double dt, const double *f, int steps,
                             ebv_step_stats *stats);
/* `steps` steps from HOST buffers: copies u_host, p_host to the device, runs
 * the steps (as ebv_advance_graph), copies the result back.  Uses the
 * context's own device copies. */
ebv_status ebv_advance_host(ebv_ctx *ctx, double *u_host, double *p_host, int steps, double dt,
                            ebv_step_stats *last);
/* Drag F_z on the body (Eq. drag-force, surface normal into the fluid) and the
 * unyielded fluid volume fraction (||tau|| <= (1 + 1e-3) tau0), host outputs. */
ebv_status ebv_drag(ebv_ctx *ctx, const double *u, const double *p, double *fz_host,
                    double *yield_frac_host);

/* The drag and unyielded fraction of ebv_drag for callers that cannot allocate
 * GPU memory (they run inside a memory pool they do not own, must not grow
 * device memory after start-up, or may only touch the buffers they are given).
 * The paper has no counterpart: this is a deployment variant, not a step of
 * the method.  It needs no context: the caller passes the grid and parameters,
 * the geometry as returned by ebv_get_geometry (alpha, area, nrm, bcen, flag),
 * the ascending list `cut` of the ncut cells with flag 2, the fields u and p,
 * and `out` (2 doubles: F_z, unyielded fraction) -- all device pointers -- and
 * a cudaStream_t (NULL: legacy default stream).  Nothing is allocated; the
 * working storage is a fixed array of about 6.3 MB that every GPU loading the
 * library holds until the process exits, so grids of more than 262,144 cells
 * (e.g. 64^3) or more than 65,536 cut cells return EBV_ERR_TOO_LARGE.  The
 * first call on each device looks up that array's device address (with the
 * device current); make that first call before any stream capture.  All calls
 * share the one array and every call writes what it reads, so nothing carries
 * over between calls, but calls whose work overlaps on the GPU (other streams,
 * other threads) race on it and must be serialised by the caller.  Work is
 * queued asynchronously on `stream`; `out` is valid once it completes.
 * The device address is looked up once per device and kept for the life of
 * the process: after a cudaDeviceReset the array may move, so a process that
 * resets a device must not call this entry again (restart the process).
 * The C side cannot see buffer sizes: the caller guarantees that u holds
 * 3 x cells, p the nodes, and every entry of `cut` lies in [0, cells) (an
 * entry outside is skipped).  EBV_ERR_INVALID for a NULL pointer, a
 * non-positive size or h <= 0; EBV_ERR_CUDA_PENDING if an error of earlier
 * work was pending on entry (nothing is queued then). */
ebv_status ebv_drag_noalloc(const ebv_grid *grid, const ebv_params *params, const double *alpha,
                            const double *area, const double *nrm, const double *bcen,
                            const unsigned char *flag, const int *cut, int ncut, const double *u,
                            const double *p, double *out, void *stream);

/* Fault injection on the host, for tests of the out-of-memory path: device
 * allocations the library makes after this call fail as out-of-memory once
 * they total more than `bytes` (the call that fails reports EBV_ERR_OOM and
 * frees what it took); bytes < 0 removes the limit.  Process-wide; the
 * device is never actually exhausted. */
void ebv_set_alloc_limit(long long bytes);

/* The smoother's waits on its asynchronous (TMA) tile loads are bounded:
 * one wait gives up after `cycles` cycles of the SM clock (default about one
 * second: cycles < 0 restores it), and the solve then ends with
 * EBV_ERR_TIMEOUT.  cycles = 0 makes every such wait give up at once, which
 * exercises that path without any fault or hang (for tests).  Process-wide;
 * read when a step is issued or captured. */
void ebv_set_spin_limit(long long cycles);

/* How FP32 multigrid levels whose x size is a multiple of 16 run a red-black
 * sweep: 0 as two colour passes, 1 (default) as whichever of the two colour
 * passes and the fused one-pass sweep was faster when the context's solvers
 * were set up (instances of an ebv_batch keep the colour passes: their steps
 * run side by side, where a lone kernel's time does not decide), 2 always as
 * the fused sweep.  All give the same results bit
 * for bit; the switch exists to show that and to measure the difference.
 * Process-wide; read when a step is issued or captured. */
void ebv_set_fused_sweep(int mode);

/* EBV_FP32_REFINE / EBV_FP32_MIXED: the factor by which each FP32 correction
 * solve of the iterative refinement reduces its residual before the FP64
 * residual is formed again (default 1e-4; the last correction of a solve aims
 * only for what the tolerance still needs).  Values outside (0, 1) restore
 * the default.  Changes the number of corrections and inner iterations, not
 * the tolerance the solves meet.  Process-wide; read when a step is issued or
 * captured. */
void ebv_set_inner_drop(double drop);

/* Measurement hook: the times (ms, four launches each) that chose the form
 * of one kind of red-black sweep on level `level` of the MAC hierarchy when
 * the context's solvers were set up (ebv_set_fused_sweep mode 1): kind 0 the
 * sweep from zero, 1 the plain sweep, 2 the sweep after the coarse
 * correction, 3 the sweep that also forms the r.z partials; *fused_ms the
 * one-pass sweep, *passes_ms its two colour passes.  A form that was not
 * timed (the level does not fuse, an FP64 context, no correction on the
 * coarsest level, a batch instance) reads 1e30 and 0.  EBV_ERR_INVALID for a
 * null argument or a level or kind out of range; the values are only
 * meaningful after the first step. */
ebv_status ebv_sweep_timing(const ebv_ctx *ctx, int level, int kind, float *fused_ms, float *passes_ms);

/* Counters for the measurement harness: kernel launches queued since the
 * context was created (host counter). */
long long ebv_launch_count(const ebv_ctx *ctx);

/* Measurement hook, no part of the method: between begin and end every kernel
 * launch of the context is bracketed by two CUDA events on its stream.
 * ebv_profile_end synchronises, aggregates per kernel name and returns the
 * number of entries; ebv_profile_entry(i) gives an entry's name (static
 * string), launch count, summed kernel time in ms and summed algorithmic bytes
 * (the data the method must move, stated for the kernels whose roofline is
 * reported; 0 for the others). */
ebv_status ebv_profile_begin(ebv_ctx *ctx);
ebv_status ebv_profile_end(ebv_ctx *ctx, int *entries);
ebv_status ebv_profile_entry(ebv_ctx *ctx, int i, const char **name, long long *launches,
                             double *ms, double *bytes);
const char *ebv_last_error(const ebv_ctx *ctx);
void ebv_destroy(ebv_ctx *ctx);

/* ---- Adjoint (drag sensitivities) ----------------------------------------
 * Reverse mode of the step of Algorithm 1 at a fixed dt, in the form the
 * context's `advect` selects (1: with the convective term; 0: creeping flow,
 * as in the paper's evaluation at Re = 1e-3, Sec. "Cylinder moving through
 * Bingham fluid"), for the sensitivities of the drag of Eq. drag-force to the
 * yield stress tau0, the plastic viscosity mu and a per-cell body force f:
 * hand-written adjoints of the limited slopes, upwinded face states, MAC
 * projection and convective fluxes, of the strain-rate/viscosity update, the
 * explicit viscous term (face fluxes, EB wall flux of Eq. dudn,
 * redistribution), the eta-dependence of the semi-implicit viscous operator,
 * the nodal projection and the drag; the adjoint solves reuse the
 * (symmetric) projection, viscous and nodal multigrid-CG solves in the
 * context's precision.  The limiter and the upwinding are piecewise linear:
 * the reverse pass takes the branch the forward took.  Rheologies: Newtonian, Bingham,
 * Herschel-Bulkley, power law.  dt, which Eq. cfl:dt ties to u and f, is a
 * fixed input (its own sensitivity is not propagated).  The first adjoint
 * call allocates the context's adjoint workspace (about 150 doubles per
 * cell); forward steps never allocate.  EBV_ERR_INVALID if dt <= 0 or the
 * rheology has no adjoint.
 *
 * One step: given the state (u, p) at the step's start (device, unchanged),
 * dt and f (3 x cells or NULL), and in u_bar, p_bar the adjoints of the
 * step's outputs, overwrites u_bar, p_bar with the adjoints of its inputs,
 * adds the adjoint of f to f_bar (3 x cells, device, or NULL) and adds
 * dJ/dtau0, dJ/dmu of this step to grads[0], grads[1] (host). */
ebv_status ebv_adjoint_step(ebv_ctx *ctx, const double *u, const double *p, double dt, const double *f,
                            double *u_bar, double *p_bar, double *f_bar, double *grads);
/* Adds w times the gradient of the drag F_z(u, p) (eta from u) to u_bar,
 * p_bar (device) and its tau0, mu parts to grads[0..1] (host). */
ebv_status ebv_drag_adjoint(ebv_ctx *ctx, const double *u, const double *p, double w, double *u_bar,
                            double *p_bar, double *grads);
/* Doubles of device workspace ebv_drag_gradient needs for (steps, every). */
ebv_status ebv_drag_gradient_workspace(const ebv_ctx *ctx, int steps, int every, long long *ndoubles);
/* J = (1/steps) sum_{s=1..steps} F_z(u_s, p_s) over `steps` steps from (u0, p0) (device, unchanged) at fixed dt with body force f
 * (3 x cells or NULL), and its gradient: grads[0] = dJ/dtau0, grads[1] =
 * dJ/dmu (host), f_bar = dJ/df (3 x cells, device, or NULL).  Stores (u, p)
 * every `every` steps in `work` (device, ebv_drag_gradient_workspace doubles)
 * and recomputes each segment's states before reversing it. */
ebv_status ebv_drag_gradient(ebv_ctx *ctx, const double *u0, const double *p0, const double *f, double dt,
                             int steps, int every, double *work, double *J, double *grads, double *f_bar);

/* ---- Batches ------------------------------------------------------------
 * A parameter sweep of independent problems (the paper computes drag
 * coefficients over a range of Bingham numbers, Sec. "Evaluation", flows past
 * a cylinder and a sphere; running many such problems at once is this
 * library's own deployment form, not a step of the method).  Instance i has
 * its own grid, parameters, geometry, work fields and hierarchies, exactly as
 * a context from ebv_create; every step of all instances is ONE launch of a
 * graph that forks into one branch per instance (each branch the instance's
 * captured step, its solver loops conditional nodes of its own), so
 * instances converge independently while their kernels share the GPU. */
typedef struct ebv_batch ebv_batch;
/* n instances: grids[i], params[i]; work queued on `stream` (cudaStream_t).
 * Allocates everything up front; errors as ebv_create (first failing one). */
ebv_status ebv_batch_create(int n, const ebv_grid *grids, const ebv_params *params, void *stream,
                            ebv_batch **out);
/* Sphere geometry per instance: c_r holds n rows (cx, cy, cz, r), host
 * memory.  The host builders run in parallel threads; then each instance's
 * hierarchies are set up and its smoother launch shapes autotuned. */
ebv_status ebv_batch_build_spheres(ebv_batch *batch, const double *c_r);
/* Instance i's context (owned by the batch: do not destroy), NULL if out of
 * range; any single-context call may be made on it between batch steps. */
ebv_ctx *ebv_batch_instance(ebv_batch *batch, int i);
/* `steps` CFL steps of every instance: u[i] (3 x cells) and p[i] (nodes) are
 * device pointers (host arrays of n pointers), updated in place.  The graph
 * is captured on the first call and again when a pointer changes; one
 * synchronisation at the end.  A failed solve gives the status of the first
 * failing instance (named in ebv_batch_last_error).  stats: n entries (host)
 * for the last step, or NULL. */
ebv_status ebv_batch_advance(ebv_batch *batch, double *const *u, double *const *p, int steps,
                             ebv_step_stats *stats);
/* Sum of the instances' kernel launch counters (see ebv_launch_count). */
long long ebv_batch_launch_count(const ebv_batch *batch);
const char *ebv_batch_last_error(const ebv_batch *batch);
/* Destroys the instances and the batch graph. */
void ebv_batch_destroy(ebv_batch *batch);

#ifdef __cplusplus
}
#endif
#endif
