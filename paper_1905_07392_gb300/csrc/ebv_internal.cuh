// Internal declarations of the sm_103a library behind include/ebvisc.h.
//
// Data layout (device, all no-ghost, x fastest):
//   cell arrays n0*n1*n2; x-faces (n0+1)*n1*n2; y-faces n0*(n1+1)*n2;
//   z-faces n0*n1*(n2+1); nodes (n0+1)*(n1+1)*(n2+1).
// Cell availability for stencils is "inside the box and flag != 0".
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "ebvisc.h"

namespace ebv {

constexpr int kMaxLevels = 16;
constexpr int kBottomMax = 512;      // largest dense bottom system (unknowns)
constexpr int kReduceBlocks = 1216;  // 8 per SM on 152 SMs; fixed for determinism
constexpr int kSolveSlots = 16;       // solve statistics slots (10 per step)
// sstat: [3 s] iterations, [3 s + 1] relative residual, [3 s + 2] outer passes
// of the last solve in slot s; from kSstatAcc: per slot, running sums of
// iterations and of outer-body passes (launch accounting of captured steps).
constexpr int kSstatAcc = 3 * kSolveSlots;
constexpr int kSstatLen = kSstatAcc + 2 * kSolveSlots;
// control words: loop conditions, iteration counters, error words
enum { C_COND_OUT = 0, C_COND_IN = 1, C_IT = 2, C_K = 3, C_NOUT = 4, C_STALL = 5, C_ERR = 6, C_ZERO = 7,
       C_STEPERR = 8, C_LEN = 16 };
enum { E_NAN = 1, E_NOTCONV = 2, E_TIMEOUT = 3, E_SMEM = 4 };

struct GridD {
    int nx, ny, nz;
    double h;
    double ih;   // 1 / h, so kernels multiply instead of dividing in FP64
    double lo[3];
    int bc[6];
    double u_in[3];
};

// A box with no outflow side (velocity prescribed or walls all round: the
// paper's cylinder and sphere runs with U on every boundary, the Taylor-Green
// vortex between slip walls) leaves both pressure problems pure Neumann,
// fixed only up to a constant.  One Dirichlet point fixes them: the x- face
// of cell (0,0,0) acts as an outflow face (phi = 0 beyond it) in the
// cell-centred projection, and node (0,0,0) is a Dirichlet node (p = 0) in
// the nodal one.  With a consistent right-hand side (zero net boundary flux)
// the solution is the pure-Neumann one that vanishes at that point.  Every
// level of a hierarchy carries the box sides, so the rule holds on each.
__host__ __device__ inline bool no_outflow(const GridD &g)
{
    for (int s = 0; s < 6; s++)
        if (g.bc[s] == EBV_OUTFLOW) return false;
    return true;
}
__host__ __device__ inline bool pin_face(const GridD &g, int d, int i, int j, int k)
{
    return d == 0 && i == 0 && j == 0 && k == 0 && no_outflow(g);
}
__host__ __device__ inline bool pin_node(const GridD &g, int i, int j, int k)
{
    return i == 0 && j == 0 && k == 0 && no_outflow(g);
}

struct GeomD {
    const double *alpha, *ax, *ay, *az, *area, *nrm, *bcen;
    const uint8_t *flag;
    const int *cut;   // linear indices of cut cells with EB area > 0
    int ncut;
    int ncell;
};

struct ParamsD {
    double rho, mu, tau0, m, n_flow, eta0;
    int model;
    double delta_min;
    double inv_m;  // 1/m (the floor of the strain rate in the power laws)
};

__host__ __device__ inline int cidx(const GridD &g, int i, int j, int k)
{
    return (k * g.ny + j) * g.nx + i;
}
__host__ __device__ inline int nidx(const GridD &g, int i, int j, int k)
{
    return (k * (g.ny + 1) + j) * (g.nx + 1) + i;
}
// Face with normal d whose low corner has integer position (i,j,k).
__host__ __device__ inline int fidx(const GridD &g, int d, int i, int j, int k)
{
    if (d == 0) return (k * g.ny + j) * (g.nx + 1) + i;
    if (d == 1) return (k * (g.ny + 1) + j) * g.nx + i;
    return (k * g.ny + j) * g.nx + i;
}
__host__ __device__ inline int nface(const GridD &g, int d)
{
    return (g.nx + (d == 0)) * (g.ny + (d == 1)) * (g.nz + (d == 2));
}
__host__ __device__ inline int ncell(const GridD &g) { return g.nx * g.ny * g.nz; }
__host__ __device__ inline int nnode(const GridD &g) { return (g.nx + 1) * (g.ny + 1) * (g.nz + 1); }
__host__ __device__ inline int dimn(const GridD &g, int d) { return d == 0 ? g.nx : (d == 1 ? g.ny : g.nz); }

__device__ inline bool inbox(const GridD &g, int i, int j, int k)
{
    return (unsigned)i < (unsigned)g.nx && (unsigned)j < (unsigned)g.ny && (unsigned)k < (unsigned)g.nz;
}
__device__ inline bool avail(const GridD &g, const uint8_t *flag, int i, int j, int k)
{
    return inbox(g, i, j, k) && flag[cidx(g, i, j, k)] != 0;
}

// Dirichlet value of velocity component `comp` on box side `side`; false for Neumann.
__host__ __device__ inline bool side_dirichlet(const GridD &g, int side, int comp, double *val)
{
    int d = side >> 1;
    switch (g.bc[side]) {
    case EBV_INFLOW: *val = g.u_in[comp]; return true;
    case EBV_NOSLIP: *val = 0.0; return true;
    case EBV_SLIP: *val = 0.0; return comp == d;
    default: *val = 0.0; return false;
    }
}

// The device-side time step: dt and the scalars every cell would otherwise
// derive from it with an FP64 division, computed once where dt is set.
enum { DT_DT = 0, DT_DT_RHO = 1, DT_RHO_DT = 2, DT_DTH2 = 3, DT_NSCALAR = 4 };
__device__ inline void store_dt(double *d, double dt, double rho, double h)
{
    d[DT_DT] = dt;
    d[DT_DT_RHO] = dt / rho;
    d[DT_RHO_DT] = rho / dt;
    d[DT_DTH2] = dt / (h * h);
}

// Apparent viscosity of the rheology table at strain rate sr, given its
// reciprocal rsr (the laws take their sr -> 0 limits at sr = 0).
__device__ inline double eta_of(const ParamsD &p, double sr, double rsr)
{
    // (1 - exp(-m sr)) / sr; once m sr > 40, exp(-m sr) < 2^-57 and
    // -expm1(-m sr) rounds to 1 exactly, so the exponential is skipped.
    const double msr = p.m * sr;
    double yield = (sr > 0.0) ? (msr > 40.0 ? 1.0 : -expm1(-msr)) * rsr : p.m;
    double srf = sr > p.inv_m ? sr : p.inv_m;
    switch (p.model) {
    case EBV_NEWTONIAN: return p.mu;
    case EBV_BINGHAM: return p.mu + p.tau0 * yield;
    case EBV_HERSCHEL_BULKLEY: return p.mu * pow(srf, p.n_flow - 1.0) + p.tau0 * yield;
    case EBV_POWER_LAW: return p.mu * pow(srf, p.n_flow - 1.0);
    case EBV_SOUZA_MENDES_DUTRA: {
        double y2 = (sr > 0.0) ? -expm1(-p.eta0 * sr / p.tau0) * rsr : p.eta0 / p.tau0;
        return p.mu * pow(srf, p.n_flow - 1.0) + p.tau0 * y2;
    }
    }
    return p.mu;
}

inline dim3 block3() { return dim3(32, 4, 2); }
inline dim3 grid3(int nx, int ny, int nz) { return dim3((nx + 31) / 32, (ny + 3) / 4, (nz + 1) / 2); }

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

struct CcLevel {
    GridD g;            // dims and h of this level (bc shared)
    double *extra_d = nullptr, *diag_d = nullptr, *bf_d[3] = {nullptr, nullptr, nullptr};
    float *extra_f = nullptr, *bf_f[3] = {nullptr, nullptr, nullptr};
    // FP32 multigrid: the V-cycle operator has BF16 face coefficients (bf_h,
    // rounded from bf_f) and the diagonal diag_f formed from those rounded
    // faces; the level-0 Krylov operator keeps the FP32 faces with diag_a.
    float *diag_f = nullptr, *diag_a = nullptr;
    float *dinv_f = nullptr;   // 1/diag_f (0 where diag_f <= 0), the smoother's multiplier
    __nv_bfloat16 *bf_h[3] = {nullptr, nullptr, nullptr};
    uint8_t *cov = nullptr;  // 1 where the cell is covered (identity row)
    void *bxp = nullptr;     // padded x faces of the fused sweep (V-cycle face type), or none
    // per kind of sweep (from zero, plain, after the coarse correction, with
    // r.z): the times of the fused sweep [0] and of its colour passes [1],
    // measured when the solvers are set up (fused never chosen if untimed)
    float rb_ms[4][2] = {{1e30f, 0.f}, {1e30f, 0.f}, {1e30f, 0.f}, {1e30f, 0.f}};
    int rb_kz = 0;           // its planes per block (timed), 0 for the model's choice
    dim3 gs_blk = dim3(32, 4, 2);  // colour-pass block shape (autotuned per level)
    dim3 gs4_blk = dim3(32, 4, 2); // the same for the vectorised FP32 pass
    int gs4_pz = 2;                // its planes per thread (1 or 2, autotuned)
};

struct CcHier {
    int L = 0;                 // number of levels (level L-1 is the bottom)
    CcLevel lv[kMaxLevels];
    double *binv = nullptr;    // bottom inverse of the selected variant, nb x nb
    double *bmat = nullptr;    // scratch for the bottom factorisations, nvar x nb x 2nb
    int nb = 0;
    // Variants of one operator that differ only in which box faces enter the
    // diagonal (the three velocity components of the viscous solve: a slip
    // wall is a Dirichlet side for the normal component only).  A box face
    // couples no two cells, so extra and the face arrays are shared; each
    // variant has its own diagonals and bottom inverse, and select_variant()
    // points lv[].diag_d / diag_f and binv at those of one variant.
    int nvar = 1;
    unsigned side_mask[3] = {0x3fu, 0x3fu, 0x3fu};  // bit s: box side s enters the diagonal
    double *vdiag_d[3][kMaxLevels] = {};
    float *vdiag_f[3][kMaxLevels] = {};
    float *vdinv_f[3][kMaxLevels] = {};
    float *vdiag_a[3] = {};   // level 0, FP32 Krylov operator
    double *vbinv[3] = {};
};

inline void select_variant(CcHier &H, int q)
{
    for (int l = 0; l < H.L; l++) {
        H.lv[l].diag_d = H.vdiag_d[q][l];
        H.lv[l].diag_f = H.vdiag_f[q][l];
        H.lv[l].dinv_f = H.vdinv_f[q][l];
    }
    H.lv[0].diag_a = H.vdiag_a[q];
    H.binv = H.vbinv[q];
}

struct NdLevel {
    GridD g;                     // cell dims of this level
    double *alpha_d = nullptr;   // cell volume fractions at this level
    float *alpha_f = nullptr;
    uint8_t *act = nullptr;      // 1 for active nodes
    uint8_t *reg = nullptr;      // 1 where all 8 cells around the node are full (levels that
                                 // take the plane march, else null)
    int *irr = nullptr;          // with reg: the active nodes that are not regular, ascending
    int nirr = 0;
    double lam_max = 2.0;        // bound of the spectrum of D^-1 A
    dim3 ch_blk = dim3(32, 4, 2);  // Chebyshev-step block shape (autotuned per level)
};

struct NdHier {
    int L = 0;
    NdLevel lv[kMaxLevels];
    double *binv = nullptr;      // bottom inverse for the unit-coefficient operator
    double *bmat = nullptr;
    int nb = 0;
};

// Measurement hook (ebv_profile_begin/end): while on, every launch is
// bracketed by two CUDA events on the context stream and keyed by kernel name.
struct ProfEvents {
    std::vector<cudaEvent_t> ev;   // pairs (start, stop)
    std::vector<int> key;          // kernel name index of each pair
    std::vector<double> bytes;     // algorithmic bytes of each pair (0: not stated)
    std::vector<const char *> names;
    size_t used = 0;
    // aggregated by ebv_profile_end
    std::vector<long long> agg_launches;
    std::vector<double> agg_ms, agg_bytes;
};

struct Ctx {
    GridD g;
    ebv_params prm;
    cudaStream_t stream = nullptr;
    std::string err;
    long long launches = 0;
    int device = 0;
    bool prof_on = false;
    ProfEvents prof;

    bool have_geom = false;
    // an instance of a batch: its steps run beside the other instances', so
    // the smoother keeps the colour passes in switch mode 1 (the fused sweep
    // wins a lone timing on small grids but takes two blocks' shared memory
    // per SM; the batch measured 7 % slower with it)
    bool batched = false;
    // geometry (device)
    double *alpha = nullptr, *ax = nullptr, *ay = nullptr, *az = nullptr, *area = nullptr;
    double *nrm = nullptr, *bcen = nullptr;
    uint8_t *flag = nullptr;
    int *cut = nullptr;
    int ncut = 0;
    uint8_t *nearm = nullptr;    // 1 for fluid cells that are cut or have a cut neighbour
    int *nearl = nullptr;        // those cells, ascending
    int nnear = 0;

    // work fields (device)
    double *Cm = nullptr, *Vm = nullptr, *Cs = nullptr, *Vs = nullptr;
    double *em = nullptr, *es = nullptr, *psi = nullptr, *ut = nullptr, *us = nullptr;
    double *ps = nullptr, *uf = nullptr, *phi = nullptr, *G = nullptr, *DC = nullptr;
    double *gpa = nullptr;       // (dt/rho) grad p of the stage's old pressure, for the projection's add-back
    double *dD = nullptr, *Dh = nullptr, *wts = nullptr, *dudn = nullptr, *srate = nullptr;
    double *ff = nullptr;        // face fluxes: 3 components x face triple
    double *rhs_c = nullptr;     // cell rhs scratch
    double *rhs_n = nullptr;     // nodal rhs scratch
    double *u_host_dev = nullptr, *p_host_dev = nullptr;  // device copies for host-buffer steps
    double *dt_dev = nullptr;    // device-side time step and its derived scalars (DT_*)
    unsigned long long *cfl_max = nullptr;  // [0] convective, [1] forcing (bit patterns)

    // solvers
    CcHier mac, visc;
    NdHier nd;
    // per-level vectors, shared by the hierarchies (sized for the larger of cells/nodes)
    void *lx[kMaxLevels] = {}, *lb[kMaxLevels] = {}, *lr[kMaxLevels] = {}, *ld[kMaxLevels] = {};
    void *lt[kMaxLevels] = {};
    // Krylov vectors (FP64)
    double *kr = nullptr, *kz = nullptr, *kp = nullptr, *kq = nullptr;
    // FP32 inner Krylov vectors of the refinement solver
    float *kr32 = nullptr, *kz32 = nullptr, *kp32 = nullptr, *kq32 = nullptr, *ke32 = nullptr;
    double *part = nullptr;      // block partial sums
    double *scal = nullptr;      // device scalars
    double *scal_host = nullptr; // pinned mirror
    size_t vec_len = 0;

    // Solver loop control lives on the device: the convergence tests run in
    // one-thread kernels that write a condition word (read back by the host
    // loop in eager mode) and, inside a captured graph, set the handle of a
    // conditional WHILE node, so a whole step runs without the host.
    int *ctl = nullptr;           // condition words, counters, error words
    int *ctl_host = nullptr;      // pinned mirror
    double *sstat = nullptr;      // per solve slot: iterations, relative residual, outer passes
    double *sstat_host = nullptr; // pinned mirror
    int cur_slot = 0;             // slot of the solve being issued
    bool capturing = false;       // issuing into a graph capture
    int cap_depth = 0;            // nesting of conditional bodies being captured
    cudaStream_t cap_stream[4] = {};
    std::string cap_err;          // first failure while capturing
    struct LoopRec { int slot, per_outer, per_inner; };
    std::vector<LoopRec> loop_recs;   // launches per loop pass of each captured solve
    long long graph_top_launches = 0; // launches of the captured step outside loop bodies
    // adjoint workspace (allocated by the first adjoint call)
    double *adj = nullptr;
    size_t adj_len = 0;
    // the cut cells by colour for the wall-gradient adjoint (built on first
    // use per geometry): wall_col[wall_col_off[q] .. wall_col_off[q+1]) colour q
    int *wall_col = nullptr;
    std::vector<int> wall_col_off;
    bool wall_col_ok = false;
    // the captured step (one graph launch = one step)
    cudaGraphExec_t step_exec = nullptr;
    const void *gkey_u = nullptr, *gkey_p = nullptr, *gkey_f = nullptr;
    double gkey_dt = 0.0;

    // per-phase CUDA events of an eager step with statistics (created on first use)
    cudaEvent_t phase_ev[9] = {};
    bool phase_ev_ok = false;

    // TMA tensor maps of the fused smoother sweep, encoded on first use per
    // (array, box kind, level dims); the arrays live as long as the context
    struct TmaEntry {
        const void *p;
        int kind, nx, ny, nz;
        CUtensorMap m;
    };
    std::vector<TmaEntry> tma;

    ebv_status fail(ebv_status s, const std::string &m)
    {
        err = m;
        return s;
    }
};

// Process-wide switches of the smoother (ebv_set_spin_limit,
// ebv_set_fused_sweep): the bound of one wait inside a kernel in clock64
// cycles (0: give up at once, for tests of the timeout path), and whether
// FP32 levels with nx a multiple of 16 take the fused one-pass sweep: 0
// never, 1 where it timed faster than two colour passes, 2 always (same
// results in every case).  Read when a launch is issued or captured.
long long spin_limit();
int fused_sweep_mode();
void set_spin_limit(long long cycles);
void set_fused_sweep(int mode);
// The drop of the residual each FP32 correction solve of the refinement aims
// for (ebv_set_inner_drop), read when a solve is issued or captured.
double refine_inner_drop();
void set_inner_drop(double drop);
constexpr double kInnerDropDefault = 1e-4;
constexpr long long kSpinDefault = 2000000000LL;   // about 1 s at the maximum SM clock
constexpr long long kRbDrainCycles = 4000000000LL; // waiting for loads in flight after a timeout

// Launch bookkeeping: every kernel launch goes through these macros.
// EBV_LAUNCH_P names the launch and states the algorithmic bytes it must move
// (used for the roofline); EBV_LAUNCH names it after the kernel.
bool prof_begin_launch(struct Ctx *c, const char *name, double nbytes);
void prof_end_launch(struct Ctx *c);
#define EBV_LAUNCH_P(ctx, name, nbytes, kern, grid, block, smem, ...)                   \
    do {                                                                                \
        bool p_ = (ctx)->prof_on;                                                       \
        if (p_) p_ = prof_begin_launch((ctx), (name), (nbytes));                         \
        kern<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);                  \
        (ctx)->launches++;                                                              \
        if (p_) prof_end_launch((ctx));                                                 \
    } while (0)
#define EBV_LAUNCH(ctx, kern, grid, block, smem, ...) \
    EBV_LAUNCH_P(ctx, #kern, 0.0, kern, grid, block, smem, __VA_ARGS__)

#define EBV_CUDA_TRY(ctx, call)                                                          \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return (ctx)->fail(e_ == cudaErrorMemoryAllocation ? EBV_ERR_OOM : EBV_ERR_CUDA, \
                               std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

// Every device allocation of the library goes through dev_malloc, which
// enforces the optional allocation budget of ebv_set_alloc_limit (a host-side
// fault-injection hook: past the budget it fails as cudaMalloc does when the
// device is out of memory, without touching the device).
cudaError_t dev_malloc(void **p, size_t bytes);

inline GeomD geomd(const Ctx *c)
{
    GeomD q;
    q.alpha = c->alpha; q.ax = c->ax; q.ay = c->ay; q.az = c->az; q.area = c->area;
    q.nrm = c->nrm; q.bcen = c->bcen; q.flag = c->flag; q.cut = c->cut; q.ncut = c->ncut;
    q.ncell = ncell(c->g);
    return q;
}
inline ParamsD paramsd(const ebv_params &p)
{
    ParamsD q;
    q.rho = p.rho; q.mu = p.mu; q.tau0 = p.tau0; q.m = p.m; q.n_flow = p.n_flow; q.eta0 = p.eta0;
    q.model = p.model; q.delta_min = p.delta_min;
    q.inv_m = 1.0 / p.m;
    return q;
}

// geometry.cu
ebv_status build_geometry_host(Ctx *c, ebv_implicit_fn fn, void *user);
ebv_status build_geometry_bodies(Ctx *c, int n, const ebv_body *bodies);
// fields.cu
// Geometry on the host: volume fractions, face apertures (three face
// arrays), EB areas, normals and centroids (3 x cells each), flags and the
// ascending list of cut cells.
struct HostGeom {
    std::vector<double> alpha, a[3], area, nrm, bcen;
    std::vector<uint8_t> flag;
    std::vector<int> cut;
};
ebv_status install_geometry(Ctx *c, HostGeom &H);
ebv_status launch_strain_eta(Ctx *c, const double *u, double *eta, double *srate, double *G);
ebv_status launch_flow_diag(Ctx *c, const double *u, double *lam, double *sdev);
ebv_status launch_face_states(Ctx *c, const double *u, double *uf);
ebv_status launch_mac_rhs(Ctx *c, const double *uf, double *b);
ebv_status launch_mac_correct(Ctx *c, double *uf, const double *phi);
ebv_status launch_convective(Ctx *c, const double *u, const double *uf, double *C);
ebv_status launch_viscous_explicit(Ctx *c, const double *u, const double *eta, const double *G,
                                   double *V);
ebv_status launch_redistribute_into(Ctx *c, const double *DC, double sign, double div, double *out);
ebv_status launch_psi(Ctx *c, const double *u, const double *C, const double *V, const double *p,
                      const double *f, double *psi, double *gpa = nullptr);
ebv_status launch_add_stored(Ctx *c, double *u, const double *gpa);
ebv_status launch_add_gradp(Ctx *c, double *u, const double *p, double coef_sign);
ebv_status launch_nodal_rhs(Ctx *c, const double *ut, double *b);
ebv_status launch_timestep(Ctx *c, const double *u, const double *f, double dt_fixed);
ebv_status launch_average(Ctx *c, double *a, const double *b, int n);
ebv_status launch_drag(Ctx *c, const double *u, const double *p, double *fz, double *yf);
ebv_status launch_zero_covered(Ctx *c, double *u, int ncomp);
ebv_status launch_wall_dudn(Ctx *c, const double *u, double *dudn);
// adjoint.cu (reverse pieces of the creeping-flow step)
ebv_status adj_strain_eta(Ctx *c, const double *u, const double *eta_bar, const double *G_bar, double *u_bar,
                          double *grads_dev);
ebv_status adj_wall_dudn(Ctx *c, const double *dudn_bar, double *u_bar);
ebv_status adj_viscous_explicit(Ctx *c, const double *u, const double *eta, const double *G, const double *V_bar,
                                double *u_bar, double *eta_bar, double *G_bar, double *Fb, double *DCb, double *tb,
                                double *dudn_bar);
ebv_status adj_visc_eta(Ctx *c, int comp, const double *lam, const double *x, double *eta_bar);
ebv_status adj_gradp_t(Ctx *c, const double *w, double scale, double *out, int accumulate);
ebv_status adj_nodal_rhs_t(Ctx *c, const double *rb, double *ub);
ebv_status adj_drag(Ctx *c, const double *eta, double wJ, double *eta_bar, double *dudn_bar, double *p_bar);
ebv_status adj_psi(Ctx *c, const double *psib, double dt, double vs, double *ub, double *Vb, int vb_acc,
                   double *fb, double *Cb);
ebv_status adj_convective(Ctx *c, const double *u, const double *S, const double *uF, const double *Cb, double *ub,
                          double *DCb, double *tb, double *Fb, double *Sb, double *uFb, double *phib, double *bb);
ebv_status adj_mask_scale(Ctx *c, int ncomp, const double *b, double s, double *a);
ebv_status adj_alpha_times(Ctx *c, const double *lam, double *a);
ebv_status adj_axpby(Ctx *c, int n, double a, const double *x, double b, double *y);
ebv_status adj_zero_inactive_nodes(Ctx *c, double *x);
// solvers.cu
ebv_status setup_solvers(Ctx *c);
ebv_status setup_geometry_solvers(Ctx *c);
ebv_status mac_solve(Ctx *c, const double *b, double *x, int *iters, double *res);
// operators A_q(eta) of the three viscous solves (q = velocity component):
// shared coefficients, per-component diagonals and bottom inverses
ebv_status visc_build(Ctx *c, const double *eta);
// A_q x = alpha psi_q + boundary terms, after visc_build
ebv_status visc_solve(Ctx *c, const double *psi_comp, int comp, double *x, int *iters, double *res);
ebv_status nodal_solve(Ctx *c, const double *b, double *x, int *iters, double *res);
// A_q x = rhs (the viscous operator with the given right-hand side instead of
// alpha psi + boundary terms), from x = 0, after visc_build
ebv_status visc_solve_rhs(Ctx *c, int comp, const double *rhs, double *x, int *iters, double *res);
// reductions (solvers.cu)
ebv_status reduce_sum(Ctx *c, const double *part, int nblocks, double *out_dev);

}  // namespace ebv
