// C-ABI entry points (include/ebvisc.h): context life cycle, geometry, the
// stage operations of Algorithm 2 and the step of Algorithm 1.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include "ebv_internal.cuh"

#include <atomic>

#include <nvtx3/nvToolsExt.h>

using namespace ebv;

struct ebv_ctx : public Ctx {};

namespace ebv {
// Allocation budget of ebv_set_alloc_limit: bytes still allowed, or -1 for
// no limit (the default).
static std::atomic<long long> g_alloc_budget{-1};

cudaError_t dev_malloc(void **p, size_t bytes)
{
    long long b = g_alloc_budget.load();
    while (b >= 0) {
        if ((long long)bytes > b) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_alloc_budget.compare_exchange_weak(b, b - (long long)bytes)) break;
    }
    return cudaMalloc(p, bytes);
}
}  // namespace ebv

extern "C" void ebv_set_alloc_limit(long long bytes) { g_alloc_budget.store(bytes < 0 ? -1 : bytes); }
extern "C" void ebv_set_spin_limit(long long cycles) { ebv::set_spin_limit(cycles); }
extern "C" void ebv_set_fused_sweep(int mode) { ebv::set_fused_sweep(mode); }
extern "C" void ebv_set_inner_drop(double drop) { ebv::set_inner_drop(drop); }

namespace {

ebv_status check_params(const ebv_params *p, std::string &why)
{
    if (!(p->rho > 0.0)) { why = "rho must be > 0"; return EBV_ERR_INVALID; }
    if (!(p->mu >= 0.0) || !(p->tau0 >= 0.0)) { why = "mu and tau0 must be >= 0"; return EBV_ERR_INVALID; }
    if (!(p->m > 0.0)) { why = "m (1/epsilon) must be > 0"; return EBV_ERR_INVALID; }
    if (p->model < EBV_NEWTONIAN || p->model > EBV_SOUZA_MENDES_DUTRA) { why = "unknown model"; return EBV_ERR_INVALID; }
    if (p->model == EBV_SOUZA_MENDES_DUTRA && !(p->tau0 > 0.0)) { why = "SMD needs tau0 > 0"; return EBV_ERR_INVALID; }
    if (!(p->tol > 0.0) || p->max_iters < 1) { why = "tol > 0 and max_iters >= 1 required"; return EBV_ERR_INVALID; }
    if (!(p->cfl > 0.0)) { why = "cfl must be > 0"; return EBV_ERR_INVALID; }
    if (!(p->delta_min > 0.0)) { why = "delta_min must be > 0"; return EBV_ERR_INVALID; }
    if (p->precision != EBV_FP64 && p->precision != EBV_FP32_REFINE && p->precision != EBV_FP32_MIXED) {
        why = "unknown precision";
        return EBV_ERR_INVALID;
    }
    if (p->advect != 0 && p->advect != 1) { why = "advect must be 0 or 1"; return EBV_ERR_INVALID; }
    return EBV_OK;
}

// Outcome of the allocations of one ebv_create: the first failure decides
// whether the context reports EBV_ERR_OOM or EBV_ERR_CUDA.
struct AllocState {
    cudaError_t first = cudaSuccess;
};
template <class T>
bool alloc(T **p, size_t n, AllocState &a)
{
    cudaError_t e = dev_malloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess && a.first == cudaSuccess) a.first = e;
    return e == cudaSuccess;
}

double sphere_fn(const double x[3], void *user)
{
    const double *s = (const double *)user;
    double dx = x[0] - s[0], dy = x[1] - s[1], dz = x[2] - s[2];
    return sqrt(dx * dx + dy * dy + dz * dz) - s[3];
}
double plane_fn(const double x[3], void *user)
{
    const double *s = (const double *)user;
    return s[0] * x[0] + s[1] * x[1] + s[2] * x[2] - s[3];
}

void drop_step_graph(Ctx *c)
{
    if (c->step_exec) {
        cudaStreamSynchronize(c->stream);
        cudaGraphExecDestroy(c->step_exec);
        c->step_exec = nullptr;
    }
}

ebv_status need_geom(Ctx *c)
{
    if (!c->have_geom) return c->fail(EBV_ERR_GEOMETRY, "no geometry built");
    return EBV_OK;
}

__global__ void k_set_dt(double *d, double dt, double rho, double h)
{
    if (threadIdx.x == 0) store_dt(d, dt, rho, h);
}

ebv_status set_dt(Ctx *c, double dt)
{
    if (!(dt > 0.0)) return c->fail(EBV_ERR_INVALID, "dt must be > 0");
    EBV_LAUNCH(c, k_set_dt, dim3(1), dim3(32), 0, c->dt_dev, dt, c->prm.rho, c->g.h);
    return EBV_OK;
}

#define TRY(x)                          \
    do {                                \
        ebv_status s_ = (x);            \
        if (s_ != EBV_OK) return s_;    \
    } while (0)

// Algorithm 2 for velocity u: C, eta, V (and the projected face velocities in c->uf).
ebv_status derived(Ctx *c, const double *u, double *C, double *eta, double *V, int *it, double *res, int slot)
{
    if (c->prm.advect) {
        TRY(launch_face_states(c, u, c->uf));
        TRY(launch_mac_rhs(c, c->uf, c->rhs_c));
        c->cur_slot = slot;
        TRY(mac_solve(c, c->rhs_c, c->phi, it, res));
        TRY(launch_mac_correct(c, c->uf, c->phi));
        TRY(launch_convective(c, u, c->uf, C));
    } else {
        // creeping flow: no convective term, no face velocities to project
        EBV_CUDA_TRY(c, cudaMemsetAsync(C, 0, 3 * (size_t)ncell(c->g) * sizeof(double), c->stream));
        if (it) *it = 0;
        if (res) *res = 0.0;
    }
    TRY(launch_strain_eta(c, u, eta, nullptr, c->G));
    TRY(launch_viscous_explicit(c, u, eta, c->G, V));
    return EBV_OK;
}

// ut = psi / rho on fluid cells (0 on covered ones), the viscous solves'
// initial guess.  An FP64 division is about fifteen FP64-pipe instructions on
// this GPU, so when rho is a power of two (rho = 1 in the usual scaling) the
// kernel multiplies by the exact reciprocal instead: the same bits.
__global__ void k_init_guess(int n3, const uint8_t *flag, const double *psi, double rho, double inv_rho,
                             int exact_inv, double *ut)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n3; c += gridDim.x * blockDim.x) {
        const bool fl = flag[c] != 0;
        for (int q = 0; q < 3; q++) {
            const int s = q * n3 + c;
            ut[s] = fl ? (exact_inv ? psi[s] * inv_rho : psi[s] / rho) : 0.0;
        }
    }
}

ebv_status viscous_update(Ctx *c, const double *eta, const double *psi, double *ut, ebv_step_stats *st, int slot)
{
    const int N3 = ncell(c->g);
    int e2 = 0;
    const bool pow2 = frexp(c->prm.rho, &e2) == 0.5;   // rho = 2^(e2 - 1): 1/rho exact
    EBV_LAUNCH(c, k_init_guess, dim3(kReduceBlocks), dim3(256), 0, N3, c->flag, psi, c->prm.rho, 1.0 / c->prm.rho,
               pow2 ? 1 : 0, ut);
    TRY(visc_build(c, eta));
    for (int q = 0; q < 3; q++) {
        int it = 0;
        double res = 0.0;
        c->cur_slot = slot + q;
        TRY(visc_solve(c, psi + (size_t)q * N3, q, ut + (size_t)q * N3, &it, &res));
        if (st) { st->iters[slot + q] = it; st->res[slot + q] = res; }
    }
    return EBV_OK;
}

// Nodal projection of ut with old pressure p (in/out), dt on the device.
// gpa: (dt/rho) grad p stored by the k_psi of the same stage (same p), added
// back without re-forming it; null forms it from p.
ebv_status nodal_projection(Ctx *c, double *ut, double *p, ebv_step_stats *st, int slot, const double *gpa = nullptr)
{
    if (gpa) TRY(launch_add_stored(c, ut, gpa));
    else TRY(launch_add_gradp(c, ut, p, +1.0));
    TRY(launch_nodal_rhs(c, ut, c->rhs_n));
    int it = 0;
    double res = 0.0;
    c->cur_slot = slot;
    TRY(nodal_solve(c, c->rhs_n, p, &it, &res));
    if (st) { st->iters[slot] = it; st->res[slot] = res; }
    TRY(launch_add_gradp(c, ut, p, -1.0));
    return EBV_OK;
}

// The largest relative divergence the step's four projections leave: the
// cell-centred solve's relative residual is ||D u^F|| / ||D u~^F||, the nodal
// solve's is the relative residual of the (approximate) projection.
double step_div_rel(const ebv_step_stats &s)
{
    return std::max(std::max(s.res[0], s.res[4]), std::max(s.res[5], s.res[9]));
}

// Phases of an eager step with statistics, timed by CUDA events on the
// context's stream and marked as NVTX ranges: ms[0] time step, [1] predictor
// derived quantities (Algorithm 2), [2] predictor viscous solves, [3]
// predictor projection, [4..6] the same for the corrector, [7] drag and
// yielded fraction.
struct Phases {
    Ctx *c;
    bool on;
    int cur = -1;
    Phases(Ctx *c_, bool want) : c(c_), on(want)
    {
        if (on && !c->phase_ev_ok) {
            bool ok = true;
            for (cudaEvent_t &e : c->phase_ev) ok &= cudaEventCreate(&e) == cudaSuccess;
            c->phase_ev_ok = ok;
        }
        on = on && c->phase_ev_ok;
    }
    void mark(int q, const char *name)
    {
        if (cur >= 0) nvtxRangePop();
        nvtxRangePushA(name);
        cur = q;
        if (on) cudaEventRecord(c->phase_ev[q], c->stream);
    }
    void end()
    {
        if (cur >= 0) nvtxRangePop();
        cur = -1;
        if (on) cudaEventRecord(c->phase_ev[8], c->stream);
    }
    ~Phases()
    {
        if (cur >= 0) nvtxRangePop();
    }
    void read(float *ms)
    {
        if (!on) return;
        for (int q = 0; q < 8; q++)
            if (cudaEventElapsedTime(&ms[q], c->phase_ev[q], c->phase_ev[q + 1]) != cudaSuccess) ms[q] = 0.0f;
    }
};

ebv_status advance_impl(Ctx *c, double *u, double *p, double dt, const double *f, ebv_step_stats *st)
{
    const GridD &g = c->g;
    const size_t N3 = ncell(g), NN = nnode(g);
    ebv_step_stats loc;
    memset(&loc, 0, sizeof loc);
    Phases ph(c, st != nullptr);
    ph.mark(0, "ebv: time step");
    TRY(launch_timestep(c, u, f, dt));
    // Predictor
    ph.mark(1, "ebv: predictor derived quantities");
    TRY(derived(c, u, c->Cm, c->em, c->Vm, &loc.iters[0], &loc.res[0], 0));
    TRY(launch_psi(c, u, c->Cm, c->Vm, p, f, c->psi, c->gpa));
    ph.mark(2, "ebv: predictor viscous solves");
    TRY(viscous_update(c, c->em, c->psi, c->ut, &loc, 1));
    ph.mark(3, "ebv: predictor nodal projection");
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->ps, p, NN * 8, cudaMemcpyDeviceToDevice, c->stream));
    TRY(nodal_projection(c, c->ut, c->ps, &loc, 4, c->gpa));   // c->ps holds p here
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->us, c->ut, 3 * N3 * 8, cudaMemcpyDeviceToDevice, c->stream));
    // Corrector
    ph.mark(4, "ebv: corrector derived quantities");
    TRY(derived(c, c->us, c->Cs, c->es, c->Vs, &loc.iters[5], &loc.res[5], 5));
    TRY(launch_average(c, c->Cm, c->Cs, (int)(3 * N3)));
    TRY(launch_average(c, c->Vm, c->Vs, (int)(3 * N3)));
    TRY(launch_average(c, c->em, c->es, (int)N3));
    TRY(launch_psi(c, u, c->Cm, c->Vm, c->ps, f, c->psi, c->gpa));
    ph.mark(5, "ebv: corrector viscous solves");
    TRY(viscous_update(c, c->em, c->psi, c->ut, &loc, 6));
    ph.mark(6, "ebv: corrector nodal projection");
    EBV_CUDA_TRY(c, cudaMemcpyAsync(p, c->ps, NN * 8, cudaMemcpyDeviceToDevice, c->stream));
    TRY(nodal_projection(c, c->ut, p, &loc, 9, c->gpa));      // p holds c->ps here
    EBV_CUDA_TRY(c, cudaMemcpyAsync(u, c->ut, 3 * N3 * 8, cudaMemcpyDeviceToDevice, c->stream));
    if (st) {
        ph.mark(7, "ebv: drag");
        EBV_CUDA_TRY(c, cudaMemcpyAsync(&c->scal_host[14], c->dt_dev, sizeof(double), cudaMemcpyDeviceToHost,
                                        c->stream));
        ph.end();
        TRY(launch_drag(c, u, p, &loc.drag, &loc.yield_frac));  // synchronises
        loc.dt = c->scal_host[14];
        loc.div_rel = step_div_rel(loc);
        ph.read(loc.ms);
        *st = loc;
    } else {
        ph.end();
    }
    return EBV_OK;
}

// Redirects a context's issue into its capture stream (already capturing or
// joined to a capture); returns the saved state for end_ctx_capture.
struct CtxCapture {
    cudaStream_t user;
    bool prof;
    long long l0;
};
ebv_status begin_ctx_capture(Ctx *c, CtxCapture &k)
{
    for (cudaStream_t &s : c->cap_stream)
        if (!s) EBV_CUDA_TRY(c, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    k.prof = c->prof_on;
    k.user = c->stream;
    k.l0 = c->launches;
    c->prof_on = false;
    c->stream = c->cap_stream[0];
    c->capturing = true;
    c->cap_depth = 0;
    c->cap_err.clear();
    c->loop_recs.clear();
    return EBV_OK;
}
// Restores the context; records the launches captured outside loop bodies.
void end_ctx_capture(Ctx *c, const CtxCapture &k)
{
    const long long captured = c->launches - k.l0;
    c->launches = k.l0;
    c->capturing = false;
    c->stream = k.user;
    c->prof_on = k.prof;
    long long in_loops = 0;
    for (const Ctx::LoopRec &r : c->loop_recs) in_loops += r.per_outer + r.per_inner;
    c->graph_top_launches = captured - in_loops;
}
// Launches that `steps` launches of the captured step ran (from the device's
// per-slot iteration sums, read back into sstat_host).
long long graph_launches(const Ctx *c, int steps)
{
    long long n = steps * c->graph_top_launches;
    for (const Ctx::LoopRec &r : c->loop_recs)
        n += (long long)(r.per_inner * c->sstat_host[kSstatAcc + 2 * r.slot] +
                         r.per_outer * c->sstat_host[kSstatAcc + 2 * r.slot + 1]);
    return n;
}
ebv_status step_error(Ctx *c)
{
    const int fe = c->ctl_host[C_STEPERR];
    if (!fe) return EBV_OK;
    const int e = fe / 100, slot = fe % 100;
    if (e == E_SMEM)
        return c->fail(EBV_ERR_CUDA, "shared memory of the fused sweep not 128-byte aligned (solve slot " +
                                         std::to_string(slot) + ")");
    if (e == E_TIMEOUT)
        return c->fail(EBV_ERR_TIMEOUT, "a bounded wait in the smoother gave up (solve slot " +
                                            std::to_string(slot) + ")");
    return c->fail(e == E_NAN ? EBV_ERR_NAN : EBV_ERR_NOT_CONVERGED,
                   std::string(e == E_NAN ? "non-finite residual" : "linear solve did not reach the tolerance") +
                       " (solve slot " + std::to_string(slot) + ")");
}

// Captures one step of Algorithm 1 for (u, p, dt, f) into a graph: the
// solver loops become conditional WHILE nodes, so one graph launch runs a
// whole step with no host round trip.  The capture itself issues no work.
// Before a run of captured steps: clear the error word and the launch sums.
ebv_status graph_reset(Ctx *c, cudaStream_t s)
{
    EBV_CUDA_TRY(c, cudaMemsetAsync(c->ctl + C_STEPERR, 0, sizeof(int), s));
    EBV_CUDA_TRY(c, cudaMemsetAsync(c->sstat + kSstatAcc, 0, 2 * kSolveSlots * sizeof(double), s));
    return EBV_OK;
}
// After it: control words, solve statistics and dt to the pinned mirrors.
ebv_status graph_readback(Ctx *c, cudaStream_t s)
{
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->ctl_host, c->ctl, C_LEN * sizeof(int), cudaMemcpyDeviceToHost, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->sstat_host, c->sstat, kSstatLen * sizeof(double), cudaMemcpyDeviceToHost, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(&c->scal_host[14], c->dt_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
    return EBV_OK;
}

// The last captured step's statistics (sstat_host, scal_host[14] read back)
// plus drag and unyielded fraction of (u, p).
ebv_status graph_stats(Ctx *c, const double *u, const double *p, ebv_step_stats *st)
{
    ebv_step_stats loc;
    memset(&loc, 0, sizeof loc);
    for (int q = 0; q < 10; q++) {
        loc.iters[q] = (int)c->sstat_host[3 * q];
        loc.res[q] = c->sstat_host[3 * q + 1];
    }
    loc.dt = c->scal_host[14];
    loc.div_rel = step_div_rel(loc);
    TRY(launch_drag(c, u, p, &loc.drag, &loc.yield_frac));
    *st = loc;
    return EBV_OK;
}

ebv_status capture_step(Ctx *c, double *u, double *p, double dt, const double *f)
{
    drop_step_graph(c);
    CtxCapture k;
    TRY(begin_ctx_capture(c, k));
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    ebv_status st = EBV_OK;
    if (e == cudaSuccess) st = advance_impl(c, u, p, dt, f, nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = (e == cudaSuccess) ? cudaStreamEndCapture(c->stream, &g) : e;
    end_ctx_capture(c, k);
    if (st != EBV_OK || e2 != cudaSuccess || !c->cap_err.empty()) {
        if (g) cudaGraphDestroy(g);
        if (st != EBV_OK) return st;
        return c->fail(EBV_ERR_CUDA, std::string("step capture: ") +
                                         (c->cap_err.empty() ? cudaGetErrorString(e2) : c->cap_err.c_str()));
    }
    cudaError_t e3 = cudaGraphInstantiate(&c->step_exec, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
        c->step_exec = nullptr;
        return c->fail(EBV_ERR_CUDA, std::string("step graph instantiate: ") + cudaGetErrorString(e3));
    }
    c->gkey_u = u; c->gkey_p = p; c->gkey_f = f; c->gkey_dt = dt;
    return EBV_OK;
}

// `steps` launches of the captured step, then one synchronisation: the
// step's error word, the launch count and (if asked) the last step's stats.
ebv_status advance_graph_impl(Ctx *c, double *u, double *p, double dt, const double *f, int steps,
                              ebv_step_stats *st)
{
    if (!c->step_exec || c->gkey_u != u || c->gkey_p != p || c->gkey_f != f || c->gkey_dt != dt)
        TRY(capture_step(c, u, p, dt, f));
    TRY(graph_reset(c, c->stream));
    for (int s = 0; s < steps; s++) EBV_CUDA_TRY(c, cudaGraphLaunch(c->step_exec, c->stream));
    TRY(graph_readback(c, c->stream));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->launches += graph_launches(c, steps);
    TRY(step_error(c));
    if (st) TRY(graph_stats(c, u, p, st));
    return EBV_OK;
}

}  // namespace

namespace ebv {
bool prof_begin_launch(Ctx *c, const char *name, double nbytes)
{
    ProfEvents &P = c->prof;
    if (P.used * 2 + 2 > P.ev.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return false;
        if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return false; }
        P.ev.push_back(a);
        P.ev.push_back(b);
        P.key.push_back(0);
        P.bytes.push_back(0.0);
    }
    int key = -1;
    for (size_t q = 0; q < P.names.size() && key < 0; q++)
        if (P.names[q] == name || strcmp(P.names[q], name) == 0) key = (int)q;
    if (key < 0) {
        key = (int)P.names.size();
        P.names.push_back(name);  // string literals: live for the program
    }
    P.key[P.used] = key;
    P.bytes[P.used] = nbytes;
    cudaEventRecord(P.ev[2 * P.used], c->stream);
    return true;
}
void prof_end_launch(Ctx *c)
{
    ProfEvents &P = c->prof;
    cudaEventRecord(P.ev[2 * P.used + 1], c->stream);
    P.used++;
}
}  // namespace ebv

extern "C" {

ebv_status ebv_profile_begin(ebv_ctx *c)
{
    if (!c) return EBV_ERR_INVALID;
    c->prof.used = 0;
    c->prof_on = true;
    return EBV_OK;
}

ebv_status ebv_profile_end(ebv_ctx *c, int *entries)
{
    if (!c || !entries) return EBV_ERR_INVALID;
    c->prof_on = false;
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    ProfEvents &P = c->prof;
    const size_t K = P.names.size();
    P.agg_launches.assign(K, 0);
    P.agg_ms.assign(K, 0.0);
    P.agg_bytes.assign(K, 0.0);
    for (size_t q = 0; q < P.used; q++) {
        float t = 0.0f;
        EBV_CUDA_TRY(c, cudaEventElapsedTime(&t, P.ev[2 * q], P.ev[2 * q + 1]));
        P.agg_launches[P.key[q]]++;
        P.agg_ms[P.key[q]] += t;
        P.agg_bytes[P.key[q]] += P.bytes[q];
    }
    P.used = 0;
    *entries = (int)K;
    return EBV_OK;
}

ebv_status ebv_profile_entry(ebv_ctx *c, int i, const char **name, long long *launches, double *ms,
                             double *bytes)
{
    if (!c || !name || !launches || !ms || !bytes) return EBV_ERR_INVALID;
    ProfEvents &P = c->prof;
    if (i < 0 || (size_t)i >= P.agg_ms.size()) return c->fail(EBV_ERR_INVALID, "no such profile entry");
    *name = P.names[i];
    *launches = P.agg_launches[i];
    *ms = P.agg_ms[i];
    *bytes = P.agg_bytes[i];
    return EBV_OK;
}

ebv_status ebv_create(const ebv_grid *grid, const ebv_params *params, void *stream, ebv_ctx **out)
{
    if (!grid || !params || !out) return EBV_ERR_INVALID;
    *out = nullptr;
    std::string why;
    if (check_params(params, why) != EBV_OK) return EBV_ERR_INVALID;
    for (int d = 0; d < 3; d++)
        if (grid->n[d] < 1) return EBV_ERR_INVALID;
    if (!(grid->h > 0.0)) return EBV_ERR_INVALID;
    for (int s = 0; s < 6; s++)
        if (grid->bc[s] < EBV_INFLOW || grid->bc[s] > EBV_NOSLIP) return EBV_ERR_INVALID;
    long long nn = (long long)(grid->n[0] + 1) * (grid->n[1] + 1) * (grid->n[2] + 1);
    if (nn >= (1LL << 31) / 9) return EBV_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return EBV_ERR_CUDA;

    ebv_ctx *c = new (std::nothrow) ebv_ctx();
    if (!c) return EBV_ERR_INVALID;
    cudaGetDevice(&c->device);
    c->stream = (cudaStream_t)stream;
    c->prm = *params;
    GridD &g = c->g;
    g.nx = grid->n[0]; g.ny = grid->n[1]; g.nz = grid->n[2];
    g.h = grid->h;
    g.ih = 1.0 / grid->h;
    for (int d = 0; d < 3; d++) { g.lo[d] = grid->lo[d]; g.u_in[d] = grid->u_in[d]; }
    for (int s = 0; s < 6; s++) g.bc[s] = grid->bc[s];
    const size_t N3 = ncell(g), NN = nnode(g), NF = nface(g, 0) + nface(g, 1) + nface(g, 2);
    const size_t V = std::max(N3, NN);
    AllocState as;
    bool ok = true;
    ok &= alloc(&c->alpha, N3, as) && alloc(&c->ax, nface(g, 0), as) && alloc(&c->ay, nface(g, 1), as) &&
          alloc(&c->az, nface(g, 2), as) && alloc(&c->area, N3, as) && alloc(&c->nrm, 3 * N3, as) &&
          alloc(&c->bcen, 3 * N3, as) && alloc(&c->flag, N3, as);
    ok &= alloc(&c->Cm, 3 * N3, as) && alloc(&c->Vm, 3 * N3, as) && alloc(&c->Cs, 3 * N3, as) &&
          alloc(&c->Vs, 3 * N3, as);
    ok &= alloc(&c->em, N3, as) && alloc(&c->es, N3, as) && alloc(&c->psi, 3 * N3, as) &&
          alloc(&c->ut, 3 * N3, as) && alloc(&c->us, 3 * N3, as) && alloc(&c->gpa, 3 * N3, as);
    ok &= alloc(&c->ps, NN, as) && alloc(&c->uf, NF, as) && alloc(&c->phi, N3, as) && alloc(&c->G, 9 * N3, as) &&
          alloc(&c->DC, 3 * N3, as) && alloc(&c->dD, 3 * N3, as) && alloc(&c->Dh, 3 * N3, as) &&
          alloc(&c->wts, N3, as) && alloc(&c->srate, N3, as) && alloc(&c->rhs_c, std::max(N3, (size_t)1), as) &&
          alloc(&c->rhs_n, NN, as);
    ok &= alloc(&c->nearm, N3, as) && alloc(&c->ff, 3 * NF, as);
    ok &= alloc(&c->dt_dev, DT_NSCALAR, as) && alloc(&c->cfl_max, 2, as);
    ok &= alloc(&c->u_host_dev, 3 * N3, as) && alloc(&c->p_host_dev, NN, as);
    ok &= alloc(&c->kr, V, as) && alloc(&c->kz, V, as) && alloc(&c->kp, V, as) && alloc(&c->kq, V, as);
    ok &= alloc(&c->kr32, V, as) && alloc(&c->kz32, V, as) && alloc(&c->kp32, V, as) && alloc(&c->kq32, V, as) &&
          alloc(&c->ke32, V, as);
    ok &= alloc(&c->part, (size_t)1 << 20, as) && alloc(&c->scal, 32, as);
    ok &= cudaMallocHost(&c->scal_host, 32 * sizeof(double)) == cudaSuccess;
    ok &= alloc(&c->ctl, C_LEN, as) && alloc(&c->sstat, kSstatLen, as);
    ok &= cudaMallocHost(&c->ctl_host, C_LEN * sizeof(int)) == cudaSuccess;
    ok &= cudaMallocHost(&c->sstat_host, kSstatLen * sizeof(double)) == cudaSuccess;
    c->vec_len = V;
    if (!ok) {
        ebv_destroy(c);
        cudaGetLastError();  // an allocation failure leaves no error pending
        return as.first == cudaErrorMemoryAllocation ? EBV_ERR_OOM : EBV_ERR_CUDA;
    }
    if (ebv_status st = setup_solvers(c); st != EBV_OK) {
        ebv_destroy(c);
        cudaGetLastError();
        return st == EBV_ERR_OOM ? EBV_ERR_OOM : EBV_ERR_INVALID;
    }
    cudaMemsetAsync(c->scal, 0, 32 * sizeof(double), c->stream);
    cudaMemsetAsync(c->ctl, 0, C_LEN * sizeof(int), c->stream);
    cudaMemsetAsync(c->sstat, 0, kSstatLen * sizeof(double), c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        ebv_destroy(c);
        return EBV_ERR_CUDA;
    }
    *out = c;
    return EBV_OK;
}

ebv_status ebv_set_params(ebv_ctx *c, const ebv_params *params)
{
    if (!c || !params) return EBV_ERR_INVALID;
    std::string why;
    if (check_params(params, why) != EBV_OK) return c->fail(EBV_ERR_INVALID, why);
    bool prec_changed = params->precision != c->prm.precision;
    drop_step_graph(c);
    c->prm = *params;
    if (prec_changed && c->have_geom) return setup_geometry_solvers(c);
    return EBV_OK;
}

ebv_status ebv_build_geometry(ebv_ctx *c, ebv_implicit_fn fn, void *user)
{
    if (!c || !fn) return EBV_ERR_INVALID;
    drop_step_graph(c);
    TRY(build_geometry_host(c, fn, user));
    TRY(setup_geometry_solvers(c));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return EBV_OK;
}

ebv_status ebv_build_geometry_sphere(ebv_ctx *c, const double cen[3], double r)
{
    if (!c || !cen || !(r > 0.0)) return EBV_ERR_INVALID;
    double s[4] = {cen[0], cen[1], cen[2], r};
    return ebv_build_geometry(c, sphere_fn, s);
}

ebv_status ebv_build_geometry_bodies(ebv_ctx *c, int n, const ebv_body *bodies)
{
    if (!c || !bodies || n < 1) return EBV_ERR_INVALID;
    drop_step_graph(c);
    TRY(build_geometry_bodies(c, n, bodies));
    TRY(setup_geometry_solvers(c));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return EBV_OK;
}

ebv_status ebv_build_geometry_spheres(ebv_ctx *c, int n, const double *c_r)
{
    if (!c || !c_r || n < 1 || n > 16) return EBV_ERR_INVALID;
    ebv_body b[16];
    for (int q = 0; q < n; q++) {
        b[q].kind = EBV_BODY_SPHERE;
        for (int e = 0; e < 4; e++) b[q].q[e] = c_r[4 * q + e];
        b[q].q[4] = b[q].q[5] = 0.0;
    }
    return ebv_build_geometry_bodies(c, n, b);
}

ebv_status ebv_build_geometry_plane(ebv_ctx *c, const double nrm[3], double d)
{
    if (!c || !nrm) return EBV_ERR_INVALID;
    double s[4] = {nrm[0], nrm[1], nrm[2], d};
    return ebv_build_geometry(c, plane_fn, s);
}

// ---- resumable state --------------------------------------------------------
// File layout: the 8 bytes "EBVSTAT1", the ebv_grid and ebv_params structs,
// then alpha, the x/y/z apertures, the EB area, normal and centroid (doubles),
// the flags (bytes), u (3 x cells) and p (nodes) (doubles).
namespace {
const char kStateMagic[8] = {'E', 'B', 'V', 'S', 'T', 'A', 'T', '1'};

struct StateFile {
    FILE *f = nullptr;
    ~StateFile()
    {
        if (f) fclose(f);
    }
};

ebv_grid grid_of(const Ctx *c)
{
    ebv_grid g;
    memset(&g, 0, sizeof g);
    g.n[0] = c->g.nx; g.n[1] = c->g.ny; g.n[2] = c->g.nz;
    g.h = c->g.h;
    for (int d = 0; d < 3; d++) { g.lo[d] = c->g.lo[d]; g.u_in[d] = c->g.u_in[d]; }
    for (int q = 0; q < 6; q++) g.bc[q] = c->g.bc[q];
    return g;
}
}  // namespace

ebv_status ebv_save_state(ebv_ctx *c, const double *u, const double *p, const char *path)
{
    if (!c || !u || !p || !path) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    const GridD &g = c->g;
    const size_t N3 = ncell(g), NN = nnode(g);
    HostGeom H;
    H.alpha.resize(N3); H.area.resize(N3); H.nrm.resize(3 * N3); H.bcen.resize(3 * N3); H.flag.resize(N3);
    for (int d = 0; d < 3; d++) H.a[d].resize(nface(g, d));
    std::vector<double> uh(3 * N3), ph(NN);
    const double *src[7] = {c->alpha, c->ax, c->ay, c->az, c->area, c->nrm, c->bcen};
    std::vector<double> *dst[7] = {&H.alpha, &H.a[0], &H.a[1], &H.a[2], &H.area, &H.nrm, &H.bcen};
    for (int q = 0; q < 7; q++)
        EBV_CUDA_TRY(c, cudaMemcpyAsync(dst[q]->data(), src[q], dst[q]->size() * 8, cudaMemcpyDeviceToHost,
                                        c->stream));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(H.flag.data(), c->flag, N3, cudaMemcpyDeviceToHost, c->stream));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(uh.data(), u, 3 * N3 * 8, cudaMemcpyDeviceToHost, c->stream));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(ph.data(), p, NN * 8, cudaMemcpyDeviceToHost, c->stream));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    StateFile F;
    F.f = fopen(path, "wb");
    if (!F.f) return c->fail(EBV_ERR_INVALID, std::string("cannot write ") + path);
    ebv_grid gr = grid_of(c);
    bool ok = fwrite(kStateMagic, 1, 8, F.f) == 8 && fwrite(&gr, sizeof gr, 1, F.f) == 1 &&
              fwrite(&c->prm, sizeof c->prm, 1, F.f) == 1;
    for (int q = 0; q < 7 && ok; q++) ok = fwrite(dst[q]->data(), 8, dst[q]->size(), F.f) == dst[q]->size();
    ok = ok && fwrite(H.flag.data(), 1, N3, F.f) == N3 && fwrite(uh.data(), 8, 3 * N3, F.f) == 3 * N3 &&
         fwrite(ph.data(), 8, NN, F.f) == NN;
    ok = (fclose(F.f) == 0) && ok;
    F.f = nullptr;
    if (!ok) return c->fail(EBV_ERR_INVALID, std::string("write failed: ") + path);
    return EBV_OK;
}

ebv_status ebv_load_state(ebv_ctx *c, double *u, double *p, const char *path)
{
    if (!c || !u || !p || !path) return EBV_ERR_INVALID;
    StateFile F;
    F.f = fopen(path, "rb");
    if (!F.f) return c->fail(EBV_ERR_INVALID, std::string("cannot read ") + path);
    char magic[8];
    ebv_grid gr, mine = grid_of(c);
    ebv_params prm;
    if (fread(magic, 1, 8, F.f) != 8 || memcmp(magic, kStateMagic, 8) != 0)
        return c->fail(EBV_ERR_INVALID, "not a state file of this library");
    if (fread(&gr, sizeof gr, 1, F.f) != 1 || fread(&prm, sizeof prm, 1, F.f) != 1)
        return c->fail(EBV_ERR_INVALID, "truncated state file");
    if (memcmp(&gr, &mine, sizeof gr) != 0) return c->fail(EBV_ERR_INVALID, "the state was saved on another grid");
    std::string why;
    if (check_params(&prm, why) != EBV_OK) return c->fail(EBV_ERR_INVALID, "state file parameters: " + why);
    const GridD &g = c->g;
    const size_t N3 = ncell(g), NN = nnode(g);
    HostGeom H;
    H.alpha.resize(N3); H.area.resize(N3); H.nrm.resize(3 * N3); H.bcen.resize(3 * N3); H.flag.resize(N3);
    for (int d = 0; d < 3; d++) H.a[d].resize(nface(g, d));
    std::vector<double> uh(3 * N3), ph(NN);
    std::vector<double> *dst[7] = {&H.alpha, &H.a[0], &H.a[1], &H.a[2], &H.area, &H.nrm, &H.bcen};
    bool ok = true;
    for (int q = 0; q < 7 && ok; q++) ok = fread(dst[q]->data(), 8, dst[q]->size(), F.f) == dst[q]->size();
    ok = ok && fread(H.flag.data(), 1, N3, F.f) == N3 && fread(uh.data(), 8, 3 * N3, F.f) == 3 * N3 &&
         fread(ph.data(), 8, NN, F.f) == NN;
    if (!ok) return c->fail(EBV_ERR_INVALID, "truncated state file");
    for (size_t q = 0; q < N3; q++)
        if (H.flag[q] == 2) H.cut.push_back((int)q);
    drop_step_graph(c);
    c->prm = prm;
    TRY(install_geometry(c, H));
    TRY(setup_geometry_solvers(c));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(u, uh.data(), 3 * N3 * 8, cudaMemcpyHostToDevice, c->stream));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(p, ph.data(), NN * 8, cudaMemcpyHostToDevice, c->stream));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return EBV_OK;
}

ebv_status ebv_get_geometry(ebv_ctx *c, double *alpha, double *ax, double *ay, double *az, double *area,
                            double *nrm, double *bcen, unsigned char *flag)
{
    if (!c) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    const GridD &g = c->g;
    const size_t N3 = ncell(g);
    cudaStream_t s = c->stream;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
    };
    EBV_CUDA_TRY(c, cp(alpha, c->alpha, N3 * 8));
    EBV_CUDA_TRY(c, cp(ax, c->ax, nface(g, 0) * 8));
    EBV_CUDA_TRY(c, cp(ay, c->ay, nface(g, 1) * 8));
    EBV_CUDA_TRY(c, cp(az, c->az, nface(g, 2) * 8));
    EBV_CUDA_TRY(c, cp(area, c->area, N3 * 8));
    EBV_CUDA_TRY(c, cp(nrm, c->nrm, 3 * N3 * 8));
    EBV_CUDA_TRY(c, cp(bcen, c->bcen, 3 * N3 * 8));
    EBV_CUDA_TRY(c, cp(flag, c->flag, N3));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(s));
    return EBV_OK;
}

ebv_status ebv_update_viscosity(ebv_ctx *c, const double *u, double *eta, double *srate)
{
    if (!c || !u || !eta) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(launch_strain_eta(c, u, eta, srate, nullptr));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_flow_diagnostics(ebv_ctx *c, const double *u, double *lambda, double *stress_dev)
{
    if (!c || !u || !lambda || !stress_dev) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(launch_flow_diag(c, u, lambda, stress_dev));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_derived(ebv_ctx *c, const double *u, double *C, double *eta, double *V, int *iters, double *res)
{
    if (!c || !u || !C || !eta || !V) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(derived(c, u, C, eta, V, iters, res, 0));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_face_states(ebv_ctx *c, const double *u, double *uf)
{
    if (!c || !u || !uf) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(launch_face_states(c, u, uf));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_solve_mac(ebv_ctx *c, double *uf, double *phi, int *iters, double *res)
{
    if (!c || !uf || !phi) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(launch_mac_rhs(c, uf, c->rhs_c));
    c->cur_slot = 0;
    TRY(mac_solve(c, c->rhs_c, phi, iters, res));
    TRY(launch_mac_correct(c, uf, phi));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_solve_viscous(ebv_ctx *c, const double *eta, const double *psi, double dt, double *ut,
                             ebv_step_stats *st)
{
    if (!c || !eta || !psi || !ut) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(set_dt(c, dt));
    TRY(viscous_update(c, eta, psi, ut, st, 1));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_solve_projection(ebv_ctx *c, double *ut, double *p, double dt, ebv_step_stats *st)
{
    if (!c || !ut || !p) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(set_dt(c, dt));
    TRY(nodal_projection(c, ut, p, st, 4));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_timestep(ebv_ctx *c, const double *u, const double *f, double *dt_host)
{
    if (!c || !u || !dt_host) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(launch_timestep(c, u, f, 0.0));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(&c->scal_host[14], c->dt_dev, sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *dt_host = c->scal_host[14];
    return EBV_OK;
}

ebv_status ebv_advance(ebv_ctx *c, double *u, double *p, double dt, const double *f, ebv_step_stats *st)
{
    if (!c || !u || !p) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(advance_impl(c, u, p, dt, f, st));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_advance_graph(ebv_ctx *c, double *u, double *p, double dt, const double *f, int steps,
                             ebv_step_stats *st)
{
    if (!c || !u || !p || steps < 0) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(advance_graph_impl(c, u, p, dt, f, steps, st));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_advance_host(ebv_ctx *c, double *u_host, double *p_host, int steps, double dt,
                            ebv_step_stats *last)
{
    if (!c || !u_host || !p_host || steps < 0) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    const size_t N3 = ncell(c->g), NN = nnode(c->g);
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->u_host_dev, u_host, 3 * N3 * 8, cudaMemcpyHostToDevice, c->stream));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->p_host_dev, p_host, NN * 8, cudaMemcpyHostToDevice, c->stream));
    TRY(advance_graph_impl(c, c->u_host_dev, c->p_host_dev, dt, nullptr, steps, last));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(u_host, c->u_host_dev, 3 * N3 * 8, cudaMemcpyDeviceToHost, c->stream));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(p_host, c->p_host_dev, NN * 8, cudaMemcpyDeviceToHost, c->stream));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return EBV_OK;
}

ebv_status ebv_drag(ebv_ctx *c, const double *u, const double *p, double *fz, double *yf)
{
    if (!c || !u || !p || !fz || !yf) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(launch_drag(c, u, p, fz, yf));
    return EBV_OK;
}

long long ebv_launch_count(const ebv_ctx *c) { return c ? c->launches : 0; }

ebv_status ebv_sweep_timing(const ebv_ctx *c, int level, int kind, float *fused_ms, float *passes_ms)
{
    if (!c || !fused_ms || !passes_ms || level < 0 || level >= c->mac.L || kind < 0 || kind > 3)
        return EBV_ERR_INVALID;
    *fused_ms = c->mac.lv[level].rb_ms[kind][0];
    *passes_ms = c->mac.lv[level].rb_ms[kind][1];
    return EBV_OK;
}

const char *ebv_last_error(const ebv_ctx *c) { return c ? c->err.c_str() : "null context"; }

void ebv_destroy(ebv_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    if (c->phase_ev_ok)
        for (cudaEvent_t e : c->phase_ev) cudaEventDestroy(e);
    void *ptrs[] = {c->alpha, c->ax, c->ay, c->az, c->area, c->nrm, c->bcen, c->flag, c->cut, c->Cm, c->Vm,
                    c->Cs, c->Vs, c->em, c->es, c->psi, c->ut, c->us, c->ps, c->uf, c->phi, c->G, c->DC,
                    c->dD, c->Dh, c->wts, c->dudn, c->srate, c->rhs_c, c->rhs_n, c->u_host_dev, c->p_host_dev,
                    c->dt_dev, c->cfl_max, c->kr, c->kz, c->kp, c->kq, c->part, c->scal, c->nearm,
                    c->nearl, c->ff, c->kr32, c->kz32, c->kp32, c->kq32, c->ke32, c->gpa, c->wall_col};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    CcHier *hs[2] = {&c->mac, &c->visc};
    for (int h = 0; h < 2; h++) {
        CcHier *H = hs[h];
        for (int l = 0; l < H->L; l++) {
            CcLevel &L = H->lv[l];
            cudaFree(L.extra_d); cudaFree(L.extra_f);
            for (int q = 0; q < H->nvar; q++) {
                cudaFree(H->vdiag_d[q][l]); cudaFree(H->vdiag_f[q][l]); cudaFree(H->vdinv_f[q][l]);
            }
            for (int d = 0; d < 3; d++) { cudaFree(L.bf_d[d]); cudaFree(L.bf_f[d]); cudaFree(L.bf_h[d]); }
            cudaFree(L.bxp);
            if (h == 0) cudaFree(L.cov);
        }
        for (int q = 0; q < H->nvar; q++) { cudaFree(H->vbinv[q]); cudaFree(H->vdiag_a[q]); }
        cudaFree(H->bmat);
    }
    for (int l = 0; l < c->nd.L; l++) {
        NdLevel &L = c->nd.lv[l];
        if (l) cudaFree(L.alpha_d);
        cudaFree(L.alpha_f);
        cudaFree(L.act);
        cudaFree(L.reg);
        cudaFree(L.irr);
    }
    cudaFree(c->nd.binv);
    cudaFree(c->nd.bmat);

    for (int l = 0; l < kMaxLevels; l++) {
        cudaFree(c->lx[l]); cudaFree(c->lb[l]); cudaFree(c->lr[l]); cudaFree(c->ld[l]); cudaFree(c->lt[l]);
    }
    if (c->scal_host) cudaFreeHost(c->scal_host);
    drop_step_graph(c);
    cudaFree(c->ctl);
    cudaFree(c->sstat);
    if (c->adj) cudaFree(c->adj);
    if (c->ctl_host) cudaFreeHost(c->ctl_host);
    if (c->sstat_host) cudaFreeHost(c->sstat_host);
    for (cudaStream_t s : c->cap_stream)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : c->prof.ev) cudaEventDestroy(e);
    delete c;
}

// ---------------------------------------------------------------------------
// Adjoint of the creeping-flow step (advect = 0, fixed dt) and of the drag,
// for drag sensitivities with respect to tau0, mu and a body-force field.
// The forward step is recomputed from its start state, keeping what the
// reverse pass reads; the reverse pass runs the adjoint kernels of
// adjoint.cu and the transposed solves (the viscous and nodal operators are
// symmetric, so their adjoint solves are the same multigrid-CG solves).
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

struct AdjBufs {
    double *em, *es, *eb, *Gm, *Gs, *Vm, *Vs, *Va, *psi, *utm, *uts, *us, *zero3, *t3;
    double *ebm, *ebs, *ebb, *Gb, *Vbs, *Vbm, *psib, *usb, *utb, *lam, *DCb, *tb, *etad;
    double *ffb, *dudnb, *ps, *psb, *nb1, *nb2, *ua, *pa, *grads;
    // convective term: slopes and projected face velocities of both stages,
    // C of both stages and its average, their adjoints and work
    double *Sm, *Ss, *uFm, *uFs, *Cm, *Cs, *Ca, *Cbm, *Cbs, *Sb, *uFb, *phib, *bbc;
};

// Carves the adjoint workspace into B (allocated on first use, once per
// context; the forward step itself never allocates).
ebv_status adj_buffers(Ctx *c, AdjBufs &B)
{
    const size_t N3 = ncell(c->g), NN = nnode(c->g), NF = nface(c->g, 0) + nface(c->g, 1) + nface(c->g, 2);
    const size_t NC = (size_t)c->ncut + 1;
    // offsets first, pointers once the block exists
    size_t off = 0;
    std::vector<std::pair<double **, size_t>> parts;
    auto take = [&](double **dst, size_t n) { parts.push_back({dst, off}); off += n; };
    for (double **d : {&B.em, &B.es, &B.eb, &B.ebm, &B.ebs, &B.ebb, &B.lam, &B.etad, &B.phib, &B.bbc}) take(d, N3);
    for (double **d : {&B.Gm, &B.Gs, &B.Gb, &B.Sm, &B.Ss, &B.Sb}) take(d, 9 * N3);
    for (double **d : {&B.Vm, &B.Vs, &B.Va, &B.psi, &B.utm, &B.uts, &B.us, &B.zero3, &B.t3, &B.Vbs, &B.Vbm, &B.psib,
                       &B.usb, &B.utb, &B.DCb, &B.tb, &B.ua, &B.Cm, &B.Cs, &B.Ca, &B.Cbm, &B.Cbs})
        take(d, 3 * N3);
    take(&B.ffb, 3 * NF);
    for (double **d : {&B.uFm, &B.uFs, &B.uFb}) take(d, NF);
    take(&B.dudnb, 3 * NC);
    for (double **d : {&B.ps, &B.psb, &B.nb1, &B.nb2, &B.pa}) take(d, NN);
    take(&B.grads, 8);
    auto layout = [&](double *base) {
        for (auto &pr : parts) *pr.first = base + pr.second;
    };
    const size_t need = off;
    if (c->adj_len < need) {
        if (c->adj) cudaFree(c->adj);
        c->adj = nullptr;
        c->adj_len = 0;
        EBV_CUDA_TRY(c, dev_malloc((void **)&c->adj, need * sizeof(double)));
        c->adj_len = need;
    }
    layout(c->adj);
    return EBV_OK;
}

ebv_status adj_check(Ctx *c, double dt)
{
    if (c->prm.model != EBV_NEWTONIAN && c->prm.model != EBV_BINGHAM && c->prm.model != EBV_HERSCHEL_BULKLEY &&
        c->prm.model != EBV_POWER_LAW)
        return c->fail(EBV_ERR_INVALID, "no adjoint for this rheology");
    if (!(dt > 0.0)) return c->fail(EBV_ERR_INVALID, "the adjoint needs a fixed dt > 0");
    return EBV_OK;
}

// Adjoint of the nodal projection (ut, p_old) -> (u, p): given the adjoints
// (ubo, pbo) of its outputs, utb = adjoint of ut; pold_b += adjoint of p_old.
//   u1 = mask(ut + c G p_old); p = L^-1 (D u1 + bc) / c; u = mask(u1 - c G p)
ebv_status proj_adjoint(Ctx *c, AdjBufs &B, double dt, const double *ubo, const double *pbo, double *utb,
                        double *pold_b)
{
    const size_t NN = nnode(c->g);
    const double cc = dt / c->prm.rho;
    TRY(adj_mask_scale(c, 3, ubo, 1.0, B.t3));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(B.nb1, pbo, NN * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    TRY(adj_gradp_t(c, B.t3, -cc, B.nb1, 1));
    TRY(adj_zero_inactive_nodes(c, B.nb1));
    EBV_CUDA_TRY(c, cudaMemsetAsync(B.nb2, 0, NN * sizeof(double), c->stream));
    int it = 0;
    double res = 0.0;
    c->cur_slot = 13;
    TRY(nodal_solve(c, B.nb1, B.nb2, &it, &res));
    TRY(adj_nodal_rhs_t(c, B.nb2, B.t3));
    TRY(adj_mask_scale(c, 3, B.t3, 1.0, utb));
    TRY(adj_gradp_t(c, utb, cc, pold_b, 1));
    return EBV_OK;
}

// Adjoint of the three viscous solves A_q(eta) x_q = alpha psi_q + b_q(eta):
// psib = adjoint of psi, etab += adjoint of eta, from xb = adjoint of x.
ebv_status visc_adjoint(Ctx *c, AdjBufs &B, const double *eta, const double *x, const double *xb, double *psib,
                        double *etab)
{
    const size_t N3 = ncell(c->g);
    TRY(visc_build(c, eta));
    for (int q = 0; q < 3; q++) {
        int it = 0;
        double res = 0.0;
        c->cur_slot = 12;
        TRY(visc_solve_rhs(c, q, xb + q * N3, B.lam, &it, &res));
        TRY(adj_alpha_times(c, B.lam, psib + q * N3));
        TRY(adj_visc_eta(c, q, B.lam, x + q * N3, etab));
    }
    return EBV_OK;
}

// One step's reverse pass.  In: state (u, p) at the step's start, dt, f; ub,
// pb the adjoints of the step's outputs.  Out: ub, pb the adjoints of u, p;
// fb += adjoint of f (if fb); grads_dev[0..1] += d/dtau0, d/dmu.
ebv_status adjoint_step_impl(Ctx *c, const double *u, const double *p, double dt, const double *f, double *ub,
                             double *pb, double *fb, AdjBufs &B)
{
    const size_t N3 = ncell(c->g), NN = nnode(c->g);
    cudaStream_t s = c->stream;
    TRY(set_dt(c, dt));
    const bool adv = c->prm.advect != 0;
    // the convective term of state w (as derived() computes it): slopes into
    // S, projected face velocities into uF, C into C
    auto convective = [&](const double *w, double *S, double *uF, double *C) -> ebv_status {
        if (!adv) {
            EBV_CUDA_TRY(c, cudaMemsetAsync(C, 0, 3 * N3 * sizeof(double), s));
            return EBV_OK;
        }
        TRY(launch_face_states(c, w, uF));   // slopes of w in c->G
        EBV_CUDA_TRY(c, cudaMemcpyAsync(S, c->G, 9 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        TRY(launch_mac_rhs(c, uF, c->rhs_c));
        int it = 0;
        double res = 0.0;
        c->cur_slot = 10;   // the reverse pass's solves use slots 10..13
        TRY(mac_solve(c, c->rhs_c, c->phi, &it, &res));
        TRY(launch_mac_correct(c, uF, c->phi));
        TRY(launch_convective(c, w, uF, C));
        return EBV_OK;
    };
    // ---- forward, keeping the intermediates (as advance_impl)
    TRY(convective(u, B.Sm, B.uFm, B.Cm));
    TRY(launch_strain_eta(c, u, B.em, nullptr, B.Gm));
    TRY(launch_viscous_explicit(c, u, B.em, B.Gm, B.Vm));
    TRY(launch_psi(c, u, B.Cm, B.Vm, p, f, B.psi));
    TRY(viscous_update(c, B.em, B.psi, B.utm, nullptr, 1));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(B.us, B.utm, 3 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(B.ps, p, NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TRY(nodal_projection(c, B.us, B.ps, nullptr, 4));      // u*, p*
    TRY(convective(B.us, B.Ss, B.uFs, B.Cs));
    TRY(launch_strain_eta(c, B.us, B.es, nullptr, B.Gs));
    TRY(launch_viscous_explicit(c, B.us, B.es, B.Gs, B.Vs));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(B.Ca, B.Cm, 3 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TRY(launch_average(c, B.Ca, B.Cs, (int)(3 * N3)));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(B.eb, B.em, N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TRY(launch_average(c, B.eb, B.es, (int)N3));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(B.Va, B.Vm, 3 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TRY(launch_average(c, B.Va, B.Vs, (int)(3 * N3)));
    TRY(launch_psi(c, u, B.Ca, B.Va, B.ps, f, B.psi));
    TRY(viscous_update(c, B.eb, B.psi, B.uts, nullptr, 6));
    // ---- reverse
    // corrector projection: (ub, pb) -> utb (adjoint of the corrector's ut), psb (of p*)
    EBV_CUDA_TRY(c, cudaMemsetAsync(B.psb, 0, NN * sizeof(double), s));
    TRY(proj_adjoint(c, B, dt, ub, pb, B.utb, B.psb));
    // from here ub, pb accumulate the adjoints of the step's inputs u, p
    EBV_CUDA_TRY(c, cudaMemsetAsync(ub, 0, 3 * N3 * sizeof(double), s));
    EBV_CUDA_TRY(c, cudaMemsetAsync(pb, 0, NN * sizeof(double), s));
    // corrector viscous solves with eta_avg
    EBV_CUDA_TRY(c, cudaMemsetAsync(B.ebb, 0, N3 * sizeof(double), s));
    TRY(visc_adjoint(c, B, B.eb, B.uts, B.utb, B.psib, B.ebb));
    // corrector psi = rho u + dt (V_avg - grad p* + f), V_avg = (V_m + V_s) / 2:
    // V_s bar = V_m bar = dt psi bar / 2
    TRY(adj_psi(c, B.psib, dt, 0.5 * dt, ub, B.Vbs, 0, fb, adv ? B.Cbs : nullptr));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(B.Vbm, B.Vbs, 3 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (adv) EBV_CUDA_TRY(c, cudaMemcpyAsync(B.Cbm, B.Cbs, 3 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    TRY(adj_gradp_t(c, B.psib, -dt, B.psb, 1));   // psi is 0 on covered cells; k_gradp_t reads fluid cells
    // eta_avg = (eta_m + eta_s) / 2
    TRY(adj_mask_scale(c, 1, B.ebb, 0.5, B.ebs));
    TRY(adj_mask_scale(c, 1, B.ebb, 0.5, B.ebm));
    // corrector explicit viscous term and eta, G of u*
    EBV_CUDA_TRY(c, cudaMemsetAsync(B.usb, 0, 3 * N3 * sizeof(double), s));
    EBV_CUDA_TRY(c, cudaMemsetAsync(B.Gb, 0, 9 * N3 * sizeof(double), s));
    TRY(adj_viscous_explicit(c, B.us, B.es, B.Gs, B.Vbs, B.usb, B.ebs, B.Gb, B.ffb, B.DCb, B.tb, B.dudnb));
    TRY(adj_strain_eta(c, B.us, B.ebs, B.Gb, B.usb, B.grads));
    if (adv)
        TRY(adj_convective(c, B.us, B.Ss, B.uFs, B.Cbs, B.usb, B.DCb, B.tb, B.ffb, B.Sb, B.uFb, B.phib, B.bbc));
    // predictor projection: (usb, psb) -> utb, pb += (adjoint of p via u1 = ut + c G p)
    TRY(proj_adjoint(c, B, dt, B.usb, B.psb, B.utb, pb));
    // predictor viscous solves with eta_m
    TRY(visc_adjoint(c, B, B.em, B.utm, B.utb, B.psib, B.ebm));
    // predictor psi = rho u + dt (V_m - grad p + f)
    TRY(adj_psi(c, B.psib, dt, dt, ub, B.Vbm, 1, fb, adv ? B.Cbm : nullptr));
    TRY(adj_gradp_t(c, B.psib, -dt, pb, 1));
    // predictor explicit viscous term and eta, G of u
    EBV_CUDA_TRY(c, cudaMemsetAsync(B.Gb, 0, 9 * N3 * sizeof(double), s));
    TRY(adj_viscous_explicit(c, u, B.em, B.Gm, B.Vbm, ub, B.ebm, B.Gb, B.ffb, B.DCb, B.tb, B.dudnb));
    TRY(adj_strain_eta(c, u, B.ebm, B.Gb, ub, B.grads));
    if (adv) TRY(adj_convective(c, u, B.Sm, B.uFm, B.Cbm, ub, B.DCb, B.tb, B.ffb, B.Sb, B.uFb, B.phib, B.bbc));
    return EBV_OK;
}

// Adjoint of w F_z(u, p) (Eq. drag-force, eta = eta(u)): ub, pb, grads += .
// (F_z is linear in p, so p itself is not read.)
ebv_status drag_adjoint_impl(Ctx *c, const double *u, double w, double *ub, double *pb, AdjBufs &B)
{
    const size_t N3 = ncell(c->g);
    TRY(launch_strain_eta(c, u, B.etad, nullptr, nullptr));
    TRY(launch_wall_dudn(c, u, c->dudn));
    EBV_CUDA_TRY(c, cudaMemsetAsync(B.ebb, 0, N3 * sizeof(double), c->stream));
    if (c->ncut) {
        EBV_CUDA_TRY(c, cudaMemsetAsync(B.dudnb, 0, 3 * (size_t)c->ncut * sizeof(double), c->stream));
        TRY(adj_drag(c, B.etad, w, B.ebb, B.dudnb, pb));
        TRY(adj_wall_dudn(c, B.dudnb, ub));
    }
    TRY(adj_strain_eta(c, u, B.ebb, nullptr, ub, B.grads));
    return EBV_OK;
}

ebv_status read_grads(Ctx *c, AdjBufs &B, double *grads)
{
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->scal_host + 20, B.grads, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (grads) {
        grads[0] += c->scal_host[20];
        grads[1] += c->scal_host[21];
    }
    return EBV_OK;
}

}  // namespace

extern "C" {

ebv_status ebv_adjoint_step(ebv_ctx *c, const double *u, const double *p, double dt, const double *f,
                            double *u_bar, double *p_bar, double *f_bar, double *grads)
{
    if (!c || !u || !p || !u_bar || !p_bar) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(adj_check(c, dt));
    AdjBufs B;
    TRY(adj_buffers(c, B));
    EBV_CUDA_TRY(c, cudaMemsetAsync(B.grads, 0, 2 * sizeof(double), c->stream));
    TRY(adjoint_step_impl(c, u, p, dt, f, u_bar, p_bar, f_bar, B));
    TRY(read_grads(c, B, grads));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_drag_adjoint(ebv_ctx *c, const double *u, const double *p, double w, double *u_bar, double *p_bar,
                            double *grads)
{
    if (!c || !u || !p || !u_bar || !p_bar) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    if (c->prm.model == EBV_SOUZA_MENDES_DUTRA) return c->fail(EBV_ERR_INVALID, "no adjoint for this rheology");
    AdjBufs B;
    TRY(adj_buffers(c, B));
    EBV_CUDA_TRY(c, cudaMemsetAsync(B.grads, 0, 2 * sizeof(double), c->stream));
    TRY(drag_adjoint_impl(c, u, w, u_bar, p_bar, B));
    TRY(read_grads(c, B, grads));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status ebv_drag_gradient_workspace(const ebv_ctx *c, int steps, int every, long long *ndoubles)
{
    if (!c || steps < 1 || every < 1 || !ndoubles) return EBV_ERR_INVALID;
    const long long S = 3LL * ncell(c->g) + nnode(c->g);
    const long long nck = (steps + every - 1) / every;
    *ndoubles = S * (nck + std::min(every, steps) + 1);
    return EBV_OK;
}

// J = (1/steps) sum_{s=1..steps} F_z(u_s, p_s) over `steps` creeping-flow
// steps from (u0, p0) at fixed dt, and its gradient with respect to tau0, mu
// and the body force f.  Checkpoints every `every` steps; each segment is
// recomputed forward (its states kept) before its steps are reversed.
ebv_status ebv_drag_gradient(ebv_ctx *c, const double *u0, const double *p0, const double *f, double dt, int steps,
                             int every, double *work, double *J, double *grads, double *f_bar)
{
    if (!c || !u0 || !p0 || !work || !J || !grads || steps < 1 || every < 1) return EBV_ERR_INVALID;
    TRY(need_geom(c));
    TRY(adj_check(c, dt));
    const size_t N3 = ncell(c->g), NN = nnode(c->g), S = 3 * N3 + NN;
    const int nck = (steps + every - 1) / every;
    double *ck = work;                      // nck checkpoints (u, p)
    double *st = work + (size_t)nck * S;    // the states of one segment
    cudaStream_t s = c->stream;
    // forward: checkpoints and the objective
    EBV_CUDA_TRY(c, cudaMemcpyAsync(st, u0, 3 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(st + 3 * N3, p0, NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double Jsum = 0.0;
    for (int k = 0; k < steps; k++) {
        if (k % every == 0)
            EBV_CUDA_TRY(c, cudaMemcpyAsync(ck + (size_t)(k / every) * S, st, S * sizeof(double),
                                            cudaMemcpyDeviceToDevice, s));
        TRY(advance_impl(c, st, st + 3 * N3, dt, f, nullptr));
        double fz = 0.0, yf = 0.0;
        TRY(launch_drag(c, st, st + 3 * N3, &fz, &yf));
        Jsum += fz;
    }
    *J = Jsum / steps;
    // reverse: the adjoint state (ua, pa) starts at zero; each step adds its
    // objective term, then is reversed
    AdjBufs B;
    TRY(adj_buffers(c, B));
    double *ua = B.ua, *pa = B.pa;
    EBV_CUDA_TRY(c, cudaMemsetAsync(ua, 0, 3 * N3 * sizeof(double), s));
    EBV_CUDA_TRY(c, cudaMemsetAsync(pa, 0, NN * sizeof(double), s));
    EBV_CUDA_TRY(c, cudaMemsetAsync(B.grads, 0, 2 * sizeof(double), s));
    if (f_bar) EBV_CUDA_TRY(c, cudaMemsetAsync(f_bar, 0, 3 * N3 * sizeof(double), s));
    for (int q = nck - 1; q >= 0; q--) {
        const int k0 = q * every, k1 = std::min(k0 + every, steps);
        // states k0 .. k1 of this segment, recomputed from its checkpoint
        EBV_CUDA_TRY(c, cudaMemcpyAsync(st, ck + (size_t)q * S, S * sizeof(double), cudaMemcpyDeviceToDevice, s));
        for (int k = k0; k < k1; k++) {
            double *a = st + (size_t)(k - k0) * S, *b = a + S;
            EBV_CUDA_TRY(c, cudaMemcpyAsync(b, a, S * sizeof(double), cudaMemcpyDeviceToDevice, s));
            TRY(advance_impl(c, b, b + 3 * N3, dt, f, nullptr));
        }
        for (int k = k1 - 1; k >= k0; k--) {
            double *a = st + (size_t)(k - k0) * S, *b = a + S;
            TRY(drag_adjoint_impl(c, b, 1.0 / steps, ua, pa, B));
            TRY(adjoint_step_impl(c, a, a + 3 * N3, dt, f, ua, pa, f_bar, B));
        }
    }
    grads[0] = grads[1] = 0.0;
    TRY(read_grads(c, B, grads));
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

// ---------------------------------------------------------------------------
// Batches: independent instances (own grid, parameters, geometry and
// multigrid hierarchies), advanced together by ONE graph launch per step.
// The batch graph forks from an origin stream into one branch per instance;
// each branch is that instance's captured step (its solver loops are
// conditional nodes of its own), so instances converge independently and
// their kernels overlap on the GPU.
// ---------------------------------------------------------------------------
}  // extern "C"

struct ebv_batch {
    std::vector<ebv_ctx *> ctx;
    cudaStream_t stream = nullptr;     // caller's stream: graph launches
    cudaStream_t origin = nullptr;     // capture origin
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> key;     // u, p of every instance at capture
    std::string err;
    ebv_status fail(ebv_status s, const std::string &m)
    {
        err = m;
        return s;
    }
};

namespace {

void drop_batch_graph(ebv_batch *b)
{
    if (b->exec) {
        cudaStreamSynchronize(b->stream);
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
}

ebv_status capture_batch(ebv_batch *b, double *const *u, double *const *p)
{
    drop_batch_graph(b);
    const int n = (int)b->ctx.size();
    if (!b->origin && cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess)
        return b->fail(EBV_ERR_CUDA, "stream");
    if (!b->fork && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return b->fail(EBV_ERR_CUDA, "event");
    while ((int)b->join.size() < n) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return b->fail(EBV_ERR_CUDA, "event");
        b->join.push_back(e);
    }
    if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return b->fail(EBV_ERR_CUDA, "batch capture begin");
    ebv_status st = EBV_OK;
    std::string why;
    if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) { st = EBV_ERR_CUDA; why = "fork"; }
    for (int i = 0; i < n && st == EBV_OK; i++) {
        Ctx *c = b->ctx[i];
        CtxCapture k;
        if ((st = begin_ctx_capture(c, k)) != EBV_OK) { why = c->err; break; }
        if (cudaStreamWaitEvent(c->stream, b->fork, 0) != cudaSuccess) {
            end_ctx_capture(c, k);
            st = EBV_ERR_CUDA;
            why = "branch join";
            break;
        }
        st = advance_impl(c, u[i], p[i], 0.0, nullptr, nullptr);
        if (st == EBV_OK && !c->cap_err.empty()) { st = EBV_ERR_CUDA; why = c->cap_err; }
        if (st != EBV_OK && why.empty()) why = c->err;
        if (st == EBV_OK && (cudaEventRecord(b->join[i], c->stream) != cudaSuccess ||
                             cudaStreamWaitEvent(b->origin, b->join[i], 0) != cudaSuccess)) {
            st = EBV_ERR_CUDA;
            why = "branch merge";
        }
        end_ctx_capture(c, k);
        if (st != EBV_OK) why = "instance " + std::to_string(i) + ": " + why;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->origin, &g);
    if (st != EBV_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return b->fail(st != EBV_OK ? st : EBV_ERR_CUDA, "batch capture: " + (why.empty() ? cudaGetErrorString(e) : why));
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return b->fail(EBV_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
    }
    b->key.assign(2 * n, nullptr);
    for (int i = 0; i < n; i++) { b->key[2 * i] = u[i]; b->key[2 * i + 1] = p[i]; }
    return EBV_OK;
}

}  // namespace

extern "C" {

ebv_status ebv_batch_create(int n, const ebv_grid *grids, const ebv_params *params, void *stream, ebv_batch **out)
{
    if (n < 1 || !grids || !params || !out) return EBV_ERR_INVALID;
    *out = nullptr;
    ebv_batch *b = new (std::nothrow) ebv_batch();
    if (!b) return EBV_ERR_INVALID;
    b->stream = (cudaStream_t)stream;
    for (int i = 0; i < n; i++) {
        ebv_ctx *c = nullptr;
        ebv_status st = ebv_create(grids + i, params + i, stream, &c);
        if (st != EBV_OK) {
            ebv_batch_destroy(b);
            return st;
        }
        c->batched = true;
        b->ctx.push_back(c);
    }
    *out = b;
    return EBV_OK;
}

ebv_status ebv_batch_build_spheres(ebv_batch *b, const double *c_r)
{
    if (!b || !c_r) return EBV_ERR_INVALID;
    drop_batch_graph(b);
    const int n = (int)b->ctx.size();
    for (ebv_ctx *c : b->ctx) drop_step_graph(c);
    // host builders in parallel (one instance per thread, a few threads)
    std::vector<ebv_status> st(n, EBV_OK);
    const int nt = std::max(1, std::min(n, (int)std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; t++)
        pool.emplace_back([&, t]() {
            for (int i = t; i < n; i += nt) {
                double sp[4] = {c_r[4 * i], c_r[4 * i + 1], c_r[4 * i + 2], c_r[4 * i + 3]};
                st[i] = build_geometry_host(b->ctx[i], sphere_fn, sp);
            }
        });
    for (std::thread &th : pool) th.join();
    for (int i = 0; i < n; i++) {
        if (st[i] != EBV_OK) return b->fail(st[i], "instance " + std::to_string(i) + ": " + b->ctx[i]->err);
        // hierarchies and launch-shape tuning, one instance at a time
        ebv_status s2 = setup_geometry_solvers(b->ctx[i]);
        if (s2 == EBV_OK && cudaStreamSynchronize(b->ctx[i]->stream) != cudaSuccess) s2 = EBV_ERR_CUDA;
        if (s2 != EBV_OK) return b->fail(s2, "instance " + std::to_string(i) + ": " + b->ctx[i]->err);
    }
    return EBV_OK;
}

ebv_ctx *ebv_batch_instance(ebv_batch *b, int i)
{
    if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
    return b->ctx[i];
}

ebv_status ebv_batch_advance(ebv_batch *b, double *const *u, double *const *p, int steps, ebv_step_stats *stats)
{
    if (!b || !u || !p || steps < 0) return EBV_ERR_INVALID;
    const int n = (int)b->ctx.size();
    for (int i = 0; i < n; i++) {
        if (!u[i] || !p[i]) return b->fail(EBV_ERR_INVALID, "null field pointer");
        if (!b->ctx[i]->have_geom) return b->fail(EBV_ERR_GEOMETRY, "instance " + std::to_string(i) + ": no geometry");
    }
    bool same = b->exec && (int)b->key.size() == 2 * n;
    for (int i = 0; same && i < n; i++) same = b->key[2 * i] == u[i] && b->key[2 * i + 1] == p[i];
    if (!same) TRY(capture_batch(b, u, p));
    for (ebv_ctx *c : b->ctx)
        if (graph_reset(c, b->stream) != EBV_OK) return b->fail(EBV_ERR_CUDA, c->err);
    for (int s = 0; s < steps; s++)
        if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return b->fail(EBV_ERR_CUDA, "batch graph launch");
    for (ebv_ctx *c : b->ctx)
        if (graph_readback(c, b->stream) != EBV_OK) return b->fail(EBV_ERR_CUDA, c->err);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return b->fail(EBV_ERR_CUDA, "batch synchronise");
    ebv_status first = EBV_OK;
    for (int i = 0; i < n; i++) {
        Ctx *c = b->ctx[i];
        c->launches += graph_launches(c, steps);
        ebv_status e = step_error(c);
        if (e != EBV_OK && first == EBV_OK) {
            first = e;
            b->err = "instance " + std::to_string(i) + ": " + c->err;
        }
    }
    if (first != EBV_OK) return first;
    if (stats)
        for (int i = 0; i < n; i++)
            if (graph_stats(b->ctx[i], u[i], p[i], stats + i) != EBV_OK)
                return b->fail(EBV_ERR_CUDA, "instance " + std::to_string(i) + ": " + b->ctx[i]->err);
    return EBV_OK;
}

long long ebv_batch_launch_count(const ebv_batch *b)
{
    long long n = 0;
    if (b)
        for (const ebv_ctx *c : b->ctx) n += c->launches;
    return n;
}

const char *ebv_batch_last_error(const ebv_batch *b) { return b ? b->err.c_str() : "null batch"; }

void ebv_batch_destroy(ebv_batch *b)
{
    if (!b) return;
    drop_batch_graph(b);
    for (ebv_ctx *c : b->ctx) ebv_destroy(c);
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    delete b;
}

}  // extern "C"
