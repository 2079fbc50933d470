// Reverse-mode kernels of the step of Algorithm 1 (with or without the
// convective term): for each forward kernel of the step, a kernel that takes
// the adjoint of its outputs and adds the adjoint of its inputs.  Each mirrors its forward
// kernel's stencil (same branches, same weights); where the forward kernel
// gathers from several cells the reverse one gathers the transposed stencil
// where that is as simple, or scatters with plain additions in launches that
// no two threads' targets overlap in: faces of one position parity, cells of
// one colour of a map that is one-to-one on the stencil's offsets, cut cells
// of one colour of a greedy colouring by shared stencil cells.  No atomics,
// so the gradients are bitwise reproducible.
//
// Forward kernel            reverse kernel here
//   k_strain_eta              k_se_adj            (eta(||gamma||) and G = grad u)
//   k_wall_dudn               k_wall_dudn_adj     (Eq. dudn interpolation)
//   k_visc_flux               k_visc_flux_adj     (face fluxes eta (grad u)^T)
//   k_flux_div<EB>            k_flux_div_adj_faces, k_flux_div_adj_wall
//   k_redist_far/a/b          k_redist_adj_far, k_redist_adj_a, k_redist_adj_b
//   k_visc_coeffs (in eta)    k_visc_eta_adj      (-lambda^T dA/deta x + lambda^T db/deta)
//   grad_p (k_psi, k_add_gradp)  k_gradp_t
//   k_nodal_rhs (in ut)       k_nodal_rhs_t
//   k_drag_terms              k_drag_adj
//   k_slopes_march            k_slopes_adj        (MC limiter)
//   k_face_states             k_face_states_adj   (Godunov upwinding)
//   k_mac_rhs / k_mac_correct k_mac_rhs_adj / k_mac_correct_adj (with one MAC solve)
//   k_conv_flux               k_conv_flux_adj
#include <algorithm>
#include <unordered_map>

#include "ebv_internal.cuh"

namespace ebv {
namespace {

__device__ inline int3 unit3(int d) { return make_int3(d == 0, d == 1, d == 2); }

#define ADJ_CELL                                           \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   \
    const int j = blockIdx.y * blockDim.y + threadIdx.y;   \
    const int k = blockIdx.z * blockDim.z + threadIdx.z;   \
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;       \
    const int c = cidx(g, i, j, k);

// The robust derivative of the strain-rate kernel along d at (i,j,k) as a
// stencil: up to three (cell, weight) pairs; same branches as the forward
// (central; one-sided quadratic next to a covered cell; first order; none).
__device__ inline int d_robust_w(const GridD &g, const uint8_t *flag, int i, int j, int k, int d, double ih,
                                 int *idx, double *w)
{
    int3 e = unit3(d);
    const bool ip = avail(g, flag, i + e.x, j + e.y, k + e.z);
    const bool im = avail(g, flag, i - e.x, j - e.y, k - e.z);
    const int c0 = cidx(g, i, j, k);
    const int cp = cidx(g, i + e.x, j + e.y, k + e.z), cm = cidx(g, i - e.x, j - e.y, k - e.z);
    if (ip && im) {
        idx[0] = cp; w[0] = 0.5 * ih;
        idx[1] = cm; w[1] = -0.5 * ih;
        return 2;
    }
    if (im) {
        if (avail(g, flag, i - 2 * e.x, j - 2 * e.y, k - 2 * e.z)) {
            idx[0] = cidx(g, i - 2 * e.x, j - 2 * e.y, k - 2 * e.z); w[0] = 0.5 * ih;
            idx[1] = cm; w[1] = -2.0 * ih;
            idx[2] = c0; w[2] = 1.5 * ih;
            return 3;
        }
        idx[0] = c0; w[0] = ih;
        idx[1] = cm; w[1] = -ih;
        return 2;
    }
    if (ip) {
        if (avail(g, flag, i + 2 * e.x, j + 2 * e.y, k + 2 * e.z)) {
            idx[0] = c0; w[0] = -1.5 * ih;
            idx[1] = cp; w[1] = 2.0 * ih;
            idx[2] = cidx(g, i + 2 * e.x, j + 2 * e.y, k + 2 * e.z); w[2] = -0.5 * ih;
            return 3;
        }
        idx[0] = cp; w[0] = ih;
        idx[1] = c0; w[1] = -ih;
        return 2;
    }
    return 0;
}

// (1 - exp(-m s)) / s and its derivative in s, with the forward's branches
// (m s > 40: 1/s exactly; s = 0: the limit m).  Small m s uses the series of
// the derivative, -m^2 (1/2 - ms/3 + (ms)^2/8 - (ms)^3/30), to avoid the
// cancellation of the closed form.
__device__ inline void yield_term(double m, double s, double &y, double &dy)
{
    const double ms = m * s;
    if (!(s > 0.0)) {
        y = m;
        dy = -0.5 * m * m;
        return;
    }
    if (ms > 40.0) {
        y = 1.0 / s;
        dy = -1.0 / (s * s);
        return;
    }
    y = -expm1(-ms) / s;
    if (ms < 1e-3)
        dy = -m * m * (0.5 - ms / 3.0 + ms * ms / 8.0 - ms * ms * ms / 30.0);
    else
        dy = (ms * exp(-ms) + expm1(-ms)) / (s * s);
}

// d eta / d s, d eta / d tau0, d eta / d mu of the rheology table (the
// models the adjoint supports: Newtonian, Bingham-Papanastasiou,
// Herschel-Bulkley, power law).
__device__ inline void eta_partials(const ParamsD &p, double s, double &ds, double &dtau, double &dmu)
{
    double y, dy;
    yield_term(p.m, s, y, dy);
    const double sf = s > 1.0 / p.m ? s : 1.0 / p.m;
    ds = 0.0; dtau = 0.0; dmu = 0.0;
    switch (p.model) {
    case EBV_NEWTONIAN: dmu = 1.0; break;
    case EBV_BINGHAM: ds = p.tau0 * dy; dtau = y; dmu = 1.0; break;
    case EBV_HERSCHEL_BULKLEY:
        dmu = pow(sf, p.n_flow - 1.0);
        ds = (s > 1.0 / p.m ? p.mu * (p.n_flow - 1.0) * pow(s, p.n_flow - 2.0) : 0.0) + p.tau0 * dy;
        dtau = y;
        break;
    case EBV_POWER_LAW:
        dmu = pow(sf, p.n_flow - 1.0);
        ds = s > 1.0 / p.m ? p.mu * (p.n_flow - 1.0) * pow(s, p.n_flow - 2.0) : 0.0;
        break;
    }
}

template <int kThreads>
__device__ inline double block_sum_lin(double v)
{
    __shared__ double sm[kThreads / 32];
    const int t = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) sm[t >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (t < 32) {
        r = t < kThreads / 32 ? sm[t] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

// ---- strain rate + viscosity -------------------------------------------------
// In: eta_bar (per cell), G_bar (9 per cell, or NULL).  Adds the adjoint of u
// to u_bar; block partial sums of eta_bar d eta/d tau0 and eta_bar d eta/d mu
// to part[b], part[nblocks + b].  One launch per colour (i + 3j + 4k) mod 13:
// a cell scatters to itself and to its neighbours at distance 1 and 2 along
// each axis, and that map is one-to-one on those 13 offsets mod 13, so cells
// of one colour never share a target and plain additions, in launch order,
// make the result bitwise reproducible.
constexpr int kSeColours = 13;
__device__ inline int se_colour(int i, int j, int k) { return (i + 3 * j + 4 * k) % kSeColours; }
__global__ void __launch_bounds__(256) k_se_adj(GridD g, const uint8_t *__restrict__ flag,
                                                const double *__restrict__ u, ParamsD p,
                                                const double *__restrict__ eta_bar,
                                                const double *__restrict__ G_bar, double *__restrict__ u_bar,
                                                double *__restrict__ part, int colour)
{
    // thread x index t covers the cell of this colour i = i0 + 13 t of row (j, k)
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int i0 = ((colour - 3 * j - 4 * k) % kSeColours + kSeColours) % kSeColours;
    const int i = i0 + kSeColours * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    double vt = 0.0, vm = 0.0;
    if (i < g.nx && j < g.ny && k < g.nz && se_colour(i, j, k) == colour) {
        const int c = cidx(g, i, j, k);
        const int N3 = ncell(g);
        if (flag[c] != 0) {
            const double ih = g.ih;
            int idx[3][3];
            double w[3][3];
            int cnt[3];
            double Gm[3][3];
            for (int d = 0; d < 3; d++) {
                cnt[d] = d_robust_w(g, flag, i, j, k, d, ih, idx[d], w[d]);
                for (int q = 0; q < 3; q++) {
                    // the forward value, with the forward kernel's arithmetic
                    double v = 0.0;
                    const double *uq = u + q * N3;
                    int3 e = unit3(d);
                    const bool ip = avail(g, flag, i + e.x, j + e.y, k + e.z);
                    const bool im = avail(g, flag, i - e.x, j - e.y, k - e.z);
                    const double f0 = uq[c];
                    if (ip && im) {
                        v = (uq[cidx(g, i + e.x, j + e.y, k + e.z)] - uq[cidx(g, i - e.x, j - e.y, k - e.z)]) *
                            (0.5 * ih);
                    } else if (im) {
                        const double f1 = uq[cidx(g, i - e.x, j - e.y, k - e.z)];
                        if (avail(g, flag, i - 2 * e.x, j - 2 * e.y, k - 2 * e.z))
                            v = (0.5 * uq[cidx(g, i - 2 * e.x, j - 2 * e.y, k - 2 * e.z)] - 2.0 * f1 + 1.5 * f0) * ih;
                        else
                            v = (f0 - f1) * ih;
                    } else if (ip) {
                        const double f1 = uq[cidx(g, i + e.x, j + e.y, k + e.z)];
                        if (avail(g, flag, i + 2 * e.x, j + 2 * e.y, k + 2 * e.z))
                            v = (-1.5 * f0 + 2.0 * f1 - 0.5 * uq[cidx(g, i + 2 * e.x, j + 2 * e.y, k + 2 * e.z)]) * ih;
                        else
                            v = (f1 - f0) * ih;
                    }
                    Gm[d][q] = v;
                }
            }
            double s2 = 0.0;
            for (int d = 0; d < 3; d++)
                for (int q = 0; q < 3; q++) {
                    double gam = Gm[d][q] + Gm[q][d];
                    s2 += gam * gam;
                }
            const double s = sqrt(0.5 * s2);
            double ds, dtau, dmu;
            eta_partials(p, s, ds, dtau, dmu);
            const double eb = eta_bar[c];
            vt = eb * dtau;
            vm = eb * dmu;
            const double sb = s > 0.0 ? eb * ds / s : 0.0;   // d s / d G_dq = gamma_dq / s
            for (int d = 0; d < 3; d++)
                for (int q = 0; q < 3; q++) {
                    double gb = sb * (Gm[d][q] + Gm[q][d]);
                    if (G_bar) gb += G_bar[(3 * d + q) * N3 + c];
                    if (gb == 0.0) continue;
                    for (int r = 0; r < cnt[d]; r++) u_bar[q * N3 + idx[d][r]] += w[d][r] * gb;
                }
        }
    }
    vt = block_sum_lin<256>(vt);
    vm = block_sum_lin<256>(vm);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
        part[b] = vt;
        part[nb + b] = vm;
    }
}

// ---- wall-normal derivative (Eq. dudn) -----------------------------------------
// The stencil of cut cell t (the entries of geo.cut) for the wall-normal
// derivative, as k_wall_dudn forms it: with ok, 18 cells (two 3 x 3 planes
// along the normal's dominant axis); else, with near_ok, the one cell near.
struct WallSten {
    int kax, k1, k2, si, cc1[2], cc2[2], near[3], ci[3];
    double dist[2], L1[2][3], L2[2][3];
    bool ok, near_ok;
};
__device__ inline WallSten wall_stencil(const GridD &g, const GeomD &geo, int c)
{
    WallSten w;
    const int N3 = geo.ncell;
    w.ci[0] = c % g.nx; w.ci[1] = (c / g.nx) % g.ny; w.ci[2] = c / (g.nx * g.ny);
    double n[3], b[3];
    for (int e = 0; e < 3; e++) { n[e] = geo.nrm[e * N3 + c]; b[e] = geo.bcen[e * N3 + c]; }
    int kax = 0;
    if (fabs(n[1]) > fabs(n[kax])) kax = 1;
    if (fabs(n[2]) > fabs(n[kax])) kax = 2;
    w.kax = kax;
    w.k1 = (kax == 0) ? 1 : 0;
    w.k2 = (kax == 2) ? 1 : 2;
    const double s = n[kax] > 0.0 ? 1.0 : -1.0;
    w.si = n[kax] > 0.0 ? 1 : -1;
    w.dist[0] = (s - b[kax]) / n[kax];
    w.dist[1] = (2.0 * s - b[kax]) / n[kax];
    w.ok = true;
    for (int m = 0; m < 2; m++) {
        double P1 = b[w.k1] + w.dist[m] * n[w.k1], P2 = b[w.k2] + w.dist[m] * n[w.k2];
        w.cc1[m] = (int)floor(P1 + 0.5);
        w.cc2[m] = (int)floor(P2 + 0.5);
        double x1 = P1 - w.cc1[m], x2 = P2 - w.cc2[m];
        w.L1[m][0] = 0.5 * x1 * (x1 - 1.0); w.L1[m][1] = 1.0 - x1 * x1; w.L1[m][2] = 0.5 * x1 * (x1 + 1.0);
        w.L2[m][0] = 0.5 * x2 * (x2 - 1.0); w.L2[m][1] = 1.0 - x2 * x2; w.L2[m][2] = 0.5 * x2 * (x2 + 1.0);
        if (!w.ok) continue;
        for (int q1 = -1; q1 <= 1 && w.ok; q1++)
            for (int q2 = -1; q2 <= 1; q2++) {
                int id[3];
                id[kax] = w.ci[kax] + (m + 1) * w.si;
                id[w.k1] = w.ci[w.k1] + w.cc1[m] + q1;
                id[w.k2] = w.ci[w.k2] + w.cc2[m] + q2;
                if (!avail(g, geo.flag, id[0], id[1], id[2])) { w.ok = false; break; }
            }
    }
    w.near[kax] = w.ci[kax] + w.si;
    {
        double P1 = b[w.k1] + w.dist[0] * n[w.k1], P2 = b[w.k2] + w.dist[0] * n[w.k2];
        w.near[w.k1] = w.ci[w.k1] + (int)floor(P1 + 0.5);
        w.near[w.k2] = w.ci[w.k2] + (int)floor(P2 + 0.5);
    }
    w.near_ok = avail(g, geo.flag, w.near[0], w.near[1], w.near[2]);
    return w;
}
__device__ inline int wall_cell(const GridD &g, const WallSten &w, int m, int q1, int q2)
{
    int id[3];
    id[w.kax] = w.ci[w.kax] + (m + 1) * w.si;
    id[w.k1] = w.ci[w.k1] + w.cc1[m] + q1;
    id[w.k2] = w.ci[w.k2] + w.cc2[m] + q2;
    return cidx(g, id[0], id[1], id[2]);
}

// The cells each cut cell's stencil touches (kWallTargets per cut cell, -1
// unused): the host colours the cut cells so that no two of one colour share
// a target.
constexpr int kWallTargets = 18;
__global__ void k_wall_targets(GridD g, GeomD geo, int *__restrict__ tgt)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= geo.ncut) return;
    int *o = tgt + (size_t)t * kWallTargets;
    for (int r = 0; r < kWallTargets; r++) o[r] = -1;
    const int c = geo.cut[t];
    if (c < 0 || c >= geo.ncell) return;
    const WallSten w = wall_stencil(g, geo, c);
    if (w.ok) {
        int r = 0;
        for (int m = 0; m < 2; m++)
            for (int q1 = -1; q1 <= 1; q1++)
                for (int q2 = -1; q2 <= 1; q2++) o[r++] = wall_cell(g, w, m, q1, q2);
    } else if (w.near_ok) {
        o[0] = cidx(g, w.near[0], w.near[1], w.near[2]);
    }
}

// One colour of cut cells (list[0 .. n)): no two share a target, so plain
// additions, colour after colour, make u_bar bitwise reproducible.
__global__ void k_wall_dudn_adj(GridD g, GeomD geo, const int *__restrict__ list, int n,
                                const double *__restrict__ dudn_bar, double *__restrict__ u_bar)
{
    const int s_ = blockIdx.x * blockDim.x + threadIdx.x;
    if (s_ >= n) return;
    const int t = list[s_];
    const int N3 = geo.ncell;
    const int c = geo.cut[t];
    if (c < 0 || c >= N3) return;
    const WallSten w = wall_stencil(g, geo, c);
    const double d1 = w.dist[0], d2 = w.dist[1];
    for (int q = 0; q < 3; q++) {
        const double rb = dudn_bar[q * geo.ncut + t];
        if (rb == 0.0) continue;
        double *ubq = u_bar + q * N3;
        if (w.ok) {
            // r = (d2^2 uv0 - d1^2 uv1) / (d1 d2 (d2 - d1)) / h
            const double den = d1 * d2 * (d2 - d1);
            const double cm[2] = {d2 * d2 / den / g.h, -d1 * d1 / den / g.h};
            for (int m = 0; m < 2; m++)
                for (int q1 = -1; q1 <= 1; q1++)
                    for (int q2 = -1; q2 <= 1; q2++)
                        ubq[wall_cell(g, w, m, q1, q2)] += cm[m] * w.L1[m][q1 + 1] * w.L2[m][q2 + 1] * rb;
        } else if (w.near_ok) {
            ubq[cidx(g, w.near[0], w.near[1], w.near[2])] += rb / (d1 * g.h);
        }
    }
}

// ---- viscous face fluxes F_j = a_f eta_f d u_d / d x_j ---------------------
__global__ void __launch_bounds__(256) k_visc_flux_adj(GridD g, int d, const double *__restrict__ ap,
                                                       const double *__restrict__ u,
                                                       const double *__restrict__ eta,
                                                       const double *__restrict__ G,
                                                       const double *__restrict__ Fb, int nft, int off,
                                                       double *__restrict__ u_bar, double *__restrict__ eta_bar,
                                                       double *__restrict__ G_bar, int colour)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int mx = g.nx + (d == 0), my = g.ny + (d == 1), mz = g.nz + (d == 2);
    if (i >= mx || j >= my || k >= mz) return;
    const int pos = d == 0 ? i : (d == 1 ? j : k);
    if ((pos & 1) != colour) return;   // faces of one parity share no cell: plain additions
    const int f = fidx(g, d, i, j, k);
    const int N3 = ncell(g);
    const double a = ap[f];
    if (a <= 0.0) return;
    double fb[3];
    for (int jj = 0; jj < 3; jj++) fb[jj] = Fb[jj * nft + off + f];
    if (fb[0] == 0.0 && fb[1] == 0.0 && fb[2] == 0.0) return;
    int3 e = unit3(d);
    const double ih = g.ih;
    if (pos == 0 || pos == dimn(g, d)) {
        const int hs = pos != 0;
        const int c = cidx(g, i - hs * e.x, j - hs * e.y, k - hs * e.z);
        double val;
        const bool dir = side_dirichlet(g, 2 * d + hs, d, &val);
        if (dir) {
            // F_d = a eta_c (hs ? val - u_d : u_d - val) 2 / h
            const double ud = u[d * N3 + c];
            const double T = (hs ? (val - ud) : (ud - val)) * (2.0 * ih);
            eta_bar[c] += a * fb[d] * T;
            u_bar[d * N3 + c] += a * fb[d] * eta[c] * (hs ? -1.0 : 1.0) * (2.0 * ih);
        } else {
            // F_jj = a eta_c G[(3 jj + d)] for jj != d
            double eb = 0.0;
            for (int jj = 0; jj < 3; jj++) {
                if (jj == d) continue;
                eb += fb[jj] * G[(3 * jj + d) * N3 + c];
                G_bar[(3 * jj + d) * N3 + c] += a * eta[c] * fb[jj];
            }
            eta_bar[c] += a * eb;
        }
        return;
    }
    const int cL = cidx(g, i - e.x, j - e.y, k - e.z), cR = cidx(g, i, j, k);
    const double ef = 0.5 * (eta[cL] + eta[cR]);
    double efb = 0.0;
    for (int jj = 0; jj < 3; jj++) {
        const double der = (jj == d) ? (u[d * N3 + cR] - u[d * N3 + cL]) * ih
                                     : 0.5 * (G[(3 * jj + d) * N3 + cL] + G[(3 * jj + d) * N3 + cR]);
        efb += a * fb[jj] * der;
        const double derb = a * ef * fb[jj];
        if (jj == d) {
            u_bar[d * N3 + cR] += derb * ih;
            u_bar[d * N3 + cL] += -derb * ih;
        } else {
            G_bar[(3 * jj + d) * N3 + cL] += 0.5 * derb;
            G_bar[(3 * jj + d) * N3 + cR] += 0.5 * derb;
        }
    }
    eta_bar[cL] += 0.5 * efb;
    eta_bar[cR] += 0.5 * efb;
}

// ---- conservative divergence of a face flux triple ------------------------
// DC_q(c) = (sum over faces of +-F_q) / (alpha h) on fluid cells: the flux of
// face f enters its low cell with + and its high cell with -.
__global__ void k_flux_div_adj_faces(GridD g, int d, GeomD geo, const double *__restrict__ DCb, int nft,
                                     int off, double *__restrict__ Fb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int mx = g.nx + (d == 0), my = g.ny + (d == 1), mz = g.nz + (d == 2);
    if (i >= mx || j >= my || k >= mz) return;
    const int f = fidx(g, d, i, j, k);
    const int N3 = ncell(g);
    const int pos = d == 0 ? i : (d == 1 ? j : k);
    int3 e = unit3(d);
    auto sb = [&](int c, int q) -> double {
        if (geo.flag[c] == 0) return 0.0;
        const double inv = geo.flag[c] == 1 ? g.ih : 1.0 / (geo.alpha[c] * g.h);
        return DCb[q * N3 + c] * inv;
    };
    for (int q = 0; q < 3; q++) {
        double v = 0.0;
        if (pos > 0) v += sb(cidx(g, i - e.x, j - e.y, k - e.z), q);      // low cell: its high face
        if (pos < dimn(g, d)) v -= sb(cidx(g, i, j, k), q);               // high cell: its low face
        Fb[q * nft + off + f] = v;
    }
}

// The EB wall term of the viscous divergence, -eta n_q (n . du/dn) A_EB / (alpha h).
__global__ void k_flux_div_adj_wall(GridD g, GeomD geo, const double *__restrict__ DCb,
                                    const double *__restrict__ eta, const double *__restrict__ dudn,
                                    double *__restrict__ eta_bar, double *__restrict__ dudn_bar)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= geo.ncut) return;
    const int N3 = geo.ncell;
    const int c = geo.cut[t];
    if (geo.flag[c] != 2 || !(geo.area[c] > 0.0)) return;
    const double inv = 1.0 / (geo.alpha[c] * g.h);
    double n[3], sbn = 0.0, nd = 0.0;
    for (int q = 0; q < 3; q++) {
        n[q] = geo.nrm[q * N3 + c];
        sbn += DCb[q * N3 + c] * inv * n[q];
        nd += n[q] * dudn[q * geo.ncut + t];
    }
    const double A = geo.area[c];
    eta_bar[c] += -sbn * nd * A;
    for (int r = 0; r < 3; r++) dudn_bar[r * geo.ncut + t] += -eta[c] * A * n[r] * sbn;
}

// ---- redistribution ----------------------------------------------------------
// Forward: far cells out = sign DC / div; near cells (pass a) D = al DC +
// (1 - al) dnc, dD = al (1 - al)(DC - dnc), dnc = sum_nb alpha DC / sum_nb
// alpha, and (pass b) out = sign (D + sum over cut neighbours w dD) / div.
// kDiv: divide by div; without it div is 1 and no division is issued.
template <bool kDiv>
__global__ void k_redist_adj_far(GridD g, const uint8_t *__restrict__ flag, const uint8_t *__restrict__ near,
                                 const double *__restrict__ ob, double sign, double div, double *__restrict__ DCb)
{
    ADJ_CELL
    const int N3 = ncell(g);
    if (near[c]) return;
    for (int q = 0; q < 3; q++) DCb[q * N3 + c] = flag[c] ? sign * (kDiv ? ob[q * N3 + c] / div : ob[q * N3 + c]) : 0.0;
}

// Near cells: the adjoint of D (self) and, for cut cells, of dD (gathered from
// the fluid neighbours that add it) and of dnc (kept in tb, divided by the
// neighbour alpha sum, for k_redist_adj_b).
__global__ void __launch_bounds__(256) k_redist_adj_a(GridD g, const int *__restrict__ list, int nlist,
                                                      const uint8_t *__restrict__ flag,
                                                      const double *__restrict__ alpha,
                                                      const double *__restrict__ ob, double sign, double div,
                                                      double *__restrict__ DCb, double *__restrict__ tb)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nlist) return;
    const int c = list[t];
    const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    const int N3 = ncell(g);
    double Db[3];
    for (int q = 0; q < 3; q++) Db[q] = sign * ob[q * N3 + c] / div;
    if (flag[c] == 1) {
        for (int q = 0; q < 3; q++) { DCb[q * N3 + c] = Db[q]; tb[q * N3 + c] = 0.0; }
        return;
    }
    double sa = 0.0, dDb[3] = {0.0, 0.0, 0.0};
    for (int dk = -1; dk <= 1; dk++)
        for (int dj = -1; dj <= 1; dj++)
            for (int di = -1; di <= 1; di++) {
                if (!di && !dj && !dk) continue;
                if (!avail(g, flag, i + di, j + dj, k + dk)) continue;
                const int c2 = cidx(g, i + di, j + dj, k + dk);
                sa += alpha[c2];
                for (int q = 0; q < 3; q++) dDb[q] += sign * ob[q * N3 + c2] / div;
            }
    const double w = sa > 0.0 ? 1.0 / sa : 0.0;
    const double al = alpha[c];
    for (int q = 0; q < 3; q++) {
        const double ddb = w * dDb[q];
        double self = al * Db[q] + al * (1.0 - al) * ddb;
        const double dncb = (1.0 - al) * Db[q] - al * (1.0 - al) * ddb;
        double tq = 0.0;
        if (sa > 0.0) tq = dncb / sa;
        else self += dncb;
        DCb[q * N3 + c] = self;
        tb[q * N3 + c] = tq;
    }
}

__global__ void __launch_bounds__(256) k_redist_adj_b(GridD g, const int *__restrict__ list, int nlist,
                                                      const uint8_t *__restrict__ flag,
                                                      const double *__restrict__ alpha,
                                                      const double *__restrict__ tb, double *__restrict__ DCb)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nlist) return;
    const int c = list[t];
    const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    const int N3 = ncell(g);
    double s[3] = {0.0, 0.0, 0.0};
    for (int dk = -1; dk <= 1; dk++)
        for (int dj = -1; dj <= 1; dj++)
            for (int di = -1; di <= 1; di++) {
                if (!di && !dj && !dk) continue;
                if (!inbox(g, i + di, j + dj, k + dk)) continue;
                const int c2 = cidx(g, i + di, j + dj, k + dk);
                if (flag[c2] != 2) continue;
                for (int q = 0; q < 3; q++) s[q] += tb[q * N3 + c2];
            }
    const double al = alpha[c];
    for (int q = 0; q < 3; q++) DCb[q * N3 + c] += al * s[q];
}

// ---- implicit viscous operator: its dependence on eta ------------------------
// For A(eta) x = b(eta) solved for x, with lambda = A^-T xbar:
// eta_bar += lambda^T (db/deta - dA/deta x), gathered per cell over its faces
// (interior: B = dt/h^2 a (eta_L + eta_R)/2; Dirichlet box: 2 dt/h^2 a eta_c,
// also in b times the wall value) and its EB term dt eta A_EB / (h^2 delta).
__global__ void k_visc_eta_adj(GridD g, GeomD geo, ParamsD p, const double *__restrict__ dtp, int comp,
                               const double *__restrict__ lam, const double *__restrict__ x,
                               double *__restrict__ eta_bar)
{
    ADJ_CELL
    if (geo.flag[c] == 0) return;
    const int N3 = geo.ncell;
    const double h2 = g.h * g.h, dt = *dtp;
    const double dth2 = dt / h2;
    const double *A[3] = {geo.ax, geo.ay, geo.az};
    int id[3] = {i, j, k};
    const double lc = lam[c], xc = x[c];
    double eb = 0.0;
    for (int d = 0; d < 3; d++)
        for (int hs = 0; hs < 2; hs++) {
            const int pos = id[d] + hs;
            int fi[3] = {i, j, k};
            fi[d] += hs;
            const double a = A[d][fidx(g, d, fi[0], fi[1], fi[2])];
            if (!(a > 0.0)) continue;
            if (pos == 0 || pos == dimn(g, d)) {
                double val;
                if (side_dirichlet(g, 2 * d + hs, comp, &val)) eb += lc * 2.0 * dth2 * a * (val - xc);
            } else {
                int nb[3] = {i, j, k};
                nb[d] += hs ? 1 : -1;
                const int cn = cidx(g, nb[0], nb[1], nb[2]);
                eb += -0.5 * dth2 * a * (lc - lam[cn]) * (xc - x[cn]);
            }
        }
    if (geo.flag[c] == 2 && geo.area[c] > 0.0) {
        double nbv = 0.0;
        for (int q = 0; q < 3; q++) nbv += geo.nrm[q * N3 + c] * geo.bcen[q * N3 + c];
        const double del = -nbv > p.delta_min ? -nbv : p.delta_min;
        eb += -lc * xc * dt * geo.area[c] / (h2 * del);
    }
    eta_bar[c] += eb;
}

// ---- cell gradient of nodal p, transposed: node n gathers the weights
// (+-1/(4h)) it has in the gradients of its fluid cells, times w.
__global__ void k_gradp_t(GridD g, const uint8_t *__restrict__ flag, const double *__restrict__ w, double scale,
                          double *__restrict__ out, int accumulate)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int n = nidx(g, i, j, k);
    const int N3 = ncell(g);
    const double q4h = 0.25 * g.ih;
    double v = 0.0;
    for (int oc = 0; oc < 8; oc++) {
        const int ci = i - 1 + (oc & 1), cj = j - 1 + ((oc >> 1) & 1), ck = k - 1 + ((oc >> 2) & 1);
        if (!avail(g, flag, ci, cj, ck)) continue;
        const int c = cidx(g, ci, cj, ck);
        const int o[3] = {i - ci, j - cj, k - ck};
        for (int d = 0; d < 3; d++) v += (o[d] ? 1.0 : -1.0) * w[d * N3 + c];
    }
    v *= q4h * scale;
    out[n] = accumulate ? out[n] + v : v;
}

// ---- nodal right-hand side, transposed in ut: ub(d, c) += sum over the
// active corner nodes of alpha h^2/4 (+-1) rb(n) rho/dt.
__global__ void k_nodal_rhs_t(GridD g, GeomD geo, const uint8_t *__restrict__ act, const double *__restrict__ rb,
                              const double *__restrict__ dtp, double *__restrict__ ub)
{
    ADJ_CELL
    if (geo.flag[c] == 0) return;
    const int N3 = geo.ncell;
    const double h = g.h;
    const double wgt = geo.alpha[c] * h * h * 0.25 * dtp[DT_RHO_DT];
    double s[3] = {0.0, 0.0, 0.0};
    for (int oc = 0; oc < 8; oc++) {
        const int o[3] = {oc & 1, (oc >> 1) & 1, (oc >> 2) & 1};
        const int n = nidx(g, i + o[0], j + o[1], k + o[2]);
        if (!act[n]) continue;
        const double r = rb[n];
        for (int d = 0; d < 3; d++) s[d] += (o[d] ? 1.0 : -1.0) * r;
    }
    for (int d = 0; d < 3; d++) ub[d * N3 + c] += wgt * s[d];
}

// ---- drag (Eq. drag-force): adjoints of eta, du/dn and p, times wJ ---------------
// One launch per parity colour of the cut cell ((i & 1) + 2 (j & 1) + 4 (k & 1)):
// cells of one parity share no node, so the pressure adjoint takes plain
// additions (each cut cell's own entries are its alone).
__global__ void k_drag_adj(GridD g, GeomD geo, const double *__restrict__ eta, const double *__restrict__ dudn,
                           double wJ, double *__restrict__ eta_bar, double *__restrict__ dudn_bar,
                           double *__restrict__ p_bar, int colour)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= geo.ncut) return;
    const int N3 = geo.ncell;
    const int c = geo.cut[t];
    const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    if ((i & 1) + 2 * (j & 1) + 4 * (k & 1) != colour) return;
    double n[3], b[3], gq[3];
    for (int e = 0; e < 3; e++) {
        n[e] = geo.nrm[e * N3 + c];
        b[e] = geo.bcen[e * N3 + c];
        gq[e] = dudn[e * geo.ncut + t];
    }
    const double F = wJ * geo.area[c] * g.h * g.h;
    const double gn = gq[0] * n[0] + gq[1] * n[1] + gq[2] * n[2];
    eta_bar[c] += F * (n[2] * gn + gq[2]);
    for (int e = 0; e < 3; e++) dudn_bar[e * geo.ncut + t] += F * eta[c] * (n[2] * n[e] + (e == 2 ? 1.0 : 0.0));
    for (int o = 0; o < 8; o++) {
        const int oi = o & 1, oj = (o >> 1) & 1, ok = (o >> 2) & 1;
        const double w = (oi ? b[0] + 0.5 : 0.5 - b[0]) * (oj ? b[1] + 0.5 : 0.5 - b[1]) *
                         (ok ? b[2] + 0.5 : 0.5 - b[2]);
        p_bar[nidx(g, i + oi, j + oj, k + ok)] += -F * n[2] * w;
    }
}

// ---- convective term (Algorithm 2, advect = 1) -----------------------------------
// Forward: S = MC-limited slopes of u; uf = upwinded extrapolated normal
// velocities; MAC projection uF = uf - grad phi, A phi = D uf; F_q = a
// state_q uF with the state upwinded by uF; C = -R(div F).  The reverse
// pieces below take the branch each forward kernel took (the limiter's
// minimum, the Godunov case, the sign of uF), so they are exact wherever the
// forward is differentiable.

// Limited slope of f along d at (i,j,k) as a stencil (cells c-e, c, c+e):
// zero, dd/2, 2 dl or 2 dr by the forward's branch.
__device__ inline void mc_slope_w(const GridD &g, const uint8_t *flag, const double *f, int i, int j, int k, int d,
                                  int *idx, double *w)
{
    int3 e = unit3(d);
    idx[0] = cidx(g, i - e.x, j - e.y, k - e.z);
    idx[1] = cidx(g, i, j, k);
    idx[2] = cidx(g, i + e.x, j + e.y, k + e.z);
    w[0] = w[1] = w[2] = 0.0;
    if (!avail(g, flag, i + e.x, j + e.y, k + e.z) || !avail(g, flag, i - e.x, j - e.y, k - e.z)) return;
    const double f0 = f[idx[1]], fp = f[idx[2]], fm = f[idx[0]];
    const double dl = f0 - fm, dr = fp - f0, dd = fp - fm;
    if (dl == 0.0 || dr == 0.0 || (dl < 0.0) != (dr < 0.0)) return;
    // m = min(|dd|/2, 2|dl|, 2|dr|) with the sign of dd (dl, dr, dd share it)
    double m = fabs(0.5 * dd);
    int br = 0;
    if (2.0 * fabs(dl) < m) { m = 2.0 * fabs(dl); br = 1; }
    if (2.0 * fabs(dr) < m) { m = 2.0 * fabs(dr); br = 2; }
    if (br == 0) { w[2] = 0.5; w[0] = -0.5; }
    else if (br == 1) { w[1] = 2.0; w[0] = -2.0; }
    else { w[2] = 2.0; w[1] = -2.0; }
}

// One launch per colour (i + 2j + 3k) mod 7: a cell's slopes read itself and
// its two neighbours along each axis, and that map is one-to-one on those 7
// offsets mod 7, so cells of one colour share no target (plain additions).
constexpr int kSlopeColours = 7;
__global__ void __launch_bounds__(256) k_slopes_adj(GridD g, const uint8_t *__restrict__ flag,
                                                    const double *__restrict__ u, const double *__restrict__ Sb,
                                                    double *__restrict__ ub, int colour)
{
    ADJ_CELL
    if ((i + 2 * j + 3 * k) % kSlopeColours != colour) return;
    if (!flag[c]) return;
    const int N3 = ncell(g);
    for (int d = 0; d < 3; d++)
        for (int q = 0; q < 3; q++) {
            const double sb = Sb[(3 * d + q) * N3 + c];
            if (sb == 0.0) continue;
            int idx[3];
            double w[3];
            mc_slope_w(g, flag, u + q * N3, i, j, k, d, idx, w);
            for (int r = 0; r < 3; r++)
                if (w[r] != 0.0) ub[q * N3 + idx[r]] += w[r] * sb;
        }
}

// Face flux F_q = a state_q uF: adjoint of the state (to u, S) and of uF.
__global__ void __launch_bounds__(256) k_conv_flux_adj(GridD g, int d, const double *__restrict__ ap,
                                                       const double *__restrict__ u, const double *__restrict__ S,
                                                       const double *__restrict__ uFd,
                                                       const double *__restrict__ Fb, int nft, int off,
                                                       double *__restrict__ ub, double *__restrict__ Sb,
                                                       double *__restrict__ uFbd, int colour)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int mx = g.nx + (d == 0), my = g.ny + (d == 1), mz = g.nz + (d == 2);
    if (i >= mx || j >= my || k >= mz) return;
    const int pos = d == 0 ? i : (d == 1 ? j : k);
    if ((pos & 1) != colour) return;   // faces of one parity share no cell: plain additions
    const int f = fidx(g, d, i, j, k);
    const int N3 = ncell(g);
    const double a = ap[f];
    if (a <= 0.0) { uFbd[f] = 0.0; return; }
    const double w = uFd[f];
    int3 e = unit3(d);
    double wb = 0.0;
    if (pos == 0 || pos == dimn(g, d)) {
        const int hs = pos != 0;
        const int c = cidx(g, i - hs * e.x, j - hs * e.y, k - hs * e.z);
        const bool in = g.bc[2 * d + hs] == EBV_INFLOW;
        for (int q = 0; q < 3; q++) {
            const double fb = Fb[q * nft + off + f];
            const double state = in ? g.u_in[q] : u[q * N3 + c];
            wb += a * state * fb;
            if (!in) ub[q * N3 + c] += a * w * fb;
        }
        uFbd[f] = wb;
        return;
    }
    const int cL = cidx(g, i - e.x, j - e.y, k - e.z), cR = cidx(g, i, j, k);
    for (int q = 0; q < 3; q++) {
        const double fb = Fb[q * nft + off + f];
        const double sL = u[q * N3 + cL] + 0.5 * S[(3 * d + q) * N3 + cL];
        const double sR = u[q * N3 + cR] - 0.5 * S[(3 * d + q) * N3 + cR];
        const double state = w > 0.0 ? sL : (w < 0.0 ? sR : 0.5 * (sL + sR));
        wb += a * state * fb;
        const double stb = a * w * fb;
        const double wl = w > 0.0 ? 1.0 : (w < 0.0 ? 0.0 : 0.5), wr = 1.0 - wl;
        if (wl != 0.0 && stb != 0.0) {
            ub[q * N3 + cL] += wl * stb;
            Sb[(3 * d + q) * N3 + cL] += 0.5 * wl * stb;
        }
        if (wr != 0.0 && stb != 0.0) {
            ub[q * N3 + cR] += wr * stb;
            Sb[(3 * d + q) * N3 + cR] += -0.5 * wr * stb;
        }
    }
    uFbd[f] = wb;
}

// uF = uf - grad phi (faces with a > 0; outflow box faces with phi = 0 at the
// ghost, h/2 away): phi_bar(c) = sum over the cell's faces of d uF_f/d phi_c uF_bar_f.
__global__ void k_mac_correct_adj(GridD g, const double *__restrict__ ax, const double *__restrict__ ay,
                                  const double *__restrict__ az, const double *__restrict__ uFb,
                                  double *__restrict__ phib)
{
    ADJ_CELL
    const double *A[3] = {ax, ay, az};
    const int off[3] = {0, nface(g, 0), nface(g, 0) + nface(g, 1)};
    int id[3] = {i, j, k};
    double s = 0.0;
    for (int d = 0; d < 3; d++)
        for (int hs = 0; hs < 2; hs++) {
            int fi[3] = {i, j, k};
            fi[d] += hs;
            const int f = fidx(g, d, fi[0], fi[1], fi[2]);
            if (!(A[d][f] > 0.0)) continue;
            const double b = uFb[off[d] + f];
            const int pos = id[d] + hs;
            if (pos == 0 || pos == dimn(g, d)) {
                if (g.bc[2 * d + hs] != EBV_OUTFLOW && !pin_face(g, d, fi[0], fi[1], fi[2])) continue;
                // high side: uF -= (0 - phi) 2/h; low side: uF -= (phi - 0) 2/h
                s += (hs ? 1.0 : -1.0) * 2.0 * g.ih * b;
            } else {
                // interior: uF -= (phi_R - phi_L)/h; this cell is L on its high face, R on its low face
                s += (hs ? 1.0 : -1.0) * g.ih * b;
            }
        }
    phib[c] = s;
}

// b = -(1/h) sum (a uf) over the cell's faces (fluid cells): uf_bar += the transpose.
__global__ void k_mac_rhs_adj(GridD g, int d, const uint8_t *__restrict__ flag, const double *__restrict__ ap,
                              const double *__restrict__ bb, double *__restrict__ ufbd)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int mx = g.nx + (d == 0), my = g.ny + (d == 1), mz = g.nz + (d == 2);
    if (i >= mx || j >= my || k >= mz) return;
    const int f = fidx(g, d, i, j, k);
    const int pos = d == 0 ? i : (d == 1 ? j : k);
    int3 e = unit3(d);
    double v = 0.0;
    if (pos > 0) {  // low cell: this is its high face (+)
        const int cL = cidx(g, i - e.x, j - e.y, k - e.z);
        if (flag[cL]) v += bb[cL];
    }
    if (pos < dimn(g, d)) {  // high cell: its low face (-)
        const int cR = cidx(g, i, j, k);
        if (flag[cR]) v -= bb[cR];
    }
    ufbd[f] += -g.ih * ap[f] * v;
}

// Normal face velocity (extrapolated, Godunov upwinded; outflow box face: the
// cell value): its adjoint to u_d and S_dd.
__global__ void __launch_bounds__(256) k_face_states_adj(GridD g, int d, const double *__restrict__ ap,
                                                         const double *__restrict__ u, const double *__restrict__ S,
                                                         const double *__restrict__ ufbd, double *__restrict__ ub,
                                                         double *__restrict__ Sb, int colour)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int mx = g.nx + (d == 0), my = g.ny + (d == 1), mz = g.nz + (d == 2);
    if (i >= mx || j >= my || k >= mz) return;
    const int pos = d == 0 ? i : (d == 1 ? j : k);
    if ((pos & 1) != colour) return;   // faces of one parity share no cell: plain additions
    const int f = fidx(g, d, i, j, k);
    if (!(ap[f] > 0.0)) return;
    const double fb = ufbd[f];
    if (fb == 0.0) return;
    const int N3 = ncell(g);
    int3 e = unit3(d);
    if (pos == 0 || pos == dimn(g, d)) {
        const int hs = pos != 0;
        if (g.bc[2 * d + hs] == EBV_OUTFLOW)
            ub[d * N3 + cidx(g, i - hs * e.x, j - hs * e.y, k - hs * e.z)] += fb;
        return;
    }
    const int cL = cidx(g, i - e.x, j - e.y, k - e.z), cR = cidx(g, i, j, k);
    const double uL = u[d * N3 + cL] + 0.5 * S[(3 * d + d) * N3 + cL];
    const double uR = u[d * N3 + cR] - 0.5 * S[(3 * d + d) * N3 + cR];
    if (uL > 0.0 && uL + uR > 0.0) {
        ub[d * N3 + cL] += fb;
        Sb[(3 * d + d) * N3 + cL] += 0.5 * fb;
    } else if (uR < 0.0 && uL + uR < 0.0) {
        ub[d * N3 + cR] += fb;
        Sb[(3 * d + d) * N3 + cR] += -0.5 * fb;
    }
}

// ---- elementwise pieces ------------------------------------------------------------
// psi = rho u + dt (V - grad p + f) on fluid cells: u_bar += rho psi_bar,
// V_bar = vs psi_bar (or += when accumulating; vs is dt times the weight V
// has in psi), f_bar += dt psi_bar.
__global__ void k_psi_adj(int N3, const uint8_t *__restrict__ flag, const double *__restrict__ psib, double rho,
                          double dt, double vs, double *__restrict__ ub, double *__restrict__ Vb, int vb_acc,
                          double *__restrict__ fb, double *__restrict__ Cb)
{
    // psi also holds dt rho C (with V's weight): C_bar = rho vs psi_bar
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < 3 * N3; s += gridDim.x * blockDim.x) {
        const int c = s % N3;
        const double pb = flag[c] ? psib[s] : 0.0;
        ub[s] += rho * pb;
        Vb[s] = vb_acc ? Vb[s] + vs * pb : vs * pb;
        if (Cb) Cb[s] = vb_acc ? Cb[s] + rho * vs * pb : rho * vs * pb;
        if (fb) fb[s] += dt * pb;
    }
}

// a = s b on fluid cells, 0 on covered ones (ncomp components)
__global__ void k_mask_scale(int N3, int ncomp, const uint8_t *__restrict__ flag, const double *__restrict__ b,
                             double s, double *__restrict__ a)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ncomp * N3; e += gridDim.x * blockDim.x)
        a[e] = flag[e % N3] ? s * b[e] : 0.0;
}

// a = alpha lam on fluid cells (the adjoint of alpha psi)
__global__ void k_alpha_times(int N3, const uint8_t *__restrict__ flag, const double *__restrict__ alpha,
                              const double *__restrict__ lam, double *__restrict__ a)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N3; c += gridDim.x * blockDim.x)
        a[c] = flag[c] ? alpha[c] * lam[c] : 0.0;
}

__global__ void k_axpby(int n, double a, const double *__restrict__ x, double b, double *__restrict__ y)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) y[s] = a * x[s] + b * y[s];
}

__global__ void k_zero_where(int n, const uint8_t *__restrict__ act, double *__restrict__ x)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        if (!act[s]) x[s] = 0.0;
}

__global__ void __launch_bounds__(1024) k_sum2(const double *__restrict__ part, int n, double *__restrict__ out)
{
    double a = 0.0, b = 0.0;
    for (int s = threadIdx.x; s < n; s += 1024) {
        a += part[s];
        b += part[n + s];
    }
    __shared__ double sa[32], sb[32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { sa[threadIdx.x >> 5] = a; sb[threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x < 32) {
        a = sa[threadIdx.x];
        b = sb[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        if (threadIdx.x == 0) { out[0] += a; out[1] += b; }
    }
}

inline int eblocks(long long n) { return (int)std::min<long long>(kReduceBlocks, (n + 255) / 256); }

}  // namespace

// ===========================================================================
// Launchers (reverse pieces); all on the context stream.
// ===========================================================================

// (eta_bar, G_bar) -> u_bar += ..., grads_dev[0] += d/dtau0, grads_dev[1] += d/dmu
ebv_status adj_strain_eta(Ctx *c, const double *u, const double *eta_bar, const double *G_bar, double *u_bar,
                          double *grads_dev)
{
    const GridD &g = c->g;
    const dim3 gr = grid3((g.nx + kSeColours - 1) / kSeColours, g.ny, g.nz);   // one colour's cells per launch
    const int nb = gr.x * gr.y * gr.z;
    if (2 * (size_t)nb > ((size_t)1 << 20)) return c->fail(EBV_ERR_INVALID, "grid too large for the partial sums");
    for (int q = 0; q < kSeColours; q++) {   // colour by colour, each reduced in turn (fixed order)
        EBV_LAUNCH(c, k_se_adj, gr, block3(), 0, g, c->flag, u, paramsd(c->prm), eta_bar, G_bar, u_bar, c->part,
                   q);
        EBV_LAUNCH(c, k_sum2, dim3(1), dim3(1024), 0, c->part, nb, grads_dev);
    }
    return EBV_OK;
}

// Colours of the cut cells for the wall-gradient adjoint, once per geometry:
// greedy in cut-list order, a cell takes the first colour no earlier cell
// sharing one of its stencil cells has; the lists hold each colour's cut
// indices in ascending order.
ebv_status wall_colouring(Ctx *c)
{
    if (c->wall_col_ok) return EBV_OK;
    const int n = c->ncut;
    c->wall_col_off.assign(1, 0);
    if (c->wall_col) cudaFree(c->wall_col);
    c->wall_col = nullptr;
    if (n) {
        int *tgt_dev = nullptr;
        EBV_CUDA_TRY(c, dev_malloc((void **)&tgt_dev, (size_t)n * kWallTargets * sizeof(int)));
        EBV_LAUNCH(c, k_wall_targets, dim3((n + 127) / 128), dim3(128), 0, c->g, geomd(c), tgt_dev);
        std::vector<int> tgt((size_t)n * kWallTargets);
        cudaError_t e = cudaMemcpyAsync(tgt.data(), tgt_dev, tgt.size() * sizeof(int), cudaMemcpyDeviceToHost,
                                        c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(tgt_dev);
        EBV_CUDA_TRY(c, e);
        std::unordered_map<int, std::vector<int>> used;   // stencil cell -> colours of the cut cells touching it
        std::vector<int> col(n);
        int ncol = 0;
        std::vector<char> taken;
        for (int t = 0; t < n; t++) {
            taken.assign(ncol + 1, 0);
            for (int r = 0; r < kWallTargets; r++) {
                const int x = tgt[(size_t)t * kWallTargets + r];
                if (x < 0) continue;
                auto it = used.find(x);
                if (it != used.end())
                    for (int q : it->second) taken[q] = 1;
            }
            int q = 0;
            while (taken[q]) q++;
            col[t] = q;
            ncol = std::max(ncol, q + 1);
            for (int r = 0; r < kWallTargets; r++) {
                const int x = tgt[(size_t)t * kWallTargets + r];
                if (x >= 0) used[x].push_back(q);
            }
        }
        c->wall_col_off.assign(ncol + 1, 0);
        for (int t = 0; t < n; t++) c->wall_col_off[col[t] + 1]++;
        for (int q = 0; q < ncol; q++) c->wall_col_off[q + 1] += c->wall_col_off[q];
        std::vector<int> list(n), pos(c->wall_col_off.begin(), c->wall_col_off.end() - 1);
        for (int t = 0; t < n; t++) list[pos[col[t]]++] = t;
        EBV_CUDA_TRY(c, dev_malloc((void **)&c->wall_col, (size_t)n * sizeof(int)));
        EBV_CUDA_TRY(c, cudaMemcpy(c->wall_col, list.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice));
    }
    c->wall_col_ok = true;
    return EBV_OK;
}

ebv_status adj_wall_dudn(Ctx *c, const double *dudn_bar, double *u_bar)
{
    if (!c->ncut) return EBV_OK;
    const ebv_status st = wall_colouring(c);
    if (st != EBV_OK) return st;
    const int nc = (int)c->wall_col_off.size() - 1;
    for (int q = 0; q < nc; q++) {
        const int n = c->wall_col_off[q + 1] - c->wall_col_off[q];
        EBV_LAUNCH(c, k_wall_dudn_adj, dim3((n + 127) / 128), dim3(128), 0, c->g, geomd(c),
                   c->wall_col + c->wall_col_off[q], n, dudn_bar, u_bar);
    }
    return EBV_OK;
}

// V = R(FD(VF(u, eta, G), eta, dudn(u))) / rho: V_bar -> u_bar, eta_bar, G_bar
// (all accumulated).  Work: Fb (3 x faces), DCb, tb (3 x cells), dudn_bar
// (3 x cut cells).
ebv_status adj_viscous_explicit(Ctx *c, const double *u, const double *eta, const double *G, const double *V_bar,
                                double *u_bar, double *eta_bar, double *G_bar, double *Fb, double *DCb, double *tb,
                                double *dudn_bar)
{
    const GridD &g = c->g;
    GeomD geo = geomd(c);
    const int nft = nface(g, 0) + nface(g, 1) + nface(g, 2);
    // forward wall gradients of u (read by the wall term's adjoint)
    ebv_status st = launch_wall_dudn(c, u, c->dudn);
    if (st != EBV_OK) return st;
    // redistribution (sign +1, divided by rho)
    if (c->prm.rho != 1.0)
        EBV_LAUNCH(c, k_redist_adj_far<true>, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, c->nearm, V_bar, 1.0,
                   c->prm.rho, DCb);
    else
        EBV_LAUNCH(c, k_redist_adj_far<false>, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, c->nearm, V_bar, 1.0,
                   c->prm.rho, DCb);
    if (c->nnear) {
        dim3 gr((c->nnear + 127) / 128);
        EBV_LAUNCH(c, k_redist_adj_a, gr, dim3(128), 0, g, c->nearl, c->nnear, c->flag, c->alpha, V_bar, 1.0,
                   c->prm.rho, DCb, tb);
        EBV_LAUNCH(c, k_redist_adj_b, gr, dim3(128), 0, g, c->nearl, c->nnear, c->flag, c->alpha, tb, DCb);
    }
    // divergence: faces and the EB wall term
    const double *A[3] = {c->ax, c->ay, c->az};
    int off = 0;
    for (int d = 0; d < 3; d++) {
        EBV_LAUNCH(c, k_flux_div_adj_faces, grid3(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)), block3(), 0, g,
                   d, geo, DCb, nft, off, Fb);
        off += nface(g, d);
    }
    if (c->ncut) {
        EBV_CUDA_TRY(c, cudaMemsetAsync(dudn_bar, 0, 3 * (size_t)c->ncut * sizeof(double), c->stream));
        EBV_LAUNCH(c, k_flux_div_adj_wall, dim3((c->ncut + 127) / 128), dim3(128), 0, g, geo, DCb, eta, c->dudn,
                   eta_bar, dudn_bar);
        if ((st = adj_wall_dudn(c, dudn_bar, u_bar)) != EBV_OK) return st;
    }
    // face fluxes
    off = 0;
    for (int d = 0; d < 3; d++) {
        for (int q = 0; q < 2; q++)   // even, then odd face positions
            EBV_LAUNCH(c, k_visc_flux_adj, grid3(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)), block3(), 0, g,
                       d, A[d], u, eta, G, Fb, nft, off, u_bar, eta_bar, G_bar, q);
        off += nface(g, d);
    }
    return EBV_OK;
}

// C(u) = -R(div F(u, S(u), uF(u))): ub += (dC/du)^T Cb.  S: the forward
// slopes of u, uF: its projected face velocities.  Work: DCb, tb (3 x cells),
// Fb (3 x faces), Sb (9 x cells), uFb (faces), phib, bb (cells).
ebv_status adj_convective(Ctx *c, const double *u, const double *S, const double *uF, const double *Cb, double *ub,
                          double *DCb, double *tb, double *Fb, double *Sb, double *uFb, double *phib, double *bb)
{
    const GridD &g = c->g;
    GeomD geo = geomd(c);
    const int N3 = ncell(g), nft = nface(g, 0) + nface(g, 1) + nface(g, 2);
    const int offs[3] = {0, nface(g, 0), nface(g, 0) + nface(g, 1)};
    const double *A[3] = {c->ax, c->ay, c->az};
    // redistribution (sign -1, no division) and the divergence
    EBV_LAUNCH(c, k_redist_adj_far<false>, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, c->nearm, Cb, -1.0, 1.0,
               DCb);
    if (c->nnear) {
        dim3 gr((c->nnear + 127) / 128);
        EBV_LAUNCH(c, k_redist_adj_a, gr, dim3(128), 0, g, c->nearl, c->nnear, c->flag, c->alpha, Cb, -1.0, 1.0, DCb,
                   tb);
        EBV_LAUNCH(c, k_redist_adj_b, gr, dim3(128), 0, g, c->nearl, c->nnear, c->flag, c->alpha, tb, DCb);
    }
    for (int d = 0; d < 3; d++)
        EBV_LAUNCH(c, k_flux_div_adj_faces, grid3(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)), block3(), 0, g,
                   d, geo, DCb, nft, offs[d], Fb);
    // fluxes: to u, S and the projected face velocities
    EBV_CUDA_TRY(c, cudaMemsetAsync(Sb, 0, 9 * (size_t)N3 * sizeof(double), c->stream));
    for (int d = 0; d < 3; d++)
        for (int q = 0; q < 2; q++)   // even, then odd face positions
            EBV_LAUNCH(c, k_conv_flux_adj, grid3(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)), block3(), 0, g,
                       d, A[d], u, S, uF + offs[d], Fb, nft, offs[d], ub, Sb, uFb + offs[d], q);
    // MAC projection: phi_bar, the adjoint solve, then the face divergence
    EBV_LAUNCH(c, k_mac_correct_adj, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->ax, c->ay, c->az, uFb, phib);
    int it = 0;
    double res = 0.0;
    c->cur_slot = 11;
    ebv_status st = mac_solve(c, phib, bb, &it, &res);
    if (st != EBV_OK) return st;
    for (int d = 0; d < 3; d++)
        EBV_LAUNCH(c, k_mac_rhs_adj, grid3(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)), block3(), 0, g, d,
                   c->flag, A[d], bb, uFb + offs[d]);
    // face states and slopes
    for (int d = 0; d < 3; d++)
        for (int q = 0; q < 2; q++)   // even, then odd face positions
            EBV_LAUNCH(c, k_face_states_adj, grid3(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)), block3(), 0,
                       g, d, A[d], u, S, uFb + offs[d], ub, Sb, q);
    for (int q = 0; q < kSlopeColours; q++)
        EBV_LAUNCH(c, k_slopes_adj, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, u, Sb, ub, q);
    return EBV_OK;
}

ebv_status adj_visc_eta(Ctx *c, int comp, const double *lam, const double *x, double *eta_bar)
{
    const GridD &g = c->g;
    EBV_LAUNCH(c, k_visc_eta_adj, grid3(g.nx, g.ny, g.nz), block3(), 0, g, geomd(c), paramsd(c->prm), c->dt_dev,
               comp, lam, x, eta_bar);
    return EBV_OK;
}

ebv_status adj_gradp_t(Ctx *c, const double *w, double scale, double *out, int accumulate)
{
    const GridD &g = c->g;
    EBV_LAUNCH(c, k_gradp_t, grid3(g.nx + 1, g.ny + 1, g.nz + 1), block3(), 0, g, c->flag, w, scale, out,
               accumulate);
    return EBV_OK;
}

ebv_status adj_nodal_rhs_t(Ctx *c, const double *rb, double *ub)
{
    const GridD &g = c->g;
    EBV_LAUNCH(c, k_nodal_rhs_t, grid3(g.nx, g.ny, g.nz), block3(), 0, g, geomd(c), c->nd.lv[0].act, rb, c->dt_dev,
               ub);
    return EBV_OK;
}

ebv_status adj_drag(Ctx *c, const double *eta, double wJ, double *eta_bar, double *dudn_bar, double *p_bar)
{
    if (c->ncut)
        for (int q = 0; q < 8; q++)   // parity colours of the cut cells
            EBV_LAUNCH(c, k_drag_adj, dim3((c->ncut + 127) / 128), dim3(128), 0, c->g, geomd(c), eta, c->dudn, wJ,
                       eta_bar, dudn_bar, p_bar, q);
    return EBV_OK;
}

ebv_status adj_psi(Ctx *c, const double *psib, double dt, double vs, double *ub, double *Vb, int vb_acc, double *fb,
                   double *Cb)
{
    const int N3 = ncell(c->g);
    EBV_LAUNCH(c, k_psi_adj, dim3(eblocks(3LL * N3)), dim3(256), 0, N3, c->flag, psib, c->prm.rho, dt, vs, ub, Vb,
               vb_acc, fb, Cb);
    return EBV_OK;
}

ebv_status adj_mask_scale(Ctx *c, int ncomp, const double *b, double s, double *a)
{
    const int N3 = ncell(c->g);
    EBV_LAUNCH(c, k_mask_scale, dim3(eblocks((long long)ncomp * N3)), dim3(256), 0, N3, ncomp, c->flag, b, s, a);
    return EBV_OK;
}

ebv_status adj_alpha_times(Ctx *c, const double *lam, double *a)
{
    const int N3 = ncell(c->g);
    EBV_LAUNCH(c, k_alpha_times, dim3(eblocks(N3)), dim3(256), 0, N3, c->flag, c->alpha, lam, a);
    return EBV_OK;
}

ebv_status adj_axpby(Ctx *c, int n, double a, const double *x, double b, double *y)
{
    EBV_LAUNCH(c, k_axpby, dim3(eblocks(n)), dim3(256), 0, n, a, x, b, y);
    return EBV_OK;
}

ebv_status adj_zero_inactive_nodes(Ctx *c, double *x)
{
    const int NN = nnode(c->g);
    EBV_LAUNCH(c, k_zero_where, dim3(eblocks(NN)), dim3(256), 0, NN, c->nd.lv[0].act, x);
    return EBV_OK;
}

}  // namespace ebv
