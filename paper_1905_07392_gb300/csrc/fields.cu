// Streaming kernels of one Runge-Kutta stage (paper Algorithm 2 and the
// explicit parts of Algorithm 1).  One thread per cell, face or node; the
// kernels read their stencils straight from HBM/L2 (no ghost cells) and keep
// every value FP64.
#include "ebv_internal.cuh"

namespace ebv {
namespace {

__device__ inline int3 unit(int d) { return make_int3(d == 0, d == 1, d == 2); }

// The monotonised-central limiter on the differences dl = f0 - fm,
// dr = fp - f0 and dd = fp - fm of one cell and axis.
__device__ inline double mc_limit(double dl, double dr, double dd)
{
    // The limiter  m = min(|dd|/2, 2|dl|, 2|dr|)  only scales by powers of
    // two and compares, so on normal numbers it is exact on the IEEE bit
    // patterns: the integer pipe does it and FP64 issues just the three
    // differences.  dl*dr <= 0 is read off the sign bits (the product of two
    // nonzero differences of O(1) data does not underflow).
    // The 64-bit patterns are handled as (high, low) 32-bit words: the
    // exponent steps (x4, /2) only touch the high word, and a 64-bit
    // comparison is one of the high words, then of the low words on a tie:
    // the same results as 64-bit integer arithmetic (tests/test_kernel_models.py
    // checks the two forms against each other, zeros, subnormals and equal
    // high words included), which on this GPU runs at about the FP64 rate.
    const unsigned kS = 0x80000000u, kE1 = 1u << 20;   // sign bit, one exponent step
    const unsigned lh = (unsigned)__double2hiint(dl), ll = (unsigned)__double2loint(dl);
    const unsigned rh = (unsigned)__double2hiint(dr), rl = (unsigned)__double2loint(dr);
    const unsigned dh = (unsigned)__double2hiint(dd), dlo = (unsigned)__double2loint(dd);
    const unsigned alh = lh & ~kS, arh = rh & ~kS, adh = dh & ~kS;
    if ((alh | ll) == 0u || (arh | rl) == 0u || ((lh ^ rh) & kS)) return 0.0;
    // exponent fields in [3, 2044]: x4 and /2 stay normal and finite
    const unsigned lo = 3u * kE1, hi = 2044u * kE1;
    if (alh < lo || arh < lo || ((adh | dlo) != 0u && adh < lo) || alh >= hi || arh >= hi || adh >= hi) {
        double m = fabs(0.5 * dd);
        m = fmin(m, 2.0 * fabs(dl));
        m = fmin(m, 2.0 * fabs(dr));
        return dd > 0.0 ? m : -m;
    }
    // m4 = min(|dd|, 4|dl|, 4|dr|) on the patterns
    unsigned mh = alh + 2u * kE1, ml = ll;
    const unsigned bh = arh + 2u * kE1;
    if (bh < mh || (bh == mh && rl < ml)) { mh = bh; ml = rl; }
    if (adh < mh || (adh == mh && dlo < ml)) { mh = adh; ml = dlo; }
    if ((mh | ml) != 0u) mh -= kE1;                      // halved
    // the sign of dd when dd > 0 as a 64-bit pattern, else negative
    const bool pos = !(dh & kS) && (dh | dlo) != 0u;
    return __hiloint2double((int)(pos ? mh : (mh | kS)), (int)ml);
}

// Godunov state of Burgers' equation from the two extrapolated normal velocities.
__device__ inline double upwind_normal(double uL, double uR)
{
    if (uL > 0.0 && uL + uR > 0.0) return uL;
    if (uR < 0.0 && uL + uR < 0.0) return uR;
    return 0.0;
}

// Robust cell-centred derivative along d (paper Sec. "Strain rate tensor and
// apparent viscosity"): central, one-sided quadratic next to a covered cell,
// first order with a single neighbour, zero without one.
__device__ inline double d_robust(const GridD &g, const uint8_t *flag, const double *f, int i,
                                  int j, int k, int d, double ih)
{
    int3 e = unit(d);
    bool ip = avail(g, flag, i + e.x, j + e.y, k + e.z);
    bool im = avail(g, flag, i - e.x, j - e.y, k - e.z);
    double f0 = f[cidx(g, i, j, k)];
    if (ip && im)
        return (f[cidx(g, i + e.x, j + e.y, k + e.z)] - f[cidx(g, i - e.x, j - e.y, k - e.z)]) *
               (0.5 * ih);
    if (im) {
        double f1 = f[cidx(g, i - e.x, j - e.y, k - e.z)];
        if (avail(g, flag, i - 2 * e.x, j - 2 * e.y, k - 2 * e.z)) {
            double f2 = f[cidx(g, i - 2 * e.x, j - 2 * e.y, k - 2 * e.z)];
            return (0.5 * f2 - 2.0 * f1 + 1.5 * f0) * ih;
        }
        return (f0 - f1) * ih;
    }
    if (ip) {
        double f1 = f[cidx(g, i + e.x, j + e.y, k + e.z)];
        if (avail(g, flag, i + 2 * e.x, j + 2 * e.y, k + 2 * e.z)) {
            double f2 = f[cidx(g, i + 2 * e.x, j + 2 * e.y, k + 2 * e.z)];
            return (-1.5 * f0 + 2.0 * f1 - 0.5 * f2) * ih;
        }
        return (f1 - f0) * ih;
    }
    return 0.0;
}

#define CELL_INDEX                                         \
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   \
    const int j = blockIdx.y * blockDim.y + threadIdx.y;   \
    const int k = blockIdx.z * blockDim.z + threadIdx.z;   \
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;       \
    const int c = cidx(g, i, j, k);

// The apparent viscosity of eta_of in FP32 (EBV_FP32_MIXED, cells away from
// the EB): the same laws and branches, FP32 arithmetic and math functions.
__device__ inline float eta_of_f(const ParamsD &p, float sr, float rsr)
{
    const float m = (float)p.m, mu = (float)p.mu, tau0 = (float)p.tau0, nf = (float)p.n_flow;
    const float msr = m * sr;
    const float yield = (sr > 0.f) ? (msr > 20.f ? 1.f : -expm1f(-msr)) * rsr : m;
    const float srf = sr > (float)p.inv_m ? sr : (float)p.inv_m;
    switch (p.model) {
    case EBV_NEWTONIAN: return mu;
    case EBV_BINGHAM: return mu + tau0 * yield;
    case EBV_HERSCHEL_BULKLEY: return mu * powf(srf, nf - 1.f) + tau0 * yield;
    case EBV_POWER_LAW: return mu * powf(srf, nf - 1.f);
    case EBV_SOUZA_MENDES_DUTRA: {
        const float y2 = (sr > 0.f) ? -expm1f(-(float)p.eta0 * sr / tau0) * rsr : (float)p.eta0 / tau0;
        return mu * powf(srf, nf - 1.f) + tau0 * y2;
    }
    }
    return mu;
}

// ---- fused strain rate + apparent viscosity (optionally the gradient) -----
// kMixed (EBV_FP32_MIXED): cells whose six neighbours are fluid and that are
// neither cut nor next to a cut cell (nearm) form the central differences of
// u in FP64 (they cancel: u is O(1), its differences small) and the rest --
// the scaling by 1/(2h), the strain-rate norm, its reciprocal square root and
// the viscosity law -- in FP32; every other cell takes the FP64 path.  (The
// conversions between the two cost about what the FP64 arithmetic they
// replace did, here and with integer bit-field conversions, measured.)
template <bool kWriteG, bool kMixed = false>
__global__ void __launch_bounds__(256) k_strain_eta(GridD g, const uint8_t *__restrict__ flag,
                                                    const double *__restrict__ u, ParamsD p,
                                                    double *__restrict__ eta,
                                                    double *__restrict__ srate,
                                                    double *__restrict__ G,
                                                    const uint8_t *__restrict__ nearm = nullptr)
{
    CELL_INDEX
    const int N3 = ncell(g);
    if (flag[c] == 0) {
        eta[c] = 0.0;
        if (srate) srate[c] = 0.0;
        if (kWriteG)
            for (int q = 0; q < 9; q++) G[q * N3 + c] = 0.0;
        return;
    }
    if constexpr (kMixed) {
        const int sy = g.nx, sz = g.nx * g.ny;
        if (!nearm[c] && i > 0 && i < g.nx - 1 && j > 0 && j < g.ny - 1 && k > 0 && k < g.nz - 1 &&
            flag[c - 1] && flag[c + 1] && flag[c - sy] && flag[c + sy] && flag[c - sz] && flag[c + sz]) {
            const int st[3] = {1, sy, sz};
            const float hf = (float)(0.5 * g.ih);
            float Gf[3][3];
#pragma unroll
            for (int d = 0; d < 3; d++)
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    const double *uq = u + q * N3;
                    Gf[d][q] = (float)(uq[c + st[d]] - uq[c - st[d]]) * hf;
                }
            const float xy = Gf[0][1] + Gf[1][0], xz = Gf[0][2] + Gf[2][0], yz = Gf[1][2] + Gf[2][1];
            const float s = 2.f * (Gf[0][0] * Gf[0][0] + Gf[1][1] * Gf[1][1] + Gf[2][2] * Gf[2][2]) +
                            (xy * xy + xz * xz + yz * yz);
            const float rsr = s > 0.f ? rsqrtf(s) : 0.f;
            const float sr = s * rsr;
            eta[c] = (double)eta_of_f(p, sr, rsr);
            if (srate) srate[c] = (double)sr;
            if (kWriteG)
#pragma unroll
                for (int d = 0; d < 3; d++)
#pragma unroll
                    for (int q = 0; q < 3; q++) G[(3 * d + q) * N3 + c] = (double)Gf[d][q];
            return;
        }
    }
    double Gm[3][3];
    const double ih = g.ih;
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int q = 0; q < 3; q++) Gm[d][q] = d_robust(g, flag, u + q * N3, i, j, k, d, ih);
    // sr^2 = |G + G^T|^2 / 2 = 2 (G_00^2 + G_11^2 + G_22^2) + the squares of
    // the three off-diagonal sums; sr and 1/sr from one reciprocal square root
    const double xy = Gm[0][1] + Gm[1][0], xz = Gm[0][2] + Gm[2][0], yz = Gm[1][2] + Gm[2][1];
    const double s = 2.0 * (Gm[0][0] * Gm[0][0] + Gm[1][1] * Gm[1][1] + Gm[2][2] * Gm[2][2]) +
                     (xy * xy + xz * xz + yz * yz);
    const double rsr = s > 0.0 ? rsqrt(s) : 0.0;
    const double sr = s * rsr;
    eta[c] = eta_of(p, sr, rsr);
    if (srate) srate[c] = sr;
    if (kWriteG)
#pragma unroll
        for (int d = 0; d < 3; d++)
#pragma unroll
            for (int q = 0; q < 3; q++) G[(3 * d + q) * N3 + c] = Gm[d][q];
}

// ---- flow diagnostics (Sec. "Cylinder moving through Bingham fluid") ------
// Lambda of Eq. ryovar, (||g||^2 - |w|^2) / (||g||^2 + |w|^2) with w = curl u
// (0 where both vanish), and the yield-stress deviation eta ||g|| / tau0 - 1
// (0 when tau0 = 0), from the same robust gradients as k_strain_eta.
__global__ void __launch_bounds__(256) k_flow_diag(GridD g, const uint8_t *__restrict__ flag,
                                                   const double *__restrict__ u, ParamsD p,
                                                   double *__restrict__ lam, double *__restrict__ sdev)
{
    CELL_INDEX
    const int N3 = ncell(g);
    if (flag[c] == 0) {
        lam[c] = 0.0;
        sdev[c] = 0.0;
        return;
    }
    double Gm[3][3];
    const double ih = g.ih;
#pragma unroll
    for (int d = 0; d < 3; d++)
#pragma unroll
        for (int q = 0; q < 3; q++) Gm[d][q] = d_robust(g, flag, u + q * N3, i, j, k, d, ih);
    const double xy = Gm[0][1] + Gm[1][0], xz = Gm[0][2] + Gm[2][0], yz = Gm[1][2] + Gm[2][1];
    const double s = 2.0 * (Gm[0][0] * Gm[0][0] + Gm[1][1] * Gm[1][1] + Gm[2][2] * Gm[2][2]) +
                     (xy * xy + xz * xz + yz * yz);   // ||g||^2
    const double wx = Gm[1][2] - Gm[2][1], wy = Gm[2][0] - Gm[0][2], wz = Gm[0][1] - Gm[1][0];
    const double w2 = wx * wx + wy * wy + wz * wz;
    lam[c] = (s + w2) > 0.0 ? (s - w2) / (s + w2) : 0.0;
    const double rsr = s > 0.0 ? rsqrt(s) : 0.0;
    const double sr = s * rsr;
    sdev[c] = p.tau0 > 0.0 ? eta_of(p, sr, rsr) * sr / p.tau0 - 1.0 : 0.0;
}

// ---- normal face velocities (slopes, extrapolation, upwinding) ------------
__global__ void k_face_states(GridD g, int d, const double *__restrict__ S,
                              const double *__restrict__ ap, const double *__restrict__ u,
                              double *__restrict__ uf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int mx = g.nx + (d == 0), my = g.ny + (d == 1), mz = g.nz + (d == 2);
    if (i >= mx || j >= my || k >= mz) return;
    const int f = fidx(g, d, i, j, k);
    const int N3 = ncell(g);
    const double *ud = u + d * N3;
    int id[3] = {i, j, k};
    double v = 0.0;
    if (ap[f] > 0.0) {
        if (id[d] == 0 || id[d] == dimn(g, d)) {
            int hs = id[d] != 0;
            int side = 2 * d + hs;
            int cc[3] = {i, j, k};
            cc[d] -= hs;
            if (g.bc[side] == EBV_INFLOW) v = g.u_in[d];
            else if (g.bc[side] == EBV_OUTFLOW) v = ud[cidx(g, cc[0], cc[1], cc[2])];
        } else {
            int3 e = unit(d);
            const int cL = cidx(g, i - e.x, j - e.y, k - e.z), cR = cidx(g, i, j, k);
            const double *Sd = S + (3 * d + d) * N3;
            double uL = ud[cL] + 0.5 * Sd[cL];
            double uR = ud[cR] - 0.5 * Sd[cR];
            v = upwind_normal(uL, uR);
        }
    }
    uf[f] = v;
}

// ---- cell-centred projection: right-hand side and face correction ---------
__global__ void k_mac_rhs(GridD g, const uint8_t *__restrict__ flag, const double *__restrict__ ax,
                          const double *__restrict__ ay, const double *__restrict__ az,
                          const double *__restrict__ ufx, const double *__restrict__ ufy,
                          const double *__restrict__ ufz, double *__restrict__ b)
{
    CELL_INDEX
    if (flag[c] == 0) { b[c] = 0.0; return; }
    const double *A[3] = {ax, ay, az};
    const double *U[3] = {ufx, ufy, ufz};
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        int3 e = unit(d);
        int flo = fidx(g, d, i, j, k), fhi = fidx(g, d, i + e.x, j + e.y, k + e.z);
        s += A[d][fhi] * U[d][fhi] - A[d][flo] * U[d][flo];
    }
    b[c] = -s * g.ih;
}

__global__ void k_mac_correct(GridD g, int d, const double *__restrict__ ap,
                              const double *__restrict__ phi, double *__restrict__ uf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int mx = g.nx + (d == 0), my = g.ny + (d == 1), mz = g.nz + (d == 2);
    if (i >= mx || j >= my || k >= mz) return;
    const int f = fidx(g, d, i, j, k);
    if (ap[f] <= 0.0) return;
    int id[3] = {i, j, k};
    if (id[d] == 0 || id[d] == dimn(g, d)) {
        int hs = id[d] != 0;
        if (g.bc[2 * d + hs] != EBV_OUTFLOW && !pin_face(g, d, i, j, k)) return;
        int cc[3] = {i, j, k};
        cc[d] -= hs;
        double pc = phi[cidx(g, cc[0], cc[1], cc[2])];
        double grad = hs ? (0.0 - pc) * (2.0 * g.ih) : (pc - 0.0) * (2.0 * g.ih);
        uf[f] -= grad;
    } else {
        int3 e = unit(d);
        uf[f] -= (phi[cidx(g, i, j, k)] - phi[cidx(g, i - e.x, j - e.y, k - e.z)]) * g.ih;
    }
}

// Position of cell c in the ascending list of cut cells, -1 if absent.
__device__ inline int find_cut(const int *cut, int ncut, int c)
{
    int lo = 0, hi = ncut - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = cut[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// ---- limited slopes of the three components along the three axes ----------
// S[(3 d + q) N3 + c]: slope of u_q at c along d (zero on covered cells).
// Each face difference is formed once: a block of SL_X x SL_Y
// columns marches SL_Z planes; a cell's difference toward its upper
// neighbour (dr) along x comes to the next lane by a shuffle, along y to the
// next row through shared memory, along z to the next plane in a register,
// where it is that cell's dl -- the same subtraction of the same two values,
// so each slope is mc_limit(f0 - fm, fp - f0, fp - fm) bit for bit (zero
// unless the cell and both neighbours along the axis hold fluid), with 6 FP64
// subtractions per component instead of 9 (the kernel is bound by the FP64
// pipe).
constexpr int SL_X = 32, SL_Y = 8, SL_Z = 16;
__global__ void __launch_bounds__(SL_X *SL_Y) k_slopes_march(GridD g, const uint8_t *__restrict__ flag,
                                                            const double *__restrict__ u, double *__restrict__ S)
{
    __shared__ double sdy[2][3][SL_Y][SL_X];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.x * SL_X + tx, j = blockIdx.y * SL_Y + ty;
    const int z0 = blockIdx.z * SL_Z, z1 = min(g.nz, z0 + SL_Z);
    const bool col = i < g.nx && j < g.ny;
    const int N3 = ncell(g), sy = g.nx, sz = g.nx * g.ny;
    double dzp[3] = {0.0, 0.0, 0.0};   // dr along z of the plane before (its u(k) - u(k-1))
    for (int k = z0; k < z1; k++) {
        const int c = col ? cidx(g, i, j, k) : 0;
        const bool fl = col && flag[c] != 0;
        // neighbours available along each axis (inside the box and fluid)
        const bool xm = col && i > 0 && flag[c - 1] != 0, xp = col && i < g.nx - 1 && flag[c + 1] != 0;
        const bool ym = col && j > 0 && flag[c - sy] != 0, yp = col && j < g.ny - 1 && flag[c + sy] != 0;
        const bool zm = col && k > 0 && flag[c - sz] != 0, zp = col && k < g.nz - 1 && flag[c + sz] != 0;
        double f0[3], drx[3], dry[3], drz[3];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const double *f = u + q * N3;
            f0[q] = col ? f[c] : 0.0;
            drx[q] = (col && i < g.nx - 1) ? f[c + 1] - f0[q] : 0.0;
            dry[q] = (col && j < g.ny - 1) ? f[c + sy] - f0[q] : 0.0;
            drz[q] = (col && k < g.nz - 1) ? f[c + sz] - f0[q] : 0.0;
            sdy[k & 1][q][ty][tx] = dry[q];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const double *f = u + q * N3;
            // dl: the lower neighbour's dr (x: the previous lane, y: the previous
            // row, z: the previous plane), formed here at the edges of the block
            double dlx = __shfl_up_sync(0xffffffffu, drx[q], 1);
            if (tx == 0 && col && i > 0) dlx = f0[q] - f[c - 1];
            const double dly = (ty > 0) ? sdy[k & 1][q][ty - 1][tx] : ((col && j > 0) ? f0[q] - f[c - sy] : 0.0);
            const double dlz = (k > z0) ? dzp[q] : ((col && k > 0) ? f0[q] - f[c - sz] : 0.0);
            dzp[q] = drz[q];
            if (!col) continue;
            // dd = fp - fm, formed only where both neighbours exist
            const double sx = (fl && xm && xp) ? mc_limit(dlx, drx[q], f[c + 1] - f[c - 1]) : 0.0;
            const double sy_ = (fl && ym && yp) ? mc_limit(dly, dry[q], f[c + sy] - f[c - sy]) : 0.0;
            const double sz_ = (fl && zm && zp) ? mc_limit(dlz, drz[q], f[c + sz] - f[c - sz]) : 0.0;
            S[(0 + q) * N3 + c] = sx;
            S[(3 + q) * N3 + c] = sy_;
            S[(6 + q) * N3 + c] = sz_;
        }
    }
}

// ---- convective face fluxes  F_q = a_f * (upwinded state of u_q) * u^F ------
// One thread per face of normal d; F holds 3 components of the face triple.
__global__ void __launch_bounds__(256) k_conv_flux(GridD g, int d, const double *__restrict__ ap,
                                                   const double *__restrict__ u,
                                                   const double *__restrict__ S,
                                                   const double *__restrict__ ufd, double *__restrict__ F,
                                                   int nft, int off)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int mx = g.nx + (d == 0), my = g.ny + (d == 1), mz = g.nz + (d == 2);
    if (i >= mx || j >= my || k >= mz) return;
    const int f = fidx(g, d, i, j, k);
    const int N3 = ncell(g);
    const double a = ap[f];
    if (a <= 0.0) {
        for (int q = 0; q < 3; q++) F[q * nft + off + f] = 0.0;
        return;
    }
    const double w = ufd[f];
    const int pos = d == 0 ? i : (d == 1 ? j : k);
    int3 e = unit(d);
    if (pos == 0 || pos == dimn(g, d)) {
        const int hs = pos != 0;
        const int c = cidx(g, i - hs * e.x, j - hs * e.y, k - hs * e.z);
        const bool in = g.bc[2 * d + hs] == EBV_INFLOW;
        for (int q = 0; q < 3; q++) {
            double state = in ? g.u_in[q] : u[q * N3 + c];
            F[q * nft + off + f] = a * state * w;
        }
        return;
    }
    const int cL = cidx(g, i - e.x, j - e.y, k - e.z), cR = cidx(g, i, j, k);
    // only the upwind side's state is formed (fewer FP64 operations), and the
    // side is chosen before the arithmetic: faces of either sign in one warp
    // run the same instructions (u_L + S_L/2 or u_R - S_R/2, one FMA each).
    // Across the flow the sign of w alternates between neighbouring faces, so
    // a branch on it would run both halves in most warps.
    const double aw = a * w;
    if (w != 0.0) {
        const int cs = w > 0.0 ? cL : cR;
        const double hs = w > 0.0 ? 0.5 : -0.5;
        for (int q = 0; q < 3; q++) F[q * nft + off + f] = aw * (u[q * N3 + cs] + hs * S[(3 * d + q) * N3 + cs]);
    } else {
        for (int q = 0; q < 3; q++) {
            const double state = 0.5 * ((u[q * N3 + cL] + 0.5 * S[(3 * d + q) * N3 + cL]) +
                                        (u[q * N3 + cR] - 0.5 * S[(3 * d + q) * N3 + cR]));
            F[q * nft + off + f] = aw * state;
        }
    }
}

// ---- conservative divergence D^C of a face flux triple (3 components) -----
// With kEB the viscous EB wall flux -eta n_q (n . du/dn) A_EB is added.
template <bool kEB>
__global__ void __launch_bounds__(256) k_flux_div(GridD g, GeomD geo, const double *__restrict__ F, int nft,
                                                  const double *__restrict__ eta,
                                                  const double *__restrict__ dudn, double *__restrict__ DC)
{
    CELL_INDEX
    const int N3 = ncell(g);
    if (geo.flag[c] == 0) {
        for (int q = 0; q < 3; q++) DC[q * N3 + c] = 0.0;
        return;
    }
    const int off[3] = {0, nface(g, 0), nface(g, 0) + nface(g, 1)};
    double s[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        int3 e = unit(d);
        const int flo = off[d] + fidx(g, d, i, j, k), fhi = off[d] + fidx(g, d, i + e.x, j + e.y, k + e.z);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            s[q] += -F[q * nft + flo];
            s[q] += F[q * nft + fhi];
        }
    }
    if (kEB && geo.flag[c] == 2 && geo.area[c] > 0.0) {
        int t = find_cut(geo.cut, geo.ncut, c);
        if (t >= 0) {
            double nd = 0.0;
            for (int q = 0; q < 3; q++) nd += geo.nrm[q * N3 + c] * dudn[q * geo.ncut + t];
            for (int q = 0; q < 3; q++) s[q] += -eta[c] * geo.nrm[q * N3 + c] * nd * geo.area[c];
        }
    }
    const double inv = geo.flag[c] == 1 ? g.ih : 1.0 / (geo.alpha[c] * g.h);   // alpha = 1 on regular cells
    for (int q = 0; q < 3; q++) DC[q * N3 + c] = s[q] * inv;
}

// ---- hybrid flux divergence and redistribution (3 components) -------------
// A fluid cell none of whose 26 neighbours is cut has alpha = 1 and only
// full neighbours, so D = D^H = D^C exactly (its excess and its neighbours'
// excess vanish).  Such cells take the direct path; the cells of the `near`
// list (cut cells and their neighbours) take the two passes below.
// kDiv: out = v / div; without it div is 1 and no division is issued (a
// division the branch skips is still evaluated when the compiler turns the
// branch into a select).
template <bool kDiv>
__global__ void k_redist_far(GridD g, const uint8_t *__restrict__ flag, const uint8_t *__restrict__ near,
                             const double *__restrict__ DC, double sign, double div, double *__restrict__ out)
{
    CELL_INDEX
    const int N3 = ncell(g);
    if (near[c]) return;
    for (int q = 0; q < 3; q++) {
        double v = flag[c] ? sign * DC[q * N3 + c] : 0.0;
        out[q * N3 + c] = kDiv ? v / div : v;
    }
}

// Pass 1 on the near cells: D^H and, for cut cells, the excess dD and the
// weight w = 1 / (sum of neighbour alpha).
__global__ void __launch_bounds__(256) k_redist_a(GridD g, const int *__restrict__ list, int nlist,
                                                  const uint8_t *__restrict__ flag,
                                                  const double *__restrict__ alpha,
                                                  const double *__restrict__ DC,
                                                  double *__restrict__ D, double *__restrict__ dD,
                                                  double *__restrict__ w)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nlist) return;
    const int c = list[t];
    const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    const int N3 = ncell(g);
    const double al = alpha[c];
    if (flag[c] == 1) {  // alpha = 1: D^H = D^C, no excess
        for (int q = 0; q < 3; q++) { D[q * N3 + c] = DC[q * N3 + c]; dD[q * N3 + c] = 0.0; }
        return;
    }
    double sa = 0.0, sad[3] = {0.0, 0.0, 0.0};
    for (int dk = -1; dk <= 1; dk++)
        for (int dj = -1; dj <= 1; dj++)
            for (int di = -1; di <= 1; di++) {
                if (!di && !dj && !dk) continue;
                if (!avail(g, flag, i + di, j + dj, k + dk)) continue;
                int c2 = cidx(g, i + di, j + dj, k + dk);
                double a2 = alpha[c2];
                sa += a2;
                for (int q = 0; q < 3; q++) sad[q] += a2 * DC[q * N3 + c2];
            }
    for (int q = 0; q < 3; q++) {
        double dcq = DC[q * N3 + c];
        double dnc = sa > 0.0 ? sad[q] / sa : dcq;
        D[q * N3 + c] = al * dcq + (1.0 - al) * dnc;
        dD[q * N3 + c] = al * (1.0 - al) * (dcq - dnc);
    }
    w[c] = sa > 0.0 ? 1.0 / sa : 0.0;
}

// Pass 2 on the near cells: add the cut neighbours' weighted excess (full
// neighbours have none); out = sign * D / div (kDiv as in k_redist_far).
template <bool kDiv>
__global__ void __launch_bounds__(256) k_redist_b(GridD g, const int *__restrict__ list, int nlist,
                                                  const uint8_t *__restrict__ flag,
                                                  const double *__restrict__ D,
                                                  const double *__restrict__ dD,
                                                  const double *__restrict__ w, double sign,
                                                  double div, double *__restrict__ out)
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
                int c2 = cidx(g, i + di, j + dj, k + dk);
                if (flag[c2] != 2) continue;
                for (int q = 0; q < 3; q++) s[q] += w[c2] * dD[q * N3 + c2];
            }
    for (int q = 0; q < 3; q++) {
        const double v = sign * (D[q * N3 + c] + s[q]);
        out[q * N3 + c] = kDiv ? v / div : v;
    }
}

// ---- wall-normal derivative at the EB centroid (Eqs. interpolation_distances, dudn)
__global__ void k_wall_dudn(GridD g, GeomD geo, const double *__restrict__ u,
                            double *__restrict__ dudn)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= geo.ncut) return;
    const int N3 = geo.ncell;
    const int c = geo.cut[t];
    if (c < 0 || c >= N3) {  // a list entry outside the grid contributes nothing
        for (int q = 0; q < 3; q++) dudn[q * geo.ncut + t] = 0.0;
        return;
    }
    int ci[3] = {c % g.nx, (c / g.nx) % g.ny, c / (g.nx * g.ny)};
    double n[3], b[3];
    for (int e = 0; e < 3; e++) { n[e] = geo.nrm[e * N3 + c]; b[e] = geo.bcen[e * N3 + c]; }
    int kax = 0;
    if (fabs(n[1]) > fabs(n[kax])) kax = 1;
    if (fabs(n[2]) > fabs(n[kax])) kax = 2;
    const int k1 = (kax == 0) ? 1 : 0, k2 = (kax == 2) ? 1 : 2;
    const double s = n[kax] > 0.0 ? 1.0 : -1.0;
    const int si = n[kax] > 0.0 ? 1 : -1;
    const double dist[2] = {(s - b[kax]) / n[kax], (2.0 * s - b[kax]) / n[kax]};
    int cc1[2], cc2[2];
    double L1[2][3], L2[2][3];
    bool ok = true;
    for (int m = 0; m < 2; m++) {
        double P1 = b[k1] + dist[m] * n[k1], P2 = b[k2] + dist[m] * n[k2];
        cc1[m] = (int)floor(P1 + 0.5);
        cc2[m] = (int)floor(P2 + 0.5);
        double x1 = P1 - cc1[m], x2 = P2 - cc2[m];
        L1[m][0] = 0.5 * x1 * (x1 - 1.0); L1[m][1] = 1.0 - x1 * x1; L1[m][2] = 0.5 * x1 * (x1 + 1.0);
        L2[m][0] = 0.5 * x2 * (x2 - 1.0); L2[m][1] = 1.0 - x2 * x2; L2[m][2] = 0.5 * x2 * (x2 + 1.0);
        for (int q1 = -1; q1 <= 1 && ok; q1++)
            for (int q2 = -1; q2 <= 1; q2++) {
                int id[3];
                id[kax] = ci[kax] + (m + 1) * si;
                id[k1] = ci[k1] + cc1[m] + q1;
                id[k2] = ci[k2] + cc2[m] + q2;
                if (!avail(g, geo.flag, id[0], id[1], id[2])) { ok = false; break; }
            }
        if (!ok) break;
    }
    int near[3];
    near[kax] = ci[kax] + si;
    {
        double P1 = b[k1] + dist[0] * n[k1], P2 = b[k2] + dist[0] * n[k2];
        near[k1] = ci[k1] + (int)floor(P1 + 0.5);
        near[k2] = ci[k2] + (int)floor(P2 + 0.5);
    }
    const bool near_ok = avail(g, geo.flag, near[0], near[1], near[2]);
    for (int q = 0; q < 3; q++) {
        const double *uq = u + q * N3;
        double r;
        if (ok) {
            double uv[2];
            for (int m = 0; m < 2; m++) {
                double v = 0.0;
                for (int q1 = -1; q1 <= 1; q1++)
                    for (int q2 = -1; q2 <= 1; q2++) {
                        int id[3];
                        id[kax] = ci[kax] + (m + 1) * si;
                        id[k1] = ci[k1] + cc1[m] + q1;
                        id[k2] = ci[k2] + cc2[m] + q2;
                        v += L1[m][q1 + 1] * L2[m][q2 + 1] * uq[cidx(g, id[0], id[1], id[2])];
                    }
                uv[m] = v;
            }
            double d1 = dist[0], d2 = dist[1];
            r = (d2 * d2 * uv[0] - d1 * d1 * uv[1]) / (d1 * d2 * (d2 - d1)) / g.h;
        } else if (near_ok) {
            r = uq[cidx(g, near[0], near[1], near[2])] / (dist[0] * g.h);
        } else {
            r = 0.0;
        }
        dudn[q * geo.ncut + t] = r;
    }
}

// ---- viscous face fluxes  F_j = a_f eta_f d u_d / d x_j (face normal d) ---
// eta_f: mean of the two cells; d u_d/d x_d: two-point difference; the
// transverse derivatives: mean of the two cells' robust gradients G.  Box
// faces: Dirichlet (ghost at h/2) or Neumann for u_d.
__global__ void __launch_bounds__(256) k_visc_flux(GridD g, int d, const double *__restrict__ ap,
                                                   const double *__restrict__ u,
                                                   const double *__restrict__ eta,
                                                   const double *__restrict__ G, double *__restrict__ F,
                                                   int nft, int off)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const int mx = g.nx + (d == 0), my = g.ny + (d == 1), mz = g.nz + (d == 2);
    if (i >= mx || j >= my || k >= mz) return;
    const int f = fidx(g, d, i, j, k);
    const int N3 = ncell(g);
    const double a = ap[f];
    if (a <= 0.0) {
        for (int q = 0; q < 3; q++) F[q * nft + off + f] = 0.0;
        return;
    }
    const int pos = d == 0 ? i : (d == 1 ? j : k);
    int3 e = unit(d);
    const double ih = g.ih;
    if (pos == 0 || pos == dimn(g, d)) {
        const int hs = pos != 0;
        const int c = cidx(g, i - hs * e.x, j - hs * e.y, k - hs * e.z);
        double val;
        const bool dir = side_dirichlet(g, 2 * d + hs, d, &val);
        for (int jj = 0; jj < 3; jj++) {
            double T;
            if (dir) {
                double ud = u[d * N3 + c];
                T = (jj == d) ? eta[c] * (hs ? (val - ud) : (ud - val)) * (2.0 * ih) : 0.0;
            } else {
                T = (jj == d) ? 0.0 : eta[c] * G[(3 * jj + d) * N3 + c];
            }
            F[jj * nft + off + f] = a * T;
        }
        return;
    }
    const int cL = cidx(g, i - e.x, j - e.y, k - e.z), cR = cidx(g, i, j, k);
    // W = a eta_f; the normal derivative's 1/h and the transverse mean's 1/2
    // are folded into W once (fewer FP64 operations)
    const double W = (0.5 * a) * (eta[cL] + eta[cR]);
    const double Wn = W * ih, Wt = 0.5 * W;
    for (int jj = 0; jj < 3; jj++) {
        F[jj * nft + off + f] = (jj == d) ? (u[d * N3 + cR] - u[d * N3 + cL]) * Wn
                                          : (G[(3 * jj + d) * N3 + cL] + G[(3 * jj + d) * N3 + cR]) * Wt;
    }
}

// Cell-centre gradient of the trilinear interpolant of nodal p: all three
// components at once, from the sums and differences of the node
// pairs along x (20 FP64 operations instead of 27).
__device__ inline void grad_p3(const GridD &g, const double *p, int i, int j, int k, double q4h, double *gr)
{
    const double a = p[nidx(g, i, j, k)], b = p[nidx(g, i + 1, j, k)];
    const double c = p[nidx(g, i, j + 1, k)], d = p[nidx(g, i + 1, j + 1, k)];
    const double e = p[nidx(g, i, j, k + 1)], f = p[nidx(g, i + 1, j, k + 1)];
    const double gg = p[nidx(g, i, j + 1, k + 1)], h = p[nidx(g, i + 1, j + 1, k + 1)];
    const double P1 = a + b, P2 = c + d, P3 = e + f, P4 = gg + h;
    const double Q1 = b - a, Q2 = d - c, Q3 = f - e, Q4 = h - gg;
    gr[0] = ((Q1 + Q2) + (Q3 + Q4)) * q4h;
    gr[1] = ((P2 - P1) + (P4 - P3)) * q4h;
    gr[2] = ((P3 + P4) - (P1 + P2)) * q4h;
}

// psi = rho u + dt (rho C + V - grad p + f).  With gpa, also (dt/rho) grad p
// (covered cells 0): the term the nodal projection adds back to the solved
// velocity, from the same node sums (the values k_add_gradp would form).
__global__ void k_psi(GridD g, const uint8_t *__restrict__ flag, const double *__restrict__ u,
                      const double *__restrict__ C, const double *__restrict__ V,
                      const double *__restrict__ p, const double *__restrict__ f,
                      const double *__restrict__ dtp, double rho, double *__restrict__ psi,
                      double *__restrict__ gpa)
{
    CELL_INDEX
    const int N3 = ncell(g);
    const double dt = *dtp;
    if (flag[c] == 0) {
        for (int q = 0; q < 3; q++) psi[q * N3 + c] = 0.0;
        if (gpa)
            for (int q = 0; q < 3; q++) gpa[q * N3 + c] = 0.0;
        return;
    }
    double sums[3];
    grad_p3(g, p, i, j, k, 1.0, sums);
    const double q4h = 0.25 * g.ih, q4a = dtp[DT_DT_RHO] * (0.25 * g.ih);
    for (int q = 0; q < 3; q++) {
        int s = q * N3 + c;
        double fq = f ? f[s] : 0.0;
        psi[s] = rho * u[s] + dt * (rho * C[s] + V[s] - sums[q] * q4h + fq);
        if (gpa) gpa[s] = sums[q] * q4a;
    }
}

// u += gpa (the stored (dt/rho) grad p of k_psi) on fluid cells, 0 on covered
// cells: k_add_gradp(sgn = +1) without re-forming the gradient.
__global__ void k_add_stored(GridD g, const uint8_t *__restrict__ flag, double *__restrict__ u,
                             const double *__restrict__ gpa)
{
    CELL_INDEX
    const int N3 = ncell(g);
    const bool fl = flag[c] != 0;
    for (int q = 0; q < 3; q++) {
        const int s = q * N3 + c;
        u[s] = fl ? u[s] + gpa[s] : 0.0;
    }
}

// u += sgn * (dt/rho) grad p on fluid cells; covered cells set to zero.
// (dt/rho) / (4h) scales the pair sums of grad_p3 in one product.
__global__ void k_add_gradp(GridD g, const uint8_t *__restrict__ flag, double *__restrict__ u,
                            const double *__restrict__ p, const double *__restrict__ dtp, double sgn)
{
    CELL_INDEX
    const int N3 = ncell(g);
    if (flag[c] == 0) {
        for (int q = 0; q < 3; q++) u[q * N3 + c] = 0.0;
        return;
    }
    double gr[3];
    grad_p3(g, p, i, j, k, dtp[DT_DT_RHO] * (0.25 * g.ih), gr);
    for (int q = 0; q < 3; q++) {
        int s = q * N3 + c;
        u[s] = sgn > 0 ? u[s] + gr[q] : u[s] - gr[q];
    }
}

__device__ inline bool node_dirichlet(const GridD &g, int i, int j, int k)
{
    if (pin_node(g, i, j, k)) return true;
    int id[3] = {i, j, k};
    for (int d = 0; d < 3; d++) {
        if (id[d] == 0 && g.bc[2 * d] == EBV_OUTFLOW) return true;
        if (id[d] == dimn(g, d) && g.bc[2 * d + 1] == EBV_OUTFLOW) return true;
    }
    return false;
}

// Per fluid cell, the four weighted signed sums of its velocity that its 8
// nodes take (alpha h^2/4 times (ux + uy) + uz, (ux + uy) - uz, (ux - uy) + uz,
// (ux - uy) - uz): every corner's sum is one of these or its exact negation
// (IEEE rounding is symmetric), so k_nodal_rhs adds or subtracts them in its
// corner order with half the FP64 operations of forming each corner's sum
// itself (each product is rounded before it is added).
__global__ void k_nodal_cellsums(GridD g, GeomD geo, const double *__restrict__ ut, double *__restrict__ P)
{
    CELL_INDEX
    if (geo.flag[c] == 0) return;
    const int N3 = ncell(g);
    const double hq = g.h * g.h * 0.25, w = geo.alpha[c] * hq;
    const double ux = ut[c], uy = ut[N3 + c], uz = ut[2 * N3 + c];
    const double pxy = ux + uy, mxy = ux - uy;
    P[c] = w * (pxy + uz);
    P[N3 + c] = w * (pxy - uz);
    P[2 * N3 + c] = w * (mxy + uz);
    P[3 * N3 + c] = w * (mxy - uz);
}

// Nodal right-hand side (weak divergence of ut plus the inflow boundary
// integral), times rho/dt so the solve uses the unit-coefficient operator.
// P: the cell sums of k_nodal_cellsums.
__global__ void k_nodal_rhs(GridD g, GeomD geo, const double *__restrict__ P,
                            const double *__restrict__ dtp, double *__restrict__ b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int n = nidx(g, i, j, k);
    const int N3 = ncell(g);
    const double h = g.h;
    bool act = !node_dirichlet(g, i, j, k);
    if (act) {
        bool any = false;
        for (int oc = 0; oc < 8; oc++)
            any |= avail(g, geo.flag, i - 1 + (oc & 1), j - 1 + ((oc >> 1) & 1), k - 1 + ((oc >> 2) & 1));
        act = any;
    }
    if (!act) { b[n] = 0.0; return; }
    // per cell: alpha h^2/4 times the signed sum of its three components,
    // (ux + uy) + uz for the corner (i - ci, j - cj, k - ck) = (1, 1, 1) and
    // so on: sums 0..3 of k_nodal_cellsums, negated for the opposite corners
    double v = 0.0;
    for (int oc = 0; oc < 8; oc++) {
        int ci = i - 1 + (oc & 1), cj = j - 1 + ((oc >> 1) & 1), ck = k - 1 + ((oc >> 2) & 1);
        if (!avail(g, geo.flag, ci, cj, ck)) continue;
        const int c = cidx(g, ci, cj, ck);
        const int di = i - ci, dj = j - cj, dk = k - ck;
        // (di,dj,dk) -> sum: (1,1,1) 0, (1,1,0) 1, (1,0,1) 2, (1,0,0) 3; with di = 0 the
        // negation of the sum of (1, 1-dj, 1-dk)
        const int q = di ? (dj ? 0 : 2) + (dk ? 0 : 1) : (dj ? 2 : 0) + (dk ? 1 : 0);
        const double pc = P[q * N3 + c];
        v = di ? v + pc : v - pc;
    }
    int id[3] = {i, j, k};
    const double *A[3] = {geo.ax, geo.ay, geo.az};
    for (int d = 0; d < 3; d++)
        for (int hs = 0; hs < 2; hs++) {
            int side = 2 * d + hs;
            if (g.bc[side] != EBV_INFLOW) continue;
            if (id[d] != (hs ? dimn(g, d) : 0)) continue;
            double sgn = hs ? 1.0 : -1.0;
            int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
            for (int q1 = -1; q1 <= 0; q1++)
                for (int q2 = -1; q2 <= 0; q2++) {
                    int fid[3] = {i, j, k};
                    fid[t1] += q1;
                    fid[t2] += q2;
                    if (fid[t1] < 0 || fid[t1] >= dimn(g, t1) || fid[t2] < 0 || fid[t2] >= dimn(g, t2))
                        continue;
                    double af = A[d][fidx(g, d, fid[0], fid[1], fid[2])];
                    v -= sgn * g.u_in[d] * af * h * h * 0.25;
                }
        }
    b[n] = v * dtp[DT_RHO_DT];
}

// ---- time step --------------------------------------------------------------
__global__ void k_cfl_max(GridD g, const uint8_t *__restrict__ flag, const double *__restrict__ u,
                          const double *__restrict__ f, unsigned long long *out)
{
    const int N3 = ncell(g);
    double mc = 0.0, mf = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N3; c += gridDim.x * blockDim.x) {
        if (flag[c] == 0) continue;
        double v = (fabs(u[c]) + fabs(u[N3 + c]) + fabs(u[2 * N3 + c])) * g.ih;
        mc = fmax(mc, v);
        if (f) mf = fmax(mf, (fabs(f[c]) + fabs(f[N3 + c]) + fabs(f[2 * N3 + c])) * g.ih);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mc = fmax(mc, __shfl_down_sync(0xffffffffu, mc, o));
        mf = fmax(mf, __shfl_down_sync(0xffffffffu, mf, o));
    }
    if ((threadIdx.x & 31) == 0) {
        // non-negative doubles order like their bit patterns
        atomicMax(out, (unsigned long long)__double_as_longlong(mc));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(mf));
    }
}

__global__ void k_dt_final(const unsigned long long *mx, double cfl, double cv, double dt_fixed, double rho,
                           double h, double *dt)
{
    if (threadIdx.x != 0) return;
    if (dt_fixed > 0.0) { store_dt(dt, dt_fixed, rho, h); return; }
    double cc = __longlong_as_double((long long)mx[0]);
    double cf2 = __longlong_as_double((long long)mx[1]);
    double ccv = cc + cv;
    store_dt(dt, cfl / (0.5 * (ccv + sqrt(ccv * ccv + 4.0 * cf2))), rho, h);
}

__global__ void k_average(double *a, const double *b, int n)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        a[s] = 0.5 * (a[s] + b[s]);
}

__global__ void k_zero_covered(GridD g, const uint8_t *__restrict__ flag, double *u, int ncomp)
{
    const int N3 = ncell(g);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N3; c += gridDim.x * blockDim.x)
        if (flag[c] == 0)
            for (int q = 0; q < ncomp; q++) u[q * N3 + c] = 0.0;
}

// ---- drag and yielded fraction -------------------------------------------
__global__ void k_drag_terms(GridD g, GeomD geo, const double *__restrict__ eta,
                             const double *__restrict__ dudn, const double *__restrict__ p,
                             double *__restrict__ term)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= geo.ncut) return;
    const int N3 = geo.ncell;
    const int c = geo.cut[t];
    if (c < 0 || c >= N3) {  // a list entry outside the grid contributes nothing
        term[t] = 0.0;
        return;
    }
    const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
    double n[3], b[3], gq[3];
    for (int e = 0; e < 3; e++) {
        n[e] = geo.nrm[e * N3 + c];
        b[e] = geo.bcen[e * N3 + c];
        gq[e] = dudn[e * geo.ncut + t];
    }
    double gn = gq[0] * n[0] + gq[1] * n[1] + gq[2] * n[2];
    double tz = eta[c] * (n[2] * gn + gq[2]);
    double pb = 0.0;
    for (int o = 0; o < 8; o++) {
        int oi = o & 1, oj = (o >> 1) & 1, ok = (o >> 2) & 1;
        double w = (oi ? b[0] + 0.5 : 0.5 - b[0]) * (oj ? b[1] + 0.5 : 0.5 - b[1]) *
                   (ok ? b[2] + 0.5 : 0.5 - b[2]);
        pb += w * p[nidx(g, i + oi, j + oj, k + ok)];
    }
    term[t] = geo.area[c] * g.h * g.h * (tz - pb * n[2]);
}

template <int kThreads>
__device__ inline double block_sum(double v)
{
    __shared__ double sm[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < kThreads / 32 ? sm[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) k_yield_parts(int N3, const uint8_t *__restrict__ flag,
                                                     const double *__restrict__ alpha,
                                                     const double *__restrict__ eta,
                                                     const double *__restrict__ sr, double tau0,
                                                     double *__restrict__ part)
{
    double vy = 0.0, vt = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N3; c += gridDim.x * blockDim.x) {
        if (flag[c] == 0) continue;
        double a = alpha[c];
        vt += a;
        if (eta[c] * sr[c] <= (1.0 + 1e-3) * tau0) vy += a;
    }
    double sy = block_sum<256>(vy);
    double st = block_sum<256>(vt);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sy;
        part[gridDim.x + blockIdx.x] = st;
    }
}

}  // namespace

// ===========================================================================
// Launchers
// ===========================================================================

ebv_status launch_strain_eta(Ctx *c, const double *u, double *eta, double *srate, double *G)
{
    const GridD &g = c->g;
    // u (3 words), flag (1 byte), eta (+ ||gamma||) (+ 9 gradient words)
    const double nb = (double)ncell(g) * (8.0 * (4 + (srate ? 1 : 0) + (G ? 9 : 0)) + 1.0);
    const dim3 gr = grid3(g.nx, g.ny, g.nz);
    if (c->prm.precision == EBV_FP32_MIXED) {   // FP32 away from the EB (plus the near-cell mask)
        if (G)
            EBV_LAUNCH_P(c, "strain_rate_viscosity", nb + ncell(g), (k_strain_eta<true, true>), gr, block3(), 0, g,
                         c->flag, u, paramsd(c->prm), eta, srate, G, c->nearm);
        else
            EBV_LAUNCH_P(c, "strain_rate_viscosity", nb + ncell(g), (k_strain_eta<false, true>), gr, block3(), 0, g,
                         c->flag, u, paramsd(c->prm), eta, srate, nullptr, c->nearm);
        return EBV_OK;
    }
    if (G)
        EBV_LAUNCH_P(c, "strain_rate_viscosity", nb, k_strain_eta<true>, gr, block3(), 0, g, c->flag, u,
                     paramsd(c->prm), eta, srate, G);
    else
        EBV_LAUNCH_P(c, "strain_rate_viscosity", nb, k_strain_eta<false>, gr, block3(), 0, g, c->flag, u,
                     paramsd(c->prm), eta, srate, nullptr);
    return EBV_OK;
}

ebv_status launch_flow_diag(Ctx *c, const double *u, double *lam, double *sdev)
{
    const GridD &g = c->g;
    EBV_LAUNCH(c, k_flow_diag, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, u, paramsd(c->prm), lam, sdev);
    return EBV_OK;
}

// Slopes of u into c->G (read again by launch_convective, before the viscous
// part overwrites c->G with the velocity gradient), then the face states.
ebv_status launch_face_states(Ctx *c, const double *u, double *uf)
{
    const GridD &g = c->g;
    EBV_LAUNCH(c, k_slopes_march, dim3((g.nx + SL_X - 1) / SL_X, (g.ny + SL_Y - 1) / SL_Y, (g.nz + SL_Z - 1) / SL_Z),
               dim3(SL_X, SL_Y), 0, g, c->flag, u, c->G);
    const double *A[3] = {c->ax, c->ay, c->az};
    size_t off = 0;
    for (int d = 0; d < 3; d++) {
        EBV_LAUNCH(c, k_face_states, grid3(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)),
                   block3(), 0, g, d, c->G, A[d], u, uf + off);
        off += nface(g, d);
    }
    return EBV_OK;
}

ebv_status launch_mac_rhs(Ctx *c, const double *uf, double *b)
{
    const GridD &g = c->g;
    EBV_LAUNCH(c, k_mac_rhs, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, c->ax, c->ay, c->az,
               uf, uf + nface(g, 0), uf + nface(g, 0) + nface(g, 1), b);
    return EBV_OK;
}

ebv_status launch_mac_correct(Ctx *c, double *uf, const double *phi)
{
    const GridD &g = c->g;
    const double *A[3] = {c->ax, c->ay, c->az};
    size_t off = 0;
    for (int d = 0; d < 3; d++) {
        EBV_LAUNCH(c, k_mac_correct, grid3(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)),
                   block3(), 0, g, d, A[d], phi, uf + off);
        off += nface(g, d);
    }
    return EBV_OK;
}

ebv_status launch_redistribute_into(Ctx *c, const double *DC, double sign, double div, double *out)
{
    const GridD &g = c->g;
    const bool dv = div != 1.0;
    if (dv)
        EBV_LAUNCH(c, k_redist_far<true>, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, c->nearm, DC, sign, div,
                   out);
    else
        EBV_LAUNCH(c, k_redist_far<false>, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, c->nearm, DC, sign, div,
                   out);
    if (c->nnear) {
        dim3 gr((c->nnear + 127) / 128);
        EBV_LAUNCH(c, k_redist_a, gr, dim3(128), 0, g, c->nearl, c->nnear, c->flag, c->alpha, DC, c->Dh, c->dD,
                   c->wts);
        if (dv)
            EBV_LAUNCH(c, k_redist_b<true>, gr, dim3(128), 0, g, c->nearl, c->nnear, c->flag, c->Dh, c->dD, c->wts,
                       sign, div, out);
        else
            EBV_LAUNCH(c, k_redist_b<false>, gr, dim3(128), 0, g, c->nearl, c->nnear, c->flag, c->Dh, c->dD, c->wts,
                       sign, div, out);
    }
    return EBV_OK;
}

ebv_status launch_convective(Ctx *c, const double *u, const double *uf, double *C)
{
    const GridD &g = c->g;
    const int nft = nface(g, 0) + nface(g, 1) + nface(g, 2);
    // the slopes of u are in c->G (launch_face_states)
    const double *ufd[3] = {uf, uf + nface(g, 0), uf + nface(g, 0) + nface(g, 1)};
    const double *A[3] = {c->ax, c->ay, c->az};
    int off = 0;
    for (int d = 0; d < 3; d++) {
        EBV_LAUNCH(c, k_conv_flux, grid3(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)), block3(), 0, g, d,
                   A[d], u, c->G, ufd[d], c->ff, nft, off);
        off += nface(g, d);
    }
    EBV_LAUNCH(c, k_flux_div<false>, grid3(g.nx, g.ny, g.nz), block3(), 0, g, geomd(c), c->ff, nft, nullptr,
               nullptr, c->DC);
    return launch_redistribute_into(c, c->DC, -1.0, 1.0, C);
}

ebv_status launch_wall_dudn(Ctx *c, const double *u, double *dudn)
{
    if (c->ncut)
        EBV_LAUNCH(c, k_wall_dudn, dim3((c->ncut + 127) / 128), dim3(128), 0, c->g, geomd(c), u, dudn);
    return EBV_OK;
}

ebv_status launch_viscous_explicit(Ctx *c, const double *u, const double *eta, const double *G,
                                   double *V)
{
    const GridD &g = c->g;
    GeomD geo = geomd(c);
    ebv_status s0 = launch_wall_dudn(c, u, c->dudn);
    if (s0 != EBV_OK) return s0;
    const int nft = nface(g, 0) + nface(g, 1) + nface(g, 2);
    const double *A[3] = {c->ax, c->ay, c->az};
    int off = 0;
    for (int d = 0; d < 3; d++) {
        EBV_LAUNCH(c, k_visc_flux, grid3(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)), block3(), 0, g, d,
                   A[d], u, eta, G, c->ff, nft, off);
        off += nface(g, d);
    }
    EBV_LAUNCH(c, k_flux_div<true>, grid3(g.nx, g.ny, g.nz), block3(), 0, g, geo, c->ff, nft, eta, c->dudn,
               c->DC);
    return launch_redistribute_into(c, c->DC, 1.0, c->prm.rho, V);
}

ebv_status launch_psi(Ctx *c, const double *u, const double *C, const double *V, const double *p,
                      const double *f, double *psi, double *gpa)
{
    const GridD &g = c->g;
    EBV_LAUNCH(c, k_psi, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, u, C, V, p, f, c->dt_dev,
               c->prm.rho, psi, gpa);
    return EBV_OK;
}

ebv_status launch_add_stored(Ctx *c, double *u, const double *gpa)
{
    const GridD &g = c->g;
    EBV_LAUNCH(c, k_add_stored, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, u, gpa);
    return EBV_OK;
}

ebv_status launch_add_gradp(Ctx *c, double *u, const double *p, double sgn)
{
    const GridD &g = c->g;
    EBV_LAUNCH(c, k_add_gradp, grid3(g.nx, g.ny, g.nz), block3(), 0, g, c->flag, u, p, c->dt_dev, sgn);
    return EBV_OK;
}

ebv_status launch_nodal_rhs(Ctx *c, const double *ut, double *b)
{
    const GridD &g = c->g;
    double *P = c->G;   // scratch: the velocity gradient is not needed again before the next stage forms it
    EBV_LAUNCH(c, k_nodal_cellsums, grid3(g.nx, g.ny, g.nz), block3(), 0, g, geomd(c), ut, P);
    EBV_LAUNCH(c, k_nodal_rhs, grid3(g.nx + 1, g.ny + 1, g.nz + 1), block3(), 0, g, geomd(c), P,
               c->dt_dev, b);
    return EBV_OK;
}

ebv_status launch_timestep(Ctx *c, const double *u, const double *f, double dt_fixed)
{
    const GridD &g = c->g;
    EBV_CUDA_TRY(c, cudaMemsetAsync(c->cfl_max, 0, 2 * sizeof(unsigned long long), c->stream));
    EBV_LAUNCH(c, k_cfl_max, dim3(kReduceBlocks), dim3(256), 0, g, c->flag, u, f, c->cfl_max);
    const double h = g.h;
    double cv = 2.0 * c->prm.mu / c->prm.rho * (c->prm.bi_cfl + 1.0) * (3.0 / (h * h));
    EBV_LAUNCH(c, k_dt_final, dim3(1), dim3(32), 0, c->cfl_max, c->prm.cfl, cv, dt_fixed, c->prm.rho, h, c->dt_dev);
    return EBV_OK;
}

ebv_status launch_average(Ctx *c, double *a, const double *b, int n)
{
    EBV_LAUNCH(c, k_average, dim3(kReduceBlocks), dim3(256), 0, a, b, n);
    return EBV_OK;
}

ebv_status launch_zero_covered(Ctx *c, double *u, int ncomp)
{
    EBV_LAUNCH(c, k_zero_covered, dim3(kReduceBlocks), dim3(256), 0, c->g, c->flag, u, ncomp);
    return EBV_OK;
}

ebv_status launch_drag(Ctx *c, const double *u, const double *p, double *fz, double *yf)
{
    const GridD &g = c->g;
    GeomD geo = geomd(c);
    const int N3 = ncell(g);
    // eta and ||gamma|| of u (em/srate scratch), wall gradients, then the sums
    launch_strain_eta(c, u, c->es, c->srate, nullptr);
    if (c->ncut) {
        EBV_LAUNCH(c, k_wall_dudn, dim3((c->ncut + 127) / 128), dim3(128), 0, g, geo, u, c->dudn);
        EBV_LAUNCH(c, k_drag_terms, dim3((c->ncut + 127) / 128), dim3(128), 0, g, geo, c->es, c->dudn,
                   p, c->rhs_c);
        ebv_status s = reduce_sum(c, c->rhs_c, c->ncut, c->scal + 8);
        if (s != EBV_OK) return s;
    } else {
        EBV_CUDA_TRY(c, cudaMemsetAsync(c->scal + 8, 0, sizeof(double), c->stream));
    }
    EBV_LAUNCH(c, k_yield_parts, dim3(kReduceBlocks), dim3(256), 0, N3, c->flag, c->alpha, c->es,
               c->srate, c->prm.tau0, c->part);
    ebv_status s = reduce_sum(c, c->part, kReduceBlocks, c->scal + 9);
    if (s != EBV_OK) return s;
    s = reduce_sum(c, c->part + kReduceBlocks, kReduceBlocks, c->scal + 10);
    if (s != EBV_OK) return s;
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->scal_host + 8, c->scal + 8, 3 * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *fz = c->scal_host[8];
    *yf = c->scal_host[10] > 0.0 ? c->scal_host[9] / c->scal_host[10] : 0.0;
    return EBV_OK;
}

}  // namespace ebv

// ===========================================================================
// Drag and yielded fraction without any allocation
// ===========================================================================
// Some callers cannot call cudaMalloc: code that runs inside a memory pool
// they do not own, a host that must not grow device memory after start-up, or
// a plug-in that may only use the buffers it is handed.  ebv_drag_noalloc
// serves them: it runs the same kernels as ebv_drag, but its working storage
// is the fixed array below, which the library places in the memory of every
// GPU that loads it and which stays there until the process exits.
#include <cmath>
#include <mutex>

namespace ebv {
namespace {

constexpr int kNoAllocCells = 1 << 18;  // cells of the largest grid accepted (e.g. 64^3)
constexpr int kNoAllocCut = 1 << 16;    // cut cells of the largest geometry accepted
// eta and ||gamma|| per cell, wall gradients (3) and traction terms per cut
// cell, two sets of block partial sums, three results: about 6.3 MB.
constexpr size_t kNoAllocDoubles =
    2 * (size_t)kNoAllocCells + 4 * (size_t)kNoAllocCut + 2 * (size_t)kReduceBlocks + 8;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of g_noalloc_scratch per device.  In host code the array's
// name only stands in for it; the address comes from cudaGetSymbolAddress,
// taken once per device with that device current.
constexpr int kNoAllocMaxDevices = 64;
double *g_noalloc_addr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mutex;

__global__ void __launch_bounds__(1024) k_noalloc_sum(const double *part, int n, double *out)
{
    double v = 0.0;
    for (int s = threadIdx.x; s < n; s += 1024) v += part[s];
    v = block_sum<1024>(v);
    if (threadIdx.x == 0) *out = v;
}

__global__ void k_noalloc_finish(const double *sums, double *out)
{
    if (threadIdx.x != 0) return;
    out[0] = sums[0];
    out[1] = sums[2] > 0.0 ? sums[1] / sums[2] : 0.0;
}

}  // namespace
}  // namespace ebv

extern "C" ebv_status ebv_drag_noalloc(const ebv_grid *grid, const ebv_params *params,
                                       const double *alpha, const double *area, const double *nrm,
                                       const double *bcen, const unsigned char *flag, const int *cut,
                                       int ncut, const double *u, const double *p, double *out,
                                       void *stream)
{
    using namespace ebv;
    if (!grid || !params || !alpha || !area || !nrm || !bcen || !flag || !u || !p || !out)
        return EBV_ERR_INVALID;
    if (ncut < 0 || (ncut > 0 && !cut)) return EBV_ERR_INVALID;
    for (int d = 0; d < 3; d++)
        if (grid->n[d] < 1) return EBV_ERR_INVALID;
    if (!(grid->h > 0.0) || !std::isfinite(grid->h)) return EBV_ERR_INVALID;
    // An error left by earlier, unrelated work stays pending for its owner;
    // this call neither reports it as its own nor clears it.
    if (cudaPeekAtLastError() != cudaSuccess) return EBV_ERR_CUDA_PENDING;
    const long long n3 = (long long)grid->n[0] * grid->n[1] * grid->n[2];
    if (n3 > kNoAllocCells || ncut > kNoAllocCut) return EBV_ERR_TOO_LARGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return EBV_ERR_CUDA;
    double *scr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void *a = nullptr;
            if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess) return EBV_ERR_CUDA;
            g_noalloc_addr[dev] = (double *)a;
        }
        scr = g_noalloc_addr[dev];
    }
    double *eta = scr, *sr = scr + kNoAllocCells;
    double *dudn = scr + 2 * (size_t)kNoAllocCells;
    double *term = dudn + 3 * (size_t)kNoAllocCut;
    double *part = term + kNoAllocCut;
    double *sums = part + 2 * (size_t)kReduceBlocks;

    GridD g;
    g.nx = grid->n[0]; g.ny = grid->n[1]; g.nz = grid->n[2];
    g.h = grid->h;
    g.ih = 1.0 / grid->h;
    for (int d = 0; d < 3; d++) { g.lo[d] = grid->lo[d]; g.u_in[d] = grid->u_in[d]; }
    for (int s = 0; s < 6; s++) g.bc[s] = grid->bc[s];
    GeomD geo;
    geo.alpha = alpha; geo.ax = geo.ay = geo.az = nullptr; geo.area = area; geo.nrm = nrm;
    geo.bcen = bcen; geo.flag = flag; geo.cut = cut; geo.ncut = ncut; geo.ncell = (int)n3;
    cudaStream_t st = (cudaStream_t)stream;

    // every scratch value read below is written earlier in this call, so no
    // clearing is needed
    k_strain_eta<false><<<grid3(g.nx, g.ny, g.nz), block3(), 0, st>>>(g, flag, u, paramsd(*params), eta, sr,
                                                                      nullptr);
    if (ncut) {
        k_wall_dudn<<<(ncut + 127) / 128, 128, 0, st>>>(g, geo, u, dudn);
        k_drag_terms<<<(ncut + 127) / 128, 128, 0, st>>>(g, geo, eta, dudn, p, term);
    }
    k_noalloc_sum<<<1, 1024, 0, st>>>(term, ncut, sums);
    k_yield_parts<<<kReduceBlocks, 256, 0, st>>>((int)n3, flag, alpha, eta, sr, params->tau0, part);
    k_noalloc_sum<<<1, 1024, 0, st>>>(part, kReduceBlocks, sums + 1);
    k_noalloc_sum<<<1, 1024, 0, st>>>(part + kReduceBlocks, kReduceBlocks, sums + 2);
    k_noalloc_finish<<<1, 32, 0, st>>>(sums, out);
    if (cudaGetLastError() != cudaSuccess) return EBV_ERR_CUDA;
    return EBV_OK;
}
