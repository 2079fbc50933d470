// Linear solvers of one step: the cell-centred projection (Poisson), the
// three semi-implicit viscous Helmholtz solves and the nodal projection
// (paper Sec. "Numerical algorithm": geometric multigrid for EB systems with a
// Krylov method at the bottom).
//
// Every solve is conjugate gradients in FP64 preconditioned by one symmetric
// multigrid V-cycle: red-black Gauss-Seidel (red first on the way down, black
// first on the way up) for the 7-point cell-centred operators, a degree-3
// Chebyshev-Jacobi smoother for the 27-point nodal operator, averaging /
// full-weighting restriction, piecewise-constant / trilinear prolongation and
// an exact dense solve at the bottom.  The V-cycle runs in FP64 or FP32
// (EBV_FP32_REFINE); residuals, Krylov vectors and solution accumulation stay
// FP64, so FP32 only enters as a preconditioner.  Dot products use fixed-order
// block partials, so results are bitwise reproducible run to run.
#include <math.h>
#include <vector>

#include <cooperative_groups.h>

#include "ebv_internal.cuh"
#include "tma.cuh"
#include "fpbits.cuh"

namespace ebv {

// ===========================================================================
// Reductions
// ===========================================================================
namespace {

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

__device__ inline int block_linear() { return (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x; }
__device__ inline int thread_linear() { return (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x; }

// 3-D blocks of 256 threads: block sum keyed on the linear thread index.
__device__ inline double block_sum3(double v)
{
    __shared__ double sm[8];
    const int t = thread_linear();
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) sm[t >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (t < 32) {
        r = t < 8 ? sm[t] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

// Block sum of per-thread partials of type T, returned in FP64.  FP64 keeps
// FP64 throughout (block_sum3).  FP32 partials are summed in FP32 within the
// warp (32 terms) and in FP64 across warps: FP64 arithmetic is scarce on this
// GPU, and per-cell FP64 work in a kernel that streams FP32 data made FP64 the
// bound of the FP32 operator apply.
template <class T>
__device__ inline double block_sum3_t(T v)
{
    if constexpr (sizeof(T) == 8) {
        return block_sum3(v);
    } else {
        __shared__ double sm[8];
        const int t = thread_linear();
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((t & 31) == 0) sm[t >> 5] = (double)v;
        __syncthreads();
        double r = 0.0;
        if (t < 32) {
            r = t < 8 ? sm[t] : 0.0;
            for (int o = 4; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
        }
        return r;
    }
}

// Sum of n block partials in a fixed order, over a cluster of kRedCtas
// blocks: block q sums the slice [q n / kRedCtas, (q + 1) n / kRedCtas)
// (strided over its threads, then its block sum) and stores that sum in
// block 0's shared memory; after the cluster barrier block 0 adds the
// kRedCtas sums in rank order.  FP64 additions issue at about one per SM and
// cycle on this GPU, so a single block spent up to 16 us on the 32,768
// partials of a 256^3 refinement residual; the cluster spreads them over
// kRedCtas SMs.  The barrier is the hardware cluster barrier (no spin).
constexpr int kRedCtas = 8, kRedThreads = 512;
__global__ void __cluster_dims__(kRedCtas, 1, 1) __launch_bounds__(kRedThreads)
    k_reduce_final(const double *part, int n, double *out)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double csum[kRedCtas];
    const int q = (int)cl.block_rank();
    const int lo = (int)((long long)n * q / kRedCtas), hi = (int)((long long)n * (q + 1) / kRedCtas);
    double v = 0.0;
    for (int s = lo + threadIdx.x; s < hi; s += kRedThreads) v += part[s];
    v = block_sum<kRedThreads>(v);
    if (threadIdx.x == 0) *cl.map_shared_rank(&csum[q], 0) = v;
    cl.sync();
    if (q == 0 && threadIdx.x == 0) {
        double t = 0.0;
        for (int r = 0; r < kRedCtas; r++) t += csum[r];
        *out = t;
    }
}

__global__ void __launch_bounds__(256) k_dot(const double *__restrict__ a, const double *__restrict__ b,
                                             int n, double *__restrict__ part)
{
    double v = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        v += a[s] * b[s];
    v = block_sum<256>(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

}  // namespace

ebv_status reduce_sum(Ctx *c, const double *part, int nblocks, double *out_dev)
{
    EBV_LAUNCH(c, k_reduce_final, dim3(kRedCtas), dim3(kRedThreads), 0, part, nblocks, out_dev);
    return EBV_OK;
}

namespace {

// ===========================================================================
// Cell-centred operator  (A x)_i = extra_i x_i + sum_faces beta_f (x_i - x_nb)
// (face coefficients include the box faces; x_nb = 0 outside the box).
// Each level stores extra (for coarsening) and the full diagonal
// diag = extra + sum of the 6 face coefficients (for the smoother and apply).
// ===========================================================================

// Cell-centred operator of one level: diagonal (precision T) and face
// coefficients (storage F, widened to T when read).
template <class T, class F = T>
struct CcOp {
    GridD g;
    const T *diag;
    const F *bx, *by, *bz;
    const T *dinv = nullptr;   // FP32 V-cycle: 1/diag (0 where diag <= 0)
};
// The V-cycle's operator: in FP32 its faces are stored in BF16 (half the
// bytes of the face arrays every colour pass reads whole); the Krylov
// operator it preconditions keeps FP32 faces (CcOp<T>).  Built with
// EBV_VCYCLE_FP32_FACES (a measurement variant of the library, not the
// default) the V-cycle reads the FP32 faces instead, with the diagonal
// formed from them unrounded; everything else is the same code.
template <class T> struct VFace { using type = T; };
#ifdef EBV_VCYCLE_FP32_FACES
template <> struct VFace<float> { using type = float; };
constexpr bool kVcycleBf16 = false;
#else
template <> struct VFace<float> { using type = __nv_bfloat16; };
constexpr bool kVcycleBf16 = true;
#endif
template <class T> using VOp = CcOp<T, typename VFace<T>::type>;

// Array layout of the cell-centred multigrid, by precision.  FP64 arrays are
// in the natural order (x fastest).  FP32 arrays -- the coefficients of every
// level, the V-cycle vectors and the inner Krylov vectors of the refinement
// solver -- are "row-split": within every x-row the even-i entries come first,
// then the odd-i ones.  A colour of a red-black pass then reads and writes
// contiguous half-rows (the cells of one colour in a row all have the same
// parity of i) instead of every other word of every sector; only the x-face
// coefficients are still read whole.  Rows keep their length and place, so
// neighbours in y and z are at the same offsets as in the natural order.
__host__ __device__ inline int spos(int m, int i) { return (i & 1) ? ((m + 1) >> 1) + (i >> 1) : (i >> 1); }
template <class T>
__host__ __device__ inline int cix(const GridD &g, int i, int j, int k)
{
    return (k * g.ny + j) * g.nx + (sizeof(T) == 4 ? spos(g.nx, i) : i);
}
template <class T>
__host__ __device__ inline int fidxT(const GridD &g, int d, int i, int j, int k)
{
    if (d == 0) return (k * g.ny + j) * (g.nx + 1) + (sizeof(T) == 4 ? spos(g.nx + 1, i) : i);
    if (d == 1) return (k * (g.ny + 1) + j) * g.nx + (sizeof(T) == 4 ? spos(g.nx, i) : i);
    return (k * g.ny + j) * g.nx + (sizeof(T) == 4 ? spos(g.nx, i) : i);
}

// Positions of cell (i,j,k), of its two x-neighbours and of its six faces in
// the level's layout (cix / fidxT), from the start of its row.  Row-split
// (FP32): with t = i/2 the even cells of a row sit at rc + t and the odd ones
// at rc + h + t (h = ceil(nx/2), rc the row's start), so the x-neighbours of
// an even cell are odd cells t-1 and t and those of an odd cell even cells t
// and t+1; x-face rows (nx+1 faces, hf = ceil((nx+1)/2)) start at rc + k ny + j.
// Natural order (FP64): the plain offsets.  In both, a y-face row is the cell
// row shifted by k nx and a z-face row the cell row itself.
struct CellPos {
    int c, xw, xe, fx0, fx1, fy0, fy1, fz0, fz1;
};
template <class T>
__device__ inline CellPos cell_pos(const GridD &g, int i, int j, int k)
{
    CellPos p;
    const int rc = (k * g.ny + j) * g.nx;
    if constexpr (sizeof(T) == 4) {
        const int t = i >> 1, odd = i & 1, h = (g.nx + 1) >> 1, hf = (g.nx + 2) >> 1;
        const int rf = rc + k * g.ny + j;
        p.c = rc + (odd ? h + t : t);
        p.xw = rc + (odd ? t : h + t - 1);
        p.xe = rc + (odd ? t + 1 : h + t);
        p.fx0 = rf + (odd ? hf + t : t);
        p.fx1 = rf + (odd ? t + 1 : hf + t);
    } else {
        p.c = rc + i;
        p.xw = p.c - 1;
        p.xe = p.c + 1;
        p.fx0 = rc + k * g.ny + j + i;
        p.fx1 = p.fx0 + 1;
    }
    p.fy0 = p.c + k * g.nx;
    p.fy1 = p.fy0 + g.nx;
    p.fz0 = p.c;
    p.fz1 = p.c + g.nx * g.ny;
    return p;
}

template <class T, class F>
__device__ inline void cc_row(const CcOp<T, F> &A, int i, int j, int k, const T *__restrict__ x,
                              T &diag, T &off)
{
    const GridD &g = A.g;
    const CellPos p = cell_pos<T>(g, i, j, k);
    const int c = p.c;
    const T bxl = T(A.bx[p.fx0]), bxh = T(A.bx[p.fx1]);
    const T byl = T(A.by[p.fy0]), byh = T(A.by[p.fy1]);
    const T bzl = T(A.bz[p.fz0]), bzh = T(A.bz[p.fz1]);
    diag = A.diag[c];
    T s = 0;
    if (i > 0) s += bxl * x[p.xw];
    if (i < g.nx - 1) s += bxh * x[p.xe];
    if (j > 0) s += byl * x[c - g.nx];
    if (j < g.ny - 1) s += byh * x[c + g.nx];
    if (k > 0) s += bzl * x[c - g.nx * g.ny];
    if (k < g.nz - 1) s += bzh * x[c + g.nx * g.ny];
    off = s;
}

// One colour of Gauss-Seidel in place: x_i = (b_i + sum beta x_nb) / diag for
// the cells of colour `color` ((i+j+k) mod 2); with zero_start the other
// colour reads as 0 (the sweep starts from x = 0) and x is not read.
// Thread (t, j, kk) owns the x-pair (2t, 2t+1) of row j on planes
// GS_PZ kk .. GS_PZ kk + GS_PZ - 1 and updates the cell of colour `color` in
// each: every lane works.  All operands of its GS_PZ updates are loaded before
// any result is stored (the updated cells are never read in the same pass), so
// the loads of all of them are in flight together.
// kCorr: the pass that follows the coarse-grid correction.  Since a pass
// never reads the old value of the cells it updates, prolongation (x += the
// coarse correction xc of the parent cell, on uncovered cells) is folded into
// the neighbour reads: x_nb + xc(parent(nb)), the very sums a separate
// prolongation kernel would store.  A covered neighbour's face coefficient is
// 0, so adding to it changes nothing either.
constexpr int GS_PZ = 2;

// The Gauss-Seidel value of cell (i,j,k): (b + sum beta x_nb) / diag, 0 on
// cells with no diagonal (see k_cc_gs for kCorr and zero_start); FP32 levels
// multiply by the stored inverse diagonal instead of dividing.
template <class T, bool kCorr>
__device__ inline T gs_cell(const VOp<T> &A, const T *__restrict__ x, const T *__restrict__ b, int i, int j,
                            int k, int zero_start, const T *__restrict__ xc, const GridD &gc)
{
    const GridD &g = A.g;
    const int sy = g.nx, sz = g.nx * g.ny;
    const CellPos p = cell_pos<T>(g, i, j, k);
    const int c = p.c;
    const T diag = sizeof(T) == 4 ? T(0) : A.diag[c], bc = b[c];
    T off = 0;
    if (!zero_start) {
        const T bxl = T(A.bx[p.fx0]), bxh = T(A.bx[p.fx1]);
        const T byl = T(A.by[p.fy0]), byh = T(A.by[p.fy1]);
        const T bzl = T(A.bz[p.fz0]), bzh = T(A.bz[p.fz1]);
        auto cor = [&](int ii, int jj, int kq) -> T {
            return kCorr ? xc[cix<T>(gc, ii >> 1, jj >> 1, kq >> 1)] : T(0);
        };
        const T xw = i > 0 ? (kCorr ? x[p.xw] + cor(i - 1, j, k) : x[p.xw]) : T(0);
        const T xe = i < g.nx - 1 ? (kCorr ? x[p.xe] + cor(i + 1, j, k) : x[p.xe]) : T(0);
        const T xs = j > 0 ? (kCorr ? x[c - sy] + cor(i, j - 1, k) : x[c - sy]) : T(0);
        const T xn = j < g.ny - 1 ? (kCorr ? x[c + sy] + cor(i, j + 1, k) : x[c + sy]) : T(0);
        const T xd = k > 0 ? (kCorr ? x[c - sz] + cor(i, j, k - 1) : x[c - sz]) : T(0);
        const T xu = k < g.nz - 1 ? (kCorr ? x[c + sz] + cor(i, j, k + 1) : x[c + sz]) : T(0);
        if (i > 0) off += bxl * xw;
        if (i < g.nx - 1) off += bxh * xe;
        if (j > 0) off += byl * xs;
        if (j < g.ny - 1) off += byh * xn;
        if (k > 0) off += bzl * xd;
        if (k < g.nz - 1) off += bzh * xu;
    }
    if constexpr (sizeof(T) == 4) return (bc + off) * A.dinv[c];
    return diag > T(0) ? (bc + off) / diag : T(0);
}

// kDot (the last pass of a V-cycle on the finest level): also block partials
// of b.x over both cells of every x-pair -- the updated one and its partner of
// the other colour, which this pass does not change -- i.e. r.z of the
// preconditioned CG, without a separate pass over both vectors.
template <class T, bool kCorr = false, bool kDot = false>
__global__ void __launch_bounds__(256) k_cc_gs(VOp<T> A, T *__restrict__ x, const T *__restrict__ b,
                                               int color, int zero_start, const T *__restrict__ xc = nullptr,
                                               GridD gc = GridD(), double *__restrict__ part = nullptr)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int kk = blockIdx.z * blockDim.z + threadIdx.z;
    const GridD &g = A.g;
    const bool act = 2 * t < g.nx && j < g.ny;
    if (!kDot && !act) return;   // (with kDot every thread reaches the block sum)
    T val[GS_PZ];
    int cc[GS_PZ];
#pragma unroll
    for (int h = 0; h < GS_PZ; h++) {
        const int k = GS_PZ * kk + h;
        const int i = 2 * t + ((j + k + color) & 1);
        cc[h] = -1;
        val[h] = T(0);
        if (!act || k >= g.nz || i >= g.nx) continue;
        cc[h] = cix<T>(g, i, j, k);
        val[h] = gs_cell<T, kCorr>(A, x, b, i, j, k, zero_start, xc, gc);
    }
    T dot = T(0);
#pragma unroll
    for (int h = 0; h < GS_PZ; h++) {
        if (zero_start) {
            const int k = GS_PZ * kk + h;
            const int io = 2 * t + 1 - ((j + k + color) & 1);
            if (k < g.nz && io < g.nx) x[cix<T>(g, io, j, k)] = T(0);
        }
        if (cc[h] >= 0) x[cc[h]] = val[h];
        if constexpr (kDot) {
            const int k = GS_PZ * kk + h;
            const int io = 2 * t + 1 - ((j + k + color) & 1);
            if (cc[h] >= 0) dot += b[cc[h]] * val[h];
            if (act && k < g.nz && io < g.nx) {
                const int co = cix<T>(g, io, j, k);
                dot += b[co] * x[co];
            }
        }
    }
    if constexpr (kDot) {
        const double sdot = block_sum3_t<T>(dot);
        if (thread_linear() == 0) part[block_linear()] = sdot;
    }
}

// The colour pass of k_cc_gs (plain form: no coarse correction, no r.z) for
// FP32 levels whose rows split into half-rows of a multiple of 4 cells (nx a
// multiple of 8): a thread updates 4 consecutive cells of its colour in one
// half-row of each of its kPz planes.  The row-split layout makes b, 1/diag,
// the y and z neighbours (the other colour at the same half-row position in
// the adjacent rows), the y and z faces and the result 16-byte (FP32) or
// 8-byte (BF16) vectors; the x neighbours are the other half-row's 4 values
// plus one beyond, the x faces 8 scalars.  Per cell the same operations in
// the same order as gs_cell, so the result is bit for bit that of k_cc_gs.
template <class F>
__device__ inline void load4(const F *p, float v[4])
{
    if constexpr (sizeof(F) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&q.x);
        const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&q.y);
        v[0] = __low2float(a); v[1] = __high2float(a); v[2] = __low2float(b); v[3] = __high2float(b);
    }
}

// kPz = 1 asks for 5 resident blocks per SM (at most 51 registers), kPz = 2
// for 4: one plane per thread and more warps, or two and more loads per warp.
// kCorr: the pass after the coarse-grid correction, as in k_cc_gs (each
// neighbour value plus its parent's coarse correction xc, level gc); its
// coarse rows in registers ask for 3 resident blocks per SM.
template <int kPz, bool kCorr = false>
__global__ void __launch_bounds__(256, kCorr ? 3 : (kPz == 1 ? 5 : 4)) k_cc_gs4(VOp<float> A, float *__restrict__ x,
                                                                 const float *__restrict__ b, int color,
                                                                 int zero_start, const float *__restrict__ xc = nullptr,
                                                                 GridD gc = GridD())
{
    using F = typename VFace<float>::type;
    const GridD &g = A.g;
    const int hx = g.nx >> 1;
    const int t0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int kb = (blockIdx.z * blockDim.z + threadIdx.z) * kPz;
    if (t0 >= hx || j >= g.ny) return;
    const int sy = g.nx, sz = g.nx * g.ny;
    float val[kPz][4];
    int pos[kPz], oth[kPz];
#pragma unroll
    for (int h = 0; h < kPz; h++) {
        const int k = kb + h;
        pos[h] = -1;
        if (k >= g.nz) continue;
        const int par = (color + j + k) & 1;            // i parity of this row's cells of the colour
        const int rc = (k * g.ny + j) * g.nx;
        const int c = rc + (par ? hx : 0) + t0;         // own half-row, cells t0 .. t0+3
        const int o = rc + (par ? 0 : hx) + t0;         // the other half-row, same positions
        pos[h] = c;
        oth[h] = o;
        float bc[4], di[4];
        load4(b + c, bc);
        load4(A.dinv + c, di);
        float off[4] = {0.f, 0.f, 0.f, 0.f};
        if (!zero_start) {
            float xo[4], xs[4], xn[4], xd[4], xu[4], fy0[4], fy1[4], fz0[4], fz1[4];
            load4(x + o, xo);
            const float xb = par ? (t0 + 4 < hx ? x[o + 4] : 0.f) : (t0 > 0 ? x[o - 1] : 0.f);
            if (j > 0) load4(x + c - sy, xs);
            if (j < g.ny - 1) load4(x + c + sy, xn);
            if (k > 0) load4(x + c - sz, xd);
            if (k < g.nz - 1) load4(x + c + sz, xu);
            load4(A.by + c + k * g.nx, fy0);
            load4(A.by + c + k * g.nx + g.nx, fy1);
            load4(A.bz + c, fz0);
            load4(A.bz + c + sz, fz1);
            const int rf = rc + k * g.ny + j, hf = (g.nx + 2) >> 1;
            // kCorr: the parents of the 4 cells' neighbours are the coarse cells
            // t0-1 .. t0+4 of the parent row and t0 .. t0+3 of the rows of the y
            // and z neighbours' parents; in the coarse row-split layout the even
            // and odd ones of t0 .. t0+3 are two 8-byte pairs of each row
            float cw[6] = {}, cs[4] = {}, cn[4] = {}, cd[4] = {}, cu[4] = {};
            if constexpr (kCorr) {
                const int hxc = gc.nx >> 1, tc = t0 >> 1;
                auto row4 = [&](int J, int K, float *o) {
                    const float *r0 = xc + (K * gc.ny + J) * gc.nx;
                    const float2 ev = *reinterpret_cast<const float2 *>(r0 + tc);
                    const float2 od = *reinterpret_cast<const float2 *>(r0 + hxc + tc);
                    o[0] = ev.x; o[1] = od.x; o[2] = ev.y; o[3] = od.y;
                };
                row4(j >> 1, k >> 1, cw + 1);
                const float *r0 = xc + ((k >> 1) * gc.ny + (j >> 1)) * gc.nx;
                cw[0] = t0 > 0 ? r0[hxc + tc - 1] : 0.f;          // coarse t0 - 1 (odd)
                cw[5] = t0 + 4 < gc.nx ? r0[tc + 2] : 0.f;         // coarse t0 + 4 (even)
                if (j > 0) row4((j - 1) >> 1, k >> 1, cs);
                if (j < g.ny - 1) row4((j + 1) >> 1, k >> 1, cn);
                if (k > 0) row4(j >> 1, (k - 1) >> 1, cd);
                if (k < g.nz - 1) row4(j >> 1, (k + 1) >> 1, cu);
            }
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const int t = t0 + m, i = 2 * t + par;
                const float bxl = float(A.bx[rf + (par ? hf + t : t)]);
                const float bxh = float(A.bx[rf + (par ? t + 1 : hf + t)]);
                float xw = par ? xo[m] : (m ? xo[m - 1] : xb);
                float xe = par ? (m < 3 ? xo[m + 1] : xb) : xo[m];
                float ys = xs[m], yn = xn[m], zd = xd[m], zu = xu[m];
                if constexpr (kCorr) {
                    // parent of i - 1 is coarse t - 1 + par, of i + 1 coarse t + par
                    if (i > 0) xw = xw + (par ? cw[m + 1] : cw[m]);
                    if (i < g.nx - 1) xe = xe + (par ? cw[m + 2] : cw[m + 1]);
                    if (j > 0) ys = ys + cs[m];
                    if (j < g.ny - 1) yn = yn + cn[m];
                    if (k > 0) zd = zd + cd[m];
                    if (k < g.nz - 1) zu = zu + cu[m];
                }
                float s = 0.f;
                if (i > 0) s += bxl * xw;
                if (i < g.nx - 1) s += bxh * xe;
                if (j > 0) s += fy0[m] * ys;
                if (j < g.ny - 1) s += fy1[m] * yn;
                if (k > 0) s += fz0[m] * zd;
                if (k < g.nz - 1) s += fz1[m] * zu;
                off[m] = s;
            }
        }
#pragma unroll
        for (int m = 0; m < 4; m++) val[h][m] = (bc[m] + off[m]) * di[m];
    }
#pragma unroll
    for (int h = 0; h < kPz; h++) {
        if (pos[h] < 0) continue;
        if (zero_start) *reinterpret_cast<float4 *>(x + oth[h]) = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4 *>(x + pos[h]) = make_float4(val[h][0], val[h][1], val[h][2], val[h][3]);
    }
}
inline bool gs4_ok(const GridD &g) { return (g.nx & 7) == 0; }
inline dim3 gs4_grid(const GridD &g, dim3 bk, int pz)
{
    const int nq = (g.nx >> 1) / 4, nzg = (g.nz + pz - 1) / pz;
    return dim3((nq + bk.x - 1) / bk.x, (g.ny + bk.y - 1) / bk.y, (nzg + bk.z - 1) / bk.z);
}
inline void launch_gs4(cudaStream_t st, dim3 bk, int pz, const VOp<float> &A, float *x, const float *b, int color,
                       int zs)
{
    if (pz == 1) k_cc_gs4<1><<<gs4_grid(A.g, bk, 1), bk, 0, st>>>(A, x, b, color, zs);
    else k_cc_gs4<2><<<gs4_grid(A.g, bk, 2), bk, 0, st>>>(A, x, b, color, zs);
}

// ---------------------------------------------------------------------------
// A whole red-black sweep in one pass (FP32 levels with nx a multiple of 16):
// the cells of colour c0 from the old values of the other colour, then the
// other colour from the new c0 values, read from x_in and written to x_out
// (the two passes in place give the same values, bit for bit: each cell is
// formed by the same operations in the same order as in gs_cell).
//
// A block owns a tile of RB_TX x RB_TY cells of every plane of a chunk of
// planes [z0, z1) and marches it in z.  Step m forms the first colour on
// plane m over the tile and a one-cell ring around it (the ring's values are
// the neighbours of the tile's second-colour cells; neighbouring blocks form
// them too), keeping three planes of these in shared memory, then the second
// colour on plane m-1 and writes plane m-1 (both colours).  Every operand
// comes in by TMA tile loads two steps ahead, completed on mbarriers: x (tile
// + 2-cell ring), b and 1/diag (tile + 1-cell ring), and the x, y and z face
// coefficients -- the x faces from a copy whose rows are padded to 16-byte
// strides (bxp: even faces then odd faces, each half RB_HXP(nx) long), since
// the stored rows hold nx + 1 entries.  No global load is left inside a
// step.  Per sweep every array is read once from DRAM (the rings come from
// L2) and x written once: 22 bytes per cell with BF16 faces instead of 28
// for two colour passes.
//
// Out-of-range tile coordinates load as zeros and the cells there are
// skipped; a neighbour outside the box is not read (the same tests as in
// gs_cell).  Each wait on a load is bounded (spin cycles of clock64); a wait
// that gives up sets E_TIMEOUT in ctl[C_ERR], waits (bounded) for the loads
// still in flight and ends the block, so the solve stops with that status
// instead of hanging.
// kZero: x_in is zero (not read).  kCorr: the first colour reads
// x_in + the coarse correction of the neighbour's parent (prolongation
// folded in, as in k_cc_gs); the coarse planes of the tile's parents come by
// TMA too (a RB_KW x 2 x RB_KR box per coarse plane, a three-slot ring, one
// new plane every other step), and each cell reads its four distinct parent
// values (its own parent and, per axis, the next coarse cell on the
// neighbour's side) once.  The first colour's results keep only that
// colour's half of each row.  kDot: also the partial b.x_out of every
// (plane, tile), part[plane * ntiles + tile], summed over the same cells in
// the same order as k_cc_gs2_dot, which forms them with the colour passes:
// in FP32 over a thread's cells and within the warp, in FP64 over the warps
// (FP64 arithmetic is scarce on this GPU: FP64 warp sums made each plane's
// partial cost more than the plane's loads).
constexpr int RB_TX = 64;                 // tile cells along x
constexpr int RB_HW = RB_TX / 2;          // half-row positions per tile
constexpr int RB_TY = 16;                 // tile rows
constexpr int RB_THREADS = RB_TY * (RB_HW / 2);   // one thread per 2 positions of a tile row
constexpr int RB_XW = RB_HW + 8;          // x / cell box width (FP32): 4 positions each side
constexpr int RB_FW = RB_HW + 16;         // face box width: 8 positions each side
constexpr int RB_XR = RB_TY + 4;          // rows of the x box
constexpr int RB_CR = RB_TY + 2;          // rows of the cell boxes (b, 1/diag, x and z faces, results)
constexpr int RB_YR = RB_TY + 3;          // rows of the y-face box
constexpr int RB_NBAR = 3;                // mbarriers (steps in flight + 1)
constexpr int RB_KW = 24;                 // coarse box width (half-row positions of the coarse level)
constexpr int RB_KR = RB_TY / 2 + 2;      // coarse box rows
static_assert(RB_THREADS == 256, "one thread per 2 positions of each tile row");
// half-row length of the padded x-face copy: nx/2 + 1 even faces, rounded up to 8
__host__ __device__ inline int rb_hxp(int nx) { return ((nx / 2 + 1) + 7) / 8 * 8; }

constexpr int al128(int b) { return (b + 127) / 128 * 128; }
template <class F>
struct RbSmem {
    static constexpr int bX = RB_XW * 2 * RB_XR * 4, bC = RB_XW * 2 * RB_CR * 4;
    static constexpr int bY = RB_FW * 2 * RB_YR * (int)sizeof(F), bZ = RB_FW * 2 * RB_CR * (int)sizeof(F);
    static constexpr int bR = RB_XW * RB_CR * 4, bK = RB_KW * 2 * RB_KR * 4;
    static constexpr int kX = al128(bX), kC = al128(bC), kY = al128(bY), kZ = al128(bZ);
    static constexpr int kR = al128(bR), kK = al128(bK);
    // x: planes m-1, m, m+1 and one ahead; b, 1/diag, x and y faces: m-1, m
    // and one ahead; z faces: face planes m-1 .. m+1 and one ahead; results
    // of the first colour (only its half of each row): planes m-2 .. m;
    // coarse correction (kCorr): coarse planes (m-1)/2 .. (m+1)/2 and one ahead
    static constexpr int oX = 0, oB = oX + 4 * kX, oD = oB + 3 * kC, oY = oD + 3 * kC, oZ = oY + 3 * kY;
    static constexpr int oXF = oZ + 4 * kZ, oR = oXF + 3 * kZ, oK = oR + 3 * kR, oBar = oK + 3 * kK;
    static constexpr int oMisc = oBar + 64;
    static constexpr int bytes = oMisc + 128;
};

template <class F>
struct RbArgs {
    GridD g;                // this level
    float *xout;
    double *part;           // kDot partials
    int *ctl;
    int c0, kz;             // first colour, planes per chunk
    long long spin;         // bound of one wait, clock64 cycles
};

struct RbMaps {
    CUtensorMap x, b, d, fx, fy, fz, xc;   // xc: the coarse correction (kCorr)
};

// Coarse planes step q loads (kCorr): step m needs coarse planes (m-1)/2 ..
// (m+1)/2 (floor division); the first step loads both of its, every later
// step the plane (m+1)/2 when it is new (m+1 even).  With three ring slots a
// load never lands on a slot a step in flight still reads.
__device__ inline int rb_coarse_count(int q, int m) { return q == 0 ? 2 : (((m + 1) & 1) == 0 ? 1 : 0); }

template <class F>
__device__ inline void rb_issue(unsigned char *sm, uint64_t *bar, int q, int m0, int p0, int y0, bool zero,
                                bool corr, const RbMaps &tm)
{
    using S = RbSmem<F>;
    const int m = m0 + q;
    uint64_t *b = bar + q % RB_NBAR;
    uint32_t bytes = 2 * S::bC + S::bY + 2 * S::bZ;
    if (!zero) bytes += (q == 0 ? 3 : 1) * S::bX;
    if (q == 0) bytes += S::bZ;
    if (corr) bytes += rb_coarse_count(q, m) * S::bK;
    mbar_arrive_expect_tx(b, bytes);
    if (corr) {
        const int nk = rb_coarse_count(q, m), cfirst = q == 0 ? ((m - 1) >> 1) : ((m + 1) >> 1);
        for (int t = 0; t < nk; t++) {
            const int C = cfirst + t;
            tma_load_4d(sm + S::oK + ((C + 3) % 3) * S::kK, &tm.xc, p0 / 2 - 4, 0, y0 / 2 - 1, C, b);
        }
    }
    if (!zero) {
        if (q == 0) {
            tma_load_4d(sm + S::oX + ((m - 1 + 8) & 3) * S::kX, &tm.x, p0 - 4, 0, y0 - 2, m - 1, b);
            tma_load_4d(sm + S::oX + ((m + 8) & 3) * S::kX, &tm.x, p0 - 4, 0, y0 - 2, m, b);
        }
        tma_load_4d(sm + S::oX + ((m + 1 + 8) & 3) * S::kX, &tm.x, p0 - 4, 0, y0 - 2, m + 1, b);
    }
    const int sb = (m + 3) % 3;
    tma_load_4d(sm + S::oB + sb * S::kC, &tm.b, p0 - 4, 0, y0 - 1, m, b);
    tma_load_4d(sm + S::oD + sb * S::kC, &tm.d, p0 - 4, 0, y0 - 1, m, b);
    tma_load_4d(sm + S::oY + sb * S::kY, &tm.fy, p0 - 8, 0, y0 - 1, m, b);
    tma_load_4d(sm + S::oXF + sb * S::kZ, &tm.fx, p0 - 8, 0, y0 - 1, m, b);
    if (q == 0) tma_load_4d(sm + S::oZ + ((m + 8) & 3) * S::kZ, &tm.fz, p0 - 8, 0, y0 - 1, m, b);
    tma_load_4d(sm + S::oZ + ((m + 1 + 8) & 3) * S::kZ, &tm.fz, p0 - 8, 0, y0 - 1, m + 1, b);
}

// Two consecutive face coefficients from shared memory (4- or 8-byte aligned) as floats.
template <class F>
__device__ inline float2 ld2f(const F *p)
{
    if constexpr (sizeof(F) == 4) {
        return *reinterpret_cast<const float2 *>(p);
    } else {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(p);
        return make_float2(__low2float(v), __high2float(v));
    }
}

template <class F, bool kZero, bool kCorr, bool kDot>
__global__ void __launch_bounds__(RB_THREADS, 2)
    k_cc_rb_sweep(const __grid_constant__ RbMaps tm, const RbArgs<F> a)
{
    using S = RbSmem<F>;
    extern __shared__ __align__(128) unsigned char sm[];
    const GridD &g = a.g;
    const int hx = g.nx >> 1;
    const int p0 = blockIdx.x * RB_HW, y0 = blockIdx.y * RB_TY;
    const int z0 = blockIdx.z * a.kz, z1 = min(g.nz, z0 + a.kz);
    if (z0 >= z1) return;
    const int tid = threadIdx.x, c1 = 1 - a.c0;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + S::oBar);
    int *flag = reinterpret_cast<int *>(sm + S::oMisc);
    double *wsum = reinterpret_cast<double *>(sm + S::oMisc + 16);
    const int m0 = z0 - 1, nstep = z1 - z0 + 2;
    auto X = [&](int pl) { return reinterpret_cast<const float *>(sm + S::oX + ((pl + 8) & 3) * S::kX); };
    auto Bv = [&](int pl) { return reinterpret_cast<const float *>(sm + S::oB + ((pl + 3) % 3) * S::kC); };
    auto Dv = [&](int pl) { return reinterpret_cast<const float *>(sm + S::oD + ((pl + 3) % 3) * S::kC); };
    auto FX = [&](int pl) { return reinterpret_cast<const F *>(sm + S::oXF + ((pl + 3) % 3) * S::kZ); };
    auto FY = [&](int pl) { return reinterpret_cast<const F *>(sm + S::oY + ((pl + 3) % 3) * S::kY); };
    auto FZ = [&](int pl) { return reinterpret_cast<const F *>(sm + S::oZ + ((pl + 8) & 3) * S::kZ); };
    // results of the first colour: row r, position q of that row's first-colour half
    auto R = [&](int pl) { return reinterpret_cast<float *>(sm + S::oR + ((pl + 3) % 3) * S::kR); };
    // the staged coarse correction (kCorr): coarse plane K, the entry of
    // coarse cell I in box row rw (a row offset from cor_row)
    auto Kpl = [&](int K) { return reinterpret_cast<const float *>(sm + S::oK + ((K + 3) % 3) * S::kK); };
    auto cor_row = [&](int J) { return (J - (y0 / 2 - 1)) * 2 * RB_KW; };
    auto cor_col = [&](int I) { return (I & 1) * RB_KW + (I >> 1) - (p0 / 2 - 4); };
    if (smem_u32(sm) & 127) {   // tile destinations must be 128-byte aligned: report, load nothing
        if (tid == 0) atomicCAS(a.ctl + C_ERR, 0, E_SMEM);
        return;
    }
    if (tid == 0) {
        for (int s = 0; s < RB_NBAR; s++) mbar_init(bar + s, 1);
        *flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        rb_issue<F>(sm, bar, 0, m0, p0, y0, kZero, kCorr, tm);
        rb_issue<F>(sm, bar, 1, m0, p0, y0, kZero, kCorr, tm);
    }
    // second colour and output: thread -> positions pq, pq+1 of both halves of tile row r
    const int r = tid >> 4, pq = p0 + 2 * (tid & 15);
    const int j2 = y0 + r;
    const bool own = j2 < g.ny && pq < hx;
    for (int q = 0; q < nstep; q++) {
        const int m = m0 + q;
        if (!mbar_wait_bounded(bar + q % RB_NBAR, (q / RB_NBAR) & 1, a.spin)) atomicExch(flag, 1);
        // first colour on plane m over the tile (two positions per thread)
        // and its one-cell ring (82 cells)
        if (m >= 0 && m < g.nz) {
            const float *X0 = X(m - 1), *X1 = X(m), *X2 = X(m + 1), *Bm = Bv(m), *Dm = Dv(m);
            const F *Fx = FX(m), *Fy = FY(m), *Fz0 = FZ(m), *Fz1 = FZ(m + 1);
            float *Rm = R(m);
            const int k = m;
            // coarse planes of the parents (k >> 1) and of the other z neighbour
            const float *Kk = nullptr, *Ko = nullptr;
            if (kCorr) {
                Kk = Kpl(k >> 1);
                Ko = Kpl((k >> 1) - 1 + 2 * (k & 1));
            }
            auto XI = [&](const float *Xp, int rr, int h2, int qq) { return Xp[(rr * 2 + h2) * RB_XW + qq]; };
            // one cell (i = 2p + h, j) of box row r1: the operations of gs_cell
            auto cell = [&](int r1, int j, int h, int p) {
                const int i = 2 * p + h, qx = p - p0 + 4, qf = p - p0 + 8;
                const int cc = (r1 * 2 + h) * RB_XW + qx;
                float off = 0.f;
                if (!kZero) {
                    const int rx = r1 + 1;
                    // x faces i (lo) and i + 1 (hi): even faces in half 0, odd in half 1
                    const float bxl = float(Fx[(r1 * 2 + h) * RB_FW + qf]);
                    const float bxh = float(Fx[(r1 * 2 + 1 - h) * RB_FW + qf + h]);
                    const float fy0 = float(Fy[(r1 * 2 + h) * RB_FW + qf]);
                    const float fy1 = float(Fy[((r1 + 1) * 2 + h) * RB_FW + qf]);
                    const float fz0 = float(Fz0[(r1 * 2 + h) * RB_FW + qf]);
                    const float fz1 = float(Fz1[(r1 * 2 + h) * RB_FW + qf]);
                    float xw = h ? XI(X1, rx, 0, qx) : XI(X1, rx, 1, qx - 1);
                    float xe = h ? XI(X1, rx, 0, qx + 1) : XI(X1, rx, 1, qx);
                    float xs = XI(X1, rx - 1, h, qx), xn = XI(X1, rx + 1, h, qx);
                    float xd = XI(X0, rx, h, qx), xu = XI(X2, rx, h, qx);
                    if (kCorr) {
                        // the neighbours' parents: this cell's (I = p, J, K) or, one
                        // per axis, the next coarse cell on the neighbour's side
                        const int rj = cor_row(j >> 1), ro = cor_row((j >> 1) - 1 + 2 * (j & 1));
                        const float co = Kk[rj + cor_col(p)], cx = Kk[rj + cor_col(h ? p + 1 : p - 1)];
                        const float cy = Kk[ro + cor_col(p)], cz = Ko[rj + cor_col(p)];
                        if (i > 0) xw = xw + (h ? co : cx);
                        if (i < g.nx - 1) xe = xe + (h ? cx : co);
                        if (j > 0) xs = xs + ((j & 1) ? co : cy);
                        if (j < g.ny - 1) xn = xn + ((j & 1) ? cy : co);
                        if (k > 0) xd = xd + ((k & 1) ? co : cz);
                        if (k < g.nz - 1) xu = xu + ((k & 1) ? cz : co);
                    }
                    if (i > 0) off += bxl * xw;
                    if (i < g.nx - 1) off += bxh * xe;
                    if (j > 0) off += fy0 * xs;
                    if (j < g.ny - 1) off += fy1 * xn;
                    if (k > 0) off += fz0 * xd;
                    if (k < g.nz - 1) off += fz1 * xu;
                }
                Rm[r1 * RB_XW + qx] = (Bm[cc] + off) * Dm[cc];
            };
            {   // the tile: positions p, p + 1 of row y0 + r, paired shared-memory loads
                const int j = y0 + r, h = (a.c0 + j + m) & 1, p = pq;
                if (own) {
                    const int r1 = r + 1, rx = r1 + 1, qx = p - p0 + 4, qf = p - p0 + 8;
                    const int ch = (r1 * 2 + h) * RB_XW + qx, cx = (rx * 2 + h) * RB_XW + qx;
                    const int co = (rx * 2 + 1 - h) * RB_XW + qx;   // the other half, same positions
                    const float2 bb = *reinterpret_cast<const float2 *>(Bm + ch);
                    const float2 dd = *reinterpret_cast<const float2 *>(Dm + ch);
                    float v[2];
                    if (!kZero) {
                        const float2 xs = *reinterpret_cast<const float2 *>(X1 + cx - 2 * RB_XW);
                        const float2 xn = *reinterpret_cast<const float2 *>(X1 + cx + 2 * RB_XW);
                        const float2 xd = *reinterpret_cast<const float2 *>(X0 + cx);
                        const float2 xu = *reinterpret_cast<const float2 *>(X2 + cx);
                        const float2 xo = *reinterpret_cast<const float2 *>(X1 + co);
                        // h = 1: neighbours (p, p+1 | p+1, p+2) of half 0; h = 0: (p-1, p | p, p+1) of half 1
                        const float xb = h ? X1[co + 2] : X1[co - 1];
                        const float xw2[2] = {h ? xo.x : xb, h ? xo.y : xo.x};
                        const float xe2[2] = {h ? xo.y : xo.x, h ? xb : xo.y};
                        const float2 fxl = ld2f(Fx + (r1 * 2 + h) * RB_FW + qf);
                        const float fxh0 = float(Fx[(r1 * 2 + 1 - h) * RB_FW + qf + h]);
                        const float fxh1 = float(Fx[(r1 * 2 + 1 - h) * RB_FW + qf + h + 1]);
                        const float2 fy0 = ld2f(Fy + (r1 * 2 + h) * RB_FW + qf);
                        const float2 fy1 = ld2f(Fy + ((r1 + 1) * 2 + h) * RB_FW + qf);
                        const float2 fz0 = ld2f(Fz0 + (r1 * 2 + h) * RB_FW + qf);
                        const float2 fz1 = ld2f(Fz1 + (r1 * 2 + h) * RB_FW + qf);
                        const float bxl[2] = {fxl.x, fxl.y}, bxh[2] = {fxh0, fxh1};
                        const float ys0[2] = {fy0.x, fy0.y}, ys1[2] = {fy1.x, fy1.y};
                        const float zs0[2] = {fz0.x, fz0.y}, zs1[2] = {fz1.x, fz1.y};
                        const float vs[2] = {xs.x, xs.y}, vn[2] = {xn.x, xn.y}, vd[2] = {xd.x, xd.y};
                        const float vu[2] = {xu.x, xu.y}, bv[2] = {bb.x, bb.y}, dv[2] = {dd.x, dd.y};
                        // the parents of the neighbours of cells 2(p+e)+h: coarse cells
                        // p+e (co) and, per axis, the next one on the neighbour's side
                        float co[2] = {0.f, 0.f}, cx[2] = {0.f, 0.f}, cy[2] = {0.f, 0.f}, cz[2] = {0.f, 0.f};
                        if (kCorr) {
                            const int rj = cor_row(j >> 1), ro = cor_row((j >> 1) - 1 + 2 * (j & 1));
                            const int i0 = cor_col(p), i1 = cor_col(p + 1);
                            co[0] = Kk[rj + i0];
                            co[1] = Kk[rj + i1];
                            const float ce = Kk[rj + cor_col(h ? p + 2 : p - 1)];
                            cx[0] = h ? co[1] : ce;
                            cx[1] = h ? ce : co[0];
                            cy[0] = Kk[ro + i0];
                            cy[1] = Kk[ro + i1];
                            cz[0] = Ko[rj + i0];
                            cz[1] = Ko[rj + i1];
                        }
#pragma unroll
                        for (int e = 0; e < 2; e++) {
                            const int i = 2 * (p + e) + h;
                            float xw = xw2[e], xe = xe2[e], xs_ = vs[e], xn_ = vn[e], xd_ = vd[e], xu_ = vu[e];
                            if (kCorr) {
                                if (i > 0) xw = xw + (h ? co[e] : cx[e]);
                                if (i < g.nx - 1) xe = xe + (h ? cx[e] : co[e]);
                                if (j > 0) xs_ = xs_ + ((j & 1) ? co[e] : cy[e]);
                                if (j < g.ny - 1) xn_ = xn_ + ((j & 1) ? cy[e] : co[e]);
                                if (k > 0) xd_ = xd_ + ((k & 1) ? co[e] : cz[e]);
                                if (k < g.nz - 1) xu_ = xu_ + ((k & 1) ? cz[e] : co[e]);
                            }
                            float off = 0.f;
                            if (i > 0) off += bxl[e] * xw;
                            if (i < g.nx - 1) off += bxh[e] * xe;
                            if (j > 0) off += ys0[e] * xs_;
                            if (j < g.ny - 1) off += ys1[e] * xn_;
                            if (k > 0) off += zs0[e] * xd_;
                            if (k < g.nz - 1) off += zs1[e] * xu_;
                            v[e] = (bv[e] + off) * dv[e];
                        }
                    } else {
                        v[0] = (bb.x + 0.f) * dd.x;
                        v[1] = (bb.y + 0.f) * dd.y;
                    }
                    *reinterpret_cast<float2 *>(Rm + r1 * RB_XW + qx) = make_float2(v[0], v[1]);
                }
            }
            // the ring: item t = tid / 3 of every third thread, spread over all warps
            const int t = tid / 3;
            if (tid % 3 == 0 && t < 2 * (RB_HW + 1) + RB_TY) {
                int r1, p;
                const int w = t < RB_HW + 1 ? t : t - (RB_HW + 1);
                if (t < 2 * (RB_HW + 1)) {
                    r1 = t < RB_HW + 1 ? 0 : RB_CR - 1;
                    const int j = y0 - 1 + r1, h = (a.c0 + j + m) & 1;
                    p = (h ? p0 - 1 : p0) + w;
                } else {
                    r1 = t - 2 * (RB_HW + 1) + 1;
                    const int j = y0 - 1 + r1, h = (a.c0 + j + m) & 1;
                    p = h ? p0 - 1 : p0 + RB_HW;
                }
                const int j = y0 - 1 + r1, h = (a.c0 + j + m) & 1;
                if (j >= 0 && j < g.ny && p >= 0 && p < hx) cell(r1, j, h, p);
            }
        }
        __syncthreads();
        if (*flag) {
            // a load did not arrive in time: record it, let the loads in
            // flight land (bounded) and stop this block
            if (tid == 0) {
                atomicCAS(a.ctl + C_ERR, 0, E_TIMEOUT);
                for (int s = q; s < min(nstep, q + 2); s++)
                    mbar_wait_bounded(bar + s % RB_NBAR, (s / RB_NBAR) & 1, kRbDrainCycles);
            }
            return;
        }
        // second colour on plane mm = m - 1, and the plane's output
        const int mm = m - 1;
        if (q >= 2) {
            float dsum = 0.f;   // (a thread's 4 cells, then the warp: FP32; the 8 warps: FP64)
            if (own) {
                const float *Rc = R(mm), *Bm = Bv(mm);
                const int rc = r + 1, qx = pq - p0 + 4, h2 = (c1 + j2 + mm) & 1;
                float s2[2], s1[2];   // second colour (computed), first colour (from R)
                {
                    const float *Rl = R(mm - 1), *Rh = R(mm + 1), *Dm = Dv(mm);
                    const F *Fx = FX(mm), *Fy = FY(mm), *Fz0 = FZ(mm), *Fz1 = FZ(mm + 1);
                    const int k = mm, j = j2, hh = h2, qf = qx + 4;
                    const int ch = (rc * 2 + hh) * RB_XW + qx, cr = rc * RB_XW + qx;
                    // paired loads: own half (b, 1/diag), and the first colour's results:
                    // the y and z neighbours (rows rc -+ 1, planes mm -+ 1) and the x
                    // neighbours (row rc) -- each row's first-colour half
                    const float2 bb = *reinterpret_cast<const float2 *>(Bm + ch);
                    const float2 dd = *reinterpret_cast<const float2 *>(Dm + ch);
                    const float2 xs = *reinterpret_cast<const float2 *>(Rc + cr - RB_XW);
                    const float2 xn = *reinterpret_cast<const float2 *>(Rc + cr + RB_XW);
                    const float2 xd = *reinterpret_cast<const float2 *>(Rl + cr);
                    const float2 xu = *reinterpret_cast<const float2 *>(Rh + cr);
                    const float2 xo = *reinterpret_cast<const float2 *>(Rc + cr);
                    const float xb = hh ? Rc[cr + 2] : Rc[cr - 1];
                    const float xw2[2] = {hh ? xo.x : xb, hh ? xo.y : xo.x};
                    const float xe2[2] = {hh ? xo.y : xo.x, hh ? xb : xo.y};
                    const float2 fxl = ld2f(Fx + (rc * 2 + hh) * RB_FW + qf);
                    const float bxh[2] = {float(Fx[(rc * 2 + 1 - hh) * RB_FW + qf + hh]),
                                          float(Fx[(rc * 2 + 1 - hh) * RB_FW + qf + hh + 1])};
                    const float2 fy0 = ld2f(Fy + (rc * 2 + hh) * RB_FW + qf);
                    const float2 fy1 = ld2f(Fy + ((rc + 1) * 2 + hh) * RB_FW + qf);
                    const float2 fz0 = ld2f(Fz0 + (rc * 2 + hh) * RB_FW + qf);
                    const float2 fz1 = ld2f(Fz1 + (rc * 2 + hh) * RB_FW + qf);
                    const float bxl[2] = {fxl.x, fxl.y}, ys0[2] = {fy0.x, fy0.y}, ys1[2] = {fy1.x, fy1.y};
                    const float zs0[2] = {fz0.x, fz0.y}, zs1[2] = {fz1.x, fz1.y};
                    const float vs[2] = {xs.x, xs.y}, vn[2] = {xn.x, xn.y}, vd[2] = {xd.x, xd.y};
                    const float vu[2] = {xu.x, xu.y}, bv[2] = {bb.x, bb.y}, dv[2] = {dd.x, dd.y};
                    s1[0] = xo.x;
                    s1[1] = xo.y;
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const int i = 2 * (pq + e) + hh;
                        float off = 0.f;
                        if (i > 0) off += bxl[e] * xw2[e];
                        if (i < g.nx - 1) off += bxh[e] * xe2[e];
                        if (j > 0) off += ys0[e] * vs[e];
                        if (j < g.ny - 1) off += ys1[e] * vn[e];
                        if (k > 0) off += zs0[e] * vd[e];
                        if (k < g.nz - 1) off += zs1[e] * vu[e];
                        s2[e] = (bv[e] + off) * dv[e];
                    }
                }
                float v[2][2];
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    v[0][e] = h2 ? s1[e] : s2[e];
                    v[1][e] = h2 ? s2[e] : s1[e];
                }
                float *o = a.xout + (size_t)(mm * g.ny + j2) * g.nx + pq;
                *reinterpret_cast<float2 *>(o) = make_float2(v[0][0], v[0][1]);
                *reinterpret_cast<float2 *>(o + hx) = make_float2(v[1][0], v[1][1]);
                if constexpr (kDot) {
                    float d = 0.f;
#pragma unroll
                    for (int h = 0; h < 2; h++)
#pragma unroll
                        for (int e = 0; e < 2; e++) d += Bm[(rc * 2 + h) * RB_XW + qx + e] * v[h][e];
                    dsum = d;
                }
            }
            if constexpr (kDot) {
                for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
                if ((tid & 31) == 0) wsum[tid >> 5] = (double)dsum;
            }
        }
        __syncthreads();
        // the plane's partial from the warp sums (FP64) in warp 1, so that
        // thread 0 issues the next loads at once
        if (kDot && q >= 2 && tid == 32) {
            double s = 0.0;
            for (int w = 0; w < RB_THREADS / 32; w++) s += wsum[w];
            a.part[(size_t)mm * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x] = s;
        }
        if (tid == 0 && q + 2 < nstep) {
            fence_proxy_async();
            rb_issue<F>(sm, bar, q + 2, m0, p0, y0, kZero, kCorr, tm);
        }
    }
}

// The padded copy of the x-face coefficients that k_cc_rb_sweep loads: per
// row, the nx/2 + 1 even faces then, from position rb_hxp(nx), the nx/2 odd
// ones (zeros in the padding), converted as the V-cycle's copy is.
template <class F>
__global__ void k_xface_pad(GridD g, const float *__restrict__ bf, F *__restrict__ out)
{
    const int hxp = rb_hxp(g.nx), hf = g.nx / 2 + 1, hx = g.nx / 2;
    const long long n = 2LL * hxp * g.ny * g.nz;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int pos = (int)(s % hxp);
        const long long rh = s / hxp;
        const int half = (int)(rh & 1);
        const long long row = rh >> 1;
        const long long rf = row * (g.nx + 1);
        float v = 0.f;
        if (half == 0 && pos < hf) v = bf[rf + pos];
        if (half == 1 && pos < hx) v = bf[rf + hf + pos];
        if constexpr (sizeof(F) == 2) out[s] = __float2bfloat16_rn(v);
        else out[s] = v;
    }
}

// The fused sweep's face type: the V-cycle's.
using RbF = typename VFace<float>::type;

// The second colour pass of a sweep (colour c1, plain) together with the
// (plane, tile) partials of b.x that k_cc_rb_sweep<kDot> forms: the same
// threads (positions pq, pq+1 of both halves of a tile row), cells, order
// and sums, so the colour passes end with the fused sweep's r.z bit for bit.
// Each c1 cell is formed by the operations of gs_cell; the other colour is
// read (unchanged by this pass) for the partial.  A block covers
// kGs2Planes planes of its tile (the loads of all of them in flight
// together), each plane's partial reduced on its own.  Grid (tiles x,
// tiles y, ceil(nz / kGs2Planes)).
constexpr int kGs2Planes = 4;
__global__ void __launch_bounds__(RB_THREADS) k_cc_gs2_dot(VOp<float> A, float *__restrict__ x,
                                                            const float *__restrict__ b, int c1,
                                                            double *__restrict__ part)
{
    __shared__ double wsum[kGs2Planes][RB_THREADS / 32];
    const GridD &g = A.g;
    const int tid = threadIdx.x, hx = g.nx >> 1, hf = (g.nx + 2) >> 1;
    const int r = tid >> 4;
    const int j = blockIdx.y * RB_TY + r, pq = blockIdx.x * RB_HW + 2 * (tid & 15);
    const int sy = g.nx, sz = g.nx * g.ny;
    float dsum[kGs2Planes];
#pragma unroll
    for (int pl = 0; pl < kGs2Planes; pl++) {
        const int k = blockIdx.z * kGs2Planes + pl;
        dsum[pl] = 0.f;
        if (j >= g.ny || pq >= hx || k >= g.nz) continue;
        const int h2 = (c1 + j + k) & 1;
        const int rc = (k * g.ny + j) * g.nx;
        const int c = rc + (h2 ? hx : 0) + pq, o = rc + (h2 ? 0 : hx) + pq;
        const float2 bb = *reinterpret_cast<const float2 *>(b + c);
        const float2 bo = *reinterpret_cast<const float2 *>(b + o);
        const float2 di = *reinterpret_cast<const float2 *>(A.dinv + c);
        const float2 xo = *reinterpret_cast<const float2 *>(x + o);
        const float xb = h2 ? (pq + 2 < hx ? x[o + 2] : 0.f) : (pq > 0 ? x[o - 1] : 0.f);
        float2 xs = make_float2(0.f, 0.f), xn = xs, xd = xs, xu = xs;
        if (j > 0) xs = *reinterpret_cast<const float2 *>(x + c - sy);
        if (j < g.ny - 1) xn = *reinterpret_cast<const float2 *>(x + c + sy);
        if (k > 0) xd = *reinterpret_cast<const float2 *>(x + c - sz);
        if (k < g.nz - 1) xu = *reinterpret_cast<const float2 *>(x + c + sz);
        const float2 fy0 = ld2f(A.by + c + k * g.nx), fy1 = ld2f(A.by + c + k * g.nx + g.nx);
        const float2 fz0 = ld2f(A.bz + c), fz1 = ld2f(A.bz + c + sz);
        const float xw2[2] = {h2 ? xo.x : xb, h2 ? xo.y : xo.x};
        const float xe2[2] = {h2 ? xo.y : xo.x, h2 ? xb : xo.y};
        const float ys0[2] = {fy0.x, fy0.y}, ys1[2] = {fy1.x, fy1.y}, zs0[2] = {fz0.x, fz0.y}, zs1[2] = {fz1.x, fz1.y};
        const float vs[2] = {xs.x, xs.y}, vn[2] = {xn.x, xn.y}, vd[2] = {xd.x, xd.y}, vu[2] = {xu.x, xu.y};
        const float bv[2] = {bb.x, bb.y}, dv[2] = {di.x, di.y};
        const int rf = rc + k * g.ny + j;
        float s2[2];
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int t = pq + e, i = 2 * t + h2;
            const float bxl = float(A.bx[rf + (h2 ? hf + t : t)]);
            const float bxh = float(A.bx[rf + (h2 ? t + 1 : hf + t)]);
            float off = 0.f;
            if (i > 0) off += bxl * xw2[e];
            if (i < g.nx - 1) off += bxh * xe2[e];
            if (j > 0) off += ys0[e] * vs[e];
            if (j < g.ny - 1) off += ys1[e] * vn[e];
            if (k > 0) off += zs0[e] * vd[e];
            if (k < g.nz - 1) off += zs1[e] * vu[e];
            s2[e] = (bv[e] + off) * dv[e];
        }
        *reinterpret_cast<float2 *>(x + c) = make_float2(s2[0], s2[1]);
        // b.x over the 4 cells, half 0 then half 1, as k_cc_rb_sweep<kDot>
        const float b0[2] = {h2 ? bo.x : bb.x, h2 ? bo.y : bb.y}, b1[2] = {h2 ? bb.x : bo.x, h2 ? bb.y : bo.y};
        const float v0[2] = {h2 ? xo.x : s2[0], h2 ? xo.y : s2[1]}, v1[2] = {h2 ? s2[0] : xo.x, h2 ? s2[1] : xo.y};
        float d = 0.f;
        d += b0[0] * v0[0];
        d += b0[1] * v0[1];
        d += b1[0] * v1[0];
        d += b1[1] * v1[1];
        dsum[pl] = d;
    }
    // per warp in FP32, across the 8 warps in FP64 (as k_cc_rb_sweep<kDot>)
#pragma unroll
    for (int pl = 0; pl < kGs2Planes; pl++) {
        float v = dsum[pl];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) wsum[pl][tid >> 5] = (double)v;
    }
    __syncthreads();
    if (tid < kGs2Planes) {
        const int k = blockIdx.z * kGs2Planes + tid;
        if (k < g.nz) {
            double s = 0.0;
            for (int w = 0; w < RB_THREADS / 32; w++) s += wsum[tid][w];
            part[(size_t)k * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x] = s;
        }
    }
}

// Residual of the 8 children of coarse cell (I,J,K), averaged.
template <class T>
__device__ inline T rr_cell(const VOp<T> &A, const T *__restrict__ x, const T *__restrict__ b, int I, int J,
                            int K)
{
    // child by child with the layout's index functions: with the children's
    // parities known after unrolling these fold to row offsets in few
    // registers (this kernel is latency-bound: occupancy counts more).
    // Only the 4 red children ((i+j+k) even) are summed: the restriction
    // follows pre-smoothing whose last pass updated every black cell from its
    // current neighbours, so a black cell's residual is 0 up to rounding.
    const GridD &g = A.g;
    T s = 0;
#pragma unroll
    for (int o = 0; o < 8; o++) {
        if (__popc(o) & 1) continue;   // black child
        const int i = 2 * I + (o & 1), j = 2 * J + ((o >> 1) & 1), k = 2 * K + ((o >> 2) & 1);
        const int c = cix<T>(g, i, j, k);
        const T bxl = T(A.bx[fidxT<T>(g, 0, i, j, k)]), bxh = T(A.bx[fidxT<T>(g, 0, i + 1, j, k)]);
        const T byl = T(A.by[fidxT<T>(g, 1, i, j, k)]), byh = T(A.by[fidxT<T>(g, 1, i, j + 1, k)]);
        const T bzl = T(A.bz[fidxT<T>(g, 2, i, j, k)]), bzh = T(A.bz[fidxT<T>(g, 2, i, j, k + 1)]);
        T off = 0;
        if (i > 0) off += bxl * x[cix<T>(g, i - 1, j, k)];
        if (i < g.nx - 1) off += bxh * x[cix<T>(g, i + 1, j, k)];
        if (j > 0) off += byl * x[c - g.nx];
        if (j < g.ny - 1) off += byh * x[c + g.nx];
        if (k > 0) off += bzl * x[c - g.nx * g.ny];
        if (k < g.nz - 1) off += bzh * x[c + g.nx * g.ny];
        s += b[c] - (A.diag[c] * x[c] - off);
    }
    return s * T(0.125);
}

// Residual of the 8 children, averaged into the coarse right-hand side.
template <class T>
__global__ void __launch_bounds__(256) k_cc_resid_restrict(VOp<T> A, const T *__restrict__ x,
                                                           const T *__restrict__ b, GridD gc,
                                                           T *__restrict__ bc)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z * blockDim.z + threadIdx.z;
    if (I >= gc.nx || J >= gc.ny || K >= gc.nz) return;
    bc[cix<T>(gc, I, J, K)] = rr_cell<T>(A, x, b, I, J, K);
}

// k_cc_resid_restrict for FP32 levels with nx a multiple of 8: a thread
// forms coarse cells I0 .. I0+3 (I0 = 4t) of coarse row (J, K).  Their red
// children lie in one half of each of the 4 fine rows (2J+jj, 2K+kk) -- the
// half of parity (j + k) & 1 -- at the consecutive positions I0 .. I0+3, so
// x, b, the diagonal, the y and z neighbours and faces are 16-byte (8-byte
// BF16) vectors, as in k_cc_gs4.  Children and operations in the order of
// rr_cell (rows (2J,2K), (2J+1,2K), (2J,2K+1), (2J+1,2K+1)), so the results
// are the same bits; the coarse values go out as two 8-byte pairs (even and
// odd coarse cells are the two halves of the coarse row).  Bound by load
// latency: capped at 64 registers (from 75) for four blocks per SM, 16 %
// faster at 256^3.
__global__ void __launch_bounds__(256, 4) k_cc_rr4(VOp<float> A, const float *__restrict__ x,
                                               const float *__restrict__ b, GridD gc, float *__restrict__ bc)
{
    const GridD &g = A.g;
    const int hx = g.nx >> 1, hf = (g.nx + 2) >> 1;
    const int I0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z * blockDim.z + threadIdx.z;
    if (I0 >= gc.nx || J >= gc.ny || K >= gc.nz) return;
    const int sy = g.nx, sz = g.nx * g.ny;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 2; kk++)
#pragma unroll
        for (int jj = 0; jj < 2; jj++) {
            const int j = 2 * J + jj, k = 2 * K + kk, h = (j + k) & 1;
            const int rc = (k * g.ny + j) * g.nx;
            const int c = rc + (h ? hx : 0) + I0, o = rc + (h ? 0 : hx) + I0;
            float xc4[4], bb[4], dg[4], xo[4], xs[4], xn[4], xd[4], xu[4], fy0[4], fy1[4], fz0[4], fz1[4];
            load4(x + c, xc4);
            load4(b + c, bb);
            load4(A.diag + c, dg);
            load4(x + o, xo);
            const float xb = h ? (I0 + 4 < hx ? x[o + 4] : 0.f) : (I0 > 0 ? x[o - 1] : 0.f);
            if (j > 0) load4(x + c - sy, xs);
            if (j < g.ny - 1) load4(x + c + sy, xn);
            if (k > 0) load4(x + c - sz, xd);
            if (k < g.nz - 1) load4(x + c + sz, xu);
            load4(A.by + c + k * g.nx, fy0);
            load4(A.by + c + k * g.nx + g.nx, fy1);
            load4(A.bz + c, fz0);
            load4(A.bz + c + sz, fz1);
            const int rf = rc + k * g.ny + j;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int t = I0 + e, i = 2 * t + h;
                const float bxl = float(A.bx[rf + (h ? hf + t : t)]);
                const float bxh = float(A.bx[rf + (h ? t + 1 : hf + t)]);
                const float xw = h ? xo[e] : (e ? xo[e - 1] : xb);
                const float xe = h ? (e < 3 ? xo[e + 1] : xb) : xo[e];
                float off = 0.f;
                if (i > 0) off += bxl * xw;
                if (i < g.nx - 1) off += bxh * xe;
                if (j > 0) off += fy0[e] * xs[e];
                if (j < g.ny - 1) off += fy1[e] * xn[e];
                if (k > 0) off += fz0[e] * xd[e];
                if (k < g.nz - 1) off += fz1[e] * xu[e];
                acc[e] += bb[e] - (dg[e] * xc4[e] - off);
            }
        }
    const int hxc = gc.nx >> 1;
    float *row = bc + (K * gc.ny + J) * gc.nx;
    *reinterpret_cast<float2 *>(row + (I0 >> 1)) = make_float2(acc[0] * 0.125f, acc[2] * 0.125f);
    *reinterpret_cast<float2 *>(row + hxc + (I0 >> 1)) = make_float2(acc[1] * 0.125f, acc[3] * 0.125f);
}

// Rediscretised coarse operator: face coefficient = (sum of the 4 fine faces) / 16,
// extra = sum over uncovered children / 8 (identity where all children are covered).
template <class T>
__global__ void k_cc_coarsen(GridD gf, const T *__restrict__ ef, const T *__restrict__ bxf,
                             const T *__restrict__ byf, const T *__restrict__ bzf,
                             const uint8_t *__restrict__ covf, GridD gc, const uint8_t *__restrict__ covc,
                             T *__restrict__ ec, T *__restrict__ bxc, T *__restrict__ byc,
                             T *__restrict__ bzc)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z * blockDim.z + threadIdx.z;
    if (I > gc.nx || J > gc.ny || K > gc.nz) return;
    if (I < gc.nx && J < gc.ny && K < gc.nz) {
        const int C = cix<T>(gc, I, J, K);
        if (covc[cidx(gc, I, J, K)]) {
            ec[C] = T(1);
        } else {
            T s = 0;
            for (int o = 0; o < 8; o++) {
                const int i = 2 * I + (o & 1), j = 2 * J + ((o >> 1) & 1), k = 2 * K + ((o >> 2) & 1);
                if (!covf[cidx(gf, i, j, k)]) s += ef[cix<T>(gf, i, j, k)];
            }
            ec[C] = s * T(0.125);
        }
    }
    const T *bf[3] = {bxf, byf, bzf};
    T *bcs[3] = {bxc, byc, bzc};
    const int m[3] = {gc.nx, gc.ny, gc.nz};
    for (int d = 0; d < 3; d++) {
        int id[3] = {I, J, K};
        bool ok = true;
        for (int e = 0; e < 3; e++) ok &= (e == d) ? id[e] <= m[e] : id[e] < m[e];
        if (!ok) continue;
        int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
        T s = 0;
        for (int q1 = 0; q1 < 2; q1++)
            for (int q2 = 0; q2 < 2; q2++) {
                int f[3] = {2 * I, 2 * J, 2 * K};
                f[t1] += q1;
                f[t2] += q2;
                s += bf[d][fidxT<T>(gf, d, f[0], f[1], f[2])];
            }
        bcs[d][fidxT<T>(gc, d, I, J, K)] = s * T(0.0625);
    }
}

// diag = extra + the six face coefficients of the cell, for each of nvar
// variants of the operator: a face on box side s counts for variant q only if
// bit s of side mask q (bits 6q .. 6q+5 of masks) is set.  Sums in the same
// order for every variant, so a variant with all bits set is the plain sum.
// kRound: the faces as the V-cycle stores them (rounded to BF16), so that its
// operator keeps diag = extra + sum of its own faces.
template <class T, bool kRound = false>
__global__ void k_cc_make_diag(GridD g, const T *__restrict__ extra, const T *__restrict__ bx,
                               const T *__restrict__ by, const T *__restrict__ bz, int nvar, unsigned masks,
                               T *__restrict__ d0, T *__restrict__ d1, T *__restrict__ d2,
                               T *__restrict__ i0 = nullptr, T *__restrict__ i1 = nullptr,
                               T *__restrict__ i2 = nullptr)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const int c = cix<T>(g, i, j, k);
    const T e = extra[c];
    T f[6] = {bx[fidxT<T>(g, 0, i, j, k)], bx[fidxT<T>(g, 0, i + 1, j, k)],
              by[fidxT<T>(g, 1, i, j, k)], by[fidxT<T>(g, 1, i, j + 1, k)],
              bz[fidxT<T>(g, 2, i, j, k)], bz[fidxT<T>(g, 2, i, j, k + 1)]};
    if constexpr (kRound) {
#pragma unroll
        for (int t = 0; t < 6; t++) f[t] = __bfloat162float(__float2bfloat16_rn(f[t]));
    }
    // box side of each face, -1 for a face between two cells
    const int sd[6] = {i == 0 ? 0 : -1, i == g.nx - 1 ? 1 : -1, j == 0 ? 2 : -1,
                       j == g.ny - 1 ? 3 : -1, k == 0 ? 4 : -1, k == g.nz - 1 ? 5 : -1};
    T *out[3] = {d0, d1, d2};
    T *inv[3] = {i0, i1, i2};
    for (int q = 0; q < nvar; q++) {
        const unsigned m = masks >> (6 * q);
        T s = e;
#pragma unroll
        for (int t = 0; t < 6; t++) s += (sd[t] < 0 || ((m >> sd[t]) & 1u)) ? f[t] : T(0);
        out[q][c] = s;
        if (inv[q]) inv[q][c] = s > T(0) ? T(1) / s : T(0);
    }
}

__global__ void k_cov_coarsen(GridD gf, const uint8_t *covf, GridD gc, uint8_t *covc)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z * blockDim.z + threadIdx.z;
    if (I >= gc.nx || J >= gc.ny || K >= gc.nz) return;
    int all = 1;
    for (int o = 0; o < 8; o++)
        all &= covf[cidx(gf, 2 * I + (o & 1), 2 * J + ((o >> 1) & 1), 2 * K + ((o >> 2) & 1))];
    covc[cidx(gc, I, J, K)] = (uint8_t)all;
}

__global__ void k_cov_from_flag(int n, const uint8_t *flag, uint8_t *cov)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        cov[s] = flag[s] == 0;
}

template <class S, class D>
__global__ void k_convert(const S *__restrict__ a, D *__restrict__ b, int n)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        b[s] = (D)a[s];
}

// FP64 natural-order array of cells (d < 0) or of faces of normal d -> FP32
// row-split copy.
__global__ void k_to_split(GridD g, int d, const double *__restrict__ a, float *__restrict__ b,
                           const double *__restrict__ sig = nullptr)
{
    const int mx = g.nx + (d == 0), my = g.ny + (d == 1), mz = g.nz + (d == 2);
    const int n = mx * my * mz;
    const double sc = sig ? *sig : 1.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const int i = s % mx, j = (s / mx) % my, k = s / (mx * my);
        b[d < 0 ? cix<float>(g, i, j, k) : fidxT<float>(g, d, i, j, k)] = f64_to_f32_pow2(a[s], sc);
    }
}

// r = sig * a in FP32 (the refinement solver's first residual, natural order)
__global__ void k_to32_scaled(const double *__restrict__ a, float *__restrict__ b, int n,
                              const double *__restrict__ sig)
{
    const double sc = *sig;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        b[s] = f64_to_f32_pow2(a[s], sc);
}

// FP32 face coefficients -> the V-cycle's BF16 copy (same layout)
__global__ void k_to_bf16(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, int n)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        b[s] = __float2bfloat16_rn(a[s]);
}


// Level-0 coefficients of the cell-centred projection: beta = a_f / h^2,
// 2 a_f / h^2 on outflow faces (phi = 0 there), 0 on other box faces.
__global__ void k_mac_coeffs(GridD g, const uint8_t *__restrict__ flag, const double *__restrict__ ax,
                             const double *__restrict__ ay, const double *__restrict__ az,
                             double *__restrict__ extra, double *__restrict__ bx, double *__restrict__ by,
                             double *__restrict__ bz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const double h2 = g.h * g.h;
    if (i < g.nx && j < g.ny && k < g.nz) {
        int c = cidx(g, i, j, k);
        extra[c] = flag[c] ? 0.0 : 1.0;
    }
    const double *A[3] = {ax, ay, az};
    double *B[3] = {bx, by, bz};
    int id[3] = {i, j, k};
    for (int d = 0; d < 3; d++) {
        bool ok = true;
        for (int e = 0; e < 3; e++) ok &= (e == d) ? id[e] <= dimn(g, e) : id[e] < dimn(g, e);
        if (!ok) continue;
        int f = fidx(g, d, i, j, k);
        if (id[d] == 0 || id[d] == dimn(g, d)) {
            int side = 2 * d + (id[d] != 0);
            B[d][f] = (g.bc[side] == EBV_OUTFLOW || pin_face(g, d, i, j, k)) ? 2.0 * A[d][f] / h2 : 0.0;
        } else {
            B[d][f] = A[d][f] / h2;
        }
    }
}

// Level-0 coefficients of the viscous solves (Eq. implicit-viscous,
// alpha-weighted), shared by the three velocity components:
//   extra = rho alpha + dt eta A_EB / (h^2 delta), delta = max(-n.b, delta_min)
//   beta  = dt a_f eta_f / h^2, eta_f the mean of the two cells; on a box face
//           2 dt a_f eta / h^2, the coefficient of a Dirichlet condition there.
// A box face enters the diagonal of component q only where the side is a
// Dirichlet side for q (k_cc_make_diag's side masks); its value enters the
// right-hand side (k_visc_rhs).
__global__ void k_visc_coeffs(GridD g, GeomD geo, ParamsD p, const double *__restrict__ eta,
                              const double *__restrict__ dtp, double *__restrict__ extra,
                              double *__restrict__ bx, double *__restrict__ by, double *__restrict__ bz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const double h2 = g.h * g.h, dt = dtp[DT_DT];
    const double dth2 = dtp[DT_DTH2];  // dt / h^2
    const int N3 = geo.ncell;
    const double *A[3] = {geo.ax, geo.ay, geo.az};
    double *B[3] = {bx, by, bz};
    int id[3] = {i, j, k};
    for (int d = 0; d < 3; d++) {
        bool ok = true;
        for (int e = 0; e < 3; e++) ok &= (e == d) ? id[e] <= dimn(g, e) : id[e] < dimn(g, e);
        if (!ok) continue;
        int f = fidx(g, d, i, j, k);
        double a = A[d][f];
        if (id[d] == 0 || id[d] == dimn(g, d)) {
            int cc[3] = {i, j, k};
            cc[d] -= id[d] != 0;
            B[d][f] = a > 0.0 ? 2.0 * dth2 * a * eta[cidx(g, cc[0], cc[1], cc[2])] : 0.0;
        } else {
            int lo[3] = {i, j, k};
            lo[d] -= 1;
            double ef = 0.5 * (eta[cidx(g, lo[0], lo[1], lo[2])] + eta[cidx(g, i, j, k)]);
            B[d][f] = a > 0.0 ? dth2 * a * ef : 0.0;
        }
    }
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const int c = cidx(g, i, j, k);
    if (geo.flag[c] == 0) {
        extra[c] = 1.0;
        return;
    }
    double e = p.rho * geo.alpha[c];
    if (geo.flag[c] == 2 && geo.area[c] > 0.0) {
        double nb = 0.0;
        for (int q = 0; q < 3; q++) nb += geo.nrm[q * N3 + c] * geo.bcen[q * N3 + c];
        double del = -nb > p.delta_min ? -nb : p.delta_min;
        e += dt * eta[c] * geo.area[c] / (h2 * del);
    }
    extra[c] = e;
}

// Right-hand side of the viscous solve of component comp: alpha psi plus, for
// each box face of the cell on a Dirichlet side of comp, its coefficient
// (k_visc_coeffs) times the boundary value.
__global__ void k_visc_rhs(GridD g, GeomD geo, int comp, const double *__restrict__ psi,
                           const double *__restrict__ bx, const double *__restrict__ by,
                           const double *__restrict__ bz, double *__restrict__ b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const int c = cidx(g, i, j, k);
    if (geo.flag[c] == 0) {
        b[c] = 0.0;
        return;
    }
    const double *B[3] = {bx, by, bz};
    const int id[3] = {i, j, k};
    double rb = 0.0;
    for (int d = 0; d < 3; d++)
        for (int hs = 0; hs < 2; hs++) {
            int pos = id[d] + hs;
            if (pos != 0 && pos != dimn(g, d)) continue;
            int fi[3] = {i, j, k};
            fi[d] += hs;
            double val;
            if (side_dirichlet(g, 2 * d + hs, comp, &val)) rb += B[d][fidx(g, d, fi[0], fi[1], fi[2])] * val;
        }
    b[c] = geo.alpha[c] * psi[c] + rb;
}

// q = A p (level 0) and block partials of p.q in FP64 (per thread and warp
// in T, see block_sum3_t).  Each thread handles planes 2kk and 2kk+1 of
// column (i, j).  With kRes (FP64) instead the residual r = b - A p, stored
// as an FP32 row-split vector, with block partials of |r|^2 (the refinement
// solver's true residual in one pass; |r|^2 only decides convergence, so it
// is summed from the stored FP32 values, per thread and warp in FP32).
template <class T, bool kRes = false>
__global__ void __launch_bounds__(256) k_cc_apply_dot(CcOp<T> A, const T *__restrict__ p, T *__restrict__ q,
                                                      double *__restrict__ part, const T *__restrict__ b = nullptr,
                                                      float *__restrict__ r32 = nullptr,
                                                      const double *__restrict__ sig = nullptr)
{
    const double sc = (kRes && sig) ? *sig : 1.0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int kk = blockIdx.z * blockDim.z + threadIdx.z;
    T v = 0;
    float vr = 0.0f;
    if (i < A.g.nx && j < A.g.ny) {
        T y[2], pc[2];
        int cc[2] = {-1, -1};
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int k = 2 * kk + h;
            if (k >= A.g.nz) continue;
            T diag, off;
            cc_row(A, i, j, k, p, diag, off);
            cc[h] = cix<T>(A.g, i, j, k);
            pc[h] = p[cc[h]];
            y[h] = diag * pc[h] - off;
        }
#pragma unroll
        for (int h = 0; h < 2; h++)
            if (cc[h] >= 0) {
                if constexpr (kRes) {
                    const float r = f64_to_f32_pow2(b[cc[h]] - y[h], sc);
                    r32[cix<float>(A.g, i, j, 2 * kk + h)] = r;
                    vr += r * r;
                } else {
                    q[cc[h]] = y[h];
                    v += pc[h] * y[h];
                }
            }
    }
    const double vs = kRes ? block_sum3_t<float>(vr) : block_sum3_t<T>(v);
    if (thread_linear() == 0) part[block_linear()] = vs;
}

// k_cc_apply_dot<float> for levels with nx a multiple of 8: a thread forms
// q = A p at 4 consecutive cells of one half-row (half h = tx / nq) in each of
// two planes, with 16-byte loads as in k_cc_gs4 (the x faces, rows of nx + 1,
// as scalars), and adds p.q of its 8 cells to its block's partial.  Each q is
// formed as in cc_row; the partial sums are grouped by this kernel's fixed
// block shape (kApply4Blk).  (A cap of 48 registers, for five blocks per SM,
// measures no faster than 64 registers and four blocks.)
constexpr int kApply4X = 16, kApply4Y = 8, kApply4Z = 2;
// The vectorised apply and restriction serve grids where they launch at least
// this many blocks (two per SM of 152); smaller grids keep one cell per thread.
constexpr long long kVecMinBlocks = 304;
__global__ void __launch_bounds__(256) k_cc_apply4(CcOp<float> A, const float *__restrict__ p, float *__restrict__ q,
                                                  double *__restrict__ part)
{
    const GridD &g = A.g;
    const int hx = g.nx >> 1, hf = (g.nx + 2) >> 1, nq = hx >> 2;
    const int tx = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int kk = blockIdx.z * blockDim.z + threadIdx.z;
    const int sy = g.nx, sz = g.nx * g.ny;
    float v = 0.f;
    if (tx < 2 * nq && j < g.ny) {
        const int h = tx / nq, t0 = 4 * (tx - h * nq);
#pragma unroll
        for (int hp = 0; hp < 2; hp++) {
            const int k = 2 * kk + hp;
            if (k >= g.nz) continue;
            const int rc = (k * g.ny + j) * g.nx;
            const int c = rc + (h ? hx : 0) + t0, o = rc + (h ? 0 : hx) + t0;
            float pc[4], dg[4], xo[4], xs[4], xn[4], xd[4], xu[4], fy0[4], fy1[4], fz0[4], fz1[4], y[4];
            load4(p + c, pc);
            load4(A.diag + c, dg);
            load4(p + o, xo);
            const float xb = h ? (t0 + 4 < hx ? p[o + 4] : 0.f) : (t0 > 0 ? p[o - 1] : 0.f);
            if (j > 0) load4(p + c - sy, xs);
            if (j < g.ny - 1) load4(p + c + sy, xn);
            if (k > 0) load4(p + c - sz, xd);
            if (k < g.nz - 1) load4(p + c + sz, xu);
            load4(A.by + c + k * g.nx, fy0);
            load4(A.by + c + k * g.nx + g.nx, fy1);
            load4(A.bz + c, fz0);
            load4(A.bz + c + sz, fz1);
            const int rf = rc + k * g.ny + j;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int t = t0 + e, i = 2 * t + h;
                const float bxl = A.bx[rf + (h ? hf + t : t)];
                const float bxh = A.bx[rf + (h ? t + 1 : hf + t)];
                const float xw = h ? xo[e] : (e ? xo[e - 1] : xb);
                const float xe = h ? (e < 3 ? xo[e + 1] : xb) : xo[e];
                float off = 0.f;
                if (i > 0) off += bxl * xw;
                if (i < g.nx - 1) off += bxh * xe;
                if (j > 0) off += fy0[e] * xs[e];
                if (j < g.ny - 1) off += fy1[e] * xn[e];
                if (k > 0) off += fz0[e] * xd[e];
                if (k < g.nz - 1) off += fz1[e] * xu[e];
                y[e] = dg[e] * pc[e] - off;
                v += pc[e] * y[e];
            }
            *reinterpret_cast<float4 *>(q + c) = make_float4(y[0], y[1], y[2], y[3]);
        }
    }
    const double vs = block_sum3_t<float>(v);
    if (thread_linear() == 0) part[block_linear()] = vs;
}
inline dim3 apply4_grid(const GridD &g)
{
    const int nq2 = 2 * ((g.nx >> 1) >> 2), nzh = (g.nz + 1) / 2;
    return dim3((nq2 + kApply4X - 1) / kApply4X, (g.ny + kApply4Y - 1) / kApply4Y, (nzh + kApply4Z - 1) / kApply4Z);
}

// ===========================================================================
// Nodal operator (alpha-weighted trilinear stiffness, unit coefficient):
//   (A x)_a = h sum_{cells c at a} alpha_c sum_{nodes b of c, active} K(a,b) x_b
// with K(a,b) = 1/3, 0, -1/12, -1/12 for corners differing in 0, 1, 2, 3
// coordinates.
// ===========================================================================

__constant__ double kQ1[4] = {1.0 / 3.0, 0.0, -1.0 / 12.0, -1.0 / 12.0};

template <class T>
struct NdOp {
    GridD g;               // cell dims
    T h;                   // g.h in the operator's precision
    const T *alpha;        // cells
    const uint8_t *act;    // nodes
    const uint8_t *reg;    // nodes whose 8 cells are full (level 0), else nullptr
};

// Row of the nodal operator at node (i,j,k), assembled in stencil form.  With
// a[r][q][p] the volume fraction of the cell (i-1+p, j-1+q, k-1+r) (0 outside
// the box), the element matrix gives: centre (1/3) sum a; axis neighbours 0;
// each face-diagonal neighbour -(sum of the two cells sharing that edge)/12;
// each body-diagonal neighbour -(the one cell between them)/12.  Inactive
// neighbours hold x = 0 in every vector the solvers pass here.
// Sums of the 12 face-diagonal (fd) and 8 body-diagonal (bd) neighbours of
// interior node n.
template <class T>
__device__ inline void nd_regular_sums(const GridD &g, const T *__restrict__ x, int n, T &fd, T &bd)
{
    const T *xc = x + n;
    const int sy = g.nx + 1, sz = (g.nx + 1) * (g.ny + 1);
    fd = xc[1 + sy] + xc[-1 + sy] + xc[1 - sy] + xc[-1 - sy] + xc[1 + sz] + xc[-1 + sz] + xc[1 - sz] +
         xc[-1 - sz] + xc[sy + sz] + xc[-sy + sz] + xc[sy - sz] + xc[-sy - sz];
    bd = xc[1 + sy + sz] + xc[-1 + sy + sz] + xc[1 - sy + sz] + xc[-1 - sy + sz] + xc[1 + sy - sz] +
         xc[-1 + sy - sz] + xc[1 - sy - sz] + xc[-1 - sy - sz];
}

template <class T>
__device__ inline void nd_row(const NdOp<T> &A, int i, int j, int k, const T *__restrict__ x, T &diag,
                              T &ax)
{
    const GridD &g = A.g;
    const int NXn = g.nx + 1, NYn = g.ny + 1;
    if (A.reg && A.reg[nidx(g, i, j, k)]) {
        // all 8 cells full (so the node is interior): the constant stencil
        // 8/3 at the centre, -1/6 on the 12 face diagonals, -1/12 on the 8
        // body diagonals (times h)
        T fd, bd;
        nd_regular_sums(g, x, nidx(g, i, j, k), fd, bd);
        const T hh = A.h;
        diag = hh * T(8.0 / 3.0);
        ax = diag * x[nidx(g, i, j, k)] - hh * T(1.0 / 12.0) * (T(2) * fd + bd);
        return;
    }
    T a[2][2][2];
    T sa = 0;
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int q = 0; q < 2; q++)
#pragma unroll
            for (int p = 0; p < 2; p++) {
                int ci = i - 1 + p, cj = j - 1 + q, ck = k - 1 + r;
                T v = inbox(g, ci, cj, ck) ? A.alpha[cidx(g, ci, cj, ck)] : T(0);
                a[r][q][p] = v;
                sa += v;
            }
    const int n0 = nidx(g, i, j, k);
    auto X = [&](int di, int dj, int dk) -> T {
        int ii = i + di, jj = j + dj, kk = k + dk;
        if ((unsigned)ii > (unsigned)g.nx || (unsigned)jj > (unsigned)g.ny || (unsigned)kk > (unsigned)g.nz)
            return T(0);
        return x[n0 + di + dj * NXn + dk * NXn * NYn];
    };
    T s = 0;
    // face diagonals in the xy, xz and yz planes
#pragma unroll
    for (int q = 0; q < 2; q++)
#pragma unroll
        for (int p = 0; p < 2; p++) {
            s += (a[0][q][p] + a[1][q][p]) * X(2 * p - 1, 2 * q - 1, 0);
            s += (a[q][0][p] + a[q][1][p]) * X(2 * p - 1, 0, 2 * q - 1);
            s += (a[q][p][0] + a[q][p][1]) * X(0, 2 * p - 1, 2 * q - 1);
        }
    // body diagonals
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int q = 0; q < 2; q++)
#pragma unroll
            for (int p = 0; p < 2; p++) s += a[r][q][p] * X(2 * p - 1, 2 * q - 1, 2 * r - 1);
    const T hh = A.h;
    diag = hh * sa * T(1.0 / 3.0);
    ax = diag * x[n0] - hh * T(1.0 / 12.0) * s;
}

// One Chebyshev step: r = b - A x_in; d = cd d + cr D^-1 r; x_out = x_in + d.
// Node by node: the first step from zero on every level, and all steps on the
// levels without regular-node flags (the others take the plane march).
template <class T>
__global__ void __launch_bounds__(256) k_nd_cheb(NdOp<T> A, const T *__restrict__ xin, T *__restrict__ xout,
                                                 T *__restrict__ dvec, const T *__restrict__ b, T cd, T cr,
                                                 int zero_start)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const GridD &g = A.g;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int n = nidx(g, i, j, k);
    // the node's own operands are loaded before any branch on them
    const uint8_t on = A.act[n];
    const T bn = b[n];
    T xn = T(0), dold = T(0);
    if (!zero_start) {
        xn = xin[n];
        dold = dvec[n];
    }
    if (!on) {
        xout[n] = T(0);
        dvec[n] = T(0);
        return;
    }
    T diag, ax;
    if (zero_start) {
        // x_in = 0, d = 0: only the diagonal is needed
        T dsum = 0;
        for (int oc = 0; oc < 8; oc++) {
            int ci = i - 1 + (oc & 1), cj = j - 1 + ((oc >> 1) & 1), ck = k - 1 + ((oc >> 2) & 1);
            if (!inbox(g, ci, cj, ck)) continue;
            T al = A.alpha[cidx(g, ci, cj, ck)];
            if (al > T(0)) dsum += al;
        }
        diag = A.h * dsum * T(1.0 / 3.0);
        T dn = cr * bn / diag;
        dvec[n] = dn;
        xout[n] = dn;
        return;
    }
    nd_row(A, i, j, k, xin, diag, ax);
    T r = bn - ax;
    T dn = (cd != T(0) ? cd * dold : T(0)) + cr * r / diag;
    dvec[n] = dn;
    xout[n] = xn + dn;
}

// ---- nodal passes in plane-sum form (levels with regular-node flags) ------------
// With E_x, E_y, E_z the sums of the two neighbours along one axis, the
// regular stencil's face-diagonal sum is (E_x E_y + E_x E_z + E_y E_z) x and
// its body-diagonal sum E_x E_y E_z x.  Per plane k let A_k = the four axis
// neighbours within the plane and B_k = its four in-plane diagonals; then
//   face diagonals of node k = B_k + A_{k-1} + A_{k+1},
//   body diagonals of node k = B_{k-1} + B_{k+1}.
// A block of NT_X x NT_Y threads owns as many node columns and marches NT_Z
// planes: each plane of x (with its one-node halo) is staged in shared memory
// while the next plane's loads are in flight (two buffers: the one written at
// plane kk was last read at plane kk - 2, before every thread passed plane
// kk - 1's barrier), A and B of three planes stay in registers, and the node
// operands are fetched one plane ahead.  The tile kernel takes the regular
// and the inactive nodes; the active nodes that are not regular (box faces,
// cut cells: a few per cent) are listed once and take nd_row in k_nd_irr, so
// no warp of the march diverges into the general row.  Modes:
//   ND_CHEB   one Chebyshev step, as k_nd_cheb (out = x_out, d updated);
//   ND_RESID  out = b - A x, as k_nd_resid;
//   ND_APPLY  out = A x (x on inactive nodes) with block partials of x.out;
//   ND_RES32  r = b - A x (b - x on inactive nodes) in T, stored to the FP32
//             vector out32, with block partials of |r|^2 (the refinement
//             solver's true residual; T = double).
// The sums are associated differently from the one-node kernels.
enum { ND_CHEB = 0, ND_RESID = 1, ND_APPLY = 2, ND_RES32 = 3 };
constexpr int NT_X = 32, NT_Y = 8, NT_Z = 16;
constexpr long long kTileNodes = 1 << 20;   // coarse levels with at least this many nodes march too
constexpr int NT_W = NT_X + 2, NT_H = NT_Y + 2, NT_N = NT_W * NT_H;
constexpr int NT_SLOTS = (NT_N + NT_X * NT_Y - 1) / (NT_X * NT_Y);

inline dim3 nd_tile_grid(const GridD &g)
{
    return dim3((g.nx + 1 + NT_X - 1) / NT_X, (g.ny + 1 + NT_Y - 1) / NT_Y, (g.nz + 1 + NT_Z - 1) / NT_Z);
}

template <class T, int kMode>
__global__ void __launch_bounds__(NT_X * NT_Y) k_nd_tile(NdOp<T> A, const T *__restrict__ xin, T *__restrict__ out,
                                                       T *__restrict__ dvec, const T *__restrict__ b, T cd, T cr,
                                                       double *__restrict__ part, float *__restrict__ out32,
                                                       const double *__restrict__ sig)
{
    const double sc = (kMode == ND_RES32 && sig) ? *sig : 1.0;
    __shared__ T sx[2][NT_H][NT_W];
    const GridD &g = A.g;
    const int NX = g.nx + 1, NY = g.ny + 1, NZ = g.nz + 1;
    const int sy = NX, sz = NX * NY;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * NT_X + tx;
    const int i0 = blockIdx.x * NT_X, j0 = blockIdx.y * NT_Y, k0 = blockIdx.z * NT_Z;
    const int i = i0 + tx, j = j0 + ty;
    const bool col = i < NX && j < NY;
    const int kend = min(k0 + NT_Z, NZ);   // nodes k0 .. kend-1; planes k0-1 .. kend
    // halo-tile slots of this thread: offset within a plane, -1 outside the box
    int soff[NT_SLOTS];
#pragma unroll
    for (int u = 0; u < NT_SLOTS; u++) {
        const int sl = tid + u * NT_X * NT_Y;
        const int rr = sl / NT_W, qq = sl - rr * NT_W;
        const int gi = i0 - 1 + qq, gj = j0 - 1 + rr;
        soff[u] = (sl < NT_N && gi >= 0 && gi < NX && gj >= 0 && gj < NY) ? gj * sy + gi : -1;
    }
    T pre[NT_SLOTS];
    auto fetch = [&](int kk) {
#pragma unroll
        for (int u = 0; u < NT_SLOTS; u++)
            pre[u] = (soff[u] >= 0 && kk >= 0 && kk < NZ) ? xin[kk * sz + soff[u]] : T(0);
    };
    const T dreg = A.h * T(8.0 / 3.0), h12 = A.h * T(1.0 / 12.0);
    const T crd = cr / dreg;   // regular nodes: cr / diag
    T Am = 0, Bm = 0, A0 = 0, B0 = 0, X0 = 0;
    uint8_t on_c = 0, rg_c = 0, on_n = 0, rg_n = 0;
    T b_c = 0, d_c = 0, b_n = 0, d_n = 0;
    T v = 0;          // ND_APPLY: this thread's part of x.out
    float vr = 0.0f;  // ND_RES32: its part of |r|^2, from the stored FP32 values
    fetch(k0 - 1);
    for (int kk = k0 - 1; kk <= kend; kk++) {
        T(*S)[NT_W] = sx[kk & 1];
#pragma unroll
        for (int u = 0; u < NT_SLOTS; u++) {
            const int sl = tid + u * NT_X * NT_Y;
            if (sl < NT_N) (&S[0][0])[sl] = pre[u];
        }
        if (kk < kend) fetch(kk + 1);
        // operands of node kk, finalised at the next plane
        if (col && kk >= k0 && kk < kend) {
            const int n = kk * sz + j * sy + i;
            on_n = A.act[n];
            rg_n = A.reg[n];
            if (kMode != ND_APPLY) b_n = b[n];
            if (kMode == ND_CHEB) d_n = dvec[n];
        }
        __syncthreads();
        const T xc = S[ty + 1][tx + 1];
        const T An = (S[ty + 1][tx] + S[ty + 1][tx + 2]) + (S[ty][tx + 1] + S[ty + 2][tx + 1]);
        const T Bn = (S[ty][tx] + S[ty][tx + 2]) + (S[ty + 2][tx] + S[ty + 2][tx + 2]);
        const int k = kk - 1;
        if (col && k >= k0 && k < kend) {
            const int n = k * sz + j * sy + i;
            if (!on_c) {
                if (kMode == ND_CHEB) { out[n] = T(0); dvec[n] = T(0); }
                if (kMode == ND_RESID) out[n] = T(0);
                if (kMode == ND_APPLY) { out[n] = X0; v += X0 * X0; }
                if (kMode == ND_RES32) {
                    const float r = f64_to_f32_pow2(b_c - X0, sc);
                    out32[n] = r;
                    vr += r * r;
                }
            } else if (rg_c) {
                const T ax = dreg * X0 - h12 * (T(2) * (B0 + Am + An) + (Bm + Bn));
                if (kMode == ND_CHEB) {
                    const T dn = (cd != T(0) ? cd * d_c : T(0)) + crd * (b_c - ax);
                    dvec[n] = dn;
                    out[n] = X0 + dn;
                }
                if (kMode == ND_RESID) out[n] = b_c - ax;
                if (kMode == ND_APPLY) { out[n] = ax; v += X0 * ax; }
                if (kMode == ND_RES32) {
                    const float r = f64_to_f32_pow2(b_c - ax, sc);
                    out32[n] = r;
                    vr += r * r;
                }
            }
        }
        Am = A0; Bm = B0; A0 = An; B0 = Bn; X0 = xc;
        on_c = on_n; rg_c = rg_n; b_c = b_n; d_c = d_n;
    }
    if constexpr (kMode == ND_APPLY || kMode == ND_RES32) {
        const double vs = kMode == ND_RES32 ? block_sum3_t<float>(vr) : block_sum3_t<T>(v);
        if (thread_linear() == 0) part[block_linear()] = vs;
    }
}

// The listed nodes (active, not regular) of a level-0 pass: nd_row per node,
// the same outputs as k_nd_tile's mode; ND_APPLY partials per block.
template <class T, int kMode>
__global__ void __launch_bounds__(256) k_nd_irr(NdOp<T> A, const int *__restrict__ list, int nlist,
                                                const T *__restrict__ xin, T *__restrict__ out, T *__restrict__ dvec,
                                                const T *__restrict__ b, T cd, T cr, double *__restrict__ part,
                                                float *__restrict__ out32, const double *__restrict__ sig)
{
    const double sc = (kMode == ND_RES32 && sig) ? *sig : 1.0;
    const GridD &g = A.g;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    T v = 0;
    if (t < nlist) {
        const int n = list[t];
        const int NX = g.nx + 1, NY = g.ny + 1;
        const int i = n % NX, j = (n / NX) % NY, k = n / (NX * NY);
        T diag, ax;
        nd_row(A, i, j, k, xin, diag, ax);
        if (kMode == ND_CHEB) {
            const T dn = (cd != T(0) ? cd * dvec[n] : T(0)) + cr * (b[n] - ax) / diag;
            dvec[n] = dn;
            out[n] = xin[n] + dn;
        }
        if (kMode == ND_RESID) out[n] = b[n] - ax;
        if (kMode == ND_APPLY) { out[n] = ax; v = xin[n] * ax; }
        if (kMode == ND_RES32) {
            const float r = f64_to_f32_pow2(b[n] - ax, sc);
            out32[n] = r;
            v = T(r) * T(r);
        }
    }
    if constexpr (kMode == ND_APPLY || kMode == ND_RES32) {
        const double vs = block_sum3_t<T>(v);
        if (threadIdx.x == 0) part[blockIdx.x] = vs;
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_nd_resid(NdOp<T> A, const T *__restrict__ x, const T *__restrict__ b,
                                                  T *__restrict__ r)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const GridD &g = A.g;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    const int n = nidx(g, i, j, k);
    if (!A.act[n]) { r[n] = T(0); return; }
    T diag, ax;
    nd_row(A, i, j, k, x, diag, ax);
    r[n] = b[n] - ax;
}

// Full weighting (transpose of trilinear prolongation).
template <class T>
__global__ void k_nd_restrict(GridD gf, const T *__restrict__ rf, GridD gc, const uint8_t *__restrict__ actc,
                              T *__restrict__ bc)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z * blockDim.z + threadIdx.z;
    if (I > gc.nx || J > gc.ny || K > gc.nz) return;
    const int N = nidx(gc, I, J, K);
    if (!actc[N]) { bc[N] = T(0); return; }
    T s = 0;
    for (int dk = -1; dk <= 1; dk++) {
        int k = 2 * K + dk;
        if (k < 0 || k > gf.nz) continue;
        T wk = dk ? T(0.5) : T(1);
        for (int dj = -1; dj <= 1; dj++) {
            int j = 2 * J + dj;
            if (j < 0 || j > gf.ny) continue;
            T wj = dj ? T(0.5) : T(1);
            for (int di = -1; di <= 1; di++) {
                int i = 2 * I + di;
                if (i < 0 || i > gf.nx) continue;
                T wi = di ? T(0.5) : T(1);
                s += wi * wj * wk * rf[nidx(gf, i, j, k)];
            }
        }
    }
    bc[N] = s;
}

// xout = xin + trilinear interpolation of the coarse correction (active nodes).
template <class T>
__global__ void k_nd_prolong(GridD gf, const uint8_t *__restrict__ actf, GridD gc, const T *__restrict__ xc,
                             const T *__restrict__ xin, T *__restrict__ xout)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i > gf.nx || j > gf.ny || k > gf.nz) return;
    const int n = nidx(gf, i, j, k);
    if (!actf[n]) { xout[n] = T(0); return; }
    int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
    int i1 = i0 + (i & 1), j1 = j0 + (j & 1), k1 = k0 + (k & 1);
    T wi = (i & 1) ? T(0.5) : T(1), wj = (j & 1) ? T(0.5) : T(1), wk = (k & 1) ? T(0.5) : T(1);
    T s = 0;
    s += xc[nidx(gc, i0, j0, k0)];
    if (i & 1) s += xc[nidx(gc, i1, j0, k0)];
    if (j & 1) s += xc[nidx(gc, i0, j1, k0)];
    if (k & 1) s += xc[nidx(gc, i0, j0, k1)];
    if ((i & 1) && (j & 1)) s += xc[nidx(gc, i1, j1, k0)];
    if ((i & 1) && (k & 1)) s += xc[nidx(gc, i1, j0, k1)];
    if ((j & 1) && (k & 1)) s += xc[nidx(gc, i0, j1, k1)];
    if ((i & 1) && (j & 1) && (k & 1)) s += xc[nidx(gc, i1, j1, k1)];
    xout[n] = xin[n] + wi * wj * wk * s;
}

__global__ void k_nd_alpha_coarsen(GridD gf, const double *__restrict__ af, GridD gc, double *__restrict__ ac)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z * blockDim.z + threadIdx.z;
    if (I >= gc.nx || J >= gc.ny || K >= gc.nz) return;
    double s = 0.0;
    for (int o = 0; o < 8; o++)
        s += af[cidx(gf, 2 * I + (o & 1), 2 * J + ((o >> 1) & 1), 2 * K + ((o >> 2) & 1))];
    ac[cidx(gc, I, J, K)] = 0.125 * s;
}

__global__ void k_nd_regular(GridD g, const double *__restrict__ alpha, uint8_t *__restrict__ reg)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    bool all = true;
    for (int oc = 0; oc < 8; oc++) {
        int ci = i - 1 + (oc & 1), cj = j - 1 + ((oc >> 1) & 1), ck = k - 1 + ((oc >> 2) & 1);
        if (!inbox(g, ci, cj, ck) || alpha[cidx(g, ci, cj, ck)] != 1.0) all = false;
    }
    reg[nidx(g, i, j, k)] = all ? 1 : 0;
}

__global__ void k_nd_active(GridD g, const double *__restrict__ alpha, uint8_t *__restrict__ act)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    int id[3] = {i, j, k};
    bool dir = pin_node(g, i, j, k);
    for (int d = 0; d < 3; d++) {
        if (id[d] == 0 && g.bc[2 * d] == EBV_OUTFLOW) dir = true;
        if (id[d] == dimn(g, d) && g.bc[2 * d + 1] == EBV_OUTFLOW) dir = true;
    }
    bool any = false;
    for (int oc = 0; oc < 8; oc++) {
        int ci = i - 1 + (oc & 1), cj = j - 1 + ((oc >> 1) & 1), ck = k - 1 + ((oc >> 2) & 1);
        if (inbox(g, ci, cj, ck) && alpha[cidx(g, ci, cj, ck)] > 0.0) any = true;
    }
    act[nidx(g, i, j, k)] = (!dir && any) ? 1 : 0;
}

// ===========================================================================
// Dense bottom solve
// ===========================================================================

template <class T>
__global__ void k_cc_bottom_assemble(VOp<T> A, double *__restrict__ M, int nb)
{
    const GridD &g = A.g;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nb; r += gridDim.x * blockDim.x) {
        double *row = M + (size_t)r * 2 * nb;
        for (int s = 0; s < 2 * nb; s++) row[s] = 0.0;
        row[nb + r] = 1.0;
        int i = r % g.nx, j = (r / g.nx) % g.ny, k = r / (g.nx * g.ny);
        double bxl = (double)T(A.bx[fidxT<T>(g, 0, i, j, k)]), bxh = (double)T(A.bx[fidxT<T>(g, 0, i + 1, j, k)]);
        double byl = (double)T(A.by[fidxT<T>(g, 1, i, j, k)]), byh = (double)T(A.by[fidxT<T>(g, 1, i, j + 1, k)]);
        double bzl = (double)T(A.bz[fidxT<T>(g, 2, i, j, k)]), bzh = (double)T(A.bz[fidxT<T>(g, 2, i, j, k + 1)]);
        double diag = (double)A.diag[cix<T>(g, i, j, k)];
        row[r] = diag > 0.0 ? diag : 1.0;
        if (i > 0) row[r - 1] = -bxl;
        if (i < g.nx - 1) row[r + 1] = -bxh;
        if (j > 0) row[r - g.nx] = -byl;
        if (j < g.ny - 1) row[r + g.nx] = -byh;
        if (k > 0) row[r - g.nx * g.ny] = -bzl;
        if (k < g.nz - 1) row[r + g.nx * g.ny] = -bzh;
    }
}

__global__ void k_nd_bottom_assemble(GridD g, const double *__restrict__ alpha, const uint8_t *__restrict__ act,
                                     double *__restrict__ M, int nb)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nb; r += gridDim.x * blockDim.x) {
        double *row = M + (size_t)r * 2 * nb;
        for (int s = 0; s < 2 * nb; s++) row[s] = 0.0;
        row[nb + r] = 1.0;
        int i = r % (g.nx + 1), j = (r / (g.nx + 1)) % (g.ny + 1), k = r / ((g.nx + 1) * (g.ny + 1));
        if (!act[r]) { row[r] = 1.0; continue; }
        for (int oc = 0; oc < 8; oc++) {
            int ci = i - 1 + (oc & 1), cj = j - 1 + ((oc >> 1) & 1), ck = k - 1 + ((oc >> 2) & 1);
            if (!inbox(g, ci, cj, ck)) continue;
            double al = alpha[cidx(g, ci, cj, ck)];
            if (!(al > 0.0)) continue;
            int oa = (i - ci) | ((j - cj) << 1) | ((k - ck) << 2);
            for (int ob = 0; ob < 8; ob++) {
                int n = nidx(g, ci + (ob & 1), cj + ((ob >> 1) & 1), ck + ((ob >> 2) & 1));
                if (!act[n]) continue;
                row[n] += g.h * al * kQ1[__popc(oa ^ ob)];
            }
        }
    }
}

// Gauss-Jordan elimination of [M | I] in one CTA (SPD: no pivoting needed);
// the right half becomes the inverse, copied to inv.  CTA q of the grid
// inverts matrix q of the nb x 2nb matrices stored one after another in M into
// inv_q (up to three at once: the variants of one operator).
__global__ void __launch_bounds__(1024) k_gauss_jordan(double *__restrict__ Mall, int nb, double *inv0,
                                                       double *inv1, double *inv2)
{
    __shared__ double fac[kBottomMax];
    const int w = 2 * nb;
    double *__restrict__ M = Mall + (size_t)blockIdx.x * nb * w;
    double *__restrict__ inv = blockIdx.x == 0 ? inv0 : (blockIdx.x == 1 ? inv1 : inv2);
    for (int col = 0; col < nb; col++) {
        double piv = M[(size_t)col * w + col];
        __syncthreads();
        for (int s = threadIdx.x; s < w; s += blockDim.x) M[(size_t)col * w + s] /= piv;
        __syncthreads();
        for (int r = threadIdx.x; r < nb; r += blockDim.x) fac[r] = (r == col) ? 0.0 : M[(size_t)r * w + col];
        __syncthreads();
        for (int e = threadIdx.x; e < nb * w; e += blockDim.x) {
            int r = e / w, s = e - r * w;
            if (r != col) M[e] -= fac[r] * M[(size_t)col * w + s];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int r = e / nb, s = e - r * nb;
        inv[e] = M[(size_t)r * w + nb + s];
    }
}

// x = scale inv b; the dense system is numbered in the natural order, the
// vectors of a row-split (FP32 cell-centred) level are mapped through g.
__device__ inline int bottom_pos(const GridD &g, int split, int r)
{
    if (!split) return r;
    return cix<float>(g, r % g.nx, (r / g.nx) % g.ny, r / (g.nx * g.ny));
}
template <class T>
__device__ inline void bottom_row(const double *__restrict__ inv, int nb, const T *__restrict__ b,
                                  T *__restrict__ x, double scale, const GridD &g, int split, int r)
{
    double s = 0.0;
    for (int q = 0; q < nb; q++) s += inv[(size_t)r * nb + q] * (double)b[bottom_pos(g, split, q)];
    x[bottom_pos(g, split, r)] = (T)(s * scale);
}
template <class T>
__global__ void __launch_bounds__(256) k_bottom_solve(const double *__restrict__ inv, int nb,
                                                      const T *__restrict__ b, T *__restrict__ x,
                                                      double scale, GridD g, int split)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nb; r += gridDim.x * blockDim.x)
        bottom_row(inv, nb, b, x, scale, g, split, r);
}

// ---- the coarse end of the cell-centred V-cycle in one CTA ------------------------
// Levels of at most kCoarseCells cells cannot fill the GPU, and as separate
// launches they cost more in launch latency than in work.  Below such a
// level one persistent block of 1024 threads runs the rest of the V-cycle --
// pre-smoothing, residual and restriction down to the bottom, the bottom
// solve, then correction and post-smoothing back up -- with the same steps
// and per-cell arithmetic as the per-level kernels (gs_cell, rr_cell,
// bottom_row) and a block barrier wherever those have a kernel boundary, so
// its results are bit for bit those of the per-level path.
constexpr int kCoarseCells = 4096;
constexpr int kCoarseMax = 8;
template <class T>
struct CoarseVC {
    int n;                    // levels handled; the last is the bottom
    VOp<T> A[kCoarseMax];
    T *x[kCoarseMax];
    T *b[kCoarseMax];         // b[0] given, the others written by restriction
    const double *binv;       // bottom inverse (natural numbering)
    int nb;
};

// One colour pass of the coarse kernel on level l: thread tid takes the
// (x-pair, row) slots tid, tid + 1024, ... and in each the cell of colour
// `color`; as in k_cc_gs, every operand of its (at most kCoarseSlots) updates
// is loaded before any result is stored, so the L2 round trips overlap.
// With zero_start the other cell of each slot is set to 0.
constexpr int kCoarseThreads = 1024;
constexpr int kCoarseSlots = (kCoarseCells + kCoarseThreads - 1) / kCoarseThreads;  // x-pairs: <= cells
template <class T, bool kCorr>
__device__ inline void coarse_pass(const CoarseVC<T> &D, int l, int color, int zero_start)
{
    const VOp<T> &A = D.A[l];
    const GridD &g = A.g;
    const int hx = (g.nx + 1) >> 1, slots = hx * g.ny * g.nz;
    T *x = D.x[l];
    T val[kCoarseSlots];
    int cc[kCoarseSlots], co[kCoarseSlots];
#pragma unroll
    for (int u = 0; u < kCoarseSlots; u++) {
        const int m = threadIdx.x + u * kCoarseThreads;
        cc[u] = -1;
        co[u] = -1;
        val[u] = T(0);
        if (m >= slots) continue;
        const int t = m % hx, jk = m / hx, j = jk % g.ny, k = jk / g.ny;
        const int par = (j + k + color) & 1;
        const int i = 2 * t + par, io = 2 * t + 1 - par;
        if (io < g.nx) co[u] = cix<T>(g, io, j, k);
        if (i >= g.nx) continue;
        cc[u] = cix<T>(g, i, j, k);
        val[u] = kCorr ? gs_cell<T, true>(A, x, D.b[l], i, j, k, 0, D.x[l + 1], D.A[l + 1].g)
                       : gs_cell<T, false>(A, x, D.b[l], i, j, k, zero_start, x, g);
    }
#pragma unroll
    for (int u = 0; u < kCoarseSlots; u++) {
        if (zero_start && co[u] >= 0) x[co[u]] = T(0);
        if (cc[u] >= 0) x[cc[u]] = val[u];
    }
    __syncthreads();
}

// The V-cycle from level 0 of D down to its bottom and back; bs holds the
// bottom right-hand side in natural order.
template <class T>
__device__ inline void coarse_vcycle_body(const CoarseVC<T> &D, double *bs)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int L = D.n - 1;
    for (int l = 0; l < L; l++) {
        // two red-black sweeps, red first, the first from zero
        coarse_pass<T, false>(D, l, 0, 1);
        coarse_pass<T, false>(D, l, 1, 0);
        coarse_pass<T, false>(D, l, 0, 0);
        coarse_pass<T, false>(D, l, 1, 0);
        const GridD &gc = D.A[l + 1].g;
        const int nc = ncell(gc);
        for (int s = tid; s < nc; s += nt) {
            const int I = s % gc.nx, J = (s / gc.nx) % gc.ny, K = s / (gc.nx * gc.ny);
            D.b[l + 1][cix<T>(gc, I, J, K)] = rr_cell<T>(D.A[l], D.x[l], D.b[l], I, J, K);
        }
        __syncthreads();
    }
    // bottom: x = inv b, b gathered once into natural order (same sums as bottom_row)
    {
        const GridD &gb = D.A[L].g;
        const int split = (int)(sizeof(T) == 4);
        for (int q = tid; q < D.nb; q += nt) bs[q] = (double)D.b[L][bottom_pos(gb, split, q)];
        __syncthreads();
        for (int r = tid; r < D.nb; r += nt) {
            const double *row = D.binv + (size_t)r * D.nb;
            double sum = 0.0;
#pragma unroll 8
            for (int q = 0; q < D.nb; q++) sum += row[q] * bs[q];
            D.x[L][bottom_pos(gb, split, r)] = (T)(sum * 1.0);
        }
        __syncthreads();
    }
    for (int l = L - 1; l >= 0; l--) {
        // two sweeps, black first; the first pass takes the coarse correction
        coarse_pass<T, true>(D, l, 1, 0);
        coarse_pass<T, false>(D, l, 0, 0);
        coarse_pass<T, false>(D, l, 1, 0);
        coarse_pass<T, false>(D, l, 0, 0);
    }
}

// Asynchronous global -> shared copies of n elements (cp.async, 4 or 8 bytes
// per copy, all in flight together).  2-byte elements go as 4-byte pairs:
// both addresses 4-byte aligned, and for odd n the source holds one element
// more (the face arrays of the V-cycle are allocated with one spare).
template <class E>
__device__ inline void stage_async(E *dst, const E *src, int n)
{
    static_assert(sizeof(E) == 2 || sizeof(E) == 4 || sizeof(E) == 8, "2-, 4- or 8-byte elements");
    if constexpr (sizeof(E) == 2) {
        stage_async((uint32_t *)dst, (const uint32_t *)src, (n + 1) >> 1);
    } else {
        for (int s = threadIdx.x; s < n; s += blockDim.x) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + s);
            if constexpr (sizeof(E) == 4)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src + s) : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src + s) : "memory");
        }
    }
}

// Shared-memory layout of the staged coarse V-cycle: the bottom inverse (if
// staged) first, then per level the diagonal and the three face arrays
// (levels that smooth), x and b; every array starts on a 16-byte boundary.
__host__ __device__ inline size_t stage_align(size_t b) { return (b + 15) & ~(size_t)15; }
template <class T>
__host__ __device__ inline size_t coarse_stage_bytes(const CoarseVC<T> &D, int with_binv)
{
    using F = typename VFace<T>::type;
    size_t b = with_binv ? stage_align((size_t)D.nb * D.nb * sizeof(double)) : 0;
    for (int q = 0; q < D.n; q++) {
        const GridD &g = D.A[q].g;
        if (q + 1 < D.n) {
            b += (sizeof(T) == 4 ? 2 : 1) * stage_align((size_t)ncell(g) * sizeof(T));   // diag (and 1/diag)
            for (int d = 0; d < 3; d++) b += stage_align((size_t)nface(g, d) * sizeof(F));
        }
        b += 2 * stage_align((size_t)ncell(g) * sizeof(T));
    }
    return b;
}
constexpr size_t kCoarseStageMax = 200 * 1024;  // dynamic shared memory of the staged form

// kStage: every array the V-cycle touches is first copied into shared memory
// (the level vectors need no copy: they are written before being read, and
// b of the top level is the one input), the V-cycle runs there, and x of the
// top level -- the correction the next finer level reads -- is copied back.
// Same arithmetic in the same order as the unstaged form.
template <class T, bool kStage>
__global__ void __launch_bounds__(kCoarseThreads) k_cc_coarse_vcycle(CoarseVC<T> D, int stage_binv)
{
    __shared__ double bs[kBottomMax];
    if constexpr (!kStage) {
        coarse_vcycle_body<T>(D, bs);
    } else {
        extern __shared__ __align__(16) unsigned char dyn[];
        // the staged level table lives in shared memory too (thread 0 writes it)
        __shared__ __align__(16) unsigned char tbl[sizeof(CoarseVC<T>)];
        CoarseVC<T> &S = *reinterpret_cast<CoarseVC<T> *>(tbl);
        const bool t0 = threadIdx.x == 0;
        if (t0) S = D;
        using F = typename VFace<T>::type;
        unsigned char *ptr = dyn;
        if (stage_binv) {
            double *bi = (double *)ptr;
            stage_async(bi, D.binv, D.nb * D.nb);
            if (t0) S.binv = bi;
            ptr += stage_align((size_t)D.nb * D.nb * sizeof(double));
        }
        for (int q = 0; q < D.n; q++) {
            const GridD &g = D.A[q].g;
            const int nc = ncell(g);
            if (q + 1 < D.n) {
                T *dg = (T *)ptr;
                ptr += stage_align((size_t)nc * sizeof(T));
                stage_async(dg, D.A[q].diag, nc);
                if constexpr (sizeof(T) == 4) {
                    T *di = (T *)ptr;
                    ptr += stage_align((size_t)nc * sizeof(T));
                    stage_async(di, D.A[q].dinv, nc);
                    if (t0) S.A[q].dinv = di;
                }
                F *fc[3];
                const F *src[3] = {D.A[q].bx, D.A[q].by, D.A[q].bz};
                for (int d = 0; d < 3; d++) {
                    fc[d] = (F *)ptr;
                    ptr += stage_align((size_t)nface(g, d) * sizeof(F));
                    stage_async(fc[d], src[d], nface(g, d));
                }
                if (t0) { S.A[q].diag = dg; S.A[q].bx = fc[0]; S.A[q].by = fc[1]; S.A[q].bz = fc[2]; }
            }
            T *xs = (T *)ptr;
            ptr += stage_align((size_t)nc * sizeof(T));
            T *bs2 = (T *)ptr;
            ptr += stage_align((size_t)nc * sizeof(T));
            if (q == 0) stage_async(bs2, (const T *)D.b[0], nc);
            if (t0) { S.x[q] = xs; S.b[q] = bs2; }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
        coarse_vcycle_body<T>(S, bs);
        const int n0 = ncell(D.A[0].g);
        const T *x0s = S.x[0];
        for (int s = threadIdx.x; s < n0; s += blockDim.x) D.x[0][s] = x0s[s];
    }
}

// ===========================================================================
// Krylov glue
// ===========================================================================
enum { S_BB = 0, S_RR = 1, S_RZ = 2, S_RZOLD = 3, S_PQ = 4, S_REL = 16, S_PREV = 17, S_T2 = 18, S_SIG = 19 };

// Scale of the refinement solver's FP32 residuals: a power of two near 1/|b|
// (1 when |b| is 0 or not finite), so that corrections of right-hand sides far
// below 1 (down to round-off) do not underflow in FP32.  Multiplying by a
// power of two is exact, so in the usual range every FP32 operation gives
// the same bits as without it.  The FP64 norms are scaled alike.
__global__ void k_set_sigma(double *scal, int x_zero)
{
    if (threadIdx.x) return;
    const double bb = scal[S_BB];
    double sig = 1.0;
    if (bb > 0.0 && isfinite(bb)) sig = ldexp(1.0, -ilogb(sqrt(bb)));
    scal[S_SIG] = sig;
    scal[S_BB] = bb * sig * sig;
    if (x_zero) scal[S_RR] = scal[S_BB];
}

// Writes a loop condition: the control word (polled by the host in eager
// mode) and, inside a captured graph, the conditional node's handle.
__device__ inline void set_cond(int *ctl, int slot, int v, cudaGraphConditionalHandle h, int use_h)
{
    ctl[slot] = v;
    if (use_h) cudaGraphSetConditional(h, v ? 1u : 0u);
}

__global__ void k_set_cond(int *ctl, int slot, int v, cudaGraphConditionalHandle h, int use_h)
{
    if (threadIdx.x == 0) set_cond(ctl, slot, v, h, use_h);
}

__global__ void k_solve_begin(int *ctl)
{
    if (threadIdx.x == 0) {
        ctl[C_IT] = 0; ctl[C_K] = 0; ctl[C_NOUT] = 0; ctl[C_STALL] = 0; ctl[C_ERR] = 0; ctl[C_ZERO] = 0;
    }
}

// After a true residual (S_RR = |b - A x|^2, S_BB = |b|^2): record the
// relative residual and decide whether another CG pass (FP64 path: a
// restart; refinement path: one correction solve) runs.  Passes are capped
// at max_pass, iterations at maxit; a non-finite norm stops with E_NAN; b = 0
// flags x for zeroing.  For refinement, the inner target and stall state of
// the coming correction solve are set here.
__global__ void k_outer_check(double *scal, int *ctl, double tol, int maxit, int max_pass, int refine,
                              double inner_drop, cudaGraphConditionalHandle h, int use_h)
{
    if (threadIdx.x) return;
    const double bb = scal[S_BB], rr = scal[S_RR];
    int go = 0;
    if (ctl[C_ERR] == 0) {
        if (!isfinite(rr) || !isfinite(bb)) {
            ctl[C_ERR] = E_NAN;
        } else if (bb == 0.0) {
            ctl[C_ZERO] = 1;
            scal[S_REL] = 0.0;
        } else {
            const double rel = sqrt(rr / bb);
            scal[S_REL] = rel;
            go = rel > tol && ctl[C_IT] < maxit && ctl[C_NOUT] < max_pass;
            if (go && refine) {
                const double f = fmax(inner_drop, 0.5 * tol / rel);
                scal[S_T2] = rr * f * f;
                scal[S_PREV] = rr;
                ctl[C_STALL] = 0;
            }
        }
    }
    ctl[C_NOUT]++;
    ctl[C_K] = 0;
    set_cond(ctl, C_COND_OUT, go, h, use_h);
}

// After one CG iteration (S_RR = recursive residual norm^2).  FP64 path:
// continue while |r|/|b| > tol/2.  Refinement path: continue until the
// correction's residual is below its target, or it has stalled (three
// iterations in a row that do not cut |r|^2 by 4: the FP32 round-off floor).
__device__ inline void inner_check(double *scal, int *ctl, double tol, int maxit, int refine,
                                   cudaGraphConditionalHandle h, int use_h)
{
    scal[S_RZOLD] = scal[S_RZ];
    ctl[C_IT]++;
    ctl[C_K]++;
    const double rr = scal[S_RR];
    int go = 1;
    if (!isfinite(rr)) {
        if (ctl[C_ERR] == 0) ctl[C_ERR] = E_NAN;   // (the first error word stands)
        go = 0;
    } else if (!refine) {
        go = sqrt(rr / scal[S_BB]) > 0.5 * tol;
    } else if (rr <= scal[S_T2]) {
        go = 0;
    } else {
        if (rr > 0.25 * scal[S_PREV]) {
            if (++ctl[C_STALL] >= 3) go = 0;
        } else {
            ctl[C_STALL] = 0;
        }
        scal[S_PREV] = rr;
    }
    if (ctl[C_IT] >= maxit || ctl[C_ERR]) go = 0;   // (an error word set by a kernel ends the solve)
    set_cond(ctl, C_COND_IN, go, h, use_h);
}

// S_RR = the sum of the update's n block partials, then the same decision
// (one launch instead of a reduction and a check).
__global__ void __launch_bounds__(1024) k_reduce_inner_check(const double *part, int n, double *scal, int *ctl,
                                                             double tol, int maxit, int refine,
                                                             cudaGraphConditionalHandle h, int use_h)
{
    double v = 0.0;
    for (int s = threadIdx.x; s < n; s += 1024) v += part[s];
    v = block_sum<1024>(v);
    if (threadIdx.x == 0) {
        scal[S_RR] = v;
        inner_check(scal, ctl, tol, maxit, refine, h, use_h);
    }
}

// End of a solve: per-slot statistics, and the step's first failure
// (100 x error + slot) kept in C_STEPERR.
__global__ void k_solve_end(const double *scal, int *ctl, double tol, double *sstat, int slot)
{
    if (threadIdx.x) return;
    const double rel = scal[S_REL];
    sstat[3 * slot] = ctl[C_IT];
    sstat[3 * slot + 1] = rel;
    sstat[3 * slot + 2] = ctl[C_NOUT];
    int e = ctl[C_ERR];
    if (e == 0 && !(rel <= tol)) e = E_NOTCONV;
    if (e) ctl[C_ERR] = e;
    if (e && ctl[C_STEPERR] == 0) ctl[C_STEPERR] = 100 * e + slot;
    sstat[kSstatAcc + 2 * slot] += ctl[C_IT];
    sstat[kSstatAcc + 2 * slot + 1] += ctl[C_NOUT] - 1;
}

__global__ void k_zero_if(double *x, int n, const int *ctl)
{
    if (!ctl[C_ZERO]) return;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) x[s] = 0.0;
}

__global__ void __launch_bounds__(256) k_resid_init(const double *__restrict__ b, const double *__restrict__ q,
                                                    double *__restrict__ r, int n, double *__restrict__ part)
{
    double v = 0.0, w = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        double rs = b[s] - q[s];
        r[s] = rs;
        v += rs * rs;
        w += b[s] * b[s];
    }
    v = block_sum<256>(v);
    w = block_sum<256>(w);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = v;
        part[gridDim.x + blockIdx.x] = w;
    }
}

__global__ void __launch_bounds__(256) k_cg_update(double *__restrict__ x, double *__restrict__ r,
                                                   const double *__restrict__ p, const double *__restrict__ q,
                                                   const double *__restrict__ scal, int n, double *__restrict__ part)
{
    const double a = scal[S_RZ] / scal[S_PQ];
    double v = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        x[s] += a * p[s];
        double rs = r[s] - a * q[s];
        r[s] = rs;
        v += rs * rs;
    }
    v = block_sum<256>(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
}

__global__ void k_cg_pupdate(double *__restrict__ p, const double *__restrict__ z, const double *__restrict__ scal,
                             int n, const int *__restrict__ ctl)
{
    const int first = ctl[C_K] == 0;
    const double beta = first ? 0.0 : scal[S_RZ] / scal[S_RZOLD];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        p[s] = first ? z[s] : z[s] + beta * p[s];
}

// --- refinement: FP64 residual into an FP32 vector, FP32 inner CG, FP64 update.
// Per-thread sums of the FP32 kernels stay FP32 (a few dozen terms), block and
// final sums are FP64.

__global__ void __launch_bounds__(256) k_dot32(const float *__restrict__ a, const float *__restrict__ b, int n,
                                               double *__restrict__ part)
{
    float v = 0.0f;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) v += a[s] * b[s];
    double dv = block_sum<256>((double)v);
    if (threadIdx.x == 0) part[blockIdx.x] = dv;
}

// r -= a q with a = rz/pq, partials of r.r.  (The solution update e += a p
// of the same iteration is deferred to the next k_cg_pupdate32, which reads
// p anyway, and after the last iteration to k_add32to64*.)
__global__ void __launch_bounds__(256) k_cg_update32(float *__restrict__ r, const float *__restrict__ q,
                                                     const double *__restrict__ scal, int n,
                                                     double *__restrict__ part)
{
    const float a = (float)(scal[S_RZ] / scal[S_PQ]);
    float v = 0.0f;
    // 16-byte vectors (the arrays come from cudaMalloc), then the n % 4 tail:
    // four independent loads per thread keep enough bytes in flight
    const int n4 = n >> 2, t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    float4 *r4 = reinterpret_cast<float4 *>(r);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    for (int s = t0; s < n4; s += st) {
        float4 rs = r4[s];
        const float4 qs = q4[s];
        rs.x = rs.x - a * qs.x;
        rs.y = rs.y - a * qs.y;
        rs.z = rs.z - a * qs.z;
        rs.w = rs.w - a * qs.w;
        r4[s] = rs;
        v += rs.x * rs.x;
        v += rs.y * rs.y;
        v += rs.z * rs.z;
        v += rs.w * rs.w;
    }
    for (int s = 4 * n4 + t0; s < n; s += st) {
        const float rs = r[s] - a * q[s];
        r[s] = rs;
        v += rs * rs;
    }
    double dv = block_sum<256>((double)v);
    if (threadIdx.x == 0) part[blockIdx.x] = dv;
}

// Iteration k of the FP32 CG: p = z (k = 0) or z + beta p, beta = rz/rz_old;
// for k >= 1 first the previous iteration's solution update with the old p,
// e = a p (k = 1) or e + a p, a = rz_old/pq (that iteration's step).
__global__ void k_cg_pupdate32(float *__restrict__ p, float *__restrict__ e, const float *__restrict__ z,
                               const double *__restrict__ scal, int n, const int *__restrict__ ctl)
{
    const int k = ctl[C_K];
    const float beta = k == 0 ? 0.0f : (float)(scal[S_RZ] / scal[S_RZOLD]);
    const float a = k == 0 ? 0.0f : (float)(scal[S_RZOLD] / scal[S_PQ]);
    // one element (each lane of a vector, and the tail)
    auto upd = [&](float &pv, float &ev, float zv) {
        if (k == 0) {
            pv = zv;
        } else {
            const float po = pv;
            ev = k == 1 ? a * po : ev + a * po;
            pv = zv + beta * po;
        }
    };
    // 16-byte vectors (cudaMalloc'd arrays), then the n % 4 tail
    const int n4 = n >> 2, t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
    float4 *p4 = reinterpret_cast<float4 *>(p), *e4 = reinterpret_cast<float4 *>(e);
    const float4 *z4 = reinterpret_cast<const float4 *>(z);
    for (int s = t0; s < n4; s += st) {
        const float4 zv = z4[s];
        float4 pv = k == 0 ? zv : p4[s];
        float4 ev = k >= 2 ? e4[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        upd(pv.x, ev.x, zv.x);
        upd(pv.y, ev.y, zv.y);
        upd(pv.z, ev.z, zv.z);
        upd(pv.w, ev.w, zv.w);
        p4[s] = pv;
        if (k >= 1) e4[s] = ev;
    }
    for (int s = 4 * n4 + t0; s < n; s += st) {
        float pv = k == 0 ? z[s] : p[s], ev = k >= 2 ? e[s] : 0.f;
        upd(pv, ev, z[s]);
        p[s] = pv;
        if (k >= 1) e[s] = ev;
    }
}

// After the last of the correction solve's k = ctl[C_K] iterations: its
// deferred solution update (a = rz_old/pq of that iteration) as in
// k_cg_pupdate32, then the FP64 solution x += e.
__device__ inline float final_e(const float *__restrict__ e, const float *__restrict__ p, float a, int k, int s)
{
    return k == 1 ? a * p[s] : e[s] + a * p[s];
}

__global__ void k_add32to64(double *__restrict__ x, const float *__restrict__ e, const float *__restrict__ p,
                            const double *__restrict__ scal, const int *__restrict__ ctl, int n)
{
    const int k = ctl[C_K];
    const float a = (float)(scal[S_RZOLD] / scal[S_PQ]);
    const double isig = 1.0 / scal[S_SIG];   // exact: a power of two
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        x[s] += (double)final_e(e, p, a, k, s) * isig;
}

// k_add32to64 with e and p FP32 row-split vectors
__global__ void k_add32to64_split(GridD g, double *__restrict__ x, const float *__restrict__ e,
                                  const float *__restrict__ p, const double *__restrict__ scal,
                                  const int *__restrict__ ctl)
{
    const int n = ncell(g);
    const int k = ctl[C_K];
    const float a = (float)(scal[S_RZOLD] / scal[S_PQ]);
    const double isig = 1.0 / scal[S_SIG];   // exact: a power of two
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        x[s] += (double)final_e(e, p, a, k, cix<float>(g, s % g.nx, (s / g.nx) % g.ny, s / (g.nx * g.ny))) * isig;
}

__global__ void k_fill(double *a, int n, double v)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) a[s] = v;
}

__global__ void k_zero_inactive(int n, const uint8_t *__restrict__ act, double *__restrict__ x)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        if (!act[s]) x[s] = 0.0;
}

inline dim3 cgrid(const GridD &g) { return grid3(g.nx, g.ny, g.nz); }
inline dim3 ngrid(const GridD &g) { return grid3(g.nx + 1, g.ny + 1, g.nz + 1); }
inline int nblocks3(dim3 b) { return b.x * b.y * b.z; }

// The Krylov operator of level L (FP32: level 0 only, FP32 faces, diag_a).
template <class T>
CcOp<T> ccop(const CcLevel &L)
{
    CcOp<T> A;
    A.g = L.g;
    if constexpr (sizeof(T) == 8) {
        A.diag = (const T *)L.diag_d; A.bx = (const T *)L.bf_d[0]; A.by = (const T *)L.bf_d[1]; A.bz = (const T *)L.bf_d[2];
    } else {
        A.diag = (const T *)L.diag_a; A.bx = (const T *)L.bf_f[0]; A.by = (const T *)L.bf_f[1]; A.bz = (const T *)L.bf_f[2];
    }
    return A;
}

// The V-cycle operator of level L (FP32: BF16 faces, diag_f).
template <class T>
VOp<T> vop(const CcLevel &L)
{
    VOp<T> A;
    A.g = L.g;
    if constexpr (sizeof(T) == 8) {
        A.diag = (const T *)L.diag_d; A.bx = (const T *)L.bf_d[0]; A.by = (const T *)L.bf_d[1]; A.bz = (const T *)L.bf_d[2];
    } else {
        A.diag = (const T *)L.diag_f;
        if constexpr (kVcycleBf16) {
            A.bx = L.bf_h[0]; A.by = L.bf_h[1]; A.bz = L.bf_h[2];
        } else {
            A.bx = (const typename VFace<T>::type *)L.bf_f[0];
            A.by = (const typename VFace<T>::type *)L.bf_f[1];
            A.bz = (const typename VFace<T>::type *)L.bf_f[2];
        }
        A.dinv = (const T *)L.dinv_f;
    }
    return A;
}

// diagonals of every variant of level l from its extra and faces, in precision
// T (FP32: the V-cycle's, from the faces rounded as it stores them).
template <class T>
void cc_make_diag(Ctx *c, CcHier &H, int l)
{
    const CcLevel &L = H.lv[l];
    unsigned masks = 0;
    for (int q = 0; q < H.nvar; q++) masks |= (H.side_mask[q] & 0x3fu) << (6 * q);
    if constexpr (sizeof(T) == 8)
        EBV_LAUNCH(c, k_cc_make_diag<double>, cgrid(L.g), block3(), 0, L.g, L.extra_d, L.bf_d[0], L.bf_d[1],
                   L.bf_d[2], H.nvar, masks, H.vdiag_d[0][l], H.vdiag_d[1][l], H.vdiag_d[2][l]);
    else
        EBV_LAUNCH(c, (k_cc_make_diag<float, kVcycleBf16>), cgrid(L.g), block3(), 0, L.g, L.extra_f, L.bf_f[0], L.bf_f[1],
                   L.bf_f[2], H.nvar, masks, H.vdiag_f[0][l], H.vdiag_f[1][l], H.vdiag_f[2][l], H.vdinv_f[0][l],
                   H.vdinv_f[1][l], H.vdinv_f[2][l]);
}

// The V-cycle's BF16 copy of the FP32 faces of level L, and the padded copy
// of its x faces that the fused sweep loads (in the V-cycle's face type).
inline void cc_faces_bf16(Ctx *c, CcLevel &L)
{
    if (L.bxp)
        EBV_LAUNCH(c, k_xface_pad<RbF>, dim3(kReduceBlocks), dim3(256), 0, L.g, L.bf_f[0], (RbF *)L.bxp);
    if constexpr (!kVcycleBf16) return;
    for (int d = 0; d < 3; d++) {
        const int n = nface(L.g, d);
        EBV_LAUNCH(c, k_to_bf16, dim3(std::min(kReduceBlocks, (n + 255) / 256)), dim3(256), 0, L.bf_f[d], L.bf_h[d], n);
    }
}

template <class T>
NdOp<T> ndop(const NdLevel &L)
{
    NdOp<T> A;
    A.g = L.g;
    A.h = (T)L.g.h;
    if constexpr (sizeof(T) == 8) A.alpha = (const T *)L.alpha_d;
    else A.alpha = (const T *)L.alpha_f;
    A.act = L.act;
    A.reg = L.reg;
    return A;
}

// ---------------------------------------------------------------------------
// V-cycles
// ---------------------------------------------------------------------------

// Profiling labels of the colour passes per precision and level (level 0 is
// HBM-bound; the coarse levels are latency- and launch-bound): plain passes
// (from zero or not), the pass after the coarse correction, and the pass
// that also forms r.z; and of the residual-restriction per level.
static const char *const kGsName[2][8] = {
    {"cc_gs_colour_pass<double> L0", "cc_gs_colour_pass<double> L1", "cc_gs_colour_pass<double> L2",
     "cc_gs_colour_pass<double> L3", "cc_gs_colour_pass<double> L4", "cc_gs_colour_pass<double> L5",
     "cc_gs_colour_pass<double> L6", "cc_gs_colour_pass<double> L7+"},
    {"cc_gs_colour_pass<float> L0", "cc_gs_colour_pass<float> L1", "cc_gs_colour_pass<float> L2",
     "cc_gs_colour_pass<float> L3", "cc_gs_colour_pass<float> L4", "cc_gs_colour_pass<float> L5",
     "cc_gs_colour_pass<float> L6", "cc_gs_colour_pass<float> L7+"}};
static const char *const kGsCorrName[2][8] = {
    {"cc_gs_correction_pass<double> L0", "cc_gs_correction_pass<double> L1", "cc_gs_correction_pass<double> L2",
     "cc_gs_correction_pass<double> L3", "cc_gs_correction_pass<double> L4", "cc_gs_correction_pass<double> L5",
     "cc_gs_correction_pass<double> L6", "cc_gs_correction_pass<double> L7+"},
    {"cc_gs_correction_pass<float> L0", "cc_gs_correction_pass<float> L1", "cc_gs_correction_pass<float> L2",
     "cc_gs_correction_pass<float> L3", "cc_gs_correction_pass<float> L4", "cc_gs_correction_pass<float> L5",
     "cc_gs_correction_pass<float> L6", "cc_gs_correction_pass<float> L7+"}};
static const char *const kGsDotName[2] = {"cc_gs_rz_pass<double> L0", "cc_gs_rz_pass<float> L0"};
static const char *const kRrName[2][4] = {
    {"cc_residual_restrict<double> L0", "cc_residual_restrict<double> L1", "cc_residual_restrict<double> L2",
     "cc_residual_restrict<double> L3+"},
    {"cc_residual_restrict<float> L0", "cc_residual_restrict<float> L1", "cc_residual_restrict<float> L2",
     "cc_residual_restrict<float> L3+"}};

// Two red-black Gauss-Seidel sweeps in place (the first from x = 0 when
// zero_start), each as two colour passes.
inline dim3 gs_grid(const GridD &g, dim3 bk)
{
    const int nzg = (g.nz + GS_PZ - 1) / GS_PZ;
    return dim3(((g.nx + 1) / 2 + bk.x - 1) / bk.x, (g.ny + bk.y - 1) / bk.y, (nzg + bk.z - 1) / bk.z);
}
inline dim3 ch_grid(const GridD &g, dim3 bk)
{
    return dim3((g.nx + 1 + bk.x - 1) / bk.x, (g.ny + 1 + bk.y - 1) / bk.y, (g.nz + 1 + bk.z - 1) / bk.z);
}


// ---- the fused sweep on the host: where it applies, tensor maps, shape -----
enum { RB_ZERO = 0, RB_PLAIN = 1, RB_CORR = 2, RB_DOT = 3 };
constexpr size_t kPartLen = (size_t)1 << 20;   // doubles in c->part

inline int rb_ntiles(const GridD &g) { return ((g.nx / 2 + RB_HW - 1) / RB_HW) * ((g.ny + RB_TY - 1) / RB_TY); }

// FP32 levels whose half-rows are whole multiples of 8 positions (16-byte TMA
// strides for the BF16 face rows); their r.z partials are per (plane, tile).
inline bool rb_fusable(const GridD &g)
{
    return g.nx % 16 == 0 && g.nx >= 16 && (size_t)rb_ntiles(g) * g.nz <= kPartLen;
}

// Tensor map of one array of the level, by box kind: 0 x (FP32 cells, tile +
// 2 rows each side), 1 FP32 cells (tile + 1 row), 2 y faces, 3 z faces, 4 the
// padded x faces, 5 the coarse correction (g the coarse level: the parents
// of the tile and its ring); the array viewed as (half-row position, half,
// row, plane).
bool rb_map(Ctx *c, const void *p, int kind, const GridD &g, CUtensorMap *out)
{
    if (!p) return false;
    for (const auto &e : c->tma)
        if (e.p == p && e.kind == kind && e.nx == g.nx && e.ny == g.ny && e.nz == g.nz) {
            *out = e.m;
            return true;
        }
    const bool face = kind >= 2 && kind <= 4;
    const uint64_t es = face ? sizeof(RbF) : 4;
    const uint64_t hx = kind == 4 ? (uint64_t)rb_hxp(g.nx) : (uint64_t)g.nx / 2;
    const uint64_t rows = kind == 2 ? g.ny + 1 : g.ny, planes = kind == 3 ? g.nz + 1 : g.nz;
    const uint64_t dims[4] = {hx, 2, rows, planes};
    const uint64_t st[3] = {hx * es, 2 * hx * es, rows * 2 * hx * es};
    const uint32_t box[4] = {(uint32_t)(kind == 5 ? RB_KW : (face ? RB_FW : RB_XW)), 2u,
                             (uint32_t)(kind == 0 ? RB_XR : (kind == 2 ? RB_YR : (kind == 5 ? RB_KR : RB_CR))), 1u};
    const CUtensorMapDataType ty = (face && sizeof(RbF) == 2) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                              : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    Ctx::TmaEntry e;
    e.p = p;
    e.kind = kind;
    e.nx = g.nx;
    e.ny = g.ny;
    e.nz = g.nz;
    if (!tma_encode_4d(&e.m, ty, const_cast<void *>(p), dims, st, box)) return false;
    c->tma.push_back(e);
    *out = e.m;
    return true;
}

template <bool kZero, bool kCorr, bool kDot>
void rb_attr()
{
    static bool done = false;
    if (!done) {
        done = true;
        cudaFuncSetAttribute(k_cc_rb_sweep<RbF, kZero, kCorr, kDot>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             RbSmem<RbF>::bytes);
    }
}

// Blocks of the fused sweep resident on the device at once.
int rb_resident()
{
    static int res = 0;
    if (!res) {
        rb_attr<false, false, false>();
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cc_rb_sweep<RbF, false, false, false>, RB_THREADS,
                                                      RbSmem<RbF>::bytes);
        res = std::max(1, per) * std::max(1, sms);
    }
    return res;
}

// Planes per chunk of a block: the fewest waves of resident blocks times the
// steps of one block (its planes and the two of the chunk's start).
int rb_kz(const GridD &g)
{
    const long long nt = rb_ntiles(g), res = rb_resident();
    long long best = -1;
    int bkz = g.nz;
    for (int nc = 1; nc <= g.nz; nc++) {
        const int kz = (g.nz + nc - 1) / nc, ncr = (g.nz + kz - 1) / kz;
        const long long cost = ((nt * ncr + res - 1) / res) * (kz + 2);
        if (best < 0 || cost < best) {
            best = cost;
            bkz = kz;
        }
    }
    return bkz;
}

// One fused sweep (maps already encoded by rb_maps).
void rb_launch(Ctx *c, const char *name, const GridD &g, const RbMaps &tm, float *xout, int c0, int mode,
               double *part, int kz = 0)
{
    RbArgs<RbF> a;
    a.g = g;
    a.xout = xout;
    a.part = part;
    a.ctl = c->ctl;
    a.c0 = c0;
    a.kz = kz > 0 ? kz : rb_kz(g);
    a.spin = spin_limit();
    const dim3 gr((g.nx / 2 + RB_HW - 1) / RB_HW, (g.ny + RB_TY - 1) / RB_TY, (g.nz + a.kz - 1) / a.kz);
    // algorithmic bytes: x written, x read (not from zero), b, 1/diag, three
    // faces, the coarse correction (1/8 word per cell)
    const double nb = (double)ncell(g) * (4.0 + (mode == RB_ZERO ? 0.0 : 4.0) + 8.0 + 3.0 * sizeof(RbF) +
                                          (mode == RB_CORR ? 0.5 : 0.0));
    const int sb = RbSmem<RbF>::bytes;
    switch (mode) {
    case RB_ZERO:
        rb_attr<true, false, false>();
        EBV_LAUNCH_P(c, name, nb, (k_cc_rb_sweep<RbF, true, false, false>), gr, dim3(RB_THREADS), sb, tm, a);
        break;
    case RB_CORR:
        rb_attr<false, true, false>();
        EBV_LAUNCH_P(c, name, nb, (k_cc_rb_sweep<RbF, false, true, false>), gr, dim3(RB_THREADS), sb, tm, a);
        break;
    case RB_DOT:
        rb_attr<false, false, true>();
        EBV_LAUNCH_P(c, name, nb, (k_cc_rb_sweep<RbF, false, false, true>), gr, dim3(RB_THREADS), sb, tm, a);
        break;
    default:
        rb_attr<false, false, false>();
        EBV_LAUNCH_P(c, name, nb, (k_cc_rb_sweep<RbF, false, false, false>), gr, dim3(RB_THREADS), sb, tm, a);
    }
}

const char *const kRbName[8] = {"cc_rb_sweep<float> L0", "cc_rb_sweep<float> L1", "cc_rb_sweep<float> L2",
                                "cc_rb_sweep<float> L3", "cc_rb_sweep<float> L4", "cc_rb_sweep<float> L5",
                                "cc_rb_sweep<float> L6", "cc_rb_sweep<float> L7+"};

// Two red-black sweeps' worth of smoothing is two calls; this is one sweep
// pair as the V-cycle uses it: sweep 1 (from zero, or after the coarse
// correction) then sweep 2 (plain, or with r.z partials).
// dot_part: the last pass also writes partials of b.x -- per (plane, tile)
// (k_cc_rb_sweep<kDot> or k_cc_gs2_dot) on levels the fused sweep applies
// to, else per block of k_cc_gs<kDot>; returns their number (0 without
// dot_part).  FP32 levels with nx a multiple of 16 can run each sweep as one
// fused pass (x -> t -> x) or as two colour passes, with the same results bit
// for bit: ebv_set_fused_sweep picks the passes (0), the faster of the two as
// timed when the solvers are set up (1, the default) or the fused pass (2).
template <class T>
int cc_smooth2(Ctx *c, const CcLevel &L, int l, T *x, T *t, const T *b, bool red_first, bool zero_start,
               const T *xc = nullptr, const GridD *gc = nullptr, double *dot_part = nullptr)
{
    VOp<T> A = vop<T>(L);
    const int c0 = red_first ? 0 : 1;
    const GridD &g = L.g;
    bool tiles = false;   // r.z partials per (plane, tile)
    if constexpr (sizeof(T) == 4) {
        if (rb_fusable(g)) {
            tiles = true;
            RbMaps m1, m2;
            // each kind of sweep (from zero, plain, after the coarse correction,
            // with r.z) was timed on its own against its colour passes
            const int mode = fused_sweep_mode();
            const int k1 = zero_start ? RB_ZERO : (xc ? RB_CORR : RB_PLAIN), k2 = dot_part ? RB_DOT : RB_PLAIN;
            // (the pair runs x -> t -> x fused, or in place as passes: one form for both)
            const bool faster = L.rb_ms[k1][0] + L.rb_ms[k2][0] < L.rb_ms[k1][1] + L.rb_ms[k2][1];
            bool use = (mode == 2 || (mode == 1 && faster)) && rb_map(c, x, 0, g, &m1.x) &&
                       rb_map(c, t, 0, g, &m2.x) && rb_map(c, b, 1, g, &m1.b) && rb_map(c, A.dinv, 1, g, &m1.d) &&
                       rb_map(c, L.bxp, 4, g, &m1.fx) && rb_map(c, A.by, 2, g, &m1.fy) &&
                       rb_map(c, A.bz, 3, g, &m1.fz);
            if (use) {
                m2.b = m1.b;
                m2.d = m1.d;
                m2.fx = m1.fx;
                m2.fy = m1.fy;
                m2.fz = m1.fz;
                m1.xc = m2.xc = m1.b;   // (read by the correction sweep only)
                if (k1 == RB_CORR) use = rb_map(c, xc, 5, *gc, &m1.xc);
            }
            if (use) {
                const char *nm = kRbName[l < 7 ? l : 7];
                rb_launch(c, nm, g, m1, t, c0, k1, nullptr, L.rb_kz);
                rb_launch(c, nm, g, m2, x, c0, k2, dot_part, L.rb_kz);
                return dot_part ? rb_ntiles(g) * g.nz : 0;
            }
        }
    }
    // algorithmic bytes of one colour pass: half of one sweep's x read and
    // write, b, diagonal and 3 face coefficients (in their storage type)
    const double nb = 0.5 * ((4.0 * sizeof(T) + 3.0 * sizeof(typename VFace<T>::type)) * (double)ncell(g));
    // threads: x-pairs x rows x groups of GS_PZ planes, in the level's block shape
    const dim3 bk = L.gs_blk, gr = gs_grid(g, bk);
    const char *name = kGsName[sizeof(T) == 4][l < 7 ? l : 7];
    for (int s = 0; s < 2; s++) {
        const int z = (s == 0 && zero_start) ? 1 : 0;
        // the plain passes of FP32 levels with half-rows of a multiple of 4
        // cells take the vectorised form (same results)
        auto plain = [&](int color, int zs) {
            if constexpr (sizeof(T) == 4) {
                if (gs4_ok(g)) {
                    if (L.gs4_pz == 1)
                        EBV_LAUNCH_P(c, name, nb, (k_cc_gs4<1>), gs4_grid(g, L.gs4_blk, 1), L.gs4_blk, 0, A, x, b,
                                     color, zs);
                    else
                        EBV_LAUNCH_P(c, name, nb, (k_cc_gs4<2>), gs4_grid(g, L.gs4_blk, 2), L.gs4_blk, 0, A, x, b,
                                     color, zs);
                    return;
                }
            }
            EBV_LAUNCH_P(c, name, nb, (k_cc_gs<T, false>), gr, bk, 0, A, x, b, color, zs, nullptr, GridD());
        };
        if (s == 0 && xc) {  // the first pass after the coarse-grid correction (+ the coarse array)
            const char *nmc = kGsCorrName[sizeof(T) == 4][l < 7 ? l : 7];
            const double nbc = nb + 0.125 * sizeof(T) * (double)ncell(g);
            bool done = false;
            if constexpr (sizeof(T) == 4) {
                if (gs4_ok(g)) {   // vectorised, same results
                    if (L.gs4_pz == 1)
                        EBV_LAUNCH_P(c, nmc, nbc, (k_cc_gs4<1, true>), gs4_grid(g, L.gs4_blk, 1), L.gs4_blk, 0, A, x, b,
                                     c0, z, xc, *gc);
                    else
                        EBV_LAUNCH_P(c, nmc, nbc, (k_cc_gs4<2, true>), gs4_grid(g, L.gs4_blk, 2), L.gs4_blk, 0, A, x, b,
                                     c0, z, xc, *gc);
                    done = true;
                }
            }
            if (!done) EBV_LAUNCH_P(c, nmc, nbc, (k_cc_gs<T, true>), gr, bk, 0, A, x, b, c0, z, xc, *gc);
        }
        else
            plain(c0, z);
        if (s == 1 && dot_part && tiles) {
            // the fused sweep's r.z partials, per (plane, tile), with the last pass
            if constexpr (sizeof(T) == 4) {
                const dim3 gt((g.nx / 2 + RB_HW - 1) / RB_HW, (g.ny + RB_TY - 1) / RB_TY,
                              (g.nz + kGs2Planes - 1) / kGs2Planes);
                EBV_LAUNCH_P(c, kGsDotName[1], nb, k_cc_gs2_dot, gt, dim3(RB_THREADS), 0, A, x, b, 1 - c0, dot_part);
                return rb_ntiles(g) * g.nz;
            }
        } else if (s == 1 && dot_part) {
            // fixed block shape: the grouping of its partial sums must not
            // follow the autotuned shape, or results would depend on timing
            EBV_LAUNCH_P(c, kGsDotName[sizeof(T) == 4], nb, (k_cc_gs<T, false, true>), gs_grid(g, block3()), block3(),
                         0, A, x, b, 1 - c0, 0, nullptr, GridD(), dot_part);
        } else {
            plain(1 - c0, 0);
        }
    }
    if (!dot_part) return 0;
    const dim3 gd = gs_grid(g, block3());
    return (int)(gd.x * gd.y * gd.z);
}

// One V-cycle x0 = M b0.  dot_part: the finest level's last pass also
// writes block partials of b0.x0; returns their number (0 when the whole
// V-cycle runs in the coarse kernel, or without dot_part).
template <class T>
int cc_vcycle(Ctx *c, CcHier &H, const T *b0, T *x0, double *dot_part = nullptr)
{
    const int Lb = H.L - 1;
    // levels l0 .. Lb (each at most kCoarseCells cells) run in one CTA
    int l0 = Lb;
    while (l0 > 0 && ncell(H.lv[l0 - 1].g) <= kCoarseCells && Lb - l0 + 2 <= kCoarseMax) l0--;
    for (int l = 0; l < l0; l++) {
        const CcLevel &L = H.lv[l];
        T *x = l ? (T *)c->lx[l] : x0;
        const T *b = l ? (const T *)c->lb[l] : b0;
        cc_smooth2<T>(c, L, l, x, (T *)c->lt[l], b, true, true);
        const CcLevel &Lc = H.lv[l + 1];
        // x, b, diagonal, 3 faces (storage type) read, 1/8 word written
        const double nbr = ((3.0 + 1.0 / 8.0) * sizeof(T) + 3.0 * sizeof(typename VFace<T>::type)) * (double)ncell(L.g);
        const char *nmr = kRrName[sizeof(T) == 4][l < 3 ? l : 3];
        bool vec = false;
        if constexpr (sizeof(T) == 4) {
            const dim3 bk(8, 8, 4), gr((Lc.g.nx / 4 + bk.x - 1) / bk.x, (Lc.g.ny + bk.y - 1) / bk.y,
                                        (Lc.g.nz + bk.z - 1) / bk.z);
            // four coarse cells per thread, vector loads (same results), where
            // that still gives two blocks per SM (small levels keep the scalar kernel)
            if (gs4_ok(L.g) && (long long)gr.x * gr.y * gr.z >= kVecMinBlocks) {
                EBV_LAUNCH_P(c, nmr, nbr, k_cc_rr4, gr, bk, 0, vop<float>(L), x, b, Lc.g, (float *)c->lb[l + 1]);
                vec = true;
            }
        }
        if (!vec)
            EBV_LAUNCH_P(c, nmr, nbr, k_cc_resid_restrict<T>, cgrid(Lc.g), block3(), 0, vop<T>(L), x, b, Lc.g,
                         (T *)c->lb[l + 1]);
    }
    if (l0 < Lb) {
        CoarseVC<T> D;
        D.n = Lb - l0 + 1;
        for (int q = 0; q < D.n; q++) {
            const int l = l0 + q;
            D.A[q] = vop<T>(H.lv[l]);
            D.x[q] = l ? (T *)c->lx[l] : x0;
            D.b[q] = l ? (T *)c->lb[l] : (T *)b0;
        }
        D.binv = H.binv;
        D.nb = H.nb;
        // staged in shared memory when it fits (with the bottom inverse if that fits too)
        int sb = coarse_stage_bytes(D, 1) <= kCoarseStageMax;
        const size_t bytes = coarse_stage_bytes(D, sb);
        if (bytes <= kCoarseStageMax)
            EBV_LAUNCH_P(c, sizeof(T) == 4 ? "cc_coarse_vcycle<float>" : "cc_coarse_vcycle<double>", 0.0,
                         (k_cc_coarse_vcycle<T, true>), dim3(1), dim3(kCoarseThreads), bytes, D, sb);
        else
            EBV_LAUNCH_P(c, sizeof(T) == 4 ? "cc_coarse_vcycle<float>" : "cc_coarse_vcycle<double>", 0.0,
                         (k_cc_coarse_vcycle<T, false>), dim3(1), dim3(kCoarseThreads), 0, D, 0);
    } else {
        T *x = Lb ? (T *)c->lx[Lb] : x0;
        const T *b = Lb ? (const T *)c->lb[Lb] : b0;
        EBV_LAUNCH(c, k_bottom_solve<T>, dim3((H.nb + 255) / 256), dim3(256), 0, H.binv, H.nb, b, x, 1.0,
                   H.lv[Lb].g, (int)(sizeof(T) == 4));
    }
    for (int l = l0 - 1; l >= 0; l--) {
        const CcLevel &L = H.lv[l];
        T *x = l ? (T *)c->lx[l] : x0;
        const T *b = l ? (const T *)c->lb[l] : b0;
        // prolongation folded into the first colour pass of the post-smoothing
        const int nd = cc_smooth2<T>(c, L, l, x, (T *)c->lt[l], b, false, false, (const T *)c->lx[l + 1],
                                     &H.lv[l + 1].g, l == 0 ? dot_part : nullptr);
        if (l == 0) return nd;
    }
    return 0;
}

// Chebyshev coefficients on [lam_max / 8, lam_max] of D^-1 A, degree 3.
struct ChebCoef { double cd[3], cr[3]; };
inline ChebCoef cheb_coef(double lmax)
{
    const double lmin = lmax / 8.0;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    ChebCoef k;
    double rho0 = 1.0 / sigma;
    k.cd[0] = 0.0;
    k.cr[0] = 1.0 / theta;
    for (int s = 1; s < 3; s++) {
        double rho1 = 1.0 / (2.0 * sigma - rho0);
        k.cd[s] = rho1 * rho0;
        k.cr[s] = 2.0 * rho1 / delta;
        rho0 = rho1;
    }
    return k;
}

// Three Chebyshev steps on A x = b, ending in x.  From zero: (0) -> x -> t -> x.
// Otherwise the start is in t: t -> x -> t -> x.  d is the level's direction.
// A nodal pass on a level with regular-node flags: the plane march over the
// regular and inactive nodes, then the listed nodes (their ND_APPLY partials
// follow the march's).
inline int nd_tile_blocks(const GridD &g)
{
    const dim3 gr = nd_tile_grid(g);
    return (int)(gr.x * gr.y * gr.z);
}
template <class T, int kMode>
void nd_tile_pass(Ctx *c, const NdLevel &L, const char *name, double nbytes, const T *xin, T *out, T *d,
                const T *b, T cd, T cr, double *part, float *out32 = nullptr, const double *sig = nullptr)
{
    const NdOp<T> A = ndop<T>(L);
    EBV_LAUNCH_P(c, name, nbytes, (k_nd_tile<T, kMode>), nd_tile_grid(L.g), dim3(NT_X, NT_Y), 0, A, xin, out, d, b,
                 cd, cr, part, out32, sig);
    static const char *const kIrrName[4] = {"nodal_listed_nodes chebyshev", "nodal_listed_nodes residual",
                                            "nodal_listed_nodes apply", "nodal_listed_nodes refinement residual"};
    if (L.nirr)
        EBV_LAUNCH_P(c, kIrrName[kMode], 0.0, (k_nd_irr<T, kMode>), dim3((L.nirr + 255) / 256), dim3(256), 0, A, L.irr,
                     L.nirr, xin, out, d, b, cd, cr, part ? part + nd_tile_blocks(L.g) : nullptr, out32, sig);
}
// partial sums written by nd_tile_pass on level L
inline int nd_tile_parts(const NdLevel &L) { return nd_tile_blocks(L.g) + (L.nirr ? (L.nirr + 255) / 256 : 0); }

template <class T>
void nd_smooth(Ctx *c, const NdLevel &L, int l, T *x, T *t, const T *b, bool zero_start)
{
    NdOp<T> A = ndop<T>(L);
    ChebCoef k = cheb_coef(L.lam_max);
    T *d = (T *)c->ld[l];
    T *src = zero_start ? x : t, *dst = x;
    for (int s = 0; s < 3; s++) {
        // per node: x in/out, d in/out, b, alpha of one cell (the first step
        // from zero reads only b and alpha and writes d, x)
        const bool z0 = s == 0 && zero_start;
        const double nb = (z0 ? 4.0 : 6.0) * sizeof(T) * (double)nnode(L.g);
        if (!z0 && L.reg)   // levels with regular-node flags: plane-sum form
            nd_tile_pass<T, ND_CHEB>(c, L,
                                   sizeof(T) == 4 ? (l ? "nodal_chebyshev_step<float> L1+" : "nodal_chebyshev_step<float> L0")
                                                  : (l ? "nodal_chebyshev_step<double> L1+" : "nodal_chebyshev_step<double> L0"),
                                   nb, src, dst, d, b, (T)k.cd[s], (T)k.cr[s], nullptr);
        else
            EBV_LAUNCH_P(c, sizeof(T) == 4 ? "nodal_chebyshev_step<float>" : "nodal_chebyshev_step<double>", nb,
                         k_nd_cheb<T>, ch_grid(L.g, L.ch_blk), L.ch_blk, 0, A, src, dst, d, b, (T)k.cd[s],
                         (T)k.cr[s], (int)z0);
        src = dst;
        dst = (dst == x) ? t : x;
    }
}

template <class T>
void nd_vcycle(Ctx *c, NdHier &H, const T *b0, T *x0)
{
    const int Lb = H.L - 1;
    for (int l = 0; l < Lb; l++) {
        const NdLevel &L = H.lv[l];
        T *x = l ? (T *)c->lx[l] : x0;
        const T *b = l ? (const T *)c->lb[l] : b0;
        nd_smooth<T>(c, L, l, x, (T *)c->lt[l], b, true);
        if (L.reg)
            nd_tile_pass<T, ND_RESID>(c, L, l ? "k_nd_resid<T> tiled L1+" : "k_nd_resid<T> tiled L0", 0.0, x, (T *)c->lr[l], nullptr, b, T(0), T(0),
                                    nullptr);
        else
            EBV_LAUNCH(c, k_nd_resid<T>, ngrid(L.g), block3(), 0, ndop<T>(L), x, b, (T *)c->lr[l]);
        const NdLevel &Lc = H.lv[l + 1];
        EBV_LAUNCH(c, k_nd_restrict<T>, ngrid(Lc.g), block3(), 0, L.g, (const T *)c->lr[l], Lc.g, Lc.act,
                   (T *)c->lb[l + 1]);
    }
    {
        T *x = Lb ? (T *)c->lx[Lb] : x0;
        const T *b = Lb ? (const T *)c->lb[Lb] : b0;
        EBV_LAUNCH(c, k_bottom_solve<T>, dim3((H.nb + 255) / 256), dim3(256), 0, H.binv, H.nb, b, x, 1.0,
                   H.lv[Lb].g, 0);
    }
    for (int l = Lb - 1; l >= 0; l--) {
        const NdLevel &L = H.lv[l];
        T *x = l ? (T *)c->lx[l] : x0;
        const T *b = l ? (const T *)c->lb[l] : b0;
        // t = x + P x_coarse, then smooth from t back into x
        EBV_LAUNCH(c, k_nd_prolong<T>, ngrid(L.g), block3(), 0, L.g, L.act, H.lv[l + 1].g,
                   (const T *)c->lx[l + 1], x, (T *)c->lt[l]);
        nd_smooth<T>(c, L, l, x, (T *)c->lt[l], b, false);
    }
}

// ---------------------------------------------------------------------------
// Preconditioned conjugate gradients
// ---------------------------------------------------------------------------

struct Problem {
    virtual ~Problem() {}
    virtual int n() const = 0;
    virtual int apply_blocks() const = 0;      // partial sums written by apply_dot
    virtual int apply_blocks32() const { return apply_blocks(); }   // by apply_dot32
    virtual int resid_blocks() const { return apply_blocks(); }     // by resid32
    // q = A p with block partials of p.q in c->part, in FP64 or FP32
    virtual void apply_dot(Ctx *c, const double *p, double *q) = 0;
    virtual void apply_dot32(Ctx *c, const float *p, float *q) = 0;
    // z = one V-cycle applied to r, in FP64 or FP32
    virtual void precond(Ctx *c, const double *r, double *z) = 0;
    virtual void precond32(Ctx *c, const float *r, float *z) = 0;
    // precond32 that may also leave block partials of r.z in c->part:
    // returns their number, 0 if it did not
    virtual int precond32_dot(Ctx *c, const float *r, float *z)
    {
        precond32(c, r, z);
        return 0;
    }
    // FP64 <-> FP32 vectors of the refinement solver (the FP32 side in the
    // layout of the problem's FP32 multigrid): r = b - A x in FP64 with
    // resid_blocks() block partials of |r|^2 in c->part; x += e
    virtual void resid32(Ctx *c, const double *b, const double *x, float *r) = 0;
    virtual void to32(Ctx *c, const double *b, float *r) = 0;   // r = b in the FP32 layout
    // x += e + the deferred last step of the correction solve (search direction p)
    virtual void add32(Ctx *c, double *x, const float *e, const float *p) = 0;
};

inline int vblocks(int n) { return std::min(kReduceBlocks, (n + 255) / 256); }

// A loop whose condition is decided on the device.  Eager mode: next()
// reads the condition word back (one synchronisation per pass).  Capture
// mode: the first next() adds a conditional WHILE node after the work issued
// so far and redirects the context's stream into the node's body graph; the
// second ends the body capture.  The kernel that sets the condition before
// the loop and the last kernel of the body take (h, use_h).
struct DevLoop {
    Ctx *c;
    int slot;
    cudaGraphConditionalHandle h = 0;
    int use_h = 0;
    int pass = 0;
    cudaStream_t saved = nullptr, body = nullptr;
    long long l0 = 0;
    int inner_count = 0;   // launches of a nested loop's body (capture mode)

    DevLoop(Ctx *c_, int slot_) : c(c_), slot(slot_)
    {
        if (!c->capturing) return;
        cudaStreamCaptureStatus st;
        cudaGraph_t g = nullptr;
        if (cudaStreamGetCaptureInfo(c->stream, &st, nullptr, &g) != cudaSuccess ||
            st != cudaStreamCaptureStatusActive ||
            cudaGraphConditionalHandleCreate(&h, g, 0, 0) != cudaSuccess) {
            if (c->cap_err.empty()) c->cap_err = "conditional handle";
            return;
        }
        use_h = 1;
    }

    bool next()
    {
        if (!c->capturing) {
            if (cudaMemcpyAsync(c->ctl_host + slot, c->ctl + slot, sizeof(int), cudaMemcpyDeviceToHost,
                                c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                return false;
            return c->ctl_host[slot] != 0;
        }
        if (pass == 0) {
            pass = 1;
            if (!use_h || c->cap_depth + 1 >= 4) {
                if (c->cap_err.empty()) c->cap_err = "loop nesting";
                return false;
            }
            cudaStreamCaptureStatus st;
            cudaGraph_t g = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            if (cudaStreamGetCaptureInfo(c->stream, &st, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess ||
                cudaGraphAddNode(&node, g, deps, nullptr, nd, &np) != cudaSuccess ||
                cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies) != cudaSuccess) {
                if (c->cap_err.empty()) c->cap_err = "conditional node";
                return false;
            }
            body = c->cap_stream[++c->cap_depth];
            if (cudaStreamBeginCaptureToGraph(body, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                c->cap_depth--;
                if (c->cap_err.empty()) c->cap_err = "body capture";
                return false;
            }
            saved = c->stream;
            c->stream = body;
            l0 = c->launches;
            return true;
        }
        if (pass == 1) {
            pass = 2;
            cudaGraph_t gb = nullptr;
            if (cudaStreamEndCapture(body, &gb) != cudaSuccess && c->cap_err.empty()) c->cap_err = "body end";
            c->stream = saved;
            c->cap_depth--;
        }
        return false;
    }
    // launches captured in the body (valid after the loop in capture mode)
    int body_launches() const { return (int)(c->launches - l0); }
};

// Issues the end-of-solve kernels and, in eager mode, reads the solve's
// statistics and status back.
ebv_status finish_solve(Ctx *c, double *x, int n, int *iters, double *res)
{
    EBV_LAUNCH(c, k_zero_if, dim3(vblocks(n)), dim3(256), 0, x, n, c->ctl);
    EBV_LAUNCH(c, k_solve_end, dim3(1), dim3(32), 0, c->scal, c->ctl, c->prm.tol, c->sstat, c->cur_slot);
    if (c->capturing) {
        if (iters) *iters = 0;
        if (res) *res = 0.0;
        return EBV_OK;
    }
    const int s = c->cur_slot;
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->sstat_host + 3 * s, c->sstat + 3 * s, 3 * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->ctl_host + C_ERR, c->ctl + C_ERR, sizeof(int), cudaMemcpyDeviceToHost,
                                    c->stream));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (iters) *iters = (int)c->sstat_host[3 * s];
    if (res) *res = c->sstat_host[3 * s + 1];
    if (c->ctl_host[C_ERR] == E_NAN)
        return c->fail(EBV_ERR_NAN, "non-finite residual (solve slot " + std::to_string(s) + ")");
    if (c->ctl_host[C_ERR] == E_SMEM)
        return c->fail(EBV_ERR_CUDA, "shared memory of the fused sweep not 128-byte aligned (solve slot " +
                                         std::to_string(s) + ")");
    if (c->ctl_host[C_ERR] == E_TIMEOUT)
        return c->fail(EBV_ERR_TIMEOUT, "a bounded wait in the smoother gave up (solve slot " + std::to_string(s) + ")");
    if (c->ctl_host[C_ERR] == E_NOTCONV)
        return c->fail(EBV_ERR_NOT_CONVERGED, "linear solve did not reach the tolerance (solve slot " +
                                                  std::to_string(s) + ", relative residual " +
                                                  std::to_string(c->sstat_host[3 * s + 1]) + ", " +
                                                  std::to_string((int)c->sstat_host[3 * s]) + " iterations)");
    return EBV_OK;
}

// Preconditioned CG in FP64, restarted from the true residual whenever the
// recursive one has dropped below tol/2 but the true one is still above tol
// (at most 20 passes).
ebv_status pcg(Ctx *c, Problem &P, const double *b, double *x, int *iters, double *res)
{
    const int n = P.n();
    const double tol = c->prm.tol;
    const int maxit = c->prm.max_iters;
    double *r = c->kr, *z = c->kz, *p = c->kp, *q = c->kq;
    auto true_residual = [&]() {
        P.apply_dot(c, x, q);
        EBV_LAUNCH(c, k_resid_init, dim3(vblocks(n)), dim3(256), 0, b, q, r, n, c->part);
        reduce_sum(c, c->part, vblocks(n), c->scal + S_RR);
        reduce_sum(c, c->part + vblocks(n), vblocks(n), c->scal + S_BB);
    };
    EBV_LAUNCH(c, k_solve_begin, dim3(1), dim3(32), 0, c->ctl);
    DevLoop outer(c, C_COND_OUT);
    true_residual();
    EBV_LAUNCH(c, k_outer_check, dim3(1), dim3(32), 0, c->scal, c->ctl, tol, maxit, 20, 0, 0.0, outer.h,
               outer.use_h);
    int inner_count = 0;
    while (outer.next()) {
        DevLoop inner(c, C_COND_IN);
        EBV_LAUNCH(c, k_set_cond, dim3(1), dim3(32), 0, c->ctl, C_COND_IN, 1, inner.h, inner.use_h);
        while (inner.next()) {
            P.precond(c, r, z);
            EBV_LAUNCH(c, k_dot, dim3(vblocks(n)), dim3(256), 0, r, z, n, c->part);
            reduce_sum(c, c->part, vblocks(n), c->scal + S_RZ);
            EBV_LAUNCH(c, k_cg_pupdate, dim3(vblocks(n)), dim3(256), 0, p, z, c->scal, n, c->ctl);
            P.apply_dot(c, p, q);
            reduce_sum(c, c->part, P.apply_blocks(), c->scal + S_PQ);
            EBV_LAUNCH(c, k_cg_update, dim3(vblocks(n)), dim3(256), 0, x, r, p, q, c->scal, n, c->part);
            EBV_LAUNCH(c, k_reduce_inner_check, dim3(1), dim3(1024), 0, c->part, vblocks(n), c->scal, c->ctl, tol,
                       maxit, 0, inner.h, inner.use_h);
        }
        inner_count = inner.body_launches();
        true_residual();
        EBV_LAUNCH(c, k_outer_check, dim3(1), dim3(32), 0, c->scal, c->ctl, tol, maxit, 20, 0, 0.0, outer.h,
                   outer.use_h);
    }
    if (c->capturing)
        c->loop_recs.push_back({c->cur_slot, outer.body_launches() - inner_count, inner_count});
    if (!c->cap_err.empty() && c->capturing) return c->fail(EBV_ERR_CUDA, "graph capture: " + c->cap_err);
    return finish_solve(c, x, n, iters, res);
}

// Iterative refinement for the FP32 path: the residual r = b - A x and the
// solution update x += e are FP64; each correction e solves A e = r with
// conjugate gradients run entirely in FP32 (vectors, operator with FP32
// coefficients, V-cycle) until its residual drops by `inner_drop` (or it
// stalls), so FP64 arithmetic is spent once per refinement step instead of in
// every Krylov iteration.  At most 60 corrections.
ebv_status pcg_refine(Ctx *c, Problem &P, const double *b, double *x, int *iters, double *res, bool x_zero)
{
    const int n = P.n();
    const double tol = c->prm.tol;
    const int maxit = c->prm.max_iters;
    const double inner_drop = refine_inner_drop();
    float *r = c->kr32, *z = c->kz32, *p = c->kp32, *q = c->kq32, *e = c->ke32;
    // x_zero: the first residual is b itself (its norm is |b|^2, reduced below)
    bool first_is_b = x_zero;
    auto true_residual = [&]() {
        if (first_is_b) {
            first_is_b = false;
            P.to32(c, b, r);
            return;
        }
        P.resid32(c, b, x, r);
        reduce_sum(c, c->part, P.resid_blocks(), c->scal + S_RR);
    };
    EBV_LAUNCH(c, k_solve_begin, dim3(1), dim3(32), 0, c->ctl);
    EBV_LAUNCH(c, k_dot, dim3(vblocks(n)), dim3(256), 0, b, b, n, c->part);
    reduce_sum(c, c->part, vblocks(n), c->scal + S_BB);
    EBV_LAUNCH(c, k_set_sigma, dim3(1), dim3(32), 0, c->scal, x_zero ? 1 : 0);
    DevLoop outer(c, C_COND_OUT);
    true_residual();
    EBV_LAUNCH(c, k_outer_check, dim3(1), dim3(32), 0, c->scal, c->ctl, tol, maxit, 60, 1, inner_drop, outer.h,
               outer.use_h);
    int inner_count = 0;
    while (outer.next()) {
        DevLoop inner(c, C_COND_IN);
        EBV_LAUNCH(c, k_set_cond, dim3(1), dim3(32), 0, c->ctl, C_COND_IN, 1, inner.h, inner.use_h);
        while (inner.next()) {
            const int nd = P.precond32_dot(c, r, z);
            if (!nd) EBV_LAUNCH(c, k_dot32, dim3(vblocks(n)), dim3(256), 0, r, z, n, c->part);
            reduce_sum(c, c->part, nd ? nd : vblocks(n), c->scal + S_RZ);
            EBV_LAUNCH(c, k_cg_pupdate32, dim3(vblocks(n)), dim3(256), 0, p, e, z, c->scal, n, c->ctl);
            P.apply_dot32(c, p, q);
            reduce_sum(c, c->part, P.apply_blocks32(), c->scal + S_PQ);
            EBV_LAUNCH(c, k_cg_update32, dim3(vblocks(n)), dim3(256), 0, r, q, c->scal, n, c->part);
            EBV_LAUNCH(c, k_reduce_inner_check, dim3(1), dim3(1024), 0, c->part, vblocks(n), c->scal, c->ctl, tol,
                       maxit, 1, inner.h, inner.use_h);
        }
        inner_count = inner.body_launches();
        P.add32(c, x, e, p);
        true_residual();
        EBV_LAUNCH(c, k_outer_check, dim3(1), dim3(32), 0, c->scal, c->ctl, tol, maxit, 60, 1, inner_drop,
                   outer.h, outer.use_h);
    }
    if (c->capturing)
        c->loop_recs.push_back({c->cur_slot, outer.body_launches() - inner_count, inner_count});
    if (!c->cap_err.empty() && c->capturing) return c->fail(EBV_ERR_CUDA, "graph capture: " + c->cap_err);
    return finish_solve(c, x, n, iters, res);
}

struct CcProblem : Problem {
    CcHier *H;
    int n() const override { return ncell(H->lv[0].g); }
    // two planes per thread
    dim3 agrid() const { const GridD &g = H->lv[0].g; return grid3(g.nx, g.ny, (g.nz + 1) / 2); }
    int apply_blocks() const override { return nblocks3(agrid()); }
    void apply_dot(Ctx *c, const double *p, double *q) override
    {
        // p, diagonal, 3 faces, q: 6 words per cell
        EBV_LAUNCH_P(c, "cc_apply_fp64", 48.0 * n(), k_cc_apply_dot<double>, agrid(), block3(), 0,
                     ccop<double>(H->lv[0]), p, q, c->part);
    }
    // FP32 levels with nx a multiple of 8 large enough for two blocks per SM:
    // the vectorised apply (its own partials; the choice follows the grid only)
    bool vec32() const
    {
        return gs4_ok(H->lv[0].g) && nblocks3(apply4_grid(H->lv[0].g)) >= kVecMinBlocks;
    }
    int apply_blocks32() const override { return vec32() ? nblocks3(apply4_grid(H->lv[0].g)) : apply_blocks(); }
    void apply_dot32(Ctx *c, const float *p, float *q) override
    {
        if (vec32())
            EBV_LAUNCH_P(c, "cc_apply_fp32", 24.0 * n(), k_cc_apply4, apply4_grid(H->lv[0].g),
                         dim3(kApply4X, kApply4Y, kApply4Z), 0, ccop<float>(H->lv[0]), p, q, c->part);
        else
            EBV_LAUNCH_P(c, "cc_apply_fp32", 24.0 * n(), k_cc_apply_dot<float>, agrid(), block3(), 0,
                         ccop<float>(H->lv[0]), p, q, c->part);
    }
    void precond(Ctx *c, const double *r, double *z) override { cc_vcycle<double>(c, *H, r, z); }
    void precond32(Ctx *c, const float *r, float *z) override { cc_vcycle<float>(c, *H, r, z); }
    int precond32_dot(Ctx *c, const float *r, float *z) override { return cc_vcycle<float>(c, *H, r, z, c->part); }
    void resid32(Ctx *c, const double *b, const double *x, float *r) override
    {
        // x, diagonal, 3 faces, b read, r (FP32) written: 6.5 words per cell
        EBV_LAUNCH_P(c, "cc_resid_fp64", 52.0 * n(), (k_cc_apply_dot<double, true>), agrid(), block3(), 0,
                     ccop<double>(H->lv[0]), x, (double *)nullptr, c->part, b, r, c->scal + S_SIG);
    }
    void add32(Ctx *c, double *x, const float *e, const float *p) override
    {
        EBV_LAUNCH(c, k_add32to64_split, dim3(vblocks(n())), dim3(256), 0, H->lv[0].g, x, e, p, c->scal, c->ctl);
    }
    void to32(Ctx *c, const double *b, float *r) override
    {
        EBV_LAUNCH(c, k_to_split, dim3(vblocks(n())), dim3(256), 0, H->lv[0].g, -1, b, r, c->scal + S_SIG);
    }
};

struct NdProblem : Problem {
    NdHier *H;
    int n() const override { return nnode(H->lv[0].g); }
    int apply_blocks() const override { return nd_tile_parts(H->lv[0]); }
    void apply_dot(Ctx *c, const double *p, double *q) override
    {
        // p read, q written, act and reg flags: 2.25 words per node
        nd_tile_pass<double, ND_APPLY>(c, H->lv[0], "nodal_apply_fp64", 18.0 * n(), p, q, nullptr, nullptr, 0.0, 0.0,
                                       c->part);
    }
    void apply_dot32(Ctx *c, const float *p, float *q) override
    {
        nd_tile_pass<float, ND_APPLY>(c, H->lv[0], "nodal_apply_fp32", 12.0 * n(), p, q, nullptr, nullptr, 0.0f,
                                    0.0f, c->part);
    }
    void precond(Ctx *c, const double *r, double *z) override { nd_vcycle<double>(c, *H, r, z); }
    void precond32(Ctx *c, const float *r, float *z) override { nd_vcycle<float>(c, *H, r, z); }
    void resid32(Ctx *c, const double *b, const double *x, float *r) override
    {
        // x, b read, r (FP32) written, act and reg flags: 5.25 words per node
        nd_tile_pass<double, ND_RES32>(c, H->lv[0], "nodal_resid_fp64", 22.0 * n(), x, nullptr, nullptr, b, 0.0,
                                       0.0, c->part, r, c->scal + S_SIG);
    }
    void add32(Ctx *c, double *x, const float *e, const float *p) override
    {
        EBV_LAUNCH(c, k_add32to64, dim3(vblocks(n())), dim3(256), 0, x, e, p, c->scal, c->ctl, n());
    }
    void to32(Ctx *c, const double *b, float *r) override
    {
        EBV_LAUNCH(c, k_to32_scaled, dim3(vblocks(n())), dim3(256), 0, b, r, n(), c->scal + S_SIG);
    }
};

// x_zero: x holds zeros on entry (lets the refinement solver skip its first
// operator application)
ebv_status solve(Ctx *c, Problem &P, const double *b, double *x, int *iters, double *res, bool x_zero = false)
{
    if (c->prm.precision != EBV_FP64) return pcg_refine(c, P, b, x, iters, res, x_zero);
    return pcg(c, P, b, x, iters, res);
}

// Coarse levels of a cell-centred hierarchy whose level-0 FP64 coefficients
// are set: the diagonals of every variant, in FP32 also the level-0 Krylov
// operator and on every level the V-cycle's BF16 faces with the diagonal (and
// its inverse) formed from them; then the bottom inverses of all variants.
ebv_status cc_finish_hierarchy(Ctx *c, CcHier &H, bool fp32)
{
    CcLevel &L0 = H.lv[0];
    cc_make_diag<double>(c, H, 0);
    if (fp32) {
        // level 0 in FP32: the Krylov operator (the FP64 diagonal rounded),
        // then the V-cycle's BF16 faces and the diagonal formed from them
        const int n = ncell(L0.g);
        EBV_LAUNCH(c, k_to_split, dim3(vblocks(n)), dim3(256), 0, L0.g, -1, L0.extra_d, L0.extra_f);
        for (int q = 0; q < H.nvar; q++)
            EBV_LAUNCH(c, k_to_split, dim3(vblocks(n)), dim3(256), 0, L0.g, -1, H.vdiag_d[q][0], H.vdiag_a[q]);
        for (int d = 0; d < 3; d++)
            EBV_LAUNCH(c, k_to_split, dim3(vblocks(nface(L0.g, d))), dim3(256), 0, L0.g, d, L0.bf_d[d], L0.bf_f[d]);
        cc_faces_bf16(c, L0);
        cc_make_diag<float>(c, H, 0);
    }
    for (int l = 0; l + 1 < H.L; l++) {
        CcLevel &F = H.lv[l], &Cc = H.lv[l + 1];
        dim3 gr = grid3(Cc.g.nx + 1, Cc.g.ny + 1, Cc.g.nz + 1);
        if (fp32) {
            EBV_LAUNCH(c, k_cc_coarsen<float>, gr, block3(), 0, F.g, F.extra_f, F.bf_f[0], F.bf_f[1], F.bf_f[2], F.cov,
                       Cc.g, Cc.cov, Cc.extra_f, Cc.bf_f[0], Cc.bf_f[1], Cc.bf_f[2]);
            cc_faces_bf16(c, Cc);
            cc_make_diag<float>(c, H, l + 1);
        } else {
            EBV_LAUNCH(c, k_cc_coarsen<double>, gr, block3(), 0, F.g, F.extra_d, F.bf_d[0], F.bf_d[1], F.bf_d[2],
                       F.cov, Cc.g, Cc.cov, Cc.extra_d, Cc.bf_d[0], Cc.bf_d[1], Cc.bf_d[2]);
            cc_make_diag<double>(c, H, l + 1);
        }
    }
    const int lb = H.L - 1;
    const size_t msz = (size_t)H.nb * 2 * H.nb;
    for (int q = 0; q < H.nvar; q++) {
        if (fp32) {
            VOp<float> A = vop<float>(H.lv[lb]);
            A.diag = H.vdiag_f[q][lb];
            EBV_LAUNCH(c, k_cc_bottom_assemble<float>, dim3((H.nb + 127) / 128), dim3(128), 0, A, H.bmat + q * msz,
                       H.nb);
        } else {
            VOp<double> A = vop<double>(H.lv[lb]);
            A.diag = H.vdiag_d[q][lb];
            EBV_LAUNCH(c, k_cc_bottom_assemble<double>, dim3((H.nb + 127) / 128), dim3(128), 0, A, H.bmat + q * msz,
                       H.nb);
        }
    }
    EBV_LAUNCH(c, k_gauss_jordan, dim3(H.nvar), dim3(1024), 0, H.bmat, H.nb, H.vbinv[0], H.vbinv[1], H.vbinv[2]);
    select_variant(H, 0);
    return EBV_OK;
}

// Level dimensions: halve while every dimension is even and the level has
// more than 64 cells (cell-centred) / 125 nodes (nodal).
int plan_levels(const GridD &g0, GridD *out, bool nodal)
{
    int L = 0;
    GridD g = g0;
    out[L++] = g;
    while (L < kMaxLevels) {
        long long sz = nodal ? (long long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1) : (long long)g.nx * g.ny * g.nz;
        if (sz <= (nodal ? 125 : 64)) break;
        if ((g.nx & 1) || (g.ny & 1) || (g.nz & 1)) break;
        g.nx /= 2; g.ny /= 2; g.nz /= 2;
        g.h *= 2.0;
        g.ih *= 0.5;
        out[L++] = g;
    }
    return L;
}

template <class T>
T *dalloc(size_t n, cudaError_t &e)
{
    T *p = nullptr;
    cudaError_t r = dev_malloc((void **)&p, n * sizeof(T));
    if (r != cudaSuccess) e = r;
    return p;
}

}  // namespace

// ===========================================================================
// Set-up and public solver entry points
// ===========================================================================

ebv_status setup_solvers(Ctx *c)
{
    const GridD &g = c->g;
    cudaError_t e = cudaSuccess;
    // the staged coarse V-cycle takes up to kCoarseStageMax of dynamic shared memory
    EBV_CUDA_TRY(c, cudaFuncSetAttribute(k_cc_coarse_vcycle<float, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseStageMax));
    EBV_CUDA_TRY(c, cudaFuncSetAttribute(k_cc_coarse_vcycle<double, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseStageMax));
    GridD gl[kMaxLevels];
    // cell-centred hierarchies (projection and viscous)
    int L = plan_levels(g, gl, false);
    long long nbc = (long long)gl[L - 1].nx * gl[L - 1].ny * gl[L - 1].nz;
    if (nbc > kBottomMax) return c->fail(EBV_ERR_INVALID, "grid cannot be coarsened to a small bottom level");
    CcHier *hs[2] = {&c->mac, &c->visc};
    // the projection operator has one variant; the viscous one a variant per
    // velocity component, whose diagonals take the box faces of its Dirichlet sides
    c->mac.nvar = 1;
    c->mac.side_mask[0] = 0x3fu;
    c->visc.nvar = 3;
    for (int q = 0; q < 3; q++) {
        unsigned m = 0;
        double val;
        for (int sd = 0; sd < 6; sd++)
            if (side_dirichlet(g, sd, q, &val)) m |= 1u << sd;
        c->visc.side_mask[q] = m;
    }
    for (CcHier *H : hs) {
        H->L = L;
        H->nb = (int)nbc;
        for (int l = 0; l < L; l++) {
            CcLevel &Lv = H->lv[l];
            Lv.g = gl[l];
            size_t nc = ncell(gl[l]);
            Lv.extra_d = dalloc<double>(nc, e);
            Lv.extra_f = dalloc<float>(nc, e);
            for (int q = 0; q < H->nvar; q++) {
                H->vdiag_d[q][l] = dalloc<double>(nc, e);
                H->vdiag_f[q][l] = dalloc<float>(nc, e);
                H->vdinv_f[q][l] = dalloc<float>(nc, e);
                if (l == 0) H->vdiag_a[q] = dalloc<float>(nc, e);
            }
            for (int d = 0; d < 3; d++) {
                Lv.bf_d[d] = dalloc<double>(nface(gl[l], d), e);
                Lv.bf_f[d] = dalloc<float>(nface(gl[l], d), e);
                // one spare element: the coarse kernel stages BF16 arrays in 4-byte pairs
                Lv.bf_h[d] = dalloc<__nv_bfloat16>(nface(gl[l], d) + 1, e);
            }
            if (rb_fusable(gl[l]))
                Lv.bxp = dalloc<RbF>((size_t)2 * rb_hxp(gl[l].nx) * gl[l].ny * gl[l].nz, e);
            if (H == &c->mac) Lv.cov = dalloc<uint8_t>(nc, e);
            else Lv.cov = c->mac.lv[l].cov;
        }
        for (int q = 0; q < H->nvar; q++) H->vbinv[q] = dalloc<double>((size_t)nbc * nbc, e);
        H->bmat = dalloc<double>((size_t)H->nvar * nbc * 2 * nbc, e);
        select_variant(*H, 0);
    }
    // nodal hierarchy
    GridD gn[kMaxLevels];
    int Ln = plan_levels(g, gn, true);
    long long nbn = (long long)(gn[Ln - 1].nx + 1) * (gn[Ln - 1].ny + 1) * (gn[Ln - 1].nz + 1);
    if (nbn > kBottomMax) return c->fail(EBV_ERR_INVALID, "grid cannot be coarsened to a small nodal bottom");
    c->nd.L = Ln;
    c->nd.nb = (int)nbn;
    for (int l = 0; l < Ln; l++) {
        NdLevel &Lv = c->nd.lv[l];
        Lv.g = gn[l];
        size_t nc = ncell(gn[l]);
        Lv.alpha_d = l ? dalloc<double>(nc, e) : c->alpha;
        Lv.alpha_f = dalloc<float>(nc, e);
        Lv.act = dalloc<uint8_t>(nnode(gn[l]), e);
        // regular-node flags (and the plane march) where the level is large
        // enough to fill the GPU with marching blocks
        Lv.reg = (l == 0 || nnode(gn[l]) >= kTileNodes) ? dalloc<uint8_t>(nnode(gn[l]), e) : nullptr;
        Lv.lam_max = 2.0;
    }
    c->nd.binv = dalloc<double>((size_t)nbn * nbn, e);
    c->nd.bmat = dalloc<double>((size_t)nbn * 2 * nbn, e);
    // level vectors: large enough for nodes of that level (>= cells)
    int Lmax = std::max(L, Ln);
    for (int l = 0; l < Lmax; l++) {
        const GridD &gg = l < Ln ? gn[l] : gl[l];
        size_t m = (size_t)nnode(gg);
        c->lx[l] = dalloc<double>(m, e);
        c->lb[l] = dalloc<double>(m, e);
        c->lr[l] = dalloc<double>(m, e);
        c->ld[l] = dalloc<double>(m, e);
        c->lt[l] = dalloc<double>(m, e);
    }
    if (e != cudaSuccess)
        return c->fail(e == cudaErrorMemoryAllocation ? EBV_ERR_OOM : EBV_ERR_CUDA,
                       std::string("allocation: ") + cudaGetErrorString(e));
    return EBV_OK;
}

// Geometry-dependent solver data: projection coefficients, coverage, nodal
// volume fractions and active nodes, both bottom inverses.
ebv_status autotune_shapes(Ctx *c);

ebv_status setup_geometry_solvers(Ctx *c)
{
    const GridD &g = c->g;
    // coverage per level
    EBV_LAUNCH(c, k_cov_from_flag, dim3(vblocks(ncell(g))), dim3(256), 0, ncell(g), c->flag, c->mac.lv[0].cov);
    for (int l = 0; l + 1 < c->mac.L; l++)
        EBV_LAUNCH(c, k_cov_coarsen, cgrid(c->mac.lv[l + 1].g), block3(), 0, c->mac.lv[l].g, c->mac.lv[l].cov,
                   c->mac.lv[l + 1].g, c->mac.lv[l + 1].cov);
    // projection operator
    CcLevel &M0 = c->mac.lv[0];
    EBV_LAUNCH(c, k_mac_coeffs, grid3(g.nx + 1, g.ny + 1, g.nz + 1), block3(), 0, g, c->flag, c->ax, c->ay, c->az,
               M0.extra_d, M0.bf_d[0], M0.bf_d[1], M0.bf_d[2]);
    // both precisions of the projection hierarchy are kept
    ebv_status s = cc_finish_hierarchy(c, c->mac, false);
    if (s != EBV_OK) return s;
    if (c->prm.precision != EBV_FP64) {
        // FP32 levels derived from FP64 fine coefficients; the bottom inverse
        // from the FP32 coarse operator
        s = cc_finish_hierarchy(c, c->mac, true);
        if (s != EBV_OK) return s;
    }
    // nodal
    NdHier &N = c->nd;
    for (int l = 0; l < N.L; l++) {
        NdLevel &Lv = N.lv[l];
        if (l) EBV_LAUNCH(c, k_nd_alpha_coarsen, cgrid(Lv.g), block3(), 0, N.lv[l - 1].g, N.lv[l - 1].alpha_d, Lv.g,
                          Lv.alpha_d);
        int nc = ncell(Lv.g);
        EBV_LAUNCH(c, (k_convert<double, float>), dim3(vblocks(nc)), dim3(256), 0, Lv.alpha_d, Lv.alpha_f, nc);
        EBV_LAUNCH(c, k_nd_active, ngrid(Lv.g), block3(), 0, Lv.g, Lv.alpha_d, Lv.act);
        if (Lv.reg) EBV_LAUNCH(c, k_nd_regular, ngrid(Lv.g), block3(), 0, Lv.g, Lv.alpha_d, Lv.reg);
    }
    for (int l = 0; l < N.L; l++) {
        // levels with regular-node flags: the active nodes that are not
        // regular, in ascending order, for the listed half of their passes
        NdLevel &Lv = N.lv[l];
        if (!Lv.reg) continue;
        const int nn = nnode(Lv.g);
        std::vector<uint8_t> act(nn), reg(nn);
        EBV_CUDA_TRY(c, cudaMemcpyAsync(act.data(), Lv.act, nn, cudaMemcpyDeviceToHost, c->stream));
        EBV_CUDA_TRY(c, cudaMemcpyAsync(reg.data(), Lv.reg, nn, cudaMemcpyDeviceToHost, c->stream));
        EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        std::vector<int> irr;
        for (int n = 0; n < nn; n++)
            if (act[n] && !reg[n]) irr.push_back(n);
        if (Lv.irr) cudaFree(Lv.irr);
        Lv.irr = nullptr;
        Lv.nirr = (int)irr.size();
        if (Lv.nirr) {
            EBV_CUDA_TRY(c, dev_malloc((void **)&Lv.irr, irr.size() * sizeof(int)));
            EBV_CUDA_TRY(c, cudaMemcpy(Lv.irr, irr.data(), irr.size() * sizeof(int), cudaMemcpyHostToDevice));
        }
    }
    const NdLevel &B = N.lv[N.L - 1];
    EBV_LAUNCH(c, k_nd_bottom_assemble, dim3((N.nb + 127) / 128), dim3(128), 0, B.g, B.alpha_d, B.act, N.bmat, N.nb);
    EBV_LAUNCH(c, k_gauss_jordan, dim3(1), dim3(1024), 0, N.bmat, N.nb, N.binv, (double *)nullptr,
               (double *)nullptr);
    EBV_CUDA_TRY(c, cudaGetLastError());
    return autotune_shapes(c);
}

// Launch-shape autotuner.  For every level it times each candidate block
// shape of the colour pass (on the projection operator) and of the nodal
// Chebyshev step, on zeroed scratch vectors in the precision the solves
// use, and keeps the fastest; the viscous hierarchy shares the shapes of the
// projection hierarchy (same level sizes).  The smoothers' results do not
// depend on the shape: every update of a pass reads only values that the
// pass does not write (the one pass that also sums r.z keeps the default
// shape, so its partial sums are grouped the same way).
template <class T>
ebv_status autotune_shapes_t(Ctx *c)
{
    static const dim3 cand[] = {dim3(32, 4, 2), dim3(32, 8, 1), dim3(32, 2, 4), dim3(16, 8, 2),
                                dim3(64, 4, 1), dim3(64, 2, 2), dim3(16, 16, 1), dim3(128, 2, 1)};
    const int nc = (int)(sizeof(cand) / sizeof(cand[0]));
    T *x = (T *)(sizeof(T) == 4 ? (void *)c->kz32 : (void *)c->kz);
    T *y = (T *)(sizeof(T) == 4 ? (void *)c->kp32 : (void *)c->kp);
    T *d = (T *)(sizeof(T) == 4 ? (void *)c->kq32 : (void *)c->kq);
    T *b = (T *)(sizeof(T) == 4 ? (void *)c->kr32 : (void *)c->kr);
    for (T *v : {x, y, d, b}) EBV_CUDA_TRY(c, cudaMemsetAsync(v, 0, c->vec_len * sizeof(T), c->stream));
    cudaEvent_t e0, e1;
    EBV_CUDA_TRY(c, cudaEventCreate(&e0));
    EBV_CUDA_TRY(c, cudaEventCreate(&e1));
    auto time_it = [&](auto launch) -> float {
        launch();
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 4; r++) launch();
        cudaEventRecord(e1, c->stream);
        float ms = 1e30f;
        if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    for (int l = 0; l < c->mac.L; l++) {
        CcLevel &L = c->mac.lv[l];
        VOp<T> A = vop<T>(L);
        float best = 1e30f;
        for (int q = 0; q < nc; q++) {
            const dim3 bk = cand[q], gr = gs_grid(L.g, bk);
            float ms = time_it([&]() { k_cc_gs<T, false><<<gr, bk, 0, c->stream>>>(A, x, b, 0, 0, nullptr, GridD()); });
            if (ms < best) { best = ms; L.gs_blk = bk; }
        }
        c->visc.lv[l].gs_blk = L.gs_blk;
        if constexpr (sizeof(T) == 4) {
            // the vectorised pass: a thread covers 4 cells of a half-row, so
            // narrow blocks suit the levels whose rows are short
            static const dim3 c4[] = {dim3(32, 4, 2), dim3(32, 8, 1), dim3(16, 8, 2), dim3(16, 16, 1),
                                      dim3(8, 16, 2), dim3(8, 32, 1), dim3(4, 32, 2), dim3(4, 16, 4)};
            if (gs4_ok(L.g)) {
                float best4 = 1e30f;
                for (int pz = 1; pz <= 2; pz++)
                    for (const dim3 &bk : c4) {
                        if (bk.x > 2 * (unsigned)((L.g.nx >> 3) + 1)) continue;   // no block wider than twice a row
                        float ms = time_it([&]() { launch_gs4(c->stream, bk, pz, A, x, b, 0, 0); });
                        if (ms < best4) { best4 = ms; L.gs4_blk = bk; L.gs4_pz = pz; }
                    }
                c->visc.lv[l].gs4_blk = L.gs4_blk;
                c->visc.lv[l].gs4_pz = L.gs4_pz;
            }
            // the fused one-pass sweep against its two colour passes (same
            // results), per kind of sweep: the faster serves it in switch mode 1
            RbMaps m;
            for (int q = 0; q < 4; q++) L.rb_ms[q][0] = 1e30f, L.rb_ms[q][1] = 0.f;
            if (!c->batched && rb_fusable(L.g) && gs4_ok(L.g) && rb_map(c, x, 0, L.g, &m.x) && rb_map(c, b, 1, L.g, &m.b) &&
                rb_map(c, A.dinv, 1, L.g, &m.d) && rb_map(c, L.bxp, 4, L.g, &m.fx) && rb_map(c, A.by, 2, L.g, &m.fy) &&
                rb_map(c, A.bz, 3, L.g, &m.fz)) {
                const long long nl = c->launches;
                // planes per block: the model's choice, the most planes that
                // still fill one wave, and half that (results do not depend on it)
                const int nt = rb_ntiles(L.g), res = rb_resident(), nz = L.g.nz;
                const int one = std::max(1, res / std::max(1, nt));   // chunks per wave
                const int kzc[3] = {rb_kz(L.g), (nz + one - 1) / one, (nz + 2 * one - 1) / (2 * one)};
                float best = 1e30f;
                for (int kz : kzc) {
                    const float ms = time_it(
                        [&]() { rb_launch(c, "autotune", L.g, m, y, 0, RB_PLAIN, nullptr, kz); });
                    if (ms < best) { best = ms; L.rb_kz = kz; }
                }
                // the correction sweep reads a coarse array: a zeroed vector with the next level's dims
                const bool has_c = l + 1 < c->mac.L;
                const GridD gc = has_c ? c->mac.lv[l + 1].g : GridD();
                const dim3 gt((L.g.nx / 2 + RB_HW - 1) / RB_HW, (L.g.ny + RB_TY - 1) / RB_TY,
                              (L.g.nz + kGs2Planes - 1) / kGs2Planes);
                const dim3 bk = L.gs_blk, grc = gs_grid(L.g, bk);
                for (int kind = 0; kind < 4; kind++) {
                    if (kind == RB_CORR && !has_c) continue;   // (no correction sweep on the last level)
                    RbMaps mk = m;
                    mk.xc = m.b;
                    if (kind == RB_CORR && !rb_map(c, d, 5, gc, &mk.xc)) continue;
                    const float ms_f = time_it([&]() {
                        rb_launch(c, "autotune", L.g, mk, y, 0, kind, kind == RB_DOT ? c->part : nullptr, L.rb_kz);
                    });
                    const float ms_p = time_it([&]() {
                        if (kind == RB_CORR) {
                            if (L.gs4_pz == 1)
                                k_cc_gs4<1, true><<<gs4_grid(L.g, L.gs4_blk, 1), L.gs4_blk, 0, c->stream>>>(A, x, b, 0, 0, d, gc);
                            else
                                k_cc_gs4<2, true><<<gs4_grid(L.g, L.gs4_blk, 2), L.gs4_blk, 0, c->stream>>>(A, x, b, 0, 0, d, gc);
                        }
                        else
                            launch_gs4(c->stream, L.gs4_blk, L.gs4_pz, A, x, b, 0, kind == RB_ZERO ? 1 : 0);
                        if (kind == RB_DOT) k_cc_gs2_dot<<<gt, RB_THREADS, 0, c->stream>>>(A, x, b, 1, c->part);
                        else launch_gs4(c->stream, L.gs4_blk, L.gs4_pz, A, x, b, 1, 0);
                    });
                    L.rb_ms[kind][0] = ms_f;
                    L.rb_ms[kind][1] = ms_p;
                }
                c->launches = nl;
            }
            for (int q = 0; q < 4; q++) c->visc.lv[l].rb_ms[q][0] = L.rb_ms[q][0], c->visc.lv[l].rb_ms[q][1] = L.rb_ms[q][1];
            c->visc.lv[l].rb_kz = L.rb_kz;
        }
    }
    ChebCoef k = cheb_coef(2.0);
    for (int l = 0; l < c->nd.L; l++) {
        NdLevel &L = c->nd.lv[l];
        NdOp<T> A = ndop<T>(L);
        float best = 1e30f;
        for (int q = 0; q < nc; q++) {
            const dim3 bk = cand[q], gr = ch_grid(L.g, bk);
            float ms = time_it([&]() {
                k_nd_cheb<T><<<gr, bk, 0, c->stream>>>(A, x, y, d, b, (T)k.cd[1], (T)k.cr[1], 0);
            });
            if (ms < best) { best = ms; L.ch_blk = bk; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    EBV_CUDA_TRY(c, cudaGetLastError());
    return EBV_OK;
}

ebv_status autotune_shapes(Ctx *c)
{
    return c->prm.precision != EBV_FP64 ? autotune_shapes_t<float>(c) : autotune_shapes_t<double>(c);
}

ebv_status mac_solve(Ctx *c, const double *b, double *x, int *iters, double *res)
{
    CcProblem P;
    P.H = &c->mac;
    EBV_LAUNCH(c, k_fill, dim3(vblocks(ncell(c->g))), dim3(256), 0, x, ncell(c->g), 0.0);
    return solve(c, P, b, x, iters, res, true);
}

ebv_status visc_build(Ctx *c, const double *eta)
{
    const GridD &g = c->g;
    CcLevel &V0 = c->visc.lv[0];
    EBV_LAUNCH(c, k_visc_coeffs, grid3(g.nx + 1, g.ny + 1, g.nz + 1), block3(), 0, g, geomd(c), paramsd(c->prm), eta,
               c->dt_dev, V0.extra_d, V0.bf_d[0], V0.bf_d[1], V0.bf_d[2]);
    return cc_finish_hierarchy(c, c->visc, c->prm.precision != EBV_FP64);
}

ebv_status visc_solve(Ctx *c, const double *psi_comp, int comp, double *x, int *iters, double *res)
{
    const GridD &g = c->g;
    CcLevel &V0 = c->visc.lv[0];
    EBV_LAUNCH(c, k_visc_rhs, cgrid(g), block3(), 0, g, geomd(c), comp, psi_comp, V0.bf_d[0], V0.bf_d[1],
               V0.bf_d[2], c->rhs_c);
    select_variant(c->visc, comp);
    CcProblem P;
    P.H = &c->visc;
    return solve(c, P, c->rhs_c, x, iters, res);
}

ebv_status visc_solve_rhs(Ctx *c, int comp, const double *rhs, double *x, int *iters, double *res)
{
    const int n = ncell(c->g);
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->rhs_c, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    select_variant(c->visc, comp);
    EBV_LAUNCH(c, k_fill, dim3(vblocks(n)), dim3(256), 0, x, n, 0.0);
    CcProblem P;
    P.H = &c->visc;
    return solve(c, P, c->rhs_c, x, iters, res, true);
}

ebv_status nodal_solve(Ctx *c, const double *b, double *x, int *iters, double *res)
{
    const int nn = nnode(c->g);
    EBV_LAUNCH(c, k_zero_inactive, dim3(vblocks(nn)), dim3(256), 0, nn, c->nd.lv[0].act, x);
    NdProblem P;
    P.H = &c->nd;
    return solve(c, P, b, x, iters, res);
}


// ---- process-wide switches and the TMA encoder --------------------------
namespace {
long long g_spin = kSpinDefault;
int g_fused = 1;
double g_inner_drop = kInnerDropDefault;
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
}  // namespace
long long spin_limit() { return g_spin; }
int fused_sweep_mode() { return g_fused; }
void set_spin_limit(long long cycles) { g_spin = cycles < 0 ? kSpinDefault : cycles; }
void set_fused_sweep(int mode) { g_fused = mode < 0 ? 0 : (mode > 2 ? 2 : mode); }
double refine_inner_drop() { return g_inner_drop; }
void set_inner_drop(double drop) { g_inner_drop = (drop > 0.0 && drop < 1.0) ? drop : kInnerDropDefault; }

bool tma_encode_4d(CUtensorMap *tm, CUtensorMapDataType type, void *base, const uint64_t dims[4],
                   const uint64_t strides[3], const uint32_t box[4])
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess && f)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        else
            cudaGetLastError();
    }
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    const cuuint64_t d[4] = {dims[0], dims[1], dims[2], dims[3]};
    const cuuint64_t st[3] = {strides[0], strides[1], strides[2]};
    const cuuint32_t bx[4] = {box[0], box[1], box[2], box[3]};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(tm, type, 4, base, d, st, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace ebv
