/*
 * ebv_oracle.cpp -- TEST INFRASTRUCTURE ONLY (see ebv_oracle.h).
 *
 * A plain FP64 restatement of the embedded-boundary (EB) viscoplastic flow
 * step of Sverdrup, Almgren & Nikiforakis (arXiv:1905.07392), written for a
 * reader who checks it against the paper: no blocking, no fusion, loops in the
 * order of the equations.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark load it.
 *
 * Passages followed (paper section / equation / algorithm):
 *   - EB geometry: Sec. "Embedded boundaries" (flags, alpha, normal into the
 *     fluid, face apertures, EB centroid), planar cut per cell.
 *   - Strain rate, its norm and eta: Sec. "Governing partial differential
 *     equations" (gamma = grad u + grad u^T, ||g|| = sqrt(tr(g g^T)/2)),
 *     Table "Generalised Newtonian fluid models", Sec. "Strain rate tensor and
 *     apparent viscosity" (central / one-sided quadratic differences).
 *   - Time step: Eqs. cfl:dt, cfl:convective, cfl:forcing, cfl:viscous:new.
 *   - Algorithm 1 (Advance) and Algorithm 2 (DerivedQuantities).
 *   - Cell-centred projection: Eq. helmholtz and the Poisson equation after it.
 *   - Flux divergence: Eqs. divergence_conservative ... divergence_final.
 *   - Viscous wall flux: Eqs. interpolation_distances, dudn; Appendix A.
 *   - Semi-implicit viscous update: Eq. implicit-viscous.
 *   - Nodal projection: Sec. "Incompressibility constraint".
 *   - Drag: Eq. drag-force; yield criterion ||tau|| <= (1 + delta) tau0.
 * Where the paper is silent this oracle reads it as: a face-centred EB
 * operator, an alpha-weighted trilinear nodal operator, the MC limiter, the
 * upwind rule, a lower bound of the wall distance, and fallbacks of the wall
 * gradient when its stencil leaves the fluid.
 *
 * Scalar type.  Every function that carries flow quantities (velocity,
 * pressure, viscosity and the operators built from them) is a template on its
 * scalar R.  R = double is the oracle; R = Dual (og_dual.h) runs the same
 * code in forward-mode dual numbers and gives exact directional derivatives
 * (og_drag_tangent).  The geometry is always double.  A linear solve in dual
 * numbers solves for the value part and then, with the same operator, for the
 * derivative part (the derivative of A x = b is A x' = b' - A' x).
 *
 * Threads.  Loops over cells, faces and nodes run in OpenMP threads; each
 * iteration writes only its own entries, so the results do not depend on the
 * thread count.  Sums (dot products, drag) add fixed chunks in a fixed order,
 * also independent of the thread count.
 *
 * og_drag is pinned in both parts: the pressure part by the buoyancy
 * identity, the viscous traction by plane walls in a Newtonian shear or
 * extension flow, where Eq. dudn is exact.  The convective term is pinned by
 * linear, step and quadratic fields, conservation, and the cut-cell flux of a
 * uniform state; the rheologies by their closed values.
 */
#include "ebv_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <functional>
#include <vector>

#include "og_dual.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#define NX (g->n[0])
#define NY (g->n[1])
#define NZ (g->n[2])

namespace {

using std::vector;

template <class R>
struct Par {  // og_params with the differentiable parameters in R
    R rho, mu, tau0, m, n_flow, eta0;
    int model;
    double cfl, bi_cfl, tol;
    int max_iters;
    double delta_min;
    int advect;
};

template <class R>
Par<R> par_of(const og_params *p)
{
    Par<R> q;
    q.rho = p->rho; q.mu = p->mu; q.tau0 = p->tau0; q.m = p->m; q.n_flow = p->n_flow; q.eta0 = p->eta0;
    q.model = p->model; q.cfl = p->cfl; q.bi_cfl = p->bi_cfl; q.tol = p->tol;
    q.max_iters = p->max_iters; q.delta_min = p->delta_min; q.advect = p->advect;
    return q;
}

size_t cidx(const og_grid *g, int i, int j, int k) { return ((size_t)k * NY + j) * NX + i; }
size_t nidx(const og_grid *g, int i, int j, int k) { return ((size_t)k * (NY + 1) + j) * (NX + 1) + i; }
/* Face with normal d whose low corner has integer position (i,j,k); along d
 * the index runs 0..n[d]. */
size_t fidx(const og_grid *g, int d, int i, int j, int k)
{
    if (d == 0) return ((size_t)k * NY + j) * (NX + 1) + i;
    if (d == 1) return ((size_t)k * (NY + 1) + j) * NX + i;
    return ((size_t)k * NY + j) * NX + i;
}
size_t nface(const og_grid *g, int d)
{
    size_t m = 1;
    for (int e = 0; e < 3; e++) m *= (size_t)(g->n[e] + (e == d));
    return m;
}
const double *farr(const og_geom *geo, int d) { return d == 0 ? geo->ax : (d == 1 ? geo->ay : geo->az); }
int inside(const og_grid *g, int i, int j, int k)
{
    return i >= 0 && j >= 0 && k >= 0 && i < NX && j < NY && k < NZ;
}
/* A cell whose value may enter a stencil: inside the box and not covered. */
int avail(const og_grid *g, const og_geom *geo, int i, int j, int k)
{
    return inside(g, i, j, k) && geo->alpha[cidx(g, i, j, k)] > 0.0;
}

/* Sum of a[q] b[q] over q < n in 256 fixed chunks, added in chunk order. */
template <class R>
R dot(const R *a, const R *b, size_t n)
{
    const long nch = 256;
    vector<R> part(nch);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < nch; c++) {
        size_t lo = n * (size_t)c / nch, hi = n * (size_t)(c + 1) / nch;
        R s = 0.0;
        for (size_t q = lo; q < hi; q++) s += a[q] * b[q];
        part[c] = s;
    }
    R s = 0.0;
    for (long c = 0; c < nch; c++) s += part[c];
    return s;
}

}  // namespace

extern "C" size_t og_ncell(const og_grid *g) { return (size_t)NX * NY * NZ; }
extern "C" size_t og_nnode(const og_grid *g) { return (size_t)(NX + 1) * (NY + 1) * (NZ + 1); }

/* Threads the oracle's loops run on (1 without OpenMP). */
extern "C" int og_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Geometry (double only)                                                    */
/* ------------------------------------------------------------------------ */

extern "C" double og_phi(const og_shape *s, const double x[3])
{
    if (s->kind == OG_SHAPE_SPHERE) {
        double dx = x[0] - s->p[0], dy = x[1] - s->p[1], dz = x[2] - s->p[2];
        return sqrt(dx * dx + dy * dy + dz * dz) - s->p[3];
    }
    if (s->kind == OG_SHAPE_PLANE) return s->p[0] * x[0] + s->p[1] * x[1] + s->p[2] * x[2] - s->p[3];
    if (s->kind == OG_SHAPE_UNION) {
        /* outside every body: the smallest of the bodies' functions */
        double v = 1e300;
        for (int b = 0; b < s->nbody; b++) {
            const double *q = s->bq[b];
            double w;
            if (s->bkind[b] == OG_BODY_SPHERE) {
                w = sqrt((x[0] - q[0]) * (x[0] - q[0]) + (x[1] - q[1]) * (x[1] - q[1]) +
                         (x[2] - q[2]) * (x[2] - q[2])) - q[3];
            } else if (s->bkind[b] == OG_BODY_BOX) {
                /* signed distance to the box: outside, the distance to its
                 * nearest point; inside, minus the distance to its surface */
                double o2 = 0.0, in = -1e300;
                for (int d = 0; d < 3; d++) {
                    double below = q[d] - x[d], above = x[d] - q[3 + d];
                    double gap = below > above ? below : above;
                    if (gap > 0.0) o2 += gap * gap;
                    if (gap > in) in = gap;
                }
                w = sqrt(o2) + (in < 0.0 ? in : 0.0);
            } else {
                int ax = (int)q[0], a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
                w = sqrt((x[a1] - q[1]) * (x[a1] - q[1]) + (x[a2] - q[2]) * (x[a2] - q[2])) - q[3];
            }
            if (w < v) v = w;
        }
        return v;
    }
    return 1.0;
}

namespace {

int is_fluid(double phi) { return phi > 0.0; }

/* Point on the segment P->Q where phi changes sign, by bisection. */
void edge_root(const og_shape *s, const double P[3], const double Q[3], double out[3])
{
    double x[3], a = 0.0, b = 1.0;
    int fa = is_fluid(og_phi(s, P));
    for (int it = 0; it < 200 && b - a > 1e-16; it++) {
        double m = 0.5 * (a + b);
        for (int d = 0; d < 3; d++) x[d] = P[d] + m * (Q[d] - P[d]);
        if (is_fluid(og_phi(s, x)) == fa) a = m; else b = m;
    }
    double t = 0.5 * (a + b);
    for (int d = 0; d < 3; d++) out[d] = P[d] + t * (Q[d] - P[d]);
}

void node_pos(const og_grid *g, int i, int j, int k, double x[3])
{
    x[0] = g->lo[0] + i * g->h;
    x[1] = g->lo[1] + j * g->h;
    x[2] = g->lo[2] + k * g->h;
}

/* Fluid aperture of one face: the polygon made of the fluid corners and the
 * edge crossings, walked around the square; area by the shoelace formula. */
double face_fraction(const og_grid *g, const og_shape *s, int d, int i, int j, int k)
{
    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    static const int cu[4] = {0, 1, 1, 0}, cv[4] = {0, 0, 1, 1};
    double X[4][3];
    int fl[4], nfl = 0;
    for (int c = 0; c < 4; c++) {
        int id[3] = {i, j, k};
        id[t1] += cu[c];
        id[t2] += cv[c];
        node_pos(g, id[0], id[1], id[2], X[c]);
        fl[c] = is_fluid(og_phi(s, X[c]));
        nfl += fl[c];
    }
    if (nfl == 4) return 1.0;
    if (nfl == 0) return 0.0;
    double pu[8], pv[8];
    int np = 0;
    for (int c = 0; c < 4; c++) {
        int c2 = (c + 1) % 4;
        if (fl[c]) { pu[np] = cu[c]; pv[np] = cv[c]; np++; }
        if (fl[c] != fl[c2]) {
            double r[3];
            edge_root(s, X[c], X[c2], r);
            double o[3];
            node_pos(g, i, j, k, o);
            pu[np] = (r[t1] - o[t1]) / g->h;
            pv[np] = (r[t2] - o[t2]) / g->h;
            np++;
        }
    }
    double a2 = 0.0;
    for (int q = 0; q < np; q++) {
        int q2 = (q + 1) % np;
        a2 += pu[q] * pv[q2] - pu[q2] * pv[q];
    }
    double a = 0.5 * fabs(a2);
    if (a < 1e-12) a = 0.0;
    if (a > 1.0 - 1e-12) a = 1.0;
    return a;
}

struct og_pt {
    double ang;
    double p[3];
};
int cmp_pt(const void *a, const void *b)
{
    double x = ((const og_pt *)a)->ang, y = ((const og_pt *)b)->ang;
    return (x > y) - (x < y);
}

}  // namespace

extern "C" void og_build_geometry(const og_grid *g, const og_shape *s, og_geom *geo)
{
    const double h = g->h;
    for (int d = 0; d < 3; d++) {
        double *a = (double *)farr(geo, d);
        int m[3] = {NX, NY, NZ};
        m[d] += 1;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) a[fidx(g, d, i, j, k)] = face_fraction(g, s, d, i, j, k);
    }
    size_t N3 = og_ncell(g);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                double X[2][2][2][3];
                int fl[2][2][2], nfl = 0;
                for (int c2 = 0; c2 < 2; c2++)
                    for (int b2 = 0; b2 < 2; b2++)
                        for (int a2 = 0; a2 < 2; a2++) {
                            node_pos(g, i + a2, j + b2, k + c2, X[a2][b2][c2]);
                            fl[a2][b2][c2] = is_fluid(og_phi(s, X[a2][b2][c2]));
                            nfl += fl[a2][b2][c2];
                        }
                for (int d = 0; d < 3; d++) {
                    geo->nrm[d * N3 + c] = 0.0;
                    geo->bcen[d * N3 + c] = 0.0;
                }
                geo->area[c] = 0.0;
                if (nfl == 8) { geo->alpha[c] = 1.0; geo->flag[c] = 1; continue; }
                if (nfl == 0) { geo->alpha[c] = 0.0; geo->flag[c] = 0; continue; }
                /* EB area vector by closure of the fluid region's boundary. */
                double alo[3], ahi[3], An[3], suma = 0.0;
                for (int d = 0; d < 3; d++) {
                    int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                    hi[d] += 1;
                    alo[d] = farr(geo, d)[fidx(g, d, lo[0], lo[1], lo[2])];
                    ahi[d] = farr(geo, d)[fidx(g, d, hi[0], hi[1], hi[2])];
                    An[d] = ahi[d] - alo[d];
                    suma += alo[d] + ahi[d];
                }
                double A = sqrt(An[0] * An[0] + An[1] * An[1] + An[2] * An[2]);
                if (A < 1e-12) {
                    /* The cut only touches the cell: it is full or empty. */
                    if (suma > 3.0) { geo->alpha[c] = 1.0; geo->flag[c] = 1; }
                    else { geo->alpha[c] = 0.0; geo->flag[c] = 0; }
                    continue;
                }
                double n[3] = {An[0] / A, An[1] / A, An[2] / A};
                /* Crossings on the 12 edges, relative to the cell centre, in h. */
                og_pt P[12];
                int np = 0;
                double cc[3] = {g->lo[0] + (i + 0.5) * h, g->lo[1] + (j + 0.5) * h, g->lo[2] + (k + 0.5) * h};
                for (int d = 0; d < 3; d++) {
                    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
                    for (int q1 = 0; q1 < 2; q1++)
                        for (int q2 = 0; q2 < 2; q2++) {
                            int o0[3] = {0, 0, 0}, o1[3];
                            o0[t1] = q1;
                            o0[t2] = q2;
                            memcpy(o1, o0, sizeof o1);
                            o1[d] = 1;
                            if (fl[o0[0]][o0[1]][o0[2]] == fl[o1[0]][o1[1]][o1[2]]) continue;
                            double r[3];
                            edge_root(s, X[o0[0]][o0[1]][o0[2]], X[o1[0]][o1[1]][o1[2]], r);
                            for (int e = 0; e < 3; e++) P[np].p[e] = (r[e] - cc[e]) / h;
                            np++;
                        }
                }
                /* Area centroid of the crossing polygon, seen along n. */
                double M[3] = {0, 0, 0};
                for (int q = 0; q < np; q++)
                    for (int e = 0; e < 3; e++) M[e] += P[q].p[e] / np;
                double e1[3], e2[3];
                {
                    double t[3] = {0, 0, 0};
                    int amin = 0;
                    for (int e = 1; e < 3; e++)
                        if (fabs(n[e]) < fabs(n[amin])) amin = e;
                    t[amin] = 1.0;
                    double tn = t[0] * n[0] + t[1] * n[1] + t[2] * n[2];
                    for (int e = 0; e < 3; e++) e1[e] = t[e] - tn * n[e];
                    double l = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
                    for (int e = 0; e < 3; e++) e1[e] /= l;
                    e2[0] = n[1] * e1[2] - n[2] * e1[1];
                    e2[1] = n[2] * e1[0] - n[0] * e1[2];
                    e2[2] = n[0] * e1[1] - n[1] * e1[0];
                }
                for (int q = 0; q < np; q++) {
                    double x = 0, y = 0;
                    for (int e = 0; e < 3; e++) {
                        x += (P[q].p[e] - M[e]) * e1[e];
                        y += (P[q].p[e] - M[e]) * e2[e];
                    }
                    P[q].ang = atan2(y, x);
                }
                qsort(P, np, sizeof(og_pt), cmp_pt);
                /* Fan of triangles (M, P_q, P_q+1) around the vertex mean, so
                 * the result does not depend on where the cycle starts. */
                double bw = 0.0, bsum[3] = {0, 0, 0};
                for (int q = 0; q < np; q++) {
                    int q2 = (q + 1) % np;
                    double u1[3], u2[3], cr[3];
                    for (int e = 0; e < 3; e++) {
                        u1[e] = P[q].p[e] - M[e];
                        u2[e] = P[q2].p[e] - M[e];
                    }
                    cr[0] = u1[1] * u2[2] - u1[2] * u2[1];
                    cr[1] = u1[2] * u2[0] - u1[0] * u2[2];
                    cr[2] = u1[0] * u2[1] - u1[1] * u2[0];
                    double w = 0.5 * (cr[0] * n[0] + cr[1] * n[1] + cr[2] * n[2]);
                    for (int e = 0; e < 3; e++) bsum[e] += w * (M[e] + P[q].p[e] + P[q2].p[e]) / 3.0;
                    bw += w;
                }
                double b[3];
                for (int e = 0; e < 3; e++) b[e] = fabs(bw) > 1e-300 ? bsum[e] / bw : M[e];
                /* Volume by the divergence theorem: each axis face sits at
                 * distance 1/2 from the centre, the EB plane passes through b. */
                double alpha = (0.5 * suma - A * (b[0] * n[0] + b[1] * n[1] + b[2] * n[2])) / 3.0;
                if (alpha < 1e-12) alpha = 0.0;
                if (alpha > 1.0 - 1e-12) alpha = 1.0;
                geo->alpha[c] = alpha;
                geo->flag[c] = alpha > 0.0 ? 2 : 0;
                if (alpha > 0.0) {
                    geo->area[c] = A;
                    for (int e = 0; e < 3; e++) {
                        geo->nrm[e * N3 + c] = n[e];
                        geo->bcen[e * N3 + c] = b[e];
                    }
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Strain rate and apparent viscosity                                        */
/* ------------------------------------------------------------------------ */

namespace {

template <class R>
R eta_of(const Par<R> &p, const R &sr)
{
    /* (1 - exp(-sr*m)) / sr, with its limit m at sr = 0. */
    R yield = (sr > 0.0) ? -expm1(-p.m * sr) / sr : p.m;
    R floor_ = 1.0 / p.m;
    R srf = sr > floor_ ? sr : floor_;
    switch (p.model) {
    case OG_NEWTONIAN: return p.mu;
    case OG_BINGHAM: return p.mu + p.tau0 * yield;
    case OG_HB: return p.mu * pow(srf, p.n_flow - 1.0) + p.tau0 * yield;
    case OG_POWERLAW: return p.mu * pow(srf, p.n_flow - 1.0);
    case OG_SMD: {
        R y2 = (sr > 0.0) ? -expm1(-p.eta0 * sr / p.tau0) / sr : p.eta0 / p.tau0;
        return p.mu * pow(srf, p.n_flow - 1.0) + p.tau0 * y2;
    }
    }
    return p.mu;
}

/* du/dx_d at a cell from cell values, following the robust stencils:
 * central when both neighbours exist, the one-sided quadratic when one side
 * is missing, first order if only one neighbour exists, zero otherwise. */
template <class R>
R d_cell(const og_grid *g, const og_geom *geo, const R *f, int i, int j, int k, int d)
{
    int e[3] = {0, 0, 0};
    e[d] = 1;
    double h = g->h;
    int ip = avail(g, geo, i + e[0], j + e[1], k + e[2]);
    int im = avail(g, geo, i - e[0], j - e[1], k - e[2]);
    R f0 = f[cidx(g, i, j, k)];
    if (ip && im)
        return (f[cidx(g, i + e[0], j + e[1], k + e[2])] - f[cidx(g, i - e[0], j - e[1], k - e[2])]) / (2.0 * h);
    if (im) {
        R f1 = f[cidx(g, i - e[0], j - e[1], k - e[2])];
        if (avail(g, geo, i - 2 * e[0], j - 2 * e[1], k - 2 * e[2])) {
            R f2 = f[cidx(g, i - 2 * e[0], j - 2 * e[1], k - 2 * e[2])];
            return (0.5 * f2 - 2.0 * f1 + 1.5 * f0) / h;
        }
        return (f0 - f1) / h;
    }
    if (ip) {
        R f1 = f[cidx(g, i + e[0], j + e[1], k + e[2])];
        if (avail(g, geo, i + 2 * e[0], j + 2 * e[1], k + 2 * e[2])) {
            R f2 = f[cidx(g, i + 2 * e[0], j + 2 * e[1], k + 2 * e[2])];
            return (-1.5 * f0 + 2.0 * f1 - 0.5 * f2) / h;
        }
        return (f1 - f0) / h;
    }
    return 0.0;
}

template <class R>
void cell_gradient(const og_grid *g, const og_geom *geo, const R *u, R *grad)
{
    size_t N3 = og_ncell(g);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                for (int d = 0; d < 3; d++)
                    for (int q = 0; q < 3; q++)
                        grad[(3 * d + q) * N3 + c] =
                            geo->alpha[c] > 0.0 ? d_cell(g, geo, u + q * N3, i, j, k, d) : R(0.0);
            }
}

template <class R>
void strain_eta(const og_grid *g, const og_geom *geo, const Par<R> &p, const R *u, R *eta, R *srate)
{
    size_t N3 = og_ncell(g);
    vector<R> G(9 * N3);
    cell_gradient(g, geo, u, G.data());
#pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)N3; c++) {
        if (geo->alpha[c] <= 0.0) {
            eta[c] = 0.0;
            if (srate) srate[c] = 0.0;
            continue;
        }
        R s2 = 0.0;
        for (int d = 0; d < 3; d++)
            for (int q = 0; q < 3; q++) {
                R gam = G[(3 * d + q) * N3 + c] + G[(3 * q + d) * N3 + c];
                s2 += gam * gam;
            }
        R sr = sqrt(0.5 * s2);
        eta[c] = eta_of(p, sr);
        if (srate) srate[c] = sr;
    }
}

/* ------------------------------------------------------------------------ */
/* Generic cell-centred operator and its CG solver                           */
/* ------------------------------------------------------------------------ */

template <class R>
const R *barr(int d, const R *bx, const R *by, const R *bz)
{
    return d == 0 ? bx : (d == 1 ? by : bz);
}

template <class R>
void cc_apply(const og_grid *g, const R *extra, const R *bx, const R *by, const R *bz, const R *x, R *y)
{
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                R v = extra[c] * x[c];
                for (int d = 0; d < 3; d++) {
                    const R *B = barr(d, bx, by, bz);
                    int id[3] = {i, j, k};
                    R blo = B[fidx(g, d, id[0], id[1], id[2])];
                    id[d] += 1;
                    R bhi = B[fidx(g, d, id[0], id[1], id[2])];
                    int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                    lo[d] -= 1;
                    hi[d] += 1;
                    R xlo = inside(g, lo[0], lo[1], lo[2]) ? x[cidx(g, lo[0], lo[1], lo[2])] : R(0.0);
                    R xhi = inside(g, hi[0], hi[1], hi[2]) ? x[cidx(g, hi[0], hi[1], hi[2])] : R(0.0);
                    v += blo * (x[c] - xlo) + bhi * (x[c] - xhi);
                }
                y[c] = v;
            }
}

/* Jacobi-preconditioned conjugate gradients on an SPD operator; stops at
 * ||b - A x|| <= tol ||b|| (true residual checked), or at once when a
 * residual is not finite (the result is then reported as that residual). */
int pcg_real(const std::function<void(const double *, double *)> &A, const double *diag, const double *b,
             double *x, size_t n, double tol, int max_iters, double *res_out)
{
    vector<double> r(n), z(n), pp(n), q(n);
    double bn = sqrt(dot(b, b, n));
    int it = 0;
    double rel = 0.0;
    if (bn == 0.0) {
        memset(x, 0, n * sizeof(double));
        if (res_out) *res_out = rel;
        return it;
    }
    for (int restart = 0; restart < 20; restart++) {
        A(x, q.data());
#pragma omp parallel for schedule(static)
        for (long s = 0; s < (long)n; s++) r[s] = b[s] - q[s];
        rel = sqrt(dot(r.data(), r.data(), n)) / bn;
        if (rel <= tol || it >= max_iters || !std::isfinite(rel)) break;
#pragma omp parallel for schedule(static)
        for (long s = 0; s < (long)n; s++) { z[s] = r[s] / diag[s]; pp[s] = z[s]; }
        double rz = dot(r.data(), z.data(), n);
        while (it < max_iters) {
            A(pp.data(), q.data());
            double a = rz / dot(pp.data(), q.data(), n);
#pragma omp parallel for schedule(static)
            for (long s = 0; s < (long)n; s++) { x[s] += a * pp[s]; r[s] -= a * q[s]; }
            it++;
            double rn = sqrt(dot(r.data(), r.data(), n));
            if (rn <= 0.5 * tol * bn || !std::isfinite(rn)) break;
#pragma omp parallel for schedule(static)
            for (long s = 0; s < (long)n; s++) z[s] = r[s] / diag[s];
            double rz2 = dot(r.data(), z.data(), n);
#pragma omp parallel for schedule(static)
            for (long s = 0; s < (long)n; s++) pp[s] = z[s] + (rz2 / rz) * pp[s];
            rz = rz2;
        }
    }
    if (res_out) *res_out = rel;
    return it;
}

/* The solve in the scalar type R.  For double it is pcg_real.  For Dual
 * the value part x solves A x = b, then the derivative part x' solves
 * A x' = b' - A' x with the same (value) operator, each to tol. */
template <class R>
int pcg(const std::function<void(const R *, R *)> &A, const R *diag, const R *b, R *x, size_t n, double tol,
        int max_iters, double *res_out);

template <>
int pcg<double>(const std::function<void(const double *, double *)> &A, const double *diag, const double *b,
                double *x, size_t n, double tol, int max_iters, double *res_out)
{
    return pcg_real(A, diag, b, x, n, tol, max_iters, res_out);
}

template <>
int pcg<Dual>(const std::function<void(const Dual *, Dual *)> &A, const Dual *diag, const Dual *b, Dual *x,
              size_t n, double tol, int max_iters, double *res_out)
{
    vector<Dual> xin(n), yout(n);
    auto Av = [&](const double *xr, double *yr) {
        for (size_t s = 0; s < n; s++) xin[s] = Dual(xr[s], 0.0);
        A(xin.data(), yout.data());
        for (size_t s = 0; s < n; s++) yr[s] = yout[s].v;
    };
    vector<double> dv(n), bv(n), xv(n), rd(n), xd(n);
    for (size_t s = 0; s < n; s++) {
        dv[s] = diag[s].v;
        bv[s] = b[s].v;
        xv[s] = x[s].v;
        xd[s] = x[s].d;
    }
    int it = pcg_real(Av, dv.data(), bv.data(), xv.data(), n, tol, max_iters, res_out);
    for (size_t s = 0; s < n; s++) xin[s] = Dual(xv[s], 0.0);
    A(xin.data(), yout.data());
    for (size_t s = 0; s < n; s++) rd[s] = b[s].d - yout[s].d;
    pcg_real(Av, dv.data(), rd.data(), xd.data(), n, tol, max_iters, nullptr);
    for (size_t s = 0; s < n; s++) x[s] = Dual(xv[s], xd[s]);
    return it;
}

template <class R>
int cc_solve(const og_grid *g, const R *extra, const R *bx, const R *by, const R *bz, const R *b, R *x, double tol,
             int max_iters, double *res_out)
{
    size_t N3 = og_ncell(g);
    vector<R> diag(N3);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                R v = extra[c];
                for (int d = 0; d < 3; d++) {
                    const R *B = barr(d, bx, by, bz);
                    int id[3] = {i, j, k};
                    v += B[fidx(g, d, id[0], id[1], id[2])];
                    id[d] += 1;
                    v += B[fidx(g, d, id[0], id[1], id[2])];
                }
                diag[c] = v > 0.0 ? v : R(1.0);
            }
    auto A = [&](const R *xx, R *yy) { cc_apply(g, extra, bx, by, bz, xx, yy); };
    return pcg<R>(A, diag.data(), b, x, N3, tol, max_iters, res_out);
}

/* A box with no outflow side (velocity prescribed or walls all round, as in
 * the paper's cylinder and sphere runs with U on every boundary, or the
 * Taylor-Green vortex between slip walls) leaves both pressure problems pure
 * Neumann: their solutions are fixed only up to a constant.  One Dirichlet
 * point fixes them: the x- face of cell (0,0,0) acts as an outflow face
 * (phi = 0 beyond it) in the cell-centred projection, and node (0,0,0) is a
 * Dirichlet node (p = 0) in the nodal one.  With a consistent right-hand side
 * (zero net boundary flux) the solution is the pure-Neumann one that is zero
 * at that point. */
int no_outflow(const og_grid *g)
{
    for (int s = 0; s < 6; s++)
        if (g->bc[s] == OG_OUTFLOW) return 0;
    return 1;
}
int pin_face(const og_grid *g, int d, int i, int j, int k)
{
    return d == 0 && i == 0 && j == 0 && k == 0 && no_outflow(g);
}

/* Boundary condition of velocity component `comp` on box side `side`:
 * returns 1 and the value for Dirichlet, 0 for Neumann. */
int side_dirichlet(const og_grid *g, int side, int comp, double *val)
{
    int d = side / 2;
    switch (g->bc[side]) {
    case OG_INFLOW: *val = g->u_in[comp]; return 1;
    case OG_NOSLIP: *val = 0.0; return 1;
    case OG_SLIP: *val = 0.0; return comp == d;
    default: *val = 0.0; return 0;
    }
}

/* Cell-centred projection operator: alpha-weighted EB Poisson (face-centred
 * fluxes weighted by the apertures), Dirichlet phi = 0 at outflow sides,
 * Neumann elsewhere and on the EB. */
template <class R>
void mac_coeffs(const og_grid *g, const og_geom *geo, R *extra, R *bx, R *by, R *bz)
{
    const double h2 = g->h * g->h;
    for (size_t c = 0; c < og_ncell(g); c++) extra[c] = geo->alpha[c] > 0.0 ? 0.0 : 1.0;
    for (int d = 0; d < 3; d++) {
        R *B = (R *)barr<R>(d, bx, by, bz);
        const double *a = farr(geo, d);
        int m[3] = {NX, NY, NZ};
        m[d] += 1;
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    int id[3] = {i, j, k};
                    size_t f = fidx(g, d, i, j, k);
                    if (id[d] == 0 || id[d] == g->n[d]) {
                        int side = 2 * d + (id[d] == g->n[d]);
                        B[f] = (g->bc[side] == OG_OUTFLOW || pin_face(g, d, i, j, k)) ? 2.0 * a[f] / h2 : 0.0;
                    } else {
                        B[f] = a[f] / h2;
                    }
                }
    }
}

/* Semi-implicit viscous operator for one component (Eq. implicit-viscous),
 * alpha-weighted: rho*alpha*u + dt/h^2 sum a_f eta_f (u_i - u_nb)
 * + dt/h^2 eta_i A_EB / delta_i u_i, with delta_i the distance from the EB
 * centroid plane to the cell centre (cell units, bounded below). */
template <class R>
void visc_coeffs(const og_grid *g, const og_geom *geo, const Par<R> &p, const R *eta, double dt, int comp, R *extra,
                 R *bx, R *by, R *bz, R *rhs_bc)
{
    const double h2 = g->h * g->h;
    size_t N3 = og_ncell(g);
    for (size_t c = 0; c < N3; c++) {
        if (geo->alpha[c] <= 0.0) { extra[c] = 1.0; if (rhs_bc) rhs_bc[c] = 0.0; continue; }
        R e = p.rho * geo->alpha[c];
        if (geo->flag[c] == 2 && geo->area[c] > 0.0) {
            double nb = 0.0;
            for (int q = 0; q < 3; q++) nb += geo->nrm[q * N3 + c] * geo->bcen[q * N3 + c];
            double del = -nb > p.delta_min ? -nb : p.delta_min;
            e += dt * eta[c] * geo->area[c] / (h2 * del);
        }
        extra[c] = e;
        if (rhs_bc) rhs_bc[c] = 0.0;
    }
    for (int d = 0; d < 3; d++) {
        R *B = (R *)barr<R>(d, bx, by, bz);
        const double *a = farr(geo, d);
        int m[3] = {NX, NY, NZ};
        m[d] += 1;
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    int id[3] = {i, j, k};
                    size_t f = fidx(g, d, i, j, k);
                    if (id[d] == 0 || id[d] == g->n[d]) {
                        int hi = id[d] == g->n[d];
                        int side = 2 * d + hi;
                        int cc[3] = {i, j, k};
                        if (hi) cc[d] -= 1;
                        size_t c = cidx(g, cc[0], cc[1], cc[2]);
                        double val;
                        if (a[f] > 0.0 && side_dirichlet(g, side, comp, &val)) {
                            B[f] = 2.0 * dt * a[f] * eta[c] / h2;
                            if (rhs_bc) rhs_bc[c] += B[f] * val;
                        } else {
                            B[f] = 0.0;
                        }
                    } else {
                        int lo[3] = {i, j, k};
                        lo[d] -= 1;
                        R ef = 0.5 * (eta[cidx(g, lo[0], lo[1], lo[2])] + eta[cidx(g, i, j, k)]);
                        B[f] = a[f] > 0.0 ? dt * a[f] * ef / h2 : R(0.0);
                    }
                }
    }
}

/* ------------------------------------------------------------------------ */
/* Nodal projection                                                          */
/* ------------------------------------------------------------------------ */

/* Trilinear (Q1) stiffness on the unit cube, int grad N_a . grad N_b, from the
 * 1-D integrals: int phi_p phi_q = 1/3 or 1/6, int phi_p' phi_q' = +1 or -1. */
double q1_stiff(int oa, int ob)
{
    double v = 0.0;
    for (int d = 0; d < 3; d++) {
        double t = 1.0;
        for (int e = 0; e < 3; e++) {
            int pa = (oa >> e) & 1, pb = (ob >> e) & 1;
            if (e == d) t *= (pa == pb) ? 1.0 : -1.0;
            else t *= (pa == pb) ? 1.0 / 3.0 : 1.0 / 6.0;
        }
        v += t;
    }
    return v;
}

int node_dirichlet(const og_grid *g, int i, int j, int k)
{
    if (i == 0 && j == 0 && k == 0 && no_outflow(g)) return 1;  /* the pinned node */
    int id[3] = {i, j, k};
    for (int d = 0; d < 3; d++) {
        if (id[d] == 0 && g->bc[2 * d] == OG_OUTFLOW) return 1;
        if (id[d] == g->n[d] && g->bc[2 * d + 1] == OG_OUTFLOW) return 1;
    }
    return 0;
}
/* A node is active when it is not a Dirichlet node and touches fluid. */
int node_active(const og_grid *g, const og_geom *geo, int i, int j, int k)
{
    if (node_dirichlet(g, i, j, k)) return 0;
    for (int o = 0; o < 8; o++) {
        int ci = i - 1 + (o & 1), cj = j - 1 + ((o >> 1) & 1), ck = k - 1 + ((o >> 2) & 1);
        if (avail(g, geo, ci, cj, ck)) return 1;
    }
    return 0;
}
/* node_active of every node, evaluated once per call (a table, not a change
 * of the arithmetic). */
vector<unsigned char> active_nodes(const og_grid *g, const og_geom *geo)
{
    vector<unsigned char> act(og_nnode(g));
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= NZ; k++)
        for (int j = 0; j <= NY; j++)
            for (int i = 0; i <= NX; i++) act[nidx(g, i, j, k)] = (unsigned char)node_active(g, geo, i, j, k);
    return act;
}

template <class R>
void nodal_apply(const og_grid *g, const og_geom *geo, double coef, const R *p, R *y)
{
    double K[8][8];
    for (int a = 0; a < 8; a++)
        for (int b = 0; b < 8; b++) K[a][b] = q1_stiff(a, b);
    vector<unsigned char> act = active_nodes(g, geo);
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= NZ; k++)
        for (int j = 0; j <= NY; j++)
            for (int i = 0; i <= NX; i++) {
                size_t n = nidx(g, i, j, k);
                if (!act[n]) { y[n] = p[n]; continue; }
                R v = 0.0;
                for (int oc = 0; oc < 8; oc++) {
                    /* cell with this node at local corner oa */
                    int ci = i - 1 + (oc & 1), cj = j - 1 + ((oc >> 1) & 1), ck = k - 1 + ((oc >> 2) & 1);
                    if (!inside(g, ci, cj, ck)) continue;
                    double al = geo->alpha[cidx(g, ci, cj, ck)];
                    if (al <= 0.0) continue;
                    int oa = (i - ci) | ((j - cj) << 1) | ((k - ck) << 2);
                    for (int ob = 0; ob < 8; ob++) {
                        int bi = ci + (ob & 1), bj = cj + ((ob >> 1) & 1), bk = ck + ((ob >> 2) & 1);
                        if (!act[nidx(g, bi, bj, bk)]) continue;
                        v += al * K[oa][ob] * p[nidx(g, bi, bj, bk)];
                    }
                }
                y[n] = coef * g->h * v;
            }
}

/* Right-hand side of the nodal Poisson equation in weak form:
 * sum over cells of alpha_c h^3 grad N_a(centre) . u_c, minus the boundary
 * integral of N_a u_bc . n on inflow sides (zero on walls). */
template <class R>
void nodal_rhs(const og_grid *g, const og_geom *geo, const R *ut, R *rhs)
{
    size_t N3 = og_ncell(g);
    const double h = g->h;
    vector<unsigned char> act = active_nodes(g, geo);
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= NZ; k++)
        for (int j = 0; j <= NY; j++)
            for (int i = 0; i <= NX; i++) {
                size_t n = nidx(g, i, j, k);
                if (!act[n]) { rhs[n] = 0.0; continue; }
                R v = 0.0;
                for (int oc = 0; oc < 8; oc++) {
                    int ci = i - 1 + (oc & 1), cj = j - 1 + ((oc >> 1) & 1), ck = k - 1 + ((oc >> 2) & 1);
                    if (!avail(g, geo, ci, cj, ck)) continue;
                    size_t c = cidx(g, ci, cj, ck);
                    int o[3] = {i - ci, j - cj, k - ck};
                    for (int d = 0; d < 3; d++)
                        v += geo->alpha[c] * h * h * 0.25 * (o[d] ? 1.0 : -1.0) * ut[d * N3 + c];
                }
                int id[3] = {i, j, k};
                for (int d = 0; d < 3; d++)
                    for (int hs = 0; hs < 2; hs++) {
                        int side = 2 * d + hs;
                        if (g->bc[side] != OG_INFLOW) continue;
                        if (id[d] != (hs ? g->n[d] : 0)) continue;
                        double sgn = hs ? 1.0 : -1.0; /* outward normal */
                        int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
                        for (int q1 = -1; q1 <= 0; q1++)
                            for (int q2 = -1; q2 <= 0; q2++) {
                                int fid[3] = {i, j, k};
                                fid[t1] += q1;
                                fid[t2] += q2;
                                if (fid[t1] < 0 || fid[t1] >= g->n[t1] || fid[t2] < 0 || fid[t2] >= g->n[t2])
                                    continue;
                                double af = farr(geo, d)[fidx(g, d, fid[0], fid[1], fid[2])];
                                v -= sgn * g->u_in[d] * af * h * h * 0.25;
                            }
                    }
                rhs[n] = v;
            }
}

template <class R>
int nodal_solve(const og_grid *g, const og_geom *geo, double coef, const R *b, R *p, double tol, int max_iters,
                double *res_out)
{
    size_t NN = og_nnode(g);
    vector<R> diag(NN);
    double K00 = q1_stiff(0, 0);
    vector<unsigned char> act = active_nodes(g, geo);
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= NZ; k++)
        for (int j = 0; j <= NY; j++)
            for (int i = 0; i <= NX; i++) {
                size_t n = nidx(g, i, j, k);
                double v = 0.0;
                if (act[n]) {
                    for (int oc = 0; oc < 8; oc++) {
                        int ci = i - 1 + (oc & 1), cj = j - 1 + ((oc >> 1) & 1), ck = k - 1 + ((oc >> 2) & 1);
                        if (avail(g, geo, ci, cj, ck)) v += geo->alpha[cidx(g, ci, cj, ck)] * K00;
                    }
                    v *= coef * g->h;
                } else {
                    p[n] = 0.0;
                }
                diag[n] = v > 0.0 ? v : 1.0;
            }
    auto A = [&](const R *xx, R *yy) { nodal_apply(g, geo, coef, xx, yy); };
    return pcg<R>(A, diag.data(), b, p, NN, tol, max_iters, res_out);
}

/* Gradient of the trilinear interpolant of nodal p at each cell centre. */
template <class R>
void cell_grad_p(const og_grid *g, const R *p, R *gp)
{
    size_t N3 = og_ncell(g);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                for (int d = 0; d < 3; d++) {
                    int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
                    R s = 0.0;
                    for (int q1 = 0; q1 < 2; q1++)
                        for (int q2 = 0; q2 < 2; q2++) {
                            int lo[3] = {i, j, k};
                            lo[t1] += q1;
                            lo[t2] += q2;
                            int hi[3] = {lo[0], lo[1], lo[2]};
                            hi[d] += 1;
                            s += p[nidx(g, hi[0], hi[1], hi[2])] - p[nidx(g, lo[0], lo[1], lo[2])];
                        }
                    gp[d * N3 + c] = s / (4.0 * g->h);
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Derived quantities (Algorithm 2)                                          */
/* ------------------------------------------------------------------------ */

/* Monotonised-central limited slope (difference across one cell); zero when
 * a neighbour in that direction is covered or outside the box. */
template <class R>
R slope(const og_grid *g, const og_geom *geo, const R *f, int i, int j, int k, int d)
{
    int e[3] = {0, 0, 0};
    e[d] = 1;
    if (!avail(g, geo, i + e[0], j + e[1], k + e[2]) || !avail(g, geo, i - e[0], j - e[1], k - e[2])) return 0.0;
    R f0 = f[cidx(g, i, j, k)];
    R fp = f[cidx(g, i + e[0], j + e[1], k + e[2])];
    R fm = f[cidx(g, i - e[0], j - e[1], k - e[2])];
    R dl = f0 - fm, dr = fp - f0, dc = 0.5 * (fp - fm);
    if (dl * dr <= 0.0) return 0.0;
    R m = fabs(dc);
    if (2.0 * fabs(dl) < m) m = 2.0 * fabs(dl);
    if (2.0 * fabs(dr) < m) m = 2.0 * fabs(dr);
    return dc > 0.0 ? m : -m;
}

/* Upwinding of the face-normal velocity from the two extrapolated states. */
template <class R>
R upwind_normal(const R &uL, const R &uR)
{
    if (uL > 0.0 && uL + uR > 0.0) return uL;
    if (uR < 0.0 && uL + uR < 0.0) return uR;
    return 0.0;
}

template <class R>
void face_states(const og_grid *g, const og_geom *geo, const R *u, R *uf)
{
    size_t N3 = og_ncell(g);
    size_t off = 0;
    for (int d = 0; d < 3; d++) {
        const double *a = farr(geo, d);
        const R *ud = u + d * N3;
        int m[3] = {NX, NY, NZ};
        m[d] += 1;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    int id[3] = {i, j, k};
                    size_t f = fidx(g, d, i, j, k);
                    R v = 0.0;
                    if (a[f] > 0.0) {
                        int lo[3] = {i, j, k};
                        lo[d] -= 1;
                        if (id[d] == 0 || id[d] == g->n[d]) {
                            int hs = id[d] == g->n[d];
                            int side = 2 * d + hs;
                            int cc[3] = {i, j, k};
                            if (hs) cc[d] -= 1;
                            switch (g->bc[side]) {
                            case OG_INFLOW: v = g->u_in[d]; break;
                            case OG_OUTFLOW: v = ud[cidx(g, cc[0], cc[1], cc[2])]; break;
                            default: v = 0.0;
                            }
                        } else {
                            R uL = ud[cidx(g, lo[0], lo[1], lo[2])] + 0.5 * slope(g, geo, ud, lo[0], lo[1], lo[2], d);
                            R uR = ud[cidx(g, i, j, k)] - 0.5 * slope(g, geo, ud, i, j, k, d);
                            v = upwind_normal(uL, uR);
                        }
                    }
                    uf[off + f] = v;
                }
        off += nface(g, d);
    }
}

template <class R>
int mac_project(const og_grid *g, const og_geom *geo, R *uf, R *phi, double tol, int max_iters, double *res_out)
{
    size_t N3 = og_ncell(g);
    size_t nf[3] = {nface(g, 0), nface(g, 1), nface(g, 2)};
    R *ufd[3] = {uf, uf + nf[0], uf + nf[0] + nf[1]};
    vector<R> extra(N3), b(N3), B0(nf[0]), B1(nf[1]), B2(nf[2]);
    R *B[3] = {B0.data(), B1.data(), B2.data()};
    mac_coeffs(g, geo, extra.data(), B[0], B[1], B[2]);
    const double h = g->h;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                if (geo->alpha[c] <= 0.0) { b[c] = 0.0; continue; }
                R s = 0.0;
                for (int d = 0; d < 3; d++) {
                    int id[3] = {i, j, k};
                    size_t flo = fidx(g, d, id[0], id[1], id[2]);
                    id[d] += 1;
                    size_t fhi = fidx(g, d, id[0], id[1], id[2]);
                    s += farr(geo, d)[fhi] * ufd[d][fhi] - farr(geo, d)[flo] * ufd[d][flo];
                }
                b[c] = -s / h;
            }
    for (size_t c = 0; c < N3; c++) phi[c] = 0.0;
    int it = cc_solve(g, extra.data(), B[0], B[1], B[2], b.data(), phi, tol, max_iters, res_out);
    for (int d = 0; d < 3; d++) {
        const double *a = farr(geo, d);
        int m[3] = {NX, NY, NZ};
        m[d] += 1;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    int id[3] = {i, j, k};
                    size_t f = fidx(g, d, i, j, k);
                    if (a[f] <= 0.0) continue;
                    if (id[d] == 0 || id[d] == g->n[d]) {
                        int hs = id[d] == g->n[d];
                        if (g->bc[2 * d + hs] != OG_OUTFLOW && !pin_face(g, d, i, j, k)) continue;
                        int cc[3] = {i, j, k};
                        if (hs) cc[d] -= 1;
                        R pc = phi[cidx(g, cc[0], cc[1], cc[2])];
                        R grad = hs ? (0.0 - pc) / (0.5 * h) : (pc - 0.0) / (0.5 * h);
                        ufd[d][f] -= grad;
                    } else {
                        int lo[3] = {i, j, k};
                        lo[d] -= 1;
                        ufd[d][f] -= (phi[cidx(g, i, j, k)] - phi[cidx(g, lo[0], lo[1], lo[2])]) / h;
                    }
                }
    }
    return it;
}

/* Neighbourhood average, hybridisation and redistribution of the excess
 * (Eqs. divergence_nonconservative .. divergence_final), with the
 * neighbourhood read as the 26 surrounding cells that hold fluid. */
template <class R>
void redistribute(const og_grid *g, const og_geom *geo, const R *DC, R *D)
{
    size_t N3 = og_ncell(g);
    vector<R> dD(N3, R(0.0));
    vector<double> w(N3, 0.0);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                double al = geo->alpha[c];
                if (al <= 0.0) { D[c] = 0.0; continue; }
                double sa = 0.0;
                R sad = 0.0;
                for (int dk = -1; dk <= 1; dk++)
                    for (int dj = -1; dj <= 1; dj++)
                        for (int di = -1; di <= 1; di++) {
                            if (!di && !dj && !dk) continue;
                            if (!avail(g, geo, i + di, j + dj, k + dk)) continue;
                            size_t c2 = cidx(g, i + di, j + dj, k + dk);
                            sa += geo->alpha[c2];
                            sad += geo->alpha[c2] * DC[c2];
                        }
                R dnc = sa > 0.0 ? sad / sa : DC[c];
                D[c] = al * DC[c] + (1.0 - al) * dnc; /* hybrid D^H */
                dD[c] = al * (1.0 - al) * (DC[c] - dnc);
                w[c] = sa > 0.0 ? 1.0 / sa : 0.0;
            }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                if (geo->alpha[c] <= 0.0) continue;
                R s = 0.0;
                for (int dk = -1; dk <= 1; dk++)
                    for (int dj = -1; dj <= 1; dj++)
                        for (int di = -1; di <= 1; di++) {
                            if (!di && !dj && !dk) continue;
                            if (!avail(g, geo, i + di, j + dj, k + dk)) continue;
                            size_t c2 = cidx(g, i + di, j + dj, k + dk);
                            s += w[c2] * dD[c2];
                        }
                D[c] += s;
            }
}

/* Convective term C = -div(u (x) u^F) with zero EB flux; advected states are
 * the slope-extrapolated cell values upwinded by the projected face velocity. */
template <class R>
void convective(const og_grid *g, const og_geom *geo, const R *u, const R *uf, R *C)
{
    size_t N3 = og_ncell(g);
    size_t nf[3] = {nface(g, 0), nface(g, 1), nface(g, 2)};
    const R *ufd[3] = {uf, uf + nf[0], uf + nf[0] + nf[1]};
    const double h = g->h;
    vector<R> DC(N3), D(N3);
    for (int q = 0; q < 3; q++) {
        const R *uq = u + q * N3;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < NZ; k++)
            for (int j = 0; j < NY; j++)
                for (int i = 0; i < NX; i++) {
                    size_t c = cidx(g, i, j, k);
                    if (geo->alpha[c] <= 0.0) { DC[c] = 0.0; continue; }
                    R s = 0.0;
                    for (int d = 0; d < 3; d++)
                        for (int hs = 0; hs < 2; hs++) {
                            int id[3] = {i, j, k};
                            id[d] += hs;
                            size_t f = fidx(g, d, id[0], id[1], id[2]);
                            double a = farr(geo, d)[f];
                            if (a <= 0.0) continue;
                            R w = ufd[d][f], state;
                            if (id[d] == 0 || id[d] == g->n[d]) {
                                int side = 2 * d + hs;
                                if (g->bc[side] == OG_INFLOW) state = g->u_in[q];
                                else state = uq[c];
                            } else {
                                int L[3] = {id[0], id[1], id[2]};
                                L[d] -= 1;
                                int Rr[3] = {id[0], id[1], id[2]};
                                R sL = uq[cidx(g, L[0], L[1], L[2])] + 0.5 * slope(g, geo, uq, L[0], L[1], L[2], d);
                                R sR = uq[cidx(g, Rr[0], Rr[1], Rr[2])] - 0.5 * slope(g, geo, uq, Rr[0], Rr[1], Rr[2], d);
                                state = w > 0.0 ? sL : (w < 0.0 ? sR : 0.5 * (sL + sR));
                            }
                            s += (hs ? 1.0 : -1.0) * a * state * w;
                        }
                    DC[c] = s / (geo->alpha[c] * h);
                }
        redistribute(g, geo, DC.data(), D.data());
        for (size_t c = 0; c < N3; c++) C[q * N3 + c] = -D[c];
    }
}

/* Normal derivative of velocity component `comp` at the EB centroid of a cut
 * cell (Eqs. interpolation_distances and dudn), u_EB = 0.  Interpolation planes
 * are the cell-centre planes one and two cells away along the axis of the
 * largest |n_d|; values come from biquadratic Lagrange interpolation on the
 * 3x3 cells nearest to the crossing point.  If a needed cell is covered, the
 * nearest cell of the first plane gives a one-point estimate. */
template <class R>
R wall_dudn(const og_grid *g, const og_geom *geo, const R *u, int cell, int comp)
{
    size_t N3 = og_ncell(g);
    const R *uq = u + (size_t)comp * N3;
    double n[3], b[3];
    for (int e = 0; e < 3; e++) {
        n[e] = geo->nrm[e * N3 + cell];
        b[e] = geo->bcen[e * N3 + cell];
    }
    int ci[3];
    ci[0] = cell % NX;
    ci[1] = (cell / NX) % NY;
    ci[2] = cell / (NX * NY);
    int kax = 0;
    for (int e = 1; e < 3; e++)
        if (fabs(n[e]) > fabs(n[kax])) kax = e;
    int k1 = (kax == 0) ? 1 : 0, k2 = (kax == 2) ? 1 : 2;
    double s = n[kax] > 0.0 ? 1.0 : -1.0;
    double dist[2] = {(s - b[kax]) / n[kax], (2.0 * s - b[kax]) / n[kax]};
    R uv[2];
    int ok = 1, near[3] = {0, 0, 0};
    for (int m = 0; m < 2 && ok; m++) {
        double P[3];
        for (int e = 0; e < 3; e++) P[e] = b[e] + dist[m] * n[e];
        int c1 = (int)floor(P[k1] + 0.5), c2 = (int)floor(P[k2] + 0.5);
        double x1 = P[k1] - c1, x2 = P[k2] - c2;
        double L1[3] = {0.5 * x1 * (x1 - 1.0), 1.0 - x1 * x1, 0.5 * x1 * (x1 + 1.0)};
        double L2[3] = {0.5 * x2 * (x2 - 1.0), 1.0 - x2 * x2, 0.5 * x2 * (x2 + 1.0)};
        if (m == 0) {
            near[kax] = ci[kax] + (int)s;
            near[k1] = ci[k1] + c1;
            near[k2] = ci[k2] + c2;
        }
        R v = 0.0;
        for (int q1 = -1; q1 <= 1 && ok; q1++)
            for (int q2 = -1; q2 <= 1; q2++) {
                int id[3];
                id[kax] = ci[kax] + (m + 1) * (int)s;
                id[k1] = ci[k1] + c1 + q1;
                id[k2] = ci[k2] + c2 + q2;
                if (!avail(g, geo, id[0], id[1], id[2])) { ok = 0; break; }
                v += L1[q1 + 1] * L2[q2 + 1] * uq[cidx(g, id[0], id[1], id[2])];
            }
        uv[m] = v;
    }
    const double h = g->h;
    if (ok) {
        double d1 = dist[0], d2 = dist[1];
        return (d2 * d2 * uv[0] - d1 * d1 * uv[1]) / (d1 * d2 * (d2 - d1)) / h;
    }
    if (avail(g, geo, near[0], near[1], near[2])) return uq[cidx(g, near[0], near[1], near[2])] / (dist[0] * h);
    return 0.0;
}

/* Explicit viscous term V = (1/rho) div(eta (grad u)^T) (Eq. explicit-viscous)
 * with face fluxes eta_f d u_d / d x_j, the EB wall flux from the wall-normal
 * derivative, and the same hybrid redistribution as the convective term. */
template <class R>
void viscous_explicit(const og_grid *g, const og_geom *geo, const Par<R> &p, const R *u, const R *eta, R *V)
{
    size_t N3 = og_ncell(g);
    const double h = g->h;
    vector<R> G(9 * N3), DC(3 * N3), D(N3), dudn(3 * N3, R(0.0));
    cell_gradient(g, geo, u, G.data());
#pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)N3; c++)
        if (geo->flag[c] == 2 && geo->area[c] > 0.0)
            for (int q = 0; q < 3; q++) dudn[q * N3 + c] = wall_dudn(g, geo, u, (int)c, q);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                for (int jj = 0; jj < 3; jj++) DC[jj * N3 + c] = 0.0;
                if (geo->alpha[c] <= 0.0) continue;
                for (int jj = 0; jj < 3; jj++) {
                    R s = 0.0;
                    for (int d = 0; d < 3; d++)
                        for (int hs = 0; hs < 2; hs++) {
                            int id[3] = {i, j, k};
                            id[d] += hs;
                            size_t f = fidx(g, d, id[0], id[1], id[2]);
                            double a = farr(geo, d)[f];
                            if (a <= 0.0) continue;
                            R T;
                            if (id[d] == 0 || id[d] == g->n[d]) {
                                int side = 2 * d + hs;
                                double val;
                                if (side_dirichlet(g, side, d, &val)) {
                                    R ud = u[d * N3 + c];
                                    T = (jj == d) ? eta[c] * (hs ? (val - ud) : (ud - val)) / (0.5 * h) : R(0.0);
                                } else {
                                    T = (jj == d) ? R(0.0) : eta[c] * G[(3 * jj + d) * N3 + c];
                                }
                            } else {
                                int L[3] = {id[0], id[1], id[2]};
                                L[d] -= 1;
                                size_t cL = cidx(g, L[0], L[1], L[2]);
                                size_t cR = cidx(g, id[0], id[1], id[2]);
                                R ef = 0.5 * (eta[cL] + eta[cR]);
                                R der = (jj == d) ? (u[d * N3 + cR] - u[d * N3 + cL]) / h
                                                  : 0.5 * (G[(3 * jj + d) * N3 + cL] + G[(3 * jj + d) * N3 + cR]);
                                T = ef * der;
                            }
                            s += (hs ? 1.0 : -1.0) * a * T;
                        }
                    if (geo->flag[c] == 2 && geo->area[c] > 0.0) {
                        R nd = 0.0;
                        for (int q = 0; q < 3; q++) nd += geo->nrm[q * N3 + c] * dudn[q * N3 + c];
                        /* outward normal of the fluid region on the EB is -n */
                        s += -eta[c] * geo->nrm[jj * N3 + c] * nd * geo->area[c];
                    }
                    DC[jj * N3 + c] = s / (geo->alpha[c] * h);
                }
            }
    for (int q = 0; q < 3; q++) {
        redistribute(g, geo, DC.data() + q * N3, D.data());
        for (size_t c = 0; c < N3; c++) V[q * N3 + c] = D[c] / p.rho;
    }
}

template <class R>
void derived(const og_grid *g, const og_geom *geo, const Par<R> &p, const R *u, R *C, R *eta, R *V, R *srate,
             og_stats *st)
{
    size_t N3 = og_ncell(g);
    size_t nft = nface(g, 0) + nface(g, 1) + nface(g, 2);
    vector<R> uf(nft), phi(N3);
    double res = 0.0;
    if (p.advect) {
        face_states(g, geo, u, uf.data());
        int it = mac_project(g, geo, uf.data(), phi.data(), p.tol, p.max_iters, &res);
        if (st) { st->iters[0] = it; st->res[0] = res; }
        convective(g, geo, u, uf.data(), C);
    } else {
        /* creeping flow (the paper's evaluation, Re = 1e-3): no convective term */
        for (size_t s = 0; s < 3 * N3; s++) C[s] = 0.0;
        if (st) { st->iters[0] = 0; st->res[0] = 0.0; }
    }
    strain_eta(g, geo, p, u, eta, srate);
    viscous_explicit(g, geo, p, u, eta, V);
}

template <class R>
int viscous_solve(const og_grid *g, const og_geom *geo, const Par<R> &p, const R *eta, const R *psi, double dt, R *ut,
                  og_stats *st, int slot)
{
    size_t N3 = og_ncell(g);
    vector<R> extra(N3), rb(N3), b(N3), B0(nface(g, 0)), B1(nface(g, 1)), B2(nface(g, 2));
    int tot = 0;
    for (int q = 0; q < 3; q++) {
        visc_coeffs(g, geo, p, eta, dt, q, extra.data(), B0.data(), B1.data(), B2.data(), rb.data());
        for (size_t c = 0; c < N3; c++) {
            b[c] = geo->alpha[c] > 0.0 ? geo->alpha[c] * psi[q * N3 + c] + rb[c] : R(0.0);
            ut[q * N3 + c] = geo->alpha[c] > 0.0 ? psi[q * N3 + c] / p.rho : R(0.0);
        }
        double res = 0.0;
        int it = cc_solve(g, extra.data(), B0.data(), B1.data(), B2.data(), b.data(), ut + q * N3, p.tol,
                          p.max_iters, &res);
        if (st) { st->iters[slot + q] = it; st->res[slot + q] = res; }
        tot += it;
    }
    return tot;
}

template <class R>
int nodal_project(const og_grid *g, const og_geom *geo, const Par<R> &p, double dt, R *ut, R *pres, og_stats *st,
                  int slot)
{
    size_t N3 = og_ncell(g), NN = og_nnode(g);
    vector<R> gp(3 * N3), rhs(NN);
    double coef = dt / value_of(p.rho);
    cell_grad_p(g, pres, gp.data());
    for (int q = 0; q < 3; q++)
        for (size_t c = 0; c < N3; c++)
            ut[q * N3 + c] = geo->alpha[c] > 0.0 ? ut[q * N3 + c] + coef * gp[q * N3 + c] : R(0.0);
    nodal_rhs(g, geo, ut, rhs.data());
    double res = 0.0;
    int it = nodal_solve(g, geo, coef, rhs.data(), pres, p.tol, p.max_iters, &res);
    if (st) { st->iters[slot] = it; st->res[slot] = res; }
    cell_grad_p(g, pres, gp.data());
    for (int q = 0; q < 3; q++)
        for (size_t c = 0; c < N3; c++)
            ut[q * N3 + c] = geo->alpha[c] > 0.0 ? ut[q * N3 + c] - coef * gp[q * N3 + c] : R(0.0);
    return it;
}

template <class R>
void drag(const og_grid *g, const og_geom *geo, const Par<R> &p, const R *u, const R *pres, R *fz, double *yield_frac)
{
    size_t N3 = og_ncell(g);
    vector<R> eta(N3), sr(N3);
    strain_eta(g, geo, p, u, eta.data(), sr.data());
    const double h = g->h;
    R F = 0.0;
    double vy = 0.0, vt = 0.0;
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                double al = geo->alpha[c];
                if (al <= 0.0) continue;
                vt += al;
                if (eta[c] * sr[c] <= (1.0 + 1e-3) * p.tau0) vy += al;
                if (geo->flag[c] != 2 || geo->area[c] <= 0.0) continue;
                double n[3], b[3];
                R gq[3];
                for (int e = 0; e < 3; e++) {
                    n[e] = geo->nrm[e * N3 + c];
                    b[e] = geo->bcen[e * N3 + c];
                    gq[e] = wall_dudn(g, geo, u, (int)c, e);
                }
                R gn = gq[0] * n[0] + gq[1] * n[1] + gq[2] * n[2];
                R tz = eta[c] * (n[2] * gn + gq[2]);
                R pb = 0.0;
                for (int o = 0; o < 8; o++) {
                    int oi = o & 1, oj = (o >> 1) & 1, ok = (o >> 2) & 1;
                    double w = (oi ? b[0] + 0.5 : 0.5 - b[0]) * (oj ? b[1] + 0.5 : 0.5 - b[1]) *
                               (ok ? b[2] + 0.5 : 0.5 - b[2]);
                    pb += w * pres[nidx(g, i + oi, j + oj, k + ok)];
                }
                F += geo->area[c] * h * h * (tz - pb * n[2]);
            }
    *fz = F;
    *yield_frac = vt > 0.0 ? vy / vt : 0.0;
}

/* Algorithm 1: predictor and corrector with a semi-implicit viscous update
 * and a nodal projection each, at the time step dt (> 0). */
template <class R>
void advance(const og_grid *g, const og_geom *geo, const Par<R> &p, R *u, R *pres, double dt, const R *f,
             og_stats *st, R *drag_out)
{
    size_t N3 = og_ncell(g), V3 = 3 * N3, NN = og_nnode(g);
    vector<R> Cm(V3), Vm(V3), Cs(V3), Vs(V3), em(N3), es(N3), psi(V3), ut(V3), gp(V3), ps(NN);
    og_stats loc;
    memset(&loc, 0, sizeof loc);
    og_stats tmp;
    memset(&tmp, 0, sizeof tmp);

    /* Predictor */
    derived(g, geo, p, u, Cm.data(), em.data(), Vm.data(), (R *)nullptr, &tmp);
    loc.iters[0] = tmp.iters[0];
    loc.res[0] = tmp.res[0];
    cell_grad_p(g, pres, gp.data());
    for (int q = 0; q < 3; q++)
        for (size_t c = 0; c < N3; c++) {
            size_t s = q * N3 + c;
            R fq = f ? f[s] : R(0.0);
            psi[s] = geo->alpha[c] > 0.0 ? p.rho * u[s] + dt * (p.rho * Cm[s] + Vm[s] - gp[s] + fq) : R(0.0);
        }
    viscous_solve(g, geo, p, em.data(), psi.data(), dt, ut.data(), &loc, 1);
    for (size_t s = 0; s < NN; s++) ps[s] = pres[s];
    nodal_project(g, geo, p, dt, ut.data(), ps.data(), &loc, 4);
    /* ut now holds u*, ps holds p* */

    /* Corrector */
    derived(g, geo, p, ut.data(), Cs.data(), es.data(), Vs.data(), (R *)nullptr, &tmp);
    loc.iters[5] = tmp.iters[0];
    loc.res[5] = tmp.res[0];
    for (size_t s = 0; s < V3; s++) {
        Cm[s] = 0.5 * (Cm[s] + Cs[s]);
        Vm[s] = 0.5 * (Vm[s] + Vs[s]);
    }
    for (size_t c = 0; c < N3; c++) em[c] = 0.5 * (em[c] + es[c]);
    cell_grad_p(g, ps.data(), gp.data());
    for (int q = 0; q < 3; q++)
        for (size_t c = 0; c < N3; c++) {
            size_t s = q * N3 + c;
            R fq = f ? f[s] : R(0.0);
            psi[s] = geo->alpha[c] > 0.0 ? p.rho * u[s] + dt * (p.rho * Cm[s] + Vm[s] - gp[s] + fq) : R(0.0);
        }
    viscous_solve(g, geo, p, em.data(), psi.data(), dt, ut.data(), &loc, 6);
    for (size_t s = 0; s < NN; s++) pres[s] = ps[s];
    nodal_project(g, geo, p, dt, ut.data(), pres, &loc, 9);
    for (size_t s = 0; s < V3; s++) u[s] = ut[s];

    loc.dt = dt;
    R fz;
    drag(g, geo, p, u, pres, &fz, &loc.yield_frac);
    loc.drag = value_of(fz);
    if (drag_out) *drag_out = fz;
    if (st) *st = loc;
}

}  // namespace

/* Flow diagnostics of Sec. "Cylinder moving through Bingham fluid": the flow
 * topology parameter of Eq. ryovar, Lambda = (||g||^2 - |w|^2) / (||g||^2 +
 * |w|^2) with ||g|| the strain-rate norm and w = curl u (0 where both vanish),
 * and the relative deviation from the yield stress, ||tau|| / tau0 - 1 with
 * ||tau|| = eta ||g|| (0 when tau0 = 0).  Gradients are the robust cell
 * gradients of the strain-rate step; covered cells get 0. */
template <class R>
void flow_diagnostics(const og_grid *g, const og_geom *geo, const Par<R> &p, const R *u, R *lam, R *sdev)
{
    size_t N3 = og_ncell(g);
    vector<R> G(9 * N3), eta(N3), sr(N3);
    cell_gradient(g, geo, u, G.data());
    strain_eta(g, geo, p, u, eta.data(), sr.data());
#pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)N3; c++) {
        if (geo->alpha[c] <= 0.0) { lam[c] = 0.0; sdev[c] = 0.0; continue; }
        auto D = [&](int d, int q) -> R { return G[(3 * d + q) * N3 + c]; };  /* du_q / dx_d */
        R wx = D(1, 2) - D(2, 1), wy = D(2, 0) - D(0, 2), wz = D(0, 1) - D(1, 0);
        R w2 = wx * wx + wy * wy + wz * wz;
        R s2 = sr[c] * sr[c];
        lam[c] = (s2 + w2) > 0.0 ? (s2 - w2) / (s2 + w2) : R(0.0);
        sdev[c] = p.tau0 > 0.0 ? eta[c] * sr[c] / p.tau0 - 1.0 : R(0.0);
    }
}

/* ------------------------------------------------------------------------ */
/* C entry points (double)                                                   */
/* ------------------------------------------------------------------------ */

extern "C" double og_eta_of(const og_params *p, double sr) { return eta_of(par_of<double>(p), sr); }

extern "C" void og_strain_eta(const og_grid *g, const og_geom *geo, const og_params *p, const double *u, double *eta,
                              double *srate)
{
    strain_eta(g, geo, par_of<double>(p), u, eta, srate);
}

extern "C" void og_flow_diagnostics(const og_grid *g, const og_geom *geo, const og_params *p, const double *u,
                                    double *lam, double *sdev)
{
    flow_diagnostics(g, geo, par_of<double>(p), u, lam, sdev);
}

extern "C" void og_cell_gradient(const og_grid *g, const og_geom *geo, const double *u, double *grad)
{
    cell_gradient(g, geo, u, grad);
}

extern "C" void og_cc_apply(const og_grid *g, const double *extra, const double *bx, const double *by,
                            const double *bz, const double *x, double *y)
{
    cc_apply(g, extra, bx, by, bz, x, y);
}

extern "C" int og_cc_solve(const og_grid *g, const double *extra, const double *bx, const double *by,
                           const double *bz, const double *b, double *x, double tol, int max_iters, double *res_out)
{
    return cc_solve(g, extra, bx, by, bz, b, x, tol, max_iters, res_out);
}

extern "C" void og_mac_coeffs(const og_grid *g, const og_geom *geo, double *extra, double *bx, double *by,
                              double *bz)
{
    mac_coeffs(g, geo, extra, bx, by, bz);
}

extern "C" void og_visc_coeffs(const og_grid *g, const og_geom *geo, const og_params *p, const double *eta, double dt,
                               int comp, double *extra, double *bx, double *by, double *bz, double *rhs_bc)
{
    visc_coeffs(g, geo, par_of<double>(p), eta, dt, comp, extra, bx, by, bz, rhs_bc);
}

extern "C" void og_nodal_apply(const og_grid *g, const og_geom *geo, double coef, const double *p, double *y)
{
    nodal_apply(g, geo, coef, p, y);
}

extern "C" void og_nodal_rhs(const og_grid *g, const og_geom *geo, const double *ut, double *rhs)
{
    nodal_rhs(g, geo, ut, rhs);
}

extern "C" int og_nodal_solve(const og_grid *g, const og_geom *geo, double coef, const double *b, double *p,
                              double tol, int max_iters, double *res_out)
{
    return nodal_solve(g, geo, coef, b, p, tol, max_iters, res_out);
}

extern "C" void og_cell_grad_p(const og_grid *g, const double *p, double *gp) { cell_grad_p(g, p, gp); }

extern "C" void og_face_states(const og_grid *g, const og_geom *geo, const double *u, double *uf)
{
    face_states(g, geo, u, uf);
}

extern "C" int og_mac_project(const og_grid *g, const og_geom *geo, double *uf, double *phi, double tol,
                              int max_iters, double *res_out)
{
    return mac_project(g, geo, uf, phi, tol, max_iters, res_out);
}

extern "C" void og_convective(const og_grid *g, const og_geom *geo, const double *u, const double *uf, double *C)
{
    convective(g, geo, u, uf, C);
}

extern "C" void og_redistribute(const og_grid *g, const og_geom *geo, const double *DC, double *D)
{
    redistribute(g, geo, DC, D);
}

extern "C" void og_viscous_explicit(const og_grid *g, const og_geom *geo, const og_params *p, const double *u,
                                    const double *eta, double *V)
{
    viscous_explicit(g, geo, par_of<double>(p), u, eta, V);
}

extern "C" double og_wall_dudn(const og_grid *g, const og_geom *geo, const double *u, int cell, int comp)
{
    return wall_dudn(g, geo, u, cell, comp);
}

extern "C" void og_derived(const og_grid *g, const og_geom *geo, const og_params *p, const double *u, double *C,
                           double *eta, double *V, double *srate, og_stats *st)
{
    derived(g, geo, par_of<double>(p), u, C, eta, V, srate, st);
}

/* Eqs. cfl:dt, cfl:convective, cfl:forcing, cfl:viscous:new. */
extern "C" double og_timestep(const og_grid *g, const og_geom *geo, const og_params *p, const double *u,
                              const double *f)
{
    size_t N3 = og_ncell(g);
    const double h = g->h;
    double cc = 0.0, cf2 = 0.0;
    for (size_t c = 0; c < N3; c++) {
        if (geo->alpha[c] <= 0.0) continue;
        double v = (fabs(u[c]) + fabs(u[N3 + c]) + fabs(u[2 * N3 + c])) / h;
        if (v > cc) cc = v;
        if (f) {
            double w = (fabs(f[c]) + fabs(f[N3 + c]) + fabs(f[2 * N3 + c])) / h;
            if (w > cf2) cf2 = w;
        }
    }
    double cv = 2.0 * p->mu / p->rho * (p->bi_cfl + 1.0) * (3.0 / (h * h));
    double ccv = cc + cv;
    return p->cfl / (0.5 * (ccv + sqrt(ccv * ccv + 4.0 * cf2)));
}

extern "C" int og_viscous_solve(const og_grid *g, const og_geom *geo, const og_params *p, const double *eta,
                                const double *psi, double dt, double *ut, og_stats *st, int slot)
{
    return viscous_solve(g, geo, par_of<double>(p), eta, psi, dt, ut, st, slot);
}

extern "C" int og_nodal_project(const og_grid *g, const og_geom *geo, const og_params *p, double dt, double *ut,
                                double *pres, og_stats *st, int slot)
{
    return nodal_project(g, geo, par_of<double>(p), dt, ut, pres, st, slot);
}

extern "C" void og_drag(const og_grid *g, const og_geom *geo, const og_params *p, const double *u,
                        const double *pres, double *fz, double *yield_frac)
{
    drag(g, geo, par_of<double>(p), u, pres, fz, yield_frac);
}

extern "C" int og_advance(const og_grid *g, const og_geom *geo, const og_params *p, double *u, double *pres,
                          double dt_in, const double *f, og_stats *st)
{
    double dt = dt_in > 0.0 ? dt_in : og_timestep(g, geo, p, u, f);
    advance(g, geo, par_of<double>(p), u, pres, dt, f, st, (double *)nullptr);
    return 0;
}

/* Forward-mode derivative of the time-averaged drag (the objective of the
 * drag sensitivities): J = (1/S) sum_{s=1..S} F_z(u_s, p_s) over S = steps
 * steps of Algorithm 1 from (u0, p0) at the fixed time step dt, with the
 * body force f (or none).  The whole run is made in dual numbers with
 * tau0 + dtau0 e, mu + dmu e and f + df e, so dJ is the exact directional
 * derivative of J along (dtau0, dmu, df). */
extern "C" int og_drag_tangent(const og_grid *g, const og_geom *geo, const og_params *p, const double *u0,
                               const double *p0, const double *f, const double *df, double dtau0, double dmu,
                               double dt, int steps, double *J, double *dJ)
{
    if (!(dt > 0.0) || steps < 1) return -1;
    size_t N3 = og_ncell(g), NN = og_nnode(g);
    Par<Dual> q = par_of<Dual>(p);
    q.tau0 = Dual(p->tau0, dtau0);
    q.mu = Dual(p->mu, dmu);
    vector<Dual> u(3 * N3), pr(NN), fd;
    for (size_t s = 0; s < 3 * N3; s++) u[s] = Dual(u0[s], 0.0);
    for (size_t s = 0; s < NN; s++) pr[s] = Dual(p0[s], 0.0);
    if (f || df) {
        fd.resize(3 * N3);
        for (size_t s = 0; s < 3 * N3; s++) fd[s] = Dual(f ? f[s] : 0.0, df ? df[s] : 0.0);
    }
    Dual acc = 0.0;
    for (int s = 0; s < steps; s++) {
        Dual fz;
        advance(g, geo, q, u.data(), pr.data(), dt, fd.empty() ? (const Dual *)nullptr : fd.data(),
                (og_stats *)nullptr, &fz);
        acc += fz;
    }
    acc /= Dual((double)steps);
    *J = acc.v;
    *dJ = acc.d;
    return 0;
}
