// EB geometry from an implicit function (paper Sec. "Embedded boundaries").
//
// The body surface is cut by each cell as a plane: phi is sampled at the grid
// nodes, every edge with a sign change gets its crossing by bisection, the
// face apertures are the fluid polygons of the faces, the EB area vector of a
// cell closes its fluid region (sum of outward area vectors is zero), the EB
// centroid is the area centroid of the crossing polygon, and the volume
// fraction follows from the divergence theorem with the EB plane through that
// centroid.  Two builders share these steps (the functions below run on the
// host and on the device alike): one evaluates a host callback on the host,
// the other runs on the device for bodies made of spheres, boxes and
// cylinders (their union).  Both hand the arrays to install_geometry; the
// steps are not timed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ebv_internal.cuh"

namespace ebv {
namespace {

__host__ __device__ inline bool fluid(double v) { return v > 0.0; }

__host__ __device__ inline void node_pos(const GridD &g, int i, int j, int k, double x[3])
{
    x[0] = g.lo[0] + i * g.h;
    x[1] = g.lo[1] + j * g.h;
    x[2] = g.lo[2] + k * g.h;
}

// Crossing on the segment P->Q (P, Q on opposite sides of the surface), as
// the fraction t from P, by bisection of the sign of phi.
template <class Phi>
__host__ __device__ double crossing(const Phi &phi, const double P[3], const double Q[3])
{
    double x[3], lo = 0.0, hi = 1.0;
    bool fp = fluid(phi(P));
    for (int it = 0; it < 200 && hi - lo > 1e-16; it++) {
        double m = 0.5 * (lo + hi);
        for (int d = 0; d < 3; d++) x[d] = P[d] + m * (Q[d] - P[d]);
        if (fluid(phi(x)) == fp) lo = m; else hi = m;
    }
    return 0.5 * (lo + hi);
}

// Edge arrays: edges along axis d have n[d] segments and n[e]+1 positions across.
__host__ __device__ inline int edge_index(const GridD &g, int d, int i, int j, int k)
{
    int mx = g.nx + (d != 0), my = g.ny + (d != 1);
    return (k * my + j) * mx + i;
}
__host__ __device__ inline int edge_count(const GridD &g, int d)
{
    return (g.nx + (d != 0)) * (g.ny + (d != 1)) * (g.nz + (d != 2));
}

// Fluid aperture of the face with normal d at (i,j,k): walk the square's
// corners (u along t1, v along t2), keep the fluid corners and the edge
// crossings, shoelace area.  nfl: node signs; et[e]: crossing fractions of
// the edges along e (NaN where none).
__host__ __device__ double face_aperture(const GridD &g, int d, int i, int j, int k, const uint8_t *nfl,
                                         const double *const *et)
{
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const int cu[4] = {0, 1, 1, 0}, cv[4] = {0, 0, 1, 1};
    bool f[4];
    int cnt = 0;
    for (int q = 0; q < 4; q++) {
        int id[3] = {i, j, k};
        id[t1] += cu[q];
        id[t2] += cv[q];
        f[q] = nfl[nidx(g, id[0], id[1], id[2])] != 0;
        cnt += f[q];
    }
    if (cnt == 4) return 1.0;
    if (cnt == 0) return 0.0;
    double pu[8], pv[8];
    int np = 0;
    for (int q = 0; q < 4; q++) {
        int q2 = (q + 1) & 3;
        if (f[q]) { pu[np] = cu[q]; pv[np] = cv[q]; np++; }
        if (f[q] == f[q2]) continue;
        // the edge between corners q and q2 runs along t1 (q even) or t2
        int ax = (q == 0 || q == 2) ? t1 : t2;
        int lo[3] = {i, j, k};
        lo[t1] += cu[q] < cu[q2] ? cu[q] : cu[q2];
        lo[t2] += cv[q] < cv[q2] ? cv[q] : cv[q2];
        double t = et[ax][edge_index(g, ax, lo[0], lo[1], lo[2])];
        double u0 = cu[q] < cu[q2] ? cu[q] : cu[q2], v0 = cv[q] < cv[q2] ? cv[q] : cv[q2];
        if (ax == t1) { pu[np] = u0 + t; pv[np] = v0; }
        else { pu[np] = u0; pv[np] = v0 + t; }
        np++;
    }
    double s = 0.0;
    for (int q = 0; q < np; q++) {
        int q2 = (q + 1) % np;
        s += pu[q] * pv[q2] - pu[q2] * pv[q];
    }
    double area = 0.5 * fabs(s);
    if (area < 1e-12) area = 0.0;
    if (area > 1.0 - 1e-12) area = 1.0;
    return area;
}

struct CellGeo {
    double alpha, area, n[3], b[3];
    uint8_t flag;
};

// Volume fraction, EB area, normal (into the fluid) and centroid (relative to
// the centre, units of h) and flag of cell (i,j,k) from the node signs, the
// edge crossings and the face apertures a[d].
__host__ __device__ CellGeo cell_geometry(const GridD &g, int i, int j, int k, const uint8_t *nfl,
                                          const double *const *et, const double *const *a)
{
    CellGeo r;
    r.alpha = 0.0; r.area = 0.0; r.flag = 0;
    for (int e = 0; e < 3; e++) { r.n[e] = 0.0; r.b[e] = 0.0; }
    int cnt = 0;
    for (int o = 0; o < 8; o++) cnt += nfl[nidx(g, i + (o & 1), j + ((o >> 1) & 1), k + ((o >> 2) & 1))] != 0;
    if (cnt == 8) { r.alpha = 1.0; r.flag = 1; return r; }
    if (cnt == 0) return r;
    double An[3], suma = 0.0;
    for (int d = 0; d < 3; d++) {
        int hi[3] = {i, j, k};
        hi[d] += 1;
        double alo = a[d][fidx(g, d, i, j, k)];
        double ahi = a[d][fidx(g, d, hi[0], hi[1], hi[2])];
        An[d] = ahi - alo;
        suma += alo + ahi;
    }
    double A = sqrt(An[0] * An[0] + An[1] * An[1] + An[2] * An[2]);
    if (A < 1e-12) {
        if (suma > 3.0) { r.alpha = 1.0; r.flag = 1; }
        return r;
    }
    double n[3] = {An[0] / A, An[1] / A, An[2] / A};
    // crossings of the 12 cell edges, relative to the centre (units of h)
    double ang[12], P[12][3];
    int np = 0;
    for (int d = 0; d < 3; d++)
        for (int o = 0; o < 4; o++) {
            int off[3] = {0, 0, 0};
            off[(d + 1) % 3] = o & 1;
            off[(d + 2) % 3] = o >> 1;
            double t = et[d][edge_index(g, d, i + off[0], j + off[1], k + off[2])];
            if (isnan(t)) continue;
            for (int e = 0; e < 3; e++) P[np][e] = off[e] - 0.5;
            P[np][d] += t;
            np++;
        }
    double M[3] = {0, 0, 0};
    for (int q = 0; q < np; q++)
        for (int e = 0; e < 3; e++) M[e] += P[q][e] / np;
    // in-plane basis: the axis least aligned with n, made orthogonal
    int amin = 0;
    for (int e = 1; e < 3; e++)
        if (fabs(n[e]) < fabs(n[amin])) amin = e;
    double e1[3] = {0, 0, 0}, e2[3];
    e1[amin] = 1.0;
    double tn = n[amin];
    for (int e = 0; e < 3; e++) e1[e] -= tn * n[e];
    double l = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int e = 0; e < 3; e++) e1[e] /= l;
    e2[0] = n[1] * e1[2] - n[2] * e1[1];
    e2[1] = n[2] * e1[0] - n[0] * e1[2];
    e2[2] = n[0] * e1[1] - n[1] * e1[0];
    for (int q = 0; q < np; q++) {
        double x = 0, y = 0;
        for (int e = 0; e < 3; e++) {
            x += (P[q][e] - M[e]) * e1[e];
            y += (P[q][e] - M[e]) * e2[e];
        }
        ang[q] = atan2(y, x);
    }
    // order the crossings by angle (insertion sort: stable, at most 12)
    for (int q = 1; q < np; q++) {
        double a0 = ang[q], p0[3] = {P[q][0], P[q][1], P[q][2]};
        int t = q - 1;
        while (t >= 0 && ang[t] > a0) {
            ang[t + 1] = ang[t];
            for (int e = 0; e < 3; e++) P[t + 1][e] = P[t][e];
            t--;
        }
        ang[t + 1] = a0;
        for (int e = 0; e < 3; e++) P[t + 1][e] = p0[e];
    }
    double bw = 0.0, bs[3] = {0, 0, 0};
    for (int q = 0; q < np; q++) {
        const double *A1 = P[q], *A2 = P[(q + 1) % np];
        double u1[3] = {A1[0] - M[0], A1[1] - M[1], A1[2] - M[2]};
        double u2[3] = {A2[0] - M[0], A2[1] - M[1], A2[2] - M[2]};
        double w = 0.5 * ((u1[1] * u2[2] - u1[2] * u2[1]) * n[0] + (u1[2] * u2[0] - u1[0] * u2[2]) * n[1] +
                          (u1[0] * u2[1] - u1[1] * u2[0]) * n[2]);
        for (int e = 0; e < 3; e++) bs[e] += w * (M[e] + A1[e] + A2[e]) / 3.0;
        bw += w;
    }
    double b[3];
    for (int e = 0; e < 3; e++) b[e] = fabs(bw) > 1e-300 ? bs[e] / bw : M[e];
    double al = (0.5 * suma - A * (b[0] * n[0] + b[1] * n[1] + b[2] * n[2])) / 3.0;
    if (al < 1e-12) al = 0.0;
    if (al > 1.0 - 1e-12) al = 1.0;
    r.alpha = al;
    if (al > 0.0) {
        r.flag = 2;
        r.area = A;
        for (int e = 0; e < 3; e++) { r.n[e] = n[e]; r.b[e] = b[e]; }
    }
    return r;
}

// ---- host builder: implicit function given as a host callback -----------------
struct HostPhi {
    ebv_implicit_fn fn;
    void *user;
    double operator()(const double x[3]) const { return fn(x, user); }
};

// ---- device builder: union of primitive bodies --------------------------------
// phi of one primitive, > 0 outside it (in the fluid): a sphere (centre, r),
// an axis-aligned box (low and high corners; its signed distance), or a
// circular cylinder along an axis (axis, the two other centre coordinates, r).
__host__ __device__ inline double prim_phi(const ebv_body &P, const double x[3])
{
    if (P.kind == EBV_BODY_SPHERE) {
        double dx = x[0] - P.q[0], dy = x[1] - P.q[1], dz = x[2] - P.q[2];
        return sqrt(dx * dx + dy * dy + dz * dz) - P.q[3];
    }
    if (P.kind == EBV_BODY_BOX) {
        double out = 0.0, in = -1e300;
        for (int d = 0; d < 3; d++) {
            double q = fmax(P.q[d] - x[d], x[d] - P.q[3 + d]);
            out += q > 0.0 ? q * q : 0.0;
            in = fmax(in, q);
        }
        return sqrt(out) + fmin(in, 0.0);
    }
    // cylinder: axis q[0] (0, 1, 2), centre (q[1], q[2]) in the two other axes, radius q[3]
    int ax = (int)P.q[0], a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    double d1 = x[a1] - P.q[1], d2 = x[a2] - P.q[2];
    return sqrt(d1 * d1 + d2 * d2) - P.q[3];
}

constexpr int kMaxBodies = 16;
struct Bodies {
    int n;
    ebv_body b[kMaxBodies];
    // the fluid is outside every body: phi = min over the bodies
    __host__ __device__ double operator()(const double x[3]) const
    {
        double v = prim_phi(b[0], x);
        for (int q = 1; q < n; q++) v = fmin(v, prim_phi(b[q], x));
        return v;
    }
};

__global__ void k_geo_nodes(GridD g, Bodies B, uint8_t *__restrict__ nfl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i > g.nx || j > g.ny || k > g.nz) return;
    double x[3];
    node_pos(g, i, j, k, x);
    nfl[nidx(g, i, j, k)] = fluid(B(x));
}

__global__ void k_geo_edges(GridD g, int d, Bodies B, const uint8_t *__restrict__ nfl, double *__restrict__ et)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= g.nx + (d != 0) || j >= g.ny + (d != 1) || k >= g.nz + (d != 2)) return;
    int hi[3] = {i, j, k};
    hi[d] += 1;
    double t = NAN;
    if (nfl[nidx(g, i, j, k)] != nfl[nidx(g, hi[0], hi[1], hi[2])]) {
        double P[3], Q[3];
        node_pos(g, i, j, k, P);
        node_pos(g, hi[0], hi[1], hi[2], Q);
        t = crossing(B, P, Q);
    }
    et[edge_index(g, d, i, j, k)] = t;
}

struct EdgePtrs {
    const double *e[3];
};
struct FacePtrs {
    double *a[3];
};

__global__ void k_geo_faces(GridD g, int d, const uint8_t *__restrict__ nfl, EdgePtrs E, double *__restrict__ a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= g.nx + (d == 0) || j >= g.ny + (d == 1) || k >= g.nz + (d == 2)) return;
    a[fidx(g, d, i, j, k)] = face_aperture(g, d, i, j, k, nfl, E.e);
}

__global__ void k_geo_cells(GridD g, const uint8_t *__restrict__ nfl, EdgePtrs E, FacePtrs F,
                            double *__restrict__ alpha, double *__restrict__ area, double *__restrict__ nrm,
                            double *__restrict__ bcen, uint8_t *__restrict__ flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    if (i >= g.nx || j >= g.ny || k >= g.nz) return;
    const double *af[3] = {F.a[0], F.a[1], F.a[2]};
    CellGeo r = cell_geometry(g, i, j, k, nfl, E.e, af);
    const int c = cidx(g, i, j, k), N3 = ncell(g);
    alpha[c] = r.alpha;
    area[c] = r.area;
    flag[c] = r.flag;
    for (int e = 0; e < 3; e++) {
        nrm[e * N3 + c] = r.n[e];
        bcen[e * N3 + c] = r.b[e];
    }
}

inline dim3 geo_grid(int mx, int my, int mz) { return dim3((mx + 31) / 32, (my + 3) / 4, (mz + 1) / 2); }

}  // namespace

ebv_status build_geometry_host(Ctx *c, ebv_implicit_fn fn, void *user)
{
    const GridD &g = c->g;
    HostPhi S{fn, user};
    const int NX = g.nx, NY = g.ny, NZ = g.nz;
    const size_t N3 = (size_t)NX * NY * NZ, NN = (size_t)nnode(g);

    // 1. node signs
    std::vector<uint8_t> nfl(NN);
    for (int k = 0; k <= NZ; k++)
        for (int j = 0; j <= NY; j++)
            for (int i = 0; i <= NX; i++) {
                double x[3];
                node_pos(g, i, j, k, x);
                nfl[nidx(g, i, j, k)] = fluid(S(x));
            }
    // 2. edge crossings, as the fraction from the low node (NaN: no crossing)
    std::vector<double> et[3];
    for (int d = 0; d < 3; d++) {
        et[d].assign(edge_count(g, d), NAN);
        int m[3] = {NX + (d != 0), NY + (d != 1), NZ + (d != 2)};
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    int hi[3] = {i, j, k};
                    hi[d] += 1;
                    if (nfl[nidx(g, i, j, k)] == nfl[nidx(g, hi[0], hi[1], hi[2])]) continue;
                    double P[3], Q[3];
                    node_pos(g, i, j, k, P);
                    node_pos(g, hi[0], hi[1], hi[2], Q);
                    et[d][edge_index(g, d, i, j, k)] = crossing(S, P, Q);
                }
    }
    const double *ep[3] = {et[0].data(), et[1].data(), et[2].data()};
    HostGeom H;
    // 3. face apertures
    for (int d = 0; d < 3; d++) {
        H.a[d].assign(nface(g, d), 0.0);
        int m[3] = {NX, NY, NZ};
        m[d] += 1;
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) H.a[d][fidx(g, d, i, j, k)] = face_aperture(g, d, i, j, k, nfl.data(), ep);
    }
    // 4. cells
    const double *ap[3] = {H.a[0].data(), H.a[1].data(), H.a[2].data()};
    H.alpha.assign(N3, 0.0);
    H.area.assign(N3, 0.0);
    H.nrm.assign(3 * N3, 0.0);
    H.bcen.assign(3 * N3, 0.0);
    H.flag.assign(N3, 0);
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                CellGeo r = cell_geometry(g, i, j, k, nfl.data(), ep, ap);
                H.alpha[c] = r.alpha;
                H.area[c] = r.area;
                H.flag[c] = r.flag;
                for (int e = 0; e < 3; e++) {
                    H.nrm[e * N3 + c] = r.n[e];
                    H.bcen[e * N3 + c] = r.b[e];
                }
                if (r.flag == 2) H.cut.push_back((int)c);
            }
    return install_geometry(c, H);
}

// The same steps on the device for a union of primitive bodies; the arrays
// are then read back for install_geometry (which derives the lists on the
// host).  Scratch: the node signs in c->kz, the edge crossings in c->ff.
ebv_status build_geometry_bodies(Ctx *c, int n, const ebv_body *bodies)
{
    if (n < 1 || n > kMaxBodies) return c->fail(EBV_ERR_INVALID, "between 1 and 16 bodies");
    Bodies B;
    B.n = n;
    for (int q = 0; q < n; q++) {
        const ebv_body &b = bodies[q];
        if (b.kind == EBV_BODY_SPHERE && !(b.q[3] > 0.0)) return c->fail(EBV_ERR_INVALID, "sphere radius must be > 0");
        if (b.kind == EBV_BODY_BOX && !(b.q[3] > b.q[0] && b.q[4] > b.q[1] && b.q[5] > b.q[2]))
            return c->fail(EBV_ERR_INVALID, "box corners must be ordered");
        if (b.kind == EBV_BODY_CYLINDER && (!(b.q[3] > 0.0) || !(b.q[0] == 0.0 || b.q[0] == 1.0 || b.q[0] == 2.0)))
            return c->fail(EBV_ERR_INVALID, "cylinder axis 0, 1 or 2 and radius > 0");
        if (b.kind < EBV_BODY_SPHERE || b.kind > EBV_BODY_CYLINDER) return c->fail(EBV_ERR_INVALID, "unknown body");
        B.b[q] = b;
    }
    const GridD &g = c->g;
    const size_t N3 = ncell(g), NN = nnode(g);
    uint8_t *nfl = (uint8_t *)c->kz;       // NN bytes <= vec_len doubles
    double *et[3];
    et[0] = c->ff;                          // 3 x (faces) doubles >= the three edge arrays
    et[1] = et[0] + edge_count(g, 0);
    et[2] = et[1] + edge_count(g, 1);
    EBV_LAUNCH(c, k_geo_nodes, geo_grid(g.nx + 1, g.ny + 1, g.nz + 1), dim3(32, 4, 2), 0, g, B, nfl);
    for (int d = 0; d < 3; d++)
        EBV_LAUNCH(c, k_geo_edges, geo_grid(g.nx + (d != 0), g.ny + (d != 1), g.nz + (d != 2)), dim3(32, 4, 2), 0, g,
                   d, B, nfl, et[d]);
    EdgePtrs E{{et[0], et[1], et[2]}};
    double *ad[3] = {c->ax, c->ay, c->az};
    for (int d = 0; d < 3; d++)
        EBV_LAUNCH(c, k_geo_faces, geo_grid(g.nx + (d == 0), g.ny + (d == 1), g.nz + (d == 2)), dim3(32, 4, 2), 0, g,
                   d, nfl, E, ad[d]);
    FacePtrs F{{c->ax, c->ay, c->az}};
    EBV_LAUNCH(c, k_geo_cells, geo_grid(g.nx, g.ny, g.nz), dim3(32, 4, 2), 0, g, nfl, E, F, c->alpha, c->area,
               c->nrm, c->bcen, c->flag);
    EBV_CUDA_TRY(c, cudaGetLastError());
    HostGeom H;
    H.alpha.resize(N3); H.area.resize(N3); H.nrm.resize(3 * N3); H.bcen.resize(3 * N3); H.flag.resize(N3);
    for (int d = 0; d < 3; d++) H.a[d].resize(nface(g, d));
    const double *src[7] = {c->alpha, c->ax, c->ay, c->az, c->area, c->nrm, c->bcen};
    std::vector<double> *dst[7] = {&H.alpha, &H.a[0], &H.a[1], &H.a[2], &H.area, &H.nrm, &H.bcen};
    for (int q = 0; q < 7; q++)
        EBV_CUDA_TRY(c, cudaMemcpyAsync(dst[q]->data(), src[q], dst[q]->size() * 8, cudaMemcpyDeviceToHost,
                                        c->stream));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(H.flag.data(), c->flag, N3, cudaMemcpyDeviceToHost, c->stream));
    EBV_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    (void)NN;
    for (size_t q = 0; q < N3; q++)
        if (H.flag[q] == 2) H.cut.push_back((int)q);
    return install_geometry(c, H);
}

// Checks the geometry, derives the cells next to the EB and uploads
// everything; shared by the builders and ebv_load_state.
ebv_status install_geometry(Ctx *c, HostGeom &H)
{
    const GridD &g = c->g;
    const int NX = g.nx, NY = g.ny, NZ = g.nz;
    const size_t N3 = (size_t)NX * NY * NZ;
    {
        size_t nfluid = 0;
        for (size_t q = 0; q < N3; q++) nfluid += H.flag[q] != 0;
        if (nfluid == 0) return c->fail(EBV_ERR_GEOMETRY, "the body covers every cell: no fluid left");
    }
    // the pressure reference of a box without outflow needs fluid at the x-
    // face of cell (0,0,0) (see pin_face)
    if (no_outflow(g) && !(H.a[0][fidx(g, 0, 0, 0, 0)] > 0.0))
        return c->fail(EBV_ERR_GEOMETRY, "a box without an outflow side needs fluid on the x- face of cell (0,0,0)");

    // 5. cells next to the EB: fluid cells that are cut or have a cut cell
    //    among their 26 neighbours (the only cells redistribution changes)
    std::vector<uint8_t> nearm(N3, 0);
    std::vector<int> nearl;
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c0 = cidx(g, i, j, k);
                if (H.flag[c0] == 0) continue;
                bool nb = false;
                for (int dk = -1; dk <= 1 && !nb; dk++)
                    for (int dj = -1; dj <= 1 && !nb; dj++)
                        for (int di = -1; di <= 1; di++) {
                            int ii = i + di, jj = j + dj, kk = k + dk;
                            if (ii < 0 || jj < 0 || kk < 0 || ii >= NX || jj >= NY || kk >= NZ) continue;
                            if (H.flag[cidx(g, ii, jj, kk)] == 2) { nb = true; break; }
                        }
                if (nb) {
                    nearm[c0] = 1;
                    nearl.push_back((int)c0);
                }
            }

    // 6. upload
    cudaStream_t s = c->stream;
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->nearm, nearm.data(), N3, cudaMemcpyHostToDevice, s));
    if (c->nearl) cudaFree(c->nearl);
    c->nearl = nullptr;
    c->nnear = (int)nearl.size();
    if (c->nnear) {
        EBV_CUDA_TRY(c, dev_malloc((void **)&c->nearl, c->nnear * sizeof(int)));
        EBV_CUDA_TRY(c, cudaMemcpyAsync(c->nearl, nearl.data(), c->nnear * sizeof(int),
                                        cudaMemcpyHostToDevice, s));
    }
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->alpha, H.alpha.data(), N3 * 8, cudaMemcpyHostToDevice, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->ax, H.a[0].data(), H.a[0].size() * 8, cudaMemcpyHostToDevice, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->ay, H.a[1].data(), H.a[1].size() * 8, cudaMemcpyHostToDevice, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->az, H.a[2].data(), H.a[2].size() * 8, cudaMemcpyHostToDevice, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->area, H.area.data(), N3 * 8, cudaMemcpyHostToDevice, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->nrm, H.nrm.data(), 3 * N3 * 8, cudaMemcpyHostToDevice, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->bcen, H.bcen.data(), 3 * N3 * 8, cudaMemcpyHostToDevice, s));
    EBV_CUDA_TRY(c, cudaMemcpyAsync(c->flag, H.flag.data(), N3, cudaMemcpyHostToDevice, s));
    if (c->cut) cudaFree(c->cut);
    c->cut = nullptr;
    c->ncut = (int)H.cut.size();
    if (c->dudn) cudaFree(c->dudn);
    c->dudn = nullptr;
    if (c->ncut) {
        EBV_CUDA_TRY(c, dev_malloc((void **)&c->cut, c->ncut * sizeof(int)));
        EBV_CUDA_TRY(c, dev_malloc((void **)&c->dudn, 3 * (size_t)c->ncut * sizeof(double)));
        EBV_CUDA_TRY(c, cudaMemcpyAsync(c->cut, H.cut.data(), c->ncut * sizeof(int),
                                        cudaMemcpyHostToDevice, s));
    }
    EBV_CUDA_TRY(c, cudaStreamSynchronize(s));
    c->have_geom = true;
    c->wall_col_ok = false;   // the wall-gradient adjoint's colouring follows the geometry
    return EBV_OK;
}

}  // namespace ebv
