// EB geometry from an implicit function (paper Sec. "Embedded boundaries").
//
// The body surface is cut by each cell as a plane: phi is sampled at the grid
// nodes, every edge with a sign change gets its crossing by bisection, the
// face apertures are the fluid polygons of the faces, the EB area vector of a
// cell closes its fluid region (sum of outward area vectors is zero), the EB
// centroid is the area centroid of the crossing polygon, and the volume
// fraction follows from the divergence theorem with the EB plane through that
// centroid.  Runs once per geometry on the host (the implicit function is a
// host callback) and uploads the arrays; the steps are not timed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ebv_internal.cuh"

namespace ebv {
namespace {

struct HostGeom {
    std::vector<double> alpha, a[3], area, nrm, bcen;
    std::vector<uint8_t> flag;
    std::vector<int> cut;
};

inline bool fluid(double v) { return v > 0.0; }

struct Sampler {
    const GridD &g;
    ebv_implicit_fn fn;
    void *user;
    double eval(const double x[3]) const { return fn(x, user); }
    void node(int i, int j, int k, double x[3]) const
    {
        x[0] = g.lo[0] + i * g.h;
        x[1] = g.lo[1] + j * g.h;
        x[2] = g.lo[2] + k * g.h;
    }
    // Crossing on the segment P->Q (P, Q on opposite sides), as the fraction t.
    double crossing(const double P[3], const double Q[3]) const
    {
        double x[3], lo = 0.0, hi = 1.0;
        bool fp = fluid(eval(P));
        for (int it = 0; it < 200 && hi - lo > 1e-16; it++) {
            double m = 0.5 * (lo + hi);
            for (int d = 0; d < 3; d++) x[d] = P[d] + m * (Q[d] - P[d]);
            if (fluid(eval(x)) == fp) lo = m; else hi = m;
        }
        return 0.5 * (lo + hi);
    }
};

// Edge arrays: edges along axis d have n[d] segments and n[e]+1 positions across.
inline int edge_index(const GridD &g, int d, int i, int j, int k)
{
    int mx = g.nx + (d != 0), my = g.ny + (d != 1);
    return (k * my + j) * mx + i;
}
inline int edge_count(const GridD &g, int d)
{
    return (g.nx + (d != 0)) * (g.ny + (d != 1)) * (g.nz + (d != 2));
}

}  // namespace

ebv_status build_geometry_host(Ctx *c, ebv_implicit_fn fn, void *user)
{
    const GridD &g = c->g;
    Sampler S{g, fn, user};
    const int NX = g.nx, NY = g.ny, NZ = g.nz;
    const size_t N3 = (size_t)NX * NY * NZ, NN = (size_t)nnode(g);

    // 1. node values and fluid signs
    std::vector<double> phi(NN);
    std::vector<uint8_t> nfl(NN);
    for (int k = 0; k <= NZ; k++)
        for (int j = 0; j <= NY; j++)
            for (int i = 0; i <= NX; i++) {
                double x[3];
                S.node(i, j, k, x);
                size_t n = nidx(g, i, j, k);
                phi[n] = S.eval(x);
                nfl[n] = fluid(phi[n]);
            }
    auto nf = [&](int i, int j, int k) { return nfl[nidx(g, i, j, k)] != 0; };

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
                    if (nf(i, j, k) == nf(hi[0], hi[1], hi[2])) continue;
                    double P[3], Q[3];
                    S.node(i, j, k, P);
                    S.node(hi[0], hi[1], hi[2], Q);
                    et[d][edge_index(g, d, i, j, k)] = S.crossing(P, Q);
                }
    }

    HostGeom H;
    // 3. face apertures: walk the square's corners (u along t1, v along t2),
    //    keep fluid corners and edge crossings, shoelace area.
    for (int d = 0; d < 3; d++) {
        const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
        H.a[d].assign(nface(g, d), 0.0);
        int m[3] = {NX, NY, NZ};
        m[d] += 1;
        for (int k = 0; k < m[2]; k++)
            for (int j = 0; j < m[1]; j++)
                for (int i = 0; i < m[0]; i++) {
                    const int cu[4] = {0, 1, 1, 0}, cv[4] = {0, 0, 1, 1};
                    bool f[4];
                    int cnt = 0;
                    for (int q = 0; q < 4; q++) {
                        int id[3] = {i, j, k};
                        id[t1] += cu[q];
                        id[t2] += cv[q];
                        f[q] = nf(id[0], id[1], id[2]);
                        cnt += f[q];
                    }
                    double area;
                    if (cnt == 4) area = 1.0;
                    else if (cnt == 0) area = 0.0;
                    else {
                        double pu[8], pv[8];
                        int np = 0;
                        for (int q = 0; q < 4; q++) {
                            int q2 = (q + 1) & 3;
                            if (f[q]) { pu[np] = cu[q]; pv[np] = cv[q]; np++; }
                            if (f[q] == f[q2]) continue;
                            // the edge between corners q and q2 runs along t1 (q even) or t2
                            int ax = (q == 0 || q == 2) ? t1 : t2;
                            int lo[3] = {i, j, k};
                            lo[t1] += std::min(cu[q], cu[q2]);
                            lo[t2] += std::min(cv[q], cv[q2]);
                            double t = et[ax][edge_index(g, ax, lo[0], lo[1], lo[2])];
                            double u0 = std::min(cu[q], cu[q2]), v0 = std::min(cv[q], cv[q2]);
                            if (ax == t1) { pu[np] = u0 + t; pv[np] = v0; }
                            else { pu[np] = u0; pv[np] = v0 + t; }
                            np++;
                        }
                        double s = 0.0;
                        for (int q = 0; q < np; q++) {
                            int q2 = (q + 1) % np;
                            s += pu[q] * pv[q2] - pu[q2] * pv[q];
                        }
                        area = 0.5 * fabs(s);
                        if (area < 1e-12) area = 0.0;
                        if (area > 1.0 - 1e-12) area = 1.0;
                    }
                    H.a[d][fidx(g, d, i, j, k)] = area;
                }
    }

    // 4. cells
    H.alpha.assign(N3, 0.0);
    H.area.assign(N3, 0.0);
    H.nrm.assign(3 * N3, 0.0);
    H.bcen.assign(3 * N3, 0.0);
    H.flag.assign(N3, 0);
    for (int k = 0; k < NZ; k++)
        for (int j = 0; j < NY; j++)
            for (int i = 0; i < NX; i++) {
                size_t c = cidx(g, i, j, k);
                int cnt = 0;
                for (int o = 0; o < 8; o++) cnt += nf(i + (o & 1), j + ((o >> 1) & 1), k + ((o >> 2) & 1));
                if (cnt == 8) { H.alpha[c] = 1.0; H.flag[c] = 1; continue; }
                if (cnt == 0) continue;
                double An[3], suma = 0.0;
                for (int d = 0; d < 3; d++) {
                    int hi[3] = {i, j, k};
                    hi[d] += 1;
                    double alo = H.a[d][fidx(g, d, i, j, k)];
                    double ahi = H.a[d][fidx(g, d, hi[0], hi[1], hi[2])];
                    An[d] = ahi - alo;
                    suma += alo + ahi;
                }
                double A = sqrt(An[0] * An[0] + An[1] * An[1] + An[2] * An[2]);
                if (A < 1e-12) {
                    if (suma > 3.0) { H.alpha[c] = 1.0; H.flag[c] = 1; }
                    continue;
                }
                double n[3] = {An[0] / A, An[1] / A, An[2] / A};
                // crossings of the 12 cell edges, relative to the centre (units of h)
                struct Pt { double ang, p[3]; };
                Pt P[12];
                int np = 0;
                for (int d = 0; d < 3; d++)
                    for (int o = 0; o < 4; o++) {
                        int off[3] = {0, 0, 0};
                        off[(d + 1) % 3] = o & 1;
                        off[(d + 2) % 3] = o >> 1;
                        double t = et[d][edge_index(g, d, i + off[0], j + off[1], k + off[2])];
                        if (std::isnan(t)) continue;
                        for (int e = 0; e < 3; e++) P[np].p[e] = off[e] - 0.5;
                        P[np].p[d] += t;
                        np++;
                    }
                double M[3] = {0, 0, 0};
                for (int q = 0; q < np; q++)
                    for (int e = 0; e < 3; e++) M[e] += P[q].p[e] / np;
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
                        x += (P[q].p[e] - M[e]) * e1[e];
                        y += (P[q].p[e] - M[e]) * e2[e];
                    }
                    P[q].ang = atan2(y, x);
                }
                std::stable_sort(P, P + np, [](const Pt &a, const Pt &b) { return a.ang < b.ang; });
                double bw = 0.0, bs[3] = {0, 0, 0};
                for (int q = 0; q < np; q++) {
                    const double *A1 = P[q].p, *A2 = P[(q + 1) % np].p;
                    double u1[3] = {A1[0] - M[0], A1[1] - M[1], A1[2] - M[2]};
                    double u2[3] = {A2[0] - M[0], A2[1] - M[1], A2[2] - M[2]};
                    double w = 0.5 * ((u1[1] * u2[2] - u1[2] * u2[1]) * n[0] +
                                      (u1[2] * u2[0] - u1[0] * u2[2]) * n[1] +
                                      (u1[0] * u2[1] - u1[1] * u2[0]) * n[2]);
                    for (int e = 0; e < 3; e++) bs[e] += w * (M[e] + A1[e] + A2[e]) / 3.0;
                    bw += w;
                }
                double b[3];
                for (int e = 0; e < 3; e++) b[e] = fabs(bw) > 1e-300 ? bs[e] / bw : M[e];
                double al = (0.5 * suma - A * (b[0] * n[0] + b[1] * n[1] + b[2] * n[2])) / 3.0;
                if (al < 1e-12) al = 0.0;
                if (al > 1.0 - 1e-12) al = 1.0;
                H.alpha[c] = al;
                if (al > 0.0) {
                    H.flag[c] = 2;
                    H.area[c] = A;
                    for (int e = 0; e < 3; e++) {
                        H.nrm[e * N3 + c] = n[e];
                        H.bcen[e * N3 + c] = b[e];
                    }
                    H.cut.push_back((int)c);
                }
            }

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
        EBV_CUDA_TRY(c, cudaMalloc(&c->nearl, c->nnear * sizeof(int)));
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
        EBV_CUDA_TRY(c, cudaMalloc(&c->cut, c->ncut * sizeof(int)));
        EBV_CUDA_TRY(c, cudaMalloc(&c->dudn, 3 * (size_t)c->ncut * sizeof(double)));
        EBV_CUDA_TRY(c, cudaMemcpyAsync(c->cut, H.cut.data(), c->ncut * sizeof(int),
                                        cudaMemcpyHostToDevice, s));
    }
    EBV_CUDA_TRY(c, cudaStreamSynchronize(s));
    c->have_geom = true;
    return EBV_OK;
}

}  // namespace ebv
