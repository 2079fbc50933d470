/*
 * ebv_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU restatement of the embedded-boundary viscoplastic flow
 * step (Sverdrup, Almgren & Nikiforakis, arXiv:1905.07392).  It exists so the
 * tests can check the CUDA library against an independent implementation and
 * so the benchmark can time a CPU baseline.  The product path never links,
 * loads or calls it; it shares no code, header or table with the library.
 *
 * Layout: cell arrays are nx*ny*nz, x fastest.  x-face arrays are
 * (nx+1)*ny*nz, y-face nx*(ny+1)*nz, z-face nx*ny*(nz+1).  Node arrays are
 * (nx+1)*(ny+1)*(nz+1).  Vector cell fields are three consecutive components
 * (SoA).  Cells are cubes of side h; the box starts at lo.
 *
 * Parity notes: every elliptic solution is defined as the exact solution of
 * its discrete system; the oracle reaches it with Jacobi-preconditioned CG.
 *
 * The implementation (ebv_oracle.cpp) is C++ with C linkage for every entry
 * point below; its flow arithmetic is written once for a generic scalar and
 * instantiated in double and in forward-mode dual numbers (og_drag_tangent).
 */
#ifndef EBV_ORACLE_H
#define EBV_ORACLE_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Domain side types (sides ordered x-, x+, y-, y+, z-, z+). */
enum { OG_INFLOW = 0, OG_OUTFLOW = 1, OG_SLIP = 2, OG_NOSLIP = 3 };
/* Rheology (Table "Generalised Newtonian fluid models"). */
enum { OG_NEWTONIAN = 0, OG_BINGHAM = 1, OG_HB = 2, OG_POWERLAW = 3, OG_SMD = 4 };
/* Implicit functions (fluid where phi > 0). */
enum { OG_SHAPE_NONE = 0, OG_SHAPE_SPHERE = 1, OG_SHAPE_PLANE = 2, OG_SHAPE_UNION = 3 };
/* Bodies of OG_SHAPE_UNION (the fluid is outside all of them):
 * sphere: centre, radius; box: low and high corners (axis-aligned);
 * cylinder: axis, centre in the two other axes ((axis+1)%3, (axis+2)%3), radius. */
enum { OG_BODY_SPHERE = 0, OG_BODY_BOX = 1, OG_BODY_CYLINDER = 2 };

typedef struct {
    int n[3];
    double lo[3];
    double h;
    int bc[6];
    double u_in[3];
} og_grid;

typedef struct {
    double rho, mu, tau0, m, n_flow, eta0; /* mu is kappa for HB / power law */
    int model;
    double cfl;
    double bi_cfl;      /* Bingham number entering the viscous CFL limit */
    double tol;         /* relative residual for every linear solve */
    int max_iters;
    double delta_min;   /* lower bound of wall distance (cell units) in the implicit EB term */
    int advect;         /* 1: Algorithm 1 as printed; 0: creeping flow, convective term C = 0 */
} og_params;

typedef struct {
    int kind;
    double p[8];        /* sphere: cx,cy,cz,r ; plane: nx,ny,nz,d (fluid where n.x > d) */
    int nbody;          /* OG_SHAPE_UNION: number of bodies (<= 16) */
    int bkind[16];
    double bq[16][6];
} og_shape;

typedef struct {
    double *alpha;          /* volume fraction, N3 */
    double *ax, *ay, *az;   /* face aperture fractions */
    double *area;           /* EB area / h^2, N3 */
    double *nrm;            /* EB unit normal into the fluid, 3*N3 */
    double *bcen;           /* EB centroid relative to cell centre, in units of h, 3*N3 */
    unsigned char *flag;    /* 0 covered, 1 regular, 2 cut */
} og_geom;

typedef struct {
    double dt, drag, yield_frac;
    int iters[10];
    double res[10];
} og_stats;

double og_phi(const og_shape *s, const double x[3]);
void og_build_geometry(const og_grid *g, const og_shape *s, og_geom *geo);

/* Rate of strain magnitude and apparent viscosity (fused step a6). */
double og_eta_of(const og_params *p, double sr);
void og_strain_eta(const og_grid *g, const og_geom *geo, const og_params *p,
                   const double *u, double *eta, double *srate);
/* Flow topology parameter Lambda (Eq. ryovar) and yield-stress deviation
 * eta ||g|| / tau0 - 1 per cell (Sec. "Cylinder moving through Bingham fluid"). */
void og_flow_diagnostics(const og_grid *g, const og_geom *geo, const og_params *p, const double *u,
                         double *lam, double *sdev);
void og_cell_gradient(const og_grid *g, const og_geom *geo, const double *u,
                      double *grad /* 9*N3: grad[(3*d+c)*N3+cell] = du_c/dx_d */);

/* Generic cell-centred operator  (A x)_i = extra_i x_i + sum_faces beta_f (x_i - x_nb). */
void og_cc_apply(const og_grid *g, const double *extra, const double *bx, const double *by,
                 const double *bz, const double *x, double *y);
int og_cc_solve(const og_grid *g, const double *extra, const double *bx, const double *by,
                const double *bz, const double *b, double *x, double tol, int max_iters,
                double *res_out);
void og_mac_coeffs(const og_grid *g, const og_geom *geo, double *extra, double *bx,
                   double *by, double *bz);
void og_visc_coeffs(const og_grid *g, const og_geom *geo, const og_params *p, const double *eta,
                    double dt, int comp, double *extra, double *bx, double *by, double *bz,
                    double *rhs_bc /* N3, Dirichlet contributions, may be NULL */);

/* Nodal operator, divergence and cell gradient (step a10). */
void og_nodal_apply(const og_grid *g, const og_geom *geo, double coef, const double *p,
                    double *y);
void og_nodal_rhs(const og_grid *g, const og_geom *geo, const double *ut, double *rhs);
int og_nodal_solve(const og_grid *g, const og_geom *geo, double coef, const double *b,
                   double *p, double tol, int max_iters, double *res_out);
void og_cell_grad_p(const og_grid *g, const double *p, double *gp /* 3*N3 */);

/* Derived quantities (Algorithm 2) and their parts. */
void og_face_states(const og_grid *g, const og_geom *geo, const double *u,
                    double *uf /* normal face velocities, 3 face arrays concatenated */);
int og_mac_project(const og_grid *g, const og_geom *geo, double *uf, double *phi, double tol,
                   int max_iters, double *res_out);
void og_convective(const og_grid *g, const og_geom *geo, const double *u, const double *uf,
                   double *C);
void og_redistribute(const og_grid *g, const og_geom *geo, const double *DC, double *D);
void og_viscous_explicit(const og_grid *g, const og_geom *geo, const og_params *p,
                         const double *u, const double *eta, double *V);
double og_wall_dudn(const og_grid *g, const og_geom *geo, const double *u, int cell, int comp);
void og_derived(const og_grid *g, const og_geom *geo, const og_params *p, const double *u,
                double *C, double *eta, double *V, double *srate, og_stats *st);

double og_timestep(const og_grid *g, const og_geom *geo, const og_params *p, const double *u,
                   const double *f);
int og_viscous_solve(const og_grid *g, const og_geom *geo, const og_params *p, const double *eta,
                     const double *psi, double dt, double *ut, og_stats *st, int slot);
int og_nodal_project(const og_grid *g, const og_geom *geo, const og_params *p, double dt,
                     double *ut, double *pres, og_stats *st, int slot);
int og_advance(const og_grid *g, const og_geom *geo, const og_params *p, double *u, double *pres,
               double dt_in, const double *f, og_stats *st);
void og_drag(const og_grid *g, const og_geom *geo, const og_params *p, const double *u,
             const double *pres, double *fz, double *yield_frac);

/* Forward-mode (dual-number) derivative of J = (1/steps) sum_{s=1..steps}
 * F_z(u_s, p_s), the drag of Eq. drag-force averaged over `steps` steps of
 * Algorithm 1 from (u0, p0) at the fixed time step dt > 0 with body force f
 * (3*N3 or NULL), along the direction tau0 += dtau0, mu += dmu, f += df (df
 * 3*N3 or NULL).  Writes J and its exact directional derivative dJ; returns
 * 0, or -1 for dt <= 0 or steps < 1. */
int og_drag_tangent(const og_grid *g, const og_geom *geo, const og_params *p, const double *u0,
                    const double *p0, const double *f, const double *df, double dtau0, double dmu,
                    double dt, int steps, double *J, double *dJ);

size_t og_ncell(const og_grid *g);
size_t og_nnode(const og_grid *g);
/* Threads the oracle's loops run on (its OpenMP team size; 1 without OpenMP). */
int og_threads(void);

#ifdef __cplusplus
}
#endif
#endif
