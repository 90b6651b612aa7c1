/*
 * fvlbm_oracle.c -- plain, slow, double-precision CPU oracle of the time step of the
 * simplified finite-volume lattice Boltzmann method with k-omega SST and three-stage IMEX
 * Runge-Kutta (Wang, Zhong, Cao, Zhuo, arXiv 1812.00394, Part II).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load this file.  It shares no code, header, table or helper with the CUDA
 * library; the product path never calls it.
 *
 * Each function restates one passage of the paper, cell by cell, in the paper's order and
 * notation, in FP64, without blocking, fusion or reordering:
 *   feq()            D2Q9 equilibrium (Sec. 3.1 names D2Q9 of Qian et al.; form of Part I)
 *   lsq_gradient()   cell gradient of a field (Sec. 3.2 Step 2; method of Part I)
 *   boundary_f()     face values f_{alpha,bc} on boundary faces (Step 2; Part I)
 *   convection()     Gamma^a of Eq. (advection)
 *   imex_step()      Eqs. (imexone), (imextwo) with the tableau of Sec. 3.1, the moment
 *                    elimination of Eqs. (sumimeximplicitnew) and (fnewstage)
 *   sst_update()     Sec. 2 (k-omega SST), discretised per Eq. (SSTequint); tau by
 *                    Eq. (turbtau); coupled once per step before the stages (Step 1)
 *   forces()         momentum flux through wall faces -> C_D, C_L, Cp (Sec. 4.3 table)
 *   euler_step()     the explicit Euler scheme of Part I, for the comparison of Sec. 4.1
 *
 * Where Part I (not available) or the text is silent, the reading taken is stated beside the
 * code; each is listed with its reason in the design notes of this repository.
 *
 * Parity status.
 *   - Pinned by tests against closed forms and invariants: f^eq, the IMEX tableau, the moment
 *     elimination, the gradient, the flux, the wall boundary, mass conservation, Couette flow
 *     and the SST point functions.
 *   - Pinned on tiny meshes against an independent NumPy restatement of the same equations:
 *     one whole step, laminar and turbulent, with every boundary kind.
 *   - Unpinned: the turbulent cases as a whole (the inlet, outlet and far-field readings
 *     together with SST transport) have no closed form, so the readings themselves stay
 *     unpinned beyond those checks.
 *
 * Built with ORACLE_COMPLEX_STEP, the same source is the oracle's own tangent (complex-step
 * method, see `real` below); its real parts equal the double build's values exactly, and its
 * derivatives are pinned against central differences of the double build (laminar cavity; SST
 * step and airfoil from a developed state).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Threads of the per-cell loops (1 unless oracle_set_threads asks for more, and only in a
 * build with OpenMP).  Every loop so marked writes per-cell results from per-cell arithmetic
 * in the same order as the serial loop, so the results are bitwise the same for any thread
 * count; sums over cells (residual, mass) stay serial. */
static int g_threads = 1;
void oracle_set_threads(int n) { g_threads = n > 0 ? n : 1; }
#ifdef _OPENMP
#define OMP_FOR _Pragma("omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)")
#define OMP_FOR_MAX_DEFECT \
    _Pragma("omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1) reduction(max : defect)")
#else
#define OMP_FOR
#define OMP_FOR_MAX_DEFECT
#endif

/* The state arithmetic (f, the macros, k, omega, nu_t, tau, the boundary values and every
 * quantity formed from them) is done in the type `real`: double, or -- when this file is
 * compiled with ORACLE_COMPLEX_STEP -- double complex, for the complex-step derivative of the
 * step (Squire and Trapp 1998): with the inputs seeded as x + i h d, every analytic operation
 * carries f(x) + i h f'(x) d + O(h^2), so Im(J)/h is the directional derivative of J to
 * rounding, with no difference taken.  Branches (upwind choice, limiters, clips, min / max)
 * act on real parts, so the derivative is that of the branch the value takes; sqrt uses its
 * first-order rule with derivative 0 at 0, the convention of the GPU tangent.  The geometry
 * stays double.  In the double build every expression is the one the plain oracle evaluates. */
#ifdef ORACLE_COMPLEX_STEP
#include <complex.h>
typedef double complex real;
#define RE(x) creal(x)
static real rsqrt(real x)
{
    double v = creal(x), s = v > 0.0 ? sqrt(v) : 0.0;
    return s > 0.0 ? s + I * (cimag(x) / (2.0 * s)) : 0.0;
}
#define rtanh(x) ctanh(x)
#else
typedef double real;
#define RE(x) (x)
#define rsqrt(x) sqrt(x)
#define rtanh(x) tanh(x)
#endif
/* min / max of two reals by value, keeping the first argument on ties */
static real rmin(real a, real b) { return RE(b) < RE(a) ? b : a; }
static real rmax(real a, real b) { return RE(b) > RE(a) ? b : a; }

#define Q 9
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* D2Q9 velocities e_alpha and weights w_alpha (Part I reading): rest, 4 axis, 4 diagonal. */
static const double EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const double EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 of D2Q9 (text under Eq. turbtau) */

/* IMEX tableau, Sec. 3.1: explicit mt[J][k], implicit m[J][k], weights nt[J], n[J]. */
static const double MT[3][3] = {{0, 0, 0}, {0.5, 0, 0}, {0.5, 0.5, 0}};
static const double MI[3][3] = {{0.25, 0, 0}, {0, 0.25, 0}, {1.0 / 3, 1.0 / 3, 1.0 / 3}};
static const double NT[3] = {1.0 / 3, 1.0 / 3, 1.0 / 3};
static const double NI[3] = {1.0 / 3, 1.0 / 3, 1.0 / 3};

/* SST constants listed after the f2 definition in Sec. 2. */
static const double A1 = 0.31, BSTAR = 0.09, KAPPA = 0.41;
static const double SK1 = 0.85, SW1 = 0.5, B1 = 0.075;
static const double SK2 = 1.0, SW2 = 0.856, B2 = 0.0828;

enum { BC_WALL = 0, BC_INLET = 1, BC_OUTLET = 2, BC_FARFIELD = 3, BC_PERIODIC = 4 };

typedef struct {
    int nbr;        /* neighbour cell, or -1 on a boundary face */
    int bedge;      /* boundary edge when nbr == -1 */
    double nx, ny;  /* unit normal out of this cell */
    double len;     /* Delta l */
    double xm, ym;  /* face midpoint */
    double sx, sy;  /* neighbour centroid seen from this cell = centroid(nbr) + (sx, sy) */
} oface;

typedef struct oracle {
    int nc, nb;
    int *nface;
    oface *face;                 /* [nc * 4] */
    double *area, *cx, *cy, *wdist;
    int *btype, *bcell;
    real *bval;                  /* [nb * 5]: rho_b, u_b, v_b, k_b, omega_b */
    double *bxm, *bym, *bnx, *bny, *blen;
    double nu, rho0, dt, uref, lref, alpha_deg;
    double *dtc;                 /* local time stepping: dt of each cell (NULL: dt everywhere) */
    int variant;                 /* reading variants (bit mask): 1 limiter on the gradient of f,
                                    2 non-orthogonal correction of the SST diffusion, 4 SST
                                    re-solved before every stage, 8 production limiter */
    int sst;
    int scheme;                  /* 0: IMEX Runge-Kutta (Part II); 1: explicit Euler (Part I) */
    real *f;                     /* [nc * Q], cell-major */
    real *rho, *ux, *uy, *k, *om, *nut, *tau;
    double residual, moment_defect;
    long steps;
    /* work arrays */
    real *fn, *fst, *ga[3], *gc[3], *gradf, *fbc, *feqs, *X;
    real *gu, *gv, *gk, *gw, *rk, *rw, *f1, *Sabs;
} oracle;

/* Time step of cell i: its own under local time stepping, else the global one. */
static double cell_dt(const struct oracle *o, int i) { return o->dtc ? o->dtc[i] : o->dt; }

/* ------------------------------------------------------------------ equilibrium */
/* f^eq_alpha(rho, u) = w_alpha rho [1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u]: the second-order
 * D2Q9 equilibrium with c = 1 (Part I; Sec. 3.1 names the lattice). */
static void feq_r(real rho, real u, real v, real *feq)
{
    real uu = u * u + v * v;
    for (int a = 0; a < Q; a++) {
        real eu = EX[a] * u + EY[a] * v;
        feq[a] = WQ[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}
#ifndef ORACLE_COMPLEX_STEP
void oracle_feq(double rho, double u, double v, double *feq) { feq_r(rho, u, v, feq); }
#endif

/* rho = sum_alpha f_alpha, rho u = sum_alpha e_alpha f_alpha (collision invariants). */
static void moments(const real *f, real *rho, real *u, real *v)
{
    real r = 0, mx = 0, my = 0;
    for (int a = 0; a < Q; a++) {
        r += f[a];
        mx += EX[a] * f[a];
        my += EY[a] * f[a];
    }
    *rho = r;
    *u = mx / r;
    *v = my / r;
}

/* ------------------------------------------------------------------ mesh */
typedef struct { long long key; int cell, local; } edge_rec;

static int cmp_edge(const void *a, const void *b)
{
    long long x = ((const edge_rec *)a)->key, y = ((const edge_rec *)b)->key;
    return (x > y) - (x < y);
}

static long long edge_key(int a, int b)
{
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return ((long long)lo << 32) | (long long)(unsigned)hi;
}

static double seg_dist(double px, double py, double ax, double ay, double bx, double by)
{
    double dx = bx - ax, dy = by - ay;
    double t = ((px - ax) * dx + (py - ay) * dy) / (dx * dx + dy * dy);
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    double qx = ax + t * dx - px, qy = ay + t * dy - py;
    return sqrt(qx * qx + qy * qy);
}

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

void oracle_destroy(oracle *o);

/* params: [nu, rho0, dt, cfl, sst, uref, lref, alpha_deg, scheme, local_dt, variant] */
oracle *oracle_create(int n_nodes, const double *xy, int n_cells, const int *cell_ptr,
                      const int *cell_nodes, int n_bedges, const int *bedge_nodes,
                      const int *bedge_type, const double *bedge_val, int n_periodic,
                      const int *periodic_pairs, const double *periodic_shift,
                      const double *rho_init, const double *u_init, const double *v_init,
                      const double *k_init, const double *w_init, const double *params)
{
    (void)n_nodes;
    oracle *o = (oracle *)calloc(1, sizeof(oracle));
    int nc = n_cells, nb = n_bedges;
    o->nc = nc;
    o->nb = nb;
    o->nu = params[0];
    o->rho0 = params[1];
    o->dt = params[2];
    double cfl = params[3];
    o->sst = params[4] != 0.0;
    o->uref = params[5];
    o->lref = params[6];
    o->alpha_deg = params[7];
    o->scheme = (int)params[8];
    int local_dt = params[9] != 0.0;
    o->variant = (int)params[10];
    if (local_dt && !(cfl > 0.0)) { /* local steps are CFL * the cell's limit: need a CFL */
        free(o);
        return NULL;
    }

    o->nface = (int *)xcalloc(nc, sizeof(int));
    o->face = (oface *)xcalloc((size_t)nc * 4, sizeof(oface));
    o->area = (double *)xcalloc(nc, sizeof(double));
    o->cx = (double *)xcalloc(nc, sizeof(double));
    o->cy = (double *)xcalloc(nc, sizeof(double));
    o->wdist = (double *)xcalloc(nc, sizeof(double));
    o->btype = (int *)xcalloc(nb, sizeof(int));
    o->bcell = (int *)xcalloc(nb, sizeof(int));
    o->bval = (real *)xcalloc((size_t)nb * 5, sizeof(real));
    o->bxm = (double *)xcalloc(nb, sizeof(double));
    o->bym = (double *)xcalloc(nb, sizeof(double));
    o->bnx = (double *)xcalloc(nb, sizeof(double));
    o->bny = (double *)xcalloc(nb, sizeof(double));
    o->blen = (double *)xcalloc(nb, sizeof(double));
    memcpy(o->btype, bedge_type, sizeof(int) * (size_t)nb);
    for (size_t q = 0; q < 5 * (size_t)nb; q++) o->bval[q] = bedge_val[q];

    /* cell area and centroid (polygon formulas, taken relative to the first node) */
    for (int i = 0; i < nc; i++) {
        int p0 = cell_ptr[i], nv = cell_ptr[i + 1] - p0;
        double x0 = xy[2 * cell_nodes[p0]], y0 = xy[2 * cell_nodes[p0] + 1];
        double A2 = 0, sx = 0, sy = 0;
        for (int l = 0; l < nv; l++) {
            int a = cell_nodes[p0 + l], b = cell_nodes[p0 + (l + 1) % nv];
            double xa = xy[2 * a] - x0, ya = xy[2 * a + 1] - y0;
            double xb = xy[2 * b] - x0, yb = xy[2 * b + 1] - y0;
            double cr = xa * yb - xb * ya;
            A2 += cr;
            sx += (xa + xb) * cr;
            sy += (ya + yb) * cr;
        }
        o->area[i] = 0.5 * A2;
        o->cx[i] = x0 + sx / (3.0 * A2);
        o->cy[i] = y0 + sy / (3.0 * A2);
        o->nface[i] = nv;
    }

    /* faces: every cell edge a->b (counter-clockwise) has outward normal (dy, -dx)/|d| */
    long ne = cell_ptr[nc];
    edge_rec *er = (edge_rec *)xcalloc((size_t)ne, sizeof(edge_rec));
    for (int i = 0; i < nc; i++) {
        int p0 = cell_ptr[i], nv = cell_ptr[i + 1] - p0;
        for (int l = 0; l < nv; l++) {
            int a = cell_nodes[p0 + l], b = cell_nodes[p0 + (l + 1) % nv];
            double dx = xy[2 * b] - xy[2 * a], dy = xy[2 * b + 1] - xy[2 * a + 1];
            double len = sqrt(dx * dx + dy * dy);
            oface *F = &o->face[4 * i + l];
            F->nbr = -1;
            F->bedge = -1;
            F->nx = dy / len;
            F->ny = -dx / len;
            F->len = len;
            F->xm = 0.5 * (xy[2 * a] + xy[2 * b]);
            F->ym = 0.5 * (xy[2 * a + 1] + xy[2 * b + 1]);
            er[p0 + l].key = edge_key(a, b);
            er[p0 + l].cell = i;
            er[p0 + l].local = l;
        }
    }
    qsort(er, (size_t)ne, sizeof(edge_rec), cmp_edge);
    for (long e = 0; e + 1 < ne; e++) {
        if (er[e].key == er[e + 1].key) {
            o->face[4 * er[e].cell + er[e].local].nbr = er[e + 1].cell;
            o->face[4 * er[e + 1].cell + er[e + 1].local].nbr = er[e].cell;
            e++;
        }
    }
    /* boundary edges: find the owning cell face by key */
    int ok = 1;
    for (int b = 0; b < nb; b++) {
        long long key = edge_key(bedge_nodes[2 * b], bedge_nodes[2 * b + 1]);
        long lo = 0, hi = ne - 1, hit = -1;
        while (lo <= hi) {
            long mid = (lo + hi) / 2;
            if (er[mid].key == key) { hit = mid; break; }
            if (er[mid].key < key) lo = mid + 1; else hi = mid - 1;
        }
        if (hit < 0) { ok = 0; break; }
        oface *F = &o->face[4 * er[hit].cell + er[hit].local];
        if (F->nbr >= 0) { ok = 0; break; }
        F->bedge = b;
        o->bcell[b] = er[hit].cell;
        o->bxm[b] = F->xm;
        o->bym[b] = F->ym;
        o->bnx[b] = F->nx;
        o->bny[b] = F->ny;
        o->blen[b] = F->len;
    }
    /* periodic pairs: edge b is edge a translated by s; glue the two owner cells */
    for (int p = 0; p < n_periodic && ok; p++) {
        int ea = periodic_pairs[2 * p], eb = periodic_pairs[2 * p + 1];
        double sx = periodic_shift[2 * p], sy = periodic_shift[2 * p + 1];
        int ca = o->bcell[ea], cb = o->bcell[eb];
        oface *Fa = NULL, *Fb = NULL;
        for (int l = 0; l < o->nface[ca]; l++)
            if (o->face[4 * ca + l].bedge == ea) Fa = &o->face[4 * ca + l];
        for (int l = 0; l < o->nface[cb]; l++)
            if (o->face[4 * cb + l].bedge == eb) Fb = &o->face[4 * cb + l];
        if (!Fa || !Fb) { ok = 0; break; }
        Fa->nbr = cb; Fa->bedge = -1; Fa->sx = -sx; Fa->sy = -sy;
        Fb->nbr = ca; Fb->bedge = -1; Fb->sx = sx; Fb->sy = sy;
        Fb->nx = -Fa->nx; Fb->ny = -Fa->ny; Fb->len = Fa->len;
        o->btype[ea] = o->btype[eb] = BC_PERIODIC;
    }
    free(er);
    for (int i = 0; i < nc && ok; i++)
        for (int l = 0; l < o->nface[i]; l++)
            if (o->face[4 * i + l].nbr < 0 && o->face[4 * i + l].bedge < 0) ok = 0;
    if (!ok) { oracle_destroy(o); return NULL; }

    /* wall distance d of Sec. 2: centroid to the nearest wall segment */
    for (int i = 0; i < nc; i++) {
        double d = 1e30;
        for (int b = 0; b < nb; b++) {
            if (o->btype[b] != BC_WALL) continue;
            int a0 = bedge_nodes[2 * b], a1 = bedge_nodes[2 * b + 1];
            double s = seg_dist(o->cx[i], o->cy[i], xy[2 * a0], xy[2 * a0 + 1], xy[2 * a1],
                                xy[2 * a1 + 1]);
            if (s < d) d = s;
        }
        o->wdist[i] = d;
    }

    /* state and work arrays */
    size_t nq = (size_t)nc * Q;
    o->f = (real *)xcalloc(nq, sizeof(real));
    o->fn = (real *)xcalloc(nq, sizeof(real));
    o->fst = (real *)xcalloc(nq, sizeof(real));
    o->feqs = (real *)xcalloc(nq, sizeof(real));
    o->X = (real *)xcalloc(nq, sizeof(real));
    for (int J = 0; J < 3; J++) {
        o->ga[J] = (real *)xcalloc(nq, sizeof(real));
        o->gc[J] = (real *)xcalloc(nq, sizeof(real));
    }
    o->gradf = (real *)xcalloc(nq * 2, sizeof(real));
    o->fbc = (real *)xcalloc((size_t)nb * Q, sizeof(real));
    o->rho = (real *)xcalloc(nc, sizeof(real));
    o->ux = (real *)xcalloc(nc, sizeof(real));
    o->uy = (real *)xcalloc(nc, sizeof(real));
    o->k = (real *)xcalloc(nc, sizeof(real));
    o->om = (real *)xcalloc(nc, sizeof(real));
    o->nut = (real *)xcalloc(nc, sizeof(real));
    o->tau = (real *)xcalloc(nc, sizeof(real));
    o->gu = (real *)xcalloc((size_t)nc * 2, sizeof(real));
    o->gv = (real *)xcalloc((size_t)nc * 2, sizeof(real));
    o->gk = (real *)xcalloc((size_t)nc * 2, sizeof(real));
    o->gw = (real *)xcalloc((size_t)nc * 2, sizeof(real));
    o->rk = (real *)xcalloc(nc, sizeof(real));
    o->rw = (real *)xcalloc(nc, sizeof(real));
    o->f1 = (real *)xcalloc(nc, sizeof(real));
    o->Sabs = (real *)xcalloc(nc, sizeof(real));

    /* Step 0: f = f^eq(rho, u); k, omega initial; nu_t^0 = k / omega; tau from Eq. turbtau */
    for (int i = 0; i < nc; i++) {
        double r = rho_init ? rho_init[i] : o->rho0;
        double u = u_init ? u_init[i] : 0.0, v = v_init ? v_init[i] : 0.0;
        feq_r(r, u, v, &o->f[(size_t)i * Q]);
        moments(&o->f[(size_t)i * Q], &o->rho[i], &o->ux[i], &o->uy[i]);
        o->k[i] = k_init ? k_init[i] : 0.0;
        o->om[i] = w_init ? w_init[i] : 1.0;
        o->nut[i] = o->sst ? o->k[i] / o->om[i] : 0.0;
        o->tau[i] = (o->nu + o->nut[i]) / CS2;
    }

    /* time step: given, or CFL * (forward-Euler upwind limit) when dt <= 0.  The limit of cell
     * i is 1 / max_alpha sum_m max(e_alpha . n_m, 0) Delta l_m / A_i; the global step takes the
     * smallest over the cells.  Local time stepping (steady-state acceleration, not in the
     * paper) gives every cell its own dt_i = CFL * limit_i instead; dt then reports the
     * smallest of them, which is the global step. */
    if (o->dt <= 0.0 || local_dt) {
        if (local_dt) o->dtc = (double *)xcalloc(nc, sizeof(double));
        double lim = 0.0;
        for (int i = 0; i < nc; i++) {
            double rate = 0.0;
            for (int a = 0; a < Q; a++) {
                double s = 0.0;
                for (int l = 0; l < o->nface[i]; l++) {
                    const oface *F = &o->face[4 * i + l];
                    double en = EX[a] * F->nx + EY[a] * F->ny;
                    if (en > 0) s += en * F->len;
                }
                s /= o->area[i];
                if (s > rate) rate = s;
            }
            if (rate > lim) lim = rate;
            if (local_dt) o->dtc[i] = cfl / rate;
        }
        o->dt = cfl / lim;
    }
    return o;
}

void oracle_destroy(oracle *o)
{
    if (!o) return;
    free(o->nface); free(o->face); free(o->area); free(o->cx); free(o->cy); free(o->wdist);
    free(o->btype); free(o->bcell); free(o->bval);
    free(o->bxm); free(o->bym); free(o->bnx); free(o->bny); free(o->blen);
    free(o->f); free(o->fn); free(o->fst); free(o->feqs); free(o->X);
    for (int J = 0; J < 3; J++) { free(o->ga[J]); free(o->gc[J]); }
    free(o->gradf); free(o->fbc);
    free(o->rho); free(o->ux); free(o->uy); free(o->k); free(o->om); free(o->nut); free(o->tau); free(o->dtc);
    free(o->gu); free(o->gv); free(o->gk); free(o->gw); free(o->rk); free(o->rw);
    free(o->f1); free(o->Sabs);
    free(o);
}

/* ------------------------------------------------------------------ gradient */
/* Unweighted least-squares gradient (Part I method, reading): data points are the
 * neighbour centroids (periodic ones shifted) with their cell values and, on boundary faces,
 * the face midpoint with the boundary value.  g = M^{-1} sum_m d_m (phi_m - phi_i),
 * M = sum_m d_m d_m^T.  phi is strided (value of cell i at phi[i*stride]). */
static void lsq_gradient(const oracle *o, int i, const real *phi, int stride,
                         const real *phib, int bstride, real *gx, real *gy)
{
    double mxx = 0, mxy = 0, myy = 0;
    real bx = 0, by = 0;
    real pi = phi[(size_t)i * stride];
    for (int l = 0; l < o->nface[i]; l++) {
        const oface *F = &o->face[4 * i + l];
        double dx, dy;
        real dp;
        if (F->nbr >= 0) {
            dx = o->cx[F->nbr] + F->sx - o->cx[i];
            dy = o->cy[F->nbr] + F->sy - o->cy[i];
            dp = phi[(size_t)F->nbr * stride] - pi;
        } else {
            dx = F->xm - o->cx[i];
            dy = F->ym - o->cy[i];
            dp = phib[(size_t)F->bedge * bstride] - pi;
        }
        mxx += dx * dx;
        mxy += dx * dy;
        myy += dy * dy;
        bx += dx * dp;
        by += dy * dp;
    }
    double det = mxx * myy - mxy * mxy;
    *gx = (myy * bx - mxy * by) / det;
    *gy = (mxx * by - mxy * bx) / det;
}

/* ------------------------------------------------------------------ boundary values */
/* f_{alpha,bc} on boundary faces from the owner cell P (Part I not available; readings):
 *   wall / inlet:  f^eq(rho_P, u_b) + [f_P - f^eq(rho_P, u_P)]   (non-equilibrium extrapolation)
 *   outlet:        f^eq(rho_b, u_P) + [f_P - f^eq(rho_P, u_P)]
 *   far field:     f^eq(rho_b, u_b) where e.n < 0 (incoming), f_P where e.n >= 0 (outgoing) */
static void boundary_f(const oracle *o, const real *f, real *fbc)
{
    OMP_FOR
    for (int b = 0; b < o->nb; b++) {
        int t = o->btype[b];
        if (t == BC_PERIODIC) continue;
        int P = o->bcell[b];
        const real *fp = &f[(size_t)P * Q];
        const real *bv = &o->bval[5 * (size_t)b];
        real *out = &fbc[(size_t)b * Q];
        real rP, uP, vP, eqP[Q], eqB[Q];
        moments(fp, &rP, &uP, &vP);
        feq_r(rP, uP, vP, eqP);
        if (t == BC_WALL || t == BC_INLET) {
            feq_r(rP, bv[1], bv[2], eqB);
            for (int a = 0; a < Q; a++) out[a] = eqB[a] + (fp[a] - eqP[a]);
        } else if (t == BC_OUTLET) {
            feq_r(bv[0], uP, vP, eqB);
            for (int a = 0; a < Q; a++) out[a] = eqB[a] + (fp[a] - eqP[a]);
        } else { /* BC_FARFIELD */
            feq_r(bv[0], bv[1], bv[2], eqB);
            for (int a = 0; a < Q; a++) {
                double en = EX[a] * o->bnx[b] + EY[a] * o->bny[b];
                out[a] = en < 0.0 ? eqB[a] : fp[a];
            }
        }
    }
}

/* Venkatakrishnan limiter of the reconstruction of f (variant 1; a reading of Part I's
 * reconstruction with a limiter, which Sec. 3.2 does not state): with D1 the distance from f_i
 * to the max (min) over the cell, its face neighbours and its boundary face values and D2 the
 * reconstructed increment g . (x_f - x_i) to face m, phi_m = [(D1^2 + e2) D2 + 2 D2^2 D1] /
 * [D1^2 + 2 D2^2 + D1 D2 + e2] / D2 (1 where D2 = 0), and phi = min_m phi_m.  e2 = (K h)^3
 * with h = sqrt(A_i) and K = 1 keeps smooth regions unlimited. */
static real vk_limiter(const oracle *o, int i, const real *phi, int stride,
                       const real *phib, int bstride, real gx, real gy)
{
    real pi = phi[(size_t)i * stride], lo = pi, hi = pi;
    for (int l = 0; l < o->nface[i]; l++) {
        const oface *F = &o->face[4 * i + l];
        real q = F->nbr >= 0 ? phi[(size_t)F->nbr * stride] : phib[(size_t)F->bedge * bstride];
        if (RE(q) < RE(lo)) lo = q;
        if (RE(q) > RE(hi)) hi = q;
    }
    double h = sqrt(o->area[i]);
    double e2 = h * h * h;
    real psi = 1.0;
    for (int l = 0; l < o->nface[i]; l++) {
        const oface *F = &o->face[4 * i + l];
        real d2 = gx * (F->xm - o->cx[i]) + gy * (F->ym - o->cy[i]);
        if (RE(d2) == 0.0) continue;
        real d1 = RE(d2) > 0.0 ? hi - pi : lo - pi;
        real r = ((d1 * d1 + e2) * d2 + 2.0 * d2 * d2 * d1) /
                 (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + e2) / d2;
        if (RE(r) < RE(psi)) psi = r;
    }
    return psi;
}

/* ------------------------------------------------------------------ convection */
/* Gamma^a_alpha = -(1/A) sum_m [(e_alpha . n) f_{alpha,bc} Delta l]_m, Eq. (advection).
 * Interior face values: upwind by the sign of e_alpha . n (n out of this cell), linear
 * reconstruction f + grad f . (x_face - x_cell) from the upwind cell (Part I reading).
 * Boundary faces use boundary_f(). */
static void convection(oracle *o, const real *f, real *ga)
{
    int nc = o->nc;
    boundary_f(o, f, o->fbc);
    OMP_FOR
    for (int i = 0; i < nc; i++)
        for (int a = 0; a < Q; a++) {
            real gx, gy;
            lsq_gradient(o, i, f + a, Q, o->fbc + a, Q, &gx, &gy);
            if (o->variant & 1) {
                real phi = vk_limiter(o, i, f + a, Q, o->fbc + a, Q, gx, gy);
                gx *= phi;
                gy *= phi;
            }
            o->gradf[((size_t)i * Q + a) * 2] = gx;
            o->gradf[((size_t)i * Q + a) * 2 + 1] = gy;
        }
    OMP_FOR
    for (int i = 0; i < nc; i++) {
        for (int a = 0; a < Q; a++) {
            real sum = 0.0;
            for (int l = 0; l < o->nface[i]; l++) {
                const oface *F = &o->face[4 * i + l];
                double en = EX[a] * F->nx + EY[a] * F->ny;
                real fv;
                if (F->nbr < 0) {
                    fv = o->fbc[(size_t)F->bedge * Q + a];
                } else if (en >= 0.0) {
                    const real *g = &o->gradf[((size_t)i * Q + a) * 2];
                    fv = f[(size_t)i * Q + a] + g[0] * (F->xm - o->cx[i]) + g[1] * (F->ym - o->cy[i]);
                } else {
                    int j = F->nbr;
                    const real *g = &o->gradf[((size_t)j * Q + a) * 2];
                    fv = f[(size_t)j * Q + a] + g[0] * (F->xm - (o->cx[j] + F->sx)) +
                         g[1] * (F->ym - (o->cy[j] + F->sy));
                }
                sum += en * fv * F->len;
            }
            ga[(size_t)i * Q + a] = -sum / o->area[i];
        }
    }
}

/* ------------------------------------------------------------------ SST */
/* Point functions of Sec. 2 in kinematic form (rho divided out; reading):
 * CD_kw = max(2 sigma_w2 / omega grad k . grad omega, 1e-20);
 * arg1 = min(max(sqrt(k)/(0.09 omega d), 500 nu/(omega d^2)), 4 sigma_w2 k/(CD_kw d^2));
 * f1 = tanh(arg1^4); arg2 = max(2 sqrt(k)/(0.09 omega d), 500 nu/(omega d^2)); f2 = tanh(arg2^2);
 * nu_t = a1 k / max(a1 omega, S f2). */
static real sst_cdkw(real w, real gkx, real gky, real gwx, real gwy)
{
    real c = 2.0 * SW2 / w * (gkx * gwx + gky * gwy);
    return RE(c) > 1e-20 ? c : 1e-20;
}

static real sst_f1(real k, real w, double d, double nu, real cdkw)
{
    real a = rsqrt(k) / (BSTAR * w * d);
    real b = 500.0 * nu / (w * d * d);
    real c = 4.0 * SW2 * k / (cdkw * d * d);
    real arg1 = rmin(rmax(a, b), c);
    return rtanh(arg1 * arg1 * arg1 * arg1);
}

static real sst_f2(real k, real w, double d, double nu)
{
    real arg2 = rmax(2.0 * rsqrt(k) / (BSTAR * w * d), 500.0 * nu / (w * d * d));
    return rtanh(arg2 * arg2);
}

static real sst_nut(real k, real w, real S, real f2)
{
    return A1 * k / rmax(A1 * w, S * f2);
}

#ifndef ORACLE_COMPLEX_STEP
/* out = {f1, f2, CD_kw, nu_t} at one point (for tests). */
void oracle_sst_point(double k, double w, double d, double gkx, double gky, double gwx,
                      double gwy, double S, double nu, double *out)
{
    double cd = sst_cdkw(w, gkx, gky, gwx, gwy);
    double f2 = sst_f2(k, w, d, nu);
    out[0] = sst_f1(k, w, d, nu, cd);
    out[1] = f2;
    out[2] = cd;
    out[3] = sst_nut(k, w, S, f2);
}
#endif

/* Boundary values of u, v, k, omega for the SST gradients and face fluxes (Menter 1994
 * boundary conditions, Sec. 3.2; readings): wall k = 0, omega = 60 nu / (beta1 d^2) with d
 * the wall cell's wall distance; inlet / far field k_b, omega_b given; outlet zero gradient.
 * Velocity: wall / inlet / far field u_b; outlet the cell velocity. */
static void sst_boundary(const oracle *o, int b, real *ub, real *vb, real *kb, real *wb)
{
    int P = o->bcell[b];
    const real *bv = &o->bval[5 * (size_t)b];
    switch (o->btype[b]) {
    case BC_WALL:
        *ub = bv[1]; *vb = bv[2]; *kb = 0.0;
        *wb = 60.0 * o->nu / (B1 * o->wdist[P] * o->wdist[P]);
        break;
    case BC_OUTLET:
        *ub = o->ux[P]; *vb = o->uy[P]; *kb = o->k[P]; *wb = o->om[P];
        break;
    default: /* inlet, far field */
        *ub = bv[1]; *vb = bv[2]; *kb = bv[3]; *wb = bv[4];
        break;
    }
}

/* Barth-Jespersen limiter of a reconstructed field (reading of the second-order upwind
 * scheme of Sec. 3.2 on unstructured cells): the largest psi in [0, 1] such that every face
 * value phi_i + psi grad phi . (x_f - x_i) stays within the min / max of phi_i, its face
 * neighbours and its boundary values. */
static real bj_limiter(const oracle *o, int i, const real *phi, const real *phib,
                       int bstride, const real *g)
{
    real lo = phi[i], hi = phi[i];
    for (int l = 0; l < o->nface[i]; l++) {
        const oface *F = &o->face[4 * i + l];
        real q = F->nbr >= 0 ? phi[F->nbr] : phib[(size_t)F->bedge * bstride];
        if (RE(q) < RE(lo)) lo = q;
        if (RE(q) > RE(hi)) hi = q;
    }
    real psi = 1.0;
    for (int l = 0; l < o->nface[i]; l++) {
        const oface *F = &o->face[4 * i + l];
        real d = g[0] * (F->xm - o->cx[i]) + g[1] * (F->ym - o->cy[i]);
        real r = 1.0;
        if (RE(d) > 0.0) r = (hi - phi[i]) / d;
        else if (RE(d) < 0.0) r = (lo - phi[i]) / d;
        if (RE(r) < RE(psi)) psi = r;
    }
    return psi;
}

/* One SST update of size dt from the macros at t^n (Step 1; readings): explicit face
 * convection (second-order upwind with the mean face velocity, Barth-Jespersen limited) and
 * central diffusion with
 * the mean face coefficient, explicit production and cross diffusion, point-implicit
 * destruction, then f2, nu_t and tau = (nu + nu_t) / cs^2 (Eq. turbtau). */
static void sst_update(oracle *o)
{
    int nc = o->nc, nb = o->nb;
    real *ubc = (real *)xcalloc((size_t)nb * 4, sizeof(real));
    for (int b = 0; b < nb; b++)
        if (o->btype[b] != BC_PERIODIC)
            sst_boundary(o, b, &ubc[4 * b], &ubc[4 * b + 1], &ubc[4 * b + 2], &ubc[4 * b + 3]);
    OMP_FOR
    for (int i = 0; i < nc; i++) {
        lsq_gradient(o, i, o->ux, 1, ubc + 0, 4, &o->gu[2 * i], &o->gu[2 * i + 1]);
        lsq_gradient(o, i, o->uy, 1, ubc + 1, 4, &o->gv[2 * i], &o->gv[2 * i + 1]);
        lsq_gradient(o, i, o->k, 1, ubc + 2, 4, &o->gk[2 * i], &o->gk[2 * i + 1]);
        lsq_gradient(o, i, o->om, 1, ubc + 3, 4, &o->gw[2 * i], &o->gw[2 * i + 1]);
    }
    /* limited gradients for the upwind face values of k and omega */
    real *lk = (real *)xcalloc((size_t)nc * 2, sizeof(real));
    real *lw = (real *)xcalloc((size_t)nc * 2, sizeof(real));
    OMP_FOR
    for (int i = 0; i < nc; i++) {
        real pk = bj_limiter(o, i, o->k, ubc + 2, 4, &o->gk[2 * i]);
        real pw = bj_limiter(o, i, o->om, ubc + 3, 4, &o->gw[2 * i]);
        lk[2 * i] = pk * o->gk[2 * i];
        lk[2 * i + 1] = pk * o->gk[2 * i + 1];
        lw[2 * i] = pw * o->gw[2 * i];
        lw[2 * i + 1] = pw * o->gw[2 * i + 1];
    }
    real *sk = (real *)xcalloc(nc, sizeof(real));
    real *sw = (real *)xcalloc(nc, sizeof(real));
    real *SS = (real *)xcalloc(nc, sizeof(real));
    real *dv = (real *)xcalloc(nc, sizeof(real));
    OMP_FOR
    for (int i = 0; i < nc; i++) {
        real s11 = o->gu[2 * i], s22 = o->gv[2 * i + 1];
        real s12 = 0.5 * (o->gu[2 * i + 1] + o->gv[2 * i]);
        SS[i] = s11 * s11 + s22 * s22 + 2.0 * s12 * s12; /* S_ij S_ij */
        dv[i] = s11 + s22;
        o->Sabs[i] = rsqrt(2.0 * SS[i]);
        real cd = sst_cdkw(o->om[i], o->gk[2 * i], o->gk[2 * i + 1], o->gw[2 * i], o->gw[2 * i + 1]);
        o->f1[i] = sst_f1(o->k[i], o->om[i], o->wdist[i], o->nu, cd);
        sk[i] = o->f1[i] * SK1 + (1.0 - o->f1[i]) * SK2;
        sw[i] = o->f1[i] * SW1 + (1.0 - o->f1[i]) * SW2;
    }
    OMP_FOR
    for (int i = 0; i < nc; i++) {
        real ck = 0, cw = 0, dk = 0, dw = 0;
        for (int l = 0; l < o->nface[i]; l++) {
            const oface *F = &o->face[4 * i + l];
            double rx = F->xm - o->cx[i], ry = F->ym - o->cy[i];
            real uf, vf, kup, wup;
            real kin = o->k[i] + lk[2 * i] * rx + lk[2 * i + 1] * ry;
            real win = o->om[i] + lw[2 * i] * rx + lw[2 * i + 1] * ry;
            if (F->nbr >= 0) {
                int j = F->nbr;
                double xj = o->cx[j] + F->sx, yj = o->cy[j] + F->sy;
                uf = 0.5 * (o->ux[i] + o->ux[j]);
                vf = 0.5 * (o->uy[i] + o->uy[j]);
                real un = uf * F->nx + vf * F->ny;
                double sx = F->xm - xj, sy = F->ym - yj;
                kup = RE(un) >= 0.0 ? kin : o->k[j] + lk[2 * j] * sx + lk[2 * j + 1] * sy;
                wup = RE(un) >= 0.0 ? win : o->om[j] + lw[2 * j] * sx + lw[2 * j + 1] * sy;
                double dist = sqrt((xj - o->cx[i]) * (xj - o->cx[i]) + (yj - o->cy[i]) * (yj - o->cy[i]));
                real gkf = 0.5 * ((o->nu + sk[i] * o->nut[i]) + (o->nu + sk[j] * o->nut[j]));
                real gwf = 0.5 * ((o->nu + sw[i] * o->nut[i]) + (o->nu + sw[j] * o->nut[j]));
                ck += un * kup * F->len;
                cw += un * wup * F->len;
                real ck_n = (o->k[j] - o->k[i]) / dist, cw_n = (o->om[j] - o->om[i]) / dist;
                if (o->variant & 2) {
                    /* non-orthogonal correction (variant 2): grad phi . n = (phi_j - phi_i)/|d|
                     * + mean grad phi . (n - d/|d|) */
                    double tx = F->nx - (xj - o->cx[i]) / dist, ty = F->ny - (yj - o->cy[i]) / dist;
                    ck_n += 0.5 * ((o->gk[2 * i] + o->gk[2 * j]) * tx + (o->gk[2 * i + 1] + o->gk[2 * j + 1]) * ty);
                    cw_n += 0.5 * ((o->gw[2 * i] + o->gw[2 * j]) * tx + (o->gw[2 * i + 1] + o->gw[2 * j + 1]) * ty);
                }
                dk += gkf * ck_n * F->len;
                dw += gwf * cw_n * F->len;
            } else {
                const real *ub = &ubc[4 * F->bedge];
                real un = ub[0] * F->nx + ub[1] * F->ny;
                kup = RE(un) >= 0.0 ? kin : ub[2];
                wup = RE(un) >= 0.0 ? win : ub[3];
                double dist = sqrt(rx * rx + ry * ry);
                ck += un * kup * F->len;
                cw += un * wup * F->len;
                real ck_n = (ub[2] - o->k[i]) / dist, cw_n = (ub[3] - o->om[i]) / dist;
                if (o->variant & 2) {
                    double tx = F->nx - rx / dist, ty = F->ny - ry / dist;
                    ck_n += o->gk[2 * i] * tx + o->gk[2 * i + 1] * ty;
                    cw_n += o->gw[2 * i] * tx + o->gw[2 * i + 1] * ty;
                }
                dk += (o->nu + sk[i] * o->nut[i]) * ck_n * F->len;
                dw += (o->nu + sw[i] * o->nut[i]) * cw_n * F->len;
            }
        }
        real f1 = o->f1[i];
        real gam = f1 * (B1 / BSTAR - SW1 * KAPPA * KAPPA / sqrt(BSTAR)) +
                   (1.0 - f1) * (B2 / BSTAR - SW2 * KAPPA * KAPPA / sqrt(BSTAR));
        /* production P / rho = nu_t (2 S_ij S_ij - 2/3 (div u)^2) - 2/3 k div u */
        real pk = o->nut[i] * (2.0 * SS[i] - 2.0 / 3.0 * dv[i] * dv[i]) - 2.0 / 3.0 * o->k[i] * dv[i];
        /* variant 8: Menter's production limiter P_k <= 10 beta* omega k (not in the paper) */
        if ((o->variant & 8) && RE(pk) > RE(10.0 * BSTAR * o->om[i] * o->k[i])) pk = 10.0 * BSTAR * o->om[i] * o->k[i];
        /* gamma P / nu_t, with the k div u / nu_t part taken as 0 when nu_t = 0 */
        real pw = gam * (2.0 * SS[i] - 2.0 / 3.0 * dv[i] * dv[i]);
        if (RE(o->nut[i]) > 0.0) pw -= 2.0 / 3.0 * gam * o->k[i] * dv[i] / o->nut[i];
        real cross = 2.0 * (1.0 - f1) * SW2 / o->om[i] *
                       (o->gk[2 * i] * o->gw[2 * i] + o->gk[2 * i + 1] * o->gw[2 * i + 1]);
        o->rk[i] = (-ck + dk) / o->area[i] + pk;
        o->rw[i] = (-cw + dw) / o->area[i] + pw + cross;
    }
    double wmin = 1e-12 * o->uref / o->lref;
    OMP_FOR
    for (int i = 0; i < nc; i++) {
        real f1 = o->f1[i];
        real beta = f1 * B1 + (1.0 - f1) * B2;
        double dt = cell_dt(o, i);
        real kn = (o->k[i] + dt * o->rk[i]) / (1.0 + dt * BSTAR * o->om[i]);
        real wn = (o->om[i] + dt * o->rw[i]) / (1.0 + dt * beta * o->om[i]);
        o->k[i] = RE(kn) > 0.0 ? kn : 0.0;
        o->om[i] = RE(wn) > wmin ? wn : wmin;
    }
    OMP_FOR
    for (int i = 0; i < nc; i++) {
        real f2 = sst_f2(o->k[i], o->om[i], o->wdist[i], o->nu);
        o->nut[i] = sst_nut(o->k[i], o->om[i], o->Sabs[i], f2);
        o->tau[i] = (o->nu + o->nut[i]) / CS2;
    }
    free(ubc); free(sk); free(sw); free(SS); free(dv); free(lk); free(lw);
}

/* ------------------------------------------------------------------ IMEX step */
/* One time step, Steps 1-7 of Sec. 3.2.  Stage J (J = 1, 2, 3):
 *   rho^(J), (rho u)^(J) = moments of f^n + dt sum_{k<J} mt_Jk Gamma^a(k)   Eq. (sumimeximplicitnew)
 *   f^(J) = [f^n + dt sum_{k<J} (mt_Jk Gamma^a(k) + m_Jk Gamma^c(k)) + dt/tau m_JJ f^eq(J)]
 *           / (1 + dt/tau m_JJ)                                           Eq. (fnewstage)
 *   Gamma^c(J) = -(f^(J) - f^eq(J)) / tau                                 Eq. (collision)
 *   Gamma^a(J) = convection of f^(J)                                      Eq. (advection)
 * then f^{n+1} = f^n + dt sum nt_J Gamma^a(J) + dt sum n_J Gamma^c(J)      Eq. (imextwo). */
static int finish_step(oracle *o);

static int imex_step(oracle *o)
{
    int nc = o->nc;
    size_t nq = (size_t)nc * Q;
    /* Variant 4 (the other reading of Step 5, "repeat Steps 1-4" per stage): before every stage
     * the SST update is solved again from (k, omega, nu_t) of t^n with the macros of the latest
     * stage value (f^n, f^(1), f^(2)), and the stage uses the resulting tau; the last solve
     * gives k, omega at t^{n+1}. */
    int per_stage = o->sst && (o->variant & 4);
    real *k0 = NULL, *w0 = NULL, *nt0 = NULL;
    if (per_stage) {
        k0 = (real *)xcalloc(nc, sizeof(real));
        w0 = (real *)xcalloc(nc, sizeof(real));
        nt0 = (real *)xcalloc(nc, sizeof(real));
        memcpy(k0, o->k, nc * sizeof(real));
        memcpy(w0, o->om, nc * sizeof(real));
        memcpy(nt0, o->nut, nc * sizeof(real));
    }
    if (o->sst) sst_update(o); /* Step 1 */
    else
        for (int i = 0; i < nc; i++) o->tau[i] = o->nu / CS2;
    memcpy(o->fn, o->f, nq * sizeof(real));
    double defect = 0.0;
    for (int J = 0; J < 3; J++) {
        if (per_stage && J > 0) {
            memcpy(o->k, k0, nc * sizeof(real));
            memcpy(o->om, w0, nc * sizeof(real));
            memcpy(o->nut, nt0, nc * sizeof(real));
            for (int i = 0; i < nc; i++) moments(&o->fst[(size_t)i * Q], &o->rho[i], &o->ux[i], &o->uy[i]);
            sst_update(o);
        }
        OMP_FOR_MAX_DEFECT
        for (int i = 0; i < nc; i++) {
            real tau = o->tau[i];
            double dt = cell_dt(o, i);
            real *X = &o->X[(size_t)i * Q];
            const real *fn = &o->fn[(size_t)i * Q];
            for (int a = 0; a < Q; a++) {
                real s = fn[a];
                for (int k = 0; k < J; k++) s += dt * MT[J][k] * o->ga[k][(size_t)i * Q + a];
                X[a] = s;
            }
            real r, u, v, eq[Q];
            moments(X, &r, &u, &v);
            feq_r(r, u, v, eq);
            real zJ = dt / tau * MI[J][J];
            real *fs = &o->fst[(size_t)i * Q];
            for (int a = 0; a < Q; a++) {
                real num = fn[a];
                for (int k = 0; k < J; k++)
                    num += dt * (MT[J][k] * o->ga[k][(size_t)i * Q + a] +
                                 MI[J][k] * o->gc[k][(size_t)i * Q + a]);
                num += zJ * eq[a];
                fs[a] = num / (1.0 + zJ);
                o->gc[J][(size_t)i * Q + a] = -(fs[a] - eq[a]) / tau;
            }
            /* moment elimination check: sum f^(J) psi must equal the moments of X */
            real r2, u2, v2;
            moments(fs, &r2, &u2, &v2);
            double dd = fabs(RE(r2 - r)) + fabs(RE(r2 * u2 - r * u)) + fabs(RE(r2 * v2 - r * v));
            if (dd > defect) defect = dd;
        }
        convection(o, o->fst, o->ga[J]); /* Step 2 for the next stage / the final update */
    }
    OMP_FOR
    for (size_t q = 0; q < nq; q++) {
        double dt = cell_dt(o, (int)(q / Q));
        real s = o->fn[q];
        for (int J = 0; J < 3; J++) s += dt * (NT[J] * o->ga[J][q] + NI[J] * o->gc[J][q]);
        o->f[q] = s;
    }
    o->moment_defect = defect;
    if (per_stage) {
        /* finish_step measures the change of u from t^n */
        for (int i = 0; i < nc; i++) moments(&o->fn[(size_t)i * Q], &o->rho[i], &o->ux[i], &o->uy[i]);
        free(k0); free(w0); free(nt0);
    }
    return finish_step(o);
}

/* Step 7: macros; velocity residual e (reading: relative L2 change of u over the step). */
static int finish_step(oracle *o)
{
    int nc = o->nc;
    double num = 0.0, den = 0.0;
    int bad = 0;
    for (int i = 0; i < nc; i++) {
        real r, u, v;
        moments(&o->f[(size_t)i * Q], &r, &u, &v);
        num += RE((u - o->ux[i]) * (u - o->ux[i]) + (v - o->uy[i]) * (v - o->uy[i]));
        den += RE(u * u + v * v);
        o->rho[i] = r;
        o->ux[i] = u;
        o->uy[i] = v;
        if (!(RE(r) == RE(r)) || !(RE(u) == RE(u)) || !(RE(v) == RE(v))) bad = 1;
    }
    o->residual = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
    o->steps++;
    return bad ? -1 : 0;
}

/* Explicit Euler FVLBM (the original scheme of Part I that the IMEX method replaces; Sec. 3.1
 * states its collision limit dt < 2 tau, Sec. 4.1 compares the two):
 * f^{n+1} = f^n + dt [Gamma^a(f^n) + Gamma^c(f^n)], Eqs. (semibgk), (advection), (collision). */
static int euler_step(oracle *o)
{
    int nc = o->nc;
    if (o->sst) sst_update(o);
    else
        for (int i = 0; i < nc; i++) o->tau[i] = o->nu / CS2;
    convection(o, o->f, o->ga[0]);
    OMP_FOR
    for (int i = 0; i < nc; i++) {
        double dt = cell_dt(o, i);
        real *f = &o->f[(size_t)i * Q];
        real r, u, v, eq[Q];
        moments(f, &r, &u, &v);
        feq_r(r, u, v, eq);
        for (int a = 0; a < Q; a++) {
            real gc = -(f[a] - eq[a]) / o->tau[i];
            f[a] = f[a] + dt * (o->ga[0][(size_t)i * Q + a] + gc);
        }
    }
    return finish_step(o);
}

/* ------------------------------------------------------------------ public entry points */
int oracle_step(oracle *o, int n)
{
    for (int s = 0; s < n; s++)
        if ((o->scheme == 1 ? euler_step(o) : imex_step(o)) != 0) return -1;
    return 0;
}

int oracle_n_cells(const oracle *o) { return o->nc; }
double oracle_dt(const oracle *o) { return o->dt; }

/* dt of every cell (the global dt everywhere unless local time stepping is on). */
void oracle_dt_cells(const oracle *o, double *out)
{
    for (int i = 0; i < o->nc; i++) out[i] = cell_dt(o, i);
}
double oracle_residual(const oracle *o) { return o->residual; }
double oracle_moment_defect(const oracle *o) { return o->moment_defect; }

void oracle_get_f(const oracle *o, double *f)
{
    for (size_t q = 0; q < (size_t)o->nc * Q; q++) f[q] = RE(o->f[q]);
}

void oracle_set_f(oracle *o, const double *f)
{
    for (size_t q = 0; q < (size_t)o->nc * Q; q++) o->f[q] = f[q];
    for (int i = 0; i < o->nc; i++) moments(&o->f[(size_t)i * Q], &o->rho[i], &o->ux[i], &o->uy[i]);
}

/* k, omega, nu_t of every cell (state access for a mesh split into parts that exchange
 * ghost cells; no arithmetic). */
void oracle_set_turb(oracle *o, const double *k, const double *w, const double *nut)
{
    for (int i = 0; i < o->nc; i++) {
        o->k[i] = k[i];
        o->om[i] = w[i];
        o->nut[i] = nut[i];
    }
}

/* The wall distance of every cell, replacing the one computed from this mesh's own wall edges
 * (a part of a split mesh takes the whole mesh's). */
void oracle_set_wdist(oracle *o, const double *d)
{
    for (int i = 0; i < o->nc; i++) o->wdist[i] = d[i];
}

void oracle_get_fields(const oracle *o, double *rho, double *u, double *v, double *k,
                       double *w, double *nut)
{
    for (int i = 0; i < o->nc; i++) {
        if (rho) rho[i] = RE(o->rho[i]);
        if (u) u[i] = RE(o->ux[i]);
        if (v) v[i] = RE(o->uy[i]);
        if (k) k[i] = RE(o->k[i]);
        if (w) w[i] = RE(o->om[i]);
        if (nut) nut[i] = RE(o->nut[i]);
    }
}

void oracle_geometry(const oracle *o, double *area, double *cx, double *cy, double *wdist)
{
    for (int i = 0; i < o->nc; i++) {
        area[i] = o->area[i];
        cx[i] = o->cx[i];
        cy[i] = o->cy[i];
        wdist[i] = o->wdist[i];
    }
}

/* Total mass sum_i rho_i A_i. */
double oracle_mass(const oracle *o)
{
    double m = 0.0;
    for (int i = 0; i < o->nc; i++) {
        real r = 0.0;
        for (int a = 0; a < Q; a++) r += o->f[(size_t)i * Q + a];
        m += RE(r) * o->area[i];
    }
    return m;
}

#ifndef ORACLE_COMPLEX_STEP
/* Gradient of a per-cell field phi with boundary values phib (one per boundary edge). */
/* The limiter value of the f reconstruction (variant 1) for a scalar field phi with boundary
 * values phib [n_bedges], at its least-squares gradient, per cell (test access). */
void oracle_limiter(oracle *o, const double *phi, const double *phib, double *psi)
{
    for (int i = 0; i < o->nc; i++) {
        double gx, gy;
        lsq_gradient(o, i, phi, 1, phib, 1, &gx, &gy);
        psi[i] = vk_limiter(o, i, phi, 1, phib, 1, gx, gy);
    }
}

/* The Barth-Jespersen limiter value of the SST reconstruction (bj_limiter) for a scalar
 * field phi with boundary values phib [n_bedges], at its least-squares gradient, per cell
 * (test access). */
void oracle_bj_limiter(oracle *o, const double *phi, const double *phib, double *psi)
{
    for (int i = 0; i < o->nc; i++) {
        double g[2];
        lsq_gradient(o, i, phi, 1, phib, 1, &g[0], &g[1]);
        psi[i] = bj_limiter(o, i, phi, phib, 1, g);
    }
}

/* The SST boundary values (sst_boundary) of every non-periodic boundary edge at the current
 * state: out [4 n_bedges] = u_b, v_b, k_b, omega_b (test access). */
void oracle_sst_bvals(oracle *o, double *out)
{
    for (int b = 0; b < o->nb; b++) {
        if (o->btype[b] == BC_PERIODIC) continue;
        sst_boundary(o, b, &out[4 * b], &out[4 * b + 1], &out[4 * b + 2], &out[4 * b + 3]);
    }
}

void oracle_gradient(oracle *o, const double *phi, const double *phib, double *g)
{
    for (int i = 0; i < o->nc; i++) lsq_gradient(o, i, phi, 1, phib, 1, &g[2 * i], &g[2 * i + 1]);
}

/* Gamma^a of a given f [nc * Q] with the mesh's boundary conditions. */
void oracle_convection(oracle *o, const double *f, double *ga) { convection(o, f, ga); }
#endif

/* Force on the walls (reading): F = sum_{wall faces} sum_alpha e_alpha (e_alpha . n) f_{alpha,bc}
 * Delta l, n out of the fluid cell -- the momentum flux of the face values of Eq. (advection).
 * out = {Fx, Fy, C_D, C_L} with C_D, C_L along / normal to the free-stream angle and
 * normalised by 0.5 rho0 U^2 L; cp[b] = (cs^2 rho_P - cs^2 rho0) / (0.5 rho0 U^2) on wall
 * edges, 0 elsewhere; fxe / fye (optional) receive the force on each wall edge. */
static void forces_r(oracle *o, real *out, double *cp, double *fxe, double *fye)
{
    boundary_f(o, o->f, o->fbc);
    real fx = 0.0, fy = 0.0;
    double q = 0.5 * o->rho0 * o->uref * o->uref;
    for (int b = 0; b < o->nb; b++) {
        if (cp) cp[b] = 0.0;
        if (fxe) fxe[b] = 0.0;
        if (fye) fye[b] = 0.0;
        if (o->btype[b] != BC_WALL) continue;
        real ex = 0.0, ey = 0.0;
        for (int a = 0; a < Q; a++) {
            double en = EX[a] * o->bnx[b] + EY[a] * o->bny[b];
            real m = en * o->fbc[(size_t)b * Q + a] * o->blen[b];
            ex += EX[a] * m;
            ey += EY[a] * m;
        }
        fx += ex;
        fy += ey;
        if (fxe) fxe[b] = RE(ex);
        if (fye) fye[b] = RE(ey);
        if (cp) {
            real r = 0.0;
            for (int a = 0; a < Q; a++) r += o->f[(size_t)o->bcell[b] * Q + a];
            cp[b] = RE((CS2 * r - CS2 * o->rho0) / q);
        }
    }
    double al = o->alpha_deg * M_PI / 180.0;
    out[0] = fx;
    out[1] = fy;
    out[2] = (fx * cos(al) + fy * sin(al)) / (q * o->lref);
    out[3] = (-fx * sin(al) + fy * cos(al)) / (q * o->lref);
}

void oracle_forces(oracle *o, double *out, double *cp, double *fxe, double *fye)
{
    real r[4];
    forces_r(o, r, cp, fxe, fye);
    for (int c = 0; c < 4; c++) out[c] = RE(r[c]);
}

#ifdef ORACLE_COMPLEX_STEP
/* Complex-step seeding: the boundary values [5 * n_bedges] and f [n_cells * 9] (either may be
 * NULL) take imaginary parts h * d; the macros follow f. */
void oracle_cs_seed(oracle *o, const double *dbval, const double *df, double h)
{
    if (dbval)
        for (size_t q = 0; q < 5 * (size_t)o->nb; q++) o->bval[q] += I * (h * dbval[q]);
    if (df) {
        for (size_t q = 0; q < (size_t)o->nc * Q; q++) o->f[q] += I * (h * df[q]);
        for (int i = 0; i < o->nc; i++) moments(&o->f[(size_t)i * Q], &o->rho[i], &o->ux[i], &o->uy[i]);
    }
}

/* Fx, Fy, C_D, C_L (real parts) and their derivatives along the seeded direction (imaginary
 * parts / h). */
void oracle_cs_forces(oracle *o, double h, double *val, double *der)
{
    real r[4];
    forces_r(o, r, NULL, NULL, NULL);
    for (int c = 0; c < 4; c++) {
        val[c] = creal(r[c]);
        der[c] = cimag(r[c]) / h;
    }
}
#endif
