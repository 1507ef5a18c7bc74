/*
 * sph_oracle.c -- plain FP64 CPU oracle for the weakly compressible SPH
 * hot path (cell list, neighbour search, pair sums, time integration).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or constant with the CUDA path; every definition below is written from the
 * paper (Valdez-Balderas et al., "Towards accelerating SPH simulations for
 * free-surface flows on multi-GPU clusters"):
 *
 *   Eq. 7   continuity:  d rho_i/dt = sum_j m_j v_ij . grad_i W_ij
 *   Eq. 8   position:    d r_i/dt   = v_i
 *   Eq. 9   momentum:    d v_i/dt   = -sum_j m_j (P_i + P_j + Pi_ij) grad_i W_ij + g
 *   Sec. 2.2 artificial viscosity Pi_ij, Tait equation of state, eta = 0.1 h
 *   Sec. 2.3 dynamic boundary particles (density evolves, position and
 *            velocity stay fixed)
 *   Sec. 3.1 cell list of cell size 2h, sort by cell label, first index per cell
 *   Sec. 3.2 27-cell neighbour search, pair sums of Eqs. 7-9
 *   Sec. 3.3 time integration with a CFL-limited variable step
 *   Sec. 4.3 sort of particle ids by label, ties kept in id order
 *
 * Readings where the paper is silent or garbled (each one is also listed in
 * the project's design notes):
 *   - Eq. 9 prints p/rho; the dimensionally consistent, momentum-conserving
 *     form P = p/rho^2 is used.
 *   - rho_ij in Pi_ij is the pair mean (rho_i + rho_j)/2.
 *   - c_i = sqrt(dp/drho at rho_i) = c0 (rho_i/rho0)^((gamma-1)/2).
 *   - Kernel: Wendland C2 with h = 1.3 dp, or the paper's own cubic spline
 *     (Sec. 2.2, or_params.kernel = 1); support |r_ij| < 2h strictly.
 *   - Integrator: the symplectic predictor-corrector (position-Verlet
 *     midpoint form) with two force evaluations per step; the step size is
 *     set from the first evaluation of each step.  Or the paper's own
 *     "second-order Verlet" (Sec. 3.3), one force evaluation per step, in
 *     the form of the SPHysics formulation it cites: a leapfrog over two
 *     steps, with an Euler step every N_s steps (the caller chooses which
 *     steps; the first step, which has no earlier state, is one).
 *   - CFL step: dt = CFL * min( min_i sqrt(h/|a_i|),  h/(c_max + mu_max) ),
 *     mu_max = max over pairs of h |v_ij . r_ij| / (r_ij^2 + eta^2).
 *   - Particles outside the cell-grid domain are excluded (no interactions)
 *     and frozen.
 *
 * Floating point: compiled with -ffp-contract=off so that every expression
 * rounds exactly as written (the cell keys and the neighbour predicate are
 * compared bit for bit against the GPU).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double dp, h, rho0, gamma, c0, alpha, eta2_coef;
    double g[3];
    double cfl, mass;
    double dmin[3], dmax[3];
    int64_t n_bound;          /* ids below n_bound are boundary particles */
    int64_t kernel;           /* 0: Wendland C2, 1: cubic spline (Sec. 2.2) */
} or_params;

/* ---------------------------------------------------------------- grid -- */

int or_grid_dims(const or_params *P, int64_t nc[3])
{
    const double cs = 2.0 * P->h;
    for (int a = 0; a < 3; ++a) {
        double t = ceil((P->dmax[a] - P->dmin[a]) / cs);
        nc[a] = (t < 1.0) ? 1 : (int64_t)t;
    }
    return 0;
}

/* Cell coordinate floor((x - x0) * (1/(2h))), with 1/(2h) rounded once.
 * (Sec. 3.1 fixes cells of size 2h but not the arithmetic; this form is the
 * reading both implementations share so that labels agree bit for bit.) */
static int coord(double x, double x0, double inv_cs, int64_t n, int64_t *c)
{
    double t = (x - x0) * inv_cs;
    if (!(t >= 0.0) || !(t < (double)n)) return 0;   /* also rejects NaN */
    *c = (int64_t)floor(t);
    return 1;
}

/* Sec. 3.1: the cell label of each particle, x fastest.  Particles outside
 * the domain (or with non-finite coordinates) get the label ncells.
 * Returns the number of such particles. */
int64_t or_cell_keys(const or_params *P, int64_t n, const double *x,
                     const double *y, const double *z, uint32_t *key)
{
    int64_t nc[3];
    or_grid_dims(P, nc);
    const double inv_cs = 1.0 / (2.0 * P->h);
    const uint64_t ncells = (uint64_t)nc[0] * nc[1] * nc[2];
    int64_t nout = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx, cy, cz;
        if (coord(x[i], P->dmin[0], inv_cs, nc[0], &cx) &&
            coord(y[i], P->dmin[1], inv_cs, nc[1], &cy) &&
            coord(z[i], P->dmin[2], inv_cs, nc[2], &cz)) {
            key[i] = (uint32_t)(cx + nc[0] * (cy + nc[1] * cz));
        } else {
            key[i] = (uint32_t)ncells;
            ++nout;
        }
    }
    return nout;
}

typedef struct { uint32_t key, id; int64_t idx; } kid_t;

static int cmp_kid(const void *a, const void *b)
{
    const kid_t *p = (const kid_t *)a, *q = (const kid_t *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    if (p->id != q->id) return p->id < q->id ? -1 : 1;
    return 0;
}

/* Sec. 3.1 / Sec. 4.3: order particles by (label, id); perm[k] is the input
 * index of the k-th particle in that order. */
void or_sort_by_key_id(int64_t n, const uint32_t *key, const uint32_t *id,
                       int64_t *perm)
{
    kid_t *t = (kid_t *)malloc(sizeof(kid_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { t[i].key = key[i]; t[i].id = id[i]; t[i].idx = i; }
    qsort(t, (size_t)n, sizeof(kid_t), cmp_kid);
    for (int64_t i = 0; i < n; ++i) perm[i] = t[i].idx;
    free(t);
}

/* Sec. 3.1: index of the first particle of each cell in the sorted order,
 * for cells 0..ncells (cell ncells holds the excluded particles), plus the
 * total at the end: off has ncells + 2 entries. */
void or_cell_offsets(int64_t ncells, int64_t n, const uint32_t *sorted_key,
                     uint32_t *off)
{
    int64_t k = 0;
    for (int64_t c = 0; c <= ncells + 1; ++c) {
        while (k < n && (int64_t)sorted_key[k] < c) ++k;
        off[c] = (uint32_t)k;
    }
}

/* Neighbour-search acceleration structure private to the oracle: a counting
 * sort of particle indices by cell (stable in input order). */
typedef struct {
    int64_t nc[3], ncells;
    uint32_t *key;     /* per particle */
    uint32_t *start;   /* ncells + 2 */
    uint32_t *item;    /* particle indices grouped by cell */
} grid_t;

static void grid_build(const or_params *P, int64_t n, const double *x,
                       const double *y, const double *z, grid_t *G)
{
    or_grid_dims(P, G->nc);
    G->ncells = G->nc[0] * G->nc[1] * G->nc[2];
    G->key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    G->start = (uint32_t *)calloc((size_t)G->ncells + 2, sizeof(uint32_t));
    G->item = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    or_cell_keys(P, n, x, y, z, G->key);
    for (int64_t i = 0; i < n; ++i) G->start[G->key[i] + 1]++;
    for (int64_t c = 0; c <= G->ncells; ++c) G->start[c + 1] += G->start[c];
    uint32_t *fill = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)G->ncells + 1));
    memcpy(fill, G->start, sizeof(uint32_t) * ((size_t)G->ncells + 1));
    for (int64_t i = 0; i < n; ++i) G->item[fill[G->key[i]]++] = (uint32_t)i;
    free(fill);
}

static void grid_free(grid_t *G)
{
    free(G->key); free(G->start); free(G->item);
}

/* The squared support radius (2h)^2, rounded once. */
static double support2(const or_params *P)
{
    const double s = 2.0 * P->h;
    return s * s;
}

/* Squared distance, evaluated as (dx*dx + dy*dy) + dz*dz. */
static double dist2(double dx, double dy, double dz)
{
    double d2 = dx * dx + dy * dy;
    d2 = d2 + dz * dz;
    return d2;
}

/* Growable list of neighbour indices (one per worker thread). */
typedef struct { int64_t *j; int64_t n, cap; } nlist_t;

static void nlist_push(nlist_t *L, int64_t j)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 256;
        L->j = (int64_t *)realloc(L->j, sizeof(int64_t) * (size_t)L->cap);
    }
    L->j[L->n++] = j;
}

static int within(const double *x, const double *y, const double *z,
                  int64_t i, int64_t j, double r2max)
{
    return dist2(x[i] - x[j], y[i] - y[j], z[i] - z[j]) < r2max;
}

/* The neighbours j != i of particle i: |r_ij| < 2h, both inside the domain.
 * Found through the 27 cells around i's cell (Sec. 3.2), or by brute force
 * over all particles. */
static void neighbours(const grid_t *G, int brute, int64_t n, int64_t i,
                       const double *x, const double *y, const double *z,
                       double r2max, nlist_t *L)
{
    L->n = 0;
    const uint32_t out = (uint32_t)G->ncells;
    if (G->key[i] == out) return;
    if (brute) {
        for (int64_t j = 0; j < n; ++j)
            if (j != i && G->key[j] != out && within(x, y, z, i, j, r2max))
                nlist_push(L, j);
        return;
    }
    const int64_t k = G->key[i];
    const int64_t cx = k % G->nc[0];
    const int64_t cy = (k / G->nc[0]) % G->nc[1];
    const int64_t cz = k / (G->nc[0] * G->nc[1]);
    for (int64_t zz = cz - 1; zz <= cz + 1; ++zz) {
        if (zz < 0 || zz >= G->nc[2]) continue;
        for (int64_t yy = cy - 1; yy <= cy + 1; ++yy) {
            if (yy < 0 || yy >= G->nc[1]) continue;
            for (int64_t xx = cx - 1; xx <= cx + 1; ++xx) {
                if (xx < 0 || xx >= G->nc[0]) continue;
                const int64_t c = xx + G->nc[0] * (yy + G->nc[1] * zz);
                for (uint32_t t = G->start[c]; t < G->start[c + 1]; ++t) {
                    const int64_t j = G->item[t];
                    if (j != i && within(x, y, z, i, j, r2max)) nlist_push(L, j);
                }
            }
        }
    }
}

/* Number of neighbours of each in-domain particle (0 for excluded ones). */
void or_neighbour_counts(const or_params *P, int64_t n, const double *x,
                         const double *y, const double *z, int brute,
                         uint32_t *count)
{
    grid_t G;
    grid_build(P, n, x, y, z, &G);
    const double r2max = support2(P);
#pragma omp parallel
    {
        nlist_t L = {0, 0, 0};
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; ++i) {
            neighbours(&G, brute, n, i, x, y, z, r2max, &L);
            count[i] = (uint32_t)L.n;
        }
        free(L.j);
    }
    grid_free(&G);
}

/* ------------------------------------------------------------- physics -- */

/* Smoothing kernels, q = r/h, compact support q < 2 (Sec. 2.2).
 *
 * Wendland C2:  W = aD (1 - q/2)^4 (2q + 1),  aD = 21/(16 pi h^3).
 * Cubic spline (the kernel of the paper's results), aD = 1/(pi h^3):
 *   W = aD (1 - 3/2 q^2 + 3/4 q^3)   for 0 <= q < 1,
 *   W = aD/4 (2 - q)^3               for 1 <= q < 2. */
double or_kernel_w(const or_params *P, double r)
{
    const double h = P->h;
    const double q = r / h;
    if (q >= 2.0) return 0.0;
    if (P->kernel == 1) {
        const double aD = 1.0 / (M_PI * h * h * h);
        if (q < 1.0) return aD * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
        const double w = 2.0 - q;
        return 0.25 * aD * w * w * w;
    }
    const double aD = 21.0 / (16.0 * M_PI * h * h * h);
    const double w = 1.0 - 0.5 * q;
    return aD * w * w * w * w * (2.0 * q + 1.0);
}

/* grad_i W_ij = F(r) r_ij, F = (dW/dr)/r:
 *   Wendland C2:   F = -5 aD/h^2 (1 - q/2)^3
 *   cubic spline:  F = aD/h^2 (9/4 q - 3)           for q < 1,
 *                  F = -3/4 aD/h^2 (2 - q)^2 / q    for 1 <= q < 2. */
double or_kernel_f(const or_params *P, double r)
{
    const double h = P->h;
    const double q = r / h;
    if (q >= 2.0) return 0.0;
    if (P->kernel == 1) {
        const double aD = 1.0 / (M_PI * h * h * h);
        if (q < 1.0) return aD / (h * h) * (2.25 * q - 3.0);
        const double w = 2.0 - q;
        return -0.75 * aD / (h * h) * w * w / q;
    }
    const double aD = 21.0 / (16.0 * M_PI * h * h * h);
    const double w = 1.0 - 0.5 * q;
    return -5.0 * aD / (h * h) * w * w * w;
}

/* Tait equation of state (Sec. 2.2): p = B [(rho/rho0)^gamma - 1],
 * B = c0^2 rho0 / gamma. */
double or_pressure(const or_params *P, double rho)
{
    const double B = P->c0 * P->c0 * P->rho0 / P->gamma;
    return B * (pow(rho / P->rho0, P->gamma) - 1.0);
}

/* Speed of sound sqrt(dp/drho) = c0 (rho/rho0)^((gamma-1)/2). */
double or_sound_speed(const or_params *P, double rho)
{
    return P->c0 * pow(rho / P->rho0, 0.5 * (P->gamma - 1.0));
}

/* Specific internal energy e(rho) = int_{rho0}^{rho} p(s)/s^2 ds, closed
 * form for the Tait law (used only by the diagnostics). */
double or_internal_energy(const or_params *P, double rho)
{
    const double B = P->c0 * P->c0 * P->rho0 / P->gamma;
    const double g = P->gamma;
    return B * ((pow(rho, g - 1.0) - pow(P->rho0, g - 1.0)) /
                ((g - 1.0) * pow(P->rho0, g)) + 1.0 / rho - 1.0 / P->rho0);
}

/* Right-hand sides of Eqs. 7 and 9 for particles i in [i0, i1).
 *
 * Outputs (indexed by i, left untouched outside [i0, i1)):
 *   a[3*i..]   acceleration, gravity included (computed for boundary
 *              particles too; the integrator never applies it to them)
 *   drho[i]    density rate
 *   sa[i], sd[i]  sums of the magnitudes of the pair terms (+|g| for sa):
 *              the scale used to judge relative errors where terms cancel
 *   nnb[i]     number of neighbours
 *   terms[0..2]: max |a_i| over fluid i, max c_i over all in-domain i,
 *              max over pairs with fluid i of h |v_ij.r_ij| / (r^2 + eta^2)
 * Excluded particles get zeros.  Returns the number of pairs visited. */
int64_t or_interact(const or_params *P, int64_t n,
                    const double *x, const double *y, const double *z,
                    const double *vx, const double *vy, const double *vz,
                    const double *rho, const uint32_t *id, int brute,
                    int64_t i0, int64_t i1,
                    double *a, double *drho, double *sa, double *sd,
                    uint32_t *nnb, double *terms)
{
    grid_t G;
    grid_build(P, n, x, y, z, &G);
    const double r2max = support2(P);
    const double h = P->h, m = P->mass;
    const double eta2 = P->eta2_coef * h * h;
    const double gnorm = sqrt(P->g[0] * P->g[0] + P->g[1] * P->g[1] + P->g[2] * P->g[2]);
    double amax = 0.0, cmax = 0.0, mumax = 0.0;
    int64_t npairs = 0;
    if (i0 < 0) i0 = 0;
    if (i1 > n) i1 = n;

#pragma omp parallel reduction(max: amax, cmax, mumax) reduction(+: npairs)
    {
        nlist_t L = {0, 0, 0};
#pragma omp for schedule(dynamic, 128)
        for (int64_t i = i0; i < i1; ++i) {
            if (G.key[i] == (uint32_t)G.ncells) {
                a[3 * i] = a[3 * i + 1] = a[3 * i + 2] = 0.0;
                drho[i] = 0.0; sa[i] = sd[i] = 0.0; nnb[i] = 0;
                continue;
            }
            const int fluid = (int64_t)id[i] >= P->n_bound;
            const double Pi_ = or_pressure(P, rho[i]) / (rho[i] * rho[i]);
            const double ci = or_sound_speed(P, rho[i]);
            double ax = 0, ay = 0, az = 0, dr = 0, s_a = 0, s_d = 0, mu = 0;
            neighbours(&G, brute, n, i, x, y, z, r2max, &L);
            for (int64_t t = 0; t < L.n; ++t) {
                const int64_t j = L.j[t];
                const double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
                const double d2 = dist2(dx, dy, dz);
                const double r = sqrt(d2);
                const double F = or_kernel_f(P, r);
                const double dvx = vx[i] - vx[j], dvy = vy[i] - vy[j], dvz = vz[i] - vz[j];
                const double vr = dvx * dx + dvy * dy + dvz * dz;
                /* Eq. 7 */
                dr += m * vr * F;
                s_d += fabs(m * vr * F);
                /* Sec. 2.2: artificial viscosity for approaching pairs */
                const double nu = h * vr / (d2 + eta2);
                double visc = 0.0;
                if (vr < 0.0) {
                    const double cbar = 0.5 * (ci + or_sound_speed(P, rho[j]));
                    const double rbar = 0.5 * (rho[i] + rho[j]);
                    visc = -P->alpha * cbar * nu / rbar;
                }
                /* Eq. 9 with P = p / rho^2 */
                const double Pj = or_pressure(P, rho[j]) / (rho[j] * rho[j]);
                const double coef = m * (Pi_ + Pj + visc) * F;
                ax -= coef * dx; ay -= coef * dy; az -= coef * dz;
                s_a += fabs(coef) * r;
                if (fabs(nu) > mu) mu = fabs(nu);
            }
            ax += P->g[0]; ay += P->g[1]; az += P->g[2];
            a[3 * i] = ax; a[3 * i + 1] = ay; a[3 * i + 2] = az;
            drho[i] = dr; sa[i] = s_a + gnorm; sd[i] = s_d; nnb[i] = (uint32_t)L.n;
            npairs += L.n;
            if (ci > cmax) cmax = ci;
            if (fluid) {
                const double an = sqrt(ax * ax + ay * ay + az * az);
                if (an > amax) amax = an;
                if (mu > mumax) mumax = mu;
            }
        }
        free(L.j);
    }
    terms[0] = amax; terms[1] = cmax; terms[2] = mumax;
    grid_free(&G);
    return npairs;
}

/* Sec. 3.3: CFL-limited step from the reduction terms of one evaluation. */
double or_dt(const or_params *P, const double *terms)
{
    const double h = P->h;
    double dtf = INFINITY;
    if (terms[0] > 0.0) dtf = sqrt(h / terms[0]);
    const double dtcv = h / (terms[1] + terms[2]);
    return P->cfl * (dtf < dtcv ? dtf : dtcv);
}

static int is_in(const or_params *P, const int64_t nc[3], double x, double y,
                 double z)
{
    int64_t c;
    const double inv_cs = 1.0 / (2.0 * P->h);
    return coord(x, P->dmin[0], inv_cs, nc[0], &c) && coord(y, P->dmin[1], inv_cs, nc[1], &c) &&
           coord(z, P->dmin[2], inv_cs, nc[2], &c);
}

/* Predictor half step (symplectic scheme):
 *   fluid:  r' = r + (dt/2) v,  v' = v + (dt/2) a
 *   all:    rho' = rho + (dt/2) drho
 * Boundary particles keep r and v (Sec. 2.3); excluded particles are left
 * unchanged.  Arrays are updated in place. */
void or_predict(const or_params *P, int64_t n, double *x, double *y, double *z,
                double *vx, double *vy, double *vz, double *rho,
                const uint32_t *id, const double *a, const double *drho,
                double dt)
{
    int64_t nc[3];
    or_grid_dims(P, nc);
    const double hdt = 0.5 * dt;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (!is_in(P, nc, x[i], y[i], z[i])) continue;
        if ((int64_t)id[i] >= P->n_bound) {
            x[i] = x[i] + hdt * vx[i];
            y[i] = y[i] + hdt * vy[i];
            z[i] = z[i] + hdt * vz[i];
            vx[i] = vx[i] + hdt * a[3 * i];
            vy[i] = vy[i] + hdt * a[3 * i + 1];
            vz[i] = vz[i] + hdt * a[3 * i + 2];
        }
        rho[i] = rho[i] + hdt * drho[i];
    }
}

/* Corrector (symplectic scheme), from the state at the start of the step
 * (x0.., v0.., rho0_) and the half-step density rhoh with the rates a, drho
 * evaluated at the half step:
 *   fluid:  v1 = v0 + dt a,   r1 = r0 + (dt/2) (v1 + v0)
 *   all:    eps = -drho dt / rhoh,  rho1 = rho0 (2 - eps) / (2 + eps)
 * Particles excluded at the half step keep their half-step state (passed in
 * x,y,z,vx,vy,vz,rho on entry); results overwrite those arrays. */
void or_correct(const or_params *P, int64_t n,
                const double *x0, const double *y0, const double *z0,
                const double *vx0, const double *vy0, const double *vz0,
                const double *rho0_,
                double *x, double *y, double *z, double *vx, double *vy,
                double *vz, double *rho, const uint32_t *id, const double *a,
                const double *drho, double dt)
{
    int64_t nc[3];
    or_grid_dims(P, nc);
    const double hdt = 0.5 * dt;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (!is_in(P, nc, x[i], y[i], z[i])) continue;
        if ((int64_t)id[i] >= P->n_bound) {
            const double ux = vx0[i] + dt * a[3 * i];
            const double uy = vy0[i] + dt * a[3 * i + 1];
            const double uz = vz0[i] + dt * a[3 * i + 2];
            x[i] = x0[i] + hdt * (ux + vx0[i]);
            y[i] = y0[i] + hdt * (uy + vy0[i]);
            z[i] = z0[i] + hdt * (uz + vz0[i]);
            vx[i] = ux; vy[i] = uy; vz[i] = uz;
        }
        const double eps = -(drho[i] * dt) / rho[i];
        rho[i] = rho0_[i] * ((2.0 - eps) / (2.0 + eps));
    }
}

/* One full step: evaluate at S^n, set dt (or use dt_fixed > 0), predictor,
 * evaluate at the half step, corrector.  The cell list is rebuilt before each
 * evaluation.  State arrays are updated in place; returns the dt used. */
double or_step(const or_params *P, int64_t n, double *x, double *y, double *z,
               double *vx, double *vy, double *vz, double *rho,
               const uint32_t *id, double dt_fixed, int brute,
               int64_t *pairs_out)
{
    const size_t N = (size_t)(n > 0 ? n : 1);
    double *a = (double *)malloc(sizeof(double) * 3 * N);
    double *dr = (double *)malloc(sizeof(double) * N);
    double *sa = (double *)malloc(sizeof(double) * N);
    double *sd = (double *)malloc(sizeof(double) * N);
    uint32_t *nn = (uint32_t *)malloc(sizeof(uint32_t) * N);
    double *s0 = (double *)malloc(sizeof(double) * 7 * N);
    double terms[3];
    int64_t pairs = or_interact(P, n, x, y, z, vx, vy, vz, rho, id, brute, 0, n,
                                a, dr, sa, sd, nn, terms);
    const double dt = dt_fixed > 0.0 ? dt_fixed : or_dt(P, terms);
    memcpy(s0 + 0 * N, x, sizeof(double) * (size_t)n);
    memcpy(s0 + 1 * N, y, sizeof(double) * (size_t)n);
    memcpy(s0 + 2 * N, z, sizeof(double) * (size_t)n);
    memcpy(s0 + 3 * N, vx, sizeof(double) * (size_t)n);
    memcpy(s0 + 4 * N, vy, sizeof(double) * (size_t)n);
    memcpy(s0 + 5 * N, vz, sizeof(double) * (size_t)n);
    memcpy(s0 + 6 * N, rho, sizeof(double) * (size_t)n);
    or_predict(P, n, x, y, z, vx, vy, vz, rho, id, a, dr, dt);
    pairs += or_interact(P, n, x, y, z, vx, vy, vz, rho, id, brute, 0, n,
                         a, dr, sa, sd, nn, terms);
    or_correct(P, n, s0, s0 + N, s0 + 2 * N, s0 + 3 * N, s0 + 4 * N, s0 + 5 * N,
               s0 + 6 * N, x, y, z, vx, vy, vz, rho, id, a, dr, dt);
    if (pairs_out) *pairs_out = pairs;
    free(a); free(dr); free(sa); free(sd); free(nn); free(s0);
    return dt;
}

/* Verlet update (Sec. 3.3, in the SPHysics form): from the state S^n (x..rho,
 * updated in place), the state one step earlier (vxm, vym, vzm, rhom) and
 * the rates at S^n (a, drho):
 *   fluid:          r1 = r + dt v + (dt^2/2) a
 *                   v1 = vm + 2 dt a      (leapfrog step)
 *                   v1 = v  + dt a        (Euler step, euler != 0)
 *   all in-domain:  rho1 = rhom + 2 dt drho  (leapfrog)
 *                   rho1 = rho  + dt drho    (Euler)
 * Boundary particles keep r and v (Sec. 2.3).  On return (vxm.., rhom) holds
 * the state on entry, i.e. S^n becomes the earlier state of the next step.
 * Excluded particles are left unchanged (both states). */
void or_verlet_update(const or_params *P, int64_t n, double *x, double *y,
                      double *z, double *vx, double *vy, double *vz,
                      double *rho, double *vxm, double *vym, double *vzm,
                      double *rhom, const uint32_t *id, const double *a,
                      const double *drho, double dt, int euler)
{
    int64_t nc[3];
    or_grid_dims(P, nc);
    const double dt2h = 0.5 * dt * dt;
    const double dtv = euler ? dt : 2.0 * dt;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (!is_in(P, nc, x[i], y[i], z[i])) continue;
        const double ux = vx[i], uy = vy[i], uz = vz[i], r = rho[i];
        if ((int64_t)id[i] >= P->n_bound) {
            x[i] = x[i] + (dt * ux + dt2h * a[3 * i]);
            y[i] = y[i] + (dt * uy + dt2h * a[3 * i + 1]);
            z[i] = z[i] + (dt * uz + dt2h * a[3 * i + 2]);
            vx[i] = (euler ? ux : vxm[i]) + dtv * a[3 * i];
            vy[i] = (euler ? uy : vym[i]) + dtv * a[3 * i + 1];
            vz[i] = (euler ? uz : vzm[i]) + dtv * a[3 * i + 2];
        }
        rho[i] = (euler ? r : rhom[i]) + dtv * drho[i];
        vxm[i] = ux; vym[i] = uy; vzm[i] = uz; rhom[i] = r;
    }
}

/* One Verlet step: evaluate at S^n (cell list rebuilt), set dt from that
 * evaluation (or use dt_fixed > 0), update.  Returns the dt used. */
double or_verlet_step(const or_params *P, int64_t n, double *x, double *y,
                      double *z, double *vx, double *vy, double *vz,
                      double *rho, double *vxm, double *vym, double *vzm,
                      double *rhom, const uint32_t *id, double dt_fixed,
                      int euler, int brute, int64_t *pairs_out)
{
    const size_t N = (size_t)(n > 0 ? n : 1);
    double *a = (double *)malloc(sizeof(double) * 3 * N);
    double *dr = (double *)malloc(sizeof(double) * N);
    double *sa = (double *)malloc(sizeof(double) * N);
    double *sd = (double *)malloc(sizeof(double) * N);
    uint32_t *nn = (uint32_t *)malloc(sizeof(uint32_t) * N);
    double terms[3];
    const int64_t pairs = or_interact(P, n, x, y, z, vx, vy, vz, rho, id, brute,
                                      0, n, a, dr, sa, sd, nn, terms);
    const double dt = dt_fixed > 0.0 ? dt_fixed : or_dt(P, terms);
    or_verlet_update(P, n, x, y, z, vx, vy, vz, rho, vxm, vym, vzm, rhom, id,
                     a, dr, dt, euler);
    if (pairs_out) *pairs_out = pairs;
    free(a); free(dr); free(sa); free(sd); free(nn);
    return dt;
}

/* Sec. 4.2-4.3: labels of a one-dimensional decomposition along x, for the
 * sub-domain [xlo, xhi) that holds this particle set.
 *   mode 0, edge (the data that builds the neighbours' halos):
 *       1 if xlo <= x < xlo + 2h   (left edge)
 *       2 if xhi - 2h <= x < xhi   (right edge)
 *       0 otherwise
 *   mode 1, migration: 1 if x < xlo (moved to the left neighbour),
 *       2 if x >= xhi (moved to the right neighbour), 0 otherwise.
 * xlo + 2h and xhi - 2h are each rounded once.  The edge mode needs
 * xhi - xlo >= 4h, so that no particle belongs to both edges.  Particles
 * outside the cell-grid domain get 0.  Returns the number labelled 1 or 2. */
int64_t or_subdomain_labels(const or_params *P, int64_t n, const double *x,
                            const double *y, const double *z, int mode,
                            double xlo, double xhi, uint32_t *label)
{
    int64_t nc[3];
    or_grid_dims(P, nc);
    const double cs = 2.0 * P->h;
    const double lo_edge = xlo + cs, hi_edge = xhi - cs;
    int64_t sel = 0;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t l = 0;
        if (is_in(P, nc, x[i], y[i], z[i])) {
            if (mode == 0) {
                if (x[i] >= xlo && x[i] < lo_edge) l = 1;
                else if (x[i] >= hi_edge && x[i] < xhi) l = 2;
            } else {
                if (x[i] < xlo) l = 1;
                else if (x[i] >= xhi) l = 2;
            }
        }
        label[i] = l;
        sel += l != 0;
    }
    return sel;
}

/* Conservation diagnostics over in-domain particles:
 * out[0] total mass, out[1..3] fluid momentum, out[4] fluid kinetic energy,
 * out[5] fluid potential energy -m g.r, out[6] internal energy sum m e(rho)
 * over all in-domain particles, out[7] number of excluded particles. */
void or_diagnostics(const or_params *P, int64_t n, const double *x,
                    const double *y, const double *z, const double *vx,
                    const double *vy, const double *vz, const double *rho,
                    const uint32_t *id, double *out)
{
    int64_t nc[3];
    or_grid_dims(P, nc);
    const double m = P->mass;
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = 0; i < n; ++i) {
        if (!is_in(P, nc, x[i], y[i], z[i])) { s[7] += 1.0; continue; }
        s[0] += m;
        s[6] += m * or_internal_energy(P, rho[i]);
        if ((int64_t)id[i] >= P->n_bound) {
            s[1] += m * vx[i]; s[2] += m * vy[i]; s[3] += m * vz[i];
            s[4] += 0.5 * m * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]);
            s[5] -= m * (P->g[0] * x[i] + P->g[1] * y[i] + P->g[2] * z[i]);
        }
    }
    memcpy(out, s, sizeof(s));
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
