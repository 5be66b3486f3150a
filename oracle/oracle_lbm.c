/*
 * oracle_lbm.c -- plain, slow, FP64 CPU oracle of the two-component
 * pseudopotential D3Q19 lattice Boltzmann time step of Sedahmed, Coelho,
 * Araujo, Wahba, Warda, "Study of fluid displacement in three-dimensional
 * porous media with an improved multi-component pseudopotential lattice
 * Boltzmann method", Phys. Fluids (2022), arXiv 2207.01534.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The product (the CUDA
 * library and its Python binding) never links, imports or calls it, and it
 * shares no code, table or helper with the product.
 *
 * Deliberately unlike the GPU path:
 *   - dense nx*ny*nz arrays with a solid mask (no compaction),
 *   - two population arrays with pull streaming (no in-place A-A),
 *   - neighbour coordinates by direct arithmetic with modulo wrap,
 *   - FP64 everywhere, compiled with -ffp-contract=off.
 *
 * One time step, in this order (Section 2, with a reading noted wherever the paper is silent or garbled):
 *   1. densities and momenta of every fluid node              (Eqs. 3-4)
 *   2. virtual solid density of every solid node               (Eqs. 14-15)
 *   3. total force: cohesion + adhesion + body force          (Eqs. 10, 11, 13)
 *      with mirrored pseudopotential beyond open planes       (Section 2)
 *   4. mixture relaxation time and equilibrium velocity       (Eqs. 6-8)
 *   5. collision with the explicit-forcing source term        (Eqs. 1, 2, 9)
 *   6. pull streaming with half-way bounce-back, periodic wrap
 *      and frozen missing populations at the open planes      (Eq. 1, Section 2)
 *   7. non-equilibrium extrapolation (or the Zou-He method) for
 *      the prescribed component at the inlet (component 1) and
 *      outlet (2)                                              (Section 2, 4.1)
 *
 * Parity pins: every function is checked by tests against closed forms,
 * conservation laws, symmetries and the paper's printed physics (tests marked
 * "not gpu").  The porous-medium P_c-S_w values of Section 4 are dataset
 * specific: parity unpinned for those outputs.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* D3Q19 velocities, written column by column from the matrix printed in
 * Section 2 (rows are the x, y and z components). */
static const int EX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
/* D3Q19 weights, Section 2. */
static const double WT[Q] = {1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                             1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* Lattice sound speed squared, c_s^2 = 1/3 (Section 2, dx = dt = 1). */
static const double CS2 = 1.0 / 3.0;

typedef struct ora {
    int n[3];          /* nx, ny, nz (x fastest) */
    long nv;           /* nx*ny*nz */
    unsigned char *solid;
    int periodic[3];
    int open_axis;     /* -1: none; else the axis of the inlet (coordinate 0)
                          and outlet (coordinate n-1) planes */
    double *xi;        /* per-voxel wettability parameter xi (Eq. 15 chi) */
    double tau[2];     /* tau^(1), tau^(2) */
    double G;          /* G_coh^(sigma sigma-bar) */
    double rho_in1;    /* prescribed component-1 density at the inlet */
    double rho_out2;   /* prescribed component-2 density at the outlet */
    double g[3];       /* body acceleration, F^b = rho^sigma g */
    int velocity_shift;/* 0: Eq. 8 with Eq. 4 moments; 1: add F/2 to momenta */
    int opp[Q];
    int mirror[Q];     /* direction reflected across the open planes */
    double *f[2];      /* post-stream populations, [i*nv + v] */
    double *fs[2];     /* post-collision scratch, [i*nv + v] */
    double *f0[2];     /* populations at initialisation (frozen values) */
    double *rho[2];    /* fluid: rho^sigma; solid: rho-tilde^sigma */
    double *mom[2];    /* sum_i e_i f_i, [3*v + a] */
    double *F[2];      /* total force, [3*v + a] */
    long step;
    int bc;            /* 0: non-equilibrium extrapolation, 1: Zou-He */
    double *tape;      /* recorded states for the adjoint: (tape_len) x [2][Q*nv] */
    long tape_len;
} ora_t;

void ora_destroy(ora_t *o);

static void set_err(char *err, int errlen, const char *msg)
{
    if (err && errlen > 0) {
        strncpy(err, msg, (size_t)errlen - 1);
        err[errlen - 1] = 0;
    }
}

/* Index of the direction whose velocity equals (cx, cy, cz), -1 if none. */
static int find_dir(int cx, int cy, int cz)
{
    for (int j = 0; j < Q; ++j)
        if (EX[j] == cx && EY[j] == cy && EZ[j] == cz) return j;
    return -1;
}

void ora_lattice(int *e, double *w, int *opp)
{
    for (int i = 0; i < Q; ++i) {
        e[3 * i + 0] = EX[i];
        e[3 * i + 1] = EY[i];
        e[3 * i + 2] = EZ[i];
        w[i] = WT[i];
        opp[i] = find_dir(-EX[i], -EY[i], -EZ[i]);
    }
}

/* Mirror map across a plane normal to `axis` (Section 2, generalised from the
 * printed left-boundary example: psi(x + e_j) := psi(x + e_mirror[j]) where
 * e_mirror[j] is e_j with its axis component negated). */
void ora_mirror_map(int axis, int *map)
{
    for (int i = 0; i < Q; ++i) {
        int c[3] = {EX[i], EY[i], EZ[i]};
        c[axis] = -c[axis];
        map[i] = find_dir(c[0], c[1], c[2]);
    }
}

/* Equilibrium distribution, Eq. 2. */
static double feq_i(int i, double rho, const double u[3])
{
    double eu = EX[i] * u[0] + EY[i] * u[1] + EZ[i] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return WT[i] * rho * (1.0 + eu / CS2 + (eu * eu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Explicit-forcing source term, Eq. 9. */
static double src_i(int i, const double u[3], const double F[3])
{
    double e[3] = {(double)EX[i], (double)EY[i], (double)EZ[i]};
    double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
    double s = 0.0;
    for (int a = 0; a < 3; ++a) s += ((e[a] - u[a]) / CS2 + eu * e[a] / (CS2 * CS2)) * F[a];
    return WT[i] * s;
}

void ora_feq(double rho, const double *u, double *out)
{
    for (int i = 0; i < Q; ++i) out[i] = feq_i(i, rho, u);
}

void ora_source(const double *u, const double *F, double *out)
{
    for (int i = 0; i < Q; ++i) out[i] = src_i(i, u, F);
}

static long vid(const ora_t *o, const int c[3]) { return c[0] + (long)o->n[0] * (c[1] + (long)o->n[1] * c[2]); }

static void coords(const ora_t *o, long v, int c[3])
{
    c[0] = (int)(v % o->n[0]);
    c[1] = (int)((v / o->n[0]) % o->n[1]);
    c[2] = (int)(v / ((long)o->n[0] * o->n[1]));
}

/* Neighbour of voxel c in direction (dx, dy, dz): 0 and *out set when it lies
 * in the domain (after periodic wrap), 1 when it lies outside. */
static int neighbour(const ora_t *o, const int c[3], int dx, int dy, int dz, long *out)
{
    int d[3] = {dx, dy, dz};
    int m[3];
    for (int a = 0; a < 3; ++a) {
        m[a] = c[a] + d[a];
        if (m[a] < 0 || m[a] >= o->n[a]) {
            if (!o->periodic[a]) return 1;
            m[a] = (m[a] + o->n[a]) % o->n[a];
        }
    }
    *out = vid(o, m);
    return 0;
}

ora_t *ora_create(int nx, int ny, int nz, const unsigned char *solid, const int *periodic, int open_axis,
                  const double *xi_field, double xi, const double *tau, double G, double rho_in1,
                  double rho_out2, const double *g, int velocity_shift, char *err, int errlen)
{
    if (nx < 1 || ny < 1 || nz < 1) {
        set_err(err, errlen, "dimensions must be positive");
        return NULL;
    }
    if (open_axis < -1 || open_axis > 2) {
        set_err(err, errlen, "open_axis must be -1, 0, 1 or 2");
        return NULL;
    }
    int n[3] = {nx, ny, nz};
    if (open_axis >= 0 && (periodic[open_axis] || n[open_axis] < 3)) {
        set_err(err, errlen, "the open axis must be non-periodic and at least 3 voxels long");
        return NULL;
    }
    ora_t *o = (ora_t *)calloc(1, sizeof(ora_t));
    for (int a = 0; a < 3; ++a) {
        o->n[a] = n[a];
        o->periodic[a] = periodic[a] ? 1 : 0;
        o->g[a] = g ? g[a] : 0.0;
    }
    o->nv = (long)nx * ny * nz;
    o->open_axis = open_axis;
    o->tau[0] = tau[0];
    o->tau[1] = tau[1];
    o->G = G;
    o->rho_in1 = rho_in1;
    o->rho_out2 = rho_out2;
    o->velocity_shift = velocity_shift;
    for (int i = 0; i < Q; ++i) o->opp[i] = find_dir(-EX[i], -EY[i], -EZ[i]);
    if (open_axis >= 0)
        ora_mirror_map(open_axis, o->mirror);
    else
        for (int i = 0; i < Q; ++i) o->mirror[i] = i;
    o->solid = (unsigned char *)malloc((size_t)o->nv);
    o->xi = (double *)malloc(sizeof(double) * (size_t)o->nv);
    for (long v = 0; v < o->nv; ++v) {
        o->solid[v] = solid[v] ? 1 : 0;
        o->xi[v] = xi_field ? xi_field[v] : xi;
    }
    for (int s = 0; s < 2; ++s) {
        o->f[s] = (double *)calloc((size_t)o->nv * Q, sizeof(double));
        o->fs[s] = (double *)calloc((size_t)o->nv * Q, sizeof(double));
        o->f0[s] = (double *)calloc((size_t)o->nv * Q, sizeof(double));
        o->rho[s] = (double *)calloc((size_t)o->nv, sizeof(double));
        o->mom[s] = (double *)calloc((size_t)o->nv * 3, sizeof(double));
        o->F[s] = (double *)calloc((size_t)o->nv * 3, sizeof(double));
    }
    /* A fluid node may only see outside the domain across the open planes:
     * non-periodic lateral faces must be closed by solid voxels. */
    for (long v = 0; v < o->nv; ++v) {
        if (o->solid[v]) continue;
        int c[3];
        coords(o, v, c);
        for (int i = 1; i < Q; ++i) {
            int e[3] = {EX[i], EY[i], EZ[i]};
            for (int a = 0; a < 3; ++a) {
                int m = c[a] + e[a];
                if ((m < 0 || m >= n[a]) && !o->periodic[a] && a != open_axis) {
                    set_err(err, errlen, "a fluid voxel touches a closed (non-periodic, non-open) face");
                    ora_destroy(o);
                    return NULL;
                }
            }
        }
    }
    /* The non-equilibrium extrapolation needs a fluid interior neighbour. */
    if (open_axis >= 0) {
        for (long v = 0; v < o->nv; ++v) {
            if (o->solid[v]) continue;
            int c[3];
            coords(o, v, c);
            int k = c[open_axis];
            if (k != 0 && k != n[open_axis] - 1) continue;
            int d[3] = {0, 0, 0};
            d[open_axis] = (k == 0) ? 1 : -1;
            long nb;
            neighbour(o, c, d[0], d[1], d[2], &nb);
            if (o->solid[nb]) {
                set_err(err, errlen, "an open-plane fluid voxel has a solid interior neighbour");
                ora_destroy(o);
                return NULL;
            }
        }
    }
    return o;
}

void ora_destroy(ora_t *o)
{
    if (!o) return;
    for (int s = 0; s < 2; ++s) {
        free(o->f[s]);
        free(o->fs[s]);
        free(o->f0[s]);
        free(o->rho[s]);
        free(o->mom[s]);
        free(o->F[s]);
    }
    free(o->solid);
    free(o->xi);
    free(o->tape);
    free(o);
}

static void snapshot_frozen(ora_t *o)
{
    for (int s = 0; s < 2; ++s) memcpy(o->f0[s], o->f[s], sizeof(double) * (size_t)o->nv * Q);
}

/* Rest equilibrium (Eq. 2 with u = 0) for given component densities. */
int ora_init_densities(ora_t *o, const double *rho1, const double *rho2)
{
    const double *r[2] = {rho1, rho2};
    double u0[3] = {0, 0, 0};
    for (int s = 0; s < 2; ++s)
        for (long v = 0; v < o->nv; ++v)
            for (int i = 0; i < Q; ++i) o->f[s][i * o->nv + v] = o->solid[v] ? 0.0 : feq_i(i, r[s][v], u0);
    snapshot_frozen(o);
    o->step = 0;
    return 0;
}

int ora_set_pops(ora_t *o, const double *f1, const double *f2)
{
    const double *src[2] = {f1, f2};
    for (int s = 0; s < 2; ++s)
        for (long k = 0; k < o->nv * Q; ++k) o->f[s][k] = o->solid[k % o->nv] ? 0.0 : src[s][k];
    snapshot_frozen(o);
    return 0;
}

void ora_get_pops(const ora_t *o, double *f1, double *f2)
{
    memcpy(f1, o->f[0], sizeof(double) * (size_t)o->nv * Q);
    memcpy(f2, o->f[1], sizeof(double) * (size_t)o->nv * Q);
}

void ora_set_inlet(ora_t *o, double rho_in1) { o->rho_in1 = rho_in1; }

long ora_step_count(const ora_t *o) { return o->step; }

/* Step 1: Eqs. 3-4 on fluid nodes. */
static void compute_moments(ora_t *o)
{
    const long nv = o->nv;
#pragma omp parallel for schedule(static)
    for (long v = 0; v < nv; ++v) {
        for (int s = 0; s < 2; ++s) {
            double r = 0, m[3] = {0, 0, 0};
            if (!o->solid[v]) {
                for (int i = 0; i < Q; ++i) {
                    double fi = o->f[s][i * nv + v];
                    r += fi;
                    m[0] += EX[i] * fi;
                    m[1] += EY[i] * fi;
                    m[2] += EZ[i] * fi;
                }
            }
            o->rho[s][v] = r;
            for (int a = 0; a < 3; ++a) o->mom[s][3 * v + a] = m[a];
        }
    }
}

/* Step 2: virtual solid density, Eqs. 14-15, with chi^(1) = 1 + xi and
 * chi^(2) = 1 - xi (Section 2).  Neighbours outside the domain take part in
 * neither sum; a solid with no fluid neighbour gets 0 (never read). */
static void compute_virtual_density(ora_t *o)
{
    const long nv = o->nv;
#pragma omp parallel for schedule(static)
    for (long v = 0; v < nv; ++v) {
        if (!o->solid[v]) continue;
        int c[3];
        coords(o, v, c);
        double num[2] = {0, 0}, den = 0;
        for (int i = 1; i < Q; ++i) {
            long nb;
            if (neighbour(o, c, EX[i], EY[i], EZ[i], &nb)) continue;
            double phi = o->solid[nb] ? 1.0 : 0.0;
            num[0] += WT[i] * o->rho[0][nb] * (1.0 - phi);
            num[1] += WT[i] * o->rho[1][nb] * (1.0 - phi);
            den += WT[i] * (1.0 - phi);
        }
        double chi[2] = {1.0 + o->xi[v], 1.0 - o->xi[v]};
        for (int s = 0; s < 2; ++s) o->rho[s][v] = (den > 0) ? chi[s] * num[s] / den : 0.0;
    }
}

/* Step 3: F^tot = F^ff + F^fs + F^b (Eqs. 10, 11, 13).  psi = rho on fluid
 * neighbours (Eq. 11); s = phi * rho-tilde on solid neighbours (Eqs. 13-14);
 * beyond an open plane the neighbour value is taken from the mirrored
 * direction (Section 2).  G^(sigma sigma) = 0: only the other component acts. */
static void compute_forces(ora_t *o)
{
    const long nv = o->nv;
#pragma omp parallel for schedule(static)
    for (long v = 0; v < nv; ++v) {
        if (o->solid[v]) continue;
        int c[3];
        coords(o, v, c);
        for (int s = 0; s < 2; ++s) {
            int sb = 1 - s;
            double acc[3] = {0, 0, 0};
            for (int i = 1; i < Q; ++i) {
                long nb;
                if (neighbour(o, c, EX[i], EY[i], EZ[i], &nb)) {
                    int j = o->mirror[i];
                    if (neighbour(o, c, EX[j], EY[j], EZ[j], &nb)) continue; /* cannot happen */
                }
                double psi_nb = o->rho[sb][nb]; /* rho on fluid, rho-tilde on solid */
                acc[0] += WT[i] * psi_nb * EX[i];
                acc[1] += WT[i] * psi_nb * EY[i];
                acc[2] += WT[i] * psi_nb * EZ[i];
            }
            for (int a = 0; a < 3; ++a)
                o->F[s][3 * v + a] = -o->G * o->rho[s][v] * acc[a] + o->rho[s][v] * o->g[a];
        }
    }
}

/* Eqs. 6-7 (with nu = c_s^2 (tau - 1/2)) and Eq. 8 at one fluid node. */
static void relaxation_and_velocity(const ora_t *o, long v, double *tau_s, double u[3])
{
    double r1 = o->rho[0][v], r2 = o->rho[1][v];
    double rho = r1 + r2;
    double nu1 = CS2 * (o->tau[0] - 0.5), nu2 = CS2 * (o->tau[1] - 0.5);
    *tau_s = (r1 * nu1 + r2 * nu2) / (rho * CS2) + 0.5;
    double den = r1 / *tau_s + r2 / *tau_s;
    for (int a = 0; a < 3; ++a) {
        double p1 = o->mom[0][3 * v + a], p2 = o->mom[1][3 * v + a];
        if (o->velocity_shift) {
            p1 += 0.5 * o->F[0][3 * v + a];
            p2 += 0.5 * o->F[1][3 * v + a];
        }
        u[a] = (p1 / *tau_s + p2 / *tau_s) / den;
    }
}

/* Step 5: Eq. 1 right-hand side into fs. */
static void collide(ora_t *o)
{
    const long nv = o->nv;
#pragma omp parallel for schedule(static)
    for (long v = 0; v < nv; ++v) {
        if (o->solid[v]) continue;
        double tau_s, u[3];
        relaxation_and_velocity(o, v, &tau_s, u);
        for (int s = 0; s < 2; ++s) {
            const double *F = &o->F[s][3 * v];
            for (int i = 0; i < Q; ++i) {
                double fi = o->f[s][i * nv + v];
                double fe = feq_i(i, o->rho[s][v], u);
                o->fs[s][i * nv + v] = fi - (fi - fe) / tau_s + (1.0 - 1.0 / (2.0 * tau_s)) * src_i(i, u, F);
            }
        }
    }
}

/* Step 6: pull streaming.  Source x - e_i solid: half-way bounce-back,
 * f_i(x) = f*_opp(i)(x).  Source outside an open plane: the population is
 * missing and keeps its initial value (Section 2, open boundary rule 2). */
static void stream(ora_t *o)
{
    const long nv = o->nv;
#pragma omp parallel for schedule(static)
    for (long v = 0; v < nv; ++v) {
        if (o->solid[v]) continue;
        int c[3];
        coords(o, v, c);
        for (int s = 0; s < 2; ++s) {
            o->f[s][v] = o->fs[s][v]; /* rest population */
            for (int i = 1; i < Q; ++i) {
                long src;
                double val;
                if (neighbour(o, c, -EX[i], -EY[i], -EZ[i], &src))
                    val = o->f0[s][i * nv + v];
                else if (o->solid[src])
                    val = o->fs[s][o->opp[i] * nv + v];
                else
                    val = o->fs[s][i * nv + src];
                o->f[s][i * nv + v] = val;
            }
        }
    }
}

/* Step 7: non-equilibrium extrapolation (Section 2 rule 1, Section 4.1) of
 * the prescribed component at an open plane node xb from its first interior
 * node xi: f(xb) = f^eq(rho_b, u(xi)) + f(xi) - f^eq(rho(xi), u(xi)), where u
 * is the post-stream barycentric velocity (sum of momenta over total density)
 * of the interior node. */
static void neem_plane(ora_t *o, int plane, int comp, double rho_b, int inward)
{
    const int ax = o->open_axis;
    const long nv = o->nv;
    int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
#pragma omp parallel for schedule(static)
    for (int p2 = 0; p2 < o->n[a2]; ++p2) {
        for (int p1 = 0; p1 < o->n[a1]; ++p1) {
            int c[3];
            c[ax] = plane;
            c[a1] = p1;
            c[a2] = p2;
            long xb = vid(o, c);
            if (o->solid[xb]) continue;
            c[ax] = plane + inward;
            long xi = vid(o, c);
            double r[2] = {0, 0}, m[3] = {0, 0, 0};
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < Q; ++i) {
                    double fi = o->f[s][i * nv + xi];
                    r[s] += fi;
                    m[0] += EX[i] * fi;
                    m[1] += EY[i] * fi;
                    m[2] += EZ[i] * fi;
                }
            double u[3] = {m[0] / (r[0] + r[1]), m[1] / (r[0] + r[1]), m[2] / (r[0] + r[1])};
            for (int i = 0; i < Q; ++i)
                o->f[comp][i * nv + xb] = feq_i(i, rho_b, u) + o->f[comp][i * nv + xi] - feq_i(i, r[comp], u);
        }
    }
}

/* Step 7 with the Zou-He method (Section 2 rule 1, Zou and He 1997): at an
 * open-plane node xb the prescribed component's populations that enter from
 * outside are unknown after streaming.  They are set so that the node's
 * component density is rho_b, its velocity is normal to the plane (no
 * tangential velocity), and the non-equilibrium parts of each unknown and its
 * opposite agree up to a tangential correction:
 *   f_i = f_opp(i) + 6 w_i rho_b (e_i . n) u_n - (e_i,t1 N_t1 + e_i,t2 N_t2),
 * with n the inward normal, u_n the normal velocity fixed by the density,
 *   rho_b u_n = rho_b - (sum of the in-plane populations
 *                        + 2 sum of the outgoing populations),
 * and N_t = (1/2) sum over in-plane populations of e_t f (so the tangential
 * momentum vanishes).  The other populations of the node are kept. */
static void zou_he_plane(ora_t *o, int plane, int comp, double rho_b, int inward)
{
    const int ax = o->open_axis;
    const long nv = o->nv;
    const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
#pragma omp parallel for schedule(static)
    for (int p2 = 0; p2 < o->n[a2]; ++p2) {
        for (int p1 = 0; p1 < o->n[a1]; ++p1) {
            int c[3];
            c[ax] = plane;
            c[a1] = p1;
            c[a2] = p2;
            const long xb = vid(o, c);
            if (o->solid[xb]) continue;
            double *f = o->f[comp];
            double s0 = 0, sout = 0, nt[3] = {0, 0, 0};
            for (int i = 0; i < Q; ++i) {
                const int e[3] = {EX[i], EY[i], EZ[i]};
                const int en = e[ax] * inward; /* +1: enters the domain here */
                const double fi = f[i * nv + xb];
                if (en == 0) {
                    s0 += fi;
                    nt[a1] += e[a1] * fi;
                    nt[a2] += e[a2] * fi;
                } else if (en < 0) {
                    sout += fi;
                }
            }
            const double jn = rho_b - (s0 + 2.0 * sout); /* rho_b u_n */
            for (int i = 0; i < Q; ++i) {
                const int e[3] = {EX[i], EY[i], EZ[i]};
                if (e[ax] * inward <= 0) continue;
                const int o_i = o->opp[i];
                f[i * nv + xb] = f[o_i * nv + xb] + 6.0 * WT[i] * jn - 0.5 * (e[a1] * nt[a1] + e[a2] * nt[a2]);
            }
        }
    }
}

void ora_set_bc(ora_t *o, int bc) { o->bc = bc; }

void ora_step(ora_t *o, long nsteps)
{
    for (long t = 0; t < nsteps; ++t) {
        compute_moments(o);
        compute_virtual_density(o);
        compute_forces(o);
        collide(o);
        stream(o);
        if (o->open_axis >= 0 && o->bc == 1) {
            zou_he_plane(o, 0, 0, o->rho_in1, +1);
            zou_he_plane(o, o->n[o->open_axis] - 1, 1, o->rho_out2, -1);
        } else if (o->open_axis >= 0) {
            neem_plane(o, 0, 0, o->rho_in1, +1);
            neem_plane(o, o->n[o->open_axis] - 1, 1, o->rho_out2, -1);
        }
        o->step++;
    }
}

/* Fields of the current state: rho^sigma, u = u^eq (Eq. 8, Section 2) and the
 * pressure of Eq. 12 summed over ordered pairs sigma != sigma-bar:
 * P = c_s^2 (rho1 + rho2) + c_s^2 G rho1 rho2.  Solid voxels read 0. */
void ora_fields(ora_t *o, double *rho1, double *rho2, double *ux, double *uy, double *uz, double *P)
{
    compute_moments(o);
    compute_virtual_density(o);
    compute_forces(o);
    for (long v = 0; v < o->nv; ++v) {
        if (o->solid[v]) {
            rho1[v] = rho2[v] = ux[v] = uy[v] = uz[v] = P[v] = 0.0;
            continue;
        }
        double tau_s, u[3];
        relaxation_and_velocity(o, v, &tau_s, u);
        double r1 = o->rho[0][v], r2 = o->rho[1][v];
        rho1[v] = r1;
        rho2[v] = r2;
        ux[v] = u[0];
        uy[v] = u[1];
        uz[v] = u[2];
        P[v] = CS2 * (r1 + r2) + 0.5 * CS2 * o->G * (r1 * r2 + r2 * r1);
    }
}

/* Saturation and mass (Section 4.1): out[0] = S_w, the fraction of sample
 * fluid nodes where component 2 (water) is the majority (rho2 > rho1);
 * out[1] = smooth non-wetting saturation, mean of rho1/(rho1+rho2) over the
 * sample; out[2], out[3] = total mass of components 1 and 2 over all fluid
 * nodes.  The sample is the slab lo <= coordinate < hi along the open axis
 * (the whole domain when there is no open axis or hi <= lo). */
void ora_saturation(ora_t *o, int lo, int hi, double *out)
{
    compute_moments(o);
    double nw = 0, cnt = 0, smooth = 0, m1 = 0, m2 = 0;
    for (long v = 0; v < o->nv; ++v) {
        if (o->solid[v]) continue;
        double r1 = o->rho[0][v], r2 = o->rho[1][v];
        m1 += r1;
        m2 += r2;
        int in = 1;
        if (o->open_axis >= 0 && hi > lo) {
            int c[3];
            coords(o, v, c);
            in = (c[o->open_axis] >= lo && c[o->open_axis] < hi);
        }
        if (!in) continue;
        cnt += 1;
        if (r2 > r1) nw += 1;
        smooth += r1 / (r1 + r2);
    }
    out[0] = cnt > 0 ? nw / cnt : 0.0;
    out[1] = cnt > 0 ? smooth / cnt : 0.0;
    out[2] = m1;
    out[3] = m2;
}


/* ===========================================================================
 * Discrete adjoint of ora_step.
 *
 * TEST INFRASTRUCTURE, derived by hand from the seven stages of ora_step (the
 * paper gives no adjoint).  ora_record takes n steps and keeps every state f_t
 * (t = 0..n).  ora_adjoint then runs the transposed Jacobian of each step
 * backwards from the adjoint of the final state, lambda_n = dJ/df_n, where J
 * is the smooth non-wetting saturation of ora_saturation (or <seed, f_n> when
 * a seed is given), and accumulates dJ/dxi (per voxel, Eq. 15 chi = 1 +/- xi)
 * and dJ/drho_in1 (the inlet density of the extrapolation).  Unlike the CUDA
 * adjoint it works in scatter form on the dense grid: every forward read of a
 * value becomes an add into that value's adjoint.
 *
 * Per step, in reverse order of the forward stages:
 *   7'. extrapolation: the prescribed component at a plane node xb was
 *       overwritten, so its adjoint moves to the interior node xI through
 *       f_eq(rho_b, u_I) + f(xI) - f_eq(rho(xI), u_I), u_I = sum_s m^s / sum_s
 *       rho^s at xI;
 *   6'. streaming: each pulled value adds its adjoint to its source (the
 *       neighbour's post-collision population, the own opposite one at a
 *       solid, or the frozen value beyond an open plane);
 *   5'. collision f* = f - (f - f_eq(rho, u)) / tau + (1 - 1/(2 tau)) S(u, F)
 *       with tau(rho1, rho2) of Eqs. 6-7 and u = sum_s (m^s + F^s/2) / sum_s
 *       rho^s (Eq. 8; tau cancels there);
 *   3'. force F^s = -G rho^s A^s + rho^s g, A^s = sum_i w_i e_i psi^sbar(nb_i)
 *       with the mirrored neighbour beyond an open plane;
 *   2'. virtual density rho~^s(w) = chi^s(w) N^s(w) / D(w) (Eq. 15);
 *   1'. moments: rho^s = sum_i f_i^s, m^s = sum_i e_i f_i^s.
 * ======================================================================== */

static double dfeq_du(int i, int a, double rho, const double u[3])
{
    const double e[3] = {(double)EX[i], (double)EY[i], (double)EZ[i]};
    const double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
    return WT[i] * rho * (e[a] / CS2 + eu * e[a] / (CS2 * CS2) - u[a] / CS2);
}

static double dsrc_du(int i, int b, const double u[3], const double F[3])
{
    const double e[3] = {(double)EX[i], (double)EY[i], (double)EZ[i]};
    const double eF = e[0] * F[0] + e[1] * F[1] + e[2] * F[2];
    (void)u;
    return WT[i] * (-F[b] / CS2 + e[b] * eF / (CS2 * CS2));
}

static double dsrc_dF(int i, int a, const double u[3])
{
    const double e[3] = {(double)EX[i], (double)EY[i], (double)EZ[i]};
    const double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
    return WT[i] * ((e[a] - u[a]) / CS2 + eu * e[a] / (CS2 * CS2));
}

int ora_record(ora_t *o, long nsteps)
{
    const size_t one = (size_t)2 * Q * o->nv;
    free(o->tape);
    o->tape = (double *)malloc(sizeof(double) * one * (size_t)(nsteps + 1));
    if (!o->tape) {
        o->tape_len = 0;
        return -1;
    }
    o->tape_len = nsteps + 1;
    for (long t = 0; t <= nsteps; ++t) {
        if (t > 0) ora_step(o, 1);
        memcpy(o->tape + one * (size_t)t, o->f[0], sizeof(double) * Q * o->nv);
        memcpy(o->tape + one * (size_t)t + (size_t)Q * o->nv, o->f[1], sizeof(double) * Q * o->nv);
    }
    return 0;
}

/* Load recorded state t into o->f and recompute the forward intermediates
 * (moments, virtual densities, forces) of the step that starts from it. */
static void load_state(ora_t *o, long t)
{
    const size_t one = (size_t)2 * Q * o->nv;
    memcpy(o->f[0], o->tape + one * (size_t)t, sizeof(double) * Q * o->nv);
    memcpy(o->f[1], o->tape + one * (size_t)t + (size_t)Q * o->nv, sizeof(double) * Q * o->nv);
    compute_moments(o);
    compute_virtual_density(o);
    compute_forces(o);
}

/* 7': adjoint of neem_plane for one plane.  lam is [2][Q*nv]; fn is the
 * post-stream state (the interior node is never overwritten, so the recorded
 * next state holds the values the extrapolation read). */
static void neem_adjoint(const ora_t *o, double *lam[2], const double *fn[2], int plane, int comp, double rho_b,
                         int inward, double *g_rho_b)
{
    const int ax = o->open_axis;
    const long nv = o->nv;
    const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    for (int p2 = 0; p2 < o->n[a2]; ++p2) {
        for (int p1 = 0; p1 < o->n[a1]; ++p1) {
            int c[3];
            c[ax] = plane;
            c[a1] = p1;
            c[a2] = p2;
            const long xb = vid(o, c);
            if (o->solid[xb]) continue;
            c[ax] = plane + inward;
            const long xi = vid(o, c);
            double r[2] = {0, 0}, m[3] = {0, 0, 0};
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < Q; ++i) {
                    const double fi = fn[s][i * nv + xi];
                    r[s] += fi;
                    m[0] += EX[i] * fi;
                    m[1] += EY[i] * fi;
                    m[2] += EZ[i] * fi;
                }
            const double R = r[0] + r[1];
            const double u[3] = {m[0] / R, m[1] / R, m[2] / R};
            double rbar = 0, ubar[3] = {0, 0, 0}, gb = 0;
            for (int i = 0; i < Q; ++i) {
                const double mu = lam[comp][i * nv + xb];
                lam[comp][i * nv + xb] = 0.0;  /* overwritten: no dependence on the old value */
                lam[comp][i * nv + xi] += mu;  /* the f(xI) term */
                const double feq1 = feq_i(i, 1.0, u);
                gb += mu * feq1;       /* d f_eq(rho_b, u) / d rho_b */
                rbar -= mu * feq1;     /* - d f_eq(rho(xI), u) / d rho(xI) */
                for (int a = 0; a < 3; ++a) ubar[a] += mu * (dfeq_du(i, a, rho_b, u) - dfeq_du(i, a, r[comp], u));
            }
            for (int j = 0; j < Q; ++j) {
                lam[comp][j * nv + xi] += rbar;
                const double e[3] = {(double)EX[j], (double)EY[j], (double)EZ[j]};
                double du = 0;
                for (int a = 0; a < 3; ++a) du += ubar[a] * (e[a] - u[a]) / R;
                lam[0][j * nv + xi] += du;
                lam[1][j * nv + xi] += du;
            }
            if (g_rho_b) *g_rho_b += gb;
        }
    }
}

int ora_adjoint(ora_t *o, int lo, int hi, const double *seed, double *grad_xi, double *grad_rho_in1,
                double *grad_f, double *grad_frozen)
{
    if (!o->tape || o->tape_len < 1) return -1;
    if (o->open_axis >= 0 && o->bc != 0) return -2; /* the reverse pass covers the extrapolation only */
    const long nv = o->nv, n = o->tape_len - 1;
    const size_t one = (size_t)Q * nv;
    double *lam[2], *lamS[2], *gfz[2], *psib[2], *rhob[2];
    for (int s = 0; s < 2; ++s) {
        lam[s] = (double *)calloc(one, sizeof(double));
        lamS[s] = (double *)calloc(one, sizeof(double));
        gfz[s] = (double *)calloc(one, sizeof(double));
        psib[s] = (double *)calloc((size_t)nv, sizeof(double));
        rhob[s] = (double *)calloc((size_t)nv, sizeof(double));
    }
    double *gxi = (double *)calloc((size_t)nv, sizeof(double));
    double grin = 0.0;

    /* adjoint of the final state */
    if (seed) {
        memcpy(lam[0], seed, sizeof(double) * one);
        memcpy(lam[1], seed + one, sizeof(double) * one);
    } else {
        const double *fT[2] = {o->tape + 2 * one * (size_t)n, o->tape + 2 * one * (size_t)n + one};
        double cnt = 0;
        for (long v = 0; v < nv; ++v) {
            if (o->solid[v]) continue;
            int in = 1;
            if (o->open_axis >= 0 && hi > lo) {
                int c[3];
                coords(o, v, c);
                in = (c[o->open_axis] >= lo && c[o->open_axis] < hi);
            }
            cnt += in;
        }
        for (long v = 0; v < nv; ++v) {
            if (o->solid[v] || cnt == 0) continue;
            if (o->open_axis >= 0 && hi > lo) {
                int c[3];
                coords(o, v, c);
                if (c[o->open_axis] < lo || c[o->open_axis] >= hi) continue;
            }
            double r[2] = {0, 0};
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < Q; ++i) r[s] += fT[s][i * nv + v];
            const double R = r[0] + r[1];
            /* d/d rho1 of rho1/(rho1+rho2) = rho2/R^2, d/d rho2 = -rho1/R^2 */
            for (int i = 0; i < Q; ++i) {
                lam[0][i * nv + v] = r[1] / (R * R) / cnt;
                lam[1][i * nv + v] = -r[0] / (R * R) / cnt;
            }
        }
    }

    const double nu[2] = {CS2 * (o->tau[0] - 0.5), CS2 * (o->tau[1] - 0.5)};
    for (long t = n - 1; t >= 0; --t) {
        load_state(o, t);
        const double *fn[2] = {o->tape + 2 * one * (size_t)(t + 1), o->tape + 2 * one * (size_t)(t + 1) + one};
        /* 7' (outlet was extrapolated last, so it is undone first) */
        if (o->open_axis >= 0) {
            neem_adjoint(o, lam, fn, o->n[o->open_axis] - 1, 1, o->rho_out2, -1, NULL);
            neem_adjoint(o, lam, fn, 0, 0, o->rho_in1, +1, &grin);
        }
        /* 6' streaming, scatter form */
        for (int s = 0; s < 2; ++s) memset(lamS[s], 0, sizeof(double) * one);
        for (long v = 0; v < nv; ++v) {
            if (o->solid[v]) continue;
            int c[3];
            coords(o, v, c);
            for (int s = 0; s < 2; ++s) {
                lamS[s][v] += lam[s][v];
                for (int i = 1; i < Q; ++i) {
                    long src;
                    const double l = lam[s][i * nv + v];
                    if (neighbour(o, c, -EX[i], -EY[i], -EZ[i], &src))
                        gfz[s][i * nv + v] += l;
                    else if (o->solid[src])
                        lamS[s][o->opp[i] * nv + v] += l;
                    else
                        lamS[s][i * nv + src] += l;
                }
            }
        }
        /* 5', 3' local part, 1' (written into lam, the adjoint of state t) */
        for (int s = 0; s < 2; ++s) {
            memset(psib[s], 0, sizeof(double) * (size_t)nv);
            memset(rhob[s], 0, sizeof(double) * (size_t)nv);
        }
        for (long v = 0; v < nv; ++v) {
            if (o->solid[v]) {
                for (int s = 0; s < 2; ++s)
                    for (int i = 0; i < Q; ++i) lam[s][i * nv + v] = 0.0;
                continue;
            }
            int c[3];
            coords(o, v, c);
            const double r[2] = {o->rho[0][v], o->rho[1][v]};
            const double R = r[0] + r[1];
            double tau_s, u[3];
            relaxation_and_velocity(o, v, &tau_s, u);
            const double cf = 1.0 - 1.0 / (2.0 * tau_s);
            double rb[2] = {0, 0}, ub[3] = {0, 0, 0}, Fb[2][3] = {{0, 0, 0}, {0, 0, 0}}, mb[2][3], taub = 0;
            for (int s = 0; s < 2; ++s) {
                const double *F = &o->F[s][3 * v];
                for (int i = 0; i < Q; ++i) {
                    const double L = lamS[s][i * nv + v];
                    const double fi = o->f[s][i * nv + v];
                    const double fe = feq_i(i, r[s], u);
                    const double S = src_i(i, u, F);
                    rb[s] += L * feq_i(i, 1.0, u) / tau_s;
                    for (int a = 0; a < 3; ++a) {
                        ub[a] += L * (dfeq_du(i, a, r[s], u) / tau_s + cf * dsrc_du(i, a, u, F));
                        Fb[s][a] += L * cf * dsrc_dF(i, a, u);
                    }
                    taub += L * ((fi - fe) / (tau_s * tau_s) + S / (2.0 * tau_s * tau_s));
                }
            }
            /* tau(rho1, rho2), Eqs. 6-7 */
            rb[0] += taub * r[1] * (nu[0] - nu[1]) / (R * R * CS2);
            rb[1] += taub * r[0] * (nu[1] - nu[0]) / (R * R * CS2);
            /* u = sum_s (m^s + shift F^s / 2) / R */
            for (int s = 0; s < 2; ++s) {
                for (int a = 0; a < 3; ++a) {
                    mb[s][a] = ub[a] / R;
                    if (o->velocity_shift) Fb[s][a] += 0.5 * ub[a] / R;
                    rb[s] -= ub[a] * u[a] / R;
                }
            }
            /* F^s = -G rho^s A^s + rho^s g */
            for (int s = 0; s < 2; ++s) {
                const int sb = 1 - s;
                double A[3] = {0, 0, 0};
                long nbs[Q];
                for (int i = 1; i < Q; ++i) {
                    long nb;
                    nbs[i] = -1;
                    if (neighbour(o, c, EX[i], EY[i], EZ[i], &nb)) {
                        const int j = o->mirror[i];
                        if (neighbour(o, c, EX[j], EY[j], EZ[j], &nb)) continue; /* cannot happen */
                    }
                    nbs[i] = nb;
                    A[0] += WT[i] * o->rho[sb][nb] * EX[i];
                    A[1] += WT[i] * o->rho[sb][nb] * EY[i];
                    A[2] += WT[i] * o->rho[sb][nb] * EZ[i];
                }
                double Ab[3];
                for (int a = 0; a < 3; ++a) {
                    rb[s] += Fb[s][a] * (-o->G * A[a] + o->g[a]);
                    Ab[a] = -o->G * r[s] * Fb[s][a];
                }
                for (int i = 1; i < Q; ++i)
                    if (nbs[i] >= 0) psib[sb][nbs[i]] += WT[i] * (EX[i] * Ab[0] + EY[i] * Ab[1] + EZ[i] * Ab[2]);
            }
            /* pre-collision populations: direct term and moments */
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < Q; ++i)
                    lam[s][i * nv + v] = (1.0 - 1.0 / tau_s) * lamS[s][i * nv + v] + rb[s] +
                                         EX[i] * mb[s][0] + EY[i] * mb[s][1] + EZ[i] * mb[s][2];
        }
        /* 2': psi adjoint of a solid is that of its virtual density */
        for (long v = 0; v < nv; ++v) {
            if (!o->solid[v]) {
                for (int s = 0; s < 2; ++s) rhob[s][v] += psib[s][v];
                continue;
            }
            if (psib[0][v] == 0.0 && psib[1][v] == 0.0) continue;
            int c[3];
            coords(o, v, c);
            double num[2] = {0, 0}, den = 0;
            for (int i = 1; i < Q; ++i) {
                long nb;
                if (neighbour(o, c, EX[i], EY[i], EZ[i], &nb) || o->solid[nb]) continue;
                num[0] += WT[i] * o->rho[0][nb];
                num[1] += WT[i] * o->rho[1][nb];
                den += WT[i];
            }
            if (den <= 0) continue;
            const double chi[2] = {1.0 + o->xi[v], 1.0 - o->xi[v]};
            gxi[v] += psib[0][v] * num[0] / den - psib[1][v] * num[1] / den;
            for (int i = 1; i < Q; ++i) {
                long nb;
                if (neighbour(o, c, EX[i], EY[i], EZ[i], &nb) || o->solid[nb]) continue;
                for (int s = 0; s < 2; ++s) rhob[s][nb] += psib[s][v] * chi[s] * WT[i] / den;
            }
        }
        /* 1' for the non-local density adjoints */
        for (long v = 0; v < nv; ++v) {
            if (o->solid[v]) continue;
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < Q; ++i) lam[s][i * nv + v] += rhob[s][v];
        }
    }
    /* leave the oracle at the final recorded state */
    load_state(o, n);

    if (grad_xi) memcpy(grad_xi, gxi, sizeof(double) * (size_t)nv);
    if (grad_rho_in1) *grad_rho_in1 = grin;
    if (grad_f) {
        memcpy(grad_f, lam[0], sizeof(double) * one);
        memcpy(grad_f + one, lam[1], sizeof(double) * one);
    }
    if (grad_frozen) {
        memcpy(grad_frozen, gfz[0], sizeof(double) * one);
        memcpy(grad_frozen + one, gfz[1], sizeof(double) * one);
    }
    for (int s = 0; s < 2; ++s) {
        free(lam[s]);
        free(lamS[s]);
        free(gfz[s]);
        free(psib[s]);
        free(rhob[s]);
    }
    free(gxi);
    return 0;
}
