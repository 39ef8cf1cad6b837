/*
 * lbm_ref.c -- plain, slow FP64 CPU oracle for one time step of the BGK
 * lattice Boltzmann method on a dense masked lattice (D2Q9 and D3Q19).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file; the CUDA library never does,
 * and the two share no code, tables or headers.
 *
 * What it computes is the plain definition that the tiled method of
 * Tomczak & Szafran (arXiv:1703.08015) reorganises.  Tiles only decide where
 * the PDFs are stored; Sec. 3 lets them be updated in any order as long as
 * values crossing tile edges still propagate, so the result is that of the
 * untiled lattice.  The oracle therefore keeps every PDF on the dense grid,
 * f[i][z][y][x], and never forms a tile.
 *
 *   streaming + collision  : Eq. 7 (time-discrete BGK), pull form: the value
 *                            arriving at node r along c_i is the post-
 *                            collision value of node r - c_i (Fig. 5 gathers).
 *   collision operator     : Eq. 2, Omega = -(f - f^eq)/tau.
 *   equilibrium            : Eq. 3 (quasi-compressible), c_s^2 = 1/3 (Sec. 2.1),
 *                            or Eq. 4 (incompressible) when `model` = 1.
 *   macroscopic velocity   : Eq. 5 (u = j/rho) or Eq. 6 (u = j), each with the
 *                            half-step force correction j + F/2 (Guo forcing;
 *                            the paper has no body force).
 *   solid neighbours       : Sec. 3.2 propagates only between non-solid nodes;
 *                            the value that cannot be gathered is the node's own
 *                            post-collision value in the opposite direction
 *                            (halfway bounce-back).
 *   domain edges           : per axis either periodic or a solid wall lying
 *                            outside the last node row (the paper pads the
 *                            geometry with solid nodes, Sec. 3).
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC
 * (-ffp-contract=off keeps the arithmetic identical on x86-64 and AArch64).
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- lattice tables ------------------------------------------------------
 * The paper names D2Q9 (Fig. 1, whose drawing is lost) and D3Q19 (Sec. 2.2)
 * but prints neither the link order nor the weights w_i (Eq. 3 only names
 * them).  These are the standard sets; the tests pin them through their
 * isotropy moments. */
/* D2Q9: rest, the 4 axis links, then the 4 diagonals.  Weights 4/9, 1/9, 1/36. */
static const int C9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* D3Q19: rest, +-x, +-y, +-z, then the 12 edge diagonals in +- pairs.
 * Weights 1/3, 1/18, 1/36. */
static const int C19[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const int OPP19[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9,
                              12, 11, 14, 13, 16, 15, 18, 17};

typedef struct {
    int q, d;
    const int (*c)[3];
    const int* opp;
    double w[19];
} lattice_t;

static int get_lattice(int lattice, lattice_t* L) {
    if (lattice == 9) {
        L->q = 9; L->d = 2; L->c = C9; L->opp = OPP9;
        L->w[0] = 4.0 / 9.0;
        for (int i = 1; i <= 4; i++) L->w[i] = 1.0 / 9.0;
        for (int i = 5; i <= 8; i++) L->w[i] = 1.0 / 36.0;
        return 0;
    }
    if (lattice == 19) {
        L->q = 19; L->d = 3; L->c = C19; L->opp = OPP19;
        L->w[0] = 1.0 / 3.0;
        for (int i = 1; i <= 6; i++) L->w[i] = 1.0 / 18.0;
        for (int i = 7; i <= 18; i++) L->w[i] = 1.0 / 36.0;
        return 0;
    }
    return -1;
}

/* Export the tables so the tests can check the lattice itself. */
int ref_lattice(int lattice, int* q, int* d, int* c, double* w, int* opp) {
    lattice_t L;
    if (get_lattice(lattice, &L)) return -1;
    *q = L.q; *d = L.d;
    for (int i = 0; i < L.q; i++) {
        for (int a = 0; a < 3; a++) c[3 * i + a] = L.c[i][a];
        w[i] = L.w[i];
        opp[i] = L.opp[i];
    }
    return 0;
}

/* Eq. 3 (model 0) or Eq. 4 (model 1), with c_s^2 = 1/3:
 *   1/c_s^2 = 3, 1/(2 c_s^4) = 4.5, 1/(2 c_s^2) = 1.5. */
static void equilibrium(const lattice_t* L, int model, double rho,
                        const double u[3], double* feq) {
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L->q; i++) {
        double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        double poly = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq;
        if (model == 0)
            feq[i] = L->w[i] * rho * (1.0 + poly);
        else
            feq[i] = L->w[i] * (rho + poly);
    }
}

int ref_equilibrium(int lattice, int model, double rho, const double* u,
                    double* feq) {
    lattice_t L;
    if (get_lattice(lattice, &L)) return -1;
    double uu[3] = {u[0], u[1], u[2]};
    equilibrium(&L, model, rho, uu, feq);
    return 0;
}

/* Density and velocity of a set of q gathered values: rho = sum f (Sec. 2.1),
 * j = sum c_i f_i, then Eq. 5 (model 0) or Eq. 6 (model 1) applied to
 * j + F/2 (Guo's half-step force correction; the paper has no force). */
static void macro(const lattice_t* L, int model, const double* f,
                  const double F[3], double* rho_out, double u[3]) {
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->q; i++) {
        rho += f[i];
        for (int a = 0; a < 3; a++) j[a] += L->c[i][a] * f[i];
    }
    for (int a = 0; a < 3; a++) {
        double ja = j[a] + 0.5 * F[a];
        u[a] = (model == 0) ? ja / rho : ja;
    }
    *rho_out = rho;
}

/* BGK collision (Eq. 2 inside Eq. 7) plus the Guo forcing term
 *   S_i = (1 - 1/(2 tau)) w_i [ 3 (c_i - u).F + 9 (c_i.u)(c_i.F) ]. */
static void collide(const lattice_t* L, int model, double tau,
                    const double F[3], const double* f, double* fout) {
    double rho, u[3], feq[19];
    macro(L, model, f, F, &rho, u);
    equilibrium(L, model, rho, u, feq);
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    for (int i = 0; i < L->q; i++) {
        double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
        double cF = L->c[i][0] * F[0] + L->c[i][1] * F[1] + L->c[i][2] * F[2];
        double S = (1.0 - 1.0 / (2.0 * tau)) * L->w[i] *
                   (3.0 * (cF - uF) + 9.0 * cu * cF);
        fout[i] = f[i] - (f[i] - feq[i]) / tau + S;
    }
}

int ref_collide(int lattice, int model, double tau, const double* F,
                const double* f, double* fout) {
    lattice_t L;
    if (get_lattice(lattice, &L)) return -1;
    double FF[3] = {F[0], F[1], F[2]};
    collide(&L, model, tau, FF, f, fout);
    return 0;
}

/* ---- the dense masked lattice ------------------------------------------- */
typedef struct {
    lattice_t L;
    int n[3];        /* nx, ny, nz */
    int periodic[3];
    const uint8_t* mask; /* 1 = fluid, 0 = solid; x fastest */
    size_t N;
} grid_t;

static int make_grid(grid_t* g, int lattice, int nx, int ny, int nz,
                     const int* periodic, const uint8_t* mask) {
    if (get_lattice(lattice, &g->L)) return -1;
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    if (g->L.d == 2 && nz != 1) return -1;
    g->n[0] = nx; g->n[1] = ny; g->n[2] = nz;
    for (int a = 0; a < 3; a++) g->periodic[a] = periodic ? periodic[a] : 0;
    g->mask = mask;
    g->N = (size_t)nx * ny * nz;
    return 0;
}

/* The source node s = r - c_i of a pull along direction i.  Returns -1 when
 * no value can be gathered from it: s lies beyond a non-periodic edge or is
 * solid. */
static long long source_node(const grid_t* g, int x, int y, int z, int i) {
    int r[3] = {x, y, z};
    int s[3];
    for (int a = 0; a < 3; a++) {
        s[a] = r[a] - g->L.c[i][a];
        if (s[a] < 0 || s[a] >= g->n[a]) {
            if (!g->periodic[a]) return -1;
            s[a] = (s[a] + g->n[a]) % g->n[a];
        }
    }
    long long idx = (long long)s[0] + (long long)g->n[0] *
                    ((long long)s[1] + (long long)g->n[1] * s[2]);
    if (!g->mask[idx]) return -1;
    return idx;
}

/* Pull the q values that arrive at fluid node (x,y,z) from the post-
 * collision field fs (layout fs[i*N + node]). */
static void gather(const grid_t* g, const double* fs, int x, int y, int z,
                   double* f) {
    size_t self = (size_t)x + (size_t)g->n[0] * ((size_t)y + (size_t)g->n[1] * z);
    for (int i = 0; i < g->L.q; i++) {
        long long s = source_node(g, x, y, z, i);
        if (s >= 0)
            f[i] = fs[(size_t)i * g->N + (size_t)s];
        else /* halfway bounce-back: own value in the opposite direction */
            f[i] = fs[(size_t)g->L.opp[i] * g->N + self];
    }
}

static int threads_of(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* Equilibrium start: f*_i = f^eq_i(rho, u) at every fluid node (rho0 and
 * u = 0 when no fields are given); solid nodes hold 0. */
int ref_init(int lattice, int model, int nx, int ny, int nz,
             const uint8_t* mask, double rho0, const double* rho,
             const double* u, double* f) {
    grid_t g;
    if (make_grid(&g, lattice, nx, ny, nz, NULL, mask)) return -1;
    for (size_t n = 0; n < g.N; n++) {
        double feq[19];
        if (mask[n]) {
            double r = rho ? rho[n] : rho0;
            double uu[3] = {0.0, 0.0, 0.0};
            if (u) for (int a = 0; a < 3; a++) uu[a] = u[(size_t)a * g.N + n];
            equilibrium(&g.L, model, r, uu, feq);
        } else {
            for (int i = 0; i < g.L.q; i++) feq[i] = 0.0;
        }
        for (int i = 0; i < g.L.q; i++) f[(size_t)i * g.N + n] = feq[i];
    }
    return 0;
}

/* One time step (Eq. 7): gather, collide, store.  Every fluid node of fdst
 * is written; solid nodes of fdst are set to 0. */
int ref_step(int lattice, int model, int nx, int ny, int nz,
             const int* periodic, const uint8_t* mask, double tau,
             const double* force, const double* fsrc, double* fdst,
             int nthreads) {
    grid_t g;
    if (make_grid(&g, lattice, nx, ny, nz, periodic, mask)) return -1;
    double F[3] = {force[0], force[1], force[2]};
    long long rows = (long long)ny * nz;
#pragma omp parallel for schedule(static) num_threads(threads_of(nthreads))
    for (long long row = 0; row < rows; row++) {
        int y = (int)(row % ny), z = (int)(row / ny);
        for (int x = 0; x < nx; x++) {
            size_t n = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z);
            double f[19], fout[19];
            if (!mask[n]) {
                for (int i = 0; i < g.L.q; i++) fdst[(size_t)i * g.N + n] = 0.0;
                continue;
            }
            gather(&g, fsrc, x, y, z, f);
            collide(&g.L, model, tau, F, f, fout);
            for (int i = 0; i < g.L.q; i++) fdst[(size_t)i * g.N + n] = fout[i];
        }
    }
    return 0;
}

/* One time step evaluated only at the listed nodes (flat indices, which must
 * be fluid): out[k*q + i] = f*_i after the step at nodes[k].  This is the
 * same arithmetic as ref_step, for checking sampled outputs of a large run. */
int ref_step_nodes(int lattice, int model, int nx, int ny, int nz,
                   const int* periodic, const uint8_t* mask, double tau,
                   const double* force, const double* fsrc,
                   const int64_t* nodes, int64_t count, double* out) {
    grid_t g;
    if (make_grid(&g, lattice, nx, ny, nz, periodic, mask)) return -1;
    double F[3] = {force[0], force[1], force[2]};
    for (int64_t k = 0; k < count; k++) {
        int64_t n = nodes[k];
        if (n < 0 || (size_t)n >= g.N || !mask[n]) return -2;
        int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((int64_t)nx * ny));
        double f[19];
        gather(&g, fsrc, x, y, z, f);
        collide(&g.L, model, tau, F, f, out + (size_t)k * g.L.q);
    }
    return 0;
}

/* Density and velocity that the next step's collision will use (the pulled,
 * pre-collision values; velocity includes the F/2 correction).  Solid nodes
 * get NaN. */
int ref_moments(int lattice, int model, int nx, int ny, int nz,
                const int* periodic, const uint8_t* mask, const double* force,
                const double* fs, double* rho, double* u, int nthreads) {
    grid_t g;
    if (make_grid(&g, lattice, nx, ny, nz, periodic, mask)) return -1;
    double F[3] = {force[0], force[1], force[2]};
    long long rows = (long long)ny * nz;
#pragma omp parallel for schedule(static) num_threads(threads_of(nthreads))
    for (long long row = 0; row < rows; row++) {
        int y = (int)(row % ny), z = (int)(row / ny);
        for (int x = 0; x < nx; x++) {
            size_t n = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * z);
            if (!mask[n]) {
                rho[n] = NAN;
                for (int a = 0; a < 3; a++) u[(size_t)a * g.N + n] = NAN;
                continue;
            }
            double f[19], r, uu[3];
            gather(&g, fs, x, y, z, f);
            macro(&g.L, model, f, F, &r, uu);
            rho[n] = r;
            for (int a = 0; a < 3; a++) u[(size_t)a * g.N + n] = uu[a];
        }
    }
    return 0;
}

/* Sum of every post-collision PDF over the fluid nodes: the total mass,
 * which streaming permutes and collision conserves.  Summed with Neumaier's
 * compensated summation so the result is the exact sum to within a few
 * roundings (a plain running sum of ~10^5 small terms into a large
 * accumulator would drift by ~1e-12 relative on its own). */
double ref_total_mass(int lattice, int nx, int ny, int nz, const uint8_t* mask,
                      const double* fs) {
    lattice_t L;
    if (get_lattice(lattice, &L)) return NAN;
    size_t N = (size_t)nx * ny * nz;
    double sum = 0.0, comp = 0.0;
    for (size_t n = 0; n < N; n++) {
        if (!mask[n]) continue;
        for (int i = 0; i < L.q; i++) {
            double v = fs[(size_t)i * N + n];
            double t = sum + v;
            if (fabs(sum) >= fabs(v))
                comp += (sum - t) + v;
            else
                comp += (v - t) + sum;
            sum = t;
        }
    }
    return sum + comp;
}

/* Number of threads ref_step would use for `nthreads` (0 = all). */
int ref_threads(int nthreads) { return threads_of(nthreads); }
