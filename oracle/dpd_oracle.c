/*
 * FP64 CPU oracle for the DPD fluid step.  TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check (__graft_entry__.smoke) and the CPU-baseline
 * leg of bench.py may load this library.  The product path never calls it and
 * shares no code with it: this file includes nothing from the CUDA sources and
 * the CUDA sources include nothing from here.
 *
 * What it restates, plainly and in double precision:
 *   - the stateless pair noise xi_ij of Sec. 2.1 (symmetric in i,j, zero mean,
 *     unit variance), drawn from the Philox-4x32-R counter-based generator of
 *     Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
 *     1, 2, 3" (SC'11), with counter (min id, max id, step lo, step hi) and
 *     key (seed lo, seed hi); xi = sqrt(3) (2U - 1), U = ((u >> 8) + 1/2) 2^-24,
 *     or, as the paper states it, Gaussian: Box-Muller on words 0 and 1;
 *   - the pair force of Sec. 2.1: Eq. 3 (conservative), Eq. 4 (weight w),
 *     Eq. 5 (dissipative and random), the fluctuation-dissipation relation
 *     sigma^2 = 2 gamma kT, w_D = w_R^2, and the generalised weight
 *     w_R = w^k; the random term is divided by sqrt(dt) (time-discretised
 *     white noise);
 *   - Eq. 2 as written: F_i = sum over j != i of F_ij, an O(N^2) double loop;
 *   - the cell list of Sec. 3.2: cell sizes by counting, cell starts by an
 *     exclusive scan, then the reorder, followed by a 27-cell neighbour sum;
 *   - Newton's equations (Eq. 1) advanced by velocity-Verlet with the
 *     velocity predicted at the half step (the fused leapfrog of Sec. 3.1,
 *     item 5) in a periodic box;
 *   - the periodic Poiseuille body force of Sec. 4.2 (or a constant one);
 *   - several particle species in one box (the particle vectors of Sec. 3.1,
 *     each pair of species with its own interaction and cut-off): a_st,
 *     gamma_st and rc_st <= rc from symmetric per-pair tables, the cell list
 *     built for the largest cut-off rc;
 *   - box statistics: momentum, kinetic energy, kT, virial pressure and a
 *     binned velocity profile.
 *
 * Parity of the generator with published Philox known-answer vectors is
 * not pinned (no such vectors are available); it is pinned to an independent
 * library implementation of the same published algorithm in the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double L[3];     /* box edges */
    double a;        /* conservative coefficient (alpha in Eq. 3) */
    double gamma;    /* dissipative coefficient (Eq. 5) */
    double kT;       /* k_B T */
    double rc;       /* cut-off radius */
    double dt;       /* time step */
    double mass;     /* particle mass m (Eq. 1) */
    double kexp;     /* weight exponent k, w_R = w^k */
    double fb;       /* body-force magnitude */
    int fb_mode;     /* 0: none, 1: constant along fb_flow, 2: periodic Poiseuille */
    int fb_flow;     /* axis the body force points along */
    int fb_grad;     /* axis along which the Poiseuille force switches sign */
    int rounds;      /* Philox rounds R */
    uint64_t seed;
    int noise;       /* 0: uniform xi = sqrt(3)(2U - 1); 1: Gaussian xi (Box-Muller) */
    int nspec;       /* species in the box: 1 uses a, gamma, rc above; 2..4 the tables */
    const int32_t *species;  /* species of the particle with id k is species[k]; NULL: 0 */
    double sa[16];   /* a_st at [4 s + t] (symmetric) */
    double sg[16];   /* gamma_st */
    double src[16];  /* rc_st, at most rc */
} orc_params;

/* ----------------------------------------------------------------------
 * Philox-4x32-R.  Round multipliers and Weyl key increments are the ones
 * published with the generator.
 * -------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], int rounds, uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < rounds; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The 32-bit word behind xi_ij at a given step: word 0 of Philox applied to
 * the counter (min id, max id, step lo, step hi) under key (seed lo, seed hi).
 * Ordering the ids makes xi_ij = xi_ji (Sec. 2.1). */
uint32_t orc_pair_word(uint32_t id_i, uint32_t id_j, uint64_t step, uint64_t seed, int rounds)
{
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = id_i < id_j ? id_i : id_j;
    ctr[1] = id_i < id_j ? id_j : id_i;
    ctr[2] = (uint32_t)(step & 0xffffffffu);
    ctr[3] = (uint32_t)(step >> 32);
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32(ctr, key, rounds, out);
    return out[0];
}

/* Uniform U in (0,1) from the top 24 bits, then xi = sqrt(3)(2U - 1):
 * zero mean, unit variance. */
double orc_xi_from_word(uint32_t u)
{
    double U = ((double)(u >> 8) + 0.5) * (1.0 / 16777216.0);
    return sqrt(3.0) * (2.0 * U - 1.0);
}

/* Words 0 and 1 of the pair's Philox block (same counter and key). */
void orc_pair_words(uint32_t id_i, uint32_t id_j, uint64_t step, uint64_t seed, int rounds,
                    uint32_t out[2])
{
    uint32_t ctr[4], key[2], w[4];
    ctr[0] = id_i < id_j ? id_i : id_j;
    ctr[1] = id_i < id_j ? id_j : id_i;
    ctr[2] = (uint32_t)(step & 0xffffffffu);
    ctr[3] = (uint32_t)(step >> 32);
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32(ctr, key, rounds, w);
    out[0] = w[0];
    out[1] = w[1];
}

/* The paper's Gaussian xi (Sec. 2.1) by the Box-Muller transform of two
 * uniforms U_k = ((u_k >> 8) + 1/2) 2^-24: sqrt(-2 ln U1) cos(2 pi U2). */
double orc_xi_gauss(uint32_t u0, uint32_t u1)
{
    const double pi = 3.14159265358979323846;
    double U1 = ((double)(u0 >> 8) + 0.5) * (1.0 / 16777216.0);
    double U2 = ((double)(u1 >> 8) + 0.5) * (1.0 / 16777216.0);
    return sqrt(-2.0 * log(U1)) * cos(2.0 * pi * U2);
}

void orc_rng_gauss(int64_t n, const uint32_t *ida, const uint32_t *idb, uint64_t step,
                   uint64_t seed, int rounds, uint32_t *w0, uint32_t *w1, double *xi)
{
    for (int64_t k = 0; k < n; ++k) {
        uint32_t u[2];
        orc_pair_words(ida[k], idb[k], step, seed, rounds, u);
        if (w0) w0[k] = u[0];
        if (w1) w1[k] = u[1];
        if (xi) xi[k] = orc_xi_gauss(u[0], u[1]);
    }
}

void orc_rng(int64_t n, const uint32_t *ida, const uint32_t *idb, uint64_t step, uint64_t seed,
             int rounds, uint32_t *words, double *xi)
{
    for (int64_t k = 0; k < n; ++k) {
        uint32_t u = orc_pair_word(ida[k], idb[k], step, seed, rounds);
        if (words) words[k] = u;
        if (xi) xi[k] = orc_xi_from_word(u);
    }
}

/* ----------------------------------------------------------------------
 * Geometry helpers
 * -------------------------------------------------------------------- */
static double min_image(double d, double L)
{
    return d - L * nearbyint(d / L);
}

static double wrap_coord(double x, double L)
{
    double y = fmod(x, L);
    if (y < 0.0) y += L;
    if (y >= L) y -= L;
    return y;
}

/* ----------------------------------------------------------------------
 * Pair force F_ij = F^C + F^D + F^R (Sec. 2.1, Eqs. 3-5).
 * r_ij = r_i - r_j (minimum image), e_ij = r_ij / r_ij.
 * Writes F_ij into fij and r_ij . F^C_ij into *rfc.
 * -------------------------------------------------------------------- */
void orc_pair_force(const orc_params *p, const double *xi, const double *xj,
                    const double *vi, const double *vj, uint32_t idi, uint32_t idj,
                    uint64_t step, double *fij, double *rfc)
{
    fij[0] = fij[1] = fij[2] = 0.0;
    if (rfc) *rfc = 0.0;
    /* interaction of the pair's species (one species: the scalar parameters) */
    double a = p->a, gamma = p->gamma, rc = p->rc;
    if (p->nspec > 1) {
        int si = p->species ? p->species[idi] : 0;
        int sj = p->species ? p->species[idj] : 0;
        a = p->sa[4 * si + sj];
        gamma = p->sg[4 * si + sj];
        rc = p->src[4 * si + sj];
    }
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = min_image(xi[k] - xj[k], p->L[k]);
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(r < rc) || r == 0.0) return;
    double e[3] = {d[0] / r, d[1] / r, d[2] / r};
    double w = 1.0 - r / rc;                          /* Eq. 4 */
    double wR = (p->kexp == 1.0) ? w : pow(w, p->kexp);
    double wD = wR * wR;                              /* w_D = w_R^2 */
    double sigma = sqrt(2.0 * gamma * p->kT);         /* sigma^2 = 2 gamma kT */
    double ev = e[0] * (vi[0] - vj[0]) + e[1] * (vi[1] - vj[1]) + e[2] * (vi[2] - vj[2]);
    double xi_ij;
    if (p->noise == 1) {
        uint32_t u[2];
        orc_pair_words(idi, idj, step, p->seed, p->rounds, u);
        xi_ij = orc_xi_gauss(u[0], u[1]);
    } else {
        xi_ij = orc_xi_from_word(orc_pair_word(idi, idj, step, p->seed, p->rounds));
    }
    double FC = a * w;                                /* Eq. 3 */
    double FD = -gamma * ev * wD;                     /* Eq. 5, dissipative */
    double FR = sigma * xi_ij * wR / sqrt(p->dt);     /* Eq. 5, random */
    double s = FC + FD + FR;
    for (int k = 0; k < 3; ++k) fij[k] = s * e[k];
    if (rfc) *rfc = FC * r;
}

/* Body force on a particle at x (Sec. 4.2 periodic Poiseuille: -f below the
 * mid-plane L/2 of the gradient axis, +f above; or a constant force). */
static void body_force(const orc_params *p, const double *x, double *f)
{
    f[0] = f[1] = f[2] = 0.0;
    if (p->fb_mode == 1) {
        f[p->fb_flow] = p->fb;
    } else if (p->fb_mode == 2) {
        double half = 0.5 * p->L[p->fb_grad];
        f[p->fb_flow] = (x[p->fb_grad] <= half) ? -p->fb : p->fb;
    }
}

/* ----------------------------------------------------------------------
 * Cell list of Sec. 3.2: cells of edge h_d = L_d / n_d >= rc with
 * n_d = floor(L_d / rc); cell sizes by counting, starts by an exclusive
 * scan, then each particle placed at start + running size.
 * -------------------------------------------------------------------- */
typedef struct {
    int n[3];
    double h[3];
    int64_t ncell;
    int64_t *start;   /* ncell + 1 */
    int64_t *order;   /* particle index in cell order */
} orc_cells;

static int cell_coord(double x, double h, int n)
{
    int c = (int)floor(x / h);
    if (c < 0) c = 0;
    if (c > n - 1) c = n - 1;
    return c;
}

static int64_t cell_of(const orc_cells *cl, const double *x)
{
    int cx = cell_coord(x[0], cl->h[0], cl->n[0]);
    int cy = cell_coord(x[1], cl->h[1], cl->n[1]);
    int cz = cell_coord(x[2], cl->h[2], cl->n[2]);
    return ((int64_t)cz * cl->n[1] + cy) * cl->n[0] + cx;
}

static int cells_build(const orc_params *p, int64_t n, const double *x, orc_cells *cl)
{
    for (int k = 0; k < 3; ++k) {
        cl->n[k] = (int)floor(p->L[k] / p->rc);
        if (cl->n[k] < 3) return -1;
        cl->h[k] = p->L[k] / cl->n[k];
    }
    cl->ncell = (int64_t)cl->n[0] * cl->n[1] * cl->n[2];
    int64_t *size = calloc((size_t)cl->ncell, sizeof(int64_t));
    cl->start = calloc((size_t)cl->ncell + 1, sizeof(int64_t));
    cl->order = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!size || !cl->start || !cl->order) { free(size); return -2; }
    for (int64_t i = 0; i < n; ++i) size[cell_of(cl, x + 3 * i)]++;          /* count */
    cl->start[0] = 0;
    for (int64_t c = 0; c < cl->ncell; ++c) cl->start[c + 1] = cl->start[c] + size[c];  /* scan */
    memset(size, 0, sizeof(int64_t) * (size_t)cl->ncell);
    for (int64_t i = 0; i < n; ++i) {                                         /* reorder */
        int64_t c = cell_of(cl, x + 3 * i);
        cl->order[cl->start[c] + size[c]++] = i;
    }
    free(size);
    return 0;
}

static void cells_free(orc_cells *cl)
{
    free(cl->start);
    free(cl->order);
    cl->start = NULL;
    cl->order = NULL;
}

/* Force on particle i from every j in the 27 cells around i's cell. */
static void force_on_cells(const orc_params *p, const orc_cells *cl, int64_t i, const double *x,
                           const double *v, const uint32_t *id, uint64_t step, double *fi,
                           double *vir_i)
{
    double f[3] = {0, 0, 0}, vir = 0.0, fij[3], rfc;
    const double *xi = x + 3 * i;
    int cx = cell_coord(xi[0], cl->h[0], cl->n[0]);
    int cy = cell_coord(xi[1], cl->h[1], cl->n[1]);
    int cz = cell_coord(xi[2], cl->h[2], cl->n[2]);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int ax = (cx + dx + cl->n[0]) % cl->n[0];
                int ay = (cy + dy + cl->n[1]) % cl->n[1];
                int az = (cz + dz + cl->n[2]) % cl->n[2];
                int64_t c = ((int64_t)az * cl->n[1] + ay) * cl->n[0] + ax;
                for (int64_t s = cl->start[c]; s < cl->start[c + 1]; ++s) {
                    int64_t j = cl->order[s];
                    if (j == i) continue;
                    orc_pair_force(p, xi, x + 3 * j, v + 3 * i, v + 3 * j, id[i], id[j], step, fij, &rfc);
                    f[0] += fij[0]; f[1] += fij[1]; f[2] += fij[2];
                    vir += rfc;
                }
            }
    fi[0] = f[0]; fi[1] = f[1]; fi[2] = f[2];
    *vir_i = vir;
}

/* ----------------------------------------------------------------------
 * Total force on every particle at step index `step`.
 * mode 0: Eq. 2 as a plain O(N^2) loop over ordered pairs.
 * mode 1: the same sum restricted to the 27-cell neighbourhood.
 * f gets pair forces plus the body force; *virial = sum_{i<j} r_ij . F^C_ij.
 * Returns 0, or a negative code on bad geometry / allocation failure.
 * -------------------------------------------------------------------- */
int orc_forces(const orc_params *p, int64_t n, const double *x, const double *v,
               const uint32_t *id, uint64_t step, int mode, double *f, double *virial)
{
    double *vir = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!vir) return -2;
    if (mode == 0) {
        #pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            double fi[3] = {0, 0, 0}, fij[3], rfc, vi = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                orc_pair_force(p, x + 3 * i, x + 3 * j, v + 3 * i, v + 3 * j, id[i], id[j], step, fij, &rfc);
                fi[0] += fij[0]; fi[1] += fij[1]; fi[2] += fij[2];
                vi += rfc;
            }
            f[3 * i] = fi[0]; f[3 * i + 1] = fi[1]; f[3 * i + 2] = fi[2];
            vir[i] = vi;
        }
    } else {
        orc_cells cl;
        int rc = cells_build(p, n, x, &cl);
        if (rc) { free(vir); return rc; }
        #pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) force_on_cells(p, &cl, i, x, v, id, step, f + 3 * i, vir + i);
        cells_free(&cl);
    }
    double total = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double fb[3];
        body_force(p, x + 3 * i, fb);
        f[3 * i] += fb[0]; f[3 * i + 1] += fb[1]; f[3 * i + 2] += fb[2];
        total += vir[i];
    }
    if (virial) *virial = 0.5 * total;   /* every unordered pair was visited twice */
    free(vir);
    return 0;
}

/* Forces (pair sum + body force) on a chosen subset of particles, from the
 * cell list over all n particles.  f_out is m x 3. */
int orc_forces_subset(const orc_params *p, int64_t n, const double *x, const double *v,
                      const uint32_t *id, uint64_t step, int64_t m, const int64_t *which,
                      double *f_out)
{
    orc_cells cl;
    int rc = cells_build(p, n, x, &cl);
    if (rc) return rc;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < m; ++k) {
        double vir, fb[3];
        int64_t i = which[k];
        force_on_cells(p, &cl, i, x, v, id, step, f_out + 3 * k, &vir);
        body_force(p, x + 3 * i, fb);
        f_out[3 * k] += fb[0]; f_out[3 * k + 1] += fb[1]; f_out[3 * k + 2] += fb[2];
    }
    cells_free(&cl);
    return 0;
}

/* ----------------------------------------------------------------------
 * Time stepping (Eq. 1 by velocity-Verlet, velocity predicted at t + dt/2):
 *   v <- v + dt/2 F/m ;  x <- x + dt v (wrapped) ;  step <- step + 1 ;
 *   F <- F(x, v, step) ;  v <- v + dt/2 F/m.
 * On entry f must hold the force at step0 for the given x, v.  On exit x, v,
 * f hold the state after nsteps steps (v at the full step).  If virial is
 * given it receives the virial of the last force evaluation.
 * -------------------------------------------------------------------- */
int orc_run(const orc_params *p, int64_t n, double *x, double *v, const uint32_t *id, double *f,
            uint64_t step0, int64_t nsteps, int mode, double *virial)
{
    double h = 0.5 * p->dt / p->mass;
    for (int64_t s = 1; s <= nsteps; ++s) {
        for (int64_t i = 0; i < 3 * n; ++i) v[i] += h * f[i];
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < 3; ++k)
                x[3 * i + k] = wrap_coord(x[3 * i + k] + p->dt * v[3 * i + k], p->L[k]);
        int rc = orc_forces(p, n, x, v, id, step0 + (uint64_t)s, mode, f, virial);
        if (rc) return rc;
        for (int64_t i = 0; i < 3 * n; ++i) v[i] += h * f[i];
    }
    return 0;
}

/* Box statistics: out = {P_x, P_y, P_z, KE, kT, pressure}.
 * kT = sum m v^2 / (3 (N - 1)) (three degrees of freedom fixed by the zero
 * total momentum); pressure = rho kT + virial / (3 V). */
void orc_stats(const orc_params *p, int64_t n, const double *v, double virial, double *out)
{
    double P[3] = {0, 0, 0}, ke = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) {
            P[k] += p->mass * v[3 * i + k];
            ke += 0.5 * p->mass * v[3 * i + k] * v[3 * i + k];
        }
    }
    double V = p->L[0] * p->L[1] * p->L[2];
    double kT = (n > 1) ? 2.0 * ke / (3.0 * (double)(n - 1)) : 0.0;
    out[0] = P[0]; out[1] = P[1]; out[2] = P[2];
    out[3] = ke;
    out[4] = kT;
    out[5] = ((double)n / V) * kT + virial / (3.0 * V);
}

/* Mean of the flow-axis velocity in nbins slabs along the gradient axis. */
void orc_profile(const orc_params *p, int64_t n, const double *x, const double *v, int nbins,
                 double *prof, int64_t *counts)
{
    for (int b = 0; b < nbins; ++b) { prof[b] = 0.0; counts[b] = 0; }
    double Lg = p->L[p->fb_grad];
    for (int64_t i = 0; i < n; ++i) {
        int b = (int)floor(x[3 * i + p->fb_grad] / Lg * nbins);
        if (b < 0) b = 0;
        if (b >= nbins) b = nbins - 1;
        prof[b] += v[3 * i + p->fb_flow];
        counts[b]++;
    }
    for (int b = 0; b < nbins; ++b)
        if (counts[b]) prof[b] /= (double)counts[b];
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
