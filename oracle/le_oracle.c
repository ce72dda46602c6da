/*
 * TEST INFRASTRUCTURE ONLY — not part of the product.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of Lees-Edwards (LE)
 * shear-flow molecular dynamics as described in Xu et al., "Implementation and
 * Parallel Optimization of the Lees-Edwards Boundary Condition in ESPResSo++"
 * (arXiv 2109.11083).  Only the tests, the smoke check and the benchmark's CPU
 * baseline may build, load or call this file.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * Geometry (Sec. 2.1): flow along x, gradient along z, vorticity along y.  The
 * box is [0,Lx) x [0,Ly) x [0,Lz).  The image box above the central box is
 * displaced along x by dX(t) = gamma_dot * Lz * t (Fig. 1: 2*delta), reduced
 * modulo Lx (Eq. 4).
 *
 * Readings of the paper that this file takes (each is listed with its reason
 * in the design notes of the repository):
 *   - leaving through the top: z -= Lz, x -= dX, vx -= gamma_dot*Lz; leaving
 *     through the bottom: the mirror image (Eq. 4 with the sign of Fig. 1).
 *   - friction acts on the half-step velocity; the random force is uniform
 *     with variance 2*xi*kT*m/dt per component (the sqrt(24...)*U(-1/2,1/2)
 *     pattern of Eq. 7).
 *   - the random numbers come from Philox4x64-10 (Salmon et al., SC'11),
 *     key = (seed, system), counter = (step, particle id, 0, 0).
 *   - stress is the xz component of Eq. 15 (the text names xy, but with flow
 *     along x and gradient along z the shear component is xz).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double L[3];          /* box edges Lx, Ly, Lz */
    double shear_rate;    /* gamma_dot, Eq. 1 */
    double rc;            /* LJ cut-off radius (strict: r < rc) */
    double eps, sigma;    /* LJ parameters, Eq. 9 */
    int    lj_shift;      /* 1: energy shift of Eq. 10 (forces unchanged) */
    double fene_k, fene_R0; /* FENE, Eq. 11 */
    double mass, kT, xi, dt;
    int    thermostat;    /* 0: none, 1: Langevin on the peculiar velocity (Eq. 5),
                             2: Langevin on the absolute velocity (the xi_abs
                             variant of Sec. 2.2 and Fig. 3), 3: DPD (Eqs. 6-8) */
    uint64_t seed, system;
    int    nbins;         /* velocity-profile bins along z */
    double angle_k;       /* k_a of the bending term of Eq. 12 (0: none) */
    double force_cap;     /* > 0: LJ pair force magnitude limited to this value (the
                             push-off of overlapping initial chains, not part of the
                             method; energies stay those of Eq. 9/10) */
} ora_params;

enum { ORA_OK = 0, ORA_BOND_BROKEN = 1, ORA_BOX_TOO_SMALL = 2, ORA_NONFINITE = 3 };

/* ------------------------------------------------------------------------- */
/* Eq. 4 / Fig. 1: x-offset of the image box above the central one at step n,
 * computed from the integer step (never accumulated). */
double ora_dX(const ora_params *p, int64_t n)
{
    double t = (double)n * p->dt;
    double d = fmod(p->shear_rate * p->L[2] * t, p->L[0]);
    if (d < 0.0) d += p->L[0];
    return d;
}

/* Eq. 1: streaming velocity of the linear shear profile. */
double ora_vs(const ora_params *p, double z)
{
    return p->shear_rate * (z - 0.5 * p->L[2]);
}

/* LE minimum image of r_i - r_j with image offset dX: the image across the
 * top/bottom face is displaced along x by dX (Fig. 1); x and y are periodic. */
void ora_min_image(const ora_params *p, double dX, const double *ri,
                   const double *rj, double *d)
{
    double dx = ri[0] - rj[0], dy = ri[1] - rj[1], dz = ri[2] - rj[2];
    if (dz > 0.5 * p->L[2]) {
        dz -= p->L[2];
        dx -= dX;
    } else if (dz < -0.5 * p->L[2]) {
        dz += p->L[2];
        dx += dX;
    }
    dx -= p->L[0] * nearbyint(dx / p->L[0]);
    dy -= p->L[1] * nearbyint(dy / p->L[1]);
    d[0] = dx; d[1] = dy; d[2] = dz;
}

/* ------------------------------------------------------------------------- */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
 * multiply-xor bijection with a Weyl-sequence key schedule. */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 prod = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(prod >> 64);
    *lo = (uint64_t)prod;
}

void ora_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ULL, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Three uniforms on [-1/2, 1/2) for particle `gid` at step `n`: the top 53
 * bits of the first three Philox words, scaled by 2^-53. */
void ora_noise(const ora_params *p, int64_t n, int64_t gid, double u[3])
{
    uint64_t ctr[4] = {(uint64_t)n, (uint64_t)gid, 0, 0};
    uint64_t key[2] = {p->seed, p->system};
    uint64_t out[4];
    ora_philox4x64(ctr, key, out);
    for (int k = 0; k < 3; ++k)
        u[k] = (double)(out[k] >> 11) * 0x1.0p-53 - 0.5;
}

/* ------------------------------------------------------------------------- */
/* Pair terms.  Eq. 9 (LJ) and Eq. 10 (shifted LJ): the force is the negative
 * gradient of Eq. 9 for r < rc; the shift changes only the energy.  Returns
 * f/r so that F_i = (f/r) * d. */
static double lj_f_over_r(const ora_params *p, double r2, double *energy)
{
    double s2 = p->sigma * p->sigma / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    double e = 4.0 * p->eps * (s12 - s6);
    if (p->lj_shift) {
        double c2 = p->sigma * p->sigma / (p->rc * p->rc);
        double c6 = c2 * c2 * c2;
        e -= 4.0 * p->eps * (c6 * c6 - c6);
    }
    *energy = e;
    return 24.0 * p->eps * (2.0 * s12 - s6) / r2;
}

/* Eq. 11 (FENE): V = -1/2 k R0^2 ln(1 - (r/R0)^2) for r < R0, infinite
 * otherwise.  Returns f/r = -k / (1 - (r/R0)^2), or sets *broken. */
static double fene_f_over_r(const ora_params *p, double r2, double *energy, int *broken)
{
    double R02 = p->fene_R0 * p->fene_R0;
    double x = 1.0 - r2 / R02;
    if (!(x > 0.0)) {
        *broken = 1;
        *energy = INFINITY;
        return 0.0;
    }
    *energy = -0.5 * p->fene_k * R02 * log(x);
    return -p->fene_k / x;
}

/* ------------------------------------------------------------------------- */
/* Candidate-pair enumeration.  mode 0: every pair (i, j != i).  mode 1: a
 * cell grid of edge >= rc (at least 3 cells per dimension, otherwise mode 0
 * is used).  A neighbour row in y and z is scanned over the three adjacent x
 * cells, except across the top/bottom face where the image row is displaced
 * by dX: there the whole x row is scanned.  The candidates are a superset of
 * the pairs within rc; each is then tested with the LE minimum image. */
typedef struct {
    int nc[3];
    double lc[3];
    int *head, *next;
} cell_grid;

static int grid_build(const ora_params *p, int64_t n, const double *pos, cell_grid *g)
{
    for (int a = 0; a < 3; ++a) {
        g->nc[a] = (int)floor(p->L[a] / p->rc);
        if (g->nc[a] < 3) return 0;
        g->lc[a] = p->L[a] / g->nc[a];
    }
    int64_t ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2];
    g->head = (int *)malloc(sizeof(int) * ncell);
    g->next = (int *)malloc(sizeof(int) * n);
    for (int64_t c = 0; c < ncell; ++c) g->head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = (int)floor(pos[3 * i + a] / g->lc[a]);
            if (c[a] < 0) c[a] = 0;
            if (c[a] >= g->nc[a]) c[a] = g->nc[a] - 1;
        }
        int64_t cid = ((int64_t)c[2] * g->nc[1] + c[1]) * g->nc[0] + c[0];
        g->next[i] = g->head[cid];
        g->head[cid] = (int)i;
    }
    return 1;
}

static void grid_free(cell_grid *g)
{
    free(g->head);
    free(g->next);
}

/* Calls visit(i, j) for every candidate j of particle i (j != i). */
typedef void (*visit_fn)(void *ctx, int64_t i, int64_t j);

static void for_candidates(const ora_params *p, int64_t n, const double *pos,
                           int use_cells, void *ctx, visit_fn visit)
{
    cell_grid g;
    if (!use_cells || !grid_build(p, n, pos, &g)) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j)
                if (j != i) visit(ctx, i, j);
        return;
    }
    for (int64_t i = 0; i < n; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = (int)floor(pos[3 * i + a] / g.lc[a]);
            if (c[a] < 0) c[a] = 0;
            if (c[a] >= g.nc[a]) c[a] = g.nc[a] - 1;
        }
        for (int dz = -1; dz <= 1; ++dz) {
            int cz = c[2] + dz;
            int across = (cz < 0 || cz >= g.nc[2]);
            cz = (cz + g.nc[2]) % g.nc[2];
            for (int dy = -1; dy <= 1; ++dy) {
                int cy = (c[1] + dy + g.nc[1]) % g.nc[1];
                int x0 = across ? 0 : c[0] - 1;
                int x1 = across ? g.nc[0] - 1 : c[0] + 1;
                for (int xx = x0; xx <= x1; ++xx) {
                    int cx = (xx + g.nc[0]) % g.nc[0];
                    int64_t cid = ((int64_t)cz * g.nc[1] + cy) * g.nc[0] + cx;
                    for (int j = g.head[cid]; j >= 0; j = g.next[j])
                        if (j != i) visit(ctx, i, j);
                }
            }
        }
    }
    grid_free(&g);
}

typedef struct {
    const ora_params *p;
    double dX;
    const double *pos;
    double *F;
    double W[9];
    double epot;
} pair_ctx;

static void pair_visit(void *vctx, int64_t i, int64_t j)
{
    pair_ctx *c = (pair_ctx *)vctx;
    double d[3];
    ora_min_image(c->p, c->dX, c->pos + 3 * i, c->pos + 3 * j, d);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < c->p->rc * c->p->rc)) return;
    double e;
    double fr = lj_f_over_r(c->p, r2, &e);
    if (c->p->force_cap > 0.0) {   /* |F| = |f/r| r at most force_cap */
        double lim = c->p->force_cap / sqrt(r2);
        if (fr > lim) fr = lim;
        if (fr < -lim) fr = -lim;
    }
    for (int a = 0; a < 3; ++a) c->F[3 * i + a] += fr * d[a];
    if (i < j) {  /* each unordered pair once in the energy and the virial */
        c->epot += e;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) c->W[3 * a + b] += d[a] * fr * d[b];
    }
}

/* Conservative forces at image offset dX: LJ over all pairs within rc plus
 * FENE over the bond list.  W receives sum_{i<j} r_ij (x) F_ij (the virial
 * part of Eq. 15), epot the potential energy (Eq. 13 without the angle term).
 * Returns ORA_BOND_BROKEN if any bond reaches R0 (Eq. 11: +infinity). */
/* Eq. 12, bending term of the Kremer-Grest chains.  As printed the formula
 * is garbled (linear in the angle while called a cosine potential); read as
 * the cosine potential with its equilibrium at the stated 180 degrees,
 *   V(theta) = k_a (1 - cos(theta - pi)) = k_a (1 + cos theta),
 * theta the angle at the middle bead between its two bonds (a straight chain
 * is the minimum).  With a = r_i - r_j, c = r_k - r_j (LE minimum images)
 * and cos theta = a.c / (|a||c|):
 *   F_i = -k_a (c^ - cos theta a^) / |a|,  F_k = -k_a (a^ - cos theta c^) / |c|,
 *   F_j = -(F_i + F_k);
 * virial a (x) F_i + c (x) F_k.  The angles are every pair of bonds that
 * share a bead (one per inner bead of a linear chain). */
static void angle_forces(const ora_params *p, double dX, int64_t n, const double *pos,
                         int64_t nbond, const int32_t *bonds, double *F, double W[9],
                         double *epot)
{
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t b = 0; b < nbond; ++b) {
        ++deg[bonds[2 * b] + 1];
        ++deg[bonds[2 * b + 1] + 1];
    }
    for (int64_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * nbond + 1));
    for (int64_t i = 0; i < n; ++i) fill[i] = deg[i];
    for (int64_t b = 0; b < nbond; ++b) {
        int64_t i = bonds[2 * b], j = bonds[2 * b + 1];
        nb[fill[i]++] = j;
        nb[fill[j]++] = i;
    }
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t u = deg[j]; u < deg[j + 1]; ++u)
            for (int64_t v = u + 1; v < deg[j + 1]; ++v) {
                int64_t i = nb[u], k = nb[v];
                double a[3], c[3];
                ora_min_image(p, dX, pos + 3 * i, pos + 3 * j, a);
                ora_min_image(p, dX, pos + 3 * k, pos + 3 * j, c);
                double la = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
                double lc = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
                double ah[3], ch[3];
                for (int q = 0; q < 3; ++q) {
                    ah[q] = a[q] / la;
                    ch[q] = c[q] / lc;
                }
                double ct = ah[0] * ch[0] + ah[1] * ch[1] + ah[2] * ch[2];
                double fi[3], fk[3];
                for (int q = 0; q < 3; ++q) {
                    fi[q] = -p->angle_k * (ch[q] - ct * ah[q]) / la;
                    fk[q] = -p->angle_k * (ah[q] - ct * ch[q]) / lc;
                    F[3 * i + q] += fi[q];
                    F[3 * k + q] += fk[q];
                    F[3 * j + q] -= fi[q] + fk[q];
                }
                for (int q = 0; q < 3; ++q)
                    for (int r = 0; r < 3; ++r) W[3 * q + r] += a[q] * fi[r] + c[q] * fk[r];
                *epot += p->angle_k * (1.0 + ct);
            }
    }
    free(deg);
    free(fill);
    free(nb);
}

int ora_forces(const ora_params *p, double dX, int64_t n, const double *pos,
               int64_t nbond, const int32_t *bonds, int use_cells,
               double *F, double *W, double *epot)
{
    pair_ctx c;
    c.p = p; c.dX = dX; c.pos = pos; c.F = F; c.epot = 0.0;
    memset(c.W, 0, sizeof c.W);
    memset(F, 0, sizeof(double) * 3 * n);
    if (p->eps != 0.0) for_candidates(p, n, pos, use_cells, &c, pair_visit);
    int broken = 0;
    for (int64_t b = 0; b < nbond; ++b) {
        int64_t i = bonds[2 * b], j = bonds[2 * b + 1];
        double d[3];
        ora_min_image(p, dX, pos + 3 * i, pos + 3 * j, d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double e;
        double fr = fene_f_over_r(p, r2, &e, &broken);
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] += fr * d[a];
            F[3 * j + a] -= fr * d[a];
        }
        c.epot += e;
        for (int a = 0; a < 3; ++a)
            for (int q = 0; q < 3; ++q) c.W[3 * a + q] += d[a] * fr * d[q];
    }
    if (p->angle_k != 0.0 && nbond > 0) angle_forces(p, dX, n, pos, nbond, bonds, F, c.W, &c.epot);
    if (W) memcpy(W, c.W, sizeof c.W);
    if (epot) *epot = c.epot;
    return broken ? ORA_BOND_BROKEN : ORA_OK;
}

/* Conservative LJ force on each of the m particles idx[0..m-1] only, from
 * every particle within rc under the LE minimum image (the plain definition,
 * one particle at a time): used to check sampled particles of systems too
 * large for a full oracle step. */
void ora_forces_on(const ora_params *p, double dX, int64_t n, const double *pos,
                   int64_t m, const int64_t *idx, double *F)
{
    cell_grid g;
    int cells = grid_build(p, n, pos, &g);
    for (int64_t q = 0; q < m; ++q) {
        int64_t i = idx[q];
        double f[3] = {0.0, 0.0, 0.0};
        if (!cells) {
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double d[3];
                ora_min_image(p, dX, pos + 3 * i, pos + 3 * j, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (!(r2 < p->rc * p->rc)) continue;
                double e, fr = lj_f_over_r(p, r2, &e);
                for (int a = 0; a < 3; ++a) f[a] += fr * d[a];
            }
        } else {
            int c[3];
            for (int a = 0; a < 3; ++a) {
                c[a] = (int)floor(pos[3 * i + a] / g.lc[a]);
                if (c[a] < 0) c[a] = 0;
                if (c[a] >= g.nc[a]) c[a] = g.nc[a] - 1;
            }
            for (int dz = -1; dz <= 1; ++dz) {
                int cz = c[2] + dz;
                int across = (cz < 0 || cz >= g.nc[2]);
                cz = (cz + g.nc[2]) % g.nc[2];
                for (int dy = -1; dy <= 1; ++dy) {
                    int cy = (c[1] + dy + g.nc[1]) % g.nc[1];
                    int x0 = across ? 0 : c[0] - 1;
                    int x1 = across ? g.nc[0] - 1 : c[0] + 1;
                    for (int xx = x0; xx <= x1; ++xx) {
                        int cx = (xx + g.nc[0]) % g.nc[0];
                        int64_t cid = ((int64_t)cz * g.nc[1] + cy) * g.nc[0] + cx;
                        for (int j = g.head[cid]; j >= 0; j = g.next[j]) {
                            if (j == i) continue;
                            double d[3];
                            ora_min_image(p, dX, pos + 3 * i, pos + 3 * j, d);
                            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                            if (!(r2 < p->rc * p->rc)) continue;
                            double e, fr = lj_f_over_r(p, r2, &e);
                            for (int a = 0; a < 3; ++a) f[a] += fr * d[a];
                        }
                    }
                }
            }
        }
        for (int a = 0; a < 3; ++a) F[3 * q + a] = f[a];
    }
    if (cells) grid_free(&g);
}

/* First-order bound on the error of a force computed in a floating-point
 * format of unit roundoff u from coordinates stored relative to reference
 * points no farther than P (per component) from the particle:
 *   - each separation component carries an error of at most u*(6P + 2r)
 *     (two rounded coordinates, one rounded offset between references,
 *     two additions);
 *   - a pair force F = f(r) d then moves by at most J(r)*sqrt(3)*u*(6P + 2r)
 *     with J = |f| + r|f'| (the norm of dF/dd);
 *   - its evaluation adds 16u|F| and a sequential sum of m terms adds
 *     (m + 2)u * sum |F_ij|.
 * B[i] receives the bound for particle i (LJ of Eq. 9 and FENE of Eq. 11).
 * Test infrastructure: used only to set the tolerance of reduced-precision
 * comparisons. */
typedef struct {
    const ora_params *p;
    double dX, u, P;
    const double *pos;
    double *B, *S;
    int64_t *m;
} bound_ctx;

static void bound_add(bound_ctx *c, int64_t i, double r2, double f, double rfp)
{
    double r = sqrt(r2);
    double J = fabs(f) + fabs(rfp);
    c->B[i] += J * sqrt(3.0) * c->u * (6.0 * c->P + 2.0 * r) + 16.0 * c->u * fabs(f) * r;
    c->S[i] += fabs(f) * r;
    c->m[i] += 1;
}

static void bound_visit(void *vctx, int64_t i, int64_t j)
{
    bound_ctx *c = (bound_ctx *)vctx;
    double d[3];
    ora_min_image(c->p, c->dX, c->pos + 3 * i, c->pos + 3 * j, d);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double rc = c->p->rc;
    /* a pair within the separation error band of the cut-off may fall on
     * either side of the strict r < rc test: either answer is a correct
     * reduced-precision result, so the bound admits the whole pair force */
    double band = sqrt(3.0) * c->u * (6.0 * c->P + 2.0 * rc);
    double r = sqrt(r2);
    if (fabs(r - rc) <= band) {
        double ec, fc = lj_f_over_r(c->p, rc * rc, &ec);
        c->B[i] += fabs(fc) * rc;
    }
    if (!(r2 < rc * rc)) return;
    double e, f = lj_f_over_r(c->p, r2, &e);
    double s2 = c->p->sigma * c->p->sigma / r2, s6 = s2 * s2 * s2;
    /* r f'(r) for f = 24 eps (2 s^12 r^-2 - s^6 r^-2) */
    double rfp = 24.0 * c->p->eps * (-28.0 * s6 * s6 + 8.0 * s6) / r2;
    bound_add(c, i, r2, f, rfp);
}

void ora_force_error_bound(const ora_params *p, double dX, int64_t n, const double *pos,
                           int64_t nbond, const int32_t *bonds, double u, double P,
                           double *B)
{
    bound_ctx c;
    c.p = p; c.dX = dX; c.u = u; c.P = P; c.pos = pos; c.B = B;
    c.S = (double *)calloc((size_t)n, sizeof(double));
    c.m = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    memset(B, 0, sizeof(double) * n);
    if (p->eps != 0.0) {
        ora_params q = *p;  /* a grid edge slightly above rc also covers the band */
        q.rc = p->rc * (1.0 + 1e-4);
        for_candidates(&q, n, pos, 1, &c, bound_visit);
    }
    double R02 = p->fene_R0 * p->fene_R0;
    for (int64_t b = 0; b < nbond; ++b) {
        int64_t ends[2] = {bonds[2 * b], bonds[2 * b + 1]};
        double d[3];
        ora_min_image(p, dX, pos + 3 * ends[0], pos + 3 * ends[1], d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double x = 1.0 - r2 / R02;
        if (!(x > 0.0)) continue;
        double f = -p->fene_k / x;
        double rfp = -2.0 * p->fene_k * r2 / (R02 * x * x);
        for (int q = 0; q < 2; ++q) bound_add(&c, ends[q], r2, f, rfp);
    }
    for (int64_t i = 0; i < n; ++i) B[i] += (double)(c.m[i] + 2) * u * c.S[i];
    free(c.S);
    free(c.m);
}

/* The pairs a reduced-precision evaluation may legitimately decide either
 * way: every ordered pair (i, j) whose LE minimum-image distance lies within
 * `band` of the strict cut-off of Eq. 9/10 (|r - rc| <= band).  For each, the
 * pair force F_ij = f(r) d at its FP64 separation, and whether ora_forces
 * counts it (r < rc).  Writes at most `cap` pairs and returns how many there
 * are.  Test infrastructure: lets a comparison take either decision for such
 * a pair and count the pairs decided the other way. */
typedef struct {
    const ora_params *p;
    double dX, band;
    const double *pos;
    int64_t cap, count;
    int64_t *ij;
    double *f;
    int32_t *inside;
} band_ctx;

static void band_visit(void *vctx, int64_t i, int64_t j)
{
    band_ctx *c = (band_ctx *)vctx;
    double d[3];
    ora_min_image(c->p, c->dX, c->pos + 3 * i, c->pos + 3 * j, d);
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double rc = c->p->rc;
    if (!(fabs(r - rc) <= c->band)) return;
    if (c->count < c->cap) {
        double e, fr = lj_f_over_r(c->p, r * r, &e);
        int64_t k = c->count;
        c->ij[2 * k] = i;
        c->ij[2 * k + 1] = j;
        for (int a = 0; a < 3; ++a) c->f[3 * k + a] = fr * d[a];
        c->inside[k] = (r * r < rc * rc) ? 1 : 0;
    }
    c->count += 1;
}

int64_t ora_band_pairs(const ora_params *p, double dX, int64_t n, const double *pos,
                       double band, int64_t cap, int64_t *ij, double *f, int32_t *inside)
{
    band_ctx c;
    c.p = p; c.dX = dX; c.band = band; c.pos = pos;
    c.cap = cap; c.count = 0; c.ij = ij; c.f = f; c.inside = inside;
    if (p->eps == 0.0) return 0;
    ora_params q = *p;   /* a grid edge of rc + band covers every pair in the band */
    q.rc = p->rc + band;
    for_candidates(&q, n, pos, 1, &c, band_visit);
    return c.count;
}

/* ------------------------------------------------------------------------- */
/* Eqs. 6-8, the DPD thermostat: pairwise dissipative and random forces for
 * r < rc.  As printed both carry |r^.v_ij| and the random force has no
 * 1/sqrt(dt); read as the textbook form that satisfies the fluctuation-
 * dissipation relation with the paper's own noise pattern (Eq. 7's
 * sqrt(24 kT xi) theta, theta in U(-1/2, 1/2)):
 *   F_ij = [-xi w^2 (r^.v_ij) + sqrt(24 kT xi / dt) theta_ij w] r^,
 *   w = 1 - r/rc (Eq. 8),  r^ = d/r,  d = the LE minimum image r_i - r_j.
 * v_ij is the velocity of i relative to the image of j that d refers to:
 * the image above the box (d_z shifted by -Lz) moves at +shear_rate*Lz
 * along x, so v_ij = v_i - v_j - shear_rate*Lz e_x, mirrored below.
 * theta_ij is shared by the two members of a pair: Philox4x64-10 with key
 * (seed, system) and counter (step, min id, max id, 1) (the 1 separates it
 * from the Langevin stream), first output word to U(-1/2, 1/2) by its top
 * 53 bits.  F_ji = -F_ij exactly, so DPD conserves momentum. */
double ora_pair_uniform(const ora_params *p, int64_t n, int64_t a, int64_t b)
{
    uint64_t lo = (uint64_t)(a < b ? a : b), hi = (uint64_t)(a < b ? b : a);
    uint64_t ctr[4] = {(uint64_t)n, lo, hi, 1};
    uint64_t key[2] = {p->seed, p->system};
    uint64_t out[4];
    ora_philox4x64(ctr, key, out);
    return (double)(out[0] >> 11) * 0x1.0p-53 - 0.5;
}

typedef struct {
    const ora_params *p;
    double dX;
    int64_t step;
    const double *pos, *vel;
    double *F;
} dpd_ctx;

static void dpd_visit(void *vctx, int64_t i, int64_t j)
{
    dpd_ctx *c = (dpd_ctx *)vctx;
    const ora_params *p = c->p;
    double d[3];
    ora_min_image(p, c->dX, c->pos + 3 * i, c->pos + 3 * j, d);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < p->rc * p->rc)) return;
    double r = sqrt(r2), w = 1.0 - r / p->rc;
    double raw_dz = c->pos[3 * i + 2] - c->pos[3 * j + 2];
    double vshift = 0.0;
    if (raw_dz > 0.5 * p->L[2]) vshift = -p->shear_rate * p->L[2];
    else if (raw_dz < -0.5 * p->L[2]) vshift = p->shear_rate * p->L[2];
    double v[3] = {c->vel[3 * i] - c->vel[3 * j] + vshift,
                   c->vel[3 * i + 1] - c->vel[3 * j + 1],
                   c->vel[3 * i + 2] - c->vel[3 * j + 2]};
    double ev = (d[0] * v[0] + d[1] * v[1] + d[2] * v[2]) / r;
    double theta = ora_pair_uniform(p, c->step, i, j);
    double f = -p->xi * w * w * ev + sqrt(24.0 * p->kT * p->xi / p->dt) * theta * w;
    for (int a = 0; a < 3; ++a) c->F[3 * i + a] += f * d[a] / r;
}

/* ------------------------------------------------------------------------- */
/* Eq. 5: total force = conservative - xi*m*(v - v_s(z) e_x) + random, the
 * friction acting on the peculiar velocity.  v is the half-step velocity.
 * Thermostat 2 is the paper's comparison variant (Sec. 2.2): the same
 * friction and noise, the friction acting on the absolute velocity v. */
static void thermostat_force(const ora_params *p, int64_t step, int64_t n,
                             const double *pos, const double *vel,
                             const double *Fc, double *Ftot)
{
    double amp = sqrt(24.0 * p->xi * p->kT * p->mass / p->dt);
    if (p->thermostat == 3) {
        memcpy(Ftot, Fc, sizeof(double) * 3 * n);
        dpd_ctx c = {p, ora_dX(p, step), step, pos, vel, Ftot};
        for_candidates(p, n, pos, 1, &c, dpd_visit);
        return;
    }
    for (int64_t i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) Ftot[3 * i + a] = Fc[3 * i + a];
        if (p->thermostat != 1 && p->thermostat != 2) continue;
        double u[3];
        ora_noise(p, step, i, u);
        double vs = p->thermostat == 1 ? ora_vs(p, pos[3 * i + 2]) : 0.0;
        double vpec[3] = {vel[3 * i] - vs, vel[3 * i + 1], vel[3 * i + 2]};
        for (int a = 0; a < 3; ++a)
            Ftot[3 * i + a] += -p->xi * p->mass * vpec[a] + amp * u[a];
    }
}

/* Forces at step n for the state (pos, vel): fills Fc and Ftot.  Used to
 * start a run (with the initial velocity standing in for the half-step one). */
int ora_init_forces(const ora_params *p, int64_t step, int64_t n, const double *pos,
                    const double *vel, int64_t nbond, const int32_t *bonds,
                    int use_cells, double *Fc, double *Ftot, double *W, double *epot)
{
    int st = ora_forces(p, ora_dX(p, step), n, pos, nbond, bonds, use_cells, Fc, W, epot);
    thermostat_force(p, step, n, pos, vel, Fc, Ftot);
    return st;
}

/* Running samples (Eqs. 14-15 and the z-profiles of Sec. 3.1). */
typedef struct {
    int64_t nsamples;
    double sxz_sum;          /* sum over samples of sigma_xz */
    double stress[9];        /* last instantaneous tensor, Eq. 15 */
    double tpec;             /* last peculiar temperature (3N-3 dof) */
    double epot;             /* last potential energy */
    double *vx_sum;          /* nbins: sum of lab-frame vx */
    int64_t *count;          /* nbins */
    double *vy2_sum;         /* nbins: sum of m vy^2 (T_y profile, Sec. 3.1); may be NULL */
} ora_samples;

static void sample(const ora_params *p, int64_t n, const double *pos,
                   const double *vel, const double *W, double epot, ora_samples *s)
{
    double V = p->L[0] * p->L[1] * p->L[2];
    double K[9] = {0};
    double ke = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double u[3] = {vel[3 * i] - ora_vs(p, pos[3 * i + 2]), vel[3 * i + 1],
                       vel[3 * i + 2]};
        for (int a = 0; a < 3; ++a) {
            ke += p->mass * u[a] * u[a];
            for (int b = 0; b < 3; ++b) K[3 * a + b] += p->mass * u[a] * u[b];
        }
        if (s->vx_sum && p->nbins > 0) {
            int bin = (int)floor(pos[3 * i + 2] / p->L[2] * p->nbins);
            if (bin < 0) bin = 0;
            if (bin >= p->nbins) bin = p->nbins - 1;
            s->vx_sum[bin] += vel[3 * i];
            s->count[bin] += 1;
            if (s->vy2_sum) s->vy2_sum[bin] += p->mass * vel[3 * i + 1] * vel[3 * i + 1];
        }
    }
    for (int a = 0; a < 9; ++a) s->stress[a] = -(K[a] + W[a]) / V;
    s->sxz_sum += s->stress[2];
    s->nsamples += 1;
    s->tpec = n > 1 ? ke / (3.0 * n - 3.0) : 0.0;
    s->epot = epot;
}

/* One velocity-Verlet step n -> n+1 under LE (the order every implementation
 * in this repository follows):
 *   1. v += dt/(2m) Ftot(n)
 *   2. r += dt v
 *   3. dX(n+1) from the integer step
 *   4. LE wrap through the top/bottom face with the velocity jump; x, y periodic
 *   5. Fc(n+1): LJ + FENE with the LE minimum image at dX(n+1)
 *   6. Ftot(n+1) = Fc - xi m (v - v_s(z) e_x) + random        (Eq. 5)
 *   7. v += dt/(2m) Ftot(n+1)
 *   8. samples (Eq. 15 stress, z-profile of vx, peculiar temperature)
 * zimg (optional) counts each particle's net crossings through the top face. */
int ora_run(const ora_params *p, int64_t *step, int64_t nsteps, int64_t n,
            double *pos, double *vel, double *Fc, double *Ftot,
            int64_t nbond, const int32_t *bonds, int use_cells,
            int32_t *zimg, int sample_every, ora_samples *s)
{
    const double Lx = p->L[0], Ly = p->L[1], Lz = p->L[2];
    const double half = p->dt / (2.0 * p->mass);
    double W[9], epot;
    for (int64_t it = 0; it < nsteps; ++it) {
        for (int64_t q = 0; q < 3 * n; ++q) vel[q] += half * Ftot[q];
        for (int64_t q = 0; q < 3 * n; ++q) pos[q] += p->dt * vel[q];
        int64_t next = *step + 1;
        double dX = ora_dX(p, next);
        for (int64_t i = 0; i < n; ++i) {
            double *r = pos + 3 * i, *v = vel + 3 * i;
            if (r[2] >= Lz) {
                r[2] -= Lz;
                r[0] -= dX;
                v[0] -= p->shear_rate * Lz;
                if (zimg) zimg[i] += 1;
            } else if (r[2] < 0.0) {
                double zz = r[2] + Lz;
                if (zz < Lz) {
                    r[2] = zz;
                    r[0] += dX;
                    v[0] += p->shear_rate * Lz;
                    if (zimg) zimg[i] -= 1;
                } else {
                    /* z within rounding of 0 from below: the particle sits on
                     * the bottom face, where no image shift is needed */
                    r[2] = 0.0;
                }
            }
            r[0] -= Lx * floor(r[0] / Lx);
            r[1] -= Ly * floor(r[1] / Ly);
            /* floor-based wrapping can round up to exactly L for tiny
             * negative inputs; fold that back into [0, L) */
            if (r[0] >= Lx) r[0] -= Lx;
            if (r[1] >= Ly) r[1] -= Ly;
        }
        int st = ora_forces(p, dX, n, pos, nbond, bonds, use_cells, Fc, W, &epot);
        if (st != ORA_OK) return st;
        thermostat_force(p, next, n, pos, vel, Fc, Ftot);
        for (int64_t q = 0; q < 3 * n; ++q) vel[q] += half * Ftot[q];
        *step = next;
        for (int64_t q = 0; q < 3 * n; ++q)
            if (!isfinite(pos[q]) || !isfinite(vel[q])) return ORA_NONFINITE;
        if (s && sample_every > 0 && (next % sample_every) == 0)
            sample(p, n, pos, vel, W, epot, s);
    }
    return ORA_OK;
}

/* Instantaneous Eq. 15 tensor, peculiar temperature and potential energy of
 * a state, without advancing it. */
int ora_observe(const ora_params *p, int64_t step, int64_t n, const double *pos,
                const double *vel, int64_t nbond, const int32_t *bonds,
                int use_cells, double *stress9, double *tpec, double *epot)
{
    double *F = (double *)malloc(sizeof(double) * 3 * n);
    double W[9], e;
    int st = ora_forces(p, ora_dX(p, step), n, pos, nbond, bonds, use_cells, F, W, &e);
    free(F);
    ora_samples s;
    memset(&s, 0, sizeof s);
    sample(p, n, pos, vel, W, e, &s);
    memcpy(stress9, s.stress, sizeof s.stress);
    *tpec = s.tpec;
    *epot = e;
    return st;
}
