/*
 * lb_oracle.c -- plain, slow FP64 CPU oracle for the fluctuating D3Q19
 * lattice-Boltzmann update with frictional point-particle coupling
 * (Duenweg & Ladd, "Lattice Boltzmann simulations of soft matter systems",
 * arXiv 0803.2826).
 *
 * TEST INFRASTRUCTURE ONLY.  This file defines what the CUDA library must
 * compute; it is used by the test-suite, by the smoke check and by the
 * benchmark's CPU-baseline leg, and by nothing else.  It shares no source,
 * header, table or constant with the CUDA library.  Every table here is built
 * at start-up from the definitions printed in the paper (velocity set,
 * weights, Table 1 polynomials); nothing is hand-factorised.
 *
 * Arithmetic is IEEE double throughout, no fast-math.  Loops follow the
 * paper's steps in the paper's order.  The only parallelism is an OpenMP
 * "parallel for" over independent lattice nodes / particles, which does not
 * change any per-node result.
 *
 * Conventions that the paper leaves open (the project's readings):
 *  - velocity order: i=0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = the twelve
 *    (+-1,+-1,0), (0,+-1,+-1), (+-1,0,+-1) vectors in that group order, the
 *    two signs (of the two non-zero components, x before y before z) in the
 *    order (+,+),(+,-),(-,+),(-,-);
 *  - lattice units b = h = 1, nodes at integer coordinates 0..L-1;
 *  - population layout [19][nz][ny][nx] (x fastest), raw n_i in FP64;
 *  - the stored state is the post-collision population n*_i(r); one step is
 *    "stream (pull) then collide";
 *  - conserved-mode eigenvalues gamma_0..3 = 1;
 *  - noise: Philox4x32-10 keyed on (seed) with counter
 *    (node, step, domain<<8 | block, replica), 23-bit odd uniforms,
 *    Box-Muller pairs;
 *  - interpolation: phi_2 by default, phi_3 / phi_4 on request (Sec. 4.6);
 *    with walls a particle stays K/2 lattice units from the solid planes,
 *    K the stencil width;
 *  - the fluid receives the impulse of the drag and random forces of each
 *    sub-step, J = p' - p - h F^c (Eq. ftotal);
 *  - the exponential equilibrium (Eq. equildist_lagrange) replaces the
 *    quadratic one in the collision when params.equilibrium = 1;
 *  - solid spheres: see the section on extended particles below.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19
#define CS2 (1.0 / 3.0)

/* ------------------------------------------------------------------------ */
/* Lattice algebra (Sec. 3.3, D3Q19 weights; Sec. 3.4, Table 1)             */
/* ------------------------------------------------------------------------ */

static int g_c[Q][3];      /* velocity vectors c_i                          */
static double g_a[Q];      /* equilibrium weights a^{c_i}                   */
static double g_e[Q][Q];   /* basis vectors e_{ki} (row k, column i)        */
static double g_w[Q];      /* norms w_k = sum_i a_i e_ki^2                  */
static int g_opp[Q];       /* index of -c_i                                 */
static int g_ready = 0;

static void build_tables(void)
{
    if (g_ready) return;
    int i = 0;
    g_c[i][0] = g_c[i][1] = g_c[i][2] = 0;
    i++;
    /* six nearest neighbours: +e_alpha then -e_alpha, alpha = x, y, z */
    for (int al = 0; al < 3; al++) {
        for (int s = 0; s < 2; s++) {
            g_c[i][0] = g_c[i][1] = g_c[i][2] = 0;
            g_c[i][al] = (s == 0) ? 1 : -1;
            i++;
        }
    }
    /* twelve next-nearest neighbours: (+-1,+-1,0), (0,+-1,+-1), (+-1,0,+-1);
     * the two signs apply to the two non-zero components in x, y, z order */
    const int plane[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    const int sg[4][2] = {{1, 1}, {1, -1}, {-1, 1}, {-1, -1}};
    for (int p = 0; p < 3; p++) {
        for (int s = 0; s < 4; s++) {
            g_c[i][0] = g_c[i][1] = g_c[i][2] = 0;
            g_c[i][plane[p][0]] = sg[s][0];
            g_c[i][plane[p][1]] = sg[s][1];
            i++;
        }
    }
    /* weights by speed: a^0 = 1/3, a^1 = 1/18, a^sqrt2 = 1/36 (Sec. 3.3) */
    for (i = 0; i < Q; i++) {
        int c2 = g_c[i][0] * g_c[i][0] + g_c[i][1] * g_c[i][1] + g_c[i][2] * g_c[i][2];
        g_a[i] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
    }
    for (i = 0; i < Q; i++) {
        for (int j = 0; j < Q; j++) {
            if (g_c[j][0] == -g_c[i][0] && g_c[j][1] == -g_c[i][1] && g_c[j][2] == -g_c[i][2])
                g_opp[i] = j;
        }
    }
    /* Table 1: the nineteen polynomials in c_hat = c / (b/h) = c */
    for (i = 0; i < Q; i++) {
        double x = g_c[i][0], y = g_c[i][1], z = g_c[i][2];
        double c2 = x * x + y * y + z * z;
        g_e[0][i] = 1.0;
        g_e[1][i] = x;
        g_e[2][i] = y;
        g_e[3][i] = z;
        g_e[4][i] = c2 - 1.0;
        g_e[5][i] = 3.0 * x * x - c2;
        g_e[6][i] = y * y - z * z;
        g_e[7][i] = x * y;
        g_e[8][i] = y * z;
        g_e[9][i] = z * x;
        g_e[10][i] = (3.0 * c2 - 5.0) * x;
        g_e[11][i] = (3.0 * c2 - 5.0) * y;
        g_e[12][i] = (3.0 * c2 - 5.0) * z;
        g_e[13][i] = (y * y - z * z) * x;
        g_e[14][i] = (z * z - x * x) * y;
        g_e[15][i] = (x * x - y * y) * z;
        g_e[16][i] = 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
        g_e[17][i] = (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
        g_e[18][i] = (2.0 * c2 - 3.0) * (y * y - z * z);
    }
    /* normalising factors, Eq. (weights_unweighted) with q = a */
    for (int k = 0; k < Q; k++) {
        double s = 0.0;
        for (i = 0; i < Q; i++) s += g_a[i] * g_e[k][i] * g_e[k][i];
        g_w[k] = s;
    }
    g_ready = 1;
}

/* Threads the OpenMP loops use (1 without OpenMP). */
int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Export the tables so the tests can check them against the paper. */
void ora_tables(int *c, double *a, double *e, double *w, int *opp)
{
    build_tables();
    for (int i = 0; i < Q; i++) {
        if (c) for (int d = 0; d < 3; d++) c[3 * i + d] = g_c[i][d];
        if (a) a[i] = g_a[i];
        if (opp) opp[i] = g_opp[i];
    }
    for (int k = 0; k < Q; k++) {
        if (w) w[k] = g_w[k];
        if (e) for (int i = 0; i < Q; i++) e[Q * k + i] = g_e[k][i];
    }
}

/* ------------------------------------------------------------------------ */
/* Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,  */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from the   */
/* published round definition.                                              */
/* ------------------------------------------------------------------------ */

void ora_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;  /* Weyl increments: golden ratio, sqrt(3)-1 */
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1): the top 23 bits of a word become the odd integer
 * 2*(x>>9)+1 < 2^24, scaled by 2^-24 (exact in binary32 and binary64). */
double ora_uniform(uint32_t x)
{
    return (2.0 * (double)(x >> 9) + 1.0) * (1.0 / 16777216.0);
}

/* 16 raw words for (seed, node, step, domain, replica): four Philox blocks. */
void ora_raw16(uint64_t seed, uint32_t node, uint32_t step, uint32_t domain,
               uint32_t replica, int nblocks, uint32_t *out)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int b = 0; b < nblocks; b++) {
        uint32_t ctr[4] = {node, step, (domain << 8) | (uint32_t)b, replica};
        ora_philox4x32_10(ctr, key, out + 4 * b);
    }
}

/* The Box-Muller transform of one pair of raw words (Sec. 3.5 asks for
 * unit-variance Gaussians): sqrt(-2 ln v1) (cos, sin)(2 pi v2). */
static void box_muller_pair(uint32_t w1, uint32_t w2, double g[2])
{
    const double two_pi = 6.283185307179586476925286766559;
    double v1 = ora_uniform(w1);
    double v2 = ora_uniform(w2);
    double rad = sqrt(-2.0 * log(v1));
    g[0] = rad * cos(two_pi * v2);
    g[1] = rad * sin(two_pi * v2);
}

/* The same for npairs word pairs w[2q], w[2q+1]. */
void ora_box_muller(const uint32_t *w, long npairs, double *g)
{
#pragma omp parallel for schedule(static)
    for (long q = 0; q < npairs; q++) box_muller_pair(w[2 * q], w[2 * q + 1], g + 2 * q);
}

/* Gaussians by the Box-Muller transform on consecutive uniform pairs. */
void ora_gaussians(uint64_t seed, uint32_t node, uint32_t step, uint32_t domain,
                   uint32_t replica, int nblocks, double *g)
{
    uint32_t raw[16];
    ora_raw16(seed, node, step, domain, replica, nblocks, raw);
    for (int p = 0; p < 2 * nblocks; p++) box_muller_pair(raw[2 * p], raw[2 * p + 1], g + 2 * p);
}

/* ------------------------------------------------------------------------ */
/* Parameters                                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz;
    int walls;          /* 1: solid planes z = 0 and z = nz-1 (link bounce-back) */
    int noise_rho0;     /* 1: noise amplitude uses rho0 instead of local rho      */
    int equilibrium;    /* collision equilibrium: 0 Eq. original_equil_distrib,   */
                        /* 1 the exponential form of Eq. equildist_lagrange       */
    double rho0;
    double kT;
    double gamma_shear, gamma_bulk, gamma_odd, gamma_even;
    double body_force[3];
    uint64_t seed;
    uint32_t replica;
    uint32_t pad2_;
} ora_params;

static size_t nodes_of(const ora_params *P) { return (size_t)P->nx * P->ny * P->nz; }

static size_t lin(const ora_params *P, int x, int y, int z)
{
    return ((size_t)z * P->ny + y) * P->nx + x;
}

static int is_solid(const ora_params *P, int z)
{
    return P->walls && (z == 0 || z == P->nz - 1);
}

static int wrap(int v, int L) { return ((v % L) + L) % L; }

/* Eigenvalue gamma_k of mode k (Sec. 3.4): conserved modes 0..3 keep their
 * non-equilibrium part (gamma = 1); bulk mode 4; shear modes 5..9; kinetic
 * modes 10..15 (odd, gamma_3a = gamma_3b) and 16..18 (even, gamma_4a = gamma_4b). */
static double gamma_of(const ora_params *P, int k)
{
    if (k <= 3) return 1.0;
    if (k == 4) return P->gamma_bulk;
    if (k <= 9) return P->gamma_shear;
    if (k <= 15) return P->gamma_odd;
    return P->gamma_even;
}

/* Eq. (original_equil_distrib): quadratic equilibrium. */
static void equilibrium(double rho, const double u[3], double neq[Q])
{
    double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; i++) {
        double cu = u[0] * g_c[i][0] + u[1] * g_c[i][1] + u[2] * g_c[i][2];
        neq[i] = g_a[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - u2 / (2.0 * CS2));
    }
}

/* Eq. (equildist_lagrange): the equilibrium that maximises the entropy of
 * Eq. (boltzmann_entropy_function) under the mass and momentum constraints
 * (Eqs. constraint_mass, constraint_mom): n^eq_i = rho a_i exp(lambda.c_i) / Z,
 * Z = sum_i a_i exp(lambda.c_i) (the normalisation stands for lambda_rho),
 * with lambda the root of sum_i a_i c_i exp(lambda.c_i) / Z = u.  The root
 * is found by Newton's method (the Jacobian is the covariance of c under the
 * weights a_i exp(lambda.c_i) / Z, positive definite), started from the
 * first-order value lambda = u / c_s^2. */
static void exp_equilibrium(double rho, const double u[3], double neq[Q])
{
    double lam[3] = {u[0] / CS2, u[1] / CS2, u[2] / CS2};
    for (int it = 0; it < 60; it++) {
        double w[Q], Z = 0.0, m[3] = {0, 0, 0}, C[3][3] = {{0}};
        for (int i = 0; i < Q; i++) {
            w[i] = g_a[i] * exp(lam[0] * g_c[i][0] + lam[1] * g_c[i][1] + lam[2] * g_c[i][2]);
            Z += w[i];
        }
        for (int i = 0; i < Q; i++)
            for (int a = 0; a < 3; a++) m[a] += w[i] * g_c[i][a] / Z;
        for (int i = 0; i < Q; i++)
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) C[a][b] += w[i] * (g_c[i][a] - m[a]) * (g_c[i][b] - m[b]) / Z;
        double r[3] = {u[0] - m[0], u[1] - m[1], u[2] - m[2]};
        if (fabs(r[0]) + fabs(r[1]) + fabs(r[2]) < 1e-16) break;
        /* solve C d = r (Cramer's rule on the symmetric 3x3 system) */
        double det = C[0][0] * (C[1][1] * C[2][2] - C[1][2] * C[2][1]) - C[0][1] * (C[1][0] * C[2][2] - C[1][2] * C[2][0])
                   + C[0][2] * (C[1][0] * C[2][1] - C[1][1] * C[2][0]);
        double d[3];
        for (int k = 0; k < 3; k++) {
            double M[3][3];
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) M[a][b] = (b == k) ? r[a] : C[a][b];
            d[k] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                    + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
        }
        for (int k = 0; k < 3; k++) lam[k] += d[k];
    }
    double Z = 0.0, w[Q];
    for (int i = 0; i < Q; i++) {
        w[i] = g_a[i] * exp(lam[0] * g_c[i][0] + lam[1] * g_c[i][1] + lam[2] * g_c[i][2]);
        Z += w[i];
    }
    for (int i = 0; i < Q; i++) neq[i] = rho * w[i] / Z;
}

void ora_exp_equilibrium(double rho, const double *u, double *neq)
{
    build_tables();
    exp_equilibrium(rho, u, neq);
}

/* Equilibrium populations for given fields rho [N] and u [3][N] (NULL: rho0, 0). */
void ora_equilibrium(const ora_params *P, const double *rho, const double *u, double *pops)
{
    build_tables();
    size_t N = nodes_of(P);
    for (size_t s = 0; s < N; s++) {
        double r = rho ? rho[s] : P->rho0;
        double uu[3] = {0.0, 0.0, 0.0};
        if (u) { uu[0] = u[s]; uu[1] = u[N + s]; uu[2] = u[2 * N + s]; }
        double ne[Q];
        equilibrium(r, uu, ne);
        for (int i = 0; i < Q; i++) pops[(size_t)i * N + s] = ne[i];
    }
}

/* Pull streaming, Eq. (LBE): n_i(r) = n*_i(r - c_i).  With walls, a link
 * whose source node is solid is bounced back (Sec. 4.1, Eq. (MBB) with
 * u_b = 0): n_i(r) = n*_{opp(i)}(r). */
static void gather(const ora_params *P, const double *src, int x, int y, int z, double n[Q])
{
    size_t N = nodes_of(P);
    for (int i = 0; i < Q; i++) {
        int sx = wrap(x - g_c[i][0], P->nx);
        int sy = wrap(y - g_c[i][1], P->ny);
        int sz = z - g_c[i][2];
        if (P->walls) {
            if (sz < 0 || sz >= P->nz || is_solid(P, sz)) {
                n[i] = src[(size_t)g_opp[i] * N + lin(P, x, y, z)];
                continue;
            }
        } else {
            sz = wrap(sz, P->nz);
        }
        n[i] = src[(size_t)i * N + lin(P, sx, sy, sz)];
    }
}

/* Total force density on node s: uniform body force plus the optional field
 * (layout [3][N]). */
static void node_force(const ora_params *P, const double *force, size_t s, double f[3])
{
    size_t N = nodes_of(P);
    for (int d = 0; d < 3; d++) {
        f[d] = P->body_force[d];
        if (force) f[d] += force[(size_t)d * N + s];
    }
}

/* One collision, Sec. 3.4, 3.5 and 3.7:
 *   rho = sum n, j = sum n c + f/2, u = j / rho         (Eq. special_choice_momentum_density)
 *   n^neq = n - n^eq(rho, u)                             (Eq. original_equil_distrib)
 *   m^neq_k = sum_i e_ki n^neq_i                         (Eq. forward)
 *   m*^neq_k = gamma_k m^neq_k + phi_k sqrt(w_k mu rho) r_k,  k >= 4
 *                                                        (Eqs. lco_update, stochupdaterule1,
 *                                                         detailedbalance1, normalized_mk)
 *   n*_i = n^eq_i + a_i sum_k e_ki m*^neq_k / w_k + Delta''_i
 *                                                        (Eq. back_transformation, q = a;
 *                                                         Delta'' of Sec. 3.7)
 * mu = k_B T / (b^3 c_s^2) (Sec. 3.5).  r: 15 Gaussians r_4..r_18 or NULL. */
static void collide(const ora_params *P, const double n[Q], const double f[3],
                    const double *r, double nstar[Q])
{
    double rho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int i = 0; i < Q; i++) {
        rho += n[i];
        jx += n[i] * g_c[i][0];
        jy += n[i] * g_c[i][1];
        jz += n[i] * g_c[i][2];
    }
    double j[3] = {jx + 0.5 * f[0], jy + 0.5 * f[1], jz + 0.5 * f[2]};
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};

    double neq[Q], nneq[Q];
    if (P->equilibrium == 1)
        exp_equilibrium(rho, u, neq);
    else
        equilibrium(rho, u, neq);
    for (int i = 0; i < Q; i++) nneq[i] = n[i] - neq[i];

    double m[Q];
    for (int k = 0; k < Q; k++) {
        double s = 0.0;
        for (int i = 0; i < Q; i++) s += g_e[k][i] * nneq[i];
        m[k] = s;
    }
    double mu = P->kT / CS2;
    double rho_noise = P->noise_rho0 ? P->rho0 : rho;
    for (int k = 0; k < Q; k++) {
        double gk = gamma_of(P, k);
        double ms = gk * m[k];
        if (k >= 4 && r && P->kT > 0.0) {
            double phi = sqrt(1.0 - gk * gk);
            ms += phi * sqrt(g_w[k] * mu * rho_noise) * r[k - 4];
        }
        m[k] = ms;
    }
    /* Sigma of Eq. (moment_two_external_force) */
    double uf = u[0] * f[0] + u[1] * f[1] + u[2] * f[2];
    double Sig[3][3];
    for (int a = 0; a < 3; a++) {
        for (int b = 0; b < 3; b++) {
            double d = (a == b) ? 1.0 : 0.0;
            Sig[a][b] = 0.5 * (1.0 + P->gamma_shear) * (u[a] * f[b] + u[b] * f[a] - (2.0 / 3.0) * uf * d)
                      + (1.0 / 3.0) * (1.0 + P->gamma_bulk) * uf * d;
        }
    }
    for (int i = 0; i < Q; i++) {
        double s = 0.0;
        for (int k = 0; k < Q; k++) s += g_e[k][i] * m[k] / g_w[k];
        double fc = f[0] * g_c[i][0] + f[1] * g_c[i][1] + f[2] * g_c[i][2];
        double sc = 0.0;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                sc += Sig[a][b] * (g_c[i][a] * g_c[i][b] - CS2 * ((a == b) ? 1.0 : 0.0));
        double dforce = g_a[i] * (fc / CS2 + sc / (2.0 * CS2 * CS2));
        nstar[i] = neq[i] + g_a[i] * s + dforce;
    }
}

/* One LB step over the whole box: dst(r) = C[ S src ](r).  Solid nodes are
 * copied unchanged.  force: optional [3][N] field added to body_force. */
void ora_step(const ora_params *P, const double *src, double *dst, const double *force, uint32_t step)
{
    build_tables();
    size_t N = nodes_of(P);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; z++) {
        for (int y = 0; y < P->ny; y++) {
            for (int x = 0; x < P->nx; x++) {
                size_t s = lin(P, x, y, z);
                if (is_solid(P, z)) {
                    for (int i = 0; i < Q; i++) dst[(size_t)i * N + s] = src[(size_t)i * N + s];
                    continue;
                }
                double n[Q], ns[Q], f[3], g[16];
                gather(P, src, x, y, z, n);
                node_force(P, force, s, f);
                const double *r = NULL;
                if (P->kT > 0.0) {
                    ora_gaussians(P->seed, (uint32_t)s, step, 0u, P->replica, 4, g);
                    r = g;
                }
                collide(P, n, f, r, ns);
                for (int i = 0; i < Q; i++) dst[(size_t)i * N + s] = ns[i];
            }
        }
    }
}

/* Hydrodynamic moments of the pre-collision state (Eqs. hmodes_beg..hmodes_end
 * written directly as sums over populations): rho = sum n, j = sum n c + f/2,
 * pi_ab = sum n c_a c_b, components (xx, yy, zz, xy, yz, zx).  Layouts [N],
 * [3][N], [6][N]; any output may be NULL.  Solid nodes get rho = rho0 and
 * zero j, pi. */
void ora_moments(const ora_params *P, const double *pops, const double *force,
                 double *rho, double *j, double *pi)
{
    build_tables();
    size_t N = nodes_of(P);
    const int ab[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {1, 2}, {2, 0}};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; z++) {
        for (int y = 0; y < P->ny; y++) {
            for (int x = 0; x < P->nx; x++) {
                size_t s = lin(P, x, y, z);
                if (is_solid(P, z)) {
                    if (rho) rho[s] = P->rho0;
                    if (j) for (int d = 0; d < 3; d++) j[(size_t)d * N + s] = 0.0;
                    if (pi) for (int c = 0; c < 6; c++) pi[(size_t)c * N + s] = 0.0;
                    continue;
                }
                double n[Q], f[3];
                gather(P, pops, x, y, z, n);
                node_force(P, force, s, f);
                double r = 0.0, jj[3] = {0, 0, 0}, pp[6] = {0, 0, 0, 0, 0, 0};
                for (int i = 0; i < Q; i++) {
                    r += n[i];
                    for (int d = 0; d < 3; d++) jj[d] += n[i] * g_c[i][d];
                    for (int c = 0; c < 6; c++) pp[c] += n[i] * g_c[i][ab[c][0]] * g_c[i][ab[c][1]];
                }
                if (rho) rho[s] = r;
                if (j) for (int d = 0; d < 3; d++) j[(size_t)d * N + s] = jj[d] + 0.5 * f[d];
                if (pi) for (int c = 0; c < 6; c++) pi[(size_t)c * N + s] = pp[c];
            }
        }
    }
}

/* All nineteen moments m_k = sum_i e_ki n_i (Eq. forward) of the
 * pre-collision populations, layout [19][N]; solid nodes give zeros. */
void ora_modes(const ora_params *P, const double *pops, double *m)
{
    build_tables();
    size_t N = nodes_of(P);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; z++) {
        for (int y = 0; y < P->ny; y++) {
            for (int x = 0; x < P->nx; x++) {
                size_t s = lin(P, x, y, z);
                double n[Q];
                if (is_solid(P, z)) {
                    for (int k = 0; k < Q; k++) m[(size_t)k * N + s] = 0.0;
                    continue;
                }
                gather(P, pops, x, y, z, n);
                for (int k = 0; k < Q; k++) {
                    double acc = 0.0;
                    for (int i = 0; i < Q; i++) acc += g_e[k][i] * n[i];
                    m[(size_t)k * N + s] = acc;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Point particles: Kremer-Grest forces (Sec. 2.1), force coupling           */
/* (Sec. 4.5), linear interpolation (Sec. 4.6)                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n_chains;      /* particles k*chain_len .. (k+1)*chain_len-1 form chain k */
    int chain_len;     /* 0 or 1: no bonds                                        */
    int use_wca;       /* purely repulsive LJ between all pairs                   */
    int pad_;
    double eps, sigma; /* WCA, Eq. (ulennardjones)                                */
    double k_fene, r0; /* FENE, Eq. (ufene)                                       */
} ora_md;

/* Minimum-image separation d = a - b along each periodic axis. */
static void min_image(const ora_params *P, const double *a, const double *b, double d[3])
{
    const int L[3] = {P->nx, P->ny, P->nz};
    for (int c = 0; c < 3; c++) {
        double v = a[c] - b[c];
        int periodic = (c < 2) || !P->walls;
        if (periodic) v -= L[c] * floor(v / L[c] + 0.5);
        d[c] = v;
    }
}

/* Conservative forces F^c = -dV/dr_i, brute force over all pairs.  Returns
 * the number of FENE bonds stretched to r >= R0 (their force is left out). */
int ora_md_forces(const ora_params *P, const ora_md *md, int np, const double *pos, double *F)
{
    int broken = 0;
    double rc2 = pow(2.0, 1.0 / 3.0) * md->sigma * md->sigma;  /* (2^{1/6} sigma)^2 */
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : broken)
    for (int i = 0; i < np; i++) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < np; j++) {
            if (j == i) continue;
            double d[3];
            min_image(P, pos + 3 * i, pos + 3 * j, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (md->use_wca && r2 < rc2) {
                /* V = 4 eps [(s/r)^12 - (s/r)^6 + 1/4];  F = -dV/dr * d/r */
                double sr2 = md->sigma * md->sigma / r2;
                double sr6 = sr2 * sr2 * sr2;
                double mag = 24.0 * md->eps * (2.0 * sr6 * sr6 - sr6) / r2;
                for (int c = 0; c < 3; c++) fi[c] += mag * d[c];
            }
            if (md->chain_len > 1) {
                int ci = i / md->chain_len, cj = j / md->chain_len;
                if (ci == cj && (j == i + 1 || j == i - 1)) {
                    /* V = -(k/2) R0^2 ln(1 - r^2/R0^2);  F = -k d / (1 - r^2/R0^2) */
                    double x = r2 / (md->r0 * md->r0);
                    if (x >= 1.0) {
                        broken++;
                    } else {
                        double mag = -md->k_fene / (1.0 - x);
                        for (int c = 0; c < 3; c++) fi[c] += mag * d[c];
                    }
                }
            }
        }
        for (int c = 0; c < 3; c++) F[3 * i + c] = fi[c];
    }
    return broken;
}

/* Fluid velocity at every node for the coupling: u = (sum n c + f_ext/2)/rho
 * from the pre-collision populations (Sec. 4.5: the coupling interpolates u,
 * not j; Sec. 3.7 for the half force).  Solid nodes: u = 0. */
static void node_velocity(const ora_params *P, const double *pops, const double *force, double *u)
{
    size_t N = nodes_of(P);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; z++) {
        for (int y = 0; y < P->ny; y++) {
            for (int x = 0; x < P->nx; x++) {
                size_t s = lin(P, x, y, z);
                if (is_solid(P, z)) {
                    u[3 * s] = u[3 * s + 1] = u[3 * s + 2] = 0.0;
                    continue;
                }
                double n[Q], f[3];
                gather(P, pops, x, y, z, n);
                node_force(P, force, s, f);
                double rho = 0.0, j[3] = {0, 0, 0};
                for (int i = 0; i < Q; i++) {
                    rho += n[i];
                    for (int d = 0; d < 3; d++) j[d] += n[i] * g_c[i][d];
                }
                for (int d = 0; d < 3; d++) u[3 * s + d] = (j[d] + 0.5 * f[d]) / rho;
            }
        }
    }
}

/* phi_2, Eq. (2point). */
static double phi2(double v)
{
    double a = fabs(v);
    return a <= 1.0 ? 1.0 - a : 0.0;
}

/* The eight nodes of the linear stencil around position p and their weights
 * Delta(r - p) = phi2(x) phi2(y) phi2(z) (Eqs. Delta, 2point). */
static void stencil(const ora_params *P, const double p[3], size_t node[8], double wt[8])
{
    int b[3];
    for (int c = 0; c < 3; c++) b[c] = (int)floor(p[c]);
    int q = 0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                int nxv = b[0] + dx, nyv = b[1] + dy, nzv = b[2] + dz;
                double w = phi2(nxv - p[0]) * phi2(nyv - p[1]) * phi2(nzv - p[2]);
                nxv = wrap(nxv, P->nx);
                nyv = wrap(nyv, P->ny);
                nzv = P->walls ? nzv : wrap(nzv, P->nz);
                if (nzv < 0 || nzv >= P->nz) { nzv = 0; w = 0.0; }
                node[q] = lin(P, nxv, nyv, nzv);
                wt[q] = w;
                q++;
            }
}

/* phi_3, Eq. (3point): three nodes, moment conditions C1-C3, continuous
 * first derivative. */
static double phi3(double v)
{
    double a = fabs(v);
    if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * v * v)) / 3.0;
    if (a <= 1.5) return (5.0 - 3.0 * a - sqrt(-2.0 + 6.0 * a - 3.0 * v * v)) / 6.0;
    return 0.0;
}

/* phi_4, Eq. (4point): four nodes. */
static double phi4(double v)
{
    double a = fabs(v);
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * v * v)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * v * v)) / 8.0;
    return 0.0;
}

/* Nodes per axis of interpolation function kern (2, 3, 4) and the first of
 * them for coordinate p: every node with phi(j - p) > 0 lies in [j0, j0 + K). */
static int kernel_width(int kern) { return kern == 3 ? 3 : (kern == 4 ? 4 : 2); }

static int kernel_first(int kern, double p)
{
    if (kern == 3) return (int)floor(p + 0.5) - 1;
    if (kern == 4) return (int)floor(p) - 1;
    return (int)floor(p);
}

static double phi_of(int kern, double v)
{
    if (kern == 3) return phi3(v);
    if (kern == 4) return phi4(v);
    return phi2(v);
}

/* The K^3 nodes of Delta (Eq. Delta) with phi_kern around position p and
 * their weights, x fastest; nodes outside the box (walls) get weight 0.
 * Returns K^3.  For kern 2 it is stencil() above. */
static int stencil_k(const ora_params *P, int kern, const double p[3], size_t *node, double *wt)
{
    const int K = kernel_width(kern);
    int b[3];
    for (int c = 0; c < 3; c++) b[c] = kernel_first(kern, p[c]);
    int q = 0;
    for (int dz = 0; dz < K; dz++)
        for (int dy = 0; dy < K; dy++)
            for (int dx = 0; dx < K; dx++) {
                int nxv = b[0] + dx, nyv = b[1] + dy, nzv = b[2] + dz;
                double w = phi_of(kern, nxv - p[0]) * phi_of(kern, nyv - p[1]) * phi_of(kern, nzv - p[2]);
                nxv = wrap(nxv, P->nx);
                nyv = wrap(nyv, P->ny);
                nzv = P->walls ? nzv : wrap(nzv, P->nz);
                if (nzv < 0 || nzv >= P->nz) { nzv = 0; w = 0.0; }
                node[q] = lin(P, nxv, nyv, nzv);
                wt[q] = w;
                q++;
            }
    return q;
}

/* Put a position back into the box: periodic wrap in x, y (and z without
 * walls); with walls, specular reflection keeps z in [b, nz-1-b], b = K/2 for
 * a stencil K nodes wide, so that the stencil touches fluid nodes only (a
 * project reading; b = 1 for phi_2). */
static void confine_band(const ora_params *P, double band, double p[3], double m[3])
{
    const int L[3] = {P->nx, P->ny, P->nz};
    for (int c = 0; c < 3; c++) {
        if (c == 2 && P->walls) {
            double lo = band, hi = (double)(P->nz - 1) - band;
            if (p[2] < lo) { p[2] = 2.0 * lo - p[2]; m[2] = -m[2]; }
            if (p[2] > hi) { p[2] = 2.0 * hi - p[2]; m[2] = -m[2]; }
        } else {
            p[c] -= L[c] * floor(p[c] / L[c]);
            if (p[c] >= L[c]) p[c] -= L[c];
        }
    }
}

static void confine(const ora_params *P, double p[3], double m[3]) { confine_band(P, 1.0, p, m); }

typedef struct {
    int n_substeps;
    int noise_kind;     /* 0: Gaussian theta; 1: three-point theta in {0, +-sqrt3} */
    double dt;          /* particle time step in lattice units (h = 1 per LB step) */
    uint64_t seed;      /* particle noise key                                      */
    uint32_t md_step0;  /* global index of the first sub-step (noise counter)      */
    uint32_t kernel;    /* interpolation function phi_2 (0 or 2), phi_3, phi_4     */
    double fext[3];     /* constant external force on every particle, part of F^c  */
} ora_couple_params;

/* Particle noise theta (3 components) for particle p at sub-step t:
 * Philox domain 1, one block; Gaussian via Box-Muller, or the three-point
 * distribution of Sec. 4.5 decided on the exact integer behind the uniform. */
static void particle_theta(const ora_params *P, const ora_couple_params *C, uint32_t p,
                           uint32_t t, double th[3])
{
    if (C->noise_kind == 1) {
        uint32_t raw[4];
        ora_raw16(C->seed, p, t, 1u, P->replica, 1, raw);
        const double s3 = sqrt(3.0);
        for (int c = 0; c < 3; c++) {
            uint64_t k = 2ull * (raw[c] >> 9) + 1ull;  /* uniform = k / 2^24 */
            if (6ull * k < (1ull << 24)) th[c] = -s3;          /* v < 1/6  */
            else if (6ull * k > 5ull * (1ull << 24)) th[c] = s3; /* v > 5/6 */
            else th[c] = 0.0;
        }
    } else {
        double g[4];
        ora_gaussians(C->seed, p, t, 1u, P->replica, 1, g);
        th[0] = g[0]; th[1] = g[1]; th[2] = g[2];
    }
}

/* Frictional coupling for one LB step (Sec. 4.5, "Langevin integrator"):
 * the fluid velocity field is frozen for the n_substeps particle steps; per
 * sub-step: half drift, conservative forces, exact Ornstein-Uhlenbeck
 * momentum update (Eq. langevin_momentum_update), spreading of the impulse
 * of the drag and random forces over the sub-step as -J Delta(r - r_half)
 * into facc (layout [3][N]), Eq. (ftotal): F^c is constant during the
 * momentum update (constant coordinates), so J = p' - p - h F^c; then the
 * second half drift.  mass/gamma: per-particle.
 * Returns the number of broken FENE bonds met. */
int ora_couple(const ora_params *P, const double *pops, const double *force, int np,
               double *pos, double *mom, const double *mass, const double *gamma,
               const ora_md *md, const ora_couple_params *C, double *facc)
{
    build_tables();
    size_t N = nodes_of(P);
    double *u = (double *)malloc(sizeof(double) * 3 * N);
    double *fc = (double *)calloc((size_t)3 * (np > 0 ? np : 1), sizeof(double));
    node_velocity(P, pops, force, u);
    int broken = 0;
    double h = C->dt;
    for (int s = 0; s < C->n_substeps; s++) {
        for (int p = 0; p < np; p++) {
            for (int c = 0; c < 3; c++) pos[3 * p + c] += 0.5 * h * mom[3 * p + c] / mass[p];
            confine_band(P, 0.5 * kernel_width((int)C->kernel), pos + 3 * p, mom + 3 * p);
        }
        if (md) broken += ora_md_forces(P, md, np, pos, fc);
        for (int p = 0; p < np; p++) {
            double m = mass[p], G = gamma[p];
            double C1 = exp(-G * h / m);
            double C2 = (m / G) * (1.0 - C1);
            double C3 = sqrt(m * P->kT * (1.0 - exp(-2.0 * G * h / m)));
            size_t node[64];
            double wt[64];
            const int nq = stencil_k(P, (int)C->kernel, pos + 3 * p, node, wt);
            double up[3] = {0.0, 0.0, 0.0};
            for (int q = 0; q < nq; q++)
                for (int c = 0; c < 3; c++) up[c] += wt[q] * u[3 * node[q] + c];
            double th[3] = {0.0, 0.0, 0.0};
            if (P->kT > 0.0) particle_theta(P, C, (uint32_t)p, C->md_step0 + (uint32_t)s, th);
            double pn[3], J[3];
            for (int c = 0; c < 3; c++) {
                double Fc = (md ? fc[3 * p + c] : 0.0) + C->fext[c];
                pn[c] = C1 * mom[3 * p + c] + C2 * (Fc + G * up[c]) + C3 * th[c];
                J[c] = pn[c] - mom[3 * p + c] - h * Fc;
            }
            for (int q = 0; q < nq; q++)
                for (int c = 0; c < 3; c++) facc[(size_t)c * N + node[q]] -= J[c] * wt[q];
            for (int c = 0; c < 3; c++) mom[3 * p + c] = pn[c];
        }
        for (int p = 0; p < np; p++) {
            for (int c = 0; c < 3; c++) pos[3 * p + c] += 0.5 * h * mom[3 * p + c] / mass[p];
            confine_band(P, 0.5 * kernel_width((int)C->kernel), pos + 3 * p, mom + 3 * p);
        }
    }
    free(u);
    free(fc);
    return broken;
}

/* Interpolated fluid velocity at arbitrary positions (Eq. ufluid_discrete)
 * with interpolation function phi_kern. */
void ora_interpolate_k(const ora_params *P, int kern, const double *pops, const double *force, int np,
                       const double *pos, double *up)
{
    build_tables();
    size_t N = nodes_of(P);
    double *u = (double *)malloc(sizeof(double) * 3 * N);
    node_velocity(P, pops, force, u);
    for (int p = 0; p < np; p++) {
        size_t node[64];
        double wt[64], pp[3] = {pos[3 * p], pos[3 * p + 1], pos[3 * p + 2]};
        const int nq = stencil_k(P, kern, pp, node, wt);
        for (int c = 0; c < 3; c++) {
            double acc = 0.0;
            for (int q = 0; q < nq; q++) acc += wt[q] * u[3 * node[q] + c];
            up[3 * p + c] = acc;
        }
    }
    free(u);
}

void ora_interpolate(const ora_params *P, const double *pops, const double *force, int np,
                     const double *pos, double *up)
{
    ora_interpolate_k(P, 2, pops, force, np, pos, up);
}

/* Stencil export for the interpolation-kernel tests: K^3 nodes and weights. */
int ora_stencil_k(const ora_params *P, int kern, const double *p, long long *node, double *wt)
{
    size_t nd[64];
    const int nq = stencil_k(P, kern, p, nd, wt);
    for (int q = 0; q < nq; q++) node[q] = (long long)nd[q];
    return nq;
}

void ora_stencil(const ora_params *P, const double *p, long long *node, double *wt)
{
    ora_stencil_k(P, 2, p, node, wt);
}

/* phi_kern(v) itself, for the moment-condition tests. */
double ora_phi(int kern, double v) { return phi_of(kern, v); }

/* ------------------------------------------------------------------------ */
/* Reverse mode (kT = 0): a hand-derived adjoint of one stream-collide step  */
/* in population space, following the oracle's own formulation above:       */
/*   n* = n^eq(rho, u) + a_i sum_k e_ki gamma_k m^neq_k / w_k + Delta''(u, f) */
/* with m^neq = E (n - n^eq), rho = sum n, u = (sum n c + f/2)/rho.          */
/* ------------------------------------------------------------------------ */

/* d n^eq_i / d u_alpha at fixed rho, from Eq. (original_equil_distrib). */
static double dneq_du(int i, double rho, const double u[3], int al)
{
    double cu = u[0] * g_c[i][0] + u[1] * g_c[i][1] + u[2] * g_c[i][2];
    return g_a[i] * rho * (g_c[i][al] / CS2 + cu * g_c[i][al] / (CS2 * CS2) - u[al] / CS2);
}

/* d Sigma_bg / d u_al and d Sigma_bg / d f_al of Eq. (moment_two_external_force). */
static double dsig_du(const ora_params *P, const double f[3], int al, int b, int g)
{
    double d_ab = (al == b), d_ag = (al == g), d_bg = (b == g);
    return 0.5 * (1.0 + P->gamma_shear) * (d_ab * f[g] + d_ag * f[b] - (2.0 / 3.0) * f[al] * d_bg)
         + (1.0 / 3.0) * (1.0 + P->gamma_bulk) * f[al] * d_bg;
}

static double dsig_df(const ora_params *P, const double u[3], int al, int b, int g)
{
    double d_ab = (al == b), d_ag = (al == g), d_bg = (b == g);
    return 0.5 * (1.0 + P->gamma_shear) * (u[b] * d_ag + u[g] * d_ab - (2.0 / 3.0) * u[al] * d_bg)
         + (1.0 / 3.0) * (1.0 + P->gamma_bulk) * u[al] * d_bg;
}

/* Adjoint of collide() at one node: given lam = dL/dn*, returns dn = dL/dn
 * and adds dL/df to df. */
static void collide_adjoint(const ora_params *P, const double n[Q], const double f[3], const double lam[Q],
                            double dn[Q], double df[3])
{
    double rho = 0.0, J[3] = {0, 0, 0};
    for (int i = 0; i < Q; i++) {
        rho += n[i];
        for (int d = 0; d < 3; d++) J[d] += n[i] * g_c[i][d];
    }
    double u[3] = {(J[0] + 0.5 * f[0]) / rho, (J[1] + 0.5 * f[1]) / rho, (J[2] + 0.5 * f[2]) / rho};
    double neq[Q];
    equilibrium(rho, u, neq);
    /* through the back transform and the relaxation: mu_k = gamma_k sum_i lam_i a_i e_ki / w_k */
    double mu[Q];
    for (int k = 0; k < Q; k++) {
        double s = 0.0;
        for (int i = 0; i < Q; i++) s += lam[i] * g_a[i] * g_e[k][i];
        mu[k] = gamma_of(P, k) * s / g_w[k];
    }
    /* m^neq = E (n - n^eq): direct part g_i = sum_k e_ki mu_k, and dL/dn^eq = lam - g */
    double gvec[Q], leq[Q];
    for (int i = 0; i < Q; i++) {
        double s = 0.0;
        for (int k = 0; k < Q; k++) s += g_e[k][i] * mu[k];
        gvec[i] = s;
        leq[i] = lam[i] - s;
    }
    /* n^eq(rho, u) and Delta''(u, f) */
    double rbar = 0.0, ubar[3] = {0, 0, 0}, fbar[3] = {0, 0, 0};
    for (int i = 0; i < Q; i++) {
        rbar += leq[i] * neq[i] / rho;
        for (int al = 0; al < 3; al++) ubar[al] += leq[i] * dneq_du(i, rho, u, al);
    }
    for (int i = 0; i < Q; i++) {
        for (int al = 0; al < 3; al++) {
            double su = 0.0, sf = 0.0;
            for (int b = 0; b < 3; b++)
                for (int g = 0; g < 3; g++) {
                    double proj = g_c[i][b] * g_c[i][g] - CS2 * (b == g);
                    su += dsig_du(P, f, al, b, g) * proj;
                    sf += dsig_df(P, u, al, b, g) * proj;
                }
            ubar[al] += lam[i] * g_a[i] * su / (2.0 * CS2 * CS2);
            fbar[al] += lam[i] * g_a[i] * (g_c[i][al] / CS2 + sf / (2.0 * CS2 * CS2));
        }
    }
    /* rho = sum n, u = (sum n c + f/2) / rho */
    for (int i = 0; i < Q; i++) {
        double s = gvec[i] + rbar;
        for (int al = 0; al < 3; al++) s += ubar[al] * (g_c[i][al] - u[al]) / rho;
        dn[i] = s;
    }
    for (int al = 0; al < 3; al++) df[al] += fbar[al] + ubar[al] / (2.0 * rho);
}

/* Reverse of the pull: n_i(r) came from n*_i(r - c_i), or from n*_opp(i)(r)
 * when the source is solid; the adjoint of n_i(r) goes back to that entry. */
static void push_adjoint(const ora_params *P, double *lam_out, int x, int y, int z, const double dn[Q])
{
    size_t N = nodes_of(P);
    for (int i = 0; i < Q; i++) {
        int sx = wrap(x - g_c[i][0], P->nx);
        int sy = wrap(y - g_c[i][1], P->ny);
        int sz = z - g_c[i][2];
        if (P->walls) {
            if (sz < 0 || sz >= P->nz || is_solid(P, sz)) {
                lam_out[(size_t)g_opp[i] * N + lin(P, x, y, z)] += dn[i];
                continue;
            }
        } else {
            sz = wrap(sz, P->nz);
        }
        lam_out[(size_t)i * N + lin(P, sx, sy, sz)] += dn[i];
    }
}

/* lam_out = dL/dn*(t) from lam_in = dL/dn*(t+1) for the step that maps the
 * stored state `state` (at t) to t+1; adds dL/df into grad_f ([3][N]).
 * Requires kT = 0.  lam_out is overwritten. */
void ora_adjoint_step(const ora_params *P, const double *state, const double *force, const double *lam_in,
                      double *lam_out, double *grad_f)
{
    build_tables();
    size_t N = nodes_of(P);
    memset(lam_out, 0, sizeof(double) * Q * N);
    for (int z = 0; z < P->nz; z++) {
        if (is_solid(P, z)) continue;
        for (int y = 0; y < P->ny; y++) {
            for (int x = 0; x < P->nx; x++) {
                size_t s = lin(P, x, y, z);
                double n[Q], f[3], lam[Q], dn[Q], df[3] = {0, 0, 0};
                gather(P, state, x, y, z, n);
                node_force(P, force, s, f);
                for (int i = 0; i < Q; i++) lam[i] = lam_in[(size_t)i * N + s];
                collide_adjoint(P, n, f, lam, dn, df);
                push_adjoint(P, lam_out, x, y, z, dn);
                if (grad_f) for (int d = 0; d < 3; d++) grad_f[(size_t)d * N + s] += df[d];
            }
        }
    }
}

/* L = 1/2 sum over fluid nodes in [lo, hi) of |j|^2 / rho with j = sum n c + f/2
 * of the pre-collision state pulled from `state`; writes lam_out = dL/dstate,
 * adds dL/df into grad_f, returns L. */
double ora_kinetic_seed(const ora_params *P, const double *state, const double *force, const int lo[3],
                        const int hi[3], double *lam_out, double *grad_f)
{
    build_tables();
    size_t N = nodes_of(P);
    memset(lam_out, 0, sizeof(double) * Q * N);
    double L = 0.0;
    for (int z = lo[2]; z < hi[2]; z++) {
        if (is_solid(P, z)) continue;
        for (int y = lo[1]; y < hi[1]; y++) {
            for (int x = lo[0]; x < hi[0]; x++) {
                size_t s = lin(P, x, y, z);
                double n[Q], f[3], dn[Q];
                gather(P, state, x, y, z, n);
                node_force(P, force, s, f);
                double rho = 0.0, j[3] = {0, 0, 0};
                for (int i = 0; i < Q; i++) {
                    rho += n[i];
                    for (int d = 0; d < 3; d++) j[d] += n[i] * g_c[i][d];
                }
                for (int d = 0; d < 3; d++) j[d] += 0.5 * f[d];
                double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
                double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                L += 0.5 * (j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / rho;
                for (int i = 0; i < Q; i++)
                    dn[i] = u[0] * g_c[i][0] + u[1] * g_c[i][1] + u[2] * g_c[i][2] - 0.5 * u2;
                push_adjoint(P, lam_out, x, y, z, dn);
                if (grad_f) for (int d = 0; d < 3; d++) grad_f[(size_t)d * N + s] += 0.5 * u[d];
            }
        }
    }
    return L;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode of the coupling (kT = 0, free particles: no conservative    */
/* forces).  Each particle is then independent: replay its sub-steps of     */
/* ora_couple, then walk them back.  Per sub-step (Sec. 4.5), with          */
/* a = dt / (2 m):                                                          */
/*   r_h = confine(r + a p)             (a z reflection flips r_z and p_z)   */
/*   u_p = sum_q w_q(r_h) u_q           (Eqs. Delta, 2point)                 */
/*   p'  = C1 p~ + C2 Gamma u_p         (p~ = p after the confine)           */
/*   J   = p' - p~;  facc_q -= J w_q(r_h)                                    */
/*   r'  = confine(r_h + a p')                                               */
/* and u_q = (sum_i n_i c_i + f_q / 2) / rho_q from the pulled populations. */
/* ------------------------------------------------------------------------ */

/* Weight of stencil node (dx, dy, dz) of position p and its gradient in p:
 * w = prod_d phi2, d phi2 / d p_d = -1 for the lower node, +1 for the upper
 * (one-sided at integer positions, consistent with the floor). */
static double stencil_grad(const double p[3], int dx, int dy, int dz, double g[3])
{
    const int o[3] = {dx, dy, dz};
    double ph[3], dph[3];
    for (int c = 0; c < 3; c++) {
        double fr = p[c] - floor(p[c]);
        ph[c] = o[c] ? fr : 1.0 - fr;
        dph[c] = o[c] ? 1.0 : -1.0;
    }
    g[0] = dph[0] * ph[1] * ph[2];
    g[1] = ph[0] * dph[1] * ph[2];
    g[2] = ph[0] * ph[1] * dph[2];
    return ph[0] * ph[1] * ph[2];
}

/* confine() with the sign it applied to z (+1, or -1 after a reflection). */
static double confine_sign(const ora_params *P, double p[3], double m[3])
{
    double before = m[2];
    confine(P, p, m);
    return (before != 0.0 && m[2] == -before) ? -1.0 : 1.0;
}

/* Given the state at the start of a coupling call (pos0, mom0), the
 * populations and force field of the step, lam_facc = dL/dfacc ([3][N]) and
 * lam_pos / lam_mom = dL/d(particle state after the call) ([np][3]): replace
 * lam_pos / lam_mom by dL/d(state at the start), add dL/dpops through the
 * interpolated u into lam_pops ([Q][N]) and dL/dforce through u's f/2 term
 * into grad_f ([3][N]).  Requires kT = 0 and no conservative forces.
 * Returns -1 (nothing done) if a z reflection happened with p_z = 0, where
 * the reflection sign cannot be recovered, else 0. */
int ora_couple_adjoint(const ora_params *P, const double *pops, const double *force, int np,
                       const double *pos0, const double *mom0, const double *mass, const double *gamma,
                       const ora_couple_params *C, const double *lam_facc, double *lam_pos, double *lam_mom,
                       double *lam_pops, double *grad_f)
{
    build_tables();
    size_t N = nodes_of(P);
    double *u = (double *)malloc(sizeof(double) * 3 * N);
    double *lam_u = (double *)calloc(3 * N, sizeof(double));
    node_velocity(P, pops, force, u);
    const int S = C->n_substeps;
    const double h = C->dt;
    double *rh = (double *)malloc(sizeof(double) * 3 * S);   /* r_h of each sub-step */
    double *pt = (double *)malloc(sizeof(double) * 3 * S);   /* p~ */
    double *pn = (double *)malloc(sizeof(double) * 3 * S);   /* p' */
    double *s1 = (double *)malloc(sizeof(double) * S);       /* z sign of the first confine */
    double *s2 = (double *)malloc(sizeof(double) * S);       /* z sign of the second */
    int status = 0;
    for (int p = 0; p < np; p++) {
        const double m = mass[p], G = gamma[p], a = 0.5 * h / m;
        const double C1 = exp(-G * h / m), C2 = (m / G) * (1.0 - C1);
        double r[3], q[3];
        for (int c = 0; c < 3; c++) { r[c] = pos0[3 * p + c]; q[c] = mom0[3 * p + c]; }
        /* replay */
        for (int s = 0; s < S; s++) {
            for (int c = 0; c < 3; c++) r[c] += a * q[c];
            if (P->walls && q[2] == 0.0 && (r[2] < 1.0 || r[2] > P->nz - 2)) status = -1;
            s1[s] = P->walls ? confine_sign(P, r, q) : (confine(P, r, q), 1.0);
            size_t node[8];
            double wt[8], up[3] = {0, 0, 0};
            stencil(P, r, node, wt);
            for (int k = 0; k < 8; k++)
                for (int c = 0; c < 3; c++) up[c] += wt[k] * u[3 * node[k] + c];
            for (int c = 0; c < 3; c++) {
                rh[3 * s + c] = r[c];
                pt[3 * s + c] = q[c];
                q[c] = C1 * q[c] + C2 * G * up[c];
                pn[3 * s + c] = q[c];
                r[c] += a * q[c];
            }
            if (P->walls && q[2] == 0.0 && (r[2] < 1.0 || r[2] > P->nz - 2)) status = -1;
            s2[s] = P->walls ? confine_sign(P, r, q) : (confine(P, r, q), 1.0);
        }
        /* walk back */
        double lr[3], lp[3];
        for (int c = 0; c < 3; c++) { lr[c] = lam_pos[3 * p + c]; lp[c] = lam_mom[3 * p + c]; }
        for (int s = S - 1; s >= 0; s--) {
            const double *r_h = rh + 3 * s, *p_t = pt + 3 * s, *p_n = pn + 3 * s;
            /* second half drift + confine: r' = sz (r_h + a p'), p_stored = sz p' (z only) */
            double lrh[3], lpn[3];
            for (int c = 0; c < 3; c++) {
                double sg = (c == 2) ? s2[s] : 1.0;
                lrh[c] = sg * lr[c];
                lpn[c] = sg * (lp[c] + a * lr[c]);
            }
            /* spread facc_q -= J w_q and the update p' = C1 p~ + C2 G u_p */
            double J[3], lJ[3] = {0, 0, 0}, lu[3];
            for (int c = 0; c < 3; c++) J[c] = p_n[c] - p_t[c];
            size_t node[8];
            double wt[8];
            stencil(P, r_h, node, wt);
            int k = 0;
            for (int dz = 0; dz < 2; dz++)
                for (int dy = 0; dy < 2; dy++)
                    for (int dx = 0; dx < 2; dx++, k++) {
                        if (wt[k] == 0.0 && P->walls) {
                            /* a node outside the box: no weight, no gradient */
                            int nzv = (int)floor(r_h[2]) + dz;
                            if (nzv < 0 || nzv >= P->nz) continue;
                        }
                        double gw[3];
                        stencil_grad(r_h, dx, dy, dz, gw);
                        double lf_dot_J = 0.0;
                        for (int c = 0; c < 3; c++) {
                            double lf = lam_facc[(size_t)c * N + node[k]];
                            lJ[c] -= lf * wt[k];
                            lf_dot_J += lf * J[c];
                        }
                        for (int c = 0; c < 3; c++) lrh[c] -= lf_dot_J * gw[c];
                    }
            double lpt[3];
            for (int c = 0; c < 3; c++) {
                lpn[c] += lJ[c];
                lpt[c] = -lJ[c] + C1 * lpn[c];
                lu[c] = C2 * G * lpn[c];
            }
            /* u_p = sum_q w_q u_q */
            k = 0;
            for (int dz = 0; dz < 2; dz++)
                for (int dy = 0; dy < 2; dy++)
                    for (int dx = 0; dx < 2; dx++, k++) {
                        if (P->walls) {
                            int nzv = (int)floor(r_h[2]) + dz;
                            if (nzv < 0 || nzv >= P->nz) continue;
                        }
                        double gw[3];
                        stencil_grad(r_h, dx, dy, dz, gw);
                        double udot = 0.0;
                        for (int c = 0; c < 3; c++) {
                            lam_u[3 * node[k] + c] += wt[k] * lu[c];
                            udot += u[3 * node[k] + c] * lu[c];
                        }
                        for (int c = 0; c < 3; c++) lrh[c] += udot * gw[c];
                    }
            /* first half drift + confine: r_h = sz (r + a p), p~ = sz p */
            for (int c = 0; c < 3; c++) {
                double sg = (c == 2) ? s1[s] : 1.0;
                lr[c] = sg * lrh[c];
                lp[c] = sg * (lpt[c] + a * lrh[c]);
            }
        }
        for (int c = 0; c < 3; c++) { lam_pos[3 * p + c] = lr[c]; lam_mom[3 * p + c] = lp[c]; }
    }
    /* lam_u -> populations (through the pull) and force field */
    for (int z = 0; z < P->nz; z++) {
        if (is_solid(P, z)) continue;
        for (int y = 0; y < P->ny; y++)
            for (int x = 0; x < P->nx; x++) {
                size_t s = lin(P, x, y, z);
                const double *lu = lam_u + 3 * s;
                if (lu[0] == 0.0 && lu[1] == 0.0 && lu[2] == 0.0) continue;
                double n[Q], dn[Q], rho = 0.0;
                gather(P, pops, x, y, z, n);
                for (int i = 0; i < Q; i++) rho += n[i];
                const double *us = u + 3 * s;
                for (int i = 0; i < Q; i++) {
                    double v = 0.0;
                    for (int d = 0; d < 3; d++) v += lu[d] * (g_c[i][d] - us[d]);
                    dn[i] = v / rho;
                }
                push_adjoint(P, lam_pops, x, y, z, dn);
                if (grad_f)
                    for (int d = 0; d < 3; d++) grad_f[(size_t)d * N + s] += 0.5 * lu[d] / rho;
            }
    }
    free(u); free(lam_u); free(rh); free(pt); free(pn); free(s1); free(s2);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Extended particles: solid spheres with moving link bounce-back            */
/* (Sec. 4.1, Eqs. MBB, NodeVel; Sec. 4.2, Eqs. EOMD-1..3, force, force0,    */
/* zeta, EOMUsol and the consistency equation for the velocity U~)           */
/*                                                                           */
/* Readings (the paper leaves them open): spheres translate without          */
/* rotating (Sec. 4.2 treats the linear velocity; Omega = 0, so u_b = U); a  */
/* node is solid when its distance from the centre is below the radius a     */
/* (minimum image, periodic box, no walls); rho in Eqs. MBB and zeta is      */
/* rho0; the velocity update of Eq. EOMUsol is applied in the eigenbasis of  */
/* the symmetric matrix zeta (the exact solution of m dU/dt = -zeta U + F);  */
/* a node covered by a moving sphere gives its fluid momentum sum n c to the */
/* sphere, a node it uncovers starts from n^eq(rho0, U) and the sphere loses */
/* rho0 U, so total momentum is conserved; spheres must stay apart (a node   */
/* never passes from one sphere to another).                                 */
/* ------------------------------------------------------------------------ */

static double periodic_offset(double d, int L) { return d - L * floor(d / L + 0.5); }

static void sphere_map(const ora_params *P, int np, const double *R, double a, int *owner)
{
    for (int z = 0; z < P->nz; z++)
        for (int y = 0; y < P->ny; y++)
            for (int x = 0; x < P->nx; x++) {
                int o = -1;
                for (int p = 0; p < np && o < 0; p++) {
                    double dx = periodic_offset(x - R[3 * p], P->nx);
                    double dy = periodic_offset(y - R[3 * p + 1], P->ny);
                    double dz = periodic_offset(z - R[3 * p + 2], P->nz);
                    if (dx * dx + dy * dy + dz * dz < a * a) o = p;
                }
                owner[lin(P, x, y, z)] = o;
            }
}

/* owner[s]: sphere p whose centre lies closer than a to node s, or -1. */
void ora_sphere_owner(const ora_params *P, int np, const double *R, double a, int *owner)
{
    build_tables();
    sphere_map(P, np, R, a, owner);
}

/* Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations:
 * A = V diag(w) V^T, V's columns the eigenvectors. */
static void jacobi3(const double Ain[3][3], double w[3], double V[3][3])
{
    double A[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            A[i][j] = Ain[i][j];
            V[i][j] = (i == j) ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 50; sweep++) {
        double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
        if (off == 0.0) break;
        for (int p = 0; p < 2; p++)
            for (int q = p + 1; q < 3; q++) {
                if (A[p][q] == 0.0) continue;
                double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; k++) {  /* A <- A J */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; k++) {  /* A <- J^T A */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; k++) {  /* V <- V J */
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < 3; i++) w[i] = A[i][i];
}

/* Eq. EOMUsol for m dU/dt = -zeta U + F over h = 1 with zeta, F constant,
 * and the velocity U~ of the consistency equation, per eigen-direction of
 * zeta (alpha = lambda / m): U' = e^-alpha U + (1 - e^-alpha) F / lambda,
 * alpha U~ = (1 - e^-alpha) U + (alpha - (1 - e^-alpha)) F / lambda.  A
 * direction without links (lambda = 0) takes the limits U' = U + F / m,
 * U~ = U + F / (2 m). */
void ora_sphere_velocity(const double zeta[9], double m, const double U[3], const double F[3], double Un[3],
                         double Ut[3])
{
    double Z[3][3], w[3], V[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Z[i][j] = zeta[3 * i + j];
    jacobi3(Z, w, V);
    double ue[3], fe[3];
    for (int k = 0; k < 3; k++) {
        ue[k] = V[0][k] * U[0] + V[1][k] * U[1] + V[2][k] * U[2];
        fe[k] = V[0][k] * F[0] + V[1][k] * F[1] + V[2][k] * F[2];
    }
    double une[3], ute[3];
    for (int k = 0; k < 3; k++) {
        double al = w[k] / m;
        if (al < 1e-12) {
            une[k] = ue[k] + fe[k] / m;
            ute[k] = ue[k] + 0.5 * fe[k] / m;
        } else {
            double e1 = -expm1(-al);  /* 1 - e^-alpha */
            une[k] = (1.0 - e1) * ue[k] + e1 * fe[k] / w[k];
            ute[k] = (e1 * ue[k] + (al - e1) * fe[k] / w[k]) / al;
        }
    }
    for (int i = 0; i < 3; i++) {
        Un[i] = V[i][0] * une[0] + V[i][1] * une[1] + V[i][2] * une[2];
        Ut[i] = V[i][0] * ute[0] + V[i][1] * ute[1] + V[i][2] * ute[2];
    }
}

/* Eigen-decomposition of a symmetric n x n matrix (n <= 6) by cyclic Jacobi
 * rotations: A = V diag(w) V^T. */
static void jacobi_n(int n, const double *Ain, double *w, double *V)
{
    double A[36];
    for (int i = 0; i < n * n; i++) A[i] = Ain[i];
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) off += fabs(A[p * n + q]);
        if (off == 0.0) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                if (A[p * n + q] == 0.0) continue;
                double th = (A[q * n + q] - A[p * n + p]) / (2.0 * A[p * n + q]);
                double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; k++) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - sn * akq;
                    A[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - sn * aqk;
                    A[q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - sn * vkq;
                    V[k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; i++) w[i] = A[i * n + i];
}

/* Translation and rotation together: M dV/dt = -Z V + F for V = (U, Omega),
 * M = diag(m, m, m, I, I, I), Z the symmetric 6 x 6 friction matrix.  With
 * W = M^1/2 V and K = M^-1/2 Z M^-1/2 it is dW/dt = -K W + M^-1/2 F, solved
 * over h = 1 as Eq. EOMUsol and the U~ equation in K's eigenbasis (kappa the
 * eigenvalue, G the force component): W' = e^-kappa W + (1 - e^-kappa) G / kappa,
 * W~ = ((1 - e^-kappa) W + (kappa - (1 - e^-kappa)) G / kappa) / kappa. */
void ora_sphere_velocity6(const double Z[36], double m, double I, const double V[6], const double F[6],
                          double Vn[6], double Vt[6])
{
    double sq[6], K[36], w[6], E[36];
    for (int i = 0; i < 6; i++) sq[i] = sqrt(i < 3 ? m : I);
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) K[i * 6 + j] = Z[i * 6 + j] / (sq[i] * sq[j]);
    jacobi_n(6, K, w, E);
    double we[6], ge[6], wn[6], wt[6];
    for (int k = 0; k < 6; k++) {
        we[k] = 0.0;
        ge[k] = 0.0;
        for (int i = 0; i < 6; i++) {
            we[k] += E[i * 6 + k] * sq[i] * V[i];
            ge[k] += E[i * 6 + k] * F[i] / sq[i];
        }
        double ka = w[k];
        if (ka < 1e-12) {
            wn[k] = we[k] + ge[k];
            wt[k] = we[k] + 0.5 * ge[k];
        } else {
            double e1 = -expm1(-ka);
            wn[k] = (1.0 - e1) * we[k] + e1 * ge[k] / ka;
            wt[k] = (e1 * we[k] + (ka - e1) * ge[k] / ka) / ka;
        }
    }
    for (int i = 0; i < 6; i++) {
        double sn = 0.0, st = 0.0;
        for (int k = 0; k < 6; k++) {
            sn += E[i * 6 + k] * wn[k];
            st += E[i * 6 + k] * wt[k];
        }
        Vn[i] = sn / sq[i];
        Vt[i] = st / sq[i];
    }
}

static void cross3(const double a[3], const double b[3], double out[3])
{
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* One LB step with np spheres of radius a (h = 1, b = 1).  src: the
 * post-collision state n*(t); owner: the solid map of the previous step (or
 * of the initial placement), updated here; R, U: centres and velocities,
 * updated; Om: angular velocities [np][3], updated, or NULL for spheres that
 * do not rotate; mass[p] <= 0 holds sphere p fixed (U, Om, R unchanged,
 * U~ = U); the moment of inertia is 2/5 m a^2 (a uniform solid sphere);
 * fc: external forces F^c [np][3] or NULL; Ut_out: U~ [np][3] or NULL;
 * FT_out: the hydrodynamic force and torque of the step, F0 - Z V~ (the
 * momentum and its moment the links give the sphere) [np][6], or NULL.
 * rho_b below is the minimum-image offset from the half-step centre.
 *   1. R_half = R + U / 2                                  Eq. EOMD-1
 *   2. solid map at R_half; covered nodes give sum n c (and its moment about
 *      the centre) to their sphere, uncovered nodes get n^eq(rho0, u) with
 *      u = U + Om x rho (values at time t) and the sphere loses rho0 u
 *   3. boundary links (fluid r, r + c_b solid of sphere p), r_b = r + c_b/2:
 *      F0 = sum 2 n*_b c_b, T0 = sum 2 n*_b rho_b x c_b, and the friction
 *      (2 rho0 / c_s^2) sum a_b g g^T, g = (c_b, rho_b x c_b)   Eqs. force0, zeta
 *   4. U, Om at t + h and U~, Om~ from F0 + F^c, T0 and the friction
 *                                                          Eq. EOMUsol
 *   5. stream and collide the fluid nodes; a link whose source r - c_i is
 *      solid (sphere p) returns n_i(r) = n*_{-i}(r) + 2 a_i rho0 u_b.c_i / c_s^2,
 *      u_b = U~ + Om~ x rho_b at r_b = r - c_i/2     Eqs. MBB, NodeVel (c_b = -c_i)
 *      solid nodes keep their values
 *   6. R(t+h) = R_half + U(t+h) / 2                        Eq. EOMD-3
 * Returns 0, -1 when a node passes from one sphere to another, -2 with walls. */
int ora_step_spheres(const ora_params *P, const double *src, double *dst, const double *force, uint32_t step,
                     int *owner, int np, double a, double *R, double *U, double *Om, const double *mass,
                     const double *fc, double *Ut_out, double *FT_out)
{
    build_tables();
    if (P->walls) return -2;  /* spheres live in periodic boxes */
    size_t N = nodes_of(P);
    const int L[3] = {P->nx, P->ny, P->nz};
    const int n1 = np > 0 ? np : 1;
    double *cur = (double *)malloc(sizeof(double) * Q * N);
    memcpy(cur, src, sizeof(double) * Q * N);
    int *nown = (int *)malloc(sizeof(int) * N);
    double *Rh = (double *)malloc(sizeof(double) * 3 * n1);
    double *Vt = (double *)calloc((size_t)6 * n1, sizeof(double));
    double *F0 = (double *)calloc((size_t)6 * n1, sizeof(double));   /* force, torque */
    double *Z = (double *)calloc((size_t)36 * n1, sizeof(double));
    double *dP = (double *)calloc((size_t)6 * n1, sizeof(double));
    int status = 0;

    /* 1 */
    for (int p = 0; p < np; p++)
        for (int c = 0; c < 3; c++) {
            double v = R[3 * p + c] + (mass[p] > 0.0 ? 0.5 * U[3 * p + c] : 0.0);
            v -= L[c] * floor(v / L[c]);
            Rh[3 * p + c] = v;
        }
    /* 2 (new fluid takes the velocities at time t; the exchanges are applied after) */
    sphere_map(P, np, Rh, a, nown);
    for (int z = 0; z < P->nz; z++)
        for (int y = 0; y < P->ny; y++)
            for (int x = 0; x < P->nx; x++) {
                size_t s = lin(P, x, y, z);
                int o = owner[s], nn = nown[s];
                if (o == nn) continue;
                if (o >= 0 && nn >= 0) { status = -1; continue; }
                int p = nn >= 0 ? nn : o;
                const double rv[3] = {periodic_offset(x - Rh[3 * p], L[0]), periodic_offset(y - Rh[3 * p + 1], L[1]),
                                      periodic_offset(z - Rh[3 * p + 2], L[2])};
                double j[3] = {0.0, 0.0, 0.0}, mom[3];
                if (nn >= 0) {  /* covered: its fluid momentum goes to the sphere */
                    for (int c = 0; c < 3; c++)
                        for (int i = 0; i < Q; i++) j[c] += cur[(size_t)i * N + s] * g_c[i][c];
                } else {        /* uncovered: new fluid at the surface velocity */
                    double u[3] = {U[3 * p], U[3 * p + 1], U[3 * p + 2]}, ne[Q];
                    if (Om) {
                        double w[3];
                        cross3(Om + 3 * p, rv, w);
                        for (int c = 0; c < 3; c++) u[c] += w[c];
                    }
                    equilibrium(P->rho0, u, ne);
                    for (int i = 0; i < Q; i++) cur[(size_t)i * N + s] = ne[i];
                    for (int c = 0; c < 3; c++) j[c] = -P->rho0 * u[c];
                }
                cross3(rv, j, mom);
                for (int c = 0; c < 3; c++) {
                    dP[6 * p + c] += j[c];
                    dP[6 * p + 3 + c] += mom[c];
                }
            }
    for (int p = 0; p < np; p++)
        if (mass[p] > 0.0) {
            double I = 0.4 * mass[p] * a * a;
            for (int c = 0; c < 3; c++) {
                U[3 * p + c] += dP[6 * p + c] / mass[p];
                if (Om) Om[3 * p + c] += dP[6 * p + 3 + c] / I;
            }
        }
    memcpy(owner, nown, sizeof(int) * N);
    /* 3 */
    for (int z = 0; z < P->nz; z++)
        for (int y = 0; y < P->ny; y++)
            for (int x = 0; x < P->nx; x++) {
                size_t s = lin(P, x, y, z);
                if (owner[s] >= 0) continue;
                for (int i = 1; i < Q; i++) {
                    size_t t = lin(P, wrap(x + g_c[i][0], L[0]), wrap(y + g_c[i][1], L[1]),
                                   wrap(z + g_c[i][2], L[2]));
                    int p = owner[t];
                    if (p < 0) continue;
                    double nb = cur[(size_t)i * N + s], cb[3] = {g_c[i][0], g_c[i][1], g_c[i][2]};
                    double rb[3] = {periodic_offset(x + 0.5 * cb[0] - Rh[3 * p], L[0]),
                                    periodic_offset(y + 0.5 * cb[1] - Rh[3 * p + 1], L[1]),
                                    periodic_offset(z + 0.5 * cb[2] - Rh[3 * p + 2], L[2])};
                    double g[6];
                    g[0] = cb[0];
                    g[1] = cb[1];
                    g[2] = cb[2];
                    cross3(rb, cb, g + 3);
                    for (int c = 0; c < 6; c++) {
                        F0[6 * p + c] += 2.0 * nb * g[c];
                        for (int d = 0; d < 6; d++) Z[36 * p + 6 * c + d] += 2.0 * P->rho0 / CS2 * g_a[i] * g[c] * g[d];
                    }
                }
            }
    /* 4 */
    for (int p = 0; p < np; p++) {
        double Fp[6], Vn[6];
        for (int c = 0; c < 6; c++) Fp[c] = F0[6 * p + c] + ((fc && c < 3) ? fc[3 * p + c] : 0.0);
        if (mass[p] > 0.0) {
            if (Om) {
                double V[6] = {U[3 * p], U[3 * p + 1], U[3 * p + 2], Om[3 * p], Om[3 * p + 1], Om[3 * p + 2]};
                ora_sphere_velocity6(Z + 36 * p, mass[p], 0.4 * mass[p] * a * a, V, Fp, Vn, Vt + 6 * p);
                for (int c = 0; c < 3; c++) {
                    U[3 * p + c] = Vn[c];
                    Om[3 * p + c] = Vn[3 + c];
                }
            } else {
                double Z3[9];
                for (int c = 0; c < 3; c++)
                    for (int d = 0; d < 3; d++) Z3[3 * c + d] = Z[36 * p + 6 * c + d];
                ora_sphere_velocity(Z3, mass[p], U + 3 * p, Fp, Vn, Vt + 6 * p);
                for (int c = 0; c < 3; c++) U[3 * p + c] = Vn[c];
            }
        } else {
            for (int c = 0; c < 3; c++) {
                Vt[6 * p + c] = U[3 * p + c];
                Vt[6 * p + 3 + c] = Om ? Om[3 * p + c] : 0.0;
            }
        }
        if (Ut_out)
            for (int c = 0; c < 3; c++) Ut_out[3 * p + c] = Vt[6 * p + c];
        if (FT_out)
            for (int c = 0; c < 6; c++) {
                double zv = 0.0;
                for (int d = 0; d < 6; d++) zv += Z[36 * p + 6 * c + d] * Vt[6 * p + d];
                FT_out[6 * p + c] = F0[6 * p + c] - zv;
            }
    }
    /* 5 */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < P->nz; z++) {
        for (int y = 0; y < P->ny; y++) {
            for (int x = 0; x < P->nx; x++) {
                size_t s = lin(P, x, y, z);
                if (owner[s] >= 0) {
                    for (int i = 0; i < Q; i++) dst[(size_t)i * N + s] = cur[(size_t)i * N + s];
                    continue;
                }
                double n[Q], ns[Q], f[3], g[16];
                for (int i = 0; i < Q; i++) {
                    size_t t = lin(P, wrap(x - g_c[i][0], L[0]), wrap(y - g_c[i][1], L[1]),
                                   wrap(z - g_c[i][2], L[2]));
                    int p = owner[t];
                    if (p >= 0) {
                        const double *vt = Vt + 6 * p;
                        double ub[3] = {vt[0], vt[1], vt[2]};
                        if (Om) {
                            double rb[3] = {periodic_offset(x - 0.5 * g_c[i][0] - Rh[3 * p], L[0]),
                                            periodic_offset(y - 0.5 * g_c[i][1] - Rh[3 * p + 1], L[1]),
                                            periodic_offset(z - 0.5 * g_c[i][2] - Rh[3 * p + 2], L[2])}, w[3];
                            cross3(vt + 3, rb, w);
                            for (int c = 0; c < 3; c++) ub[c] += w[c];
                        }
                        double uc = ub[0] * g_c[i][0] + ub[1] * g_c[i][1] + ub[2] * g_c[i][2];
                        n[i] = cur[(size_t)g_opp[i] * N + s] + 2.0 * g_a[i] * P->rho0 * uc / CS2;
                    } else {
                        n[i] = cur[(size_t)i * N + t];
                    }
                }
                node_force(P, force, s, f);
                const double *r = NULL;
                if (P->kT > 0.0) {
                    ora_gaussians(P->seed, (uint32_t)s, step, 0u, P->replica, 4, g);
                    r = g;
                }
                collide(P, n, f, r, ns);
                for (int i = 0; i < Q; i++) dst[(size_t)i * N + s] = ns[i];
            }
        }
    }
    /* 6 */
    for (int p = 0; p < np; p++)
        for (int c = 0; c < 3; c++) {
            double v = Rh[3 * p + c] + (mass[p] > 0.0 ? 0.5 * U[3 * p + c] : 0.0);
            v -= L[c] * floor(v / L[c]);
            R[3 * p + c] = v;
        }
    free(cur); free(nown); free(Rh); free(Vt); free(F0); free(Z); free(dP);
    return status;
}

/* The step of ora_step restricted to the listed nodes (linear indices of
 * fluid nodes): the same pull, force and collision with the noise of the
 * node; out[k][19] receives the post-collision populations of node idx[k].
 * Lets a test check sampled nodes of a box too large to step whole. */
void ora_step_nodes(const ora_params *P, const double *src, const double *force, uint32_t step, int nsel,
                    const long long *idx, double *out)
{
    build_tables();
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nsel; k++) {
        size_t s = (size_t)idx[k];
        int x = (int)(s % (size_t)P->nx), y = (int)((s / (size_t)P->nx) % (size_t)P->ny);
        int z = (int)(s / ((size_t)P->nx * P->ny));
        double n[Q], f[3], g[16];
        gather(P, src, x, y, z, n);
        node_force(P, force, s, f);
        const double *r = NULL;
        if (P->kT > 0.0) {
            ora_gaussians(P->seed, (uint32_t)s, step, 0u, P->replica, 4, g);
            r = g;
        }
        collide(P, n, f, r, out + (size_t)Q * k);
    }
}
