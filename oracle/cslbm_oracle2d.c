/*
 * cslbm_oracle2d.c -- plain FP64 CPU oracle of the two-dimensional (D2Q9)
 * curved-space lattice Boltzmann step of arXiv 1803.07822 (the 2-D flag
 * simulations use the method on D2Q9).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA library.
 *
 * The same method and readings as the three-dimensional oracle, restated for
 * two dimensions: second-order Hermite equilibrium with the metric (App. B),
 * forcing moments A, B^i, C^ij (Eqs. forcing-A/B/C) with the trapezoidal
 * history, the isotropic lattice gradient of App. D, non-equilibrium
 * extrapolation at walls and inlets and zero-gradient outlets, the node-wise
 * chart change (Sec. IV.B).  Literal f-form: collision, then streaming, the
 * forcing history F(x, t - dt) kept as 9 values per node.
 *
 * Layouts (structure of arrays, axis 0 fastest): node = x + n0 * y;
 *   f, Fprev [9][N]; g3 [3][N] = g00, g01, g11; dg6 [6][N] = d_k g_ij at
 *   (k * 3 + ij); sqrtg [N]; ginv4 [4][N] (full 2 x 2); gam8 [8][N] Gamma^i_jk
 *   at (i * 4 + j * 2 + k); J4 [4][N] J^a_i at (a * 2 + i); face velocity of
 *   face (axis, side): [2][n of the other axis], contravariant, NULL = 0.
 *
 * Parity unpinned, as in three dimensions: the sqrt(g) factor on the
 * non-equilibrium part of the wall and inflow rule (held by convergence and
 * invariant tests only).  The Gamma rho u part of the covariant derivative
 * inside C is pinned, as in three dimensions, by a uniform Cartesian flow in
 * polar coordinates, whose covariant derivative vanishes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q2 9

enum { P2_PERIODIC = 0, P2_WALL = 1, P2_INFLOW = 2, P2_OUTFLOW = 3 };

typedef struct {
    int n[2];
    int bc_lo[2], bc_hi[2];
    double tau, theta;
    double fext[2];
} o2_params;

/* D2Q9: rest, four axis neighbours, four diagonals */
static const int C2[Q2][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};

static double w2(int l)
{
    int s = abs(C2[l][0]) + abs(C2[l][1]);
    return s == 0 ? 4.0 / 9.0 : (s == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
}

static const double CS2_2 = 1.0 / 3.0;

static long nodes2(const o2_params *p) { return (long)p->n[0] * p->n[1]; }
static long id2(const o2_params *p, int x, int y) { return x + (long)p->n[0] * y; }
static int sym3(int i, int j) { return i + j; } /* 00 -> 0, 01/10 -> 1, 11 -> 2 */

int o2_lattice(int *c18, double *w9)
{
    for (int l = 0; l < Q2; l++) {
        c18[2 * l] = C2[l][0];
        c18[2 * l + 1] = C2[l][1];
        w9[l] = w2(l);
    }
    return 0;
}

/* g^ij, sqrt(g) = sqrt(det g), Gamma^i_jk = 1/2 g^il (d_j g_kl + d_k g_jl - d_l g_jk) */
int o2_geometry(const int n[2], const double *g3, const double *dg6, double *sqrtg, double *ginv4, double *gam8)
{
    long N = (long)n[0] * n[1];
    int bad = 0;
    for (long v = 0; v < N; v++) {
        double g[2][2], gi[2][2], dg[2][2][2];
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) {
                g[i][j] = g3[sym3(i, j) * N + v];
                for (int k = 0; k < 2; k++) dg[k][i][j] = dg6[(k * 3 + sym3(i, j)) * N + v];
            }
        double det = g[0][0] * g[1][1] - g[0][1] * g[1][0];
        if (!(det > 0.0)) { bad = 1; continue; }
        gi[0][0] = g[1][1] / det;
        gi[1][1] = g[0][0] / det;
        gi[0][1] = gi[1][0] = -g[0][1] / det;
        sqrtg[v] = sqrt(det);
        for (int a = 0; a < 4; a++) ginv4[a * N + v] = gi[a / 2][a % 2];
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++)
                for (int k = 0; k < 2; k++) {
                    double s = 0.0;
                    for (int l = 0; l < 2; l++) s += gi[i][l] * (dg[j][k][l] + dg[k][j][l] - dg[l][j][k]);
                    gam8[(i * 4 + j * 2 + k) * N + v] = 0.5 * s;
                }
    }
    return bad ? -1 : 0;
}

/* f_l = w_l / sqrt(g) (a0 + a1.c / c_s^2 + a2 : (c c - c_s^2 delta) / (2 c_s^4)) */
static double recompose2(int l, double sg, double a0, const double a1[2], const double a2[2][2])
{
    double h1 = 0.0, h2 = 0.0;
    for (int i = 0; i < 2; i++) {
        h1 += a1[i] * C2[l][i];
        for (int j = 0; j < 2; j++) h2 += a2[i][j] * (C2[l][i] * C2[l][j] - CS2_2 * (i == j));
    }
    return w2(l) / sg * (a0 + h1 / CS2_2 + h2 / (2.0 * CS2_2 * CS2_2));
}

static void feq2(double rho, const double j[2], const double gi[2][2], double sg, double theta, double out[Q2])
{
    double a2[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) a2[a][b] = rho * (theta * gi[a][b] - CS2_2 * (a == b)) + j[a] * j[b] / rho;
    for (int l = 0; l < Q2; l++) out[l] = recompose2(l, sg, rho, j, a2);
}

static void forcing2(double A, const double B[2], const double C[2][2], double sg, double out[Q2])
{
    double b2[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) b2[a][b] = C[a][b] - CS2_2 * (a == b) * A;
    for (int l = 0; l < Q2; l++) out[l] = recompose2(l, sg, A, B, b2);
}

/* A, B^i, C^ij of Eqs. forcing-A/B/C, in two dimensions */
static void forcing_moments2(const double j[2], const double T[2][2], const double Dj[2][2], const double gi[2][2],
                             const double gam[2][2][2], double theta, const double fext[2], double *A, double B[2],
                             double C[2][2])
{
    double a = 0.0;
    for (int i = 0; i < 2; i++)
        for (int k = 0; k < 2; k++) a -= gam[i][i][k] * j[k] + gam[k][i][k] * j[i];
    *A = a;
    for (int i = 0; i < 2; i++) {
        double b = fext[i];
        for (int jj = 0; jj < 2; jj++)
            for (int k = 0; k < 2; k++)
                b -= gam[k][jj][k] * T[i][jj] + gam[i][jj][k] * T[jj][k] + gam[jj][jj][k] * T[k][i];
        B[i] = b;
    }
    double bard[2][2], cov[2][2];
    for (int k = 0; k < 2; k++) {
        double trace = gam[0][k][0] + gam[1][k][1];
        for (int i = 0; i < 2; i++) {
            bard[k][i] = Dj[k][i] - trace * j[i];
            double s = Dj[k][i];
            for (int l = 0; l < 2; l++) s += gam[i][k][l] * j[l];
            cov[k][i] = s;
        }
    }
    double divbar = bard[0][0] + bard[1][1], divcov = cov[0][0] + cov[1][1];
    for (int i = 0; i < 2; i++)
        for (int jj = 0; jj < 2; jj++) {
            double s = CS2_2 * (bard[jj][i] + bard[i][jj] + (i == jj ? divbar : 0.0));
            for (int k = 0; k < 2; k++) s -= theta * (cov[k][i] * gi[jj][k] + cov[k][jj] * gi[i][k]);
            s -= theta * divcov * gi[i][jj];
            C[i][jj] = s;
        }
}

typedef struct {
    const double *sqrtg, *ginv, *gam;
} geom2_t;

static void load_geom2(const geom2_t *G, long N, long v, double *sg, double gi[2][2], double gam[2][2][2])
{
    *sg = G->sqrtg[v];
    for (int a = 0; a < 4; a++) gi[a / 2][a % 2] = G->ginv[a * N + v];
    if (gam)
        for (int a = 0; a < 8; a++) gam[a / 4][(a / 2) % 2][a % 2] = G->gam[a * N + v];
}

static void moments2(const double *f, long N, long v, double sg, double *rho, double j[2], double Pi[2][2])
{
    double r = 0.0, m[2] = {0, 0}, P[2][2] = {{0}};
    for (int l = 0; l < Q2; l++) {
        double fl = f[l * N + v] * sg;
        r += fl;
        for (int a = 0; a < 2; a++) {
            m[a] += fl * C2[l][a];
            for (int b = 0; b < 2; b++) P[a][b] += fl * C2[l][a] * C2[l][b];
        }
    }
    *rho = r;
    for (int a = 0; a < 2; a++) {
        j[a] = m[a];
        if (Pi)
            for (int b = 0; b < 2; b++) Pi[a][b] = P[a][b];
    }
}

/* wall > inflow > outflow; the inner node one step inward along every
 * non-periodic face normal of the node */
static int classify2(const o2_params *p, const int r[2], int *axis, int *side, int inner[2])
{
    static const int prio[4] = {0, 3, 2, 1};
    int best = 0, rank = 0;
    for (int a = 0; a < 2; a++) inner[a] = r[a];
    for (int a = 0; a < 2; a++)
        for (int s = 0; s < 2; s++) {
            int bc = s ? p->bc_hi[a] : p->bc_lo[a];
            if (bc == P2_PERIODIC) continue;
            if (!(s ? r[a] == p->n[a] - 1 : r[a] == 0)) continue;
            inner[a] = s ? r[a] - 1 : r[a] + 1;
            if (prio[bc] > rank) {
                rank = prio[bc];
                best = bc;
                *axis = a;
                *side = s;
            }
        }
    return best;
}

static void apply_bc2(const o2_params *p, const geom2_t *G, const double *const *uface, const double *fin,
                      double *fout)
{
    long N = nodes2(p);
    for (long v = 0; v < N; v++) {
        int r[2] = {(int)(v % p->n[0]), (int)(v / p->n[0])}, in[2], axis = 0, side = 0;
        int bc = classify2(p, r, &axis, &side, in);
        if (bc == P2_PERIODIC) {
            if (fin != fout)
                for (int l = 0; l < Q2; l++) fout[l * N + v] = fin[l * N + v];
            continue;
        }
        long vi = id2(p, in[0], in[1]);
        double sgw, giw[2][2], sgi, gii[2][2];
        load_geom2(G, N, v, &sgw, giw, NULL);
        load_geom2(G, N, vi, &sgi, gii, NULL);
        if (bc == P2_OUTFLOW) {
            for (int l = 0; l < Q2; l++) fout[l * N + v] = fin[l * N + vi] * sgi / sgw;
            continue;
        }
        double rho, j[2], uw[2] = {0, 0}, jw[2], few[Q2], fei[Q2];
        moments2(fin, N, vi, sgi, &rho, j, NULL);
        const double *uf = uface[axis * 2 + side];
        if (uf) {
            int other = 1 - axis, nf = p->n[other];
            for (int a = 0; a < 2; a++) uw[a] = uf[a * (long)nf + r[other]];
        }
        for (int a = 0; a < 2; a++) jw[a] = rho * uw[a];
        feq2(rho, jw, giw, sgw, p->theta, few);
        feq2(rho, j, gii, sgi, p->theta, fei);
        for (int l = 0; l < Q2; l++) fout[l * N + v] = few[l] + (fin[l * N + vi] - fei[l]) * sgi / sgw;
    }
}

/* rho u at a site possibly one step outside: periodic wrap, or the linear
 * extrapolation 2 j(face) - j(face - normal) axis by axis */
static double jval2(const o2_params *p, const double *jf, long N, int comp, int x, int y)
{
    int r[2] = {x, y};
    for (int a = 0; a < 2; a++) {
        if (r[a] >= 0 && r[a] < p->n[a]) continue;
        if ((r[a] < 0 ? p->bc_lo[a] : p->bc_hi[a]) == P2_PERIODIC) {
            r[a] = (r[a] + p->n[a]) % p->n[a];
            continue;
        }
        int r0[2] = {r[0], r[1]}, r1[2] = {r[0], r[1]};
        if (r[a] < 0) { r0[a] = 0; r1[a] = 1; }
        else { r0[a] = p->n[a] - 1; r1[a] = p->n[a] - 2; }
        return 2.0 * jval2(p, jf, N, comp, r0[0], r0[1]) - jval2(p, jf, N, comp, r1[0], r1[1]);
    }
    return jf[comp * N + id2(p, r[0], r[1])];
}

static void forcing_field2(const o2_params *p, const geom2_t *G, const double *fb, double *F, double *feq)
{
    long N = nodes2(p);
    double *jf = (double *)malloc(sizeof(double) * 2 * N);
    for (long v = 0; v < N; v++) {
        double rho, j[2];
        moments2(fb, N, v, G->sqrtg[v], &rho, j, NULL);
        jf[v] = j[0];
        jf[N + v] = j[1];
    }
    for (long v = 0; v < N; v++) {
        int r[2] = {(int)(v % p->n[0]), (int)(v / p->n[0])};
        double sg, gi[2][2], gam[2][2][2], rho, j[2], fe[Q2];
        load_geom2(G, N, v, &sg, gi, gam);
        moments2(fb, N, v, sg, &rho, j, NULL);
        feq2(rho, j, gi, sg, p->theta, fe);
        double T[2][2] = {{0}};
        for (int l = 0; l < Q2; l++) {
            double fl = fb[l * N + v];
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++)
                    T[a][b] += (fe[l] + (1.0 - 0.5 / p->tau) * (fl - fe[l])) * C2[l][a] * C2[l][b] * sg;
        }
        double Dj[2][2] = {{0}};
        for (int l = 1; l < Q2; l++)
            for (int i = 0; i < 2; i++) {
                double jn = jval2(p, jf, N, i, r[0] + C2[l][0], r[1] + C2[l][1]);
                for (int k = 0; k < 2; k++) Dj[k][i] += w2(l) * C2[l][k] * jn / CS2_2;
            }
        double A, B[2], C[2][2], Fl[Q2];
        forcing_moments2(j, T, Dj, gi, gam, p->theta, p->fext, &A, B, C);
        forcing2(A, B, C, sg, Fl);
        for (int l = 0; l < Q2; l++) {
            F[l * N + v] = Fl[l];
            if (feq) feq[l * N + v] = fe[l];
        }
    }
    free(jf);
}

static int check2(const o2_params *p)
{
    for (int a = 0; a < 2; a++) {
        if (p->n[a] < 1) return -1;
        if ((p->bc_lo[a] == P2_PERIODIC) != (p->bc_hi[a] == P2_PERIODIC)) return -1;
        if (p->bc_lo[a] != P2_PERIODIC && p->n[a] < 3) return -1;
    }
    return p->tau > 0.5 ? 0 : -1;
}

/* single-node forcing recomposition F_l from A, B [2], C [4] (row-major), for
 * the moment identities of the tests */
int o2_forcing_recompose(double A, const double *B2, const double *C4, double sg, double *out9)
{
    const double B[2] = {B2[0], B2[1]}, C[2][2] = {{C4[0], C4[1]}, {C4[2], C4[3]}};
    forcing2(A, B, C, sg, out9);
    return 0;
}

/* A, B^i, C^ij of one node: j2 = rho u^i, T4 = T^ij, Dj4[k*2+i] = d_k(rho u^i),
 * ginv4 = g^ij, gam8 = Gamma^i_jk at (i*4 + j*2 + k); outputs A, B2, C4 (full 2 x 2) */
int o2_forcing_moments(const double *j2, const double *T4, const double *Dj4, const double *ginv4,
                       const double *gam8, double theta, const double *fext2, double *A, double *B2, double *C4)
{
    double T[2][2], Dj[2][2], gi[2][2], gam[2][2][2], C[2][2];
    for (int a = 0; a < 4; a++) {
        T[a / 2][a % 2] = T4[a];
        Dj[a / 2][a % 2] = Dj4[a];
        gi[a / 2][a % 2] = ginv4[a];
    }
    for (int a = 0; a < 8; a++) gam[a / 4][(a / 2) % 2][a % 2] = gam8[a];
    forcing_moments2(j2, T, Dj, gi, gam, theta, fext2, A, B2, C);
    for (int a = 0; a < 4; a++) C4[a] = C[a / 2][a % 2];
    return 0;
}

int o2_init(const o2_params *p, const double *sqrtg, const double *ginv4, const double *gam8, const double *rho0,
            const double *u0, const double *const *uface, double *f, double *Fprev)
{
    if (check2(p)) return -1;
    long N = nodes2(p);
    geom2_t G = {sqrtg, ginv4, gam8};
    for (long v = 0; v < N; v++) {
        double sg, gi[2][2], j[2], fe[Q2];
        load_geom2(&G, N, v, &sg, gi, NULL);
        for (int a = 0; a < 2; a++) j[a] = rho0[v] * u0[a * N + v];
        feq2(rho0[v], j, gi, sg, p->theta, fe);
        for (int l = 0; l < Q2; l++) f[l * N + v] = fe[l];
    }
    double *fb = (double *)malloc(sizeof(double) * Q2 * N);
    apply_bc2(p, &G, uface, f, fb);
    forcing_field2(p, &G, fb, Fprev, NULL);
    free(fb);
    return 0;
}

/* collision f* = f - (f - f^eq)/tau + F(t) - F(t - dt)/2, streaming
 * f(x, t + dt) = f*(x - c, t) + F(x, t)/2, the boundary rule on f(t) first */
int o2_step(const o2_params *p, const double *sqrtg, const double *ginv4, const double *gam8,
            const double *const *uface, double *f, double *Fprev, int nsteps)
{
    if (check2(p)) return -1;
    long N = nodes2(p);
    geom2_t G = {sqrtg, ginv4, gam8};
    double *fb = malloc(sizeof(double) * Q2 * N), *F = malloc(sizeof(double) * Q2 * N);
    double *fe = malloc(sizeof(double) * Q2 * N), *fs = malloc(sizeof(double) * Q2 * N);
    double om = 1.0 / p->tau;
    for (int t = 0; t < nsteps; t++) {
        apply_bc2(p, &G, uface, f, fb);
        forcing_field2(p, &G, fb, F, fe);
        for (long q = 0; q < (long)Q2 * N; q++) fs[q] = fb[q] - om * (fb[q] - fe[q]) + F[q] - 0.5 * Fprev[q];
        for (long v = 0; v < N; v++) {
            int r[2] = {(int)(v % p->n[0]), (int)(v / p->n[0])};
            for (int l = 0; l < Q2; l++) {
                int s[2], inside = 1;
                for (int a = 0; a < 2; a++) {
                    s[a] = r[a] - C2[l][a];
                    if (s[a] < 0 || s[a] >= p->n[a]) {
                        if ((s[a] < 0 ? p->bc_lo[a] : p->bc_hi[a]) == P2_PERIODIC) s[a] = (s[a] + p->n[a]) % p->n[a];
                        else inside = 0;
                    }
                }
                f[l * N + v] = inside ? fs[l * N + id2(p, s[0], s[1])] + 0.5 * F[l * N + v] : NAN;
            }
        }
        memcpy(Fprev, F, sizeof(double) * Q2 * N);
    }
    free(fb);
    free(F);
    free(fe);
    free(fs);
    return 0;
}

/* rho and u^i (or v^a = J^a_i u^i with J4) of the boundary-filled state */
int o2_moments(const o2_params *p, const double *sqrtg, const double *ginv4, const double *const *uface,
               const double *f, const double *J4, double *rho, double *u2)
{
    if (check2(p)) return -1;
    long N = nodes2(p);
    geom2_t G = {sqrtg, ginv4, NULL};
    double *fb = malloc(sizeof(double) * Q2 * N);
    apply_bc2(p, &G, uface, f, fb);
    for (long v = 0; v < N; v++) {
        double r, j[2], u[2];
        moments2(fb, N, v, sqrtg[v], &r, j, NULL);
        u[0] = j[0] / r;
        u[1] = j[1] / r;
        rho[v] = r;
        for (int a = 0; a < 2; a++) u2[a * N + v] = J4 ? J4[(a * 2) * N + v] * u[0] + J4[(a * 2 + 1) * N + v] * u[1] : u[a];
    }
    free(fb);
    return 0;
}

int o2_mass(const o2_params *p, const double *sqrtg, const double *ginv4, const double *const *uface,
            const double *f, double *out)
{
    if (check2(p)) return -1;
    long N = nodes2(p);
    geom2_t G = {sqrtg, ginv4, NULL};
    double *fb = malloc(sizeof(double) * Q2 * N), m = 0.0;
    apply_bc2(p, &G, uface, f, fb);
    for (long v = 0; v < N; v++) {
        double r, j[2];
        moments2(fb, N, v, sqrtg[v], &r, j, NULL);
        m += sqrtg[v] * r;
    }
    free(fb);
    *out = m;
    return 0;
}

/* F^a = s sum_{wall nodes} J^a_i T^{i axis} sqrt(g) (per unit depth) */
int o2_wall_force(const o2_params *p, const double *sqrtg, const double *ginv4, const double *const *uface,
                  const double *f, const double *J4, int axis, int side, double *out2)
{
    if (check2(p) || axis < 0 || axis > 1) return -1;
    long N = nodes2(p);
    geom2_t G = {sqrtg, ginv4, NULL};
    double *fb = malloc(sizeof(double) * Q2 * N), acc[2] = {0, 0}, s = side ? 1.0 : -1.0;
    apply_bc2(p, &G, uface, f, fb);
    int plane = side ? p->n[axis] - 1 : 0;
    for (long v = 0; v < N; v++) {
        int r[2] = {(int)(v % p->n[0]), (int)(v / p->n[0])};
        if (r[axis] != plane) continue;
        double sg, gi[2][2], rho, j[2], fe[Q2], T[2][2] = {{0}};
        load_geom2(&G, N, v, &sg, gi, NULL);
        moments2(fb, N, v, sg, &rho, j, NULL);
        feq2(rho, j, gi, sg, p->theta, fe);
        for (int l = 0; l < Q2; l++) {
            double fl = fb[l * N + v];
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) T[a][b] += (fe[l] + (1.0 - 0.5 / p->tau) * (fl - fe[l])) * C2[l][a] * C2[l][b] * sg;
        }
        for (int a = 0; a < 2; a++)
            for (int i = 0; i < 2; i++) acc[a] += s * J4[(a * 2 + i) * N + v] * T[i][axis] * sg;
    }
    free(fb);
    out2[0] = acc[0];
    out2[1] = acc[1];
    return 0;
}

/* node-wise chart change: D phi = Jnew^-1 Jold, a0 kept, a1 -> D a1,
 * Pi -> D Pi D^T (a2 = Pi - c_s^2 a0 delta), recomposed with the new sqrt(g);
 * the history likewise */
int o2_transform(const o2_params *p, const double *sqrtg_old, const double *ginv4_old, const double *sqrtg_new,
                 const double *Jold4, const double *Jnew4, const double *const *uface, double *f, double *Fprev)
{
    if (check2(p)) return -1;
    long N = nodes2(p);
    geom2_t G = {sqrtg_old, ginv4_old, NULL};
    double *fb = malloc(sizeof(double) * Q2 * N);
    apply_bc2(p, &G, uface, f, fb);
    for (long v = 0; v < N; v++) {
        double Jo[2][2], Jn[2][2], Jni[2][2], D[2][2];
        for (int a = 0; a < 4; a++) {
            Jo[a / 2][a % 2] = Jold4[a * N + v];
            Jn[a / 2][a % 2] = Jnew4[a * N + v];
        }
        double det = Jn[0][0] * Jn[1][1] - Jn[0][1] * Jn[1][0];
        Jni[0][0] = Jn[1][1] / det;
        Jni[1][1] = Jn[0][0] / det;
        Jni[0][1] = -Jn[0][1] / det;
        Jni[1][0] = -Jn[1][0] / det;
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) D[i][j] = Jni[i][0] * Jo[0][j] + Jni[i][1] * Jo[1][j];
        for (int pass = 0; pass < 2; pass++) {
            double *src = pass ? Fprev : fb, *dst = pass ? Fprev : f;
            double a0, a1[2], M[2][2], t1[2], t2[2][2];
            moments2(src, N, v, sqrtg_old[v], &a0, a1, M);
            for (int i = 0; i < 2; i++) t1[i] = D[i][0] * a1[0] + D[i][1] * a1[1];
            for (int i = 0; i < 2; i++)
                for (int j = 0; j < 2; j++) {
                    double s = 0.0;
                    for (int l = 0; l < 2; l++)
                        for (int m = 0; m < 2; m++) s += D[i][l] * D[j][m] * M[l][m];
                    t2[i][j] = s - CS2_2 * a0 * (i == j);
                }
            for (int l = 0; l < Q2; l++) dst[l * N + v] = recompose2(l, sqrtg_new[v], a0, t1, t2);
        }
    }
    free(fb);
    return 0;
}
