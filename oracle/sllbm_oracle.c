/*
 * sllbm_oracle.c -- plain, slow, FP64 CPU oracle of one SLLBM time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference against which
 * the CUDA path is checked.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load it.  It shares no code, header, table or
 * constant generator with the CUDA library: every quantity below is rebuilt here
 * from the paper (arXiv:2012.05537, Wilde, Kraemer, Reith, Foysi).
 *
 * Method summary, each step cited where it is implemented:
 *   - velocity set: degree-9 cubature with 45 abscissae (Sec. II.B, Fig. 2);
 *   - support points: Gauss-Lobatto-Chebyshev nodes of order p per cell (Sec. II.A, Fig. 1);
 *   - streaming: cell-oriented Lagrange interpolation at the departure point
 *     x - dt*xi_i (Eq. interpolation, and the Psi_i paragraph of Sec. II.A),
 *     evaluated here as the literal (p+1)^3 tensor sum in the enclosing cell;
 *   - moments: Eq. (moments);
 *   - equilibrium: Eq. (discreteEquilibrium) with the moments of App. A and the
 *     Hermite tensors of App. B, contracted over all 3^n index combinations;
 *   - second distribution g^eq = (2 C_v - D) T f^eq (Sec. II.A);
 *   - relaxation: tau = mu/(P dt) + 1/2 with P = rho T (Sec. II.A), mu from the
 *     Sutherland law (Sec. III.C);
 *   - BGK collision (Eq. LBM) with the optional quasi-equilibrium Prandtl
 *     correction of App. D;
 *   - diagnostics E_k, eps_s, eps_c (Sec. III.C) by per-cell interpolatory
 *     quadrature on the support points and cell-local Lagrange derivatives.
 *
 * Readings where the paper is silent or garbled (listed in the design notes):
 *   lattice units c_s^2 = T_ref = 1 (the Hermite tensors use xi/c_s with unit-variance
 *   Gaussian weight), P = rho*T, the 1/3! factor in the Prandtl term, g* = (2C_v-D) T f*,
 *   floor convention for departure points on a cell face.
 *
 * Parity unpinned: that the 45-point set below is the paper's own table (the table is
 * not printed in the paper).  The set itself is pinned by its degree-9 exactness.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 45
#define ORC_D 3

/* ------------------------------------------------------------------------ */
/* Velocity set.  Sec. II.B: 45 abscissae, degree nine, icosahedral symmetry
 * (Fig. 2, rule after Konyaev).  Built here as four orbits for the unit-variance
 * Gaussian weight: origin, an icosahedron of radius sqrt(3), a dodecahedron of
 * radius 3 (vertices = face centres of the icosahedron) and an icosahedron of
 * radius sqrt(15).  Weights solve the invariant moment equations in closed form.
 * Order: origin; inner icosahedron; dodecahedron; outer icosahedron.  Within an
 * icosahedron: for s1 in (+,-), s2 in (+,-): (0,s1,s2*phi), (s1,s2*phi,0),
 * (s2*phi,0,s1).  Within the dodecahedron: the eight (+-1,+-1,+-1) with x slowest
 * and + before -, then for s1 in (+,-), s2 in (+,-): (s1/phi,0,s2*phi),
 * (s1*phi,s2/phi,0), (0,s1*phi,s2/phi).  Each direction is normalised, then scaled.
 */
static void orc_put(double *xi, int i, double x, double y, double z, double radius)
{
    double n = sqrt(x * x + y * y + z * z);
    xi[3 * i + 0] = radius * x / n;
    xi[3 * i + 1] = radius * y / n;
    xi[3 * i + 2] = radius * z / n;
}

int orc_velset(double *xi, double *w)
{
    const double phi = 0.5 * (1.0 + sqrt(5.0));
    int i = 0;
    int s1, s2, a, b, c;
    xi[0] = xi[1] = xi[2] = 0.0;
    w[i++] = 28.0 / 135.0;
    for (s1 = 1; s1 >= -1; s1 -= 2)
        for (s2 = 1; s2 >= -1; s2 -= 2) {
            orc_put(xi, i, 0.0, s1, s2 * phi, sqrt(3.0)); w[i++] = 25.0 / 432.0;
            orc_put(xi, i, s1, s2 * phi, 0.0, sqrt(3.0)); w[i++] = 25.0 / 432.0;
            orc_put(xi, i, s2 * phi, 0.0, s1, sqrt(3.0)); w[i++] = 25.0 / 432.0;
        }
    for (a = 1; a >= -1; a -= 2)
        for (b = 1; b >= -1; b -= 2)
            for (c = 1; c >= -1; c -= 2) {
                orc_put(xi, i, a, b, c, 3.0); w[i++] = 1.0 / 216.0;
            }
    for (s1 = 1; s1 >= -1; s1 -= 2)
        for (s2 = 1; s2 >= -1; s2 -= 2) {
            orc_put(xi, i, s1 / phi, 0.0, s2 * phi, 3.0); w[i++] = 1.0 / 216.0;
            orc_put(xi, i, s1 * phi, s2 / phi, 0.0, 3.0); w[i++] = 1.0 / 216.0;
            orc_put(xi, i, 0.0, s1 * phi, s2 / phi, 3.0); w[i++] = 1.0 / 216.0;
        }
    for (s1 = 1; s1 >= -1; s1 -= 2)
        for (s2 = 1; s2 >= -1; s2 -= 2) {
            orc_put(xi, i, 0.0, s1, s2 * phi, sqrt(15.0)); w[i++] = 1.0 / 2160.0;
            orc_put(xi, i, s1, s2 * phi, 0.0, sqrt(15.0)); w[i++] = 1.0 / 2160.0;
            orc_put(xi, i, s2 * phi, 0.0, s1, sqrt(15.0)); w[i++] = 1.0 / 2160.0;
        }
    return i;
}

/* ------------------------------------------------------------------------ */
/* Support points: Gauss-Lobatto-Chebyshev nodes of order p on the reference
 * interval [-1,1] (Sec. II.A, Fig. 1): r_a = -cos(pi a / p), a = 0..p.       */
void orc_glc(int p, double *r)
{
    int a;
    for (a = 0; a <= p; ++a) r[a] = -cos(M_PI * (double)a / (double)p);
}

/* Lagrange basis psi_j(r) on the GLC nodes (Eq. interpolation), product form. */
void orc_lagrange(int p, double r, double *ell)
{
    double nodes[16];
    int j, m;
    orc_glc(p, nodes);
    for (j = 0; j <= p; ++j) {
        double v = 1.0;
        for (m = 0; m <= p; ++m)
            if (m != j) v *= (r - nodes[m]) / (nodes[j] - nodes[m]);
        ell[j] = v;
    }
}

/* Derivative of the Lagrange basis, d psi_j / dr, by the product rule. */
void orc_lagrange_deriv(int p, double r, double *dell)
{
    double nodes[16];
    int j, m, k;
    orc_glc(p, nodes);
    for (j = 0; j <= p; ++j) {
        double s = 0.0;
        for (k = 0; k <= p; ++k) {
            double v;
            if (k == j) continue;
            v = 1.0 / (nodes[j] - nodes[k]);
            for (m = 0; m <= p; ++m)
                if (m != j && m != k) v *= (r - nodes[m]) / (nodes[j] - nodes[m]);
            s += v;
        }
        dell[j] = s;
    }
}

/* Interpolatory quadrature weights on the GLC nodes, W_j = int_{-1}^{1} psi_j dr,
 * i.e. the Clenshaw-Curtis rule; obtained by solving the moment (Vandermonde)
 * system sum_j W_j r_j^k = int r^k dr, k = 0..p, with Gaussian elimination.    */
void orc_quad_weights(int p, double *W)
{
    double A[16][17];
    double nodes[16];
    int n = p + 1, i, j, k;
    orc_glc(p, nodes);
    for (k = 0; k < n; ++k) {
        for (j = 0; j < n; ++j) A[k][j] = pow(nodes[j], (double)k);
        A[k][n] = (k % 2 == 0) ? 2.0 / (double)(k + 1) : 0.0;
    }
    for (i = 0; i < n; ++i) {
        int piv = i;
        for (k = i + 1; k < n; ++k)
            if (fabs(A[k][i]) > fabs(A[piv][i])) piv = k;
        for (j = 0; j <= n; ++j) { double t = A[i][j]; A[i][j] = A[piv][j]; A[piv][j] = t; }
        for (k = 0; k < n; ++k) {
            double f;
            if (k == i) continue;
            f = A[k][i] / A[i][i];
            for (j = i; j <= n; ++j) A[k][j] -= f * A[i][j];
        }
    }
    for (i = 0; i < n; ++i) W[i] = A[i][n] / A[i][i];
}

/* Sutherland law (Sec. III.C): mu/mu_inf = 1.4042 T^1.5 / (T + 0.40417). */
double orc_sutherland(double T)
{
    return 1.4042 * pow(T, 1.5) / (T + 0.40417);
}

/* ------------------------------------------------------------------------ */
/* Equilibrium by full tensor contraction, Eq. (discreteEquilibrium):
 *   f_i^eq = w_i sum_{n=0}^{4} (1/n!) a^(n)_eq : H_i^(n),
 * moments a^(n)_eq from App. A (theta = T/T_ref, T_ref = 1 so T_ref(theta-1) = T-1),
 * Hermite tensors from App. B with c_s = 1.  Every one of the 3^n components of
 * both tensors is formed and multiplied; no symmetry is exploited.             */
static double kd(int a, int b) { return a == b ? 1.0 : 0.0; }

static double orc_a_n(int n, const int *ix, double rho, const double *u, double T)
{
    double th = T - 1.0;
    int a = ix[0], b = ix[1], c = ix[2], d = ix[3];
    switch (n) {
    case 0: return rho;
    case 1: return rho * u[a];
    case 2: return rho * (u[a] * u[b] + th * kd(a, b));
    case 3:
        return rho * (u[a] * u[b] * u[c]
                      + th * (kd(a, b) * u[c] + kd(a, c) * u[b] + kd(b, c) * u[a]));
    case 4:
        return rho * (u[a] * u[b] * u[c] * u[d]
                      + th * ((kd(a, b) * kd(c, d) + kd(a, c) * kd(b, d) + kd(a, d) * kd(b, c)) * th
                              + kd(a, b) * u[c] * u[d] + kd(a, c) * u[b] * u[d]
                              + kd(a, d) * u[b] * u[c] + kd(b, c) * u[a] * u[d]
                              + kd(b, d) * u[a] * u[c] + kd(c, d) * u[a] * u[b]));
    }
    return 0.0;
}

static double orc_H_n(int n, const int *ix, const double *x)
{
    int a = ix[0], b = ix[1], c = ix[2], d = ix[3];
    switch (n) {
    case 0: return 1.0;
    case 1: return x[a];
    case 2: return x[a] * x[b] - kd(a, b);
    case 3: return x[a] * x[b] * x[c] - (x[a] * kd(b, c) + x[b] * kd(a, c) + x[c] * kd(a, b));
    case 4: {
        double Ti = x[a] * x[b] * kd(c, d) + x[a] * x[c] * kd(b, d) + x[a] * x[d] * kd(b, c)
                  + x[b] * x[c] * kd(a, d) + x[b] * x[d] * kd(a, c) + x[c] * x[d] * kd(a, b);
        return x[a] * x[b] * x[c] * x[d] - Ti
             + (kd(a, b) * kd(c, d) + kd(a, c) * kd(b, d) + kd(a, d) * kd(b, c));
    }
    }
    return 0.0;
}

double orc_feq_one(const double *x, double w, double rho, const double *u, double T)
{
    static const double inv_fact[5] = {1.0, 1.0, 0.5, 1.0 / 6.0, 1.0 / 24.0};
    double total = 0.0;
    int n, k;
    for (n = 0; n <= 4; ++n) {
        int count = 1, ix[4] = {0, 0, 0, 0};
        double s = 0.0;
        for (k = 0; k < n; ++k) count *= 3;
        for (k = 0; k < count; ++k) {
            int m, r = k;
            for (m = 0; m < n; ++m) { ix[m] = r % 3; r /= 3; }
            s += orc_a_n(n, ix, rho, u, T) * orc_H_n(n, ix, x);
        }
        total += inv_fact[n] * s;
    }
    return w * total;
}

void orc_feq(const double *xi, const double *w, int Q, double rho, const double *u, double T,
             double *feq)
{
    int i;
    for (i = 0; i < Q; ++i) feq[i] = orc_feq_one(xi + 3 * i, w[i], rho, u, T);
}

/* ------------------------------------------------------------------------ */
/* Mesh: periodic uniform hexahedral cells, cells[d] per dimension on [0, L[d]).
 * Node index along d: n = c*p + a, a in [0,p) (the a = p node of cell c is node 0 of
 * cell c+1).  Populations are stored as pop[h][i][z][y][x], h in {f,g}.          */
typedef struct {
    int cells[3];
    int p;
    double L[3];
    double dt;
    double mu_inf;
    double gamma;
    double Pr;
    int pr_correction;
    int collide; /* 0: streaming only (used by advection tests) */
} orc_cfg;

static long orc_nodes(const orc_cfg *g)
{
    return (long)g->cells[0] * g->p * (long)g->cells[1] * g->p * (long)g->cells[2] * g->p;
}

void orc_node_coords(const orc_cfg *g, int d, double *x)
{
    int c, a, N = g->cells[d] * g->p;
    double h = g->L[d] / g->cells[d];
    for (c = 0; c < g->cells[d]; ++c)
        for (a = 0; a < g->p; ++a)
            x[c * g->p + a] = c * h + (1.0 - cos(M_PI * a / g->p)) * 0.5 * h;
    (void)N;
}

static int wrap(long v, int n)
{
    long r = v % n;
    return (int)(r < 0 ? r + n : r);
}

/* Departure search of Sec. II.A for one support point and one velocity: the departure
 * point x - dt xi is located by the floor of its cell coordinate (periodic wrap happens
 * when the support values are read), and the Lagrange basis of Eq. (interpolation) is
 * evaluated at its reference coordinate in each direction.                          */
static void orc_departure(const orc_cfg *g, double *const xs[3], const int node[3],
                          const double *xi_i, int base[3], double ell[3][16])
{
    int dd;
    for (dd = 0; dd < 3; ++dd) {
        double h = g->L[dd] / g->cells[dd];
        double y = xs[dd][node[dd]] - g->dt * xi_i[dd];
        double cf = floor(y / h);
        double r = 2.0 * (y / h - cf) - 1.0;
        base[dd] = (int)cf * g->p; /* first support node of the departure cell */
        orc_lagrange(g->p, r, ell[dd]);
    }
}

/* Semi-Lagrangian streaming, Sec. II.A: for every support point x and velocity i,
 * the departure point x - dt xi_i is located (floor of the cell coordinate, periodic
 * wrap), and h_i is evaluated there with the tensor-product Lagrange interpolant of
 * the enclosing cell's (p+1)^3 support values (Eq. interpolation).  nvel velocities
 * are given explicitly so that synthetic velocities can be streamed in tests.   */
void orc_stream(const orc_cfg *g, int nh, int nvel, const double *xi, const double *src,
                double *dst)
{
    const int p = g->p;
    const int N[3] = {g->cells[0] * p, g->cells[1] * p, g->cells[2] * p};
    const long nn = (long)N[0] * N[1] * N[2];
    double *xs[3];
    int d;
    for (d = 0; d < 3; ++d) {
        xs[d] = (double *)malloc(sizeof(double) * N[d]);
        orc_node_coords(g, d, xs[d]);
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int hq = 0; hq < nh * nvel; ++hq) {
        for (long n = 0; n < nn; ++n) {
            const int i = hq % nvel;
            const double *in = src + (long)hq * nn;
            int node[3], base[3], j, k, l;
            double ell[3][16];
            double acc = 0.0;
            node[0] = (int)(n % N[0]);
            node[1] = (int)((n / N[0]) % N[1]);
            node[2] = (int)(n / ((long)N[0] * N[1]));
            orc_departure(g, xs, node, xi + 3 * i, base, ell);
            for (l = 0; l <= p; ++l)
                for (k = 0; k <= p; ++k)
                    for (j = 0; j <= p; ++j) {
                        int sx = wrap(base[0] + j, N[0]);
                        int sy = wrap(base[1] + k, N[1]);
                        int sz = wrap(base[2] + l, N[2]);
                        acc += ell[0][j] * ell[1][k] * ell[2][l]
                             * in[((long)sz * N[1] + sy) * N[0] + sx];
                    }
            dst[(long)hq * nn + n] = acc;
        }
    }
    for (d = 0; d < 3; ++d) free(xs[d]);
}

/* Moments, Eq. (moments): rho = sum f, rho u = sum f xi, 2 rho E = sum(f|xi|^2 + g).
 * T follows from 2 rho E = rho|u|^2 + 2 C_v rho T (the energy of the equilibrium,
 * whose second moment is rho(uu + T delta) and whose g-sum is (2C_v - D) rho T).  */
static void orc_node_moments(const double *f, const double *gsum_in, const double *xi,
                             double Cv, double *rho, double *u, double *T)
{
    double r = 0.0, m[3] = {0, 0, 0}, e2 = 0.0, usq;
    int i;
    for (i = 0; i < ORC_Q; ++i) {
        double x2 = xi[3 * i] * xi[3 * i] + xi[3 * i + 1] * xi[3 * i + 1]
                  + xi[3 * i + 2] * xi[3 * i + 2];
        r += f[i];
        m[0] += f[i] * xi[3 * i];
        m[1] += f[i] * xi[3 * i + 1];
        m[2] += f[i] * xi[3 * i + 2];
        e2 += f[i] * x2;
    }
    e2 += *gsum_in;
    u[0] = m[0] / r; u[1] = m[1] / r; u[2] = m[2] / r;
    usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    *rho = r;
    *T = (e2 - r * usq) / (2.0 * Cv * r);
}

void orc_moments(const orc_cfg *g, const double *pop, double *rho, double *u, double *T)
{
    double xi[3 * ORC_Q], w[ORC_Q];
    const long nn = orc_nodes(g);
    const double Cv = 1.0 / (g->gamma - 1.0);
    orc_velset(xi, w);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < nn; ++n) {
        double f[ORC_Q], gs = 0.0, uu[3];
        int i;
        for (i = 0; i < ORC_Q; ++i) {
            f[i] = pop[(long)i * nn + n];
            gs += pop[(long)(ORC_Q + i) * nn + n];
        }
        orc_node_moments(f, &gs, xi, Cv, &rho[n], uu, &T[n]);
        u[n] = uu[0]; u[nn + n] = uu[1]; u[2 * nn + n] = uu[2];
    }
}

/* Collision at every node, Eq. (LBM) right-hand side:
 *   h_i <- h_i - (h_i - h_i^eq)/tau   [+ (1/tau - 1/tau_Pr) h_i^*, App. D],
 * g_i^eq = (2C_v - D) T f_i^eq, tau = mu/(P dt) + 1/2, P = rho T, mu = Sutherland(T) mu_inf.
 * App. D: Qbar_abc = sum_i f_i (xi-u)_a (xi-u)_b (xi-u)_c, Qbar^eq = 0 for this
 * equilibrium, h_i^* = (w_i/3!) Qbar^neq : H_i^(3), g_i^* = (2C_v - D) T f_i^*,
 * tau_Pr = (tau - 1/2)/Pr + 1/2.                                                  */
static void orc_collide_one(const orc_cfg *g, const double *xi, const double *w, double *f,
                            double *gg)
{
    const double Cv = 1.0 / (g->gamma - 1.0);
    const double gfac_c = 2.0 * Cv - 3.0;
    double feq[ORC_Q], fst[ORC_Q];
    double gs = 0.0, rho, u[3], T, mu, tau, omega, om_pr = 0.0;
    int i;
    for (i = 0; i < ORC_Q; ++i) gs += gg[i];
    orc_node_moments(f, &gs, xi, Cv, &rho, u, &T);
    mu = orc_sutherland(T) * g->mu_inf;
    tau = mu / (rho * T * g->dt) + 0.5;
    omega = 1.0 / tau;
    orc_feq(xi, w, ORC_Q, rho, u, T, feq);
    for (i = 0; i < ORC_Q; ++i) fst[i] = 0.0;
    if (g->pr_correction) {
        double Qb[3][3][3];
        int a, b, c, ix[4] = {0, 0, 0, 0};
        double tau_pr = (tau - 0.5) / g->Pr + 0.5;
        om_pr = 1.0 / tau - 1.0 / tau_pr;
        for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b)
                for (c = 0; c < 3; ++c) {
                    double s = 0.0;
                    for (i = 0; i < ORC_Q; ++i)
                        s += f[i] * (xi[3 * i + a] - u[a]) * (xi[3 * i + b] - u[b])
                           * (xi[3 * i + c] - u[c]);
                    Qb[a][b][c] = s; /* Qbar^eq = 0, so this is Qbar^neq */
                }
        for (i = 0; i < ORC_Q; ++i) {
            double s = 0.0;
            for (a = 0; a < 3; ++a)
                for (b = 0; b < 3; ++b)
                    for (c = 0; c < 3; ++c) {
                        ix[0] = a; ix[1] = b; ix[2] = c;
                        s += Qb[a][b][c] * orc_H_n(3, ix, xi + 3 * i);
                    }
            fst[i] = w[i] * s / 6.0;
        }
    }
    for (i = 0; i < ORC_Q; ++i) {
        double geq = gfac_c * T * feq[i];
        double gst = gfac_c * T * fst[i];
        f[i] = f[i] - omega * (f[i] - feq[i]) + om_pr * fst[i];
        gg[i] = gg[i] - omega * (gg[i] - geq) + om_pr * gst;
    }
}

void orc_collide(const orc_cfg *g, double *pop)
{
    double xi[3 * ORC_Q], w[ORC_Q];
    const long nn = orc_nodes(g);
    orc_velset(xi, w);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < nn; ++n) {
        double f[ORC_Q], gg[ORC_Q];
        int i;
        for (i = 0; i < ORC_Q; ++i) {
            f[i] = pop[(long)i * nn + n];
            gg[i] = pop[(long)(ORC_Q + i) * nn + n];
        }
        orc_collide_one(g, xi, w, f, gg);
        for (i = 0; i < ORC_Q; ++i) {
            pop[(long)i * nn + n] = f[i];
            pop[(long)(ORC_Q + i) * nn + n] = gg[i];
        }
    }
}

/* One or more time steps: the stored state is the post-collision population; each
 * step streams it (pull, departure points x - dt xi_i) and collides the result.
 * popA holds the input; the result ends in popA (popB is workspace).             */
void orc_step(const orc_cfg *g, double *popA, double *popB, int nsteps)
{
    double xi[3 * ORC_Q], w[ORC_Q];
    const long nn = orc_nodes(g);
    int s;
    orc_velset(xi, w);
    for (s = 0; s < nsteps; ++s) {
        orc_stream(g, 2, ORC_Q, xi, popA, popB);
        if (g->collide) orc_collide(g, popB);
        memcpy(popA, popB, sizeof(double) * 2 * ORC_Q * nn);
    }
}

/* Equilibrium initialisation from given fields: f_i = f_i^eq, g_i = (2C_v-D) T f_i^eq. */
void orc_init_fields(const orc_cfg *g, const double *rho, const double *u, const double *T,
                     double *pop)
{
    double xi[3 * ORC_Q], w[ORC_Q];
    const long nn = orc_nodes(g);
    const double gfac_c = 2.0 / (g->gamma - 1.0) - 3.0;
    orc_velset(xi, w);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < nn; ++n) {
        double feq[ORC_Q], uu[3] = {u[n], u[nn + n], u[2 * nn + n]};
        int i;
        orc_feq(xi, w, ORC_Q, rho[n], uu, T[n], feq);
        for (i = 0; i < ORC_Q; ++i) {
            pop[(long)i * nn + n] = feq[i];
            pop[(long)(ORC_Q + i) * nn + n] = gfac_c * T[n] * feq[i];
        }
    }
}

/* Taylor-Green vortex fields, Sec. III.C (constant-temperature initial condition):
 *   u = U0 sin x cos y cos z, v = -U0 cos x sin y cos z, w = 0,
 *   rho = rho0 [1 + (C/16)(cos 2x + cos 2y)(cos 2z + 2)], T = T0.               */
void orc_tgv_fields(const orc_cfg *g, double U0, double rho0, double T0, double C, double *rho,
                    double *u, double *T)
{
    const int N[3] = {g->cells[0] * g->p, g->cells[1] * g->p, g->cells[2] * g->p};
    const long nn = (long)N[0] * N[1] * N[2];
    double *xs[3];
    int d;
    for (d = 0; d < 3; ++d) {
        xs[d] = (double *)malloc(sizeof(double) * N[d]);
        orc_node_coords(g, d, xs[d]);
    }
    for (long n = 0; n < nn; ++n) {
        double x = xs[0][n % N[0]], y = xs[1][(n / N[0]) % N[1]], z = xs[2][n / ((long)N[0] * N[1])];
        u[n] = U0 * sin(x) * cos(y) * cos(z);
        u[nn + n] = -U0 * cos(x) * sin(y) * cos(z);
        u[2 * nn + n] = 0.0;
        rho[n] = rho0 * (1.0 + C / 16.0 * (cos(2 * x) + cos(2 * y)) * (cos(2 * z) + 2.0));
        T[n] = T0;
    }
    for (d = 0; d < 3; ++d) free(xs[d]);
}

/* One step from the Taylor-Green equilibrium state, evaluated only at the listed nodes:
 * the initial populations are f_i^eq and (2C_v - D) T f_i^eq of the Sec. III.C fields,
 * computed on demand at each support point a departure cell needs; the streamed values
 * then go through the collision.  out[k*90 + q] is population q of node nodes[k] after
 * the step.  Lets full-size runs be checked on a sample without the full state.      */
void orc_tgv_step_sample(const orc_cfg *g, double U0, double rho0, double T0, double C,
                         int nsample, const long *nodes, double *out)
{
    const int p = g->p;
    const int N[3] = {g->cells[0] * p, g->cells[1] * p, g->cells[2] * p};
    const double gfac_c = 2.0 / (g->gamma - 1.0) - 3.0;
    double xi[3 * ORC_Q], w[ORC_Q];
    double *xs[3];
    int d;
    orc_velset(xi, w);
    for (d = 0; d < 3; ++d) {
        xs[d] = (double *)malloc(sizeof(double) * N[d]);
        orc_node_coords(g, d, xs[d]);
    }
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < nsample; ++k) {
        long n = nodes[k];
        int node[3], base[3], i, j, kk, l;
        double ell[3][16], f[ORC_Q], gg[ORC_Q];
        node[0] = (int)(n % N[0]);
        node[1] = (int)((n / N[0]) % N[1]);
        node[2] = (int)(n / ((long)N[0] * N[1]));
        for (i = 0; i < ORC_Q; ++i) {
            double af = 0.0, ag = 0.0;
            orc_departure(g, xs, node, xi + 3 * i, base, ell);
            for (l = 0; l <= p; ++l)
                for (kk = 0; kk <= p; ++kk)
                    for (j = 0; j <= p; ++j) {
                        double x = xs[0][wrap(base[0] + j, N[0])];
                        double y = xs[1][wrap(base[1] + kk, N[1])];
                        double z = xs[2][wrap(base[2] + l, N[2])];
                        double u[3], rho, fe, wt = ell[0][j] * ell[1][kk] * ell[2][l];
                        u[0] = U0 * sin(x) * cos(y) * cos(z);
                        u[1] = -U0 * cos(x) * sin(y) * cos(z);
                        u[2] = 0.0;
                        rho = rho0 * (1.0 + C / 16.0 * (cos(2 * x) + cos(2 * y)) * (cos(2 * z) + 2.0));
                        fe = orc_feq_one(xi + 3 * i, w[i], rho, u, T0);
                        af += wt * fe;
                        ag += wt * gfac_c * T0 * fe;
                    }
            f[i] = af;
            gg[i] = ag;
        }
        if (g->collide) orc_collide_one(g, xi, w, f, gg);
        for (i = 0; i < ORC_Q; ++i) {
            out[(long)k * 2 * ORC_Q + i] = f[i];
            out[(long)k * 2 * ORC_Q + ORC_Q + i] = gg[i];
        }
    }
    for (d = 0; d < 3; ++d) free(xs[d]);
}

/* Diagnostics, Sec. III.C, normalised by the domain volume |S| and by U0:
 *   out[0] = E_k   = <rho |u|^2 / 2> / (rho_ref U0^2)
 *   out[1] = eps_s = <(mu/mu_inf) |curl u|^2> / (rho_ref Re U0^2)
 *   out[2] = eps_c = (4/3) <(mu/mu_inf) (div u)^2> / (rho_ref Re U0^2)
 * <.> is (1/|S|) times the sum over cells of the interpolatory quadrature on the
 * cell's (p+1)^3 support points; gradients are derivatives of the cell-local
 * interpolation polynomials (Sec. III.C.2 uses the same, discontinuous, gradients). */
void orc_diag(const orc_cfg *g, const double *pop, double rho_ref, double Re, double U0,
              double *out)
{
    const int p = g->p;
    const int N[3] = {g->cells[0] * p, g->cells[1] * p, g->cells[2] * p};
    const long nn = (long)N[0] * N[1] * N[2];
    const long ncell = (long)g->cells[0] * g->cells[1] * g->cells[2];
    double *rho = (double *)malloc(sizeof(double) * nn);
    double *u = (double *)malloc(sizeof(double) * 3 * nn);
    double *T = (double *)malloc(sizeof(double) * nn);
    double W[16], D[16][16], nodes[16];
    double ek = 0.0, es = 0.0, ec = 0.0, vol = g->L[0] * g->L[1] * g->L[2];
    double h[3];
    int a, d;
    orc_moments(g, pop, rho, u, T);
    orc_quad_weights(p, W);
    orc_glc(p, nodes);
    for (a = 0; a <= p; ++a) orc_lagrange_deriv(p, nodes[a], D[a]);
    for (d = 0; d < 3; ++d) h[d] = g->L[d] / g->cells[d];
#pragma omp parallel for reduction(+ : ek, es, ec) schedule(static)
    for (long cell = 0; cell < ncell; ++cell) {
        int cx = (int)(cell % g->cells[0]);
        int cy = (int)((cell / g->cells[0]) % g->cells[1]);
        int cz = (int)(cell / ((long)g->cells[0] * g->cells[1]));
        int ia, ib, ic, j, comp;
        for (ic = 0; ic <= p; ++ic)
            for (ib = 0; ib <= p; ++ib)
                for (ia = 0; ia <= p; ++ia) {
                    int nx = wrap(cx * p + ia, N[0]), ny = wrap(cy * p + ib, N[1]),
                        nz = wrap(cz * p + ic, N[2]);
                    long n = ((long)nz * N[1] + ny) * N[0] + nx;
                    double grad[3][3]; /* grad[comp][dir] = d u_comp / d x_dir */
                    double wq = W[ia] * W[ib] * W[ic] * h[0] * h[1] * h[2] / 8.0;
                    double usq = u[n] * u[n] + u[nn + n] * u[nn + n] + u[2 * nn + n] * u[2 * nn + n];
                    double mut = orc_sutherland(T[n]);
                    double cx_, cy_, cz_, dv;
                    for (comp = 0; comp < 3; ++comp) {
                        double sx = 0, sy = 0, sz = 0;
                        for (j = 0; j <= p; ++j) {
                            long mx = ((long)nz * N[1] + ny) * N[0] + wrap(cx * p + j, N[0]);
                            long my = ((long)nz * N[1] + wrap(cy * p + j, N[1])) * N[0] + nx;
                            long mz = ((long)wrap(cz * p + j, N[2]) * N[1] + ny) * N[0] + nx;
                            sx += D[ia][j] * u[comp * nn + mx];
                            sy += D[ib][j] * u[comp * nn + my];
                            sz += D[ic][j] * u[comp * nn + mz];
                        }
                        grad[comp][0] = sx * 2.0 / h[0];
                        grad[comp][1] = sy * 2.0 / h[1];
                        grad[comp][2] = sz * 2.0 / h[2];
                    }
                    cx_ = grad[2][1] - grad[1][2];
                    cy_ = grad[0][2] - grad[2][0];
                    cz_ = grad[1][0] - grad[0][1];
                    dv = grad[0][0] + grad[1][1] + grad[2][2];
                    ek += wq * 0.5 * rho[n] * usq;
                    es += wq * mut * (cx_ * cx_ + cy_ * cy_ + cz_ * cz_);
                    ec += wq * mut * dv * dv;
                }
    }
    out[0] = ek / vol / (rho_ref * U0 * U0);
    out[1] = es / vol / (rho_ref * Re * U0 * U0);
    out[2] = 4.0 / 3.0 * ec / vol / (rho_ref * Re * U0 * U0);
    free(rho); free(u); free(T);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Adjoint (reverse mode) of the step.  The paper has no adjoint: each function below is
 * the transpose of the derivative of a forward function above, built by the plainest
 * route available, so that it can be checked by eye against its definition:
 *   - streaming: the literal transpose of orc_stream -- every weight with which a
 *     support value was gathered is used to scatter the adjoint back to that value;
 *   - collision: the node-local Jacobian of orc_collide_one (90 inputs and mu_inf) by
 *     central differences with one Richardson extrapolation step (error O(delta^4)),
 *     transposed and applied to the adjoint;
 *   - kinetic energy: the derivative of the E_k quadrature sum of orc_diag, cell by cell;
 *   - equilibrium initialisation: the Jacobian of orc_feq in (rho, u, T) by the same
 *     extrapolated central differences.                                                */

/* lam_src = S^T lam_dst, with S = orc_stream (same arguments and layout). */
void orc_stream_adjoint(const orc_cfg *g, int nh, int nvel, const double *xi,
                        const double *lam_dst, double *lam_src)
{
    const int p = g->p;
    const int N[3] = {g->cells[0] * p, g->cells[1] * p, g->cells[2] * p};
    const long nn = (long)N[0] * N[1] * N[2];
    double *xs[3];
    int d;
    for (d = 0; d < 3; ++d) {
        xs[d] = (double *)malloc(sizeof(double) * N[d]);
        orc_node_coords(g, d, xs[d]);
    }
    memset(lam_src, 0, sizeof(double) * (size_t)nh * nvel * nn);
    /* one velocity/population slice per thread: the scatter stays inside the slice */
#pragma omp parallel for schedule(static)
    for (int hq = 0; hq < nh * nvel; ++hq) {
        const int i = hq % nvel;
        const double *in = lam_dst + (long)hq * nn;
        double *out = lam_src + (long)hq * nn;
        for (long n = 0; n < nn; ++n) {
            int node[3], base[3], j, k, l;
            double ell[3][16];
            node[0] = (int)(n % N[0]);
            node[1] = (int)((n / N[0]) % N[1]);
            node[2] = (int)(n / ((long)N[0] * N[1]));
            orc_departure(g, xs, node, xi + 3 * i, base, ell);
            for (l = 0; l <= p; ++l)
                for (k = 0; k <= p; ++k)
                    for (j = 0; j <= p; ++j) {
                        int sx = wrap(base[0] + j, N[0]);
                        int sy = wrap(base[1] + k, N[1]);
                        int sz = wrap(base[2] + l, N[2]);
                        out[((long)sz * N[1] + sy) * N[0] + sx]
                            += ell[0][j] * ell[1][k] * ell[2][l] * in[n];
                    }
        }
    }
    for (d = 0; d < 3; ++d) free(xs[d]);
}

/* Collision of one node as a function of its 90 inputs x = (f_0..f_44, g_0..g_44) and of
 * mu_inf: y = orc_collide_one(x). */
static void orc_collide_eval(const orc_cfg *g, const double *xi, const double *w,
                             const double *x, double mu_inf, double *y)
{
    orc_cfg gc = *g;
    gc.mu_inf = mu_inf;
    memcpy(y, x, sizeof(double) * 2 * ORC_Q);
    orc_collide_one(&gc, xi, w, y, y + ORC_Q);
}

/* Richardson-extrapolated central difference of the collision along input k (k < 90) or
 * along mu_inf (k == 90): D = (4 D(delta/2) - D(delta)) / 3.                            */
static void orc_collide_ddir(const orc_cfg *g, const double *xi, const double *w,
                             const double *x, int k, double delta, double *dy)
{
    double xp[2 * ORC_Q], yp[2 * ORC_Q], ym[2 * ORC_Q], d1[2 * ORC_Q];
    int pass, m;
    for (pass = 0; pass < 2; ++pass) {
        const double e = pass == 0 ? delta : 0.5 * delta;
        double mu_p = g->mu_inf, mu_m = g->mu_inf;
        memcpy(xp, x, sizeof(xp));
        if (k < 2 * ORC_Q) xp[k] = x[k] + e; else mu_p = g->mu_inf + e;
        orc_collide_eval(g, xi, w, xp, mu_p, yp);
        memcpy(xp, x, sizeof(xp));
        if (k < 2 * ORC_Q) xp[k] = x[k] - e; else mu_m = g->mu_inf - e;
        orc_collide_eval(g, xi, w, xp, mu_m, ym);
        for (m = 0; m < 2 * ORC_Q; ++m) {
            double dm = (yp[m] - ym[m]) / (2.0 * e);
            if (pass == 0) d1[m] = dm;
            else dy[m] = (4.0 * dm - d1[m]) / 3.0;
        }
    }
}

/* Vector-Jacobian product of the collision at every node: for streamed populations h
 * and the adjoint lam of the collided populations (both [2][45][nodes]), out = J^T lam
 * with J = d collide / d h, and dmu[0] = sum over nodes of lam . d collide / d mu_inf. */
void orc_collide_vjp(const orc_cfg *g, const double *h, const double *lam, double *out,
                     double *dmu)
{
    double xi[3 * ORC_Q], w[ORC_Q];
    const long nn = orc_nodes(g);
    double total = 0.0;
    orc_velset(xi, w);
#pragma omp parallel for reduction(+ : total) schedule(dynamic, 1)
    for (long n = 0; n < nn; ++n) {
        double x[2 * ORC_Q], l[2 * ORC_Q], dy[2 * ORC_Q];
        int k, m;
        for (k = 0; k < 2 * ORC_Q; ++k) {
            x[k] = h[(long)k * nn + n];
            l[k] = lam[(long)k * nn + n];
        }
        for (k = 0; k <= 2 * ORC_Q; ++k) {
            double s = 0.0;
            orc_collide_ddir(g, xi, w, x, k, k < 2 * ORC_Q ? 1e-4 : 1e-3 * g->mu_inf, dy);
            for (m = 0; m < 2 * ORC_Q; ++m) s += l[m] * dy[m];
            if (k < 2 * ORC_Q) out[(long)k * nn + n] = s;
            else total += s;
        }
    }
    *dmu = total;
}

/* dE_k / d pop for E_k as orc_diag defines it (out[0] there): the f entries of cell
 * point n collect w_q (xi_i . u - |u|^2/2) / (|S| rho_ref U0^2) from every cell that has
 * n as a support point; the g entries are zero.                                        */
void orc_ek_grad(const orc_cfg *g, const double *pop, double rho_ref, double U0, double *lam)
{
    const int p = g->p;
    const int N[3] = {g->cells[0] * p, g->cells[1] * p, g->cells[2] * p};
    const long nn = (long)N[0] * N[1] * N[2];
    double *rho = (double *)malloc(sizeof(double) * nn);
    double *u = (double *)malloc(sizeof(double) * 3 * nn);
    double *T = (double *)malloc(sizeof(double) * nn);
    double xi[3 * ORC_Q], w[ORC_Q], W[16], h[3];
    const double vol = g->L[0] * g->L[1] * g->L[2];
    long cell, ncell = (long)g->cells[0] * g->cells[1] * g->cells[2];
    int d;
    orc_velset(xi, w);
    orc_moments(g, pop, rho, u, T);
    orc_quad_weights(p, W);
    for (d = 0; d < 3; ++d) h[d] = g->L[d] / g->cells[d];
    memset(lam, 0, sizeof(double) * 2 * ORC_Q * nn);
    for (cell = 0; cell < ncell; ++cell) {
        int cx = (int)(cell % g->cells[0]);
        int cy = (int)((cell / g->cells[0]) % g->cells[1]);
        int cz = (int)(cell / ((long)g->cells[0] * g->cells[1]));
        int ia, ib, ic, i;
        for (ic = 0; ic <= p; ++ic)
            for (ib = 0; ib <= p; ++ib)
                for (ia = 0; ia <= p; ++ia) {
                    int nx = wrap(cx * p + ia, N[0]), ny = wrap(cy * p + ib, N[1]),
                        nz = wrap(cz * p + ic, N[2]);
                    long n = ((long)nz * N[1] + ny) * N[0] + nx;
                    double wq = W[ia] * W[ib] * W[ic] * h[0] * h[1] * h[2] / 8.0;
                    double ux = u[n], uy = u[nn + n], uz = u[2 * nn + n];
                    double usq = ux * ux + uy * uy + uz * uz;
                    double s = wq / (vol * rho_ref * U0 * U0);
                    for (i = 0; i < ORC_Q; ++i)
                        lam[(long)i * nn + n] += s * (xi[3 * i] * ux + xi[3 * i + 1] * uy
                                                      + xi[3 * i + 2] * uz - 0.5 * usq);
                }
    }
    free(rho); free(u); free(T);
}

/* Derivative of a weighted sum of the diagnostics of orc_diag,
 *   J = wk E_k + ws eps_s + wc eps_c,
 * with respect to the populations: lam = dJ/dpop ([2][45][nodes], f then g).  Written as
 * the chain rule through the node fields, in scatter form, cell by cell:
 *   - E_k's integrand at a quadrature point, rho |u|^2 / 2, sends |u|^2/2 to the point's
 *     rho adjoint and rho u to its u adjoint;
 *   - eps_s's and eps_c's integrands, mu~(T) |curl u|^2 and (4/3) mu~(T) (div u)^2, send
 *     mu~'(T) times the squared quantity to the point's T adjoint, and their derivative with
 *     respect to each gradient entry d u_c / d x_d at the point to the u_c adjoint of every
 *     support point on the point's line along d, with the cell-local Lagrange derivative
 *     weight (2/h_d) D[a][j] the forward gradient used;
 *   - then each node's (rho, u, T) adjoint becomes population adjoints through the moments
 *     rho = sum f, rho u = sum f xi, 2 C_v rho T + rho |u|^2 = sum (f |xi|^2 + g):
 *     d rho/d f_i = 1, d u/d f_i = (xi_i - u)/rho, d T/d f_i = (|xi_i - u|^2 - 2 C_v T)/(2 C_v rho),
 *     d T/d g_i = 1/(2 C_v rho), d u/d g_i = d rho/d g_i = 0.
 * mu~ is the Sutherland law of orc_sutherland; its derivative is taken analytically from
 * the printed law.                                                                     */
void orc_diag_grad(const orc_cfg *g, const double *pop, double rho_ref, double Re, double U0,
                   double wk, double ws, double wc, double *lam)
{
    const int p = g->p;
    const int N[3] = {g->cells[0] * p, g->cells[1] * p, g->cells[2] * p};
    const long nn = (long)N[0] * N[1] * N[2];
    const long ncell = (long)g->cells[0] * g->cells[1] * g->cells[2];
    const double two_cv = 2.0 / (g->gamma - 1.0);
    double *rho = (double *)malloc(sizeof(double) * nn);
    double *u = (double *)malloc(sizeof(double) * 3 * nn);
    double *T = (double *)malloc(sizeof(double) * nn);
    double *a_rho = (double *)calloc((size_t)nn, sizeof(double));
    double *a_u = (double *)calloc((size_t)3 * nn, sizeof(double));
    double *a_T = (double *)calloc((size_t)nn, sizeof(double));
    double xi[3 * ORC_Q], w[ORC_Q], W[16], D[16][16], nodes[16], h[3];
    const double vol = g->L[0] * g->L[1] * g->L[2];
    const double ke = wk / (vol * rho_ref * U0 * U0);
    const double ks = ws / (vol * rho_ref * Re * U0 * U0);
    const double kc = wc * 4.0 / 3.0 / (vol * rho_ref * Re * U0 * U0);
    long cell, n;
    int a, d, i;
    orc_velset(xi, w);
    orc_moments(g, pop, rho, u, T);
    orc_quad_weights(p, W);
    orc_glc(p, nodes);
    for (a = 0; a <= p; ++a) orc_lagrange_deriv(p, nodes[a], D[a]);
    for (d = 0; d < 3; ++d) h[d] = g->L[d] / g->cells[d];
    for (cell = 0; cell < ncell; ++cell) {
        int c[3], loc[3], comp, j;
        c[0] = (int)(cell % g->cells[0]);
        c[1] = (int)((cell / g->cells[0]) % g->cells[1]);
        c[2] = (int)(cell / ((long)g->cells[0] * g->cells[1]));
        for (loc[2] = 0; loc[2] <= p; ++loc[2])
            for (loc[1] = 0; loc[1] <= p; ++loc[1])
                for (loc[0] = 0; loc[0] <= p; ++loc[0]) {
                    long line[3][16]; /* node index of support point j on the point's line along d */
                    double grad[3][3], om[3], dv, usq, mut, dmut, wq, G;
                    long nq;
                    for (d = 0; d < 3; ++d)
                        for (j = 0; j <= p; ++j) {
                            int m[3];
                            m[0] = wrap(c[0] * p + (d == 0 ? j : loc[0]), N[0]);
                            m[1] = wrap(c[1] * p + (d == 1 ? j : loc[1]), N[1]);
                            m[2] = wrap(c[2] * p + (d == 2 ? j : loc[2]), N[2]);
                            line[d][j] = ((long)m[2] * N[1] + m[1]) * N[0] + m[0];
                        }
                    nq = line[0][loc[0]];
                    wq = W[loc[0]] * W[loc[1]] * W[loc[2]] * h[0] * h[1] * h[2] / 8.0;
                    for (comp = 0; comp < 3; ++comp)
                        for (d = 0; d < 3; ++d) {
                            double sacc = 0.0;
                            for (j = 0; j <= p; ++j) sacc += D[loc[d]][j] * u[comp * nn + line[d][j]];
                            grad[comp][d] = sacc * 2.0 / h[d];
                        }
                    om[0] = grad[2][1] - grad[1][2];
                    om[1] = grad[0][2] - grad[2][0];
                    om[2] = grad[1][0] - grad[0][1];
                    dv = grad[0][0] + grad[1][1] + grad[2][2];
                    usq = u[nq] * u[nq] + u[nn + nq] * u[nn + nq] + u[2 * nn + nq] * u[2 * nn + nq];
                    mut = orc_sutherland(T[nq]);
                    /* mu~ = A T^1.5 / (T + B): d mu~/dT = mu~ (1.5/T - 1/(T + B)) */
                    dmut = mut * (1.5 / T[nq] - 1.0 / (T[nq] + 0.40417));
                    /* kinetic energy */
                    a_rho[nq] += wq * ke * 0.5 * usq;
                    for (comp = 0; comp < 3; ++comp) a_u[comp * nn + nq] += wq * ke * rho[nq] * u[comp * nn + nq];
                    /* temperature through the Sutherland factor */
                    a_T[nq] += wq * dmut * (ks * (om[0] * om[0] + om[1] * om[1] + om[2] * om[2]) + kc * dv * dv);
                    /* gradient entries: dJ/dgrad[comp][d] */
                    for (comp = 0; comp < 3; ++comp)
                        for (d = 0; d < 3; ++d) {
                            double dcurl = 0.0;
                            if (comp == 2 && d == 1) dcurl = 2.0 * om[0];
                            if (comp == 1 && d == 2) dcurl = -2.0 * om[0];
                            if (comp == 0 && d == 2) dcurl = 2.0 * om[1];
                            if (comp == 2 && d == 0) dcurl = -2.0 * om[1];
                            if (comp == 1 && d == 0) dcurl = 2.0 * om[2];
                            if (comp == 0 && d == 1) dcurl = -2.0 * om[2];
                            G = wq * mut * (ks * dcurl + kc * (comp == d ? 2.0 * dv : 0.0));
                            if (G == 0.0) continue;
                            for (j = 0; j <= p; ++j)
                                a_u[comp * nn + line[d][j]] += G * D[loc[d]][j] * 2.0 / h[d];
                        }
                }
    }
    for (n = 0; n < nn; ++n) {
        const double r = rho[n], ux = u[n], uy = u[nn + n], uz = u[2 * nn + n];
        for (i = 0; i < ORC_Q; ++i) {
            const double cx = xi[3 * i] - ux, cy = xi[3 * i + 1] - uy, cz = xi[3 * i + 2] - uz;
            lam[(long)i * nn + n] = a_rho[n] + (a_u[n] * cx + a_u[nn + n] * cy + a_u[2 * nn + n] * cz) / r
                                  + a_T[n] * (cx * cx + cy * cy + cz * cz - two_cv * T[n]) / (two_cv * r);
            lam[(long)(ORC_Q + i) * nn + n] = a_T[n] / (two_cv * r);
        }
    }
    free(rho); free(u); free(T); free(a_rho); free(a_u); free(a_T);
}

/* Transpose of orc_init_fields: grad_rho[n], grad_u[3][n], grad_T[n] = the derivatives of
 * sum_i (lam_f_i f_i + lam_g_i g_i) at node n with respect to rho, u, T there, where
 * f_i = f_i^eq(rho, u, T) and g_i = (2C_v - D) T f_i^eq.                                */
void orc_init_fields_vjp(const orc_cfg *g, const double *rho, const double *u,
                         const double *T, const double *lam, double *grad_rho,
                         double *grad_u, double *grad_T)
{
    double xi[3 * ORC_Q], w[ORC_Q];
    const long nn = orc_nodes(g);
    const double gfac_c = 2.0 / (g->gamma - 1.0) - 3.0;
    orc_velset(xi, w);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < nn; ++n) {
        double q0[5] = {rho[n], u[n], u[nn + n], u[2 * nn + n], T[n]};
        double grad[5];
        int k, pass, i;
        for (k = 0; k < 5; ++k) {
            const double delta = 1e-4;
            double d1 = 0.0, dd = 0.0;
            for (pass = 0; pass < 2; ++pass) {
                const double e = pass == 0 ? delta : 0.5 * delta;
                double qp[5], qm[5], fp[ORC_Q], fm[ORC_Q], s = 0.0;
                memcpy(qp, q0, sizeof(qp));
                memcpy(qm, q0, sizeof(qm));
                qp[k] += e;
                qm[k] -= e;
                orc_feq(xi, w, ORC_Q, qp[0], qp + 1, qp[4], fp);
                orc_feq(xi, w, ORC_Q, qm[0], qm + 1, qm[4], fm);
                for (i = 0; i < ORC_Q; ++i) {
                    double lf = lam[(long)i * nn + n], lg = lam[(long)(ORC_Q + i) * nn + n];
                    s += lf * (fp[i] - fm[i]) + lg * gfac_c * (qp[4] * fp[i] - qm[4] * fm[i]);
                }
                s /= 2.0 * e;
                if (pass == 0) d1 = s;
                else dd = (4.0 * s - d1) / 3.0;
            }
            grad[k] = dd;
        }
        grad_rho[n] = grad[0];
        grad_u[n] = grad[1];
        grad_u[nn + n] = grad[2];
        grad_u[2 * nn + n] = grad[3];
        grad_T[n] = grad[4];
    }
}
