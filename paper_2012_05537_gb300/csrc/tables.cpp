// Host-side constant tables of the SLLBM step (see tables.h).
#include "tables.h"

#include <cmath>

namespace sllbm {

namespace {

const double kPi = 3.14159265358979323846;

// Appends the three cyclic rotations (a,b,c) -> (b,c,a) -> (c,a,b) of one direction.
int push_rotations(double xi[kQ][3], double w[kQ], int i, const double v[3], double radius,
                   double weight, bool right_rotation) {
    double n = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int r = 0; r < 3; ++r) {
        for (int d = 0; d < 3; ++d) {
            int src = right_rotation ? (d - r + 3) % 3 : (d + r) % 3;
            xi[i][d] = radius * v[src] / n;
        }
        w[i++] = weight;
    }
    return i;
}

}  // namespace

// Sec. II.B / Fig. 2: degree-9 cubature for the Gaussian weight with 45 abscissae and
// icosahedral symmetry (after Konyaev).  Four orbits for the unit-variance Gaussian:
// the origin, an icosahedron of radius sqrt(3), the dual dodecahedron of radius 3 and
// an icosahedron of radius sqrt(15); the weights are the closed-form solution of the
// invariant moment equations.  Order (the library's public convention):
//   icosahedron:  for s1, s2 in (+,-): (0,s1,s2 phi) and its two left rotations;
//   dodecahedron: the cube corners (x slowest, + first), then for s1, s2 in (+,-):
//                 (s1/phi, 0, s2 phi), (s1 phi, s2/phi, 0) and the right rotation of
//                 the latter.
void build_velocity_set(double xi[kQ][3], double w[kQ]) {
    const double phi = 0.5 * (1.0 + std::sqrt(5.0));
    const double r_in = std::sqrt(3.0), r_mid = 3.0, r_out = std::sqrt(15.0);
    const double w0 = 28.0 / 135.0, w_in = 25.0 / 432.0, w_mid = 1.0 / 216.0,
                 w_out = 1.0 / 2160.0;
    const double sgn[2] = {1.0, -1.0};
    int i = 0;
    xi[0][0] = xi[0][1] = xi[0][2] = 0.0;
    w[i++] = w0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            // dodecahedron between the two icosahedra
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int c = 0; c < 2; ++c) {
                        double n = std::sqrt(3.0);
                        xi[i][0] = r_mid * sgn[a] / n;
                        xi[i][1] = r_mid * sgn[b] / n;
                        xi[i][2] = r_mid * sgn[c] / n;
                        w[i++] = w_mid;
                    }
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    double first[3] = {sgn[a] / phi, 0.0, sgn[b] * phi};
                    double n = std::sqrt(first[0] * first[0] + first[2] * first[2]);
                    for (int d = 0; d < 3; ++d) xi[i][d] = r_mid * first[d] / n;
                    w[i++] = w_mid;
                    double second[3] = {sgn[a] * phi, sgn[b] / phi, 0.0};
                    // second and its right rotation (c,a,b)
                    double n2 = std::sqrt(second[0] * second[0] + second[1] * second[1]);
                    for (int d = 0; d < 3; ++d) xi[i][d] = r_mid * second[d] / n2;
                    w[i++] = w_mid;
                    for (int d = 0; d < 3; ++d) xi[i][d] = r_mid * second[(d + 2) % 3] / n2;
                    w[i++] = w_mid;
                }
        }
        const double radius = pass == 0 ? r_in : r_out;
        const double weight = pass == 0 ? w_in : w_out;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double v[3] = {0.0, sgn[a], sgn[b] * phi};
                i = push_rotations(xi, w, i, v, radius, weight, false);
            }
    }
}

void glc_points(int p, double* r) {
    for (int a = 0; a <= p; ++a) r[a] = -std::cos(kPi * a / p);
}

// Barycentric Lagrange evaluation (Berrut & Trefethen): psi_j(r) = (b_j/(r-r_j)) /
// sum_k b_k/(r-r_k) with b_j = 1/prod_{k!=j}(r_j - r_k); exact Kronecker at nodes.
void lagrange_at(int p, double r, double* ell) {
    double x[kMaxP + 1], b[kMaxP + 1];
    glc_points(p, x);
    for (int j = 0; j <= p; ++j) {
        double prod = 1.0;
        for (int k = 0; k <= p; ++k)
            if (k != j) prod *= (x[j] - x[k]);
        b[j] = 1.0 / prod;
    }
    for (int j = 0; j <= p; ++j)
        if (r == x[j]) {
            for (int k = 0; k <= p; ++k) ell[k] = (k == j) ? 1.0 : 0.0;
            return;
        }
    double den = 0.0;
    for (int j = 0; j <= p; ++j) den += b[j] / (r - x[j]);
    for (int j = 0; j <= p; ++j) ell[j] = (b[j] / (r - x[j])) / den;
}

// Clenshaw-Curtis weights for the n+1 Chebyshev extrema, closed form
// W_j = (c_j/n) [1 - sum_{k=1}^{n/2} b_k cos(2 k theta_j) / (4 k^2 - 1)],
// c_j = 1 at the ends and 2 inside, b_k = 1 for k = n/2 (n even) and 2 otherwise.
// theta_j = pi j / n; the points -cos(theta_j) are the GLC points in ascending order.
void clenshaw_curtis(int p, double* W) {
    const int n = p;
    for (int j = 0; j <= n; ++j) {
        double theta = kPi * j / n;
        double s = 0.0;
        for (int k = 1; k <= n / 2; ++k) {
            double bk = (2 * k == n) ? 1.0 : 2.0;
            s += bk * std::cos(2.0 * k * theta) / (4.0 * k * k - 1.0);
        }
        double cj = (j == 0 || j == n) ? 1.0 : 2.0;
        W[j] = cj / n * (1.0 - s);
    }
}

// D[a][j] = psi_j'(r_a) = (b_j/b_a)/(r_a - r_j) for a != j, D[a][a] = -sum_{j!=a} D[a][j].
void diff_matrix(int p, double D[kMaxP + 1][kMaxP + 1]) {
    double x[kMaxP + 1], b[kMaxP + 1];
    glc_points(p, x);
    for (int j = 0; j <= p; ++j) {
        double prod = 1.0;
        for (int k = 0; k <= p; ++k)
            if (k != j) prod *= (x[j] - x[k]);
        b[j] = 1.0 / prod;
    }
    for (int a = 0; a <= p; ++a) {
        double diag = 0.0;
        for (int j = 0; j <= p; ++j) {
            if (j == a) continue;
            D[a][j] = (b[j] / b[a]) / (x[a] - x[j]);
            diag -= D[a][j];
        }
        D[a][a] = diag;
    }
}

// Uniform-mesh form of the departure search and of Psi_i (Sec. II.A, Sec. IV.B): the
// departure point of local node a of any cell c is c*h + x_a - dt*xi; its cell offset
// and reference coordinate do not depend on c, so one row per (velocity, a) suffices.
void build_dir_table(int p, double h, double dt, const double xi[kQ][3], int dir,
                     DirTable* out) {
    double r[kMaxP + 1];
    glc_points(p, r);
    for (int i = 0; i < kQ; ++i)
        for (int a = 0; a < p; ++a) {
            double xa = 0.5 * (r[a] + 1.0) * h;           // node position inside cell 0
            double y = (xa - dt * xi[i][dir]) / h;        // departure, in cell units
            double cell = std::floor(y);
            double ref = 2.0 * (y - cell) - 1.0;          // reference coordinate in [-1,1)
            out->shift[i][a] = static_cast<int>(cell);
            lagrange_at(p, ref, out->weight[i][a]);
        }
}

}  // namespace sllbm
