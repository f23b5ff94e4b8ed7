// Host-side constant tables of the SLLBM step: velocity set, support points,
// separable interpolation tables, quadrature and derivative matrices.
// All built once per context in FP64 on the host; the kernels receive them by value.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define SLLBM_HD __host__ __device__
#else
#define SLLBM_HD
#endif

namespace sllbm {

constexpr int kQ = 45;      // velocities of the degree-9 cubature set (Sec. II.B)
constexpr int kMaxP = 4;    // largest supported polynomial order

SLLBM_HD constexpr int shell_of(int i) {
    return i < 1 ? 0 : (i < 13 ? 1 : (i < 33 ? 2 : 3));
}

// Velocity set: xi[45][3], w[45] in the canonical order.
void build_velocity_set(double xi[kQ][3], double w[kQ]);

// Gauss-Lobatto-Chebyshev points r_a = -cos(pi a/p), a = 0..p, on [-1, 1].
void glc_points(int p, double* r);

// Lagrange basis on the GLC points evaluated at r, barycentric form.
void lagrange_at(int p, double r, double* ell);

// Clenshaw-Curtis weights on the GLC points (closed-form cosine series), sum = 2.
void clenshaw_curtis(int p, double* W);

// Differentiation matrix D[a][j] = d psi_j/dr at r_a (barycentric formula).
void diff_matrix(int p, double D[kMaxP + 1][kMaxP + 1]);

// Separable streaming table for one direction of a uniform periodic mesh with cell
// size h: for every velocity i and local node a in [0,p) the departure point
// x_a - dt*xi_i (x_a measured from the cell's left face) lies in the cell shifted by
// shift[i][a] cells, at reference coordinate r; weight[i][a][j] = psi_j(r).
struct DirTable {
    int shift[kQ][kMaxP];
    double weight[kQ][kMaxP][kMaxP + 1];
};
void build_dir_table(int p, double h, double dt, const double xi[kQ][3], int dir, DirTable* out);

}  // namespace sllbm
