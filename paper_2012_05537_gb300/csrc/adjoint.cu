// Reverse mode of the SLLBM step (the paper has no adjoint): the transposes of the
// derivatives of the forward operators, for FP32 and FP64 storage without the Prandtl term.
//
//   * streaming S = S_x S_y S_z per velocity (Eq. interpolation on the uniform mesh: each
//     1D factor gathers p+1 support values of the departure cell with the precomputed
//     Lagrange weights).  Its transpose, in gather form: node m = c p + b receives w[a][b]
//     from every node (c - k_a) p + a, and for b = 0 also w[a][p] from (c - 1 - k_a) p + a
//     (the right-face support point of the cell to the left).  No atomics, each output
//     written once.  FP32: a tile kernel (the three transposed passes in registers and shared
//     memory); FP64 arithmetic: three 1D pass kernels.
//   * collision (Eq. LBM with Eq. moments, Eq. discreteEquilibrium in its quartic form,
//     tau = mu/(P dt) + 1/2, Sutherland mu): a node-local vector-Jacobian product through
//     the primitive variables rho, u, T and omega, derived by hand below.
//   * kinetic-energy seed and the transpose of the equilibrium initialisation.
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

#include "collide.cuh"
#include "sllbm_internal.h"
#include "trace.h"
#include "step_kernel.cuh"
#include "tables.h"

namespace sllbm {

namespace {

struct AdjVel {
    double xi[kQ][3];
    double w[kQ];
};

template <typename C>
struct PassTable {
    int shift[kQ][kMaxP];
    C w[kQ][kMaxP][kMaxP + 1];
};

template <typename C>
struct Pair;
template <>
struct Pair<float> {
    using T = float2;
};
template <>
struct Pair<double> {
    using T = double2;
};

__device__ __forceinline__ int wrap_mod(int v, int n) {
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// One 1D streaming pass along direction d on pairs (f_i, g_i) in the storage order
// [i][z][y][x][h]: forward (TR = false) out(n) = sum_j w[i][a][j] in((c + k_a) p + j), or its
// transpose (TR = true) as described at the top of the file.
template <typename C, bool TR>
__global__ void __launch_bounds__(256) pass_kernel(const C* __restrict__ in, C* __restrict__ out, int Nx, int Ny,
                                                   int d, int p, int cells_d, long long nn,
                                                   const __grid_constant__ PassTable<C> t) {
    using P2 = typename Pair<C>::T;
    const P2* src = reinterpret_cast<const P2*>(in);
    P2* dst = reinterpret_cast<P2*>(out);
    const long long total = static_cast<long long>(kQ) * nn;
    const long long sxy = static_cast<long long>(Nx) * Ny;
    for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < total;
         k += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int i = static_cast<int>(k / nn);
        const long long n = k - static_cast<long long>(i) * nn;
        const int x = static_cast<int>(n % Nx);
        const int y = static_cast<int>((n / Nx) % Ny);
        const int z = static_cast<int>(n / sxy);
        const int coord = d == 0 ? x : (d == 1 ? y : z);
        const long long stride = d == 0 ? 1 : (d == 1 ? Nx : sxy);
        const long long base = static_cast<long long>(i) * nn + (n - coord * stride);
        const int c = coord / p, a = coord - c * p;
        C af = 0, ag = 0;
        if (!TR) {
            const int c0 = wrap_mod(c + t.shift[i][a], cells_d);
            for (int j = 0; j <= p; ++j) {
                int m = c0 * p + j;
                if (m >= cells_d * p) m -= cells_d * p;
                const P2 v = src[base + m * stride];
                const C wj = t.w[i][a][j];
                af += wj * v.x;
                ag += wj * v.y;
            }
        } else {
            // here (c, a) is the receiving node: cell c, local index b = a
            const int b = a;
            for (int q = 0; q < p; ++q) {
                const int cs = wrap_mod(c - t.shift[i][q], cells_d);
                const P2 v = src[base + static_cast<long long>(cs * p + q) * stride];
                const C wq = t.w[i][q][b];
                af += wq * v.x;
                ag += wq * v.y;
                if (b == 0) {
                    const int cs1 = wrap_mod(c - 1 - t.shift[i][q], cells_d);
                    const P2 v1 = src[base + static_cast<long long>(cs1 * p + q) * stride];
                    const C wp = t.w[i][q][p];
                    af += wp * v1.x;
                    ag += wp * v1.y;
                }
            }
        }
        P2 r;
        r.x = af;
        r.y = ag;
        dst[k] = r;
    }
}

// Derivatives of the quartic f^eq/(w rho) = c0 + c1 s + c2 s^2 + s^3/6 + s^4/24 of
// collide.cuh with respect to s = xi.u, |u|^2 and th = T - 1 (from the closed forms of c0,
// c1, c2 there).
template <typename C>
struct PolyDeriv {
    C P, ds, dusq, dth;
};

template <typename C>
__device__ __forceinline__ PolyDeriv<C> poly_deriv(const EqCoef<C>& ec, int sh, C s, C usq, C th) {
    const C x2 = C(shell_xi2(sh));
    PolyDeriv<C> r;
    r.P = eq_poly(ec, sh, s);
    r.ds = ec.c1[sh] + s * (C(2) * ec.c2[sh] + s * (C(0.5) + s * C(1.0 / 6.0)));
    r.dusq = (C(-0.5) + C(0.25) * usq + C(0.25) * th * (C(5) - x2)) - C(0.5) * s - C(0.25) * s * s;
    r.dth = (C(0.5) * (x2 - C(3)) + C(0.25) * usq * (C(5) - x2)
             + C(0.25) * th * (x2 * x2 - C(10) * x2 + C(15)))
          + C(0.5) * (x2 - C(5)) * s + C(0.25) * (x2 - C(7)) * s * s;
    return r;
}

struct AdjArgs {
    double mu_over_dt;  // K = mu_inf / dt
    double inv_dt;
    double inv_2cv;
    double gfac;
};

// Vector-Jacobian product of the collision at one node.  h: streamed populations, f_i at
// h[i * hs] and g_i at h[i * hs + hg]; lam: adjoint of the collided populations and out: the
// result (J^T lam), both with f_i at [i * 2 nn] and g_i at [i * 2 nn + 1] (a state buffer's
// pair layout, offset to the node).  Returns the node's lam . d collide / d mu_inf.
//
// Forward (per node):  rho = sum f, j = sum f xi, E2 = sum (f |xi|^2 + g),
//   u = j/rho, T = (E2/rho - |u|^2)/(2 C_v), tau = K su(T)/(rho T) + 1/2, omega = 1/tau,
//   f^eq_i = w_i rho P_i(xi_i.u, |u|^2, T-1), g^eq_i = (2C_v - D) T f^eq_i,
//   f_i' = f_i + omega (f^eq_i - f_i), g_i' = g_i + omega (g^eq_i - g_i).
// Reverse: with B = sum lam . (h^eq - h), the adjoint reaching f^eq_i is
//   A_i = omega (lam_f_i + (2C_v - D) T lam_g_i), T also appears in g^eq explicitly,
//   omega depends on rho and T (and mu_inf); the primitive adjoints are mapped back to the
//   moments (rho, j, E2) and from there to the populations.
template <typename CH, typename C>
__device__ __forceinline__ double vjp_node(const CH* __restrict__ h, long long hs, long long hg,
                                           const C* __restrict__ lam, C* __restrict__ out, long long nn,
                                           const AdjArgs& aa, const AdjVel& v) {
    const C gfac = C(aa.gfac), inv_2cv = C(aa.inv_2cv), K = C(aa.mu_over_dt);
    const long long ls = 2 * nn;
    C rho = 0, jx = 0, jy = 0, jz = 0, E2 = 0;
    for (int i = 0; i < kQ; ++i) {
        const C f = C(h[i * hs]), g = C(h[i * hs + hg]);
        rho += f;
        jx += f * C(v.xi[i][0]);
        jy += f * C(v.xi[i][1]);
        jz += f * C(v.xi[i][2]);
        E2 += f * C(shell_xi2(shell_of(i))) + g;
    }
    const C ux = jx / rho, uy = jy / rho, uz = jz / rho;
    const C usq = ux * ux + uy * uy + uz * uz;
    const C T = (E2 / rho - usq) * inv_2cv;
    const C th = T - C(1);
    const C su = sutherland(T);
    const C tau = K * su / (rho * T) + C(0.5);
    const C om = C(1) / tau;
    const EqCoef<C> ec = eq_coefficients(usq, th);
    C B = 0, ATd = 0, arho = 0, aux = 0, auy = 0, auz = 0, ausq = 0, ath = 0;
    // shell by shell, so that the shell's polynomial coefficients are plain registers
#pragma unroll
    for (int sh = 0; sh < 4; ++sh) {
        const C x2 = C(shell_xi2(sh));
        const C c0 = ec.c0[sh], c1 = ec.c1[sh], c2 = ec.c2[sh];
        const C dusq0 = C(-0.5) + C(0.25) * usq + C(0.25) * th * (C(5) - x2);
        const C dth0 = C(0.5) * (x2 - C(3)) + C(0.25) * usq * (C(5) - x2) + C(0.25) * th * (x2 * x2 - C(10) * x2 + C(15));
        const C dth1 = C(0.5) * (x2 - C(5)), dth2 = C(0.25) * (x2 - C(7));
        // first velocity of each shell in the canonical order: 0, 1, 13, 33, 45
        const int i0 = sh == 0 ? 0 : (sh == 1 ? 1 : (sh == 2 ? 13 : 33));
        const int i1 = sh == 0 ? 1 : (sh == 1 ? 13 : (sh == 2 ? 33 : 45));
#pragma unroll 1
        for (int i = i0; i < i1; ++i) {
            const C x = C(v.xi[i][0]), y = C(v.xi[i][1]), z = C(v.xi[i][2]), w = C(v.w[i]);
            const C s = x * ux + y * uy + z * uz;
            // f^eq_i/(w rho) = c0 + c1 s + c2 s^2 + s^3/6 + s^4/24 and its derivatives
            const C P = c0 + s * (c1 + s * (c2 + s * (C(1.0 / 6.0) + s * C(1.0 / 24.0))));
            const C Ps = c1 + s * (C(2) * c2 + s * (C(0.5) + s * C(1.0 / 6.0)));
            const C Pusq = dusq0 - C(0.5) * s - C(0.25) * s * s;
            const C Pth = dth0 + dth1 * s + dth2 * s * s;
            const C feq = w * rho * P, geq = gfac * T * feq;
            const C lf = lam[i * ls], lg = lam[i * ls + 1];
            const C hf = C(h[i * hs]), hgv = C(h[i * hs + hg]);
            B += lf * (feq - hf) + lg * (geq - hgv);
            const C A = om * (lf + gfac * T * lg);
            ATd += om * gfac * lg * feq;
            const C Aw = A * w;
            arho += Aw * P;
            const C t = Aw * rho * Ps;
            aux += t * x;
            auy += t * y;
            auz += t * z;
            ausq += Aw * rho * Pusq;
            ath += Aw * rho * Pth;
        }
    }
    // omega = 1/tau: d omega/d tau = -omega^2; d ln su/dT = 3/(2T) - 1/(T + S)
    const C dom = -om * om;
    const C dtau_drho = -K * su / (rho * rho * T);
    const C dtau_dT = K * su / (rho * T) * (sutherland_dlog(T) - C(1) / T);
    const double dmu = static_cast<double>(B * dom * su / (rho * T)) * aa.inv_dt;
    C Arho = arho + B * dom * dtau_drho;
    const C AT = ath + ATd + B * dom * dtau_dT;
    C Aux = aux + C(2) * ux * ausq, Auy = auy + C(2) * uy * ausq, Auz = auz + C(2) * uz * ausq;
    // T = (E2/rho - |u|^2)/(2 C_v)
    const C AE2 = AT * inv_2cv / rho;
    Arho -= AT * inv_2cv * E2 / (rho * rho);
    Aux -= C(2) * AT * inv_2cv * ux;
    Auy -= C(2) * AT * inv_2cv * uy;
    Auz -= C(2) * AT * inv_2cv * uz;
    // u = j/rho
    const C Ajx = Aux / rho, Ajy = Auy / rho, Ajz = Auz / rho;
    Arho -= (Aux * ux + Auy * uy + Auz * uz) / rho;
    const C keep = C(1) - om;
    for (int i = 0; i < kQ; ++i) {
        const C x = C(v.xi[i][0]), y = C(v.xi[i][1]), z = C(v.xi[i][2]);
        const C lf = lam[i * ls], lg = lam[i * ls + 1];
        out[i * ls] = keep * lf + Arho + Ajx * x + Ajy * y + Ajz * z + AE2 * C(shell_xi2(shell_of(i)));
        out[i * ls + 1] = keep * lg + AE2;
    }
    return dmu;
}

// Block sum of a per-thread double into partials[blockIdx.x] (blockDim.x a multiple of 32).
__device__ __forceinline__ void block_partial(double x, double* partials) {
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) s += red[w];
        partials[blockIdx.x] = s;
    }
}

// The collision VJP at every node, h already streamed (a state-sized array, pair layout).
template <typename CH, typename C>
__global__ void __launch_bounds__(128) collide_vjp_kernel(const CH* __restrict__ h, const C* __restrict__ lam,
                                                          C* __restrict__ out, long long nn, AdjArgs aa,
                                                          const __grid_constant__ AdjVel v,
                                                          double* __restrict__ partials) {
    double dmu_acc = 0.0;
    for (long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; n < nn;
         n += static_cast<long long>(gridDim.x) * blockDim.x)
        dmu_acc += vjp_node<CH, C>(h + 2 * n, 2 * nn, 1, lam + 2 * n, out + 2 * n, nn, aa, v);
    block_partial(dmu_acc, partials);
}

// ---------------------------------------------------------------- transposed streaming as a tile kernel
// The transposed streaming in gather form: the 1D transpose sends node
//     m = c p + b the values of nodes (c - k_a) p + a with weights w[a][b], and for b = 0 also
//     those of (c - 1 - k_a) p + a with w[a][p]; k_a = kmin + kc[a].  A tile of cells
//     c0..c0+tc-1 therefore reads the cells c0 - 1 - kmin - span .. c0 + tc - 1 - kmin, p nodes
//     each (no shared face).

template <int CX, int CY, int CZ, int P>
struct TransShape {
    static constexpr int TX = CX * P, TY = CY * P, TZ = CZ * P;
    static constexpr int BX = (CX + 2) * P, BY = (CY + 2) * P, BZ = (CZ + 2) * P;  // with span 1
};

template <typename C, int P, int CX, int CY, int CZ, int NW>
struct TransSmem {
    using TS = TransShape<CX, CY, CZ, P>;
    // rows padded to an odd number of pairs (see adj_transpose_kernel)
    static constexpr size_t warp_pairs = size_t(TS::TZ) * TS::BY * (TS::BX | 1);
    static constexpr size_t warp_ints = TS::BX + TS::BY + TS::BZ;
    static constexpr size_t bytes = NW * warp_pairs * sizeof(typename Pair2<C>::T) + NW * warp_ints * sizeof(int);
};

// One transposed 1D pass over a column held in registers (box origin cell c0 - 1 - kmin - span):
// output o = ci P + b gets sum_a w[a][b] v[(ci + 1 + span - kc[a]) P + a], and for b = 0 also
// sum_a w[a][P] v[(ci + span - kc[a]) P + a]; span - kc[a] is 0 or 1 (a register select).
template <typename C, int P, int T, int NV>
__device__ __forceinline__ void transpose_column(const typename Pair2<C>::T (&v)[NV], const C (&w)[P][P + 1],
                                                 const signed char (&kc)[P], bool sp, typename Pair2<C>::T (&r)[T]) {
    static_assert(((T - 1) / P + 2) * P + P - 1 < NV, "column shorter than the support of its outputs");
#pragma unroll
    for (int o = 0; o < T; ++o) {
        const int ci = o / P, b = o % P;
        C fx = 0, fy = 0;
#pragma unroll
        for (int a = 0; a < P; ++a) {
            const bool d1 = sp && kc[a] == 0;
            const C wb = w[a][b];
            fx += wb * (d1 ? v[(ci + 2) * P + a].x : v[(ci + 1) * P + a].x);
            fy += wb * (d1 ? v[(ci + 2) * P + a].y : v[(ci + 1) * P + a].y);
            if (b == 0) {
                const C wp = w[a][P];
                fx += wp * (d1 ? v[(ci + 1) * P + a].x : v[ci * P + a].x);
                fy += wp * (d1 ? v[(ci + 1) * P + a].y : v[ci * P + a].y);
            }
        }
        r[o].x = fx;
        r[o].y = fy;
    }
}

// dst = S^T src (both state-sized arrays of adjoint populations, pair layout), one tile per CTA.
template <typename C, int P, int CX, int CY, int CZ, int NW>
__global__ void __launch_bounds__(NW * 32, kStepMinCtas<C, NW>)
    adj_transpose_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ StepTables<C, P> t) {
    using TS = TransShape<CX, CY, CZ, P>;
    using SM = TransSmem<C, P, CX, CY, CZ, NW>;
    using C2 = typename Pair2<C>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C2* zb = reinterpret_cast<C2*>(smem_raw) + warp * SM::warp_pairs;
    int* xo = reinterpret_cast<int*>(smem_raw + NW * SM::warp_pairs * sizeof(C2)) + warp * SM::warp_ints;
    int* yo = xo + TS::BX;
    int* zo = yo + TS::BY;
    int tile = blockIdx.x;
    const int tix = tile % a.tiles[0];
    tile /= a.tiles[0];
    const int tiy = tile % a.tiles[1];
    const int tiz = tile / a.tiles[1];
    const int c0[3] = {tix * CX, tiy * CY, tiz * CZ};
    const int tc[3] = {min(CX, a.cells[0] - c0[0]), min(CY, a.cells[1] - c0[1]), min(CZ, a.cells[2] - c0[2])};
    const int te[3] = {tc[0] * P, tc[1] * P, tc[2] * P};
    const C* __restrict__ src = static_cast<const C*>(a.src);
    C* __restrict__ dst = static_cast<C*>(a.dst);
    const int nxy = a.N[0] * a.N[1];
    for (int i = warp; i < kQ; i += NW) {
        int s[3], b0[3];
        bool sp[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            sp[d] = t.span[i][d] != 0;
            s[d] = (tc[d] + t.span[i][d] + 1) * P;
            b0[d] = (c0[d] - 1 - t.kmin[i][d] - t.span[i][d]) * P;
        }
        for (int e = lane; e < s[0]; e += 32) xo[e] = wrap_index(b0[0] + e, a.N[0]);
        for (int e = lane; e < s[1]; e += 32) yo[e] = wrap_index(b0[1] + e, a.N[1]) * a.N[0];
        for (int e = lane; e < s[2]; e += 32) zo[e] = wrap_index(b0[2] + e, a.N[2]) * nxy;
        __syncwarp();
        const C* __restrict__ sp_i = src + 2LL * i * a.nn;
        const int sx = s[0], sxy = s[0] * s[1];
        // rows of the per-warp buffer hold an odd number of pairs, so that the x pass's lanes
        // (one row each) fall on different banks; planes are s[1] such rows
        const int rs = sx | 1, ps = rs * s[1];
        C w[P][P + 1];
        signed char k[P];
        load_pass_weights<C, P>(t.lw[i][2], t.kc[i][2], w, k);
        for (int col = lane; col < sxy; col += 32) {
            const int y = col / sx;
            const int x = col - y * sx;
            const int off = yo[y] + xo[x];
            C2 v[TS::BZ];
#pragma unroll
            for (int z = 0; z < TS::BZ; ++z) {
                if (z < s[2]) {
                    v[z] = load_pair<C>(sp_i + 2LL * (zo[z] + off));
                } else {
                    v[z].x = C(0);
                    v[z].y = C(0);
                }
            }
            C2 r[TS::TZ];
            transpose_column<C, P, TS::TZ, TS::BZ>(v, w, k, sp[2], r);
#pragma unroll
            for (int oz = 0; oz < TS::TZ; ++oz)
                if (oz < te[2]) zb[oz * ps + y * rs + x] = r[oz];
        }
        __syncwarp();
        load_pass_weights<C, P>(t.lw[i][1], t.kc[i][1], w, k);
        const int ncol = te[2] * sx;
        for (int col = lane; col < ncol; col += 32) {
            const int oz = col / sx;
            const int x = col - oz * sx;
            C2* cp = zb + oz * ps + x;
            C2 v[TS::BY];
#pragma unroll
            for (int y = 0; y < TS::BY; ++y) {
                if (y < s[1]) {
                    v[y] = cp[y * rs];
                } else {
                    v[y].x = C(0);
                    v[y].y = C(0);
                }
            }
            C2 r[TS::TY];
            transpose_column<C, P, TS::TY, TS::BY>(v, w, k, sp[1], r);
#pragma unroll
            for (int oy = 0; oy < TS::TY; ++oy)
                if (oy < te[1]) cp[oy * rs] = r[oy];
        }
        __syncwarp();
        load_pass_weights<C, P>(t.lw[i][0], t.kc[i][0], w, k);
        for (int row = lane; row < TS::TY * TS::TZ; row += 32) {
            const int oz = row / TS::TY;
            const int oy = row - oz * TS::TY;
            if (oz >= te[2] || oy >= te[1]) continue;
            const C2* rp = zb + oz * ps + oy * rs;
            C2 v[TS::BX];
#pragma unroll
            for (int x = 0; x < TS::BX; ++x) {
                if (x < sx) {
                    v[x] = rp[x];
                } else {
                    v[x].x = C(0);
                    v[x].y = C(0);
                }
            }
            C2 r[TS::TX];
            transpose_column<C, P, TS::TX, TS::BX>(v, w, k, sp[0], r);
            const long long g0 = (static_cast<long long>(c0[2] * P + oz) * a.N[1] + (c0[1] * P + oy)) * a.N[0] +
                                 c0[0] * P;
            C2* dp = reinterpret_cast<C2*>(dst) + static_cast<long long>(i) * a.nn + g0;
#pragma unroll
            for (int ox = 0; ox < TS::TX; ++ox)
                if (ox < te[0]) dp[ox] = r[ox];
        }
        __syncwarp();
    }
}

// *acc += sum of partials[0..n) in a fixed order (one block).
__global__ void accumulate_kernel(const double* __restrict__ partials, int n, double* __restrict__ acc) {
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += partials[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *acc += red[0];
}

// Seed of E_k = (1/(|S| rho0 U0^2)) sum_cells sum_points w_q rho |u|^2 / 2 (the sllbm_diag
// quadrature): dE_k/df_i(n) = W_n (xi_i.u - |u|^2/2), dE_k/dg_i = 0, with W_n the node's
// total quadrature weight: prod_d W1[a_d] times scale, W1[a] = W_a (+ W_p for a = 0, the
// node being the right-face point of the neighbouring cell as well).
struct EkConst {
    double xi[kQ][3];
    double W1[kMaxP];
};

template <typename CS, typename C>
__global__ void __launch_bounds__(128) ek_seed_kernel(const CS* __restrict__ pop, C* __restrict__ lam, long long nn,
                                                      int Nx, int Ny, int p, double scale,
                                                      const __grid_constant__ EkConst kc) {
    const long long sxy = static_cast<long long>(Nx) * Ny;
    for (long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; n < nn;
         n += static_cast<long long>(gridDim.x) * blockDim.x) {
        double rho = 0, jx = 0, jy = 0, jz = 0;
        for (int i = 0; i < kQ; ++i) {
            const double f = pop[2 * (i * nn + n)];
            rho += f;
            jx += f * kc.xi[i][0];
            jy += f * kc.xi[i][1];
            jz += f * kc.xi[i][2];
        }
        const double ux = jx / rho, uy = jy / rho, uz = jz / rho;
        const double half_usq = 0.5 * (ux * ux + uy * uy + uz * uz);
        const int x = static_cast<int>(n % Nx), y = static_cast<int>((n / Nx) % Ny),
                  z = static_cast<int>(n / sxy);
        const double wn = kc.W1[x % p] * kc.W1[y % p] * kc.W1[z % p] * scale;
        for (int i = 0; i < kQ; ++i) {
            lam[2 * (i * nn + n)] = static_cast<C>(wn * (kc.xi[i][0] * ux + kc.xi[i][1] * uy + kc.xi[i][2] * uz - half_usq));
            lam[2 * (i * nn + n) + 1] = C(0);
        }
    }
}

// ---- reverse mode of the Sec. III.C diagnostics ---------------------------------------
// J = wk E_k + ws eps_s + wc eps_c as sllbm_diag computes it: per cell, the Clenshaw-Curtis
// quadrature over its (p+1)^3 support points of rho|u|^2/2, mu~(T)|curl u|^2 and
// (4/3) mu~(T)(div u)^2, with velocity gradients from the cell-local Lagrange derivative.
// dJ/dpop in three gather kernels (no atomics): the node fields; per quadrature point the
// derivatives of its integrand with respect to its nine gradient entries and to its
// temperature; per node the sum over the quadrature points whose integrand involves it,
// mapped to f and g through the moments.
struct DiagAdjConst {
    double xi[kQ][3];
    double W[kMaxP + 1];
    double D[kMaxP + 1][kMaxP + 1];  // D[a][j]: derivative of basis j at GLC point a
};

// rho, u, T (FP64, [5][nodes]) of a state in storage order.
template <typename CS>
__global__ void __launch_bounds__(128) node_fields_kernel(const CS* __restrict__ pop, long long nn, double inv_2cv,
                                                          const __grid_constant__ AdjVel v, double* __restrict__ fld) {
    for (long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; n < nn;
         n += static_cast<long long>(gridDim.x) * blockDim.x) {
        double rho = 0, mx = 0, my = 0, mz = 0, e2 = 0;
        for (int i = 0; i < kQ; ++i) {
            const double f = static_cast<double>(pop[2 * (i * nn + n)]);
            rho += f;
            mx += f * v.xi[i][0];
            my += f * v.xi[i][1];
            mz += f * v.xi[i][2];
            e2 += f * shell_xi2(shell_of(i)) + static_cast<double>(pop[2 * (i * nn + n) + 1]);
        }
        const double ux = mx / rho, uy = my / rho, uz = mz / rho;
        fld[n] = rho;
        fld[nn + n] = ux;
        fld[2 * nn + n] = uy;
        fld[3 * nn + n] = uz;
        fld[4 * nn + n] = (e2 / rho - (ux * ux + uy * uy + uz * uz)) * inv_2cv;
    }
}

// Per quadrature point (cell, local a, b, c): G[0..8] = dJ/d(du_comp/dx_dir) times the
// derivative factor 2/h_dir (index comp*3 + dir), G[9] = dJ/dT at the point.
template <int P>
__global__ void __launch_bounds__(128) diag_point_adj_kernel(const double* __restrict__ fld, long long nn, int Nx,
                                                             int Ny, int Nz, int ncx, int ncy, long long ncell,
                                                             double hx, double hy, double hz, double ks, double kc,
                                                             const __grid_constant__ DiagAdjConst dc,
                                                             double* __restrict__ G) {
    constexpr int P1 = P + 1, NPC = P1 * P1 * P1;
    const double h[3] = {hx, hy, hz};
    for (long long idx = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; idx < ncell * NPC;
         idx += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long cell = idx / NPC;
        const int q = static_cast<int>(idx - cell * NPC);
        const int loc[3] = {q % P1, (q / P1) % P1, q / (P1 * P1)};
        const int c[3] = {static_cast<int>(cell % ncx), static_cast<int>((cell / ncx) % ncy),
                          static_cast<int>(cell / (static_cast<long long>(ncx) * ncy))};
        const int Nd[3] = {Nx, Ny, Nz};
        double g[3][3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double acc[3] = {0, 0, 0};
#pragma unroll
            for (int j = 0; j < P1; ++j) {
                int m[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) m[e] = (c[e] * P + (e == d ? j : loc[e])) % Nd[e];
                const long long node = (static_cast<long long>(m[2]) * Ny + m[1]) * Nx + m[0];
#pragma unroll
                for (int comp = 0; comp < 3; ++comp) acc[comp] += dc.D[loc[d]][j] * fld[(1 + comp) * nn + node];
            }
#pragma unroll
            for (int comp = 0; comp < 3; ++comp) g[comp][d] = acc[comp] * 2.0 / h[d];
        }
        const long long nq = (static_cast<long long>((c[2] * P + loc[2]) % Nz) * Ny + (c[1] * P + loc[1]) % Ny) * Nx +
                             (c[0] * P + loc[0]) % Nx;
        const double T = fld[4 * nn + nq];
        const double wq = dc.W[loc[0]] * dc.W[loc[1]] * dc.W[loc[2]] * hx * hy * hz * 0.125;
        const double ox = g[2][1] - g[1][2], oy = g[0][2] - g[2][0], oz = g[1][0] - g[0][1];
        const double dv = g[0][0] + g[1][1] + g[2][2];
        const double mut = sutherland(T);
        const double wm = wq * mut;
        double* out = G + idx * 10;
        // d|curl u|^2 / d g[comp][dir] and d(div u)^2 / d g[comp][dir]
        const double dcurl[3][3] = {{0.0, -2.0 * oz, 2.0 * oy}, {2.0 * oz, 0.0, -2.0 * ox}, {-2.0 * oy, 2.0 * ox, 0.0}};
#pragma unroll
        for (int comp = 0; comp < 3; ++comp)
#pragma unroll
            for (int d = 0; d < 3; ++d)
                out[comp * 3 + d] = wm * (ks * dcurl[comp][d] + (comp == d ? kc * 2.0 * dv : 0.0)) * 2.0 / h[d];
        out[9] = wq * mut * sutherland_dlog(T) * (ks * (ox * ox + oy * oy + oz * oz) + kc * dv * dv);
    }
}

// Per node: the point terms of every quadrature point whose integrand involves the node
// (the node's own point in each cell that holds it, and the points on its lines in those
// cells), the kinetic-energy term, then lam_f_i = a_rho + a_u.(xi_i - u)/rho +
// a_T (|xi_i - u|^2 - 2 C_v T)/(2 C_v rho) and lam_g_i = a_T/(2 C_v rho).
template <int P, typename C>
__global__ void __launch_bounds__(128) diag_node_adj_kernel(const double* __restrict__ fld, const double* __restrict__ G,
                                                            long long nn, int Nx, int Ny, int ncx, int ncy, int ncz,
                                                            double hx, double hy, double hz, double ke, double two_cv,
                                                            const __grid_constant__ DiagAdjConst dc,
                                                            C* __restrict__ lam) {
    constexpr int P1 = P + 1, NPC = P1 * P1 * P1;
    const long long sxy = static_cast<long long>(Nx) * Ny;
    for (long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; n < nn;
         n += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x[3] = {static_cast<int>(n % Nx), static_cast<int>((n / Nx) % Ny), static_cast<int>(n / sxy)};
        const int nc[3] = {ncx, ncy, ncz};
        // the (cell, local index) pairs that hold the node, per direction: one, or two for a
        // cell-face node (local 0 of its cell and local P of the cell before, periodically)
        int cc[3][2], aa[3][2], cnt[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            cc[d][0] = x[d] / P;
            aa[d][0] = x[d] % P;
            cnt[d] = 1;
            if (aa[d][0] == 0) {
                cc[d][1] = (cc[d][0] + nc[d] - 1) % nc[d];
                aa[d][1] = P;
                cnt[d] = 2;
            }
        }
        const double rho = fld[n], ux = fld[nn + n], uy = fld[2 * nn + n], uz = fld[3 * nn + n], T = fld[4 * nn + n];
        double a_rho = 0, a_u[3] = {0, 0, 0}, a_T = 0;
        const double hv = hx * hy * hz * 0.125;
        for (int kz = 0; kz < cnt[2]; ++kz)
            for (int ky = 0; ky < cnt[1]; ++ky)
                for (int kx = 0; kx < cnt[0]; ++kx) {
                    const int lc[3] = {aa[0][kx], aa[1][ky], aa[2][kz]};
                    const long long base =
                        ((static_cast<long long>(cc[2][kz]) * ncy + cc[1][ky]) * ncx + cc[0][kx]) * NPC;
                    const long long q0 = base + (lc[2] * P1 + lc[1]) * P1 + lc[0];
                    a_T += G[q0 * 10 + 9];
                    const double wq = dc.W[lc[0]] * dc.W[lc[1]] * dc.W[lc[2]] * hv;
                    a_rho += ke * wq * 0.5 * (ux * ux + uy * uy + uz * uz);
                    a_u[0] += ke * wq * rho * ux;
                    a_u[1] += ke * wq * rho * uy;
                    a_u[2] += ke * wq * rho * uz;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
#pragma unroll
                        for (int j = 0; j < P1; ++j) {
                            int m[3] = {lc[0], lc[1], lc[2]};
                            m[d] = j;
                            const double* gq = G + (base + (m[2] * P1 + m[1]) * P1 + m[0]) * 10;
                            const double dw = dc.D[j][lc[d]];
                            a_u[0] += gq[0 * 3 + d] * dw;
                            a_u[1] += gq[1 * 3 + d] * dw;
                            a_u[2] += gq[2 * 3 + d] * dw;
                        }
                    }
                }
        const double inv_rho = 1.0 / rho, aT = a_T / (two_cv * rho);
        for (int i = 0; i < kQ; ++i) {
            const double cx = dc.xi[i][0] - ux, cy = dc.xi[i][1] - uy, cz = dc.xi[i][2] - uz;
            const double lf = a_rho + (a_u[0] * cx + a_u[1] * cy + a_u[2] * cz) * inv_rho +
                              aT * (cx * cx + cy * cy + cz * cz - two_cv * T);
            lam[2 * (i * nn + n)] = static_cast<C>(lf);
            lam[2 * (i * nn + n) + 1] = static_cast<C>(aT);
        }
    }
}

// Transpose of the equilibrium initialisation f_i = w_i rho P_i, g_i = (2C_v - D) T f_i at
// each node (FP64 arithmetic, as the initialisation itself).
template <typename C>
__global__ void __launch_bounds__(128) init_vjp_kernel(const double* __restrict__ rho_f, const double* __restrict__ u_f,
                                                       const double* __restrict__ T_f, const C* __restrict__ lam,
                                                       long long nn, double gfac, const __grid_constant__ AdjVel v,
                                                       double* __restrict__ g_rho, double* __restrict__ g_u,
                                                       double* __restrict__ g_T) {
    for (long long n = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; n < nn;
         n += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double rho = rho_f[n], ux = u_f[n], uy = u_f[nn + n], uz = u_f[2 * nn + n], T = T_f[n];
        const double usq = ux * ux + uy * uy + uz * uz, th = T - 1.0;
        const EqCoef<double> ec = eq_coefficients(usq, th);
        double arho = 0, aux = 0, auy = 0, auz = 0, ausq = 0, ath = 0, ATd = 0;
        for (int i = 0; i < kQ; ++i) {
            const double x = v.xi[i][0], y = v.xi[i][1], z = v.xi[i][2], w = v.w[i];
            const PolyDeriv<double> pd = poly_deriv(ec, shell_of(i), x * ux + y * uy + z * uz, usq, th);
            const double lf = static_cast<double>(lam[2 * (i * nn + n)]);
            const double lg = static_cast<double>(lam[2 * (i * nn + n) + 1]);
            const double Aw = (lf + gfac * T * lg) * w;
            ATd += gfac * lg * w * rho * pd.P;
            arho += Aw * pd.P;
            const double t = Aw * rho * pd.ds;
            aux += t * x;
            auy += t * y;
            auz += t * z;
            ausq += Aw * rho * pd.dusq;
            ath += Aw * rho * pd.dth;
        }
        if (g_rho) g_rho[n] = arho;
        if (g_u) {
            g_u[n] = aux + 2.0 * ux * ausq;
            g_u[nn + n] = auy + 2.0 * uy * ausq;
            g_u[2 * nn + n] = auz + 2.0 * uz * ausq;
        }
        if (g_T) g_T[n] = ath + ATd;
    }
}

unsigned adj_grid(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 65536) g = 65536;
    return static_cast<unsigned>(g < 1 ? 1 : g);
}

AdjVel adj_vel(const sllbm_ctx* ctx) {
    AdjVel v;
    std::memcpy(v.xi, ctx->xi, sizeof(v.xi));
    std::memcpy(v.w, ctx->w, sizeof(v.w));
    return v;
}

template <typename C>
PassTable<C> pass_table(const sllbm_ctx* ctx, int d) {
    PassTable<C> t;
    std::memset(&t, 0, sizeof(t));
    for (int i = 0; i < kQ; ++i)
        for (int a = 0; a < ctx->p; ++a) {
            t.shift[i][a] = ctx->dir[d].shift[i][a];
            for (int j = 0; j <= ctx->p; ++j) t.w[i][a][j] = static_cast<C>(ctx->dir[d].weight[i][a][j]);
        }
    return t;
}

int adj_fail(sllbm_ctx* ctx, cudaError_t e) {
    ctx->last_err = static_cast<int>(e);
    return SLLBM_ECUDA;
}

}  // namespace

// Two state-sized scratch buffers and the per-block partials of the mu_inf sensitivity,
// allocated on the first reverse-mode call.
int ensure_adjoint_scratch(sllbm_ctx* ctx) {
    // holds a streamed state and, in the transposed passes, adjoint populations
    const size_t lam_bytes = static_cast<size_t>(2 * kQ) * static_cast<size_t>(ctx->nn) *
                             (ctx->adj_f64 ? sizeof(double) : ctx->elem);
    const size_t need = lam_bytes > ctx->pop_bytes ? lam_bytes : ctx->pop_bytes;
    if (ctx->adj_buf[0] != nullptr && ctx->adj_bytes >= need) return SLLBM_OK;
    adjoint_release(ctx);
    // one partial per tile of the fused forward/VJP kernel (tiles are at least one cell)
    const long long ncell = static_cast<long long>(ctx->cells[0]) * ctx->cells[1] * ctx->cells[2];
    ctx->adj_blocks = static_cast<int>(ncell);
    ctx->adj_bytes = need;
    cudaError_t e = dev_alloc(&ctx->adj_buf[0], need);
    if (e == cudaSuccess) e = dev_alloc(&ctx->adj_buf[1], need);
    if (e == cudaSuccess) e = dev_alloc(&ctx->d_adj_partials, sizeof(double) * ctx->adj_blocks);
    if (e != cudaSuccess) {
        adjoint_release(ctx);
        ctx->last_err = static_cast<int>(e);
        return SLLBM_ENOMEM;
    }
    return SLLBM_OK;
}

void adjoint_release(sllbm_ctx* ctx) {
    cudaFree(ctx->adj_buf[0]);
    cudaFree(ctx->adj_buf[1]);
    cudaFree(ctx->d_adj_partials);
    ctx->adj_buf[0] = ctx->adj_buf[1] = nullptr;
    ctx->d_adj_partials = nullptr;
    ctx->adj_bytes = 0;
}

namespace {

bool adjoint_supported(const sllbm_ctx* ctx) {
    return (ctx->prm.storage == SLLBM_F32 || ctx->prm.storage == SLLBM_F64) && !ctx->prm.pr_correction &&
           ctx->prm.collide && !ctx->slab;
}

template <typename C>
int launch_pass(sllbm_ctx* ctx, const void* in, void* out, int d, bool transpose) {
    const PassTable<C> t = pass_table<C>(ctx, d);
    const unsigned grid = adj_grid(static_cast<long long>(kQ) * ctx->nn, 256);
    if (transpose)
        pass_kernel<C, true><<<grid, 256, 0, ctx->stream>>>(static_cast<const C*>(in), static_cast<C*>(out),
                                                            ctx->N[0], ctx->N[1], d, ctx->p, ctx->cells[d],
                                                            ctx->nn, t);
    else
        pass_kernel<C, false><<<grid, 256, 0, ctx->stream>>>(static_cast<const C*>(in), static_cast<C*>(out),
                                                             ctx->N[0], ctx->N[1], d, ctx->p, ctx->cells[d],
                                                             ctx->nn, t);
    ctx->launches += 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SLLBM_OK : adj_fail(ctx, e);
}

// dst = S src (transpose = false) or S^T src, through the two scratch buffers.
template <typename C>
int stream_apply_t(sllbm_ctx* ctx, const void* src, void* dst, bool transpose) {
    void* a = ctx->adj_buf[0];
    void* b = ctx->adj_buf[1];
    int rc = launch_pass<C>(ctx, src, a, 2, transpose);
    if (rc == SLLBM_OK) rc = launch_pass<C>(ctx, a, b, 1, transpose);
    if (rc == SLLBM_OK) rc = launch_pass<C>(ctx, b, dst, 0, transpose);
    return rc;
}

template <typename C, int P, int CX, int CY, int CZ, int NW>
int launch_transpose(sllbm_ctx* ctx, const void* src, void* dst) {
    using SM = TransSmem<C, P, CX, CY, CZ, NW>;
    static_assert(SM::bytes <= 227 * 1024, "shared memory budget");
    StepTables<C, P> tab;
    fill_step_tables<C, P>(ctx, &tab);
    StepArgs args;
    fill_step_args(ctx, src, dst, &args);
    args.flag = nullptr;
    args.tiles[0] = (ctx->cells[0] + CX - 1) / CX;
    args.tiles[1] = (ctx->cells[1] + CY - 1) / CY;
    args.tiles[2] = (ctx->cells[2] + CZ - 1) / CZ;
    const int ntiles = args.tiles[0] * args.tiles[1] * args.tiles[2];
    auto k = adj_transpose_kernel<C, P, CX, CY, CZ, NW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(SM::bytes));
    if (e == cudaSuccess) {
        k<<<ntiles, NW * 32, SM::bytes, ctx->stream>>>(args, tab);
        e = cudaGetLastError();
    }
    ctx->launches += 1;
    return e == cudaSuccess ? SLLBM_OK : adj_fail(ctx, e);
}

// Tiles (cells) and warps of the FP32 tile kernels of a backward step (the forward step's).
template <typename C, int P>
struct AdjTile;
template <> struct AdjTile<float, 2> { static constexpr int CX = 4, CY = 4, CZ = 2, NW = 16; };
template <> struct AdjTile<float, 3> { static constexpr int CX = 4, CY = 2, CZ = 1, NW = 9; };  // two CTAs per SM
template <> struct AdjTile<float, 4> { static constexpr int CX = 2, CY = 2, CZ = 1, NW = 16; };

// The state streamed without collision (the step kernel's tile body, stream-only mode).
template <typename CS, int P, int CX, int CY, int CZ, int NW>
int launch_stream_only(sllbm_ctx* ctx, const void* state, void* h) {
    using SM = StepSmem<CS, P, CX, CY, CZ, NW>;
    StepTables<CS, P> tab;
    fill_step_tables<CS, P>(ctx, &tab);
    StepArgs args;
    fill_step_args(ctx, state, h, &args);
    args.flag = nullptr;
    args.collide = 0;
    args.tiles[0] = (ctx->cells[0] + CX - 1) / CX;
    args.tiles[1] = (ctx->cells[1] + CY - 1) / CY;
    args.tiles[2] = (ctx->cells[2] + CZ - 1) / CZ;
    const int ntiles = args.tiles[0] * args.tiles[1] * args.tiles[2];
    auto k = step_kernel<CS, CS, P, CX, CY, CZ, NW, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(SM::bytes));
    if (e == cudaSuccess) {
        k<<<ntiles, NW * 32, SM::bytes, ctx->stream>>>(args, tab);
        e = cudaGetLastError();
    }
    ctx->launches += 1;
    return e == cudaSuccess ? SLLBM_OK : adj_fail(ctx, e);
}

// The collision VJP over a full grid, its mu_inf partials summed in a fixed order into *dmu.
template <typename CH, typename C>
int launch_vjp(sllbm_ctx* ctx, const void* h, const void* lam, void* out, double* dmu) {
    AdjArgs aa;
    aa.mu_over_dt = ctx->mu_inf / ctx->dt;
    aa.inv_dt = 1.0 / ctx->dt;
    aa.inv_2cv = 0.5 * (ctx->prm.gamma - 1.0);
    aa.gfac = 2.0 / (ctx->prm.gamma - 1.0) - 3.0;
    long long g = (ctx->nn + 127) / 128;
    if (g > ctx->adj_blocks) g = ctx->adj_blocks;
    const int nb = static_cast<int>(g);
    collide_vjp_kernel<CH, C><<<nb, 128, 0, ctx->stream>>>(static_cast<const CH*>(h), static_cast<const C*>(lam),
                                                            static_cast<C*>(out), ctx->nn, aa, adj_vel(ctx),
                                                            ctx->d_adj_partials);
    accumulate_kernel<<<1, 256, 0, ctx->stream>>>(ctx->d_adj_partials, nb, dmu);
    ctx->launches += 2;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SLLBM_OK : adj_fail(ctx, e);
}

// FP32 backward step: the state streamed by the step kernel's tile body (stream-only mode),
// the collision VJP over a full grid (one thread per node), the transposed streaming as a
// tile kernel.  (The VJP inside the streaming tile kernel was slower: only the tile's nodes,
// one thread each, share its arithmetic.)
template <int P>
int adjoint_step_tiles(sllbm_ctx* ctx, const void* state_prev, const void* lam_next, void* lam_prev, double* dmu) {
    using A = AdjTile<float, P>;
    void* mu = ctx->adj_buf[0];
    void* h = ctx->adj_buf[1];
    int rc = launch_stream_only<float, P, A::CX, A::CY, A::CZ, A::NW>(ctx, state_prev, h);
    if (rc != SLLBM_OK) return rc;
    rc = launch_vjp<float, float>(ctx, h, lam_next, mu, dmu);
    if (rc != SLLBM_OK) return rc;
    return launch_transpose<float, P, A::CX, A::CY, A::CZ, A::NW>(ctx, mu, lam_prev);
}

// Backward step with FP64 arithmetic (FP64 storage, or FP32 states with FP64 adjoint
// populations): 1D passes for the streaming and its transpose, the VJP over a full grid.
// (The tile kernels were slower here: the FP64 step kernel's register spills and its FP64
// moment arithmetic in stream-only mode.)
template <typename CS, typename C>
int adjoint_step_passes(sllbm_ctx* ctx, const void* state_prev, const void* lam_next, void* lam_prev,
                        double* dmu) {
    void* a = ctx->adj_buf[0];
    void* b = ctx->adj_buf[1];
    int rc = launch_pass<CS>(ctx, state_prev, a, 2, false);
    if (rc == SLLBM_OK) rc = launch_pass<CS>(ctx, a, b, 1, false);
    if (rc == SLLBM_OK) rc = launch_pass<CS>(ctx, b, a, 0, false);
    if (rc == SLLBM_OK) rc = launch_vjp<CS, C>(ctx, a, lam_next, b, dmu);
    if (rc == SLLBM_OK) rc = launch_pass<C>(ctx, b, a, 0, true);
    if (rc == SLLBM_OK) rc = launch_pass<C>(ctx, a, b, 1, true);
    if (rc == SLLBM_OK) rc = launch_pass<C>(ctx, b, lam_prev, 2, true);
    return rc;
}

template <typename CS, typename C>
int adjoint_step_t(sllbm_ctx* ctx, const void* state_prev, const void* lam_next, void* lam_prev, double* dmu) {
    if constexpr (std::is_same<CS, float>::value && std::is_same<C, float>::value) {
        switch (ctx->p) {
        case 2: return adjoint_step_tiles<2>(ctx, state_prev, lam_next, lam_prev, dmu);
        case 3: return adjoint_step_tiles<3>(ctx, state_prev, lam_next, lam_prev, dmu);
        case 4: return adjoint_step_tiles<4>(ctx, state_prev, lam_next, lam_prev, dmu);
        }
        return SLLBM_EINVAL;
    } else {
        return adjoint_step_passes<CS, C>(ctx, state_prev, lam_next, lam_prev, dmu);
    }
}

}  // namespace

}  // namespace sllbm

using namespace sllbm;

extern "C" {

int sllbm_stream_apply(sllbm_ctx* ctx, const void* src, void* dst, int transpose) {
    if (ctx == nullptr || src == nullptr || dst == nullptr) return SLLBM_EINVAL;
    if ((ctx->prm.storage != SLLBM_F32 && ctx->prm.storage != SLLBM_F64) || ctx->slab) return SLLBM_EINVAL;
    int rc = ensure_adjoint_scratch(ctx);
    if (rc != SLLBM_OK) return rc;
    return ctx->prm.storage == SLLBM_F64 ? stream_apply_t<double>(ctx, src, dst, transpose != 0)
                                         : stream_apply_t<float>(ctx, src, dst, transpose != 0);
}

int sllbm_adjoint_step(sllbm_ctx* ctx, const void* state_prev, const void* lam_next, void* lam_prev, double* dmu) {
    NvtxRange range("sllbm_adjoint_step");
    if (ctx == nullptr || state_prev == nullptr || lam_next == nullptr || lam_prev == nullptr || dmu == nullptr)
        return SLLBM_EINVAL;
    if (!adjoint_supported(ctx)) return SLLBM_EINVAL;
    if (lam_prev == state_prev || lam_prev == lam_next) return SLLBM_EINVAL;
    int rc = ensure_adjoint_scratch(ctx);
    if (rc != SLLBM_OK) return rc;
    if (ctx->prm.storage == SLLBM_F64) return adjoint_step_t<double, double>(ctx, state_prev, lam_next, lam_prev, dmu);
    if (ctx->adj_f64) return adjoint_step_t<float, double>(ctx, state_prev, lam_next, lam_prev, dmu);
    return adjoint_step_t<float, float>(ctx, state_prev, lam_next, lam_prev, dmu);
}

int sllbm_set_adjoint_type(sllbm_ctx* ctx, int storage) {
    if (ctx == nullptr) return SLLBM_EINVAL;
    if (storage == SLLBM_F64 && (ctx->prm.storage == SLLBM_F32 || ctx->prm.storage == SLLBM_F64)) {
        ctx->adj_f64 = ctx->prm.storage == SLLBM_F32;
        return SLLBM_OK;
    }
    if (storage == ctx->prm.storage && storage == SLLBM_F32) {
        ctx->adj_f64 = false;
        return SLLBM_OK;
    }
    return SLLBM_EINVAL;
}

int sllbm_ek_adjoint(sllbm_ctx* ctx, const void* state, void* lam) {
    if (ctx == nullptr || state == nullptr || lam == nullptr) return SLLBM_EINVAL;
    if (!adjoint_supported(ctx)) return SLLBM_EINVAL;
    EkConst kc;
    std::memcpy(kc.xi, ctx->xi, sizeof(kc.xi));
    double W[kMaxP + 1];
    clenshaw_curtis(ctx->p, W);
    for (int a = 0; a < kMaxP; ++a) kc.W1[a] = a < ctx->p ? W[a] + (a == 0 ? W[ctx->p] : 0.0) : 0.0;
    const double vol = ctx->L[0] * ctx->L[1] * ctx->L[2];
    const double scale = ctx->h[0] * ctx->h[1] * ctx->h[2] * 0.125 / (vol * ctx->prm.rho0 * ctx->U0 * ctx->U0);
    const unsigned grid = adj_grid(ctx->nn, 128);
    if (ctx->prm.storage == SLLBM_F64)
        ek_seed_kernel<double, double><<<grid, 128, 0, ctx->stream>>>(static_cast<const double*>(state),
                                                                      static_cast<double*>(lam), ctx->nn, ctx->N[0],
                                                                      ctx->N[1], ctx->p, scale, kc);
    else if (ctx->adj_f64)
        ek_seed_kernel<float, double><<<grid, 128, 0, ctx->stream>>>(static_cast<const float*>(state),
                                                                     static_cast<double*>(lam), ctx->nn, ctx->N[0],
                                                                     ctx->N[1], ctx->p, scale, kc);
    else
        ek_seed_kernel<float, float><<<grid, 128, 0, ctx->stream>>>(static_cast<const float*>(state),
                                                                    static_cast<float*>(lam), ctx->nn, ctx->N[0],
                                                                    ctx->N[1], ctx->p, scale, kc);
    ctx->launches += 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SLLBM_OK : adj_fail(ctx, e);
}

int sllbm_diag_adjoint(sllbm_ctx* ctx, const void* state, void* lam, double wk, double ws, double wc) {
    if (ctx == nullptr || state == nullptr || lam == nullptr) return SLLBM_EINVAL;
    if (!adjoint_supported(ctx)) return SLLBM_EINVAL;
    int rc = ensure_adjoint_scratch(ctx);
    if (rc != SLLBM_OK) return rc;
    DiagAdjConst dc;
    std::memcpy(dc.xi, ctx->xi, sizeof(dc.xi));
    clenshaw_curtis(ctx->p, dc.W);
    diff_matrix(ctx->p, dc.D);
    const long long ncell = static_cast<long long>(ctx->cells[0]) * ctx->cells[1] * ctx->cells[2];
    const int P1 = ctx->p + 1;
    const long long npts = ncell * P1 * P1 * P1;
    // scratch: the node fields (5 doubles per node) and the point terms (10 per quadrature
    // point) fit the two state-sized reverse-mode buffers (at least 360 bytes per node)
    if (static_cast<size_t>(5 * ctx->nn) * sizeof(double) > ctx->adj_bytes ||
        static_cast<size_t>(10 * npts) * sizeof(double) > ctx->adj_bytes)
        return SLLBM_EINVAL;
    double* fld = static_cast<double*>(ctx->adj_buf[0]);
    double* G = static_cast<double*>(ctx->adj_buf[1]);
    const double vol = ctx->L[0] * ctx->L[1] * ctx->L[2];
    const double base = vol * ctx->prm.rho0 * ctx->U0 * ctx->U0;
    const double ke = wk / base, ks = ws / (base * ctx->prm.Re), kc = wc * 4.0 / 3.0 / (base * ctx->prm.Re);
    const double inv_2cv = 0.5 * (ctx->prm.gamma - 1.0), two_cv = 1.0 / inv_2cv;
    const AdjVel v = adj_vel(ctx);
    if (ctx->prm.storage == SLLBM_F64)
        node_fields_kernel<double><<<adj_grid(ctx->nn, 128), 128, 0, ctx->stream>>>(
            static_cast<const double*>(state), ctx->nn, inv_2cv, v, fld);
    else
        node_fields_kernel<float><<<adj_grid(ctx->nn, 128), 128, 0, ctx->stream>>>(
            static_cast<const float*>(state), ctx->nn, inv_2cv, v, fld);
    const bool f64 = ctx->prm.storage == SLLBM_F64 || ctx->adj_f64;
    auto run = [&](auto pc) {
        constexpr int P = decltype(pc)::value;
        diag_point_adj_kernel<P><<<adj_grid(npts, 128), 128, 0, ctx->stream>>>(
            fld, ctx->nn, ctx->N[0], ctx->N[1], ctx->N[2], ctx->cells[0], ctx->cells[1], ncell, ctx->h[0], ctx->h[1],
            ctx->h[2], ks, kc, dc, G);
        if (f64)
            diag_node_adj_kernel<P, double><<<adj_grid(ctx->nn, 128), 128, 0, ctx->stream>>>(
                fld, G, ctx->nn, ctx->N[0], ctx->N[1], ctx->cells[0], ctx->cells[1], ctx->cells[2], ctx->h[0],
                ctx->h[1], ctx->h[2], ke, two_cv, dc, static_cast<double*>(lam));
        else
            diag_node_adj_kernel<P, float><<<adj_grid(ctx->nn, 128), 128, 0, ctx->stream>>>(
                fld, G, ctx->nn, ctx->N[0], ctx->N[1], ctx->cells[0], ctx->cells[1], ctx->cells[2], ctx->h[0],
                ctx->h[1], ctx->h[2], ke, two_cv, dc, static_cast<float*>(lam));
    };
    if (ctx->p == 2) run(std::integral_constant<int, 2>{});
    else if (ctx->p == 3) run(std::integral_constant<int, 3>{});
    else run(std::integral_constant<int, 4>{});
    ctx->launches += 3;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SLLBM_OK : adj_fail(ctx, e);
}

int sllbm_init_fields_adjoint(sllbm_ctx* ctx, const double* rho, const double* u, const double* T, const void* lam,
                              double* grad_rho, double* grad_u, double* grad_T) {
    if (ctx == nullptr || rho == nullptr || u == nullptr || T == nullptr || lam == nullptr) return SLLBM_EINVAL;
    if (!adjoint_supported(ctx)) return SLLBM_EINVAL;
    const double gfac = 2.0 / (ctx->prm.gamma - 1.0) - 3.0;
    const unsigned grid = adj_grid(ctx->nn, 128);
    if (ctx->prm.storage == SLLBM_F64 || ctx->adj_f64)
        init_vjp_kernel<double><<<grid, 128, 0, ctx->stream>>>(rho, u, T, static_cast<const double*>(lam), ctx->nn,
                                                               gfac, adj_vel(ctx), grad_rho, grad_u, grad_T);
    else
        init_vjp_kernel<float><<<grid, 128, 0, ctx->stream>>>(rho, u, T, static_cast<const float*>(lam), ctx->nn,
                                                              gfac, adj_vel(ctx), grad_rho, grad_u, grad_T);
    ctx->launches += 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SLLBM_OK : adj_fail(ctx, e);
}

}  // extern "C"
