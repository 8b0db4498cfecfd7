// Newton-Krylov solve of A_h(x) = b on one mesh level (Sec. 3.4), FP64.
//
// The paper solves each time step's nonlinear system on the coarse level
// with Newton's method (stabilisation parameters frozen in the Jacobian),
// GMRES and a geometric multigrid preconditioner with a Vanka smoother whose
// local problems are the 108 x 108 matrices of one Q2 cell; it notes that any
// coarse solver can take its place.  Here:
//   * the operator A_h is the Q1/Q1 form of Eqs. (5)-(6) with the two-level
//     local projection on groups of 8 child cells (27 nodes = one Q2 cell's
//     nodes), evaluated per group;
//   * the Jacobian is exact: forward-mode dual numbers, one direction per
//     local unknown of a group (108), with alpha_T, delta_T from the value
//     part (frozen, Eq. (8)); local 108 x 108 matrices are summed into a
//     4 x 4-block CSR matrix by a gather in group order (deterministic);
//   * the preconditioner is additive group-Vanka: the global matrix
//     restricted to each group's 108 unknowns, LU-factorised and inverted
//     once per assembly, the inverse applied to the group's residual as a
//     dense product and averaged over the groups sharing a node;
//   * right-preconditioned restarted GMRES with classical Gram-Schmidt
//     applied twice; all vectors, dot products (warp shuffles, then a second
//     pass over the blocks: fixed order) and norms in FP64;
//   * Newton re-assembles the Jacobian when the residual rate
//     rho = |r_{j+1}| / |r_j| exceeds rho_max (Sec. 3.4).
// Dirichlet velocity unknowns keep the values given in x; where no boundary
// is do-nothing the pressure is pinned at one node during the solve and
// normalised to zero mean (mass-weighted) after each update (Sec. 3.1).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace dnnmg {
namespace {

constexpr double kGaussOff = 0.28867513459481288225457439025098;

struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double s) { return {s * a.v, s * a.d}; }
__device__ __forceinline__ Dual operator+(Dual a, double s) { return {a.v + s, a.d}; }
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { a.v += b.v; a.d += b.d; return a; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) { a.v -= b.v; a.d -= b.d; return a; }
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(Dual x) { return x.v; }
template <typename T>
__device__ __forceinline__ T zero() { return T{}; }
template <>
__device__ __forceinline__ double zero<double>() { return 0.0; }
template <>
__device__ __forceinline__ Dual zero<Dual>() { return Dual{0.0, 0.0}; }
template <typename T>
__device__ __forceinline__ T lift(double x);
template <>
__device__ __forceinline__ double lift<double>(double x) { return x; }
template <>
__device__ __forceinline__ Dual lift<Dual>(double x) { return Dual{x, 0.0}; }

__device__ __forceinline__ double gpt(int i) { return i ? 0.5 + kGaussOff : 0.5 - kGaussOff; }
__device__ __forceinline__ double basis(int k, int q) {
    double r = 1.0;
    for (int d = 0; d < 3; ++d) {
        const double xi = gpt((q >> d) & 1);
        r *= ((k >> d) & 1) ? xi : 1.0 - xi;
    }
    return r;
}
__device__ __forceinline__ double dbasis(int k, int q, int e) {
    double r = 1.0;
    for (int d = 0; d < 3; ++d) {
        const double xi = gpt((q >> d) & 1);
        if (d == e)
            r *= ((k >> d) & 1) ? 1.0 : -1.0;
        else
            r *= ((k >> d) & 1) ? xi : 1.0 - xi;
    }
    return r;
}

// group node of vertex a of child t (27-node groups); a for 8-node "groups"
template <int NPG>
__device__ __forceinline__ int child_node(int t, int a) {
    if (NPG == 8) return a;
    return ((t & 1) + (a & 1)) + 3 * (((t >> 1) & 1) + ((a >> 1) & 1)) + 9 * (((t >> 2) & 1) + ((a >> 2) & 1));
}
__device__ __forceinline__ int corner_node(int K) { return 2 * (K & 1) + 6 * ((K >> 1) & 1) + 18 * ((K >> 2) & 1); }
// trilinear weight of corner K at group node iota (reference point iota / 2)
__device__ __forceinline__ double wpi(int iota, int K) {
    const int c[3] = {iota % 3, (iota / 3) % 3, iota / 9};
    double w = 1.0;
    for (int d = 0; d < 3; ++d) {
        const double x = 0.5 * c[d];
        w *= ((K >> d) & 1) ? x : 1.0 - x;
    }
    return w;
}

enum { LV_OPERATOR = 0, LV_RHS = 1, LV_MASS = 2 };

struct LvPrm {
    double m, th, nu, a0, d0;
    int lps;
};

// Contributions of child t of a group to its group's local residual R
// (NPG x 4): the Galerkin part of A_h (LV_OPERATOR), the rhs b(v_old) with no
// force (LV_RHS), or the lumped mass in row 0 (LV_MASS); with the local
// projection terms (LV_OPERATOR, lps).  X, U, PU: group node coordinates,
// values, and projected values pi U.
template <typename T, int NPG, int MODE>
__device__ void child_terms(const double (*X)[3], const T (*U)[4], const T (*PU)[4], int t, const LvPrm& p,
                            T (*R)[4]) {
    int nd[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) nd[k] = child_node<NPG>(t, k);
    double aT = 0.0, dT = 0.0;
    const bool lps = MODE == LV_OPERATOR && NPG == 27 && p.lps;
    if (lps) {
        double h = 0.0, vmax = 0.0;
        for (int a = 0; a < 8; ++a) {
            for (int b = a + 1; b < 8; ++b) {
                double s = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double t0 = X[nd[a]][d] - X[nd[b]][d];
                    s += t0 * t0;
                }
                h = fmax(h, sqrt(s));
            }
            double s = 0.0;
            for (int d = 0; d < 3; ++d) s += val(U[nd[a]][d]) * val(U[nd[a]][d]);
            vmax = fmax(vmax, sqrt(s));
        }
        const double den = p.nu / (h * h) + vmax / h + p.m;
        aT = p.a0 / den;
        dT = p.d0 / den;
    }
    T sp[8], s1[8][3], s2[8][3];
    if (lps)
        for (int k = 0; k < 8; ++k) {
            sp[k] = zero<T>();
            for (int c = 0; c < 3; ++c) s1[k][c] = s2[k][c] = zero<T>();
        }
    for (int q = 0; q < 8; ++q) {
        double J[3][3];
        for (int d = 0; d < 3; ++d)
            for (int e = 0; e < 3; ++e) {
                double s = 0.0;
                for (int k = 0; k < 8; ++k) s += X[nd[k]][d] * dbasis(k, q, e);
                J[d][e] = s;
            }
        const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        const double idet = 1.0 / det;
        double Ji[3][3];
        Ji[0][0] = c00 * idet;
        Ji[1][0] = c01 * idet;
        Ji[2][0] = c02 * idet;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * idet;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * idet;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * idet;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * idet;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * idet;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * idet;
        const double w = 0.125 * det;
        double N[8], g[8][3];
        for (int k = 0; k < 8; ++k) {
            N[k] = basis(k, q);
            for (int d = 0; d < 3; ++d)
                g[k][d] = dbasis(k, q, 0) * Ji[0][d] + dbasis(k, q, 1) * Ji[1][d] + dbasis(k, q, 2) * Ji[2][d];
        }
        if (MODE == LV_MASS) {
            for (int k = 0; k < 8; ++k) R[nd[k]][0] += lift<T>(w * N[k]);
            continue;
        }
        T v[3] = {zero<T>(), zero<T>(), zero<T>()}, pr = zero<T>();
        T Dv[3][3];
        for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) Dv[c][d] = zero<T>();
        for (int k = 0; k < 8; ++k) {
            for (int c = 0; c < 3; ++c) {
                const T u = U[nd[k]][c];
                v[c] += N[k] * u;
                for (int d = 0; d < 3; ++d) Dv[c][d] += g[k][d] * u;
            }
            if (MODE == LV_OPERATOR) pr += N[k] * U[nd[k]][3];
        }
        const double cth = MODE == LV_OPERATOR ? p.th : p.th - 1.0;   // rhs: -(1 - theta)
        T conv[3];
        for (int c = 0; c < 3; ++c) conv[c] = v[0] * Dv[c][0] + v[1] * Dv[c][1] + v[2] * Dv[c][2];
        for (int k = 0; k < 8; ++k) {
            for (int c = 0; c < 3; ++c) {
                T s = (p.m * N[k]) * v[c] + (cth * N[k]) * conv[c];
                T vis = g[k][0] * Dv[c][0] + g[k][1] * Dv[c][1] + g[k][2] * Dv[c][2];
                s += (cth * p.nu) * vis;
                if (MODE == LV_OPERATOR) s -= g[k][c] * pr;
                R[nd[k]][c] += w * s;
            }
            if (MODE == LV_OPERATOR) R[nd[k]][3] += (w * N[k]) * (Dv[0][0] + Dv[1][1] + Dv[2][2]);
        }
        if (lps) {
            T gkp[3] = {zero<T>(), zero<T>(), zero<T>()};
            T pv[3] = {zero<T>(), zero<T>(), zero<T>()};
            T Dp[3][3];
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) Dp[c][d] = zero<T>();
            for (int k = 0; k < 8; ++k) {
                const T kp = U[nd[k]][3] - PU[nd[k]][3];
                for (int d = 0; d < 3; ++d) gkp[d] += g[k][d] * kp;
                for (int c = 0; c < 3; ++c) {
                    const T pu = PU[nd[k]][c];
                    pv[c] += N[k] * pu;
                    for (int d = 0; d < 3; ++d) Dp[c][d] += g[k][d] * pu;
                }
            }
            T gv[3];
            for (int c = 0; c < 3; ++c)
                gv[c] = conv[c] - (pv[0] * Dp[c][0] + pv[1] * Dp[c][1] + pv[2] * Dp[c][2]);
            for (int k = 0; k < 8; ++k) {
                sp[k] += (aT * w) * (gkp[0] * g[k][0] + gkp[1] * g[k][1] + gkp[2] * g[k][2]);
                const T vg = v[0] * g[k][0] + v[1] * g[k][1] + v[2] * g[k][2];
                const T pvg = pv[0] * g[k][0] + pv[1] * g[k][1] + pv[2] * g[k][2];
                for (int c = 0; c < 3; ++c) {
                    s1[k][c] += (dT * w) * (gv[c] * vg);
                    s2[k][c] += (dT * w) * (gv[c] * pvg);
                }
            }
        }
    }
    if (lps) {
        for (int k = 0; k < 8; ++k) {
            R[nd[k]][3] += sp[k];
            for (int c = 0; c < 3; ++c) R[nd[k]][c] += s1[k][c];
        }
        for (int K = 0; K < 8; ++K) {
            const int cn = corner_node(K);
            for (int k = 0; k < 8; ++k) {
                const double wk = wpi(nd[k], K);
                if (wk == 0.0) continue;
                R[cn][3] -= wk * sp[k];
                for (int c = 0; c < 3; ++c) R[cn][c] -= wk * s2[k][c];
            }
        }
    }
}

// pi U at the group nodes from the 8 corners
template <typename T, int NPG>
__device__ void project_group(const T (*U)[4], T (*PU)[4]) {
    if (NPG != 27) return;
    for (int i = 0; i < 27; ++i)
        for (int c = 0; c < 4; ++c) {
            T s = zero<T>();
            for (int K = 0; K < 8; ++K) {
                const double wk = wpi(i, K);
                if (wk != 0.0) s += wk * U[corner_node(K)][c];
            }
            PU[i][c] = s;
        }
}

// Local residual / rhs / mass of each group: one thread per group.
template <int NPG, int MODE>
__global__ void __launch_bounds__(64) level_local_kernel(int64_t ng, const int32_t* __restrict__ groups,
                                                         const double* __restrict__ xyz, const double* __restrict__ x,
                                                         LvPrm p, double* __restrict__ out) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    double X[NPG][3], U[NPG][4], PU[NPG][4], R[NPG][4];
    for (int i = 0; i < NPG; ++i) {
        const int64_t n = groups[g * NPG + i];
        for (int d = 0; d < 3; ++d) X[i][d] = xyz[3 * n + d];
        for (int c = 0; c < 4; ++c) {
            U[i][c] = MODE == LV_MASS ? 0.0 : x[4 * n + c];
            R[i][c] = 0.0;
        }
    }
    if (MODE == LV_OPERATOR) project_group<double, NPG>(U, PU);
    const int children = NPG == 27 ? 8 : 1;
    for (int t = 0; t < children; ++t) child_terms<double, NPG, MODE>(X, U, PU, t, p, R);
    for (int i = 0; i < NPG; ++i)
        for (int c = 0; c < 4; ++c) out[(g * NPG + i) * 4 + c] = R[i][c];
}

// Column j (local unknown 4 i + c) of each group's local Jacobian:
// one thread per (group, j), forward-mode derivative of the local residual.
template <int NPG>
__global__ void __launch_bounds__(128) level_jacobian_kernel(int64_t ng, const int32_t* __restrict__ groups,
                                                             const double* __restrict__ xyz,
                                                             const double* __restrict__ x, LvPrm p,
                                                             double* __restrict__ Jloc) {
    constexpr int NL = 4 * NPG;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (tid >= ng * NL) return;
    const int64_t g = tid / NL;
    const int j = int(tid % NL);
    const int jn = j / 4;
    double X[NPG][3];
    Dual U[NPG][4], PU[NPG][4], R[NPG][4];
    for (int i = 0; i < NPG; ++i) {
        const int64_t n = groups[g * NPG + i];
        for (int d = 0; d < 3; ++d) X[i][d] = xyz[3 * n + d];
        for (int c = 0; c < 4; ++c) {
            U[i][c] = Dual{x[4 * n + c], (4 * i + c == j) ? 1.0 : 0.0};
            R[i][c] = Dual{0.0, 0.0};
        }
    }
    project_group<Dual, NPG>(U, PU);
    bool is_corner = false;
    if (NPG == 27)
        for (int K = 0; K < 8; ++K) is_corner |= corner_node(K) == jn;
    const int children = NPG == 27 ? 8 : 1;
    for (int t = 0; t < children; ++t) {
        bool touches = is_corner && p.lps;
        for (int k = 0; k < 8; ++k) touches |= child_node<NPG>(t, k) == jn;
        if (touches) child_terms<Dual, NPG, LV_OPERATOR>(X, U, PU, t, p, R);
    }
    double* col = Jloc + g * NL * NL + j;
    for (int i = 0; i < NPG; ++i)
        for (int c = 0; c < 4; ++c) col[int64_t(4 * i + c) * NL] = R[i][c].d;
}

// out_j = sum over (g, local) containing node j of local[g*NPG + local][0..3]
__global__ void node_gather_kernel(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                   const double* __restrict__ local, double* __restrict__ out) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double a[4] = {0, 0, 0, 0};
    for (int32_t e = ptr[j]; e < ptr[j + 1]; ++e)
        for (int c = 0; c < 4; ++c) a[c] += local[4 * int64_t(idx[e]) + c];
    for (int c = 0; c < 4; ++c) out[4 * j + c] = a[c];
}

// r = b - A(x) (or b = rhs) with Dirichlet velocity rows, the pinned pressure
// row and (rhs) pressure rows set to zero
__global__ void finish_rows_kernel(int64_t n, const double* __restrict__ b, double* __restrict__ r,
                                   const uint8_t* __restrict__ dir, int32_t pin, int negate_plus_b, int rhs) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int c = 0; c < 4; ++c) {
        double v = r[4 * j + c];
        if (negate_plus_b) v = b[4 * j + c] - v;
        if ((c < 3 && dir[j]) || (c == 3 && (j == pin || rhs))) v = 0.0;
        r[4 * j + c] = v;
    }
}

// BSR block b = sum of its local entries; 16 threads per block
template <int NPG>
__global__ void bsr_assemble_kernel(int64_t nnzb, const int32_t* __restrict__ bptr, const int32_t* __restrict__ bsrc,
                                    const double* __restrict__ Jloc, double* __restrict__ A) {
    constexpr int NL = 4 * NPG;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (tid >= nnzb * 16) return;
    const int64_t b = tid >> 4;
    const int r = int(tid & 15) >> 2, s = int(tid & 3);
    double acc = 0.0;
    for (int32_t e = bptr[b]; e < bptr[b + 1]; ++e) {
        const int32_t src = bsrc[e];
        const int64_t g = src / (NPG * NPG);
        const int li = (src / NPG) % NPG, lj = src % NPG;
        acc += Jloc[g * NL * NL + int64_t(4 * li + r) * NL + 4 * lj + s];
    }
    A[16 * b + 4 * r + s] = acc;
}

// identity rows for Dirichlet velocity unknowns and the pinned pressure
__global__ void bsr_dirichlet_kernel(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const uint8_t* __restrict__ dir, int32_t pin, double* __restrict__ A) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int r = 0; r < 4; ++r) {
        const bool fix = (r < 3 && dir[i]) || (r == 3 && i == pin);
        if (!fix) continue;
        for (int32_t b = rp[i]; b < rp[i + 1]; ++b)
            for (int s = 0; s < 4; ++s) A[16 * int64_t(b) + 4 * r + s] = (ci[b] == i && s == r) ? 1.0 : 0.0;
    }
}

__global__ void bsr_spmv_kernel(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y) {
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (tid >= 4 * n) return;
    const int64_t i = tid >> 2;
    const int r = int(tid & 3);
    double acc = 0.0;
    for (int32_t b = rp[i]; b < rp[i + 1]; ++b) {
        const double* blk = A + 16 * int64_t(b) + 4 * r;
        const double* xv = x + 4 * int64_t(ci[b]);
        acc += blk[0] * xv[0] + blk[1] * xv[1] + blk[2] * xv[2] + blk[3] * xv[3];
    }
    y[tid] = acc;
}

// Group block of the global matrix: LU with partial pivoting in shared
// memory, then its inverse (one column per thread: the pivots, a forward and
// a back substitution of a unit vector), stored column-major in Ainv so that
// applying it is a coalesced dense product.  A zero pivot gives a zero
// component, as a triangular solve with that convention would.
template <int NPG>
__global__ void vanka_factor_kernel(int64_t ng, const int32_t* __restrict__ grp_blk, const double* __restrict__ A,
                                    double* __restrict__ Ainv, int32_t* __restrict__ piv) {
    constexpr int NL = 4 * NPG;
    extern __shared__ double sm[];
    double* M = sm;                          // NL x NL
    double* X = sm + NL * NL;                // NL x NL: X[i * NL + c] = (A^{-1})_{ic}
    __shared__ int s_p;
    __shared__ int s_piv[NL];
    const int64_t g = blockIdx.x;
    for (int e = threadIdx.x; e < NL * NL; e += blockDim.x) {
        const int i = e / NL, j = e % NL;
        const int32_t b = grp_blk[(g * NPG + i / 4) * NPG + j / 4];
        M[e] = A[16 * int64_t(b) + 4 * (i % 4) + (j % 4)];
    }
    __syncthreads();
    for (int k = 0; k < NL; ++k) {
        if (threadIdx.x == 0) {
            int best = k;
            double bv = fabs(M[k * NL + k]);
            for (int i = k + 1; i < NL; ++i)
                if (fabs(M[i * NL + k]) > bv) {
                    bv = fabs(M[i * NL + k]);
                    best = i;
                }
            s_p = best;
            s_piv[k] = best;
            piv[g * NL + k] = best;
        }
        __syncthreads();
        const int pr = s_p;
        if (pr != k)
            for (int j = threadIdx.x; j < NL; j += blockDim.x) {
                const double t = M[k * NL + j];
                M[k * NL + j] = M[pr * NL + j];
                M[pr * NL + j] = t;
            }
        __syncthreads();
        const double d = M[k * NL + k];
        const double inv = d != 0.0 ? 1.0 / d : 0.0;
        for (int i = k + 1 + threadIdx.x; i < NL; i += blockDim.x) M[i * NL + k] *= inv;
        __syncthreads();
        const int rem = NL - k - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int i = k + 1 + e / rem, j = k + 1 + e % rem;
            M[i * NL + j] -= M[i * NL + k] * M[k * NL + j];
        }
        __syncthreads();
    }
    const int c = threadIdx.x;
    if (c < NL) {
        for (int i = 0; i < NL; ++i) X[i * NL + c] = i == c ? 1.0 : 0.0;
        for (int k = 0; k < NL; ++k) {
            const int pr = s_piv[k];
            if (pr != k) {
                const double t = X[k * NL + c];
                X[k * NL + c] = X[pr * NL + c];
                X[pr * NL + c] = t;
            }
        }
        for (int i = 1; i < NL; ++i) {
            double acc = X[i * NL + c];
            for (int j = 0; j < i; ++j) acc -= M[i * NL + j] * X[j * NL + c];
            X[i * NL + c] = acc;
        }
        for (int i = NL - 1; i >= 0; --i) {
            double acc = X[i * NL + c];
            for (int j = i + 1; j < NL; ++j) acc -= M[i * NL + j] * X[j * NL + c];
            const double d = M[i * NL + i];
            X[i * NL + c] = d != 0.0 ? acc / d : 0.0;
        }
    }
    __syncthreads();
    // column-major: Ainv[g][j * NL + i] = (A^{-1})_{ij}
    for (int e = threadIdx.x; e < NL * NL; e += blockDim.x) {
        const int j = e / NL, i = e % NL;
        Ainv[g * NL * NL + e] = X[i * NL + j];
    }
}

// z_g = A_g^{-1} r restricted to group g: one block per group, thread i
// computes row i of the dense product (column-major inverse: coalesced).
template <int NPG>
__global__ void __launch_bounds__(128) vanka_apply_kernel(int64_t ng, const int32_t* __restrict__ groups,
                                                          const double* __restrict__ Ainv,
                                                          const double* __restrict__ r, double* __restrict__ zloc) {
    constexpr int NL = 4 * NPG;
    __shared__ double s_r[NL];
    const int64_t g = blockIdx.x;
    for (int e = threadIdx.x; e < NL; e += blockDim.x) s_r[e] = r[4 * int64_t(groups[g * NPG + e / 4]) + e % 4];
    __syncthreads();
    const double* Ag = Ainv + g * NL * NL;
    for (int i = threadIdx.x; i < NL; i += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < NL; ++j) acc += Ag[j * NL + i] * s_r[j];
        zloc[g * NL + i] = acc;
    }
}

// z_j = (1 / valence_j) sum of the groups' local solutions at node j
__global__ void vanka_average_kernel(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                     const double* __restrict__ zloc, double* __restrict__ z) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double a[4] = {0, 0, 0, 0};
    const int32_t e0 = ptr[j], e1 = ptr[j + 1];
    for (int32_t e = e0; e < e1; ++e)
        for (int c = 0; c < 4; ++c) a[c] += zloc[4 * int64_t(idx[e]) + c];
    const double mu = 1.0 / double(e1 - e0);
    for (int c = 0; c < 4; ++c) z[4 * j + c] = a[c] * mu;
}

// ---- vector kernels (FP64, deterministic reductions) -------------------------
constexpr int kRedBlocks = 256;

// sum over a warp by shuffles (a fixed tree: deterministic)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
// sum over a block of 256 threads: warp shuffles, then the 8 warp sums by warp 0
__device__ __forceinline__ double block_sum256(double v) {
    __shared__ double ws[8];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = threadIdx.x < 8 ? ws[threadIdx.x] : 0.0;
    if (threadIdx.x < 32) t = warp_sum(t);
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(256) dot_partial_kernel(int64_t n, const double* __restrict__ a,
                                                          const double* __restrict__ b, double* __restrict__ part) {
    double acc = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        acc += a[i] * b[i];
    acc = block_sum256(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
__global__ void __launch_bounds__(256) dot_final_kernel(const double* __restrict__ part, int np,
                                                        double* __restrict__ out) {
    const double t = block_sum256(threadIdx.x < np ? part[threadIdx.x] : 0.0);
    if (threadIdx.x == 0) *out = t;
}
// Classical Gram-Schmidt pieces: part[i * gridDim.x + b] = the partial
// <w, V_i> of block b for i = blockIdx.y; then out[i] = sum over blocks
// (one block per i); then w -= sum_i h[i] V_i in order i = 0..cnt-1.
__global__ void __launch_bounds__(256) multi_dot_partial_kernel(int64_t n, const double* __restrict__ w,
                                                                const double* __restrict__ V,
                                                                double* __restrict__ part) {
    const double* v = V + int64_t(blockIdx.y) * n;
    double acc = 0.0;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x)
        acc += w[k] * v[k];
    acc = block_sum256(acc);
    if (threadIdx.x == 0) part[int64_t(blockIdx.y) * gridDim.x + blockIdx.x] = acc;
}
__global__ void __launch_bounds__(256) multi_dot_final_kernel(const double* __restrict__ part, int nb,
                                                              double* __restrict__ out) {
    const double t = block_sum256(threadIdx.x < nb ? part[int64_t(blockIdx.x) * nb + threadIdx.x] : 0.0);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
}
__global__ void multi_axpy_kernel(int64_t n, int cnt, const double* __restrict__ h, const double* __restrict__ V,
                                  double* __restrict__ w) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        double acc = w[k];
        for (int i = 0; i < cnt; ++i) acc -= h[i] * V[int64_t(i) * n + k];
        w[k] = acc;
    }
}
__global__ void add_vec_kernel(int cnt, const double* __restrict__ a, double* __restrict__ b) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) b[i] += a[i];
}
// y += sgn * coef[0] * x
__global__ void axpy_dev_kernel(int64_t n, const double* __restrict__ coef, double sgn, const double* __restrict__ x,
                                double* __restrict__ y) {
    const double a = sgn * coef[0];
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] += a * x[i];
}
// y = x / sqrt(nrm2[0]); nrm2 holds a squared norm
__global__ void scale_inv_sqrt_kernel(int64_t n, const double* __restrict__ nrm2, const double* __restrict__ x,
                                      double* __restrict__ y) {
    const double s = nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = s * x[i];
}
__global__ void axpy_kernel(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        y[i] += a * x[i];
}
// p_j -= mean (only the pressure component)
__global__ void pressure_shift_kernel(int64_t n, const double* __restrict__ mean, double* __restrict__ x) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j < n) x[4 * j + 3] -= mean[0];
}
__global__ void extract_component_kernel(int64_t n, const double* __restrict__ x, int comp, double* __restrict__ p) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j < n) p[j] = x[4 * j + comp];
}
__global__ void mean_ratio_kernel(const double* __restrict__ num, const double* __restrict__ den,
                                  double* __restrict__ out) {
    *out = den[0] != 0.0 ? num[0] / den[0] : 0.0;
}

inline unsigned nblk(int64_t n, int per) { return unsigned((n + per - 1) / per); }

}  // namespace

// ---- device level + host drivers -------------------------------------------------

struct DeviceLevel {
    HostLevel h;
    int32_t* groups = nullptr;
    double* xyz = nullptr;
    uint8_t* dir = nullptr;
    int32_t *node_ptr = nullptr, *node_idx = nullptr, *row_ptr = nullptr, *col_idx = nullptr;
    int32_t *blk_ptr = nullptr, *blk_src = nullptr, *grp_blk = nullptr;
    double* A = nullptr;        // BSR values [nnzb][4][4]
    double* Jloc = nullptr;     // [ng][4 npg][4 npg]
    double* LU = nullptr;       // [ng][4 npg][4 npg]: the inverse of each group block, column-major
    int32_t* piv = nullptr;     // [ng][4 npg]
    double* local = nullptr;    // [ng][npg][4]
    double* zloc = nullptr;     // [ng][4 npg]
    double* mass = nullptr;     // [n] lumped mass
    double* work = nullptr;     // scratch vectors
    double* scal = nullptr;     // device scalars
    double* part = nullptr;     // reduction partials
    int krylov = 0;
    std::vector<void*> allocs;
    bool has_jacobian = false;
};

namespace {

template <typename T>
cudaError_t up(DeviceLevel* L, const std::vector<T>& v, T** out) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(v.size() * sizeof(T), 1));
    if (e != cudaSuccess) return e;
    L->allocs.push_back(p);
    if (!v.empty()) {
        e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    *out = static_cast<T*>(p);
    return cudaSuccess;
}
cudaError_t dalloc(DeviceLevel* L, size_t bytes, void** out) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 1));
    if (e != cudaSuccess) return e;
    L->allocs.push_back(p);
    *out = p;
    return cudaSuccess;
}

#define CKE(x)                                  \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

}  // namespace

void destroy_level(DeviceLevel* L) {
    if (!L) return;
    for (void* p : L->allocs) cudaFree(p);
    delete L;
}

cudaError_t create_level(const HostHierarchy& hh, bool fine, int krylov, DeviceLevel** out) {
    DeviceLevel* L = new DeviceLevel();
    build_level(hh, fine, &L->h);
    const HostLevel& h = L->h;
    auto fail = [&](cudaError_t e) {
        destroy_level(L);
        return e;
    };
    cudaError_t e;
    if ((e = up(L, h.groups, &L->groups)) != cudaSuccess) return fail(e);
    if ((e = up(L, h.xyz, &L->xyz)) != cudaSuccess) return fail(e);
    if ((e = up(L, h.dir, &L->dir)) != cudaSuccess) return fail(e);
    if ((e = up(L, h.node_ptr, &L->node_ptr)) != cudaSuccess) return fail(e);
    if ((e = up(L, h.node_idx, &L->node_idx)) != cudaSuccess) return fail(e);
    if ((e = up(L, h.row_ptr, &L->row_ptr)) != cudaSuccess) return fail(e);
    if ((e = up(L, h.col_idx, &L->col_idx)) != cudaSuccess) return fail(e);
    if ((e = up(L, h.blk_ptr, &L->blk_ptr)) != cudaSuccess) return fail(e);
    if ((e = up(L, h.blk_src, &L->blk_src)) != cudaSuccess) return fail(e);
    if ((e = up(L, h.grp_blk, &L->grp_blk)) != cudaSuccess) return fail(e);
    const size_t nl = size_t(4 * h.npg);
    const size_t nnzb = h.col_idx.size();
    void* p;
    if ((e = dalloc(L, nnzb * 16 * 8, &p)) != cudaSuccess) return fail(e);
    L->A = static_cast<double*>(p);
    if ((e = dalloc(L, size_t(h.ng) * nl * nl * 8, &p)) != cudaSuccess) return fail(e);
    L->Jloc = static_cast<double*>(p);
    if ((e = dalloc(L, size_t(h.ng) * nl * nl * 8, &p)) != cudaSuccess) return fail(e);
    L->LU = static_cast<double*>(p);
    if ((e = dalloc(L, size_t(h.ng) * nl * 4, &p)) != cudaSuccess) return fail(e);
    L->piv = static_cast<int32_t*>(p);
    if ((e = dalloc(L, size_t(h.ng) * nl * 8, &p)) != cudaSuccess) return fail(e);
    L->local = static_cast<double*>(p);
    if ((e = dalloc(L, size_t(h.ng) * nl * 8, &p)) != cudaSuccess) return fail(e);
    L->zloc = static_cast<double*>(p);
    if ((e = dalloc(L, size_t(h.n) * 8, &p)) != cudaSuccess) return fail(e);
    L->mass = static_cast<double*>(p);
    L->krylov = krylov;
    // work vectors: r, dx, tmp, z, p, + (krylov + 1) basis vectors
    if ((e = dalloc(L, size_t(4 * h.n) * 8 * size_t(6 + krylov + 1), &p)) != cudaSuccess) return fail(e);
    L->work = static_cast<double*>(p);
    if ((e = dalloc(L, size_t(krylov + 2) * size_t(krylov + 2) * 8 + 64 * 8, &p)) != cudaSuccess) return fail(e);
    L->scal = static_cast<double*>(p);
    if ((e = dalloc(L, size_t(kRedBlocks) * size_t(krylov + 1) * 8, &p)) != cudaSuccess) return fail(e);
    L->part = static_cast<double*>(p);   // reduction partials, kRedBlocks per vector
    *out = L;
    return cudaSuccess;
}

int64_t level_nodes(const DeviceLevel* L) { return L->h.n; }
bool level_lps(const DeviceLevel* L) { return L->h.lps; }

namespace {

LvPrm make_prm(const OpParams& op, const dnnmg_solver_params* sp) {
    LvPrm p;
    p.m = op.m;
    p.th = op.theta;
    p.nu = op.nu;
    p.a0 = sp ? sp->alpha0 : 0.02;
    p.d0 = sp ? sp->delta0 : 0.1;
    p.lps = 1;
    return p;
}

template <int MODE>
cudaError_t local_terms(DeviceLevel* L, const double* x, LvPrm p, cudaStream_t s) {
    const HostLevel& h = L->h;
    p.lps = h.lps ? p.lps : 0;
    if (h.npg == 27)
        level_local_kernel<27, MODE><<<nblk(h.ng, 64), 64, 0, s>>>(h.ng, L->groups, L->xyz, x, p, L->local);
    else
        level_local_kernel<8, MODE><<<nblk(h.ng, 64), 64, 0, s>>>(h.ng, L->groups, L->xyz, x, p, L->local);
    CKE(cudaGetLastError());
    node_gather_kernel<<<nblk(h.n, 256), 256, 0, s>>>(h.n, L->node_ptr, L->node_idx, L->local,
                                                        L->work + 2 * 4 * h.n);   // tmp
    return cudaGetLastError();
}

cudaError_t dot(DeviceLevel* L, const double* a, const double* b, int64_t n, double* out_dev, cudaStream_t s) {
    dot_partial_kernel<<<kRedBlocks, 256, 0, s>>>(n, a, b, L->part);
    dot_final_kernel<<<1, 256, 0, s>>>(L->part, kRedBlocks, out_dev);
    return cudaGetLastError();
}

// One classical Gram-Schmidt pass against V_0..V_{cnt-1}: h = V^T w, w -= V h.
cudaError_t cgs_pass(DeviceLevel* L, double* w, const double* V, int cnt, int64_t n, double* h, cudaStream_t s) {
    multi_dot_partial_kernel<<<dim3(kRedBlocks, unsigned(cnt)), 256, 0, s>>>(n, w, V, L->part);
    multi_dot_final_kernel<<<unsigned(cnt), 256, 0, s>>>(L->part, kRedBlocks, h);
    multi_axpy_kernel<<<256, 256, 0, s>>>(n, cnt, h, V, w);
    return cudaGetLastError();
}

cudaError_t fetch(double* host, const double* dev, size_t n, cudaStream_t s) {
    CKE(cudaMemcpyAsync(host, dev, n * 8, cudaMemcpyDeviceToHost, s));
    return cudaStreamSynchronize(s);
}

// Lumped mass (integral of each basis function) into L->mass and its sum
// into the device scalar L->scal[2].
cudaError_t compute_mass(DeviceLevel* L, const OpParams& op, cudaStream_t s) {
    CKE(local_terms<LV_MASS>(L, nullptr, make_prm(op, nullptr), s));
    const int64_t n = L->h.n;
    extract_component_kernel<<<nblk(n, 256), 256, 0, s>>>(n, L->work + 2 * 4 * n, 0, L->mass);
    CKE(cudaGetLastError());
    std::vector<double> mh(static_cast<size_t>(n));
    CKE(fetch(mh.data(), L->mass, static_cast<size_t>(n), s));
    double sum = 0.0;
    for (double v : mh) sum += v;
    CKE(cudaMemcpyAsync(L->scal + 2, &sum, 8, cudaMemcpyHostToDevice, s));
    return cudaStreamSynchronize(s);
}

}  // namespace

// r = b - A(x) with Dirichlet / pin rows zero
cudaError_t level_residual(DeviceLevel* L, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                           const double* b, double* r, cudaStream_t s) {
    CKE(local_terms<LV_OPERATOR>(L, x, make_prm(op, sp), s));
    const int64_t n = L->h.n;
    CKE(cudaMemcpyAsync(r, L->work + 2 * 4 * n, size_t(4 * n) * 8, cudaMemcpyDeviceToDevice, s));
    finish_rows_kernel<<<nblk(n, 256), 256, 0, s>>>(n, b, r, L->dir, L->h.pin, 1, 0);
    return cudaGetLastError();
}

// A(x) as assembled (no row modification)
cudaError_t level_operator(DeviceLevel* L, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                           double* Ax, cudaStream_t s) {
    CKE(local_terms<LV_OPERATOR>(L, x, make_prm(op, sp), s));
    return cudaMemcpyAsync(Ax, L->work + 2 * 4 * L->h.n, size_t(4 * L->h.n) * 8, cudaMemcpyDeviceToDevice, s);
}

// b(x_old): rhs of Eq. (6), Dirichlet velocity rows and pressure rows zero
cudaError_t level_rhs(DeviceLevel* L, const OpParams& op, const double* x_old, double* b, cudaStream_t s) {
    CKE(local_terms<LV_RHS>(L, x_old, make_prm(op, nullptr), s));
    const int64_t n = L->h.n;
    CKE(cudaMemcpyAsync(b, L->work + 2 * 4 * n, size_t(4 * n) * 8, cudaMemcpyDeviceToDevice, s));
    finish_rows_kernel<<<nblk(n, 256), 256, 0, s>>>(n, nullptr, b, L->dir, -1, 0, 1);
    return cudaGetLastError();
}

// Jacobian dA/dx at x into the BSR matrix (rows of fixed unknowns = identity)
cudaError_t level_jacobian(DeviceLevel* L, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                           cudaStream_t s) {
    const HostLevel& h = L->h;
    LvPrm p = make_prm(op, sp);
    p.lps = h.lps ? 1 : 0;
    const int nl = 4 * h.npg;
    if (h.npg == 27)
        level_jacobian_kernel<27><<<nblk(h.ng * nl, 128), 128, 0, s>>>(h.ng, L->groups, L->xyz, x, p, L->Jloc);
    else
        level_jacobian_kernel<8><<<nblk(h.ng * nl, 128), 128, 0, s>>>(h.ng, L->groups, L->xyz, x, p, L->Jloc);
    CKE(cudaGetLastError());
    const int64_t nnzb = int64_t(h.col_idx.size());
    if (h.npg == 27)
        bsr_assemble_kernel<27><<<nblk(nnzb * 16, 256), 256, 0, s>>>(nnzb, L->blk_ptr, L->blk_src, L->Jloc, L->A);
    else
        bsr_assemble_kernel<8><<<nblk(nnzb * 16, 256), 256, 0, s>>>(nnzb, L->blk_ptr, L->blk_src, L->Jloc, L->A);
    CKE(cudaGetLastError());
    bsr_dirichlet_kernel<<<nblk(h.n, 128), 128, 0, s>>>(h.n, L->row_ptr, L->col_idx, L->dir, h.pin, L->A);
    CKE(cudaGetLastError());
    // group-Vanka factors
    const size_t smem = 2 * size_t(nl) * nl * 8;   // the LU and the inverse
    if (h.npg == 27) {
        CKE(cudaFuncSetAttribute(vanka_factor_kernel<27>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        vanka_factor_kernel<27><<<unsigned(h.ng), 256, smem, s>>>(h.ng, L->grp_blk, L->A, L->LU, L->piv);
    } else {
        vanka_factor_kernel<8><<<unsigned(h.ng), 256, smem, s>>>(h.ng, L->grp_blk, L->A, L->LU, L->piv);
    }
    L->has_jacobian = true;
    return cudaGetLastError();
}

// dense copy of the assembled matrix (small levels; tests)
cudaError_t level_dense_jacobian(DeviceLevel* L, double* dense_host) {
    const HostLevel& h = L->h;
    const size_t nnzb = h.col_idx.size();
    std::vector<double> A(nnzb * 16);
    CKE(cudaMemcpy(A.data(), L->A, A.size() * 8, cudaMemcpyDeviceToHost));
    const int64_t N = 4 * h.n;
    std::fill(dense_host, dense_host + N * N, 0.0);
    for (int64_t i = 0; i < h.n; ++i)
        for (int32_t b = h.row_ptr[i]; b < h.row_ptr[i + 1]; ++b)
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c)
                    dense_host[(4 * i + r) * N + 4 * int64_t(h.col_idx[b]) + c] = A[16 * size_t(b) + 4 * r + c];
    return cudaSuccess;
}

namespace {

cudaError_t precond(DeviceLevel* L, const double* r, double* z, cudaStream_t s) {
    const HostLevel& h = L->h;
    if (h.npg == 27)
        vanka_apply_kernel<27><<<unsigned(h.ng), 128, 0, s>>>(h.ng, L->groups, L->LU, r, L->zloc);
    else
        vanka_apply_kernel<8><<<unsigned(h.ng), 128, 0, s>>>(h.ng, L->groups, L->LU, r, L->zloc);
    CKE(cudaGetLastError());
    vanka_average_kernel<<<nblk(h.n, 256), 256, 0, s>>>(h.n, L->node_ptr, L->node_idx, L->zloc, z);
    return cudaGetLastError();
}

cudaError_t spmv(DeviceLevel* L, const double* x, double* y, cudaStream_t s) {
    const int64_t n = L->h.n;
    bsr_spmv_kernel<<<nblk(4 * n, 256), 256, 0, s>>>(n, L->row_ptr, L->col_idx, L->A, x, y);
    return cudaGetLastError();
}

// Right-preconditioned restarted GMRES for J dx = r (dx zero on entry).
cudaError_t gmres(DeviceLevel* L, const double* r, double* dx, double rtol, int max_it, cudaStream_t s,
                  int* iters, double* res_out) {
    const int64_t n4 = 4 * L->h.n;
    const int m = L->krylov;
    double* z = L->work + 3 * n4;
    double* w = L->work + 5 * n4;
    double* V = L->work + 6 * n4;   // (m + 1) vectors
    double* H = L->scal + 64;       // (m+1) x m column-major on the device: H[i + j*(m+1)], then m+1 scratch
    std::vector<double> Hh(size_t(m + 1) * m), cs(m), sn(m), gvec(m + 1), y(m);
    cudaMemsetAsync(dx, 0, size_t(n4) * 8, s);
    double beta0 = 0.0;
    {
        CKE(dot(L, r, r, n4, L->scal, s));
        double t;
        CKE(fetch(&t, L->scal, 1, s));
        beta0 = std::sqrt(t);
    }
    *iters = 0;
    *res_out = beta0;
    if (beta0 == 0.0) return cudaSuccess;
    // residual of the current iterate: r - J dx; start from r
    double* rr = L->work + 4 * n4;   // shares the pressure scratch: not used concurrently
    CKE(cudaMemcpyAsync(rr, r, size_t(n4) * 8, cudaMemcpyDeviceToDevice, s));
    double beta = beta0;
    while (*iters < max_it) {
        // v0 = rr / beta
        CKE(dot(L, rr, rr, n4, L->scal, s));
        scale_inv_sqrt_kernel<<<256, 256, 0, s>>>(n4, L->scal, rr, V);
        std::fill(gvec.begin(), gvec.end(), 0.0);
        gvec[0] = beta;
        int j = 0;
        for (; j < m && *iters < max_it; ++j, ++(*iters)) {
            double* vj = V + int64_t(j) * n4;
            double* vn = V + int64_t(j + 1) * n4;
            CKE(precond(L, vj, z, s));
            CKE(spmv(L, z, w, s));
            // orthogonalise against V_0..V_j: classical Gram-Schmidt twice (as
            // robust as the modified form, two multi-vector passes instead of
            // 2 (j + 1) single ones); the column gets the sum of both passes
            double* hcol = H + j * (m + 1);
            double* h2 = H + size_t(m + 1) * m;   // scratch column after H
            CKE(cgs_pass(L, w, V, j + 1, n4, hcol, s));
            CKE(cgs_pass(L, w, V, j + 1, n4, h2, s));
            add_vec_kernel<<<1, 64, 0, s>>>(j + 1, h2, hcol);
            double* hn = H + (j + 1) + j * (m + 1);
            CKE(dot(L, w, w, n4, hn, s));
            scale_inv_sqrt_kernel<<<256, 256, 0, s>>>(n4, hn, w, vn);
            CKE(fetch(Hh.data() + size_t(j) * (m + 1), H + j * (m + 1), size_t(j + 2), s));
            double* col = Hh.data() + size_t(j) * (m + 1);
            col[j + 1] = std::sqrt(std::max(col[j + 1], 0.0));
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * col[i] + sn[i] * col[i + 1];
                col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                col[i] = t;
            }
            const double den = std::hypot(col[j], col[j + 1]);
            cs[j] = den > 0 ? col[j] / den : 1.0;
            sn[j] = den > 0 ? col[j + 1] / den : 0.0;
            col[j] = den;
            col[j + 1] = 0.0;
            gvec[j + 1] = -sn[j] * gvec[j];
            gvec[j] = cs[j] * gvec[j];
            beta = std::fabs(gvec[j + 1]);
            if (beta <= rtol * beta0) {
                ++j;
                ++(*iters);
                break;
            }
        }
        // y = R^{-1} g; dx += M^{-1} V y
        for (int i = j - 1; i >= 0; --i) {
            double t = gvec[i];
            for (int k = i + 1; k < j; ++k) t -= Hh[size_t(k) * (m + 1) + i] * y[k];
            y[i] = t / Hh[size_t(i) * (m + 1) + i];
        }
        double* comb = w;
        CKE(cudaMemsetAsync(comb, 0, size_t(n4) * 8, s));
        for (int i = 0; i < j; ++i) axpy_kernel<<<256, 256, 0, s>>>(n4, y[i], V + int64_t(i) * n4, comb);
        CKE(precond(L, comb, z, s));
        axpy_kernel<<<256, 256, 0, s>>>(n4, 1.0, z, dx);
        CKE(cudaGetLastError());
        if (beta <= rtol * beta0 || *iters >= max_it) break;
        // true residual for the restart: rr = r - J dx
        CKE(spmv(L, dx, rr, s));
        CKE(cudaMemcpyAsync(w, r, size_t(n4) * 8, cudaMemcpyDeviceToDevice, s));
        axpy_kernel<<<256, 256, 0, s>>>(n4, -1.0, rr, w);
        CKE(cudaMemcpyAsync(rr, w, size_t(n4) * 8, cudaMemcpyDeviceToDevice, s));
        CKE(dot(L, rr, rr, n4, L->scal, s));
        double t;
        CKE(fetch(&t, L->scal, 1, s));
        beta = std::sqrt(t);
        if (beta <= rtol * beta0) break;
    }
    *res_out = beta;
    return cudaSuccess;
}

}  // namespace

// Newton solve of A(x) = b on level L; x holds the Dirichlet values (and the
// initial guess) on entry.
cudaError_t level_solve(DeviceLevel* L, const OpParams& op, const dnnmg_solver_params* sp, const double* b, double* x,
                        cudaStream_t s, dnnmg_solve_stats* st) {
    const int64_t n = L->h.n, n4 = 4 * n;
    double* r = L->work;
    double* dx = L->work + n4;
    dnnmg_solve_stats stats{};
    if (L->h.mean_zero_pressure) CKE(compute_mass(L, op, s));
    double r0 = -1.0, rprev = -1.0;
    bool reassemble = true;
    for (int it = 0;; ++it) {
        CKE(level_residual(L, op, sp, x, b, r, s));
        CKE(dot(L, r, r, n4, L->scal, s));
        double t;
        CKE(fetch(&t, L->scal, 1, s));
        const double rn = std::sqrt(t);
        if (!std::isfinite(rn)) {
            stats.residual = rn;
            if (st) *st = stats;
            return cudaErrorUnknown;   // reported as NaN by the caller
        }
        if (r0 < 0) r0 = rn;
        stats.residual0 = r0;
        stats.residual = rn;
        stats.newton_iterations = it;
        if (rn <= sp->newton_atol || rn <= sp->newton_rtol * r0) {
            stats.converged = 1;
            break;
        }
        if (it >= sp->newton_max) break;
        if (rprev > 0 && rn / rprev > sp->rho_max) reassemble = true;
        if (reassemble || !L->has_jacobian) {
            CKE(level_jacobian(L, op, sp, x, s));
            stats.jacobian_assemblies++;
            reassemble = false;
        }
        rprev = rn;
        int gi = 0;
        double gres = 0.0;
        CKE(gmres(L, r, dx, sp->gmres_rtol, sp->gmres_max, s, &gi, &gres));
        stats.gmres_iterations += gi;
        axpy_kernel<<<256, 256, 0, s>>>(n4, 1.0, dx, x);
        CKE(cudaGetLastError());
        if (L->h.mean_zero_pressure) {
            // p -= (mass . p) / (mass . 1)
            double* pv = L->work + 2 * n4;   // tmp (n entries used)
            extract_component_kernel<<<nblk(n, 256), 256, 0, s>>>(n, x, 3, pv);
            CKE(dot(L, L->mass, pv, n, L->scal + 1, s));
            mean_ratio_kernel<<<1, 1, 0, s>>>(L->scal + 1, L->scal + 2, L->scal + 3);
            pressure_shift_kernel<<<nblk(n, 256), 256, 0, s>>>(n, L->scal + 3, x);
            CKE(cudaGetLastError());
        }
    }
    L->has_jacobian = false;   // next solve starts with a fresh Jacobian
    if (st) *st = stats;
    return cudaSuccess;
}

}  // namespace dnnmg
