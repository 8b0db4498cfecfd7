// Newton-Krylov-multigrid solve of A_h(x) = b on one mesh level (Sec. 3.4).
//
// The paper solves each time step's nonlinear system on the coarse level
// with Newton's method (stabilisation parameters frozen in the Jacobian),
// GMRES and a geometric multigrid preconditioner with a Vanka smoother whose
// local problems are the 108 x 108 matrices of one Q2 cell.  Here:
//   * the operator A_h is the Q1/Q1 form of Eqs. (5)-(6) with the two-level
//     local projection on groups of 8 child cells (27 nodes = one Q2 cell's
//     nodes), evaluated per group in FP64; Newton residual norms are FP64;
//   * the Jacobian is the exact derivative of A_h (alpha_T, delta_T frozen,
//     Eq. (8)), formed column by column per group from closed-form
//     derivatives of every term (FP32 on the solve and smoothing levels,
//     FP64 on the coarsest level); the local 108 x 108 matrices are summed
//     into a 4 x 4-block CSR matrix by a gather in group order
//     (deterministic);
//   * the preconditioner is a geometric multigrid V-cycle over the levels
//     below (each the parents of the groups of the next finer one), with
//     additive group-Vanka smoothing in FP32: the matrix restricted to each
//     group's 108 unknowns, LU-factorised and inverted once per assembly,
//     applied as a dense product, averaged over the groups sharing a node and
//     damped; restriction R = P^T and trilinear prolongation P between
//     levels; on the coarsest level a dense LU with partial pivoting and its
//     explicit inverse in FP64.  Without coarser levels the preconditioner
//     is one group-Vanka application;
//   * flexible restarted GMRES (the preconditioned vectors are kept, so an
//     FP32 preconditioner does not limit the FP64 solution) with classical
//     Gram-Schmidt applied twice; vectors, dot products (warp shuffles, then
//     a second pass over the blocks: fixed order), norms and the Givens
//     rotations in FP64, on the device; the host reads the residual estimate
//     every few iterations only;
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

// largest coarsest multigrid level for the dense FP64 LU (unknowns): 8192^2
// doubles = 512 MiB per buffer
constexpr int64_t kMaxCoarsestUnknowns = 8192;

namespace {

constexpr double kGaussOff = 0.28867513459481288225457439025098;

__device__ __forceinline__ double val(double x) { return x; }
template <typename T>
__device__ __forceinline__ T zero() { return T{}; }
template <>
__device__ __forceinline__ double zero<double>() { return 0.0; }
template <typename T>
__device__ __forceinline__ T lift(double x);
template <>
__device__ __forceinline__ double lift<double>(double x) { return x; }

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


// Local residual / rhs / mass of 27-node groups with one thread per child
// cell: a block takes 8 groups (their coordinates, values and projected
// values in shared memory), each thread adds its child's terms into its own
// slice, and the 8 slices of a group are summed in child order.
constexpr int kChildGroups = 8;
constexpr size_t kChildSmem = size_t(kChildGroups) * (27 * 3 + 2 * 27 * 4 + 8 * 27 * 4) * sizeof(double);

template <int MODE>
__global__ void __launch_bounds__(64) level_local_child_kernel(int64_t ng, const int32_t* __restrict__ groups,
                                                               const double* __restrict__ xyz,
                                                               const double* __restrict__ x, LvPrm p,
                                                               double* __restrict__ out) {
    extern __shared__ __align__(16) double lc_smem[];
    auto X = reinterpret_cast<double (*)[27][3]>(lc_smem);
    auto U = reinterpret_cast<double (*)[27][4]>(lc_smem + kChildGroups * 81);
    auto PU = reinterpret_cast<double (*)[27][4]>(lc_smem + kChildGroups * (81 + 108));
    auto R = reinterpret_cast<double (*)[8][27][4]>(lc_smem + kChildGroups * (81 + 216));
    const int64_t g0 = int64_t(blockIdx.x) * kChildGroups;
    for (int e = threadIdx.x; e < kChildGroups * 27; e += blockDim.x) {
        const int gg = e / 27, i = e % 27;
        const int64_t g = g0 + gg;
        if (g >= ng) continue;
        const int64_t n = groups[g * 27 + i];
        for (int d = 0; d < 3; ++d) X[gg][i][d] = xyz[3 * n + d];
        for (int c = 0; c < 4; ++c) U[gg][i][c] = MODE == LV_MASS ? 0.0 : x[4 * n + c];
    }
    for (int e = threadIdx.x; e < kChildGroups * 8 * 108; e += blockDim.x) (&R[0][0][0][0])[e] = 0.0;
    __syncthreads();
    if (MODE == LV_OPERATOR)
        for (int e = threadIdx.x; e < kChildGroups * 27; e += blockDim.x) {
            const int gg = e / 27, i = e % 27;
            for (int c = 0; c < 4; ++c) {
                double a = 0.0;
                for (int K = 0; K < 8; ++K) {
                    const double wk = wpi(i, K);
                    if (wk != 0.0) a += wk * U[gg][corner_node(K)][c];
                }
                PU[gg][i][c] = a;
            }
        }
    __syncthreads();
    const int gl = threadIdx.x >> 3, t = threadIdx.x & 7;
    if (g0 + gl < ng) child_terms<double, 27, MODE>(X[gl], U[gl], PU[gl], t, p, R[gl][t]);
    __syncthreads();
    for (int e = threadIdx.x; e < kChildGroups * 108; e += blockDim.x) {
        const int gg = e / 108, k = e % 108;
        const int64_t g = g0 + gg;
        if (g >= ng) continue;
        double a = 0.0;
        for (int c = 0; c < 8; ++c) a += R[gg][c][k >> 2][k & 3];
        out[g * 108 + k] = a;
    }
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

// ---- Jacobian from closed-form derivatives ------------------------------------
//
// Column (b, e) of a group's local matrix is the derivative of the group's
// local residual with respect to unknown e of group node b.  With phi_b the
// child basis function of b, Pi_b the parent (group) trilinear function of b
// when b is a group corner (zero otherwise), and the frozen parameters:
//   velocity e: mass m phi_a phi_b delta_ce; convection theta phi_a
//     (phi_b d_e v_c + delta_ce v.grad phi_b); viscosity theta nu delta_ce
//     grad phi_a.grad phi_b; continuity phi_a d_e phi_b; projection term
//     delta_T [g'_c (v.grad phi_a) + g_c phi_b d_e phi_a] on child nodes and
//     -delta_T [g'_c (pi v.grad Pi_K) + g_c Pi_b d_e Pi_K] on corners K, with
//     g = v.grad v - pi v.grad pi v and g'_c = phi_b d_e v_c + delta_ce
//     v.grad phi_b - Pi_b d_e (pi v)_c - delta_ce pi v.grad Pi_b;
//   pressure: -d_c phi_a phi_b; alpha_T grad(phi_b - Pi_b).grad phi_a on
//     child nodes and -alpha_T grad(phi_b - Pi_b).grad Pi_K on corners.
// On a level without parents used as the coarsest multigrid level (8-node
// cells, stab != 0) the projection is taken as zero, which leaves the
// stabilisation terms with full fluctuations.

// per quadrature point of a child: everything the columns read
template <typename T>
struct QPoint {
    T w, N[8], G[8][3];      // weight x det J, child basis values, physical gradients
    T Pi[8], dPi[8][3];      // parent trilinear basis of the 8 group corners
    T v[3], Dv[3][3];        // velocity and gradient (Dv[c][d] = d v_c / d x_d)
    T pv[3], Dpv[3][3];      // projected velocity pi v and its gradient
    T gv[3];                 // v.grad v - pi v.grad pi v
};

template <typename T, int NPG>
constexpr size_t jac_smem_bytes() {
    return size_t(NPG == 27 ? 64 : 8) * sizeof(QPoint<T>) + size_t(4 * NPG) * size_t(4 * NPG) * sizeof(T);
}

template <typename T, int NPG>
__global__ void __launch_bounds__(128) jacobian_kernel(int64_t ng, const int32_t* __restrict__ groups,
                                                       const double* __restrict__ xyz,
                                                       const double* __restrict__ x, LvPrm p, int stab,
                                                       T* __restrict__ Jloc) {
    constexpr int NL = 4 * NPG;
    constexpr int NCH = NPG == 27 ? 8 : 1;
    constexpr int NQ = 8 * NCH;
    extern __shared__ __align__(16) unsigned char jac_smem[];
    QPoint<T>* P = reinterpret_cast<QPoint<T>*>(jac_smem);
    T* M = reinterpret_cast<T*>(jac_smem + size_t(NQ) * sizeof(QPoint<T>));   // [NL][NL]
    __shared__ double Xs[NPG][3];
    __shared__ T Us[NPG][4];
    __shared__ T prm_s[NCH][2];
    const int64_t g = blockIdx.x;
    for (int i = threadIdx.x; i < NPG; i += blockDim.x) {
        const int64_t n = groups[g * NPG + i];
        for (int d = 0; d < 3; ++d) Xs[i][d] = xyz[3 * n + d];
        for (int c = 0; c < 4; ++c) Us[i][c] = T(x[4 * n + c]);
    }
    for (int e = threadIdx.x; e < NL * NL; e += blockDim.x) M[e] = T(0);
    __syncthreads();
    if (threadIdx.x < NQ) {
        const int t = threadIdx.x >> 3, q = threadIdx.x & 7;
        QPoint<T>& Q = P[threadIdx.x];
        int nd[8];
        for (int k = 0; k < 8; ++k) nd[k] = child_node<NPG>(t, k);
        T J[3][3];
        for (int d = 0; d < 3; ++d)
            for (int e = 0; e < 3; ++e) {
                T s = T(0);
                for (int k = 1; k < 8; ++k) s += T(Xs[nd[k]][d] - Xs[nd[0]][d]) * T(dbasis(k, q, e));
                J[d][e] = s;
            }
        const T c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const T c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        const T det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        const T idet = T(1) / det;
        T Ji[3][3];
        Ji[0][0] = c00 * idet;
        Ji[1][0] = c01 * idet;
        Ji[2][0] = c02 * idet;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * idet;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * idet;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * idet;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * idet;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * idet;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * idet;
        Q.w = T(0.125) * det;
        for (int k = 0; k < 8; ++k) {
            Q.N[k] = T(basis(k, q));
            for (int d = 0; d < 3; ++d)
                Q.G[k][d] = T(dbasis(k, q, 0)) * Ji[0][d] + T(dbasis(k, q, 1)) * Ji[1][d] + T(dbasis(k, q, 2)) * Ji[2][d];
        }
        // parent basis at the point's parent reference coordinates (t_d + xi_d) / 2
        const bool par = NPG == 27 && stab;
        for (int K = 0; K < 8; ++K) {
            T val = T(par ? 1 : 0), dr[3] = {T(par ? 0.5 : 0), T(par ? 0.5 : 0), T(par ? 0.5 : 0)};
            if (par)
                for (int d = 0; d < 3; ++d) {
                    const T xp = T(0.5 * (((t >> d) & 1) + gpt((q >> d) & 1)));
                    const T f = ((K >> d) & 1) ? xp : T(1) - xp;
                    const T df = ((K >> d) & 1) ? T(1) : T(-1);
                    val *= f;
                    for (int e = 0; e < 3; ++e) dr[e] *= (e == d) ? df : f;
                }
            Q.Pi[K] = val;
            for (int d = 0; d < 3; ++d) Q.dPi[K][d] = dr[0] * Ji[0][d] + dr[1] * Ji[1][d] + dr[2] * Ji[2][d];
        }
        for (int c = 0; c < 3; ++c) {
            T v = T(0), pv = T(0);
            T Dv[3] = {T(0), T(0), T(0)}, Dp[3] = {T(0), T(0), T(0)};
            for (int k = 0; k < 8; ++k) {
                const T u = Us[nd[k]][c];
                v += Q.N[k] * u;
                for (int d = 0; d < 3; ++d) Dv[d] += Q.G[k][d] * u;
                const T uc = Us[corner_node(k) < NPG ? corner_node(k) : 0][c];
                if (par) {
                    pv += Q.Pi[k] * uc;
                    for (int d = 0; d < 3; ++d) Dp[d] += Q.dPi[k][d] * uc;
                }
            }
            Q.v[c] = v;
            Q.pv[c] = pv;
            for (int d = 0; d < 3; ++d) {
                Q.Dv[c][d] = Dv[d];
                Q.Dpv[c][d] = Dp[d];
            }
        }
        for (int c = 0; c < 3; ++c)
            Q.gv[c] = Q.v[0] * Q.Dv[c][0] + Q.v[1] * Q.Dv[c][1] + Q.v[2] * Q.Dv[c][2] -
                      (Q.pv[0] * Q.Dpv[c][0] + Q.pv[1] * Q.Dpv[c][1] + Q.pv[2] * Q.Dpv[c][2]);
    }
    if (threadIdx.x < NCH) {
        // frozen alpha_T, delta_T of child t (Eq. (8)) from the iterate's values
        const int t = threadIdx.x;
        double h = 0.0, vmax = 0.0;
        for (int a = 0; a < 8; ++a) {
            const int na = child_node<NPG>(t, a);
            for (int b = a + 1; b < 8; ++b) {
                const int nb = child_node<NPG>(t, b);
                double s = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double t0 = Xs[na][d] - Xs[nb][d];
                    s += t0 * t0;
                }
                h = fmax(h, sqrt(s));
            }
            double s = 0.0;
            for (int d = 0; d < 3; ++d) s += double(Us[na][d]) * double(Us[na][d]);
            vmax = fmax(vmax, sqrt(s));
        }
        const double den = p.nu / (h * h) + vmax / h + p.m;
        prm_s[t][0] = T(stab ? p.a0 / den : 0.0);
        prm_s[t][1] = T(stab ? p.d0 / den : 0.0);
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < NL) {
        const int b = j >> 2, e = j & 3;
        int Kb = -1;
        if (NPG == 27 && stab)
            for (int K = 0; K < 8; ++K)
                if (corner_node(K) == b) Kb = K;
        const T m = T(p.m), th = T(p.th), nu = T(p.nu);
        for (int t = 0; t < NCH; ++t) {
            int bl = -1, nd[8];
            for (int k = 0; k < 8; ++k) {
                nd[k] = child_node<NPG>(t, k);
                if (nd[k] == b) bl = k;
            }
            if (bl < 0 && Kb < 0) continue;
            const T aT = prm_s[t][0], dT = prm_s[t][1];
            for (int q = 0; q < 8; ++q) {
                const QPoint<T>& Q = P[t * 8 + q];
                const T w = Q.w;
                const T phib = bl >= 0 ? Q.N[bl] : T(0);
                T gb[3], gP[3];
                for (int d = 0; d < 3; ++d) {
                    gb[d] = bl >= 0 ? Q.G[bl][d] : T(0);
                    gP[d] = Kb >= 0 ? Q.dPi[Kb][d] : T(0);
                }
                const T Pib = Kb >= 0 ? Q.Pi[Kb] : T(0);
                if (e < 3) {
                    const T vgb = Q.v[0] * gb[0] + Q.v[1] * gb[1] + Q.v[2] * gb[2];
                    if (bl >= 0)
                        for (int a = 0; a < 8; ++a) {
                            const T Na = Q.N[a];
                            const T ggb = Q.G[a][0] * gb[0] + Q.G[a][1] * gb[1] + Q.G[a][2] * gb[2];
                            T* row = M + (4 * nd[a]) * NL + j;
                            for (int c = 0; c < 3; ++c) {
                                T val = th * Na * phib * Q.Dv[c][e];
                                if (c == e) val += m * Na * phib + th * Na * vgb + th * nu * ggb;
                                row[c * NL] += w * val;
                            }
                            row[3 * NL] += w * Na * gb[e];
                        }
                    if (stab) {
                        const T pvgP = Q.pv[0] * gP[0] + Q.pv[1] * gP[1] + Q.pv[2] * gP[2];
                        T gvp[3];
                        for (int c = 0; c < 3; ++c) {
                            gvp[c] = phib * Q.Dv[c][e] - Pib * Q.Dpv[c][e];
                            if (c == e) gvp[c] += vgb - pvgP;
                        }
                        for (int a = 0; a < 8; ++a) {
                            const T vGa = Q.v[0] * Q.G[a][0] + Q.v[1] * Q.G[a][1] + Q.v[2] * Q.G[a][2];
                            T* row = M + (4 * nd[a]) * NL + j;
                            for (int c = 0; c < 3; ++c) row[c * NL] += dT * w * (gvp[c] * vGa + Q.gv[c] * phib * Q.G[a][e]);
                        }
                        if (NPG == 27)
                            for (int K = 0; K < 8; ++K) {
                                const T pvdP = Q.pv[0] * Q.dPi[K][0] + Q.pv[1] * Q.dPi[K][1] + Q.pv[2] * Q.dPi[K][2];
                                T* row = M + (4 * corner_node(K)) * NL + j;
                                for (int c = 0; c < 3; ++c)
                                    row[c * NL] -= dT * w * (gvp[c] * pvdP + Q.gv[c] * Pib * Q.dPi[K][e]);
                            }
                    }
                } else {
                    if (bl >= 0)
                        for (int a = 0; a < 8; ++a) {
                            T* row = M + (4 * nd[a]) * NL + j;
                            for (int c = 0; c < 3; ++c) row[c * NL] -= w * Q.G[a][c] * phib;
                        }
                    if (stab) {
                        const T gq[3] = {gb[0] - gP[0], gb[1] - gP[1], gb[2] - gP[2]};
                        for (int a = 0; a < 8; ++a)
                            M[(4 * nd[a] + 3) * NL + j] += aT * w * (gq[0] * Q.G[a][0] + gq[1] * Q.G[a][1] + gq[2] * Q.G[a][2]);
                        if (NPG == 27)
                            for (int K = 0; K < 8; ++K)
                                M[(4 * corner_node(K) + 3) * NL + j] -=
                                    aT * w * (gq[0] * Q.dPi[K][0] + gq[1] * Q.dPi[K][1] + gq[2] * Q.dPi[K][2]);
                    }
                }
            }
        }
    }
    __syncthreads();
    T* out = Jloc + g * NL * NL;
    for (int e = threadIdx.x; e < NL * NL; e += blockDim.x) out[e] = M[e];
}

// The Jacobian of a Q2 cell (27 nodes, one element, 3 x 3 x 3 Gauss points)
// with the same closed-form column formulas as jacobian_kernel: the child
// basis is the cell's Q2 basis, and Pi_K the cell's own trilinear vertex
// functions (the range of the one-level projection pi_h: Q2 -> Q1).
template <typename T>
struct QPointQ2 {
    T w, N[27], G[27][3];    // weight x det J, Q2 basis values, physical gradients
    T Pi[8], dPi[8][3];      // trilinear vertex functions
    T v[3], Dv[3][3];
    T pv[3], Dpv[3][3];      // pi v and its gradient
    T gv[3];                 // v.grad v - pi v.grad pi v
};

template <typename T>
constexpr size_t jac_q2_smem_bytes() {
    return 27 * sizeof(QPointQ2<T>) + size_t(108) * 108 * sizeof(T);
}

__device__ __forceinline__ double g3pt_s(int i) { return i == 0 ? 0.5 - 0.38729833462074168851792653997824 : (i == 1 ? 0.5 : 0.5 + 0.38729833462074168851792653997824); }
__device__ __forceinline__ double g3wt_s(int i) { return i == 1 ? 8.0 / 18.0 : 5.0 / 18.0; }
__device__ __forceinline__ void lag2_s(double x, double (&v)[3], double (&d)[3]) {
    v[0] = 2.0 * (x - 0.5) * (x - 1.0);
    v[1] = -4.0 * x * (x - 1.0);
    v[2] = 2.0 * x * (x - 0.5);
    d[0] = 4.0 * x - 3.0;
    d[1] = 4.0 - 8.0 * x;
    d[2] = 4.0 * x - 1.0;
}

template <typename T>
__global__ void __launch_bounds__(128) jacobian_q2_kernel(int64_t ng, const int32_t* __restrict__ groups,
                                                          const double* __restrict__ xyz,
                                                          const double* __restrict__ x, LvPrm p, int stab,
                                                          T* __restrict__ Jloc) {
    constexpr int NL = 108;
    extern __shared__ __align__(16) unsigned char jq_smem[];
    QPointQ2<T>* P = reinterpret_cast<QPointQ2<T>*>(jq_smem);
    T* M = reinterpret_cast<T*>(jq_smem + 27 * sizeof(QPointQ2<T>));
    __shared__ double Xs[27][3];
    __shared__ T Us[27][4];
    __shared__ T prm_s[2];
    const int64_t g = blockIdx.x;
    for (int i = threadIdx.x; i < 27; i += blockDim.x) {
        const int64_t n = groups[g * 27 + i];
        for (int d = 0; d < 3; ++d) Xs[i][d] = xyz[3 * n + d];
        for (int c = 0; c < 4; ++c) Us[i][c] = T(x[4 * n + c]);
    }
    for (int e = threadIdx.x; e < NL * NL; e += blockDim.x) M[e] = T(0);
    __syncthreads();
    if (threadIdx.x < 27) {
        const int q = threadIdx.x;
        QPointQ2<T>& Q = P[q];
        const double xi[3] = {g3pt_s(q % 3), g3pt_s((q / 3) % 3), g3pt_s(q / 9)};
        T J[3][3], N1[8], dN1[8][3];
        for (int d = 0; d < 3; ++d)
            for (int e = 0; e < 3; ++e) J[d][e] = T(0);
        for (int k = 0; k < 8; ++k) {
            double f[3], df[3];
            for (int d = 0; d < 3; ++d) {
                f[d] = ((k >> d) & 1) ? xi[d] : 1.0 - xi[d];
                df[d] = ((k >> d) & 1) ? 1.0 : -1.0;
            }
            N1[k] = T(f[0] * f[1] * f[2]);
            dN1[k][0] = T(df[0] * f[1] * f[2]);
            dN1[k][1] = T(f[0] * df[1] * f[2]);
            dN1[k][2] = T(f[0] * f[1] * df[2]);
            const int nk = corner_node(k);
            for (int d = 0; d < 3; ++d)
                for (int e = 0; e < 3; ++e) J[d][e] += T(Xs[nk][d] - Xs[0][d]) * dN1[k][e];
        }
        const T c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const T c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        const T det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        const T idet = T(1) / det;
        T Ji[3][3];
        Ji[0][0] = c00 * idet;
        Ji[1][0] = c01 * idet;
        Ji[2][0] = c02 * idet;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * idet;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * idet;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * idet;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * idet;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * idet;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * idet;
        Q.w = T(g3wt_s(q % 3) * g3wt_s((q / 3) % 3) * g3wt_s(q / 9)) * det;
        double vx[3], dx[3], vy[3], dy[3], vz[3], dz[3];
        lag2_s(xi[0], vx, dx);
        lag2_s(xi[1], vy, dy);
        lag2_s(xi[2], vz, dz);
        for (int i = 0; i < 27; ++i) {
            const int a = i % 3, b = (i / 3) % 3, c = i / 9;
            Q.N[i] = T(vx[a] * vy[b] * vz[c]);
            const T gr[3] = {T(dx[a] * vy[b] * vz[c]), T(vx[a] * dy[b] * vz[c]), T(vx[a] * vy[b] * dz[c])};
            for (int d = 0; d < 3; ++d) Q.G[i][d] = gr[0] * Ji[0][d] + gr[1] * Ji[1][d] + gr[2] * Ji[2][d];
        }
        for (int K = 0; K < 8; ++K) {
            Q.Pi[K] = stab ? N1[K] : T(0);
            for (int d = 0; d < 3; ++d)
                Q.dPi[K][d] = stab ? dN1[K][0] * Ji[0][d] + dN1[K][1] * Ji[1][d] + dN1[K][2] * Ji[2][d] : T(0);
        }
        for (int c = 0; c < 3; ++c) {
            T v = T(0), pv = T(0), Dv[3] = {T(0), T(0), T(0)}, Dp[3] = {T(0), T(0), T(0)};
            for (int i = 0; i < 27; ++i) {
                v += Q.N[i] * Us[i][c];
                for (int d = 0; d < 3; ++d) Dv[d] += Q.G[i][d] * Us[i][c];
            }
            for (int K = 0; K < 8; ++K) {
                const T u = Us[corner_node(K)][c];
                pv += Q.Pi[K] * u;
                for (int d = 0; d < 3; ++d) Dp[d] += Q.dPi[K][d] * u;
            }
            Q.v[c] = v;
            Q.pv[c] = pv;
            for (int d = 0; d < 3; ++d) {
                Q.Dv[c][d] = Dv[d];
                Q.Dpv[c][d] = Dp[d];
            }
        }
        for (int c = 0; c < 3; ++c)
            Q.gv[c] = Q.v[0] * Q.Dv[c][0] + Q.v[1] * Q.Dv[c][1] + Q.v[2] * Q.Dv[c][2] -
                      (Q.pv[0] * Q.Dpv[c][0] + Q.pv[1] * Q.Dpv[c][1] + Q.pv[2] * Q.Dpv[c][2]);
    }
    if (threadIdx.x == 0) {
        // frozen alpha_T, delta_T (Eq. (8)): h_T the largest vertex distance,
        // |v|_inf over the cell's 27 nodes
        double h = 0.0, vmax = 0.0;
        for (int a = 0; a < 8; ++a)
            for (int b = a + 1; b < 8; ++b) {
                double s2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double t0 = Xs[corner_node(a)][d] - Xs[corner_node(b)][d];
                    s2 += t0 * t0;
                }
                h = fmax(h, sqrt(s2));
            }
        for (int i = 0; i < 27; ++i) {
            double s2 = 0.0;
            for (int d = 0; d < 3; ++d) s2 += double(Us[i][d]) * double(Us[i][d]);
            vmax = fmax(vmax, sqrt(s2));
        }
        const double den = p.nu / (h * h) + vmax / h + p.m;
        prm_s[0] = T(stab ? p.a0 / den : 0.0);
        prm_s[1] = T(stab ? p.d0 / den : 0.0);
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j < NL) {
        const int b = j >> 2, e = j & 3;
        int Kb = -1;
        if (stab)
            for (int K = 0; K < 8; ++K)
                if (corner_node(K) == b) Kb = K;
        const T m = T(p.m), th = T(p.th), nu = T(p.nu);
        const T aT = prm_s[0], dT = prm_s[1];
        for (int q = 0; q < 27; ++q) {
            const QPointQ2<T>& Q = P[q];
            const T w = Q.w;
            const T phib = Q.N[b];
            const T gb[3] = {Q.G[b][0], Q.G[b][1], Q.G[b][2]};
            T gP[3];
            for (int d = 0; d < 3; ++d) gP[d] = Kb >= 0 ? Q.dPi[Kb][d] : T(0);
            const T Pib = Kb >= 0 ? Q.Pi[Kb] : T(0);
            if (e < 3) {
                const T vgb = Q.v[0] * gb[0] + Q.v[1] * gb[1] + Q.v[2] * gb[2];
                for (int a = 0; a < 27; ++a) {
                    const T Na = Q.N[a];
                    const T ggb = Q.G[a][0] * gb[0] + Q.G[a][1] * gb[1] + Q.G[a][2] * gb[2];
                    T* row = M + (4 * a) * NL + j;
                    for (int c = 0; c < 3; ++c) {
                        T val = th * Na * phib * Q.Dv[c][e];
                        if (c == e) val += m * Na * phib + th * Na * vgb + th * nu * ggb;
                        row[c * NL] += w * val;
                    }
                    row[3 * NL] += w * Na * gb[e];
                }
                if (stab) {
                    const T pvgP = Q.pv[0] * gP[0] + Q.pv[1] * gP[1] + Q.pv[2] * gP[2];
                    T gvp[3];
                    for (int c = 0; c < 3; ++c) {
                        gvp[c] = phib * Q.Dv[c][e] - Pib * Q.Dpv[c][e];
                        if (c == e) gvp[c] += vgb - pvgP;
                    }
                    for (int a = 0; a < 27; ++a) {
                        const T vGa = Q.v[0] * Q.G[a][0] + Q.v[1] * Q.G[a][1] + Q.v[2] * Q.G[a][2];
                        T* row = M + (4 * a) * NL + j;
                        for (int c = 0; c < 3; ++c) row[c * NL] += dT * w * (gvp[c] * vGa + Q.gv[c] * phib * Q.G[a][e]);
                    }
                    for (int K = 0; K < 8; ++K) {
                        const T pvdP = Q.pv[0] * Q.dPi[K][0] + Q.pv[1] * Q.dPi[K][1] + Q.pv[2] * Q.dPi[K][2];
                        T* row = M + (4 * corner_node(K)) * NL + j;
                        for (int c = 0; c < 3; ++c)
                            row[c * NL] -= dT * w * (gvp[c] * pvdP + Q.gv[c] * Pib * Q.dPi[K][e]);
                    }
                }
            } else {
                for (int a = 0; a < 27; ++a) {
                    T* row = M + (4 * a) * NL + j;
                    for (int c = 0; c < 3; ++c) row[c * NL] -= w * Q.G[a][c] * phib;
                }
                if (stab) {
                    const T gq[3] = {gb[0] - gP[0], gb[1] - gP[1], gb[2] - gP[2]};
                    for (int a = 0; a < 27; ++a)
                        M[(4 * a + 3) * NL + j] += aT * w * (gq[0] * Q.G[a][0] + gq[1] * Q.G[a][1] + gq[2] * Q.G[a][2]);
                    for (int K = 0; K < 8; ++K)
                        M[(4 * corner_node(K) + 3) * NL + j] -=
                            aT * w * (gq[0] * Q.dPi[K][0] + gq[1] * Q.dPi[K][1] + gq[2] * Q.dPi[K][2]);
                }
            }
        }
    }
    __syncthreads();
    T* out = Jloc + g * NL * NL;
    for (int e = threadIdx.x; e < NL * NL; e += blockDim.x) out[e] = M[e];
}

// BSR block b = sum of its local entries in group order; 16 threads per block
template <typename T, int NPG>
__global__ void bsr_assemble_kernel(int64_t nnzb, const int32_t* __restrict__ bptr, const int32_t* __restrict__ bsrc,
                                    const T* __restrict__ Jloc, T* __restrict__ A) {
    constexpr int NL = 4 * NPG;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (tid >= nnzb * 16) return;
    const int64_t b = tid >> 4;
    const int r = int(tid & 15) >> 2, s = int(tid & 3);
    T acc = T(0);
    for (int32_t e = bptr[b]; e < bptr[b + 1]; ++e) {
        const int32_t src = bsrc[e];
        const int64_t g = src / (NPG * NPG);
        const int li = (src / NPG) % NPG, lj = src % NPG;
        acc += Jloc[g * NL * NL + int64_t(4 * li + r) * NL + 4 * lj + s];
    }
    A[16 * b + 4 * r + s] = acc;
}

// identity rows for Dirichlet velocity unknowns and the pinned pressure
template <typename T>
__global__ void bsr_dirichlet_kernel(int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                     const uint8_t* __restrict__ dir, int32_t pin, T* __restrict__ A) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int r = 0; r < 4; ++r) {
        const bool fix = (r < 3 && dir[i]) || (r == 3 && i == pin);
        if (!fix) continue;
        for (int32_t b = rp[i]; b < rp[i + 1]; ++b)
            for (int s = 0; s < 4; ++s) A[16 * int64_t(b) + 4 * r + s] = T((ci[b] == i && s == r) ? 1 : 0);
    }
}

template <typename TA, typename TB>
__global__ void convert_kernel(int64_t n, const TA* __restrict__ a, TB* __restrict__ b) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        b[i] = TB(a[i]);
}

// y = A x (r == null) or y = r - A x; one warp per node row: four lanes take
// one 4 x 4 block, lane 4k + rr its row rr (one 16-byte load), so a warp
// reads 8 consecutive blocks (512 bytes) per step; the row sums of the lanes
// with the same rr are reduced by a fixed shuffle tree (deterministic)
template <typename T>
__global__ void __launch_bounds__(256) bsr_spmv_kernel(int64_t n, const int32_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci, const T* __restrict__ A,
                                                       const T* __restrict__ x, const T* __restrict__ r,
                                                       T* __restrict__ y) {
    static_assert(sizeof(T) == 4, "FP32 blocks");
    const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int rr = lane & 3;
    const float4* A4 = reinterpret_cast<const float4*>(A);
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float acc = 0.f;
    for (int32_t b = rp[i] + (lane >> 2); b < rp[i + 1]; b += 8) {
        const float4 a = A4[4 * int64_t(b) + rr];
        const float4 v = x4[ci[b]];
        acc += a.x * v.x + a.y * v.y + a.z * v.z + a.w * v.w;
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (lane < 4) y[4 * i + rr] = r ? r[4 * i + rr] - acc : acc;
}

// The same product with the blocks stored in bf16 (the smoother's copy of
// the matrix): lane rr of a quad reads row rr of a block as 4 bf16 (8 bytes).
__global__ void __launch_bounds__(256) bsr_spmv_bf16_kernel(int64_t n, const int32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ ci,
                                                            const __nv_bfloat16* __restrict__ A,
                                                            const float* __restrict__ x, const float* __restrict__ r,
                                                            float* __restrict__ y) {
    const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int rr = lane & 3;
    const uint2* A2 = reinterpret_cast<const uint2*>(A);
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float acc = 0.f;
    for (int32_t b = rp[i] + (lane >> 2); b < rp[i + 1]; b += 8) {
        const uint2 raw = A2[4 * int64_t(b) + rr];
        const float2 a01 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
        const float2 a23 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
        const float4 v = x4[ci[b]];
        acc += a01.x * v.x + a01.y * v.y + a23.x * v.z + a23.y * v.w;
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 8);
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (lane < 4) y[4 * i + rr] = r ? r[4 * i + rr] - acc : acc;
}

// Group block of the global matrix inverted by Gauss-Jordan elimination
// with partial pivoting (rows swapped, the column order restored at the
// end), stored column-major in Ainv so that applying it is a coalesced dense
// product.  Thread (ty, tx) of a 16 x 16 layout keeps rows ty + 16 a and
// columns tx + 16 b of the matrix in registers for the whole elimination;
// at step k only column k (for the pivot and the multipliers) and the two
// exchanged rows go through shared memory.  A zero pivot leaves its row at
// zero (the inverse then has a zero component there, as a triangular solve
// with that convention would).
template <typename T, int NPG, typename TO>
__global__ void __launch_bounds__(256) vanka_factor_kernel(int64_t ng, const int32_t* __restrict__ grp_blk,
                                                           const T* __restrict__ A, TO* __restrict__ Ainv) {
    constexpr int NL = 4 * NPG;
    constexpr int RB = (NL + 15) / 16;   // rows (and columns) per thread
    extern __shared__ __align__(16) unsigned char vf_smem[];
    T* M = reinterpret_cast<T*>(vf_smem);   // NL x NL, row-major: the result, at the end
    __shared__ T s_col[NL];                 // column k before the row exchange
    __shared__ T s_rowk[NL];                // the new row k (old row p)
    __shared__ T s_rowp[NL];                // the new row p (old row k)
    __shared__ int s_piv[NL];
    __shared__ int s_perm[NL];
    const int64_t g = blockIdx.x;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    T R[RB][RB];
#pragma unroll
    for (int a = 0; a < RB; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int i = ty + 16 * a, j = tx + 16 * b;
            R[a][b] = T(0);
            if (i < NL && j < NL) {
                const int32_t blk = grp_blk[(g * NPG + i / 4) * NPG + j / 4];
                R[a][b] = A[16 * int64_t(blk) + 4 * (i % 4) + (j % 4)];
            }
        }
    for (int k = 0; k < NL; ++k) {
        const int kb = k >> 4;
        if (tx == (k & 15)) {
#pragma unroll
            for (int b = 0; b < RB; ++b)
                if (b == kb)
#pragma unroll
                    for (int a = 0; a < RB; ++a)
                        if (ty + 16 * a < NL) s_col[ty + 16 * a] = R[a][b];
        }
        __syncthreads();
        if (tid < 32) {
            // pivot: largest |M[i][k]|, i >= k, smallest i on ties (warp argmax)
            T bv = T(-1);
            int bi = k;
            for (int i = k + tid; i < NL; i += 32) {
                const T v = fabs(s_col[i]);
                if (v > bv) {
                    bv = v;
                    bi = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_down_sync(0xffffffffu, bv, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (tid == 0) s_piv[k] = bi;
        }
        __syncthreads();
        const int p = s_piv[k];
        // the owners of rows p and k publish them (exchanged)
        if (ty == (p & 15) || ty == (k & 15)) {
#pragma unroll
            for (int a = 0; a < RB; ++a) {
                const int i = ty + 16 * a;
                if (i != p && i != k) continue;
#pragma unroll
                for (int b = 0; b < RB; ++b) {
                    const int j = tx + 16 * b;
                    if (j >= NL) continue;
                    if (i == p) s_rowk[j] = R[a][b];
                    if (i == k) s_rowp[j] = R[a][b];
                }
            }
        }
        __syncthreads();
        const T d = s_col[p];
        const T inv = d != T(0) ? T(1) / d : T(0);
        T nr[RB];   // the normalised pivot row at this thread's columns
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int j = tx + 16 * b;
            nr[b] = j < NL ? (j == k ? T(1) : s_rowk[j]) * inv : T(0);
        }
#pragma unroll
        for (int a = 0; a < RB; ++a) {
            const int i = ty + 16 * a;
            if (i >= NL) continue;
            if (i == k) {
#pragma unroll
                for (int b = 0; b < RB; ++b) R[a][b] = nr[b];
                continue;
            }
            const T f = i == p ? s_col[k] : s_col[i];
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                const int j = tx + 16 * b;
                if (j >= NL) continue;
                const T src = i == p ? s_rowp[j] : R[a][b];
                R[a][b] = (j == k ? T(0) : src) - f * nr[b];
            }
        }
        __syncthreads();   // s_col and the rows are rewritten at the next step
    }
#pragma unroll
    for (int a = 0; a < RB; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const int i = ty + 16 * a, j = tx + 16 * b;
            if (i < NL && j < NL) M[i * NL + j] = R[a][b];
        }
    // the row swaps of the elimination become column swaps of the inverse,
    // undone in reverse order: column c of the inverse is column s_perm[c]
    if (tid == 0) {
        for (int c = 0; c < NL; ++c) s_perm[c] = c;
        for (int k = NL - 1; k >= 0; --k) {
            const int t = s_perm[k];
            s_perm[k] = s_perm[s_piv[k]];
            s_perm[s_piv[k]] = t;
        }
    }
    __syncthreads();
    // column-major: Ainv[g][j * NL + i] = (A^{-1})_{ij} (rounded once to TO)
    for (int e = tid; e < NL * NL; e += blockDim.x) {
        const int j = e / NL, i = e % NL;
        Ainv[g * NL * NL + e] = TO(M[i * NL + s_perm[j]]);
    }
}

// z_g = A_g^{-1} r restricted to group g: one block per group, thread i
// computes row i of the dense product (column-major inverse: coalesced).
template <typename T, int NPG>
__global__ void __launch_bounds__(128) vanka_apply_kernel(int64_t ng, const int32_t* __restrict__ groups,
                                                          const T* __restrict__ Ainv, const T* __restrict__ r,
                                                          T* __restrict__ zloc) {
    constexpr int NL = 4 * NPG;
    __shared__ T s_r[NL];
    const int64_t g = blockIdx.x;
    for (int e = threadIdx.x; e < NL; e += blockDim.x) s_r[e] = r[4 * int64_t(groups[g * NPG + e / 4]) + e % 4];
    __syncthreads();
    const T* Ag = Ainv + g * NL * NL;
    for (int i = threadIdx.x; i < NL; i += blockDim.x) {
        T acc = T(0);
        for (int j = 0; j < NL; ++j) acc += Ag[j * NL + i] * s_r[j];
        zloc[g * NL + i] = acc;
    }
}

// The same with bf16 inverses: thread t computes rows 2t and 2t + 1 from
// one bf16 pair per column (column-major, so a warp's pairs are contiguous).
template <int NPG>
__global__ void __launch_bounds__(64) vanka_apply_bf16_kernel(int64_t ng, const int32_t* __restrict__ groups,
                                                              const __nv_bfloat16* __restrict__ Ainv,
                                                              const float* __restrict__ r,
                                                              float* __restrict__ zloc) {
    constexpr int NL = 4 * NPG, NH = NL / 2;
    __shared__ float s_r[NL];
    const int64_t g = blockIdx.x;
    for (int e = threadIdx.x; e < NL; e += blockDim.x) s_r[e] = r[4 * int64_t(groups[g * NPG + e / 4]) + e % 4];
    __syncthreads();
    const int t = threadIdx.x;
    if (t >= NH) return;
    const __nv_bfloat162* Ag = reinterpret_cast<const __nv_bfloat162*>(Ainv + g * NL * NL) + t;
    float a0 = 0.f, a1 = 0.f;
#pragma unroll 6
    for (int j = 0; j < NL; ++j) {
        const float2 w = __bfloat1622float2(Ag[j * NH]);
        a0 = fmaf(w.x, s_r[j], a0);
        a1 = fmaf(w.y, s_r[j], a1);
    }
    zloc[g * NL + 2 * t] = a0;
    zloc[g * NL + 2 * t + 1] = a1;
}

// e_j = (first ? 0 : e_j) + omega / valence_j * (sum of the groups' local
// solutions at node j), in group order
template <typename T>
__global__ void vanka_update_kernel(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                    const T* __restrict__ zloc, T omega, int first, T* __restrict__ e) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    T a[4] = {T(0), T(0), T(0), T(0)};
    const int32_t e0 = ptr[j], e1 = ptr[j + 1];
    for (int32_t k = e0; k < e1; ++k)
        for (int c = 0; c < 4; ++c) a[c] += zloc[4 * int64_t(idx[k]) + c];
    const T mu = omega / T(e1 - e0);
    for (int c = 0; c < 4; ++c) e[4 * j + c] = (first ? T(0) : e[4 * j + c]) + a[c] * mu;
}

// One colour of a multiplicative group-Vanka sweep, in two launches so that
// every group of the colour sees the same e (no two groups of a colour share
// a node, but their rows reach each other's nodes): first the residual of
// each group's 4 NPG rows at the current e into dloc[g], then the local
// solve with the group inverse and e += omega z on the group's unknowns.
// Colours run one after another, so later colours see the earlier ones'
// updates (multiplicative between colours, fixed order: deterministic).
template <int NPG>
__global__ void __launch_bounds__(128) vanka_colour_residual_kernel(const int32_t* __restrict__ cgroups,
                                                                    const int32_t* __restrict__ groups,
                                                                    const int32_t* __restrict__ rp,
                                                                    const int32_t* __restrict__ ci,
                                                                    const float* __restrict__ A,
                                                                    const float* __restrict__ r,
                                                                    const float* __restrict__ e,
                                                                    float* __restrict__ dloc) {
    constexpr int NL = 4 * NPG;
    const int64_t g = cgroups[blockIdx.x];
    const float4* A4 = reinterpret_cast<const float4*>(A);
    const float4* e4 = reinterpret_cast<const float4*>(e);
    for (int i = threadIdx.x; i < NL; i += blockDim.x) {
        const int64_t node = groups[g * NPG + i / 4];
        const int rr = i & 3;
        float acc = 0.f;
        for (int32_t b = rp[node]; b < rp[node + 1]; ++b) {
            const float4 a = A4[4 * int64_t(b) + rr];
            const float4 v = e4[ci[b]];
            acc += a.x * v.x + a.y * v.y + a.z * v.z + a.w * v.w;
        }
        dloc[g * NL + i] = r[4 * node + rr] - acc;
    }
}

template <int NPG>
__global__ void __launch_bounds__(128) vanka_colour_update_kernel(const int32_t* __restrict__ cgroups,
                                                                  const int32_t* __restrict__ groups,
                                                                  const float* __restrict__ Ainv,
                                                                  const float* __restrict__ dloc, float omega,
                                                                  float* __restrict__ e) {
    constexpr int NL = 4 * NPG;
    __shared__ float s_d[NL];
    const int64_t g = cgroups[blockIdx.x];
    for (int i = threadIdx.x; i < NL; i += blockDim.x) s_d[i] = dloc[g * NL + i];
    __syncthreads();
    const float* Ag = Ainv + g * NL * NL;
    for (int i = threadIdx.x; i < NL; i += blockDim.x) {
        float z = 0.f;
        for (int j = 0; j < NL; ++j) z += Ag[j * NL + i] * s_d[j];
        e[4 * int64_t(groups[g * NPG + i / 4]) + (i & 3)] += omega * z;
    }
}

// coarse residual r_c = R d (rows of R = P^T in fine node order), with
// Dirichlet velocity rows and the pinned pressure row of the coarse level 0
template <typename T>
__global__ void mg_restrict_kernel(int64_t nc, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                   const float* __restrict__ w, const T* __restrict__ d,
                                   const uint8_t* __restrict__ dir, int32_t pin, T* __restrict__ rc) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    T a[4] = {T(0), T(0), T(0), T(0)};
    for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
        const T wk = T(w[k]);
        const T* dv = d + 4 * int64_t(idx[k]);
        for (int c = 0; c < 4; ++c) a[c] += wk * dv[c];
    }
    for (int c = 0; c < 4; ++c) rc[4 * i + c] = ((c < 3 && dir[i]) || (c == 3 && i == pin)) ? T(0) : a[c];
}

// e += P e_c, with the fine level's Dirichlet velocity rows and pinned
// pressure row left alone
template <typename T>
__global__ void mg_prolong_add_kernel(int64_t nf, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                      const float* __restrict__ w, const T* __restrict__ ec,
                                      const uint8_t* __restrict__ dir, int32_t pin, T* __restrict__ e) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    T a[4] = {T(0), T(0), T(0), T(0)};
    for (int32_t k = ptr[j]; k < ptr[j + 1]; ++k) {
        const T wk = T(w[k]);
        const T* ev = ec + 4 * int64_t(idx[k]);
        for (int c = 0; c < 4; ++c) a[c] += wk * ev[c];
    }
    for (int c = 0; c < 4; ++c)
        if (!((c < 3 && dir[j]) || (c == 3 && j == pin))) e[4 * j + c] += a[c];
}

// ---- coarsest level: dense LU with partial pivoting and explicit inverse (FP64)

// Dense row-major copy of a BSR matrix restricted to the free unknowns:
// cidx[4 node + c] = the compact index of unknown (node, c), -1 for a
// Dirichlet velocity or the pinned pressure (their rows are identity rows
// with zero right-hand side, so they and their columns drop out).  D (nf x
// nf) zeroed beforehand.
__global__ void dense_from_bsr_kernel(int64_t n, int nf, const int32_t* __restrict__ rp,
                                      const int32_t* __restrict__ ci, const int32_t* __restrict__ cidx,
                                      const double* __restrict__ A, double* __restrict__ D) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int r = 0; r < 4; ++r) {
        const int row = cidx[4 * i + r];
        if (row < 0) continue;
        for (int32_t b = rp[i]; b < rp[i + 1]; ++b)
            for (int c = 0; c < 4; ++c) {
                const int col = cidx[4 * int64_t(ci[b]) + c];
                if (col >= 0) D[int64_t(row) * nf + col] = A[16 * int64_t(b) + 4 * r + c];
            }
    }
}

// Elimination step k: reads the factorisation so far from Ain and writes it
// to Aout with rows k and p (the pivot: largest |A[i][k]|, i >= k, smallest
// i on ties, found by every block alike) exchanged, the multipliers of
// column k below the diagonal and the updated trailing rows; row k - 1 (final
// since the previous step) is copied, so that both buffers hold every final
// row.  A zero pivot leaves zero multipliers.
__global__ void __launch_bounds__(256) lu_step_kernel(int N, int k, const double* __restrict__ Ain,
                                                      double* __restrict__ Aout, int32_t* __restrict__ piv) {
    __shared__ double sv[8];
    __shared__ int si[8];
    double bv = -1.0;
    int bi = k;
    for (int i = k + int(threadIdx.x); i < N; i += blockDim.x) {
        const double a = fabs(Ain[int64_t(i) * N + k]);
        if (a > bv) {
            bv = a;
            bi = i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
        }
    }
    if ((threadIdx.x & 31) == 0) {
        sv[threadIdx.x >> 5] = bv;
        si[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < int(blockDim.x >> 5); ++w)
            if (sv[w] > sv[0] || (sv[w] == sv[0] && si[w] < si[0])) {
                sv[0] = sv[w];
                si[0] = si[w];
            }
        if (blockIdx.x == 0) piv[k] = si[0];
    }
    __syncthreads();
    const int p = si[0];
    const double pv = Ain[int64_t(p) * N + k];
    const int r0 = k > 0 ? k - 1 : 0;
    const int64_t total = int64_t(N - r0) * N;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int i = r0 + int(t / N), j = int(t % N);
        double out;
        if (i < k) {
            out = Ain[int64_t(i) * N + j];
        } else {
            const int src = i == k ? p : (i == p ? k : i);
            const double a = Ain[int64_t(src) * N + j];
            if (i == k || j < k) {
                out = a;
            } else {
                const double l = pv != 0.0 ? Ain[int64_t(src) * N + k] / pv : 0.0;
                out = j == k ? l : a - l * Ain[int64_t(p) * N + j];
            }
        }
        Aout[int64_t(i) * N + j] = out;
    }
}

// Column c of A^{-1} from P A = L U, one warp per column held in shared
// memory: the row exchanges, then the unit-lower forward and the upper back
// substitution; each row's sum is split over the lanes and reduced by a
// fixed shuffle tree.  A zero diagonal gives a zero component.  The result
// is stored row-major, X[i][c].
__global__ void __launch_bounds__(128) lu_inverse_kernel(int N, const double* __restrict__ LU,
                                                         const int32_t* __restrict__ piv, double* __restrict__ X) {
    extern __shared__ double inv_col[];                 // [warps][N]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = int(blockIdx.x) * int(blockDim.x >> 5) + w;
    if (c >= N) return;
    double* x = inv_col + size_t(w) * N;
    for (int i = lane; i < N; i += 32) x[i] = i == c ? 1.0 : 0.0;
    __syncwarp();
    if (lane == 0)
        for (int k = 0; k < N; ++k) {
            const int p = piv[k];
            if (p != k) {
                const double t = x[k];
                x[k] = x[p];
                x[p] = t;
            }
        }
    __syncwarp();
    for (int i = 1; i < N; ++i) {
        double acc = 0.0;
        const double* Li = LU + int64_t(i) * N;
        for (int j = lane; j < i; j += 32) acc += Li[j] * x[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) x[i] -= acc;
        __syncwarp();
    }
    for (int i = N - 1; i >= 0; --i) {
        double acc = 0.0;
        const double* Ui = LU + int64_t(i) * N;
        for (int j = i + 1 + lane; j < N; j += 32) acc += Ui[j] * x[j];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const double d = Ui[i];
            x[i] = d != 0.0 ? (x[i] - acc) / d : 0.0;
        }
        __syncwarp();
    }
    for (int i = lane; i < N; i += 32) X[int64_t(i) * N + c] = x[i];
}

// e = Ainv r on the free unknowns in FP64 (one warp per row, fixed shuffle
// tree); fixed unknowns of e are 0.  fidx[k] = the unknown 4 node + c of
// compact index k.
template <typename T>
__global__ void dense_matvec_kernel(int nf, const int32_t* __restrict__ fidx, const double* __restrict__ Ainv,
                                    const T* __restrict__ r, T* __restrict__ e) {
    const int row = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= nf) return;
    double acc = 0.0;
    for (int j = lane; j < nf; j += 32) acc += Ainv[int64_t(row) * nf + j] * double(r[fidx[j]]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) e[fidx[row]] = T(acc);
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

// ---- flexible GMRES state on the device ----------------------------------------
// st[0] = beta0 (initial residual norm), st[1] = residual estimate |g[j+1]|,
// st[2] = the iteration count at which the estimate first met the tolerance
// (-1 before)
__global__ void set_beta0_kernel(const double* __restrict__ nrm2, double* __restrict__ st) {
    st[0] = sqrt(fmax(nrm2[0], 0.0));
    st[1] = st[0];
    st[2] = -1.0;
}
__global__ void cycle_init_kernel(int m, const double* __restrict__ nrm2, double* __restrict__ g,
                                  double* __restrict__ st) {
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        g[0] = sqrt(fmax(nrm2[0], 0.0));
        st[2] = -1.0;
    }
}
// Givens rotations on column j of H (column-major, leading dimension m + 1;
// H[j+1][j] holds |w|^2): the earlier rotations, then one that zeroes
// H[j+1][j]; g follows, and |g[j+1]| is the residual norm of the iterate.
__global__ void givens_kernel(int j, int m, double* __restrict__ H, double* __restrict__ cs,
                              double* __restrict__ sn, double* __restrict__ g, double rtol,
                              double* __restrict__ st) {
    double* col = H + size_t(j) * (m + 1);
    col[j + 1] = sqrt(fmax(col[j + 1], 0.0));
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    cs[j] = den > 0.0 ? col[j] / den : 1.0;
    sn[j] = den > 0.0 ? col[j + 1] / den : 0.0;
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const double r = fabs(g[j + 1]);
    st[1] = r;
    if (st[2] < 0.0 && r <= rtol * st[0]) st[2] = double(j + 1);
}
// y = R^{-1} g for the first jn columns (back substitution, one thread)
__global__ void ls_solve_kernel(int jn, int m, const double* __restrict__ H, const double* __restrict__ g,
                                double* __restrict__ y) {
    for (int i = jn - 1; i >= 0; --i) {
        double t = g[i];
        for (int k = i + 1; k < jn; ++k) t -= H[i + size_t(k) * (m + 1)] * y[k];
        const double d = H[i + size_t(i) * (m + 1)];
        y[i] = d != 0.0 ? t / d : 0.0;
    }
}
// x += sum_i y[i] Z_i, i = 0 .. cnt - 1 in order
__global__ void multi_axpy_add_kernel(int64_t n, int cnt, const double* __restrict__ y, const double* __restrict__ Z,
                                      double* __restrict__ x) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
        double acc = x[k];
        for (int i = 0; i < cnt; ++i) acc += y[i] * Z[int64_t(i) * n + k];
        x[k] = acc;
    }
}

}  // namespace

// ---- device levels ------------------------------------------------------------

// One mesh level on the device: its structure, FP32 matrix and smoother,
// multigrid vectors, the transfer to the next coarser level, and (coarsest
// level) the FP64 matrix with its dense LU and inverse.
struct LevelData {
    HostLevel h;
    int32_t *groups = nullptr, *node_ptr = nullptr, *node_idx = nullptr, *row_ptr = nullptr, *col_idx = nullptr;
    int32_t *blk_ptr = nullptr, *blk_src = nullptr, *grp_blk = nullptr;
    double* xyz = nullptr;
    uint8_t* dir = nullptr;
    float* A = nullptr;       // BSR values [nnzb][4][4]
    float* G = nullptr;       // [ng][nl][nl]: local Jacobians, then the group inverses (column-major;
                              // in bf16, packed at the start of the same storage, when g_bf16)
    __nv_bfloat16* Ab = nullptr;   // BSR values in bf16 for the smoother's products (when g_bf16)
    bool g_bf16 = false;
    float* zloc = nullptr;    // [ng][nl]
    float *r = nullptr, *e = nullptr, *d = nullptr;   // [n][4]
    float *r2 = nullptr, *e2 = nullptr, *d2 = nullptr;  // [n][4] operands of the Krylov products (solve level)
    int32_t *P_ptr = nullptr, *P_idx = nullptr, *R_ptr = nullptr, *R_idx = nullptr;
    float *P_w = nullptr, *R_w = nullptr;
    double *J64 = nullptr, *A64 = nullptr, *D0 = nullptr, *D1 = nullptr, *Dinv = nullptr;
    int32_t* piv = nullptr;
    int32_t *cidx = nullptr, *fidx = nullptr;   // unknown -> compact free index (-1 fixed), and back
    int32_t* cgroups = nullptr;                 // groups by colour (multiplicative smoothing)
    int nfree = 0;
    bool coarsest = false;
    int stab = 0;             // stabilisation terms in the Jacobian (see jacobian_kernel)
    std::vector<void*> allocs;
};

struct DeviceLevel {
    LevelData top;                   // the level solved on
    std::vector<LevelData*> mg;      // coarser levels, mg[0] the next coarser
    int mg_pre = 2, mg_post = 2;
    int mg_smoother = 0;        // 0 additive, 1 multiplicative (coloured) group-Vanka
    int mg_bf16 = 0;            // additive smoother on bf16 copies of the matrix and the inverses
    float omega = 0.7f;
    double* local = nullptr;    // [ng][npg][4] FP64 local residuals
    double* mass = nullptr;     // [n] lumped mass
    double* work = nullptr;     // r, dx, tmp, rr, w: [5][n][4]
    double* V = nullptr;        // (krylov + 1) x [n][4]
    double* Z = nullptr;        // krylov x [n][4]
    double* scal = nullptr;     // device scalars and the small GMRES arrays
    double* part = nullptr;     // reduction partials
    int krylov = 0;
    bool has_jacobian = false, mass_ready = false;
    std::vector<void*> allocs;
};

namespace {

template <typename T>
cudaError_t up(std::vector<void*>& allocs, const std::vector<T>& v, T** out) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(v.size() * sizeof(T), 1));
    if (e != cudaSuccess) return e;
    allocs.push_back(p);
    if (!v.empty()) {
        e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    *out = static_cast<T*>(p);
    return cudaSuccess;
}
template <typename T>
cudaError_t dalloc(std::vector<void*>& allocs, size_t count, T** out) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 1));
    if (e != cudaSuccess) return e;
    allocs.push_back(p);
    *out = static_cast<T*>(p);
    return cudaSuccess;
}

#define CKE(x)                                  \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

cudaError_t upload_level(LevelData* L) {
    const HostLevel& h = L->h;
    auto& a = L->allocs;
    CKE(up(a, h.groups, &L->groups));
    CKE(up(a, h.xyz, &L->xyz));
    CKE(up(a, h.dir, &L->dir));
    CKE(up(a, h.node_ptr, &L->node_ptr));
    CKE(up(a, h.node_idx, &L->node_idx));
    CKE(up(a, h.row_ptr, &L->row_ptr));
    CKE(up(a, h.col_idx, &L->col_idx));
    CKE(up(a, h.blk_ptr, &L->blk_ptr));
    CKE(up(a, h.blk_src, &L->blk_src));
    CKE(up(a, h.grp_blk, &L->grp_blk));
    CKE(up(a, h.color_groups, &L->cgroups));
    return cudaSuccess;
}

// FP32 matrix, group inverses and multigrid vectors of a smoothing level
cudaError_t alloc_smoother(LevelData* L) {
    const HostLevel& h = L->h;
    const size_t nl = size_t(4 * h.npg);
    CKE(dalloc(L->allocs, h.col_idx.size() * 16, &L->A));
    CKE(dalloc(L->allocs, size_t(h.ng) * nl * nl, &L->G));
    CKE(dalloc(L->allocs, size_t(h.ng) * nl, &L->zloc));
    CKE(dalloc(L->allocs, size_t(4 * h.n), &L->r));
    CKE(dalloc(L->allocs, size_t(4 * h.n), &L->e));
    CKE(dalloc(L->allocs, size_t(4 * h.n), &L->d));
    return cudaSuccess;
}

cudaError_t alloc_fp64_matrix(LevelData* L) {
    if (L->A64) return cudaSuccess;
    const HostLevel& h = L->h;
    const size_t nl = size_t(4 * h.npg);
    CKE(dalloc(L->allocs, size_t(h.ng) * nl * nl, &L->J64));
    CKE(dalloc(L->allocs, h.col_idx.size() * 16, &L->A64));
    return cudaSuccess;
}

cudaError_t upload_transfer(LevelData* L, const MgTransfer& t) {
    std::vector<float> pw(t.P_w.begin(), t.P_w.end()), rw(t.R_w.begin(), t.R_w.end());   // dyadic: exact
    CKE(up(L->allocs, t.P_ptr, &L->P_ptr));
    CKE(up(L->allocs, t.P_idx, &L->P_idx));
    CKE(up(L->allocs, pw, &L->P_w));
    CKE(up(L->allocs, t.R_ptr, &L->R_ptr));
    CKE(up(L->allocs, t.R_idx, &L->R_idx));
    CKE(up(L->allocs, rw, &L->R_w));
    return cudaSuccess;
}

void free_level_data(LevelData* L) {
    for (void* p : L->allocs) cudaFree(p);
    L->allocs.clear();
}

}  // namespace

void destroy_level(DeviceLevel* D) {
    if (!D) return;
    free_level_data(&D->top);
    for (LevelData* L : D->mg) {
        free_level_data(L);
        delete L;
    }
    for (void* p : D->allocs) cudaFree(p);
    delete D;
}

cudaError_t create_level(const HostHierarchy& hh, bool fine, int krylov, int mg_levels, DeviceLevel** out) {
    DeviceLevel* D = new DeviceLevel();
    auto fail = [&](cudaError_t e) {
        destroy_level(D);
        return e;
    };
    build_level(hh, fine, &D->top.h);
    LevelData* cur = &D->top;
    for (int k = 0; k < mg_levels; ++k) {
        LevelData* c = new LevelData();
        MgTransfer t;
        if (!coarsen_level(cur->h, &c->h, &t)) {
            delete c;
            break;
        }
        cudaError_t e = upload_transfer(cur, t);
        D->mg.push_back(c);
        if (e != cudaSuccess) return fail(e);
        cur = c;
    }
    if (!D->mg.empty()) {
        LevelData* c = D->mg.back();
        c->coarsest = true;
        if (4 * c->h.n > kMaxCoarsestUnknowns) return fail(cudaErrorInvalidValue);
    }
    // stabilisation in the Jacobian: the local projection on grouped levels;
    // full fluctuations on an ungrouped coarsest multigrid level
    D->top.stab = D->top.h.npg == 27 && D->top.h.lps ? 1 : 0;
    for (LevelData* L : D->mg) L->stab = L->h.npg == 27 ? (L->h.lps ? 1 : 0) : (L->coarsest ? 1 : 0);
    cudaError_t e;
    if ((e = upload_level(&D->top)) != cudaSuccess) return fail(e);
    if ((e = alloc_smoother(&D->top)) != cudaSuccess) return fail(e);
    for (float** v : {&D->top.r2, &D->top.e2, &D->top.d2})
        if ((e = dalloc(D->top.allocs, size_t(4 * D->top.h.n), v)) != cudaSuccess) return fail(e);
    for (LevelData* L : D->mg) {
        if ((e = upload_level(L)) != cudaSuccess) return fail(e);
        if (L->coarsest) {
            // the dense system on the free unknowns only
            std::vector<int32_t> cidx(size_t(4 * L->h.n), -1), fidx;
            for (int64_t j = 0; j < L->h.n; ++j)
                for (int c = 0; c < 4; ++c)
                    if (!((c < 3 && L->h.dir[size_t(j)]) || (c == 3 && j == L->h.pin))) {
                        cidx[size_t(4 * j + c)] = int32_t(fidx.size());
                        fidx.push_back(int32_t(4 * j + c));
                    }
            L->nfree = int(fidx.size());
            if ((e = up(L->allocs, cidx, &L->cidx)) != cudaSuccess) return fail(e);
            if ((e = up(L->allocs, fidx, &L->fidx)) != cudaSuccess) return fail(e);
            const size_t N = size_t(std::max(L->nfree, 1));
            if ((e = alloc_fp64_matrix(L)) != cudaSuccess) return fail(e);
            if ((e = dalloc(L->allocs, N * N, &L->D0)) != cudaSuccess) return fail(e);
            if ((e = dalloc(L->allocs, N * N, &L->D1)) != cudaSuccess) return fail(e);
            if ((e = dalloc(L->allocs, N * N, &L->Dinv)) != cudaSuccess) return fail(e);
            if ((e = dalloc(L->allocs, N, &L->piv)) != cudaSuccess) return fail(e);
            if ((e = dalloc(L->allocs, size_t(4 * L->h.n), &L->r)) != cudaSuccess) return fail(e);
            if ((e = dalloc(L->allocs, size_t(4 * L->h.n), &L->e)) != cudaSuccess) return fail(e);
        } else if ((e = alloc_smoother(L)) != cudaSuccess) {
            return fail(e);
        }
    }
    const HostLevel& h = D->top.h;
    const size_t n4 = size_t(4 * h.n);
    const size_t nl = size_t(4 * h.npg);
    if ((e = dalloc(D->allocs, size_t(h.ng) * nl, &D->local)) != cudaSuccess) return fail(e);
    if ((e = dalloc(D->allocs, size_t(h.n), &D->mass)) != cudaSuccess) return fail(e);
    if ((e = dalloc(D->allocs, 5 * n4, &D->work)) != cudaSuccess) return fail(e);
    if ((e = dalloc(D->allocs, size_t(krylov + 1) * n4, &D->V)) != cudaSuccess) return fail(e);
    if ((e = dalloc(D->allocs, size_t(krylov) * n4, &D->Z)) != cudaSuccess) return fail(e);
    if ((e = dalloc(D->allocs, size_t(krylov + 2) * size_t(krylov + 6) + 64, &D->scal)) != cudaSuccess) return fail(e);
    if ((e = dalloc(D->allocs, size_t(kRedBlocks) * size_t(krylov + 1), &D->part)) != cudaSuccess) return fail(e);
    D->krylov = krylov;
    *out = D;
    return cudaSuccess;
}

int64_t level_nodes(const DeviceLevel* D) { return D->top.h.n; }
bool level_lps(const DeviceLevel* D) { return D->top.h.lps; }
int level_mg_depth(const DeviceLevel* D) { return int(D->mg.size()); }
int64_t level_mg_nodes(const DeviceLevel* D, int k) { return k == 0 ? D->top.h.n : D->mg[size_t(k - 1)]->h.n; }

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
cudaError_t local_terms(DeviceLevel* D, const double* x, LvPrm p, cudaStream_t s) {
    const LevelData& L = D->top;
    const HostLevel& h = L.h;
    p.lps = h.lps ? p.lps : 0;
    if (h.q2) {
        Q2Level q;
        q.n = h.n;
        q.ncell = h.ng;
        q.cells = L.groups;
        q.node_ptr = L.node_ptr;
        q.node_idx = L.node_idx;
        q.xyz = L.xyz;
        q.dir = L.dir;
        const int mode = MODE == LV_OPERATOR ? 0 : (MODE == LV_RHS ? 1 : 2);
        OpParams op{p.m, p.th, p.nu};
        CKE(q2_level_local<double>(q, mode, x, nullptr, op, p.a0, p.d0, p.lps, D->local, s));
    } else if (h.npg == 27) {
        static bool attr = false;
        if (!attr) {
            CKE(cudaFuncSetAttribute(level_local_child_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(kChildSmem)));
            attr = true;
        }
        level_local_child_kernel<MODE><<<nblk(h.ng, kChildGroups), 64, kChildSmem, s>>>(h.ng, L.groups, L.xyz, x, p,
                                                                                       D->local);
    } else
        level_local_kernel<8, MODE><<<nblk(h.ng, 64), 64, 0, s>>>(h.ng, L.groups, L.xyz, x, p, D->local);
    CKE(cudaGetLastError());
    node_gather_kernel<<<nblk(h.n, 256), 256, 0, s>>>(h.n, L.node_ptr, L.node_idx, D->local,
                                                        D->work + 2 * 4 * h.n);   // tmp
    return cudaGetLastError();
}

cudaError_t dot(DeviceLevel* D, const double* a, const double* b, int64_t n, double* out_dev, cudaStream_t s) {
    dot_partial_kernel<<<kRedBlocks, 256, 0, s>>>(n, a, b, D->part);
    dot_final_kernel<<<1, 256, 0, s>>>(D->part, kRedBlocks, out_dev);
    return cudaGetLastError();
}

// One classical Gram-Schmidt pass against V_0..V_{cnt-1}: h = V^T w, w -= V h.
cudaError_t cgs_pass(DeviceLevel* D, double* w, const double* V, int cnt, int64_t n, double* h, cudaStream_t s) {
    multi_dot_partial_kernel<<<dim3(kRedBlocks, unsigned(cnt)), 256, 0, s>>>(n, w, V, D->part);
    multi_dot_final_kernel<<<unsigned(cnt), 256, 0, s>>>(D->part, kRedBlocks, h);
    multi_axpy_kernel<<<256, 256, 0, s>>>(n, cnt, h, V, w);
    return cudaGetLastError();
}

cudaError_t fetch(double* host, const double* dev, size_t n, cudaStream_t s) {
    CKE(cudaMemcpyAsync(host, dev, n * 8, cudaMemcpyDeviceToHost, s));
    return cudaStreamSynchronize(s);
}

// Lumped mass (integral of each basis function) into D->mass and its sum
// into the device scalar D->scal[2] (once per level).
cudaError_t compute_mass(DeviceLevel* D, const OpParams& op, cudaStream_t s) {
    if (D->mass_ready) return cudaSuccess;
    CKE(local_terms<LV_MASS>(D, nullptr, make_prm(op, nullptr), s));
    const int64_t n = D->top.h.n;
    extract_component_kernel<<<nblk(n, 256), 256, 0, s>>>(n, D->work + 2 * 4 * n, 0, D->mass);
    CKE(cudaGetLastError());
    std::vector<double> mh(static_cast<size_t>(n));
    CKE(fetch(mh.data(), D->mass, static_cast<size_t>(n), s));
    double sum = 0.0;
    for (double v : mh) sum += v;
    CKE(cudaMemcpyAsync(D->scal + 2, &sum, 8, cudaMemcpyHostToDevice, s));
    CKE(cudaStreamSynchronize(s));
    D->mass_ready = true;
    return cudaSuccess;
}

template <typename T, int NPG>
cudaError_t launch_jacobian(const LevelData& L, const double* x, const LvPrm& p, T* Jloc, cudaStream_t s) {
    constexpr size_t smem = jac_smem_bytes<T, NPG>();
    static bool attr = false;
    if (!attr) {
        CKE(cudaFuncSetAttribute(jacobian_kernel<T, NPG>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        attr = true;
    }
    jacobian_kernel<T, NPG><<<unsigned(L.h.ng), 128, smem, s>>>(L.h.ng, L.groups, L.xyz, x, p, L.stab, Jloc);
    return cudaGetLastError();
}

// Jacobian at x (the first n nodes of x are this level's nodes) into the
// level's BSR matrix of element type T, Dirichlet and pinned rows identity
template <typename T>
cudaError_t assemble(const LevelData& L, const double* x, const LvPrm& p, T* Jloc, T* A, cudaStream_t s) {
    const HostLevel& h = L.h;
    if (h.q2) {
        constexpr size_t smem = jac_q2_smem_bytes<T>();
        static bool attr = false;
        if (!attr) {
            CKE(cudaFuncSetAttribute(jacobian_q2_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
            attr = true;
        }
        jacobian_q2_kernel<T><<<unsigned(h.ng), 128, smem, s>>>(h.ng, L.groups, L.xyz, x, p, L.stab, Jloc);
        CKE(cudaGetLastError());
    } else if (h.npg == 27) {
        CKE((launch_jacobian<T, 27>(L, x, p, Jloc, s)));
    } else {
        CKE((launch_jacobian<T, 8>(L, x, p, Jloc, s)));
    }
    const int64_t nnzb = int64_t(h.col_idx.size());
    if (h.npg == 27)
        bsr_assemble_kernel<T, 27><<<nblk(nnzb * 16, 256), 256, 0, s>>>(nnzb, L.blk_ptr, L.blk_src, Jloc, A);
    else
        bsr_assemble_kernel<T, 8><<<nblk(nnzb * 16, 256), 256, 0, s>>>(nnzb, L.blk_ptr, L.blk_src, Jloc, A);
    CKE(cudaGetLastError());
    bsr_dirichlet_kernel<T><<<nblk(h.n, 128), 128, 0, s>>>(h.n, L.row_ptr, L.col_idx, L.dir, h.pin, A);
    return cudaGetLastError();
}

template <int NPG>
cudaError_t launch_vanka_factor(const LevelData& L, cudaStream_t s) {
    constexpr int NL = 4 * NPG;
    constexpr size_t smem = size_t(NL) * NL * sizeof(float);
    static bool attr = false;
    if (!attr) {
        CKE(cudaFuncSetAttribute(vanka_factor_kernel<float, NPG, float>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        CKE(cudaFuncSetAttribute(vanka_factor_kernel<float, NPG, __nv_bfloat16>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        attr = true;
    }
    // the kernel reads the assembled matrix, not G, so the bf16 inverses may
    // overwrite G's local Jacobians in place
    if (L.g_bf16)
        vanka_factor_kernel<float, NPG, __nv_bfloat16><<<unsigned(L.h.ng), 256, smem, s>>>(
            L.h.ng, L.grp_blk, L.A, reinterpret_cast<__nv_bfloat16*>(L.G));
    else
        vanka_factor_kernel<float, NPG, float><<<unsigned(L.h.ng), 256, smem, s>>>(L.h.ng, L.grp_blk, L.A, L.G);
    return cudaGetLastError();
}

// FP32 matrix and group inverses of a smoothing level; with bf16 also the
// bf16 copy of the matrix for the smoother's products
cudaError_t setup_smoother(LevelData& L, const double* x, const LvPrm& p, bool bf16, cudaStream_t s) {
    CKE(assemble<float>(L, x, p, L.G, L.A, s));
    L.g_bf16 = bf16;
    if (bf16) {
        const int64_t nv = int64_t(L.h.col_idx.size()) * 16;
        if (!L.Ab) CKE(dalloc(L.allocs, size_t(nv), &L.Ab));
        convert_kernel<float, __nv_bfloat16><<<nblk(nv, 256), 256, 0, s>>>(nv, L.A, L.Ab);
        CKE(cudaGetLastError());
    }
    return L.h.npg == 27 ? launch_vanka_factor<27>(L, s) : launch_vanka_factor<8>(L, s);
}

// FP64 matrix, its dense LU and inverse on the coarsest level
cudaError_t setup_coarsest(LevelData& L, const double* x, const LvPrm& p, cudaStream_t s) {
    CKE(assemble<double>(L, x, p, L.J64, L.A64, s));
    const int N = L.nfree;
    if (N == 0) return cudaSuccess;
    CKE(cudaMemsetAsync(L.D0, 0, size_t(N) * N * 8, s));
    dense_from_bsr_kernel<<<nblk(L.h.n, 128), 128, 0, s>>>(L.h.n, N, L.row_ptr, L.col_idx, L.cidx, L.A64, L.D0);
    CKE(cudaGetLastError());
    double* buf[2] = {L.D0, L.D1};
    const int grid = std::max(1, std::min(1024, int((int64_t(N) * N + 1023) / 1024)));
    for (int k = 0; k < N; ++k) {
        lu_step_kernel<<<grid, 256, 0, s>>>(N, k, buf[k & 1], buf[(k + 1) & 1], L.piv);
        CKE(cudaGetLastError());
    }
    // one warp per column of the inverse, its column in shared memory
    const int warps = std::max(1, std::min(4, int((160 * 1024) / (size_t(N) * 8))));
    const size_t smem = size_t(warps) * N * 8;
    static bool attr = false;
    if (!attr) {
        CKE(cudaFuncSetAttribute(lu_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    lu_inverse_kernel<<<nblk(N, warps), 32 * warps, smem, s>>>(N, buf[N & 1], L.piv, L.Dinv);
    return cudaGetLastError();
}

}  // namespace

// r = b - A(x) with Dirichlet / pin rows zero
cudaError_t level_residual(DeviceLevel* D, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                           const double* b, double* r, cudaStream_t s) {
    CKE(local_terms<LV_OPERATOR>(D, x, make_prm(op, sp), s));
    const int64_t n = D->top.h.n;
    CKE(cudaMemcpyAsync(r, D->work + 2 * 4 * n, size_t(4 * n) * 8, cudaMemcpyDeviceToDevice, s));
    finish_rows_kernel<<<nblk(n, 256), 256, 0, s>>>(n, b, r, D->top.dir, D->top.h.pin, 1, 0);
    return cudaGetLastError();
}

// A(x) as assembled (no row modification)
cudaError_t level_operator(DeviceLevel* D, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                           double* Ax, cudaStream_t s) {
    CKE(local_terms<LV_OPERATOR>(D, x, make_prm(op, sp), s));
    return cudaMemcpyAsync(Ax, D->work + 2 * 4 * D->top.h.n, size_t(4 * D->top.h.n) * 8, cudaMemcpyDeviceToDevice, s);
}

// b(x_old): rhs of Eq. (6), Dirichlet velocity rows and pressure rows zero
cudaError_t level_rhs(DeviceLevel* D, const OpParams& op, const double* x_old, double* b, cudaStream_t s) {
    CKE(local_terms<LV_RHS>(D, x_old, make_prm(op, nullptr), s));
    const int64_t n = D->top.h.n;
    CKE(cudaMemcpyAsync(b, D->work + 2 * 4 * n, size_t(4 * n) * 8, cudaMemcpyDeviceToDevice, s));
    finish_rows_kernel<<<nblk(n, 256), 256, 0, s>>>(n, nullptr, b, D->top.dir, -1, 0, 1);
    return cudaGetLastError();
}

// Jacobians at x on every level (coarser levels at the injected iterate:
// their nodes are the first nodes of the finer level), the smoothers, and
// the coarsest level's dense inverse
cudaError_t level_jacobian(DeviceLevel* D, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                           cudaStream_t s) {
    const LvPrm p = make_prm(op, sp);
    const bool bf16 = D->mg_bf16 != 0 && D->mg_smoother == 0;
    CKE(setup_smoother(D->top, x, p, bf16, s));
    for (LevelData* L : D->mg) CKE(L->coarsest ? setup_coarsest(*L, x, p, s) : setup_smoother(*L, x, p, bf16, s));
    D->has_jacobian = true;
    return cudaSuccess;
}

// dense copy of the FP64 Jacobian of the solve level at x (small levels; tests)
cudaError_t level_dense_jacobian(DeviceLevel* D, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                                 double* dense_host, cudaStream_t s) {
    LevelData& L = D->top;
    CKE(alloc_fp64_matrix(&L));
    CKE(assemble<double>(L, x, make_prm(op, sp), L.J64, L.A64, s));
    const HostLevel& h = L.h;
    const size_t nnzb = h.col_idx.size();
    std::vector<double> A(nnzb * 16);
    CKE(cudaMemcpyAsync(A.data(), L.A64, A.size() * 8, cudaMemcpyDeviceToHost, s));
    CKE(cudaStreamSynchronize(s));
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

// `sweeps` multiplicative group-Vanka sweeps on L, colours in increasing
// order (reverse = decreasing, for the sweeps after the coarse correction)
cudaError_t smooth_mult(LevelData& L, int sweeps, bool e_zero, float omega, bool reverse, cudaStream_t s) {
    const HostLevel& h = L.h;
    if (e_zero) CKE(cudaMemsetAsync(L.e, 0, size_t(4 * h.n) * 4, s));
    const int nc = int(h.color_ptr.size()) - 1;
    for (int it = 0; it < sweeps; ++it)
        for (int k = 0; k < nc; ++k) {
            const int c = reverse ? nc - 1 - k : k;
            const int32_t c0 = h.color_ptr[size_t(c)], cnt = h.color_ptr[size_t(c) + 1] - c0;
            if (cnt == 0) continue;
            if (h.npg == 27) {
                vanka_colour_residual_kernel<27><<<unsigned(cnt), 128, 0, s>>>(L.cgroups + c0, L.groups, L.row_ptr,
                                                                               L.col_idx, L.A, L.r, L.e, L.zloc);
                vanka_colour_update_kernel<27><<<unsigned(cnt), 128, 0, s>>>(L.cgroups + c0, L.groups, L.G, L.zloc,
                                                                             omega, L.e);
            } else {
                vanka_colour_residual_kernel<8><<<unsigned(cnt), 32, 0, s>>>(L.cgroups + c0, L.groups, L.row_ptr,
                                                                             L.col_idx, L.A, L.r, L.e, L.zloc);
                vanka_colour_update_kernel<8><<<unsigned(cnt), 32, 0, s>>>(L.cgroups + c0, L.groups, L.G, L.zloc,
                                                                           omega, L.e);
            }
        }
    return cudaGetLastError();
}

// d = r - A e on a smoothing level (the bf16 copy of A when the smoother
// runs in bf16)
cudaError_t smoother_residual(LevelData& L, cudaStream_t s) {
    const int64_t n = L.h.n;
    if (L.g_bf16)
        bsr_spmv_bf16_kernel<<<nblk(32 * n, 256), 256, 0, s>>>(n, L.row_ptr, L.col_idx, L.Ab, L.e, L.r, L.d);
    else
        bsr_spmv_kernel<float><<<nblk(32 * n, 256), 256, 0, s>>>(n, L.row_ptr, L.col_idx, L.A, L.e, L.r, L.d);
    return cudaGetLastError();
}

// `sweeps` damped additive group-Vanka sweeps on L: e += omega V(r - A e)
// (e = omega V(r) first when e_zero)
cudaError_t smooth(LevelData& L, int sweeps, bool e_zero, float omega, cudaStream_t s) {
    const HostLevel& h = L.h;
    for (int it = 0; it < sweeps; ++it) {
        const bool first = it == 0 && e_zero;
        const float* d = L.r;
        if (!first) {
            CKE(smoother_residual(L, s));
            d = L.d;
        }
        const __nv_bfloat16* Gb = reinterpret_cast<const __nv_bfloat16*>(L.G);
        if (h.npg == 27) {
            if (L.g_bf16)
                vanka_apply_bf16_kernel<27><<<unsigned(h.ng), 64, 0, s>>>(h.ng, L.groups, Gb, d, L.zloc);
            else
                vanka_apply_kernel<float, 27><<<unsigned(h.ng), 128, 0, s>>>(h.ng, L.groups, L.G, d, L.zloc);
        } else {
            if (L.g_bf16)
                vanka_apply_bf16_kernel<8><<<unsigned(h.ng), 32, 0, s>>>(h.ng, L.groups, Gb, d, L.zloc);
            else
                vanka_apply_kernel<float, 8><<<unsigned(h.ng), 32, 0, s>>>(h.ng, L.groups, L.G, d, L.zloc);
        }
        vanka_update_kernel<float><<<nblk(h.n, 256), 256, 0, s>>>(h.n, L.node_ptr, L.node_idx, L.zloc, omega,
                                                                   first ? 1 : 0, L.e);
    }
    return cudaGetLastError();
}

// e ~ A^{-1} r on level k (0 = the solve level) by one V-cycle
cudaError_t vcycle(DeviceLevel* D, int k, cudaStream_t s) {
    LevelData& L = k == 0 ? D->top : *D->mg[size_t(k - 1)];
    const HostLevel& h = L.h;
    if (L.coarsest) {
        CKE(cudaMemsetAsync(L.e, 0, size_t(4 * h.n) * 4, s));
        if (L.nfree == 0) return cudaSuccess;
        dense_matvec_kernel<float><<<nblk(int64_t(L.nfree) * 32, 256), 256, 0, s>>>(L.nfree, L.fidx, L.Dinv, L.r, L.e);
        return cudaGetLastError();
    }
    if (size_t(k) == D->mg.size()) return smooth(L, 1, true, 1.0f, s);   // one-level: one Vanka application
    const bool mult = D->mg_smoother == 1;
    bool e_zero = true;
    if (D->mg_pre > 0) {
        CKE(mult ? smooth_mult(L, D->mg_pre, true, D->omega, false, s) : smooth(L, D->mg_pre, true, D->omega, s));
        e_zero = false;
    }
    if (e_zero) CKE(cudaMemsetAsync(L.e, 0, size_t(4 * h.n) * 4, s));
    CKE(smoother_residual(L, s));
    LevelData& C = *D->mg[size_t(k)];
    mg_restrict_kernel<float><<<nblk(C.h.n, 256), 256, 0, s>>>(C.h.n, L.R_ptr, L.R_idx, L.R_w, L.d, C.dir, C.h.pin,
                                                                C.r);
    CKE(cudaGetLastError());
    CKE(vcycle(D, k + 1, s));
    mg_prolong_add_kernel<float><<<nblk(h.n, 256), 256, 0, s>>>(h.n, L.P_ptr, L.P_idx, L.P_w, C.e, L.dir, h.pin, L.e);
    CKE(cudaGetLastError());
    return mult ? smooth_mult(L, D->mg_post, false, D->omega, true, s) : smooth(L, D->mg_post, false, D->omega, s);
}

// z = M^{-1} v (FP64 in and out, FP32 inside)
cudaError_t precond(DeviceLevel* D, const double* v, double* z, cudaStream_t s) {
    const int64_t n4 = 4 * D->top.h.n;
    convert_kernel<double, float><<<nblk(n4, 256), 256, 0, s>>>(n4, v, D->top.r);
    CKE(vcycle(D, 0, s));
    convert_kernel<float, double><<<nblk(n4, 256), 256, 0, s>>>(n4, D->top.e, z);
    return cudaGetLastError();
}

// y = J x (r == null) or y = r - J x with the FP32 Jacobian: x (and r)
// rounded to FP32, the product in FP32, the result widened to FP64.  The
// matrix is itself the Jacobian rounded to FP32, so this adds an error of
// the same order; Newton's FP64 residual decides convergence.
cudaError_t spmv64(DeviceLevel* D, const double* x, const double* r, double* y, cudaStream_t s) {
    LevelData& L = D->top;
    const int64_t n4 = 4 * L.h.n;
    convert_kernel<double, float><<<nblk(n4, 256), 256, 0, s>>>(n4, x, L.e2);
    if (r) convert_kernel<double, float><<<nblk(n4, 256), 256, 0, s>>>(n4, r, L.r2);
    bsr_spmv_kernel<float><<<nblk(32 * L.h.n, 256), 256, 0, s>>>(L.h.n, L.row_ptr, L.col_idx, L.A, L.e2,
                                                                  r ? L.r2 : nullptr, L.d2);
    convert_kernel<float, double><<<nblk(n4, 256), 256, 0, s>>>(n4, L.d2, y);
    return cudaGetLastError();
}

// Flexible right-preconditioned restarted GMRES for J dx = r (dx zero on
// entry).  The host reads the residual estimate every `check` iterations.
cudaError_t fgmres(DeviceLevel* D, const double* r, double* dx, double rtol, int max_it, cudaStream_t s,
                   int* iters, double* res_out) {
    const int64_t n4 = 4 * D->top.h.n;
    const int m = D->krylov;
    double* w = D->work + 4 * n4;
    double* rr = D->work + 3 * n4;
    double* V = D->V;
    double* Z = D->Z;
    double* st = D->scal + 8;               // beta0, residual estimate, stop
    double* nrm = D->scal + 12;
    double* h2 = D->scal + 16;              // second CGS pass: m + 1
    double* cs = h2 + (m + 1);
    double* sn = cs + m;
    double* g = sn + m;                     // m + 1
    double* y = g + (m + 1);                // m
    double* H = y + m;                      // (m + 1) x m, column-major
    const int check = D->mg.empty() ? 8 : 2;
    CKE(cudaMemsetAsync(dx, 0, size_t(n4) * 8, s));
    CKE(dot(D, r, r, n4, nrm, s));
    set_beta0_kernel<<<1, 1, 0, s>>>(nrm, st);
    double hs[3];
    CKE(fetch(hs, st, 3, s));
    *iters = 0;
    *res_out = hs[0];
    if (hs[0] == 0.0) return cudaSuccess;
    CKE(cudaMemcpyAsync(rr, r, size_t(n4) * 8, cudaMemcpyDeviceToDevice, s));
    for (;;) {
        CKE(dot(D, rr, rr, n4, nrm, s));
        scale_inv_sqrt_kernel<<<256, 256, 0, s>>>(n4, nrm, rr, V);
        cycle_init_kernel<<<1, 256, 0, s>>>(m, nrm, g, st);
        CKE(cudaGetLastError());
        int j = 0, jn = -1;
        while (j < m && *iters < max_it) {
            double* vj = V + int64_t(j) * n4;
            double* zj = Z + int64_t(j) * n4;
            double* vn = V + int64_t(j + 1) * n4;
            CKE(precond(D, vj, zj, s));
            CKE(spmv64(D, zj, nullptr, w, s));
            // orthogonalise against V_0..V_j: classical Gram-Schmidt twice;
            // the column gets the sum of both passes
            double* hcol = H + size_t(j) * (m + 1);
            CKE(cgs_pass(D, w, V, j + 1, n4, hcol, s));
            CKE(cgs_pass(D, w, V, j + 1, n4, h2, s));
            add_vec_kernel<<<1, 64, 0, s>>>(j + 1, h2, hcol);
            double* hn = hcol + (j + 1);
            CKE(dot(D, w, w, n4, hn, s));
            scale_inv_sqrt_kernel<<<256, 256, 0, s>>>(n4, hn, w, vn);
            givens_kernel<<<1, 1, 0, s>>>(j, m, H, cs, sn, g, rtol, st);
            CKE(cudaGetLastError());
            ++j;
            ++(*iters);
            if (j % check == 0 || j == m || *iters >= max_it) {
                CKE(fetch(hs, st, 3, s));
                if (hs[2] >= 0.0) {
                    jn = int(hs[2]);
                    break;
                }
            }
        }
        const bool converged = jn >= 0;
        if (jn < 0) jn = j;
        ls_solve_kernel<<<1, 1, 0, s>>>(jn, m, H, g, y);
        multi_axpy_add_kernel<<<256, 256, 0, s>>>(n4, jn, y, Z, dx);
        CKE(cudaGetLastError());
        *res_out = hs[1];
        if (converged || *iters >= max_it) break;
        CKE(spmv64(D, dx, r, rr, s));   // true residual for the restart: rr = r - J dx
    }
    return cudaSuccess;
}

}  // namespace

// Newton solve of A(x) = b on the level; x holds the Dirichlet values (and
// the initial guess) on entry.
cudaError_t level_solve(DeviceLevel* D, const OpParams& op, const dnnmg_solver_params* sp, const double* b, double* x,
                        cudaStream_t s, dnnmg_solve_stats* st) {
    const int64_t n = D->top.h.n, n4 = 4 * n;
    double* r = D->work;
    double* dx = D->work + n4;
    dnnmg_solve_stats stats{};
    D->mg_pre = sp->mg_pre;
    D->mg_post = sp->mg_post;
    D->mg_smoother = sp->mg_smoother;
    D->mg_bf16 = sp->mg_bf16;
    D->omega = float(sp->mg_omega);
    if (D->top.h.mean_zero_pressure) CKE(compute_mass(D, op, s));
    double r0 = -1.0, rprev = -1.0;
    bool reassemble = true;
    for (int it = 0;; ++it) {
        CKE(level_residual(D, op, sp, x, b, r, s));
        CKE(dot(D, r, r, n4, D->scal, s));
        double t;
        CKE(fetch(&t, D->scal, 1, s));
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
        if (reassemble || !D->has_jacobian) {
            CKE(level_jacobian(D, op, sp, x, s));
            stats.jacobian_assemblies++;
            reassemble = false;
        }
        rprev = rn;
        int gi = 0;
        double gres = 0.0;
        CKE(fgmres(D, r, dx, sp->gmres_rtol, sp->gmres_max, s, &gi, &gres));
        stats.gmres_iterations += gi;
        axpy_kernel<<<256, 256, 0, s>>>(n4, 1.0, dx, x);
        CKE(cudaGetLastError());
        if (D->top.h.mean_zero_pressure) {
            // p -= (mass . p) / (mass . 1)
            double* pv = D->work + 2 * n4;   // tmp (n entries used)
            extract_component_kernel<<<nblk(n, 256), 256, 0, s>>>(n, x, 3, pv);
            CKE(dot(D, D->mass, pv, n, D->scal + 1, s));
            mean_ratio_kernel<<<1, 1, 0, s>>>(D->scal + 1, D->scal + 2, D->scal + 3);
            pressure_shift_kernel<<<nblk(n, 256), 256, 0, s>>>(n, D->scal + 3, x);
            CKE(cudaGetLastError());
        }
    }
    D->has_jacobian = false;   // next solve starts with a fresh Jacobian
    if (st) *st = stats;
    return cudaSuccess;
}

}  // namespace dnnmg
