// Q2/Q2 elements with the one-level local projection (Sec. 3.2, Eqs. (5)-(6),
// (8)), the paper's own discretisation, on the GPU.
//
// A Q2 level is a set of hexahedral cells with 27 nodes each (local node
// a + 3 b + 9 c at the reference point (a, b, c) / 2), equal-order
// triquadratic velocity and pressure, and the trilinear geometry of the
// cell's 8 vertices.  The Q2 nodes of a mesh are the nodes of that mesh
// refined once, so with DNN-MG on Q2 the coarse level's nodes are the
// hierarchy's level L+1 and the fine level's its level L+2; a patch is a
// coarse cell with its 125 fine nodes, the layout of a two-level patch
// (Sec. 5.2), so the network input, the extension and the network are the
// J = 2 ones.
//
// The projection pi_h maps Q2 onto Q1 on each cell: the trilinear
// interpolant of the cell's 8 vertex values (kappa_h = id - pi_h).  With
// frozen alpha_T, delta_T (h_T the cell's diameter, |v|_inf,T the largest
// nodal |v| of its 27 nodes):
//   velocity rows  delta_T (v.grad v - pi v.grad pi v, v.grad phi - pi v.grad pi phi)
//   pressure rows  alpha_T (grad(p - pi p), grad(xi - pi xi))
// and the Galerkin terms of the theta-scheme as for Q1.  3 x 3 x 3 Gauss
// points.
//
// Kernels: one warp per cell, lane a < 27 owns node a (its basis function,
// its values and its residual rows); the quantities at a Gauss point
// (velocity, pressure, their gradients, the projected ones) are warp sums
// over the lanes in a fixed shuffle tree, so results are deterministic.
#include "internal.h"

namespace dnnmg {
namespace {

constexpr double kG3 = 0.38729833462074168851792653997824;   // sqrt(3/5) / 2
__device__ __forceinline__ double g3pt(int i) { return i == 0 ? 0.5 - kG3 : (i == 1 ? 0.5 : 0.5 + kG3); }
__device__ __forceinline__ double g3wt(int i) { return i == 1 ? 8.0 / 18.0 : 5.0 / 18.0; }

// 1D quadratic Lagrange basis on the nodes 0, 1/2, 1 and its derivative
template <typename T>
__device__ __forceinline__ void lag2(T x, T (&v)[3], T (&d)[3]) {
    v[0] = T(2) * (x - T(0.5)) * (x - T(1));
    v[1] = T(-4) * x * (x - T(1));
    v[2] = T(2) * x * (x - T(0.5));
    d[0] = T(4) * x - T(3);
    d[1] = T(4) - T(8) * x;
    d[2] = T(4) * x - T(1);
}

__device__ __forceinline__ int q2_corner(int K) { return 2 * (K & 1) + 6 * ((K >> 1) & 1) + 18 * ((K >> 2) & 1); }

// trilinear weight of vertex K at local node a (reference point a / 2)
template <typename T>
__device__ __forceinline__ T q2_wpi(int a, int K) {
    const int c[3] = {a % 3, (a / 3) % 3, a / 9};
    T w = T(1);
    for (int d = 0; d < 3; ++d) {
        const T x = T(0.5) * T(c[d]);
        w *= ((K >> d) & 1) ? x : T(1) - x;
    }
    return w;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;   // every lane holds the sum (butterfly: the same value everywhere)
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

enum { Q2_OPERATOR = 0, Q2_RHS = 1, Q2_MASS = 2 };

// Local residual of one Q2 cell, lane a < 27 owning node a:
//   Q2_OPERATOR: A_h's terms with the projection (lps != 0) at the values U;
//   Q2_RHS:      the rhs of Eq. (6) at the velocity U (pressure rows 0);
//   Q2_MASS:     the integral of the basis function in R[0].
// X8: the cell's 8 vertex coordinates relative to vertex 0 (all lanes).
// U: this lane's 4 values (lanes >= 27 pass zeros).  R: this lane's rows.
template <typename T, int MODE>
__device__ void q2_cell(const T (&X8)[8][3], const T (&U)[4], T m, T th, T nu, T a0, T d0, int lps, T (&R)[4]) {
    const int lane = threadIdx.x & 31;
    const bool own = lane < 27;
    const int ia = lane % 3, ja = (lane / 3) % 3, ka = (lane / 9) % 3;
    for (int c = 0; c < 4; ++c) R[c] = T(0);
    const bool stab = MODE == Q2_OPERATOR && lps;
    // projected values pi U at this lane's node: trilinear in the vertex values
    T PU[4] = {T(0), T(0), T(0), T(0)};
    T aT = T(0), dT = T(0);
    if (stab) {
        for (int K = 0; K < 8; ++K) {
            const T wk = own ? q2_wpi<T>(lane, K) : T(0);
            for (int c = 0; c < 4; ++c) PU[c] += wk * __shfl_sync(0xffffffffu, U[c], q2_corner(K));
        }
        T h = T(0);
        for (int a = 0; a < 8; ++a)
            for (int b = a + 1; b < 8; ++b) {
                T s = T(0);
                for (int d = 0; d < 3; ++d) s += (X8[a][d] - X8[b][d]) * (X8[a][d] - X8[b][d]);
                h = fmax(h, sqrt(s));
            }
        const T vn = own ? sqrt(U[0] * U[0] + U[1] * U[1] + U[2] * U[2]) : T(0);
        const T vmax = warp_max(vn);
        const T den = nu / (h * h) + vmax / h + m;
        aT = a0 / den;
        dT = d0 / den;
    }
    T sp = T(0), s1[3] = {T(0), T(0), T(0)}, s2[3] = {T(0), T(0), T(0)};
    const T cth = MODE == Q2_OPERATOR ? th : th - T(1);   // rhs: -(1 - theta)
    for (int q = 0; q < 27; ++q) {
        const int qi = q % 3, qj = (q / 3) % 3, qk = q / 9;
        const T xi[3] = {T(g3pt(qi)), T(g3pt(qj)), T(g3pt(qk))};
        const T wq = T(g3wt(qi) * g3wt(qj) * g3wt(qk));
        // trilinear geometry: J[d][e] = sum_k X8[k][d] dN_k / dxi_e
        T J[3][3];
        for (int d = 0; d < 3; ++d)
            for (int e = 0; e < 3; ++e) J[d][e] = T(0);
        T N1[8], dN1[8][3];
        for (int k = 0; k < 8; ++k) {
            T f[3], df[3];
            for (int d = 0; d < 3; ++d) {
                f[d] = ((k >> d) & 1) ? xi[d] : T(1) - xi[d];
                df[d] = ((k >> d) & 1) ? T(1) : T(-1);
            }
            N1[k] = f[0] * f[1] * f[2];
            dN1[k][0] = df[0] * f[1] * f[2];
            dN1[k][1] = f[0] * df[1] * f[2];
            dN1[k][2] = f[0] * f[1] * df[2];
            for (int d = 0; d < 3; ++d)
                for (int e = 0; e < 3; ++e) J[d][e] += X8[k][d] * dN1[k][e];
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
        const T w = wq * det;
        // this lane's Q2 basis function and its physical gradient
        T vx[3], dx[3], vy[3], dy[3], vz[3], dz[3];
        lag2(xi[0], vx, dx);
        lag2(xi[1], vy, dy);
        lag2(xi[2], vz, dz);
        const T phi = own ? vx[ia] * vy[ja] * vz[ka] : T(0);
        const T gr[3] = {own ? dx[ia] * vy[ja] * vz[ka] : T(0), own ? vx[ia] * dy[ja] * vz[ka] : T(0),
                         own ? vx[ia] * vy[ja] * dz[ka] : T(0)};
        T g[3];
        for (int d = 0; d < 3; ++d) g[d] = gr[0] * Ji[0][d] + gr[1] * Ji[1][d] + gr[2] * Ji[2][d];
        if (MODE == Q2_MASS) {
            R[0] += w * phi;
            continue;
        }
        T v[3], Dv[3][3];
        for (int c = 0; c < 3; ++c) {
            v[c] = warp_sum(phi * U[c]);
            for (int d = 0; d < 3; ++d) Dv[c][d] = warp_sum(g[d] * U[c]);
        }
        T conv[3];
        for (int c = 0; c < 3; ++c) conv[c] = v[0] * Dv[c][0] + v[1] * Dv[c][1] + v[2] * Dv[c][2];
        T p = T(0);
        if (MODE == Q2_OPERATOR) p = warp_sum(phi * U[3]);
        for (int c = 0; c < 3; ++c) {
            T s = m * phi * v[c] + cth * phi * conv[c] + cth * nu * (g[0] * Dv[c][0] + g[1] * Dv[c][1] + g[2] * Dv[c][2]);
            if (MODE == Q2_OPERATOR) s -= g[c] * p;
            R[c] += w * s;
        }
        if (MODE == Q2_OPERATOR) R[3] += w * phi * (Dv[0][0] + Dv[1][1] + Dv[2][2]);
        if (stab) {
            T pv[3], Dp[3][3], gkp[3];
            for (int c = 0; c < 3; ++c) {
                pv[c] = warp_sum(phi * PU[c]);
                for (int d = 0; d < 3; ++d) Dp[c][d] = warp_sum(g[d] * PU[c]);
            }
            for (int d = 0; d < 3; ++d) gkp[d] = warp_sum(g[d] * (U[3] - PU[3]));
            T gv[3];
            for (int c = 0; c < 3; ++c)
                gv[c] = conv[c] - (pv[0] * Dp[c][0] + pv[1] * Dp[c][1] + pv[2] * Dp[c][2]);
            sp += aT * w * (gkp[0] * g[0] + gkp[1] * g[1] + gkp[2] * g[2]);
            const T vg = v[0] * g[0] + v[1] * g[1] + v[2] * g[2];
            const T pvg = pv[0] * g[0] + pv[1] * g[1] + pv[2] * g[2];
            for (int c = 0; c < 3; ++c) {
                s1[c] += dT * w * gv[c] * vg;
                s2[c] += dT * w * gv[c] * pvg;
            }
        }
    }
    if (stab) {
        R[3] += sp;
        for (int c = 0; c < 3; ++c) R[c] += s1[c];
        // the test side's pi phi_a is vertex K's trilinear function with the
        // weight of K at node a: gathered onto the 8 vertex rows
        for (int K = 0; K < 8; ++K) {
            const T wk = own ? q2_wpi<T>(lane, K) : T(0);
            const T t3 = warp_sum(wk * sp);
            T tc[3];
            for (int c = 0; c < 3; ++c) tc[c] = warp_sum(wk * s2[c]);
            if (lane == q2_corner(K)) {
                R[3] -= t3;
                for (int c = 0; c < 3; ++c) R[c] -= tc[c];
            }
        }
    }
}

// Local rows of every cell of a Q2 level: cells [ncell][27] node ids,
// xyz [n][3] (double: vertex differences are formed before rounding), x [n][4] (MODE OPERATOR: the state; RHS: the old velocity,
// plus d [n][3] when given; MASS: unused), out [ncell][27][4].  8 cells per
// block of 256 threads.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) q2_level_kernel(int64_t ncell, const int32_t* __restrict__ cells,
                                                       const double* __restrict__ xyz, const T* __restrict__ x,
                                                       const T* __restrict__ d, T m, T th, T nu, T a0, T d0,
                                                       int lps, T* __restrict__ out) {
    const int64_t cell = int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (cell >= ncell) return;   // whole warps leave together
    const int32_t* nd = cells + cell * 27;
    T X8[8][3];
    const int64_t n0 = nd[0];
    for (int K = 0; K < 8; ++K) {
        const int64_t nk = nd[q2_corner(K)];
        for (int e = 0; e < 3; ++e) X8[K][e] = T(xyz[3 * nk + e] - xyz[3 * n0 + e]);
    }
    T U[4] = {T(0), T(0), T(0), T(0)};
    int64_t node = -1;
    if (lane < 27) {
        node = nd[lane];
        if (MODE != Q2_MASS)
            for (int c = 0; c < (MODE == Q2_OPERATOR ? 4 : 3); ++c) U[c] = x[4 * node + c];
        if (MODE == Q2_RHS && d)
            for (int c = 0; c < 3; ++c) U[c] += d[3 * node + c];
    }
    T R[4];
    q2_cell<T, MODE>(X8, U, m, th, nu, a0, d0, lps, R);
    if (lane < 27)
        for (int c = 0; c < 4; ++c) out[(cell * 27 + lane) * 4 + c] = R[c];
}

// out_j = (F_j -) sum of the cells' rows at node j in cell order; velocity
// rows zero at Dirichlet nodes; (rhs) pressure rows zero
template <typename T, int MODE>
__global__ void q2_gather_kernel(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                 const T* __restrict__ local, const uint8_t* __restrict__ dir,
                                 const T* __restrict__ F, T* __restrict__ out) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    T a[4] = {T(0), T(0), T(0), T(0)};
    for (int32_t e = ptr[j]; e < ptr[j + 1]; ++e)
        for (int c = 0; c < 4; ++c) a[c] += local[4 * int64_t(idx[e]) + c];
    for (int c = 0; c < 4; ++c) {
        T v = MODE == Q2_OPERATOR ? F[4 * j + c] - a[c] : a[c];
        if ((c < 3 && dir[j]) || (MODE == Q2_RHS && c == 3)) v = T(0);
        out[4 * j + c] = v;
    }
}

// value of coarse Q2 basis function m at patch node iota (reference point
// (a, b, c) / 4 of the coarse cell, iota = a + 5 b + 25 c)
template <typename T>
__device__ __forceinline__ T q2_patch_weight(int m, int iota) {
    T v[3][3], d[3];
    const int ab[3] = {iota % 5, (iota / 5) % 5, iota / 25};
    for (int e = 0; e < 3; ++e) lag2(T(0.25) * T(ab[e]), v[e], d);
    return v[0][m % 3] * v[1][(m / 3) % 3] * v[2][m / 9];
}

// x~ = P x^L: fine node j takes the coarse triquadratic of the first patch
// containing it (the field is continuous: every patch gives the same value)
template <typename T>
__global__ void q2_prolongate_kernel(int64_t nf, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                     const int32_t* __restrict__ pm_mid, const T* __restrict__ xc,
                                     T* __restrict__ xf) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    const int32_t e = idx[ptr[j]];
    const int64_t P = e / 125;
    const int iota = e % 125;
    T a[4] = {T(0), T(0), T(0), T(0)};
    for (int mm = 0; mm < 27; ++mm) {
        const T w = q2_patch_weight<T>(mm, iota);
        if (w == T(0)) continue;
        const int64_t nm = pm_mid[P * 27 + mm];
        for (int c = 0; c < 4; ++c) a[c] += w * xc[4 * nm + c];
    }
    for (int c = 0; c < 4; ++c) xf[4 * j + c] = a[c];
}

// Restriction R = P^T, patch part: coarse node m of patch P collects
// sum_iota w(m, iota) b[dof(P, iota)] / valence(dof(P, iota)) (velocity);
// summed over the patches containing a coarse node this is (P^T b)
template <typename T>
__global__ void q2_restrict_patch_kernel(int64_t nc, const int32_t* __restrict__ pm, const int32_t* __restrict__ ptr,
                                         const T* __restrict__ b, T* __restrict__ part) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;   // P * 27 + m
    if (e >= 27 * nc) return;
    const int64_t P = e / 27;
    const int mm = int(e % 27);
    T a[3] = {T(0), T(0), T(0)};
    for (int iota = 0; iota < 125; ++iota) {
        const T w = q2_patch_weight<T>(mm, iota);
        if (w == T(0)) continue;
        const int64_t j = pm[P * 125 + iota];
        const T s = w / T(ptr[j + 1] - ptr[j]);
        for (int c = 0; c < 3; ++c) a[c] += s * b[4 * j + c];
    }
    for (int c = 0; c < 3; ++c) part[4 * e + c] = a[c];
    part[4 * e + 3] = T(0);
}

// b^L_i = sum over (P, m) at coarse node i of the patch parts (patch order);
// Dirichlet velocity rows and pressure rows zero
template <typename T>
__global__ void q2_restrict_gather_kernel(int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                          const T* __restrict__ part, const uint8_t* __restrict__ dir,
                                          T* __restrict__ out) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T a[3] = {T(0), T(0), T(0)};
    for (int32_t e = ptr[i]; e < ptr[i + 1]; ++e)
        for (int c = 0; c < 3; ++c) a[c] += part[4 * int64_t(idx[e]) + c];
    for (int c = 0; c < 3; ++c) out[4 * i + c] = dir[i] ? T(0) : a[c];
    out[4 * i + 3] = T(0);
}

template <typename T, typename TX>
__device__ __forceinline__ TX to_x(T v) {
    return TX(v);
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_x<float, __nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// Network input rows of Q2 patches: X[P] = [x~ at the 125 patch nodes
// (u, v, w, p) | r likewise | geometry features | 0]; one thread per column
template <typename T, typename TX>
__global__ void q2_local_restrict_kernel(int64_t nc, int n_geo, int ld, const int32_t* __restrict__ pm,
                                         const T* __restrict__ xf, const T* __restrict__ r,
                                         const T* __restrict__ geo, TX* __restrict__ X) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nc * ld) return;
    const int64_t P = e / ld;
    const int col = int(e % ld);
    T v = T(0);
    if (col < 500) {
        v = xf[4 * int64_t(pm[P * 125 + col / 4]) + (col & 3)];
    } else if (col < 1000) {
        const int k = col - 500;
        v = r[4 * int64_t(pm[P * 125 + k / 4]) + (k & 3)];
    } else if (col < 1000 + n_geo) {
        v = geo[P * n_geo + (col - 1000)];
    }
    X[e] = to_x<T, TX>(v);
}

inline unsigned nb(int64_t n, int per) { return unsigned((n + per - 1) / per); }

}  // namespace

// ---- launchers ---------------------------------------------------------------

template <typename T>
cudaError_t q2_level_local(const Q2Level& L, int mode, const T* x, const T* d, OpParams op, double a0, double d0,
                           int lps, T* local, cudaStream_t s) {
    const double* xyz = L.xyz;
    const unsigned grid = nb(L.ncell, 8);
    if (L.ncell == 0) return cudaSuccess;
    if (mode == 0)
        q2_level_kernel<T, Q2_OPERATOR><<<grid, 256, 0, s>>>(L.ncell, L.cells, xyz, x, d, T(op.m), T(op.theta),
                                                             T(op.nu), T(a0), T(d0), lps, local);
    else if (mode == 1)
        q2_level_kernel<T, Q2_RHS><<<grid, 256, 0, s>>>(L.ncell, L.cells, xyz, x, d, T(op.m), T(op.theta), T(op.nu),
                                                        T(a0), T(d0), lps, local);
    else
        q2_level_kernel<T, Q2_MASS><<<grid, 256, 0, s>>>(L.ncell, L.cells, xyz, x, d, T(op.m), T(op.theta),
                                                         T(op.nu), T(a0), T(d0), lps, local);
    return cudaGetLastError();
}

template <typename T>
cudaError_t q2_gather(const Q2Level& L, int mode, const T* local, const T* F, T* out, cudaStream_t s) {
    if (mode == 0)
        q2_gather_kernel<T, Q2_OPERATOR><<<nb(L.n, 256), 256, 0, s>>>(L.n, L.node_ptr, L.node_idx, local, L.dir, F,
                                                                      out);
    else
        q2_gather_kernel<T, Q2_RHS><<<nb(L.n, 256), 256, 0, s>>>(L.n, L.node_ptr, L.node_idx, local, L.dir, F, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t q2_prolongate(const DeviceMesh& dm, const T* xc, T* xf, cudaStream_t s) {
    q2_prolongate_kernel<T><<<nb(dm.n_fine, 256), 256, 0, s>>>(dm.n_fine, dm.node_ptr, dm.node_idx, dm.patch_map_mid,
                                                               xc, xf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t q2_restrict(const DeviceMesh& dm, const T* b_fine, T* part, T* b_coarse, cudaStream_t s) {
    q2_restrict_patch_kernel<T><<<nb(27 * dm.nc, 256), 256, 0, s>>>(dm.nc, dm.patch_map, dm.node_ptr, b_fine, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    q2_restrict_gather_kernel<T><<<nb(dm.n_mid, 256), 256, 0, s>>>(dm.n_mid, dm.mid_ptr, dm.mid_idx, part,
                                                                   dm.mid_dir, b_coarse);
    return cudaGetLastError();
}

template <typename T, typename TX>
cudaError_t q2_local_restrict(const DeviceMesh& dm, const T* xf, const T* r, const T* geo, int ld, TX* X,
                              cudaStream_t s) {
    q2_local_restrict_kernel<T, TX><<<nb(dm.nc * ld, 256), 256, 0, s>>>(dm.nc, dm.n_geo, ld, dm.patch_map, xf, r, geo,
                                                                        X);
    return cudaGetLastError();
}

#define DNNMG_Q2_INST(T)                                                                                          \
    template cudaError_t q2_level_local<T>(const Q2Level&, int, const T*, const T*, OpParams, double, double, int, \
                                           T*, cudaStream_t);                                                     \
    template cudaError_t q2_gather<T>(const Q2Level&, int, const T*, const T*, T*, cudaStream_t);                \
    template cudaError_t q2_prolongate<T>(const DeviceMesh&, const T*, T*, cudaStream_t);                        \
    template cudaError_t q2_restrict<T>(const DeviceMesh&, const T*, T*, T*, cudaStream_t);
DNNMG_Q2_INST(double)
DNNMG_Q2_INST(float)
#undef DNNMG_Q2_INST
template cudaError_t q2_local_restrict<double, double>(const DeviceMesh&, const double*, const double*,
                                                       const double*, int, double*, cudaStream_t);
template cudaError_t q2_local_restrict<float, float>(const DeviceMesh&, const float*, const float*, const float*, int,
                                                     float*, cudaStream_t);
template cudaError_t q2_local_restrict<float, __nv_bfloat16>(const DeviceMesh&, const float*, const float*,
                                                             const float*, int, __nv_bfloat16*, cudaStream_t);

}  // namespace dnnmg
