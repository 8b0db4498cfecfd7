// Patch kernels of the DNN-MG correction (Sec. 5.1-5.2) for sm_103a.
//
// Data flow of one step (all device memory, one stream):
//   patch_operator<RES>  coarse x^L -> per-patch partial A(P x^L) [nc][27][4]
//   node_reduce<RES>     r_j = F_j - sum over patches containing j (patch order)
//   local_restrict       X[P] = [x~(27x4) | r(27x4) | 12 edge lengths | 0 pad]
//   (network layers)     Y = N(X)
//   extend               d_j = mu_j * sum_P Y[P][iota]  (patch order)
//   patch_operator<RHS>  per-patch partial b(x~ + d) [nc][27][4] and its
//                        restriction to the 8 corners [nc][8][4]
//   node_reduce<RHS>     b_j = sum of partials; vertex_reduce: b^L_v likewise
//
// Every reduction is a gather over a CSR list sorted by patch index, so the
// results are bitwise reproducible run to run (no floating-point atomics).
#include <cstdio>
#include <limits>
#include <mutex>
#include <type_traits>

#include "internal.h"

namespace dnnmg {
namespace {

// 0.5 / sqrt(3): the 2-point Gauss points on [0, 1] are 0.5 -+ this.
constexpr double kGaussOff = 0.28867513459481288225457439025098;

template <typename T>
struct V4 {};
template <>
struct alignas(16) V4<float> {
    float x, y, z, w;
};
template <>
struct alignas(32) V4<double> {
    double x, y, z, w;
};

template <typename T>
__device__ __forceinline__ V4<T> ld4(const T* p) {
    return *reinterpret_cast<const V4<T>*>(p);
}
template <typename T>
__device__ __forceinline__ void st4(T* p, V4<T> v) {
    *reinterpret_cast<V4<T>*>(p) = v;
}

// Three consecutive values p[0..2] of an array that is only element-aligned,
// as one aligned pair and one scalar: the pair starts at p when p is aligned
// to two elements, else at p + 1.
template <typename T>
__device__ __forceinline__ void ld3(const T* p, T (&o)[3]) {
    using P2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const bool even = (reinterpret_cast<uintptr_t>(p) & (2 * sizeof(T) - 1)) == 0;
    const P2 q = *reinterpret_cast<const P2*>(p + (even ? 0 : 1));
    const T single = p[even ? 2 : 0];
    o[0] = even ? T(q.x) : single;
    o[1] = even ? T(q.y) : T(q.x);
    o[2] = even ? single : T(q.y);
}

// Patches of J levels (Sec. 5.2): a coarse cell refined J times, NC = 2^J
// cells and NS = NC + 1 nodes per axis; node iota = a + NS b + NS^2 c.
template <int J>
struct PatchGeom {
    static constexpr int NC = 1 << J;
    static constexpr int NS = NC + 1;
    static constexpr int NPN = NS * NS * NS;   // nodes per patch (27, 125)
    static constexpr int NCELL = NC * NC * NC; // fine cells per patch (8, 64)
};

// Interpolate corner values c[8] (corner k at (k&1, (k>>1)&1, (k>>2)&1)) to
// the patch node with grid coordinates (a, b, cz) in {0..NS-1}^3: along each
// axis the node sits at t = a / (NS - 1); t = 0 takes corner 0, t = 1
// corner 1, in between (1 - t) c0 + t c1 (for t = 1/2 the mean).
template <typename T, int NS>
__device__ __forceinline__ T lerp_axis(int a, T c0, T c1) {
    if (a == 0) return c0;
    if (a == NS - 1) return c1;
    const T t = T(a) / T(NS - 1);
    return (T(1) - t) * c0 + t * c1;
}
template <typename T, int STRIDE, int NS = 3>
__device__ __forceinline__ T interp27(const T* c, int comp, int a, int b, int cz) {
    T e00 = lerp_axis<T, NS>(a, c[0 * STRIDE + comp], c[1 * STRIDE + comp]);
    T e10 = lerp_axis<T, NS>(a, c[2 * STRIDE + comp], c[3 * STRIDE + comp]);
    T e01 = lerp_axis<T, NS>(a, c[4 * STRIDE + comp], c[5 * STRIDE + comp]);
    T e11 = lerp_axis<T, NS>(a, c[6 * STRIDE + comp], c[7 * STRIDE + comp]);
    T f0 = lerp_axis<T, NS>(b, e00, e10);
    T f1 = lerp_axis<T, NS>(b, e01, e11);
    return lerp_axis<T, NS>(cz, f0, f1);
}
// trilinear weight of corner bit kd at node coordinate a (of NS per axis)
template <typename T, int NS>
__device__ __forceinline__ T corner_weight(int a, int kd) {
    const T t = T(a) / T(NS - 1);
    return kd ? t : T(1) - t;
}

enum { MODE_RESIDUAL = 0, MODE_RHS = 1 };

// A trilinear function on [0,1]^3 with nodal values f_k (k = k0 + 2 k1 +
// 4 k2) is sum_S c_S phi_S with the monomials phi_S = prod_{d in S} xi_d (S a
// bit mask over the axes).  to_monomials maps f to c in place (one
// difference per axis pair); from_moments maps moments M_S = integrals
// against phi_S back to integrals against the nodal basis,
// R_k = sum_{S >= k} (-1)^{|S|-|k|} M_S, which is the transpose map.
template <typename T>
__device__ __forceinline__ void to_monomials(T (&c)[8]) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int S = 0; S < 8; ++S)
            if (!(S & (1 << d))) c[S | (1 << d)] -= c[S];
}
// Monomial coefficients over a patch (its coarse cell, reference cube
// [0,1]^3) to those over the patch's fine cell (ci, cj, ck) of NC per axis:
// the substitution xi_d = (i_d + xi'_d) / NC, one axis at a time (c_S gains
// i_d / NC times c_{S+d}, which then scales by 1 / NC).  Exact up to
// rounding: the trilinear function restricted to a sub-box is trilinear.
template <int NC, typename T>
__device__ __forceinline__ void to_cell(T (&c)[8], int ci, int cj, int ck) {
    const int id[3] = {ci, cj, ck};
    constexpr double inv = 1.0 / NC;   // NC = 2 or 4: exact
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const T o = T(id[d]) * T(inv);
#pragma unroll
        for (int S = 0; S < 8; ++S)
            if (!(S & (1 << d))) {
                c[S] += o * c[S | (1 << d)];
                c[S | (1 << d)] *= T(inv);
            }
    }
}
template <typename T>
__device__ __forceinline__ void from_moments(T (&c)[8]) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int S = 0; S < 8; ++S)
            if (!(S & (1 << d))) c[S] -= c[S | (1 << d)];
}

// Element integrals of one fine cell whose geometry X[d] and fields U[c]
// (u, v, w, p) are given as monomial coefficients over the cell's own
// reference cube, accumulated into R[8][4] (the cell's 8 vertices), with the
// 2x2x2 Gauss rule:
//   MODE_RESIDUAL: Galerkin part of A_h (Eq. (6) left-hand side):
//     R_kc += w [ (m v_c + th conv_c) N_k + th nu Dv_c . g_k - p (g_k)_c ]
//     R_k3 += w div(v) N_k
//   MODE_RHS: right-hand side of Eq. (6) without force:
//     R_kc += w [ (m v_c - (1-th) conv_c) N_k - (1-th) nu Dv_c . g_k ]
// with g_k = J^{-T} grad_ref N_k and w = det J / 8.  Geometry and fields are
// evaluated from their monomial coefficients (J and the reference gradient
// in 4 terms each); the gradient terms are applied in reference coordinates,
// Dv_c . g_k - p (g_k)_c = sum_e dN_k/dxi_e Fhat_ce / w with
// Fhat_ce = w sum_d Jinv_ed (coef Dv_cd - p delta_cd), and the test
// functions enter through the moments of the monomials.
//
// affine: the cell is a parallelepiped (its patch's corners are), so J is
// constant; it is then formed at the first Gauss point only and reused.
template <typename T, int MODE>
__device__ __forceinline__ void element(const T (&X)[3][8], const T (&U)[4][8], T (&R)[8][4], T m, T th, T nu,
                                        bool affine) {
    T M[4][8];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int S = 0; S < 8; ++S) M[c][S] = T(0);
    T Ji[3][3], w;   // Jinv[e][d] = d xi_e / d x_d and the weight det J / 8 at the point
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const T x0 = (q & 1) ? T(0.5 + kGaussOff) : T(0.5 - kGaussOff);
        const T x1 = (q & 2) ? T(0.5 + kGaussOff) : T(0.5 - kGaussOff);
        const T x2 = (q & 4) ? T(0.5 + kGaussOff) : T(0.5 - kGaussOff);
        auto val = [&](const T (&c)[8]) {
            return c[0] + c[1] * x0 + c[2] * x1 + c[3] * (x0 * x1) + c[4] * x2 + c[5] * (x0 * x2) + c[6] * (x1 * x2) +
                   c[7] * (x0 * x1 * x2);
        };
        auto d0 = [&](const T (&c)[8]) { return c[1] + c[3] * x1 + c[5] * x2 + c[7] * (x1 * x2); };
        auto d1 = [&](const T (&c)[8]) { return c[2] + c[3] * x0 + c[6] * x2 + c[7] * (x0 * x2); };
        auto d2 = [&](const T (&c)[8]) { return c[4] + c[5] * x0 + c[6] * x1 + c[7] * (x0 * x1); };
        T Dr[3][3], v[3];   // Dr[c][e] = dv_c/dxi_e
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Dr[d][0] = d0(U[d]);
            Dr[d][1] = d1(U[d]);
            Dr[d][2] = d2(U[d]);
            v[d] = val(U[d]);
        }
        const T p = MODE == MODE_RESIDUAL ? val(U[3]) : T(0);
        if (q == 0 || !affine) {   // warp-uniform: the patches of a warp share the test's outcome but rarely
            T J[3][3];             // J[d][e] = dx_d/dxi_e
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                J[d][0] = d0(X[d]);
                J[d][1] = d1(X[d]);
                J[d][2] = d2(X[d]);
            }
            const T c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            const T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            const T c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            const T det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
            const T idet = T(1) / det;
            Ji[0][0] = c00 * idet;
            Ji[1][0] = c01 * idet;
            Ji[2][0] = c02 * idet;
            Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * idet;
            Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * idet;
            Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * idet;
            Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * idet;
            Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * idet;
            Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * idet;
            w = det * T(0.125);
        }
        T Dv[3][3];   // d v_c / d x_d
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) Dv[c][d] = Dr[c][0] * Ji[0][d] + Dr[c][1] * Ji[1][d] + Dr[c][2] * Ji[2][d];
        const T tc = MODE == MODE_RESIDUAL ? th : th - T(1);
        const T visc = tc * nu * w;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T conv = v[0] * Dv[c][0] + v[1] * Dv[c][1] + v[2] * Dv[c][2];
            const T a = w * (m * v[c] + tc * conv);
            T G[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) G[d] = visc * Dv[c][d] - (MODE == MODE_RESIDUAL && d == c ? w * p : T(0));
            const T F0 = Ji[0][0] * G[0] + Ji[0][1] * G[1] + Ji[0][2] * G[2];
            const T F1 = Ji[1][0] * G[0] + Ji[1][1] * G[1] + Ji[1][2] * G[2];
            const T F2 = Ji[2][0] * G[0] + Ji[2][1] * G[1] + Ji[2][2] * G[2];
            // a phi_S + Fhat . grad_ref phi_S for the 8 monomials
            M[c][0] += a;
            M[c][1] += a * x0 + F0;
            M[c][2] += a * x1 + F1;
            M[c][3] += a * (x0 * x1) + F0 * x1 + F1 * x0;
            M[c][4] += a * x2 + F2;
            M[c][5] += a * (x0 * x2) + F0 * x2 + F2 * x0;
            M[c][6] += a * (x1 * x2) + F1 * x2 + F2 * x1;
            M[c][7] += a * (x0 * x1 * x2) + F0 * (x1 * x2) + F1 * (x0 * x2) + F2 * (x0 * x1);
        }
        if (MODE == MODE_RESIDUAL) {
            const T s = w * (Dv[0][0] + Dv[1][1] + Dv[2][2]);
            M[3][0] += s;
            M[3][1] += s * x0;
            M[3][2] += s * x1;
            M[3][3] += s * (x0 * x1);
            M[3][4] += s * x2;
            M[3][5] += s * (x0 * x2);
            M[3][6] += s * (x1 * x2);
            M[3][7] += s * (x0 * x1 * x2);
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        from_moments(M[c]);
#pragma unroll
        for (int k = 0; k < 8; ++k) R[k][c] += M[c][k];
    }
}

// Corners cr[d][k] relative to corner 0 (cr[d][0] = 0) span a
// parallelepiped when the bilinear and trilinear monomial coefficients of
// the trilinear map vanish; "vanish" allows 16 rounding units of the edge
// vectors, far below any tolerance the results are held to.  Then every
// fine cell of the patch is a parallelepiped too, with a constant Jacobian.
template <typename T>
__device__ __forceinline__ bool is_parallelepiped(const T (&cr)[3][8]) {
    T edge = T(0), bend = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const T c3 = cr[d][3] - cr[d][2] - cr[d][1];
        const T c5 = cr[d][5] - cr[d][4] - cr[d][1];
        const T c6 = cr[d][6] - cr[d][4] - cr[d][2];
        const T c7 = cr[d][7] - cr[d][6] - cr[d][5] + cr[d][4] - c3;
        edge = fmax(edge, fmax(fabs(cr[d][1]), fmax(fabs(cr[d][2]), fabs(cr[d][4]))));
        bend = fmax(bend, fmax(fmax(fabs(c3), fabs(c5)), fmax(fabs(c6), fabs(c7))));
    }
    return bend <= T(16) * std::numeric_limits<T>::epsilon() * edge;
}

constexpr int kPatchThreads = 64;   // threads per block of the patch operator
template <int J>
constexpr int patches_per_block() { return kPatchThreads / PatchGeom<J>::NCELL; }   // 8 (J = 1), 1 (J = 2)

// One thread per fine cell; the NCELL consecutive threads of a patch share
// its corners (and, for the rhs, the correction at its nodes) in shared
// memory, and each forms its own cell's monomial coefficients from them.
// 128 registers (8 blocks of 64 threads per SM) for float: the element's
// arithmetic is latency-bound at fewer warps
template <typename T>
constexpr int patch_min_blocks() { return sizeof(T) == 4 ? 8 : 4; }

template <typename T, int MODE, int J>
__global__ void __launch_bounds__(kPatchThreads, patch_min_blocks<T>()) patch_operator_kernel(
    int64_t nc, const int32_t* __restrict__ cells, const int32_t* __restrict__ patch_map,
    const T* __restrict__ xyz, const T* __restrict__ xc, const T* __restrict__ dfine, T m, T th, T nu,
    T* __restrict__ partial, T* __restrict__ partial_c) {
    using G = PatchGeom<J>;
    constexpr int PPB = patches_per_block<J>();
    constexpr int TPP = G::NCELL;                 // threads per patch
    __shared__ T s_cx[PPB][8][3];                 // corner coordinates
    __shared__ T s_cu[PPB][8][4];                 // corner values
    // RHS: the correction d at the patch nodes, later the node sums of the
    // partial rhs (stride 5 spreads the 8 nodes a cell reads over banks)
    __shared__ T s_node[PPB][G::NPN][5];
    // per-cell contributions, one padded row of 8 x 4 per cell: the cells'
    // threads store with a stride of 33 words (no bank conflicts)
    __shared__ T s_R[PPB][G::NCELL][33];

    const int lp = threadIdx.x / TPP;   // patch within block
    const int t = threadIdx.x % TPP;    // fine cell of the patch / node / corner
    const int64_t P = int64_t(blockIdx.x) * PPB + lp;
    const bool active = P < nc;

    if (active && t < 8) {
        const int32_t v = cells[8 * P + t];
#pragma unroll
        for (int d = 0; d < 3; ++d) s_cx[lp][t][d] = xyz[3 * int64_t(v) + d];
        const V4<T> u = ld4(xc + 4 * int64_t(v));
        s_cu[lp][t][0] = u.x;
        s_cu[lp][t][1] = u.y;
        s_cu[lp][t][2] = u.z;
        s_cu[lp][t][3] = u.w;
    }
    if (MODE == MODE_RHS && active) {
        // the correction at this thread's nodes, every load issued before
        // the first is used (node ids, then their values)
        constexpr int NPT = (G::NPN + TPP - 1) / TPP;   // nodes per thread (4, 2)
        int64_t jn[NPT];
        T dn[NPT][3];
#pragma unroll
        for (int i = 0; i < NPT; ++i) {
            const int iota = t + i * TPP;
            jn[i] = iota < G::NPN ? int64_t(patch_map[G::NPN * P + iota]) : 0;
        }
#pragma unroll
        for (int i = 0; i < NPT; ++i)
#pragma unroll
            for (int d = 0; d < 3; ++d) dn[i][d] = t + i * TPP < G::NPN ? dfine[3 * jn[i] + d] : T(0);
#pragma unroll
        for (int i = 0; i < NPT; ++i)
            if (t + i * TPP < G::NPN)
#pragma unroll
                for (int d = 0; d < 3; ++d) s_node[lp][t + i * TPP][d] = dn[i][d];
    }
    __syncthreads();
    if (active) {
        // the coarse cell's corners (coordinates relative to corner 0: the
        // element needs only differences) as monomial coefficients over the
        // patch, then over this thread's fine cell
        T X[3][8], U[4][8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
#pragma unroll
            for (int d = 0; d < 3; ++d) X[d][k] = s_cx[lp][k][d] - s_cx[lp][0][d];
#pragma unroll
            for (int c = 0; c < 4; ++c) U[c][k] = s_cu[lp][k][c];
        }
        const bool affine = is_parallelepiped(X);
        const int ci = t % G::NC, cj = (t / G::NC) % G::NC, ck = t / (G::NC * G::NC);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            to_monomials(X[d]);
            to_cell<G::NC>(X[d], ci, cj, ck);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            to_monomials(U[c]);
            to_cell<G::NC>(U[c], ci, cj, ck);
        }
        if (MODE == MODE_RHS) {   // corrected velocity x~ + d, d nodal on the fine nodes
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                T dc[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int node =
                        (ci + (k & 1)) + G::NS * (cj + ((k >> 1) & 1)) + G::NS * G::NS * (ck + ((k >> 2) & 1));
                    dc[k] = s_node[lp][node][c];
                }
                to_monomials(dc);
#pragma unroll
                for (int S = 0; S < 8; ++S) U[c][S] += dc[S];
            }
        }
        T R[8][4];
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) R[k][c] = T(0);
        element<T, MODE>(X, U, R, m, th, nu, affine);
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) s_R[lp][t][4 * k + c] = R[k][c];
    }
    __syncthreads();
    // sum the contributions of the cells containing each patch node, in a fixed order
    for (int iota = t; active && iota < G::NPN; iota += TPP) {
        const int a = iota % G::NS, b = (iota / G::NS) % G::NS, c = iota / (G::NS * G::NS);
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int k2 = 0; k2 < 2; ++k2) {
            const int ck = c - k2;
            if (ck < 0 || ck >= G::NC) continue;
            for (int j2 = 0; j2 < 2; ++j2) {
                const int cj = b - j2;
                if (cj < 0 || cj >= G::NC) continue;
                for (int i2 = 0; i2 < 2; ++i2) {
                    const int ci = a - i2;
                    if (ci < 0 || ci >= G::NC) continue;
                    const int cell = ci + G::NC * cj + G::NC * G::NC * ck;
                    const int vert = i2 + 2 * j2 + 4 * k2;
#pragma unroll
                    for (int d = 0; d < 4; ++d) acc[d] += s_R[lp][cell][4 * vert + d];
                }
            }
        }
        if (MODE == MODE_RHS) acc[3] = T(0);
        st4(partial + (G::NPN * P + iota) * 4, V4<T>{acc[0], acc[1], acc[2], acc[3]});
        if (MODE == MODE_RHS) {
            // keep the node sums for the restriction below
#pragma unroll
            for (int d = 0; d < 4; ++d) s_node[lp][iota][d] = acc[d];
        }
    }
    if (MODE == MODE_RHS) {
        __syncthreads();
        if (!active || t >= 8) return;
        // restriction P^T of the patch's partial rhs onto its 8 corners:
        // corner k collects node iota with the trilinear weight of k at iota
        const int k = t;
        const int kx = k & 1, ky = (k >> 1) & 1, kz = (k >> 2) & 1;
        T acc[3] = {T(0), T(0), T(0)};
        for (int iota = 0; iota < G::NPN; ++iota) {
            const int a = iota % G::NS, b = (iota / G::NS) % G::NS, c = iota / (G::NS * G::NS);
            const T wgt = corner_weight<T, G::NS>(a, kx) * corner_weight<T, G::NS>(b, ky) *
                          corner_weight<T, G::NS>(c, kz);
            if (wgt != T(0)) {
#pragma unroll
                for (int d = 0; d < 3; ++d) acc[d] += wgt * s_node[lp][iota][d];
            }
        }
        st4(partial_c + (8 * P + k) * 4, V4<T>{acc[0], acc[1], acc[2], T(0)});
    }
}

// r_j = F_j - sum_{(P,iota) in j} partial[P][iota]  (RESIDUAL)
// b_j = sum partial (pressure row 0)                   (RHS)
// Velocity rows of Dirichlet nodes are 0.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) node_reduce_kernel(
    int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
    const T* __restrict__ partial, const uint8_t* __restrict__ dir, const T* __restrict__ F,
    T* __restrict__ out) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    const int32_t e1 = ptr[j + 1];
    for (int32_t e = ptr[j]; e < e1; ++e) {
        const V4<T> pv = ld4(partial + 4 * int64_t(idx[e]));
        acc[0] += pv.x;
        acc[1] += pv.y;
        acc[2] += pv.z;
        acc[3] += pv.w;
    }
    V4<T> o;
    if (MODE == MODE_RESIDUAL) {
        const V4<T> f = ld4(F + 4 * j);
        o = V4<T>{f.x - acc[0], f.y - acc[1], f.z - acc[2], f.w - acc[3]};
    } else {
        o = V4<T>{acc[0], acc[1], acc[2], T(0)};
    }
    if (dir[j]) {
        o.x = T(0);
        o.y = T(0);
        o.z = T(0);
    }
    st4(out + 4 * j, o);
}

// b^L_v = sum over (P, k) with cells[P][k] = v of partial_c[P][k]; Dirichlet
// velocity rows and the pressure row are 0.
template <typename T>
__global__ void __launch_bounds__(256) vertex_reduce_kernel(
    int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
    const T* __restrict__ partial_c, const uint8_t* __restrict__ dir, T* __restrict__ out) {
    const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= n) return;
    T acc[3] = {T(0), T(0), T(0)};
    const int32_t e1 = ptr[v + 1];
    for (int32_t e = ptr[v]; e < e1; ++e) {
        const V4<T> pv = ld4(partial_c + 4 * int64_t(idx[e]));
        acc[0] += pv.x;
        acc[1] += pv.y;
        acc[2] += pv.z;
    }
    if (dir[v]) acc[0] = acc[1] = acc[2] = T(0);
    st4(out + 4 * v, V4<T>{acc[0], acc[1], acc[2], T(0)});
}

// Restriction of a fine vector, patch part: corner k of patch P collects
// sum_iota w(iota, k) b[dof(P, iota)] / valence(dof(P, iota)); summed over the
// patches containing a coarse vertex (vertex_reduce) this is (P^T b)_v,
// because every patch containing a fine node contains all its parents.
template <typename T, int J>
__global__ void __launch_bounds__(256) restrict_patch_kernel(
    int64_t nc, const int32_t* __restrict__ patch_map, const int32_t* __restrict__ node_ptr,
    const T* __restrict__ b, T* __restrict__ partial_c) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;   // P * 8 + k
    if (e >= 8 * nc) return;
    const int64_t P = e >> 3;
    const int k = int(e & 7);
    const int kx = k & 1, ky = (k >> 1) & 1, kz = (k >> 2) & 1;
    using G = PatchGeom<J>;
    T acc[3] = {T(0), T(0), T(0)};
    for (int iota = 0; iota < G::NPN; ++iota) {
        const int a = iota % G::NS, bb = (iota / G::NS) % G::NS, c = iota / (G::NS * G::NS);
        const T w = corner_weight<T, G::NS>(a, kx) * corner_weight<T, G::NS>(bb, ky) *
                    corner_weight<T, G::NS>(c, kz);
        if (w == T(0)) continue;
        const int64_t j = patch_map[G::NPN * P + iota];
        const T s = w / T(node_ptr[j + 1] - node_ptr[j]);
#pragma unroll
        for (int d = 0; d < 3; ++d) acc[d] += s * b[4 * j + d];
    }
    st4(partial_c + 4 * e, V4<T>{acc[0], acc[1], acc[2], T(0)});
}

// x_fine[j] from the first patch containing j (deterministic).
template <typename T, int J>
__global__ void __launch_bounds__(256) prolongate_kernel(
    int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
    const int32_t* __restrict__ cells, const T* __restrict__ xc, T* __restrict__ xf) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    using G = PatchGeom<J>;
    const int32_t e = idx[ptr[j]];
    const int64_t P = e / G::NPN;
    const int iota = e % G::NPN;
    const int a = iota % G::NS, b = (iota / G::NS) % G::NS, c = iota / (G::NS * G::NS);
    T cu[8][4];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const V4<T> u = ld4(xc + 4 * int64_t(cells[8 * P + k]));
        cu[k][0] = u.x;
        cu[k][1] = u.y;
        cu[k][2] = u.z;
        cu[k][3] = u.w;
    }
    V4<T> o;
    o.x = interp27<T, 4, G::NS>(&cu[0][0], 0, a, b, c);
    o.y = interp27<T, 4, G::NS>(&cu[0][0], 1, a, b, c);
    o.z = interp27<T, 4, G::NS>(&cu[0][0], 2, a, b, c);
    o.w = interp27<T, 4, G::NS>(&cu[0][0], 3, a, b, c);
    st4(xf + 4 * j, o);
}

template <typename TX>
__device__ __forceinline__ TX cvt(float v);
template <>
__device__ __forceinline__ float cvt<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename TX>
__device__ __forceinline__ TX cvtd(double v);
template <>
__device__ __forceinline__ double cvtd<double>(double v) { return v; }

template <typename T, typename TX>
__device__ __forceinline__ TX to_x(T v) {
    if constexpr (sizeof(T) == 8)
        return cvtd<TX>(v);
    else
        return cvt<TX>(v);
}

// Four values of the input row as one vector store (16 bytes for float /
// bf16 pairs packed into 8 bytes; double stays scalar-pair).
template <typename TX>
struct Pack4 {};
template <>
struct alignas(8) Pack4<__nv_bfloat16> {
    __nv_bfloat162 a, b;
};
template <>
struct alignas(16) Pack4<float> {
    float a, b, c, d;
};
template <>
struct alignas(16) Pack4<double> {   // two 16-byte halves
    double a, b, c, d;
};
template <typename TX, typename T>
__device__ __forceinline__ void store4(TX* dst, T a, T b, T c, T d) {
    if constexpr (sizeof(TX) == 2) {
        Pack4<__nv_bfloat16> v{__floats2bfloat162_rn(float(a), float(b)), __floats2bfloat162_rn(float(c), float(d))};
        *reinterpret_cast<Pack4<__nv_bfloat16>*>(dst) = v;
    } else if constexpr (sizeof(TX) == 4) {
        *reinterpret_cast<Pack4<float>*>(dst) = Pack4<float>{float(a), float(b), float(c), float(d)};
    } else {
        reinterpret_cast<double2*>(dst)[0] = make_double2(double(a), double(b));
        reinterpret_cast<double2*>(dst)[1] = make_double2(double(c), double(d));
    }
}

// One warp per 2 patches (J = 1) or 1 (J = 2): X[P] = [x~ at the NPN nodes | r at the NPN nodes |
// geometry | 0] with row stride LD = 256 (J = 1) or 1024 (J = 2).  Lane l
// writes nodes l, l + 32, ... (4 values of x~ and of r as one vector each);
// the first (LD - 8 NPN) / 4 lanes write the n_geo (12 or 24) geometry
// features and the zeros after them up to the row end.  Every 4-value group
// is aligned.
template <int J>
constexpr int restrict_patches_per_warp() { return J == 1 ? 2 : 1; }   // independent gathers in flight

template <typename T, typename TX, int J>
__global__ void __launch_bounds__(256) local_restrict_kernel(
    int64_t nc, const int32_t* __restrict__ cells, const int32_t* __restrict__ patch_map,
    const T* __restrict__ xc, const T* __restrict__ r, const T* __restrict__ geo, int n_geo,
    TX* __restrict__ X) {
    using G = PatchGeom<J>;
    constexpr int LD = J == 1 ? kNInPad : kNInPadJ2;
    constexpr int NPL = (G::NPN + 31) / 32;            // nodes per lane
    constexpr int PPW = restrict_patches_per_warp<J>();
    const int lane = threadIdx.x & 31;
    const int64_t P0 = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * PPW;
    if (P0 >= nc) return;   // warp-uniform
    // issue every independent load of the warp's patches first: corner ids,
    // node ids and geometry, then the node residuals and corner values
    int32_t v[PPW], jn[PPW][NPL];
    T el[PPW];
#pragma unroll
    for (int p = 0; p < PPW; ++p) {
        const int64_t P = P0 + p;
        const bool ok = P < nc;
        v[p] = ok && lane < 8 ? __ldg(cells + 8 * P + lane) : 0;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int iota = lane + 32 * i;
            jn[p][i] = ok && iota < G::NPN ? __ldg(patch_map + int64_t(G::NPN) * P + iota) : 0;
        }
        el[p] = ok && lane < n_geo ? geo[int64_t(n_geo) * P + lane] : T(0);
    }
    V4<T> rv[PPW][NPL];
    T cu[PPW][4];
#pragma unroll
    for (int p = 0; p < PPW; ++p) {
        const bool ok = P0 + p < nc;
#pragma unroll
        for (int i = 0; i < NPL; ++i)
            rv[p][i] = ok && lane + 32 * i < G::NPN ? ld4(r + 4 * int64_t(jn[p][i])) : V4<T>{T(0), T(0), T(0), T(0)};
        V4<T> u{T(0), T(0), T(0), T(0)};
        if (ok && lane < 8) u = ld4(xc + 4 * int64_t(v[p]));
        cu[p][0] = u.x;
        cu[p][1] = u.y;
        cu[p][2] = u.z;
        cu[p][3] = u.w;
    }
#pragma unroll
    for (int p = 0; p < PPW; ++p) {
        const int64_t P = P0 + p;
        if (P >= nc) break;   // warp-uniform
        // J = 1: x~ at this lane's node as the weighted sum of the corners,
        // fetched one corner at a time (J = 2: all corners held, 4 nodes per lane)
        T xt[4] = {T(0), T(0), T(0), T(0)};
        T corner[J == 1 ? 1 : 8][4];
        if constexpr (J == 1) {
            const int a = lane % 3, b = (lane / 3) % 3, c = lane / 9;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const T wk = corner_weight<T, 3>(a, k & 1) * corner_weight<T, 3>(b, (k >> 1) & 1) *
                             corner_weight<T, 3>(c, (k >> 2) & 1);
#pragma unroll
                for (int d = 0; d < 4; ++d) xt[d] += wk * __shfl_sync(0xffffffffu, cu[p][d], k);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int d = 0; d < 4; ++d) corner[k][d] = __shfl_sync(0xffffffffu, cu[p][d], k);
        }
        // geometry features 4 lane .. 4 lane + 3 (zero past n_geo)
        T e[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const T g = __shfl_sync(0xffffffffu, el[p], (4 * lane + i) & 31);
            e[i] = 4 * lane + i < n_geo ? g : T(0);
        }
        TX* row = X + P * LD;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int iota = lane + 32 * i;
            if (iota >= G::NPN) continue;
            if constexpr (J == 1) {
                store4<TX>(row + 4 * iota, xt[0], xt[1], xt[2], xt[3]);
            } else {
                const int a = iota % G::NS, b = (iota / G::NS) % G::NS, c = iota / (G::NS * G::NS);
                store4<TX>(row + 4 * iota, interp27<T, 4, G::NS>(&corner[0][0], 0, a, b, c),
                           interp27<T, 4, G::NS>(&corner[0][0], 1, a, b, c),
                           interp27<T, 4, G::NS>(&corner[0][0], 2, a, b, c),
                           interp27<T, 4, G::NS>(&corner[0][0], 3, a, b, c));
            }
            store4<TX>(row + 4 * G::NPN + 4 * iota, rv[p][i].x, rv[p][i].y, rv[p][i].z, rv[p][i].w);
        }
        constexpr int GEO0 = 8 * G::NPN;              // first geometry column (216, 1000)
        constexpr int GEO_GROUPS = (LD - GEO0) / 4;   // 4-column groups up to the row end (10, 6)
        static_assert(GEO_GROUPS <= 32 && 4 * GEO_GROUPS >= 24 && GEO0 + 4 * GEO_GROUPS == LD, "input row layout");
        if (lane < GEO_GROUPS)   // columns GEO0 .. LD - 1: the features, then zeros
            store4<TX>(row + GEO0 + 4 * lane, e[0], e[1], e[2], e[3]);
    }
}

// d_j = mu_j * sum_{(P,iota) in j} Y[P][3 iota + c], mu_j = 1 / valence.
template <typename T>
__global__ void __launch_bounds__(256) extend_kernel(
    int64_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
    const T* __restrict__ Y, const uint8_t* __restrict__ dir, T* __restrict__ d) {
    const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    T acc[3] = {T(0), T(0), T(0)};
    const int32_t e0 = ptr[j], e1 = ptr[j + 1];
    for (int32_t e = e0; e < e1; ++e) {
        T y[3];
        ld3(Y + 3 * int64_t(idx[e]), y);   // Y[P][3 iota]: rows of 3 x nodes per patch
        acc[0] += y[0];
        acc[1] += y[1];
        acc[2] += y[2];
    }
    const T mu = T(1) / T(e1 - e0);
    const bool dj = dir[j] != 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) d[3 * j + c] = dj ? T(0) : acc[c] * mu;
}

// ---- SIMT network layer ----------------------------------------------------
template <typename T>
struct AccOf {
    using type = float;
};
template <>
struct AccOf<double> {
    using type = double;
};

template <typename T>
__device__ __forceinline__ float tof(T v) {
    return float(v);
}
template <>
__device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}
template <typename TACC, typename T>
__device__ __forceinline__ TACC toacc(T v) {
    if constexpr (sizeof(TACC) == 8)
        return TACC(v);
    else
        return tof<T>(v);
}
template <typename TC, typename TACC>
__device__ __forceinline__ TC fromacc(TACC v) {
    if constexpr (sizeof(TC) == 2)
        return __float2bfloat16_rn(float(v));
    else
        return TC(v);
}

// 64 x 64 output tile per block of 256 threads, 4 x 4 per thread, K step 16.
template <typename TA, typename TW, typename TC, typename TS, typename TACC>
__global__ void __launch_bounds__(256) layer_simt_kernel(
    const TA* __restrict__ A, int64_t lda, const TW* __restrict__ W, int64_t ldw,
    const TS* __restrict__ scale, const TS* __restrict__ shift, TC* __restrict__ C, int64_t ldc,
    const TA* __restrict__ R, int64_t ldr, int64_t M, int N, int K, int relu) {
    __shared__ TACC sA[16][64 + 1];
    __shared__ TACC sW[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = int64_t(blockIdx.x) * 64;
    const int n0 = blockIdx.y * 64;
    TACC acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = TACC(0);
    for (int k0 = 0; k0 < K; k0 += 16) {
        // load 64 x 16 of A and of W (each thread 4 elements of each)
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = threadIdx.x + 256 * l;   // 0..1023
            const int row = e >> 4, kk = e & 15;
            const int64_t gm = m0 + row;
            const int gn = n0 + row;
            sA[kk][row] = gm < M ? toacc<TACC>(A[gm * lda + k0 + kk]) : TACC(0);
            sW[kk][row] = gn < N ? toacc<TACC>(W[int64_t(gn) * ldw + k0 + kk]) : TACC(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            TACC a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sW[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tx + 16 * j;
            if (gn >= N) continue;
            TACC z = toacc<TACC>(scale[gn]) * acc[i][j] + toacc<TACC>(shift[gn]);
            if (relu) z = z > TACC(0) ? z : TACC(0);
            if (R) z += toacc<TACC>(R[gm * ldr + gn]);
            C[gm * ldc + gn] = fromacc<TC, TACC>(z);
        }
    }
}

inline unsigned blocks_for(int64_t n, int per) { return unsigned((n + per - 1) / per); }

}  // namespace

// ---- launchers ---------------------------------------------------------------
template <typename T>
static const T* xyz_of(const DeviceMesh& dm);
template <>
const double* xyz_of<double>(const DeviceMesh& dm) { return dm.xyz_d; }
template <>
const float* xyz_of<float>(const DeviceMesh& dm) { return dm.xyz_f; }
template <typename T>
static const T* edge_of(const DeviceMesh& dm);
template <>
const double* edge_of<double>(const DeviceMesh& dm) { return dm.geo_d; }
template <>
const float* edge_of<float>(const DeviceMesh& dm) { return dm.geo_f; }

template <typename T>
cudaError_t launch_prolongate(const DeviceMesh& dm, const T* xc, T* xf, cudaStream_t s) {
    if (dm.J == 2)
        prolongate_kernel<T, 2><<<blocks_for(dm.n_fine, 256), 256, 0, s>>>(dm.n_fine, dm.node_ptr, dm.node_idx,
                                                                            dm.cells, xc, xf);
    else
        prolongate_kernel<T, 1><<<blocks_for(dm.n_fine, 256), 256, 0, s>>>(dm.n_fine, dm.node_ptr, dm.node_idx,
                                                                            dm.cells, xc, xf);
    return cudaGetLastError();
}

// training targets: out[P ldt + 3 iota + c] = v[j][c] - xt[j][c] for the
// patch's node j = patch_map[P][iota], velocity components, in fp32
template <typename T>
__global__ void __launch_bounds__(256) targets_kernel(int64_t nc, int npn, const int32_t* __restrict__ pm,
                                                      const T* __restrict__ v, const T* __restrict__ xt,
                                                      float* __restrict__ out, int64_t ldt) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= nc * npn) return;
    const int64_t P = e / npn;
    const int iota = int(e - P * npn);
    const int64_t j = pm[e];
    const V4<T> a = ld4(v + 4 * j), b = ld4(xt + 4 * j);
    float* o = out + P * ldt + 3 * iota;
    o[0] = float(a.x - b.x);
    o[1] = float(a.y - b.y);
    o[2] = float(a.z - b.z);
}

template <typename T>
cudaError_t launch_targets(const DeviceMesh& dm, int npn, const T* v, const T* xt, float* out, int64_t ldt,
                           cudaStream_t s) {
    targets_kernel<T><<<blocks_for(dm.nc * npn, 256), 256, 0, s>>>(dm.nc, npn, dm.patch_map, v, xt, out, ldt);
    return cudaGetLastError();
}
template cudaError_t launch_targets<double>(const DeviceMesh&, int, const double*, const double*, float*, int64_t,
                                            cudaStream_t);
template cudaError_t launch_targets<float>(const DeviceMesh&, int, const float*, const float*, float*, int64_t,
                                           cudaStream_t);

// patch operator launch for J = 1 or 2 (64-thread blocks of 8 or 1 patches)
template <typename T, int MODE>
void launch_patch_operator(const DeviceMesh& dm, OpParams p, const T* xc, const T* dfine, T* partial, T* partial_c,
                           cudaStream_t s) {
    if (dm.J == 2)
        patch_operator_kernel<T, MODE, 2><<<blocks_for(dm.nc, patches_per_block<2>()), kPatchThreads, 0, s>>>(
            dm.nc, dm.cells, dm.patch_map, xyz_of<T>(dm), xc, dfine, T(p.m), T(p.theta), T(p.nu), partial,
            partial_c);
    else
        patch_operator_kernel<T, MODE, 1><<<blocks_for(dm.nc, patches_per_block<1>()), kPatchThreads, 0, s>>>(
            dm.nc, dm.cells, dm.patch_map, xyz_of<T>(dm), xc, dfine, T(p.m), T(p.theta), T(p.nu), partial,
            partial_c);
}

template <typename T>
cudaError_t launch_residual(const DeviceMesh& dm, OpParams p, const T* xc, const T* F, T* r, T* partial,
                            cudaStream_t s, int* launches, cudaEvent_t F_ready) {
    launch_patch_operator<T, MODE_RESIDUAL>(dm, p, xc, nullptr, partial, nullptr, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (F_ready && (e = cudaStreamWaitEvent(s, F_ready, 0)) != cudaSuccess) return e;
    node_reduce_kernel<T, MODE_RESIDUAL><<<blocks_for(dm.n_fine, 256), 256, 0, s>>>(
        dm.n_fine, dm.node_ptr, dm.node_idx, partial, dm.fine_dir, F, r);
    *launches += 2;
    return cudaGetLastError();
}

template <typename T, typename TX>
cudaError_t launch_local_restrict(const DeviceMesh& dm, const T* xc, const T* r, TX* X, cudaStream_t s) {
    // one warp per restrict_patches_per_warp<J>() patches
    if (dm.J == 2)
        local_restrict_kernel<T, TX, 2><<<blocks_for(dm.nc * 32, 256), 256, 0, s>>>(
            dm.nc, dm.cells, dm.patch_map, xc, r, edge_of<T>(dm), dm.n_geo, X);
    else
        local_restrict_kernel<T, TX, 1><<<blocks_for((dm.nc + 1) / 2 * 32, 256), 256, 0, s>>>(
            dm.nc, dm.cells, dm.patch_map, xc, r, edge_of<T>(dm), dm.n_geo, X);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const DeviceMesh& dm, const T* b_fine, T* b_coarse, T* partial_c, cudaStream_t s) {
    if (dm.J == 2)
        restrict_patch_kernel<T, 2><<<blocks_for(8 * dm.nc, 256), 256, 0, s>>>(dm.nc, dm.patch_map, dm.node_ptr,
                                                                                b_fine, partial_c);
    else
        restrict_patch_kernel<T, 1><<<blocks_for(8 * dm.nc, 256), 256, 0, s>>>(dm.nc, dm.patch_map, dm.node_ptr,
                                                                                b_fine, partial_c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    vertex_reduce_kernel<T><<<blocks_for(dm.nv, 256), 256, 0, s>>>(dm.nv, dm.vert_ptr, dm.vert_idx, partial_c,
                                                                   dm.coarse_dir, b_coarse);
    return cudaGetLastError();
}
template cudaError_t launch_restrict<double>(const DeviceMesh&, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_restrict<float>(const DeviceMesh&, const float*, float*, float*, cudaStream_t);

template <typename T>
cudaError_t launch_extend(const DeviceMesh& dm, const T* Y, T* d, cudaStream_t s) {
    extend_kernel<T><<<blocks_for(dm.n_fine, 256), 256, 0, s>>>(dm.n_fine, dm.node_ptr, dm.node_idx, Y,
                                                                dm.fine_dir, d);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rhs_restrict(const DeviceMesh& dm, OpParams p, const T* xc, const T* d, T* b_fine,
                                T* b_coarse, T* partial, T* partial_c, cudaStream_t s, int* launches) {
    launch_patch_operator<T, MODE_RHS>(dm, p, xc, d, partial, partial_c, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *launches += 1;
    if (b_fine) {
        node_reduce_kernel<T, MODE_RHS><<<blocks_for(dm.n_fine, 256), 256, 0, s>>>(
            dm.n_fine, dm.node_ptr, dm.node_idx, partial, dm.fine_dir, nullptr, b_fine);
        *launches += 1;
    }
    if (b_coarse) {
        vertex_reduce_kernel<T><<<blocks_for(dm.nv, 256), 256, 0, s>>>(dm.nv, dm.vert_ptr, dm.vert_idx,
                                                                      partial_c, dm.coarse_dir, b_coarse);
        *launches += 1;
    }
    return cudaGetLastError();
}

// FP32 form of the layer for 16-byte aligned operands with row strides that
// are multiples of 4: 128 x 128 tiles of C, 256 threads of 8 x 8 outputs
// (rows 4 ty .. 4 ty + 3 and 64 + 4 ty .. 64 + 4 ty + 3, columns likewise
// with tx), K in steps of 8 through two shared-memory buffers (the next
// step's operands are loaded into registers while the current one
// multiplies).  Every output sums over k in increasing order, as
// layer_simt_kernel does.
constexpr int kSgTile = 128, kSgK = 8;
__global__ void __launch_bounds__(256, 2) layer_sgemm_kernel(
    const float* __restrict__ A, int64_t lda, const float* __restrict__ W, int64_t ldw,
    const float* __restrict__ scale, const float* __restrict__ shift, float* __restrict__ C, int64_t ldc,
    const float* __restrict__ R, int64_t ldr, int64_t M, int N, int K, int relu) {
    __shared__ alignas(16) float sA[2][kSgK][kSgTile];
    __shared__ alignas(16) float sW[2][kSgK][kSgTile];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = int64_t(blockIdx.x) * kSgTile;
    const int n0 = blockIdx.y * kSgTile;
    // this thread's share of a step's operands: row lr, columns 4 lq .. 4 lq + 3
    const int lr = threadIdx.x >> 1, lq = threadIdx.x & 1;
    const bool a_ok = m0 + lr < M, w_ok = n0 + lr < N;
    const float* a_src = A + (a_ok ? (m0 + lr) * lda : 0) + 4 * lq;
    const float* w_src = W + (w_ok ? int64_t(n0 + lr) * ldw : 0) + 4 * lq;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 ra = a_ok ? __ldg(reinterpret_cast<const float4*>(a_src)) : zero4;
    float4 rw = w_ok ? __ldg(reinterpret_cast<const float4*>(w_src)) : zero4;
    auto stage = [&](int buf) {
        sA[buf][4 * lq + 0][lr] = ra.x;
        sA[buf][4 * lq + 1][lr] = ra.y;
        sA[buf][4 * lq + 2][lr] = ra.z;
        sA[buf][4 * lq + 3][lr] = ra.w;
        sW[buf][4 * lq + 0][lr] = rw.x;
        sW[buf][4 * lq + 1][lr] = rw.y;
        sW[buf][4 * lq + 2][lr] = rw.z;
        sW[buf][4 * lq + 3][lr] = rw.w;
    };
    stage(0);
    __syncthreads();
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    const int steps = K / kSgK;
    for (int st = 0; st < steps; ++st) {
        const int buf = st & 1;
        if (st + 1 < steps) {   // next step's operands in flight during this one
            const int k1 = (st + 1) * kSgK;
            ra = a_ok ? __ldg(reinterpret_cast<const float4*>(a_src + k1)) : zero4;
            rw = w_ok ? __ldg(reinterpret_cast<const float4*>(w_src + k1)) : zero4;
        }
#pragma unroll
        for (int kk = 0; kk < kSgK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sA[buf][kk][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sA[buf][kk][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4*>(&sW[buf][kk][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4*>(&sW[buf][kk][64 + 4 * tx]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += a[i] * b[j];
        }
        if (st + 1 < steps) {
            stage(buf ^ 1);   // the other buffer was last read before the previous barrier
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t gm = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int gn = n0 + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
            if (gn >= N) continue;
            float z = scale[gn] * acc[i][j] + shift[gn];
            if (relu) z = z > 0.f ? z : 0.f;
            if (R) z += R[gm * ldr + gn];
            C[gm * ldc + gn] = z;
        }
    }
}

template <typename TA, typename TW, typename TC, typename TS>
cudaError_t launch_layer_simt(const TA* A, int64_t lda, const TW* W, int64_t ldw, const TS* scale,
                              const TS* shift, TC* C, int64_t ldc, const TA* R, int64_t ldr, int64_t M,
                              int N, int K, bool relu, cudaStream_t s) {
    if (K % 16) return cudaErrorInvalidValue;
    if (M == 0) return cudaSuccess;
    if constexpr (std::is_same<TA, float>::value && std::is_same<TW, float>::value &&
                  std::is_same<TC, float>::value && std::is_same<TS, float>::value) {
        if (lda % 4 == 0 && ldw % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0 &&
            (reinterpret_cast<uintptr_t>(W) & 15) == 0) {
            dim3 grid(unsigned((M + kSgTile - 1) / kSgTile), unsigned((N + kSgTile - 1) / kSgTile));
            layer_sgemm_kernel<<<grid, 256, 0, s>>>(A, lda, W, ldw, scale, shift, C, ldc, R, ldr, M, N, K,
                                                    relu ? 1 : 0);
            return cudaGetLastError();
        }
    }
    using TACC = typename AccOf<TS>::type;
    dim3 grid(unsigned((M + 63) / 64), unsigned((N + 63) / 64));
    layer_simt_kernel<TA, TW, TC, TS, TACC><<<grid, 256, 0, s>>>(A, lda, W, ldw, scale, shift, C, ldc, R, ldr,
                                                                  M, N, K, relu ? 1 : 0);
    return cudaGetLastError();
}

#define DNNMG_INST(T)                                                                                  \
    template cudaError_t launch_prolongate<T>(const DeviceMesh&, const T*, T*, cudaStream_t);         \
    template cudaError_t launch_residual<T>(const DeviceMesh&, OpParams, const T*, const T*, T*, T*,  \
                                            cudaStream_t, int*, cudaEvent_t);                         \
    template cudaError_t launch_extend<T>(const DeviceMesh&, const T*, T*, cudaStream_t);             \
    template cudaError_t launch_rhs_restrict<T>(const DeviceMesh&, OpParams, const T*, const T*, T*,  \
                                                T*, T*, T*, cudaStream_t, int*);
DNNMG_INST(double)
DNNMG_INST(float)
template cudaError_t launch_local_restrict<double, double>(const DeviceMesh&, const double*, const double*,
                                                           double*, cudaStream_t);
template cudaError_t launch_local_restrict<float, float>(const DeviceMesh&, const float*, const float*, float*,
                                                         cudaStream_t);
template cudaError_t launch_local_restrict<float, __nv_bfloat16>(const DeviceMesh&, const float*, const float*,
                                                                 __nv_bfloat16*, cudaStream_t);
template cudaError_t launch_layer_simt<double, double, double, double>(const double*, int64_t, const double*,
                                                                       int64_t, const double*, const double*,
                                                                       double*, int64_t, const double*, int64_t,
                                                                       int64_t, int, int, bool, cudaStream_t);
template cudaError_t launch_layer_simt<float, float, float, float>(const float*, int64_t, const float*, int64_t,
                                                                   const float*, const float*, float*, int64_t,
                                                                   const float*, int64_t, int64_t, int, int, bool,
                                                                   cudaStream_t);
template cudaError_t launch_layer_simt<__nv_bfloat16, __nv_bfloat16, __nv_bfloat16, float>(
    const __nv_bfloat16*, int64_t, const __nv_bfloat16*, int64_t, const float*, const float*, __nv_bfloat16*,
    int64_t, const __nv_bfloat16*, int64_t, int64_t, int, int, bool, cudaStream_t);
template cudaError_t launch_layer_simt<__nv_bfloat16, __nv_bfloat16, float, float>(
    const __nv_bfloat16*, int64_t, const __nv_bfloat16*, int64_t, const float*, const float*, float*, int64_t,
    const __nv_bfloat16*, int64_t, int64_t, int, int, bool, cudaStream_t);

}  // namespace dnnmg

// ---- residual without allocation -----------------------------------------------
// Callers that may not allocate device memory (a host application that owns
// every device allocation through its own pool, or code that must not call
// cudaMalloc once set-up is over) still need the fine residual.  This entry
// point takes every array from the caller and keeps the per-patch partial
// sums in a fixed array in the library's device image instead of a context
// buffer.
static __device__ __align__(256) float g_noalloc_partial[DNNMG_NOALLOC_MAX_PATCHES * 27 * 4];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
float* g_noalloc_addr[kMaxDevices] = {};

// Device address of g_noalloc_partial on the current device (looked up once
// per device; the host-side name is not a device address).
cudaError_t noalloc_scratch(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}
}  // namespace

extern "C" dnnmg_status dnnmg_residual_noalloc(int64_t n_patches, int64_t n_fine_nodes, const int32_t* cells_dev,
                                               const float* xyz_dev, const int32_t* node_ptr_dev,
                                               const int32_t* node_idx_dev, const uint8_t* fine_dirichlet_dev,
                                               double nu, double dt, double theta, const float* x_coarse_dev,
                                               const float* F_dev, float* r_dev, void* cuda_stream) {
    using namespace dnnmg;
    if (!cells_dev || !xyz_dev || !node_ptr_dev || !node_idx_dev || !fine_dirichlet_dev || !x_coarse_dev ||
        !F_dev || !r_dev || n_patches <= 0 || n_fine_nodes <= 0 || !(dt > 0.0) || !(nu >= 0.0) ||
        !(theta >= 0.0 && theta <= 1.0))
        return DNNMG_EINVAL;
    if (n_patches > DNNMG_NOALLOC_MAX_PATCHES) return DNNMG_EINVAL;   // beyond the fixed scratch
    for (const void* f : {static_cast<const void*>(x_coarse_dev), static_cast<const void*>(F_dev),
                          static_cast<const void*>(r_dev)})
        if (reinterpret_cast<uintptr_t>(f) % 16) return DNNMG_EINVAL;   // [n][4] rows move as 16 bytes
    float* partial = nullptr;
    if (noalloc_scratch(&partial) != cudaSuccess) return DNNMG_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    patch_operator_kernel<float, MODE_RESIDUAL, 1><<<blocks_for(n_patches, patches_per_block<1>()), kPatchThreads, 0, s>>>(
        n_patches, cells_dev, nullptr, xyz_dev, x_coarse_dev, nullptr, float(1.0 / dt), float(theta), float(nu),
        partial, nullptr);
    if (cudaGetLastError() != cudaSuccess) return DNNMG_ECUDA;
    node_reduce_kernel<float, MODE_RESIDUAL><<<blocks_for(n_fine_nodes, 256), 256, 0, s>>>(
        n_fine_nodes, node_ptr_dev, node_idx_dev, partial, fine_dirichlet_dev, F_dev, r_dev);
    return cudaGetLastError() == cudaSuccess ? DNNMG_OK : DNNMG_ECUDA;
}
