// Internal declarations of libdnnmg (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dnnmg.h"

namespace dnnmg {

constexpr int kNodes = 27;     // fine nodes per patch
constexpr int kNIn = 228;      // network inputs per patch with the 12 edge lengths
constexpr int kNInGeo24 = 240; // with the 24 geometry features (edges, diagonals, angles)
constexpr int kNInPad = 256;   // row stride of X (J = 1)
constexpr int kNInPadJ2 = 1024;  // row stride of X for J = 2: 2 x 125 x 4 + 24 = 1024
constexpr int kNOutJ2 = 375;   // network outputs per patch for J = 2 (125 x 3)
constexpr int kNOut = 81;      // network outputs per patch

// Level L+1 of a coarse mesh and the patch data, built on the host.
struct HostHierarchy {
    int64_t nv = 0, nc = 0, ne = 0, nf = 0, n_fine = 0;
    std::vector<double> xyz_c;       // [nv][3]
    std::vector<int32_t> cells;      // [nc][8]
    std::vector<int32_t> bc_c;       // [nv]
    std::vector<int32_t> patch_map;  // [nc][27]
    std::vector<int32_t> kind_f;     // [n_fine]
    std::vector<int32_t> valence;    // [n_fine]
    std::vector<double> xyz_f;       // [n_fine][3]
    int J = 1;                       // refinement levels per patch (1 or 2)
    int npn = 27;                    // nodes per patch (27, 125)
    int n_geo = 12;                  // geometry features per patch: 12 or 24
    int element = 1;                 // 1 (Q1) or 2 (Q2: J = 2 layout, coarse unknowns at level L+1)
    std::vector<double> geo;         // [nc][n_geo]: 12 edge lengths (+ 4 diagonals, 8 mean dihedral angles)
    std::vector<int32_t> node_ptr, node_idx;   // fine node -> P*27+iota, patch order
    std::vector<int32_t> vert_ptr, vert_idx;   // coarse vertex -> P*8+k, patch order
    // J = 2: level L+1 kept beside level L+2 (the coarse Q2 level's nodes are
    // level L+1's, a coarse cell's 27 of them in patch_map_mid)
    int64_t n_mid = 0;
    std::vector<int32_t> patch_map_mid;        // [nc][27]
    std::vector<int32_t> kind_mid;             // [n_mid]
    std::vector<double> xyz_mid;               // [n_mid][3]
    std::vector<int32_t> mid_ptr, mid_idx;     // level L+1 node -> P*27+iota, patch order
};

// Level L+J (J = 1 or 2) of a coarse mesh and its patches; level L+2 is
// level L+1 refined once more by the same rules.
dnnmg_status build_hierarchy(const dnnmg_mesh_desc* mesh, int n_geo, int J, HostHierarchy* h, std::string* err);

// One mesh level for the Newton solve: cells in groups of 8 children of a
// parent (27 nodes per group), which is the structure the two-level local
// projection needs.  Level L+1 is always grouped (the patches); level L is
// grouped when its cells come in such groups (else it is solved as 1-cell
// "groups" without the projection terms).
struct HostLevel {
    int64_t n = 0;                   // nodes
    int64_t ng = 0;                  // groups
    int npg = 27;                    // nodes per group (27, or 8 without grouping)
    bool lps = true;
    bool mean_zero_pressure = false; // no do-nothing boundary: pressure up to a constant
    int32_t pin = -1;                // node whose pressure row is pinned (mean-zero case)
    std::vector<int32_t> groups;     // [ng][npg]
    std::vector<double> xyz;         // [n][3]
    std::vector<uint8_t> dir;        // [n] Dirichlet velocity
    std::vector<int32_t> node_ptr, node_idx;   // node -> g*npg + local, group order
    std::vector<int32_t> row_ptr, col_idx;     // node-node block sparsity (BSR, 4x4 blocks)
    std::vector<int32_t> blk_ptr, blk_src;     // block -> local entries g*npg*npg + i*npg + j
    std::vector<int32_t> grp_blk;              // [ng][npg][npg] block index
    std::vector<int32_t> color_ptr, color_groups;  // groups by colour: no two of a colour share a node
    bool q2 = false;                 // groups are Q2 cells (27 nodes, one element) instead of 8 Q1 children
};

// Level L from the coarse mesh (grouped if its cells come in consistent
// groups of 8) or level L+1 from the hierarchy.
void build_level(const HostHierarchy& h, bool fine, HostLevel* lv);

// Grid transfer between a level and the next coarser one: P (rows = fine
// nodes, trilinear weights of the parent's corners) and R = P^T (rows =
// coarse nodes, entries in increasing fine node order).
constexpr int64_t kMinFreeCoarseNodes = 8;

struct MgTransfer {
    std::vector<int32_t> P_ptr, P_idx, R_ptr, R_idx;
    std::vector<double> P_w, R_w;
};

// The next coarser level of a grouped level for geometric multigrid: the
// parents of its groups, whose corners must be nodes 0 .. n_c - 1 (meshes
// numbered coarsest level first; level L+1 of a hierarchy always is), with
// at least kMinFreeCoarseNodes nodes of free velocity.  False if the level
// cannot be coarsened.
bool coarsen_level(const HostLevel& fine, HostLevel* coarse, MgTransfer* t);

struct OpParams;
struct DeviceLevel;   // solver.cu
// The level solved on (level L, or L+1 when fine) with up to mg_levels
// coarser multigrid levels below it and a Krylov dimension of krylov.
cudaError_t create_level(const HostHierarchy& hh, bool fine, int krylov, int mg_levels, DeviceLevel** out);
void destroy_level(DeviceLevel* L);
int64_t level_nodes(const DeviceLevel* L);
bool level_lps(const DeviceLevel* L);
int level_mg_depth(const DeviceLevel* L);                // coarser levels in use
int64_t level_mg_nodes(const DeviceLevel* L, int k);     // nodes of level k (0 = the solve level)
cudaError_t level_operator(DeviceLevel* L, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                           double* Ax, cudaStream_t s);
cudaError_t level_residual(DeviceLevel* L, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                           const double* b, double* r, cudaStream_t s);
cudaError_t level_rhs(DeviceLevel* L, const OpParams& op, const double* x_old, double* b, cudaStream_t s);
cudaError_t level_jacobian(DeviceLevel* L, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                           cudaStream_t s);
cudaError_t level_dense_jacobian(DeviceLevel* L, const OpParams& op, const dnnmg_solver_params* sp, const double* x,
                                 double* dense_host, cudaStream_t s);
cudaError_t level_solve(DeviceLevel* L, const OpParams& op, const dnnmg_solver_params* sp, const double* b, double* x,
                        cudaStream_t s, dnnmg_solve_stats* st);

// Device view of a Q2 level (q2.cu): cells of 27 nodes (local node
// a + 3 b + 9 c), the node -> (cell, local) CSR in cell order, node
// coordinates (double) and Dirichlet velocity flags.
struct Q2Level {
    int64_t n = 0, ncell = 0;
    const int32_t* cells = nullptr;      // [ncell][27]
    const int32_t* node_ptr = nullptr;   // [n+1]
    const int32_t* node_idx = nullptr;   // [27 ncell]: cell * 27 + local
    const double* xyz = nullptr;         // [n][3]
    const uint8_t* dir = nullptr;        // [n]
};

// Device copy of the mesh data the kernels read.
struct DeviceMesh {
    int64_t nv = 0, nc = 0, n_fine = 0;
    const int32_t* cells = nullptr;      // [nc][8]
    const int32_t* patch_map = nullptr;  // [nc][27]
    const int32_t* node_ptr = nullptr;   // [n_fine+1]
    const int32_t* node_idx = nullptr;   // [27 nc]
    const int32_t* vert_ptr = nullptr;   // [nv+1]
    const int32_t* vert_idx = nullptr;   // [8 nc]
    const uint8_t* fine_dir = nullptr;   // [n_fine] 1 = Dirichlet velocity
    const uint8_t* coarse_dir = nullptr; // [nv]
    const double* xyz_d = nullptr;       // [nv][3] double
    const float* xyz_f = nullptr;        // [nv][3] float
    int J = 1;                           // refinement levels per patch
    int n_geo = 12;                      // geometry features per patch
    const double* geo_d = nullptr;       // [nc][n_geo]
    const float* geo_f = nullptr;        // [nc][n_geo]
    // Q2 elements (J = 2 layout): coarse Q2 nodes = level L+1 nodes
    int element = 1;                     // 1 (Q1) or 2 (Q2)
    int64_t n_mid = 0;
    const int32_t* patch_map_mid = nullptr;   // [nc][27] level L+1 nodes of each coarse cell
    const int32_t* mid_ptr = nullptr;         // [n_mid+1]
    const int32_t* mid_idx = nullptr;         // [27 nc] P*27+m, patch order
    const uint8_t* mid_dir = nullptr;         // [n_mid]
    Q2Level q2fine;                           // the fine Q2 level (level L+2 nodes, 8 cells per patch)
};

// ---- Q2 kernels (q2.cu); T = double or float; mode 0 operator, 1 rhs, 2 mass
template <typename T>
cudaError_t q2_level_local(const Q2Level& L, int mode, const T* x, const T* d, OpParams op, double a0, double d0,
                           int lps, T* local, cudaStream_t s);
template <typename T>
cudaError_t q2_gather(const Q2Level& L, int mode, const T* local, const T* F, T* out, cudaStream_t s);
template <typename T>
cudaError_t q2_prolongate(const DeviceMesh& dm, const T* xc, T* xf, cudaStream_t s);
template <typename T>
cudaError_t q2_restrict(const DeviceMesh& dm, const T* b_fine, T* part, T* b_coarse, cudaStream_t s);
template <typename T, typename TX>
cudaError_t q2_local_restrict(const DeviceMesh& dm, const T* xf, const T* r, const T* geo, int ld, TX* X,
                              cudaStream_t s);

struct OpParams {
    double m;      // 1 / dt
    double theta;
    double nu;
};


// ---- patch kernels (kernels.cu); T = double or float -------------------
template <typename T>
cudaError_t launch_prolongate(const DeviceMesh& dm, const T* xc, T* xf, cudaStream_t s);
template <typename T>
cudaError_t launch_targets(const DeviceMesh& dm, int npn, const T* v, const T* xt, float* out, int64_t ldt,
                           cudaStream_t s);
// F_ready (may be null): an event the gather waits for before reading F,
// so that F can still be arriving while the element kernel runs
template <typename T>
cudaError_t launch_residual(const DeviceMesh& dm, OpParams p, const T* xc, const T* F, T* r,
                            T* partial, cudaStream_t s, int* launches, cudaEvent_t F_ready = nullptr);
template <typename T, typename TX>
cudaError_t launch_local_restrict(const DeviceMesh& dm, const T* xc, const T* r, TX* X,
                                  cudaStream_t s);
template <typename T>
cudaError_t launch_extend(const DeviceMesh& dm, const T* Y, T* d, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict(const DeviceMesh& dm, const T* b_fine, T* b_coarse, T* partial_c, cudaStream_t s);
template <typename T>
cudaError_t launch_rhs_restrict(const DeviceMesh& dm, OpParams p, const T* xc, const T* d,
                                T* b_fine, T* b_coarse, T* partial, T* partial_c,
                                cudaStream_t s, int* launches);

// ---- network layers -------------------------------------------------------
// C[M][N] (row stride ldc) = epilogue(A[M][K] (lda) * W[N][K]^T):
//   z = scale[n] * acc + shift[n]; relu if `relu`; + R[m][n] (ldr) if R != null.
template <typename TA, typename TW, typename TC, typename TS>
cudaError_t launch_layer_simt(const TA* A, int64_t lda, const TW* W, int64_t ldw,
                              const TS* scale, const TS* shift, TC* C, int64_t ldc,
                              const TA* R, int64_t ldr, int64_t M, int N, int K, bool relu,
                              cudaStream_t s);

}  // namespace dnnmg

// The context behind the opaque handle.
struct dnnmg_ctx {
    dnnmg::HostHierarchy host;
    dnnmg::DeviceMesh dm;
    int device = 0;
    int precision = DNNMG_FP64;
    dnnmg::OpParams op{};
    cudaStream_t stream = nullptr;
    std::string last_error;
    int64_t launches = 0;
    std::vector<void*> allocations;   // freed at destroy

    // scratch and step buffers (element type by precision)
    void* partial = nullptr;     // [nc][27][4]
    void* partial_c = nullptr;   // [nc][8][4]
    void* buf_r = nullptr;       // [n_fine][4]
    void* buf_X = nullptr;       // [nc][kNInPad]
    void* buf_Y = nullptr;       // [nc][81]
    void* buf_d = nullptr;       // [n_fine][3]
    void* buf_xc = nullptr;      // [nv][4]  (host-buffer step)
    void* buf_F = nullptr;       // [n_fine][4]
    void* buf_bc = nullptr;      // [nv][4]
    cudaStream_t copy_stream = nullptr;   // host-buffer step: F upload beside the element kernel
    cudaEvent_t ev_ready = nullptr, ev_input = nullptr;

    // network
    bool has_net = false;
    int n_layers = 0;
    int skip = 0;
    std::vector<int> widths;     // true widths
    std::vector<int> kpad;       // padded K per layer (input width as stored)
    std::vector<int> npad;       // padded N per layer (rows of stored W)
    std::vector<void*> W;        // per layer [npad][kpad] in the weight dtype
    std::vector<void*> scale, shift;  // per layer [npad] (double for FP64 else float)
    void* act[2] = {nullptr, nullptr};  // [nc][max width] activations
    int64_t act_rows = 0;
    int act_ld = 0;
    int64_t net_capacity = 0;    // rows of a network-only context (no mesh)
    bool net_only = false;
    const void* last_xc = nullptr;   // coarse state (field type) of the last dnnmg_step_begin
    int* tc_err = nullptr;           // device word: a tensor-core wait of this context expired
    int wait_test_armed = 0;         // the next network launch withholds its first operand stage

    // Newton solver levels (0: L, 1: L+1), created on first use
    dnnmg::DeviceLevel* level[2] = {nullptr, nullptr};
    void* xc_field = nullptr;   // [nv][4] x^L in the field type (time stepping)
    void* bc_field = nullptr;   // [nv][4] b^L in the field type
    void* plain_b[2] = {nullptr, nullptr};   // [n][4] double rhs of dnnmg_plain_step per level
    void* buf_xf = nullptr;      // Q2: [n_fine][4] prolongated field
    void* q2_local = nullptr;    // Q2: [8 nc][27][4] rows of the fine cells
};

namespace dnnmg {
// tcgen05 BF16 layer (tc_gemm.cu): C = epilogue(A W^T), see launch_layer_simt.
cudaError_t launch_layer_tc(const __nv_bfloat16* A, int64_t lda, const __nv_bfloat16* W, int64_t ldw, int n_rows_w,
                            const float* scale, const float* shift, void* C, int64_t ldc, bool out_bf16,
                            const __nv_bfloat16* R, int64_t ldr, int64_t M, int N, int K, bool relu,
                            cudaStream_t s, int* err, int withhold_first_load = 0);
// Error code that a tensor-core kernel whose bounded wait expired recorded
// in the device word err (0 = none); reading clears it.  Synchronises s.
cudaError_t read_tc_error(int* err, cudaStream_t s, int* code);
}  // namespace dnnmg
