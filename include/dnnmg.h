/*
 * dnnmg.h -- C ABI of libdnnmg, the GB300 (sm_103a) patch-correction path of
 * the Deep Neural Network Multigrid method (DNN-MG).
 *
 * One DNN-MG time step (Sec. 5.1, Alg. 1) solves the coarse system on level L
 * and then runs the patch correction on level L+1:
 *
 *   x~   = P x^L                          prolongation           dnnmg_prolongate
 *   r    = F - A_{L+1}(x~)                fine residual, Eq. (9) dnnmg_residual
 *   X    = [Q(x~) | Q(r) | h^c]           local restriction,     dnnmg_local_restrict
 *                                         Eqs. (13)-(14) + the 12 edge lengths
 *   Y    = N(X)                           patch network, Sec. 4  dnnmg_network
 *   d    = L(Y) = mu . sum_P L(Y_P, P)    extension, Eq. (15)    dnnmg_extend
 *   b    = Rhs(v~ + d), b^L = R b         rhs of Eq. (6) on L+1, dnnmg_rhs_restrict
 *                                         restricted to level L
 *
 * dnnmg_patch_step runs all six in order on one CUDA stream.
 *
 * Conventions shared by every entry point
 *   - Every call returns a dnnmg_status; nothing throws across the ABI.
 *   - A context owns the mesh hierarchy (on the host and on the device), the
 *     network and its scratch buffers.  It is bound to the CUDA device that
 *     was current at dnnmg_create and to one stream; calls on one context
 *     must not overlap (the context is not thread-safe).
 *   - Field pointers named *_dev are device pointers owned by the caller and
 *     only borrowed for the call; *_host pointers are host memory.  Kernels
 *     are enqueued on the context's stream and the call returns without
 *     waiting, except where a function says it synchronises.
 *   - Field element type follows the context's precision:
 *       DNNMG_FP64: double fields, double network;
 *       DNNMG_FP32: float fields, float network;
 *       DNNMG_BF16: float fields, network input/activations bf16 with fp32
 *                   accumulation, network output float.
 *   - Layouts (row-major, node-major):
 *       x_coarse  [n_coarse_vertices][4]  (u, v, w, p) on level L
 *       x_fine, F, r, b_fine  [n_fine_nodes][4]
 *       d         [n_fine_nodes][3]       velocity correction
 *       b_coarse  [n_coarse_vertices][4]
 *       X         [n_patches][n_in_padded]: columns 0..107 x~ at the 27 patch
 *                 nodes (u,v,w,p), 108..215 r likewise (J = 2: 0..499 and
 *                 500..999 for the 125 nodes), then the
 *                 geometry features (12 edge lengths, or 24 features, see
 *                 dnnmg_params.features), zero after them
 *       Y         [n_patches][n_out]: 27 x (u, v, w) (J = 2: 125 x 3 = 375)
 *     Patch node iota = a + 3b + 9c, (a,b,c) in {0,1,2}^3 along the coarse
 *     cell's reference axes (J = 2: a + 5b + 25c, (a,b,c) in {0..4}^3).
 *   - Alignment of *_dev field pointers: [n][4] fields (x_coarse, x_fine,
 *     F, r, b_fine, b_coarse) to 4 elements (16 bytes in float, 32 in
 *     double), X to 16 bytes, d and Y to one element; DNNMG_EINVAL otherwise.
 *     Fresh allocations of cudaMalloc or torch meet all of them.
 *   - Dirichlet velocity rows (fine node kinds 1 and 2) of r, d and b_fine,
 *     and coarse Dirichlet velocity rows of b_coarse are zero; pressure rows
 *     of b_fine and b_coarse are zero.
 *   - Errors: DNNMG_EINVAL for null or inconsistent arguments (nothing is
 *     launched), DNNMG_ECUDA when a CUDA call fails (dnnmg_last_error has the
 *     CUDA message), DNNMG_ESTATE for calls out of order (e.g. dnnmg_network
 *     before dnnmg_set_network).
 */
#ifndef DNNMG_H
#define DNNMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DNNMG_ABI_VERSION 5

typedef struct dnnmg_ctx dnnmg_ctx;

typedef enum {
    DNNMG_OK = 0,
    DNNMG_EINVAL = -1,
    DNNMG_ENOMEM = -2,
    DNNMG_ECUDA = -3,
    DNNMG_ENOCONV = -4,
    DNNMG_ENAN = -5,
    DNNMG_ETIMEOUT = -6,
    DNNMG_ESTATE = -7,
    DNNMG_EUNSUPPORTED = -8
} dnnmg_status;

typedef enum { DNNMG_FP64 = 0, DNNMG_FP32 = 1, DNNMG_BF16 = 2 } dnnmg_precision;

/* Coarse mesh (level L).  Hexahedra with vertices in lexicographic order:
 * local vertex k sits at reference corner (k&1, (k>>1)&1, (k>>2)&1).
 * vertex_bc: 0 interior, 1 no-slip wall, 2 driven Dirichlet (lid/inflow),
 * 3 do-nothing outflow.  All arrays are copied by dnnmg_create. */
typedef struct {
    int32_t n_vertices;
    const double* xyz;             /* [n_vertices][3] */
    int32_t n_cells;
    const int32_t* cell_vertices;  /* [n_cells][8] */
    const int32_t* vertex_bc;      /* [n_vertices] */
} dnnmg_mesh_desc;

/* Time discretisation of Eq. (6) as a theta-scheme (theta = 1/2 is the
 * paper's Crank-Nicolson, theta = 1 backward Euler). */
typedef struct {
    double nu;          /* kinematic viscosity */
    double dt;          /* time step k */
    double theta;
    int32_t precision;  /* dnnmg_precision */
    int32_t features;   /* geometry features per patch in the network input
                         * (Sec. 5.2): 0 or 12 = the 12 edge lengths (228
                         * inputs); 24 = edge lengths, the 4 space diagonals
                         * (vertex k to 7 - k) and per vertex the mean of the
                         * 3 angles between the faces meeting there, in
                         * radians (240 inputs, as in Table 2) */
    int32_t patch_levels; /* J of Sec. 5.2: 0 or 1 = patches of one coarse
                           * cell refined once (27 nodes, level L+1); 2 =
                           * refined twice (125 nodes, level L+2, which is
                           * level L+1 refined again by the same rules).
                           * J = 2: n_in = 1000 + features, X row stride
                           * 1024, n_out = 375 (Table 2) */
    int32_t element;      /* 0 or 1 = Q1/Q1 on the refined mesh (27-node groups
                           * of 8 children, two-level projection); 2 = Q2/Q2,
                           * the paper's element (Sec. 3.2): triquadratic
                           * velocity and pressure with the one-level
                           * projection onto Q1 of each cell (Eq. (5)), 3 x 3
                           * x 3 Gauss points.  With Q2 the coarse level's
                           * unknowns sit at the nodes of the mesh refined
                           * once (n_coarse_nodes of dnnmg_sizes: x_coarse and
                           * b_coarse are [n_coarse_nodes][4]), the fine
                           * level's at the nodes of the mesh refined twice,
                           * and a patch is a coarse cell with those 125
                           * nodes: patch_levels must be 0 or 2 (the J = 2
                           * layout: n_in 1012 / 1024, n_out 375).  The fine
                           * level's projection terms use alpha0 = 0.02,
                           * delta0 = 0.1 (Eq. (8)). */
} dnnmg_params;

/* Patch network of Sec. 4 in inference form: layer i computes
 * z = scale_i . (W_i h) + shift_i; hidden layers apply ReLU and, when
 * skip != 0 and i >= 1 (0-based) and widths match, add their input. */
typedef struct {
    int32_t n_layers;        /* number of weight matrices, >= 1 */
    const int32_t* widths;   /* n_layers + 1 entries; widths[0] == n_in (228 or 240), widths[n_layers] == 81 */
    int32_t skip;
} dnnmg_net_desc;

typedef struct {
    int64_t n_coarse_vertices;
    int64_t n_patches;         /* = number of coarse cells */
    int64_t n_fine_nodes;
    int64_t n_coarse_edges;
    int64_t n_coarse_faces;
    int32_t n_in;              /* 8 x nodes per patch + geometry features: 228 / 240 (J = 1), 1012 / 1024 (J = 2) */
    int32_t n_in_padded;       /* row stride of X: 256 (J = 1), 1024 (J = 2) */
    int32_t n_out;             /* 3 x nodes per patch: 81 (J = 1), 375 (J = 2) */
    int32_t precision;
    int64_t n_coarse_nodes;    /* rows of x_coarse / b_coarse: n_coarse_vertices (Q1) or
                                * the nodes of the mesh refined once (Q2) */
    int32_t element;           /* 1 (Q1) or 2 (Q2) */
    int32_t reserved;
} dnnmg_sizes;

/* Mesh data a caller can read back (dnnmg_get_mesh_data). */
typedef enum {
    DNNMG_PATCH_MAP = 0,    /* int32 [n_patches][27 or 125]: dof(P, iota) of Sec. 5.2 */
    DNNMG_VALENCE = 1,      /* int32 [n_fine_nodes]: patches containing each node (1/mu) */
    DNNMG_FINE_KIND = 2,    /* int32 [n_fine_nodes]: boundary kind 0..3 */
    DNNMG_FINE_XYZ = 3,     /* double [n_fine_nodes][3] */
    DNNMG_EDGE_LENGTHS = 4, /* double [n_patches][12] */
    DNNMG_GEOMETRY = 5,     /* double [n_patches][12 or 24]: the geometry features of the input row */
    DNNMG_COARSE_XYZ = 6,   /* double [n_coarse_nodes][3]: the nodes of x_coarse (the mesh's
                             * vertices, or for Q2 the nodes of the mesh refined once) */
    DNNMG_COARSE_KIND = 7   /* int32 [n_coarse_nodes]: their boundary kinds 0..3 */
} dnnmg_mesh_item;

/* Build the level-(L+1) hierarchy of a coarse mesh on the host, upload it to
 * the current CUDA device and bind the context to `cuda_stream` (a
 * cudaStream_t; NULL = legacy default stream).  Fine nodes are numbered
 * hierarchically: coarse vertices, then one node per coarse edge, face and
 * cell in order of first appearance (cells in order; edges and faces in the
 * local order xi-, eta-, zeta-edges / xi=0, xi=1, eta=0, eta=1, zeta=0,
 * zeta=1 faces).  A coarse boundary face takes the lowest-priority kind of
 * its vertices (priority 3 < 1 < 2); a fine node on a boundary edge the
 * highest-priority kind of the boundary faces through it.
 * Errors: EINVAL (bad sizes, vertex index out of range, a boundary face with
 * an interior-marked vertex), ENOMEM, ECUDA.  On error *out is NULL. */
dnnmg_status dnnmg_create(const dnnmg_mesh_desc* mesh, const dnnmg_params* params,
                          void* cuda_stream, dnnmg_ctx** out);

/* Free every host and device resource of the context (NULL is a no-op).
 * Waits for the context's stream first. */
void dnnmg_destroy(dnnmg_ctx* ctx);

const char* dnnmg_strerror(dnnmg_status status);
/* Message of the last failing call on this context (static "" if none). */
const char* dnnmg_last_error(const dnnmg_ctx* ctx);

dnnmg_status dnnmg_get_sizes(const dnnmg_ctx* ctx, dnnmg_sizes* out);

/* Copy mesh data to host memory `host_buf` of `bytes` bytes (EINVAL if too
 * small). */
dnnmg_status dnnmg_get_mesh_data(const dnnmg_ctx* ctx, int32_t item, void* host_buf, size_t bytes);

/* The mesh hierarchy alone, built on the host with no CUDA call: the same
 * refinement, hierarchical fine numbering, patch map dof(P, iota) (Sec. 5.2),
 * valences mult_j (Eq. (15)), boundary kinds and geometry features that
 * dnnmg_create builds for its context.  It serves inspection and tests on
 * machines without a GPU.
 *   dnnmg_hierarchy_build    mesh as for dnnmg_create (copied); features
 *                            0 or 12 (edge lengths) or 24; patch_levels 0 or
 *                            1 (J = 1) or 2 (J = 2).  EINVAL for bad
 *                            arguments or an invalid mesh, ENOMEM.
 *   dnnmg_hierarchy_sizes    as dnnmg_get_sizes, precision = -1
 *   dnnmg_hierarchy_data     as dnnmg_get_mesh_data (items dnnmg_mesh_item)
 *   dnnmg_hierarchy_destroy  frees the handle (NULL is ignored)
 * The handle is immutable after build; concurrent reads are safe. */
typedef struct dnnmg_hierarchy dnnmg_hierarchy;
dnnmg_status dnnmg_hierarchy_build(const dnnmg_mesh_desc* mesh, int32_t features, int32_t patch_levels,
                                   dnnmg_hierarchy** out);
dnnmg_status dnnmg_hierarchy_sizes(const dnnmg_hierarchy* h, dnnmg_sizes* out);
dnnmg_status dnnmg_hierarchy_data(const dnnmg_hierarchy* h, int32_t item, void* host_buf, size_t bytes);
void dnnmg_hierarchy_destroy(dnnmg_hierarchy* h);

dnnmg_status dnnmg_set_stream(dnnmg_ctx* ctx, void* cuda_stream);

/* Load the patch network (Sec. 4).  W[i] points to widths[i+1] x widths[i]
 * doubles (row-major), scale[i] / shift[i] to widths[i+1] doubles (NULL =
 * 1 / 0).  Host memory; copied and converted to the context's precision.
 * Synchronises the stream.  Hidden widths need not be multiples of
 * anything: K is zero-padded to 64 (BF16) or 16 (FP32/FP64) internally.
 * Errors: EINVAL (widths[0] != n_in, widths[n_layers] != 81, a hidden
 * width outside [1, 4096]), ENOMEM, ECUDA. */
dnnmg_status dnnmg_set_network(dnnmg_ctx* ctx, const dnnmg_net_desc* net,
                               const double* const* W, const double* const* scale,
                               const double* const* shift);

/* Prolongation x~ = P x^L (Alg. 1): every fine node takes the mean of the
 * coarse vertex values of the entity it refines.
 * x_coarse_dev [n_coarse_vertices][4] -> x_fine_dev [n_fine_nodes][4]. */
dnnmg_status dnnmg_prolongate(dnnmg_ctx* ctx, const void* x_coarse_dev, void* x_fine_dev);

/* Training targets of Sec. 5.2 (the correction the network learns, used
 * with the loss of Sec. 6.4): for every patch P and patch node iota,
 *   T_dev[P * ldt + 3 iota + c] = v_fine[j][c] - (P x_coarse)[j][c],
 *   j = the fine node of (P, iota), c = 0..2 (velocity),
 * written in fp32.  x_coarse_dev [n_coarse_nodes][4] and v_fine_dev
 * [n_fine_nodes][4] are fields of the context's type (double for FP64,
 * float otherwise), aligned as for dnnmg_prolongate; P is the prolongation
 * of dnnmg_prolongate (the context's element); iota runs over the patch's
 * nodes (27 for J = 1, 125 for J = 2), so a row holds n_out values and
 * ldt >= n_out.  The first call allocates a fine-level scratch field
 * (ENOMEM if that fails).  EINVAL for NULL pointers, a network-only
 * context, ldt < n_out or a misaligned field; asynchronous on the
 * context's stream. */
dnnmg_status dnnmg_patch_targets(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* v_fine_dev, float* T_dev,
                                 int64_t ldt);

/* Fine residual r = F - A_{L+1}(P x^L) of Eq. (9), the Q1/Q1 Galerkin form
 * of Eq. (6) with 2x2x2 Gauss quadrature on every fine cell (fused with the
 * prolongation; the local projection terms vanish on prolongated fields and
 * are not evaluated).  Velocity rows at Dirichlet nodes are 0.
 * Deterministic: per-patch partial sums are reduced per node in patch
 * order.  Uses context scratch of n_patches*27*4 elements. */
dnnmg_status dnnmg_residual(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* F_dev,
                            void* r_dev);

/* Network input rows X = [Q(P x^L) | Q(r) | h^c] (Eqs. (13)-(14) and the
 * edge-length features of Sec. 5.2).  X_dev element type: double (FP64),
 * float (FP32), bf16 (BF16); row stride n_in_padded. */
dnnmg_status dnnmg_local_restrict(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* r_dev,
                                  void* X_dev);

/* Y = N(X) for n_rows rows (Sec. 4).  X_dev as produced by
 * dnnmg_local_restrict, Y_dev [n_rows][81] double (FP64) or float.
 * Errors: ESTATE before dnnmg_set_network, EINVAL if n_rows exceeds the
 * capacity fixed at dnnmg_set_network (max(n_patches, 1)). */
dnnmg_status dnnmg_network(dnnmg_ctx* ctx, const void* X_dev, void* Y_dev, int64_t n_rows);

/* Test of the failure path (the paper has no counterpart): dnnmg_network
 * with the first operand stage of the first layer armed but never filled
 * (BF16 tensor-core form only, else EUNSUPPORTED).  Every wait of the
 * tensor-core kernel is bounded (about one second), so the kernel gives up,
 * drains its copies, frees TMEM and returns; the following dnnmg_sync
 * reports DNNMG_ETIMEOUT and clears the error, and the context stays usable.
 * Takes a few seconds; Y holds no result. */
dnnmg_status dnnmg_network_wait_test(dnnmg_ctx* ctx, const void* X_dev, void* Y_dev, int64_t n_rows);

/* The same failure-path test through any entry point (the paper has no
 * counterpart): the next network launch of this context, whichever call
 * makes it (dnnmg_network, dnnmg_patch_step, dnnmg_patch_step_host,
 * dnnmg_time_step), withholds its first operand stage.  The calls that
 * synchronise (dnnmg_patch_step_host, dnnmg_time_step) then return
 * DNNMG_ETIMEOUT themselves; after an asynchronous call dnnmg_sync does.
 * The expiry is recorded in this context's own error word, so other
 * contexts on the device are not affected.  BF16 only, else EUNSUPPORTED. */
dnnmg_status dnnmg_arm_wait_test(dnnmg_ctx* ctx);

/* Extension d = mu . sum_P L(Y_P, P) of Eq. (15), mu = 1 / valence, summed
 * in patch order (deterministic, no atomics).  d_dev [n_fine_nodes][3];
 * zero at Dirichlet velocity nodes. */
dnnmg_status dnnmg_extend(dnnmg_ctx* ctx, const void* Y_dev, void* d_dev);

/* Right-hand side of Eq. (6) for the next step on level L+1 with the
 * corrected velocity P x^L + d (no force), and its restriction
 * b^L = P^T b to level L.  b_fine_dev [n_fine_nodes][4],
 * b_coarse_dev [n_coarse_vertices][4] (either may be NULL to skip it). */
dnnmg_status dnnmg_rhs_restrict(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* d_dev,
                                void* b_fine_dev, void* b_coarse_dev);

/* Restriction R = P^T of a fine vector to level L (Alg. 1, restriction of
 * the rhs): b_coarse = P^T b_fine with coarse Dirichlet velocity rows and
 * the pressure row zero (velocity components of b_fine are used).
 * b_fine_dev [n_fine_nodes][4], b_coarse_dev [n_coarse_vertices][4], field
 * type.  Deterministic (gathers in patch order). */
dnnmg_status dnnmg_restrict(dnnmg_ctx* ctx, const void* b_fine_dev, void* b_coarse_dev);

/* The whole patch correction of one time step: prolongate, residual with
 * F_dev, local restriction, network, extension, rhs and restriction.  r, X,
 * Y and d live in context buffers (readable with dnnmg_get_buffer).
 * b_fine_dev may alias F_dev (the step reads F before writing b).
 * Asynchronous: an expired bounded wait of the network (BF16) is reported
 * by the next dnnmg_sync as DNNMG_ETIMEOUT. */
dnnmg_status dnnmg_patch_step(dnnmg_ctx* ctx, const void* x_coarse_dev, const void* F_dev,
                              void* b_fine_dev, void* b_coarse_dev);

/* dnnmg_patch_step on host buffers: copies x_coarse and F to the device,
 * runs the step, copies b_fine and b_coarse back, and synchronises.  With
 * pinned host memory the copies are asynchronous: x_coarse goes on the
 * context's stream, F on a second stream of the context while the
 * residual's element kernel (which needs only x_coarse) runs, and the
 * gather that reads F waits for it.  b_fine_host or b_coarse_host may be
 * NULL (not copied back).  Returns DNNMG_ETIMEOUT if a bounded wait of the
 * network expired (the outputs are then not valid).  On any error the call
 * first waits for its copies, so the host buffers are free on return. */
dnnmg_status dnnmg_patch_step_host(dnnmg_ctx* ctx, const void* x_coarse_host, const void* F_host,
                                   void* b_fine_host, void* b_coarse_host);

typedef enum {
    DNNMG_BUF_R = 0,   /* [n_fine_nodes][4] residual of the last step */
    DNNMG_BUF_X = 1,   /* [n_patches][n_in_padded] network input */
    DNNMG_BUF_Y = 2,   /* [n_patches][81] network output */
    DNNMG_BUF_D = 3    /* [n_fine_nodes][3] correction */
} dnnmg_buffer;

/* Device pointer of a context buffer (valid until dnnmg_destroy). */
dnnmg_status dnnmg_get_buffer(dnnmg_ctx* ctx, int32_t which, void** dev_ptr);

/* Wait for the context's stream, polling at most timeout_us microseconds
 * (< 0: no limit).  ETIMEOUT if work is still pending then. */
dnnmg_status dnnmg_sync(dnnmg_ctx* ctx, int64_t timeout_us);

/* Number of kernel launches this context has issued (for accounting). */
int64_t dnnmg_launch_count(const dnnmg_ctx* ctx);

/* ---- Newton solve on a level and the DNN-MG time loop (Sec. 3.4, Alg. 1) ----
 *
 * Levels: DNNMG_LEVEL_COARSE is level L (the context's mesh), solved with the
 * two-level local projection when its cells come in consecutive groups of 8
 * children of a parent (else without it); DNNMG_LEVEL_FINE is the patches'
 * fine level, used as the fine-mesh reference: level L+1 for J = 1 (the
 * patches are its groups), level L+2 for J = 2 (one group per level-(L+1)
 * cell, 8 per patch, with its 27 level-(L+2) nodes; its multigrid passes
 * through levels L+1 and L, whose nodes are the first nodes of level L+2 in
 * the numbering of a J = 1 context on the same mesh, so the injection of a
 * level-(L+2) field onto level L+1 is its first n_fine(J = 1) rows).  Level fields are
 * double [n_nodes][4] (u, v, w, p) device arrays in every precision form.
 *
 * The solver: Newton with the exact Jacobian of A_h (stabilisation
 * parameters frozen, Sec. 3.4), re-assembled when the residual rate exceeds
 * rho_max; flexible restarted GMRES in FP64 (vectors, Gram-Schmidt, norms
 * and Givens rotations on the device), right-preconditioned by geometric
 * multigrid as in Sec. 3.4: a V-cycle over coarser levels with damped
 * additive group-Vanka smoothing (the 108 x 108 local problems of the
 * 27-node groups, LU-factorised) in FP32, and a dense LU with partial
 * pivoting in FP64 on the coarsest level.  The Jacobian is assembled in FP32
 * on the solve and smoothing levels and in FP64 on the coarsest.
 * Multigrid levels: each coarser level is made of the parents of the groups
 * of the level above, which needs a mesh whose cells come in groups of 8
 * children recursively and whose vertices are numbered coarsest level first
 * (level L+1 over level L always qualifies); mg_levels caps the depth, and
 * the hierarchy stops where a level cannot be coarsened or where the next
 * coarser level would have fewer than 8 nodes of free velocity (its
 * continuity rows would then see almost no velocity).  A coarsest level
 * without parents takes the stabilisation terms with full fluctuations (the
 * projection taken as zero).  With mg_levels = 0 the preconditioner is one
 * group-Vanka application. */
enum { DNNMG_LEVEL_COARSE = 0, DNNMG_LEVEL_FINE = 1 };

typedef struct {
    double alpha0, delta0;   /* local projection parameters of Eq. (8): 0.02, 0.1 */
    double newton_atol;      /* stop when |b - A(x)|_2 <= atol ... */
    double newton_rtol;      /* ... or <= rtol |b - A(x0)|_2 */
    int32_t newton_max;
    int32_t gmres_restart;   /* Krylov dimension per cycle (fixed at first use of a level) */
    int32_t gmres_max;       /* GMRES iterations per Newton step */
    int32_t mg_levels;       /* coarser multigrid levels below the solve level, at most
                              * (fixed at first use of a level); 0 = one-level Vanka */
    double gmres_rtol;
    double rho_max;          /* Jacobian re-assembly threshold, 0.1 or 0.05 in the paper */
    int32_t mg_pre, mg_post; /* Vanka sweeps before and after the coarse-grid correction */
    double mg_omega;         /* damping of the Vanka sweeps */
    int32_t mg_smoother;     /* 0 additive group-Vanka (local solutions averaged over the
                              * groups sharing a node); 1 multiplicative: groups in colours
                              * sharing no node, updated colour after colour (forward before,
                              * backward after the coarse-grid correction) */
    int32_t mg_bf16;         /* 1: the additive smoother reads bf16 copies of the level
                              * matrices and of the group inverses (half the bytes of its
                              * products; the Krylov products keep the FP32 matrix and
                              * Newton's residual stays FP64); 0: FP32.  The
                              * multiplicative smoother always uses FP32. */
} dnnmg_solver_params;

typedef struct {
    int32_t newton_iterations, gmres_iterations, jacobian_assemblies, converged;
    double residual0, residual;   /* l2 norms of b - A(x) at the start and the end */
} dnnmg_solve_stats;

/* Defaults: alpha0 0.02, delta0 0.1, atol 1e-11, rtol 1e-12, 25 Newton steps,
 * restart 40, 400 GMRES iterations, gmres_rtol 1e-10, rho_max 0.1,
 * mg_levels 0, 2 + 2 additive Vanka sweeps, damping 0.7, FP32 smoother
 * storage (mg_bf16 0). */
void dnnmg_solver_defaults(dnnmg_solver_params* p);

/* Number of nodes of a level and whether it uses the local projection. */
dnnmg_status dnnmg_level_info(dnnmg_ctx* ctx, int32_t level, int64_t* n_nodes, int32_t* grouped);

/* The multigrid hierarchy of a level as its solver built it (created with
 * prm's gmres_restart and mg_levels on first use): *n_levels = levels
 * including the solve level, nodes[k] = nodes of level k (0 = the solve
 * level, then coarser) for k < max_levels. */
dnnmg_status dnnmg_level_mg(dnnmg_ctx* ctx, int32_t level, const dnnmg_solver_params* prm, int32_t max_levels,
                            int32_t* n_levels, int64_t* nodes);

/* The same hierarchy on the host with no CUDA call (inspection and tests):
 * level 0 or 1 as above, at most mg_levels coarser levels. */
dnnmg_status dnnmg_hierarchy_mg(const dnnmg_hierarchy* h, int32_t level, int32_t mg_levels, int32_t max_levels,
                                int32_t* n_levels, int64_t* nodes);

/* A_h(x) of Eqs. (6), (9) on a level (no row modified).  x_dev, Ax_dev
 * double [n][4].  prm may be NULL (defaults). */
dnnmg_status dnnmg_level_operator(dnnmg_ctx* ctx, int32_t level, const dnnmg_solver_params* prm,
                                  const double* x_dev, double* Ax_dev);

/* Right-hand side of Eq. (6) on a level from the previous state x_old (no
 * force); Dirichlet velocity rows and pressure rows are 0. */
dnnmg_status dnnmg_level_rhs(dnnmg_ctx* ctx, int32_t level, const double* x_old_dev, double* b_dev);

/* The assembled Newton matrix at x as a dense row-major host array
 * [4n][4n] (rows of Dirichlet unknowns and of a pinned pressure are identity
 * rows).  For small levels: EINVAL if 4n > 8192 or bytes too small. */
dnnmg_status dnnmg_level_jacobian(dnnmg_ctx* ctx, int32_t level, const dnnmg_solver_params* prm,
                                  const double* x_dev, double* dense_host, size_t bytes);

/* Solve A_h(x) = b on a level by Newton's method.  x_dev holds the initial
 * guess and the Dirichlet values on entry, the solution on return.  Where no
 * boundary is do-nothing the pressure is normalised to zero mean.
 * Synchronises.  Returns ENOCONV (stats filled, x the last iterate) when the
 * Newton tolerance is not reached, ENAN on a non-finite residual. */
dnnmg_status dnnmg_solve(dnnmg_ctx* ctx, int32_t level, const dnnmg_solver_params* prm, const double* b_dev,
                         double* x_dev, dnnmg_solve_stats* stats);

/* n_steps DNN-MG time steps (Alg. 1): solve the coarse system with b_coarse,
 * then the patch correction with F (the previous fine rhs), which leaves the
 * next fine rhs in F and the next coarse rhs in b_coarse.
 *   x_coarse_dev double [n_coarse][4] (Dirichlet values set by the caller),
 *   b_coarse_dev double [n_coarse][4],
 *   F_dev        [n_fine][4] in the context's field type.
 * Requires dnnmg_set_network.  stats (may be NULL) are the last coarse solve's.
 * Synchronises after every step; returns DNNMG_ETIMEOUT at once if a bounded
 * wait of the network expired in that step (its correction is not valid). */
dnnmg_status dnnmg_time_step(dnnmg_ctx* ctx, int32_t n_steps, const dnnmg_solver_params* prm,
                             double* x_coarse_dev, double* b_coarse_dev, void* F_dev, dnnmg_solve_stats* stats);

/* One DNN-MG step in two halves, so that several contexts can share one
 * network launch (dnnmg_net_create) between them:
 *   dnnmg_step_begin: (solve != 0) the coarse solve with b_coarse, then the
 *     fine residual with F and the network input rows of this mesh into
 *     X_dev ([n_patches][n_in_padded], the context's X element type; may
 *     point into a larger shared buffer).  Returns ENOCONV if the coarse
 *     solve missed its tolerance (the step still proceeds).
 *   dnnmg_step_end: extension of Y_dev ([n_patches][81], the context's Y
 *     type; may point into a shared buffer), then the next fine rhs into
 *     F_dev and its restriction into b_coarse_dev (double).
 * dnnmg_time_step = begin, dnnmg_network on the context's buffers, end. */
dnnmg_status dnnmg_step_begin(dnnmg_ctx* ctx, const dnnmg_solver_params* prm, int32_t solve, double* x_coarse_dev,
                              const double* b_coarse_dev, const void* F_dev, void* X_dev, dnnmg_solve_stats* stats);
dnnmg_status dnnmg_step_end(dnnmg_ctx* ctx, const void* Y_dev, void* F_dev, double* b_coarse_dev);

/* A network-only context for serving: no mesh (the input width, 228 or 240,
 * is widths[0]); supports dnnmg_network (up
 * to max_rows rows), dnnmg_set_network, dnnmg_set_stream, dnnmg_sync,
 * dnnmg_launch_count, dnnmg_destroy; every call that needs a mesh returns
 * DNNMG_EINVAL on it.  Weights as in dnnmg_set_network.  The context
 * allocates its activations for max_rows rows once; the caller owns X and Y. */
dnnmg_status dnnmg_net_create(const dnnmg_net_desc* net, const double* const* W, const double* const* scale,
                              const double* const* shift, int32_t precision, int64_t max_rows, void* cuda_stream,
                              dnnmg_ctx** out);

/* n_steps of the plain scheme on one level (no network): b = Rhs(x_old),
 * solve A(x) = b.  x_dev double [n][4]. */
dnnmg_status dnnmg_plain_step(dnnmg_ctx* ctx, int32_t level, int32_t n_steps, const dnnmg_solver_params* prm,
                              double* x_dev, dnnmg_solve_stats* stats);

/* ---- Training of the patch network (Sec. 4; loss and optimiser, Sec. 6.4) ----
 *
 * Training form of the network: hidden layer i computes relu(W_i h + b_i)
 * (+ h where the skip applies), the last layer W_L h; the per-feature bias
 * b_i stands for the normalisation of Sec. 4 (at inference it is the shift
 * of dnnmg_set_network).  Weights and biases are caller-owned fp32 device
 * arrays, W_i row-major [widths[i+1]][widths[i]], b_i [widths[i+1]].
 * A trainer owns the saved activations of the last forward pass and the
 * backward workspace for up to max_batch rows (a multiple of 64).
 * Precision DNNMG_BF16: bf16 operands, fp32 accumulation (tensor cores);
 * DNNMG_FP32: float throughout.  Input rows X as dnnmg_local_restrict writes
 * them for a context of that precision: [batch][256], bf16 or float. */
typedef struct dnnmg_trainer dnnmg_trainer;

dnnmg_status dnnmg_trainer_create(const dnnmg_net_desc* net, int32_t precision, int64_t max_batch, void* cuda_stream,
                                  dnnmg_trainer** out);
void dnnmg_trainer_destroy(dnnmg_trainer* trainer);

/* Y_dev [batch][81] fp32 = N(X) with the given weights; saves what the
 * backward pass needs.  batch a multiple of 64, <= max_batch.  X_dev is
 * read again by dnnmg_trainer_backward (first-layer weight gradient): it
 * must stay valid and unchanged until then. */
dnnmg_status dnnmg_trainer_forward(dnnmg_trainer* trainer, const void* X_dev, const float* const* W_dev,
                                   const float* const* b_dev, float* Y_dev, int64_t batch);

/* Gradients of sum(dY . Y) with respect to every W_i and b_i for the last
 * forward pass (reverse-mode through the layers): dW_dev[i] and db_dev[i]
 * are overwritten.  ESTATE without a forward pass. */
dnnmg_status dnnmg_trainer_backward(dnnmg_trainer* trainer, const float* dY_dev, float* const* dW_dev,
                                    float* const* db_dev);

/* The l2 loss of Sec. 6.4 for one batch: loss = (1/batch) sum_P ||Y_P - T_P||^2
 * (into loss_dev[0]) and dY = 2 (Y - T) / batch (dY_dev may be NULL);
 * Y, T [batch][81] fp32. */
dnnmg_status dnnmg_mse_loss(int64_t batch, const float* Y_dev, const float* T_dev, float* loss_dev, float* dY_dev,
                            void* cuda_stream);

/* One AdamW step (decoupled weight decay, bias-corrected moments, step >= 1)
 * on n parameters w with gradient g and moments m, v (all fp32 device).
 * Hyperparameters in double: 1 - beta and the bias corrections 1 - beta^step
 * are formed in double and rounded once to fp32 for the update. */
dnnmg_status dnnmg_adamw(int64_t n, float* w_dev, const float* g_dev, float* m_dev, float* v_dev, double lr,
                         double beta1, double beta2, double eps, double weight_decay, int32_t step, void* cuda_stream);

/* Training data (Sec. 6.4: inputs standardised per feature, batches drawn
 * at random from the sample set).  Matrices are row-major device arrays,
 * row stride ld elements (ld >= cols); dtype is DNNMG_FP64 (double),
 * DNNMG_FP32 (float) or DNNMG_BF16 (bf16 storage).  All three calls are
 * asynchronous on cuda_stream (NULL: the legacy default stream) and return
 * EINVAL for NULL pointers, bad sizes or an unknown dtype, ECUDA if a
 * launch fails.
 *
 * dnnmg_column_stats: mean_dev[j] = (1/rows) sum_i A[i][j] and sd_dev[j] =
 * sqrt(sum_i (A[i][j] - mean_j)^2 / (rows - 1)) for j < cols (double device
 * arrays), accumulated in FP64 over a fixed partition of the rows (mean
 * first, then the deviations), so equal inputs give equal bits.  rows >= 2.
 * Uses stream-ordered scratch of 512 x cols doubles (ENOMEM if it fails). */
dnnmg_status dnnmg_column_stats(const void* A_dev, int32_t dtype, int64_t rows, int32_t cols, int64_t ld,
                                double* mean_dev, double* sd_dev, void* cuda_stream);

/* dnnmg_standardize: B[i][j] = (A[i][j] - shift[j]) / scale[j] for j < cols
 * (shift, scale: double device arrays [cols]), computed in float for float
 * and bf16 data and in double for double data, rounded once to the dtype;
 * B has A's dtype and stride and may be A itself.  Columns >= cols of B are
 * not written. */
dnnmg_status dnnmg_standardize(const void* A_dev, int32_t dtype, int64_t rows, int32_t cols, int64_t ld,
                               const double* shift_dev, const double* scale_dev, void* B_dev, void* cuda_stream);

/* dnnmg_gather_rows: row i of dst = row idx[i] of src for i < n, rows of
 * row_bytes bytes, packed in both (idx: int64 device array).  An index
 * outside [0, n_src) gives a zero row instead of a read.  src and dst must
 * not overlap. */
dnnmg_status dnnmg_gather_rows(const void* src_dev, int64_t n_src, int64_t row_bytes, const int64_t* idx_dev,
                               int64_t n, void* dst_dev, void* cuda_stream);

/* dnnmg_add_noise: A[i][j] += sigma z_ij for c0 <= j < c1 (in place), z_ij
 * standard normal from a counter-based generator: SplitMix64 of (seed, i,
 * j), two uniforms, the Box-Muller transform; the same seed gives the same
 * bits.  Training-time input noise (the paper has no counterpart): inputs
 * perturbed while targets stay the reference's teach the network not to
 * amplify errors that the time loop feeds back into its inputs.  Computed
 * in float (double for double data), rounded once to the dtype.  EINVAL
 * for c0 > c1, c1 > ld or sigma < 0. */
dnnmg_status dnnmg_add_noise(void* A_dev, int32_t dtype, int64_t rows, int32_t c0, int32_t c1, int64_t ld,
                             double sigma, uint64_t seed, void* cuda_stream);

/* Measured peak of the SIMT fused multiply-add pipe on the current device
 * (the paper has no counterpart: a roofline denominator for the kernels
 * bound by FP32 or FP64 arithmetic).  Every thread of blocks_per_sm x (SM
 * count) blocks of 256 threads runs 8 independent FMA chains for `iters`
 * rounds; the best of 3 timed launches after a warm-up, 2 flop per FMA,
 * is returned in *tflops.  precision DNNMG_FP32 or DNNMG_FP64.  Allocates a
 * small device buffer, a stream and two events, and synchronises. */
dnnmg_status dnnmg_probe_fma(int32_t precision, int32_t iters, int32_t blocks_per_sm, double* tflops);

/* Largest mesh dnnmg_residual_noalloc accepts (coarse cells = patches);
 * the Python binding's NOALLOC_MAX_PATCHES must equal it (a CPU test reads
 * this line). */
#define DNNMG_NOALLOC_MAX_PATCHES 16384

/* dnnmg_residual without any allocation, for callers that may not allocate
 * device memory: a host application that hands out all device memory from
 * its own pool, or a program that must not call cudaMalloc after set-up.
 * The paper has no counterpart; this is a packaging of the same FP32
 * residual kernels (prolongation fused with the Q1 element integrals, then
 * the per-node reduction in patch order), with every array supplied by the
 * caller and the per-patch partial sums (n_patches x 27 x 4 floats) kept in
 * one fixed array of DNNMG_NOALLOC_MAX_PATCHES x 27 x 4 floats (6.75 MiB)
 * that the library's device image holds on every GPU that loads it, until
 * the process exits.  No context is needed; nothing is allocated or freed.
 *
 * Arguments (device pointers, caller-owned, FP32 form only):
 *   cells_dev          int32 [n_patches][8]   coarse cells (lexicographic vertices)
 *   xyz_dev            float [n_coarse_vertices][3]
 *   node_ptr_dev       int32 [n_fine_nodes + 1] and
 *   node_idx_dev       int32 [27 n_patches]: for fine node j the entries
 *                      P*27 + iota with patch_map[P][iota] == j, sorted by P
 *   fine_dirichlet_dev uint8 [n_fine_nodes]: 1 where the velocity is prescribed
 *   x_coarse_dev       float [n_coarse_vertices][4], F_dev float [n_fine_nodes][4]
 *   r_dev              float [n_fine_nodes][4] (output)
 *   nu, dt, theta      as in dnnmg_params; cuda_stream a cudaStream_t (NULL = default)
 * The index arrays are trusted as given: nothing checks them (unlike
 * dnnmg_create, which validates a mesh).  cells_dev entries must be vertex
 * ids in [0, n_coarse_vertices), node_ptr_dev must be non-decreasing from 0
 * to 27 n_patches, and node_idx_dev entries must lie in [0, 27 n_patches);
 * an entry outside these ranges reads partial sums of an earlier call or
 * memory outside the arrays.
 * The first call on a device looks up the fixed array's device address
 * (cudaGetSymbolAddress, once per device, under a lock) and keeps it for
 * the life of the process; make that first call before any stream capture.
 * A cudaDeviceReset reloads the library's device image at a possibly
 * different address, so after one this entry point must not be called on
 * that device again in the same process.  Every call uses the same array, whose
 * contents persist between calls; each call overwrites all partial sums it
 * reads, so nothing has to be cleared, but calls that overlap on the GPU
 * (two streams, two threads) race on it.
 * Errors: DNNMG_EINVAL for a null pointer, non-positive size, bad
 * nu/dt/theta, x_coarse_dev, F_dev or r_dev not 16-byte aligned, or
 * n_patches > DNNMG_NOALLOC_MAX_PATCHES (nothing is launched); DNNMG_ECUDA if the address lookup or a launch fails. */
dnnmg_status dnnmg_residual_noalloc(int64_t n_patches, int64_t n_fine_nodes, const int32_t* cells_dev,
                                    const float* xyz_dev, const int32_t* node_ptr_dev,
                                    const int32_t* node_idx_dev, const uint8_t* fine_dirichlet_dev,
                                    double nu, double dt, double theta, const float* x_coarse_dev,
                                    const float* F_dev, float* r_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* DNNMG_H */
