/*
 * lor.h -- C ABI of the GB300 LOR-preconditioned matrix-free Poisson solver.
 *
 * Method: Pazner, "Efficient low-order refined preconditioners for high-order
 * matrix-free continuous and discontinuous Galerkin methods" (arXiv:1908.07071).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns lor_status; on failure lor_last_error(ctx) returns a
 *    message owned by the context, valid until the next call on that context.
 *  - Mesh: a structured-topology tensor mesh of nx*ny(*nz) elements, each the
 *    multilinear image of [0,1]^d of its 2^d vertices (Section 2).  Vertex
 *    coordinates are SoA float64: component c of vertex (i,j,k) at
 *    vertices[c*NV + (k*(ny+1)+j)*(nx+1)+i], NV = (nx+1)(ny+1)(nz+1).
 *    kappa[(ez*ny+ey)*nx+ex] > 0 is the piecewise-constant coefficient b of
 *    Eq. (poisson) (lor_set_coefficient replaces it by a pointwise b(x)).
 *    Both are host or device pointers, copied by lor_create.
 *  - CG vectors ("L-vectors"): float64 (or float32 where a call says so) on
 *    the full Q_p node grid Nx*Ny(*Nz), N = p*n+1 per direction, x fastest:
 *    node (I,J,K) at (K*Ny+J)*Nx+I.  Boundary (Dirichlet) entries of inputs are
 *    ignored; those of outputs are written as 0.  Vector pointers are DEVICE
 *    pointers owned by the caller, unless the name ends in _host.
 *  - DG vectors: element-major blocks of (p+1)^d GLL-nodal values, element e
 *    at offset e*(p+1)^d, node (i,j,k) of the block at (k*(p+1)+j)*(p+1)+i.
 *  - Work runs on the stream given to lor_create (NULL = legacy default
 *    stream).  Calls after lor_setup allocate no memory.
 */
#ifndef LOR_H
#define LOR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LOR_OK = 0,
  LOR_EINVAL = 1,      /* bad argument, inverted element, unsupported size   */
  LOR_ENOMEM = 2,      /* device allocation failed                           */
  LOR_ECUDA = 3,       /* a CUDA runtime call or launch failed               */
  LOR_EBREAKDOWN = 4,  /* ILU(0) met a non-positive pivot (no shifting)      */
  LOR_ENAN = 5,        /* NaN/Inf or p.Ap <= 0 in the Krylov recurrences     */
  LOR_ENOCONV = 6,     /* max_it reached before rtol                        */
  LOR_ETIMEOUT = 7,    /* a bounded device wait ran out                     */
  LOR_ESTATE = 8       /* call out of order (e.g. apply before setup)       */
} lor_status;

typedef enum { LOR_CG = 0, LOR_DG_IP = 1, LOR_DG_BR2 = 2 } lor_disc;
typedef enum { LOR_FP64 = 0, LOR_FP32 = 1, LOR_MIXED = 2 } lor_prec;

typedef struct lor_ctx lor_ctx;

typedef struct {
  int dim;          /* 2 or 3                                                  */
  int p;            /* polynomial degree, 1..8                                 */
  int nx, ny, nz;   /* elements per direction (nz ignored for dim 2)           */
  int disc;         /* lor_disc                                                */
  double eta;       /* DG penalty parameter (IP: sigma = eta p^2 kappa / h)    */
  int mg_levels;    /* patch V-cycle levels: 0 = full element-structured
                       hierarchy (Section 3.3), L >= 2 = first L-1 levels then
                       the vertex level                                        */
  int prec;         /* lor_prec used by lor_pcg_solve                          */
  double rtol;      /* stop when ||r||_2 <= rtol ||b||_2                       */
  int max_it;       /* Krylov iteration cap                                    */
  double inner_rtol;/* LOR_MIXED: relative tolerance of each FP32 inner solve  */
  int factor_bf16;  /* LOR_MIXED/FP32: store ILU factors in bf16 (1) or fp32 */
  int weighting;    /* patch sum of Eq. (as): 0 = unit weights (the paper's
                       method); 1 = scaled on both sides by D^{-1/2}, D the
                       number of patches containing each node (the counting
                       matrix Section 4.1 leaves to future work); 2 = patch j
                       scaled on both sides by sqrt(theta_j), theta_j the Q1
                       function of its vertex in element reference
                       coordinates (a partition of unity over the patches) */
} lor_options;

/* Fills *opt with defaults: dim 3, p 4, 8^3 elements, CG, eta 1, full
 * hierarchy, FP64, rtol 1e-8, max_it 1000, inner_rtol 1e-3, fp32 factors,
 * unit patch weights. */
void lor_default_options(lor_options* opt);

/* Creates a context for the mesh (Section 2).  Validates the options and sizes
 * (element count and vertex count x dim at most INT_MAX), copies the mesh
 * arrays into the context and rejects non-finite vertices and kappa <= 0
 * (LOR_EINVAL); LOR_ENOMEM if the host copy cannot be allocated.  vertices and
 * kappa may be HOST or DEVICE pointers: an array the CUDA runtime reports as
 * device or managed memory is copied to the host on `stream` (the call waits
 * for it; LOR_ECUDA if the copy fails); any other pointer, and every pointer
 * when no CUDA device is present, is read as host memory.  Nothing else of
 * CUDA is touched here.  stream: a cudaStream_t or NULL. */
lor_status lor_create(lor_ctx** ctx, const lor_options* opt,
                      const double* vertices, const double* kappa, void* stream);

/* Builds everything the iteration needs (Sections 3.1-3.4, Table 1): geometric
 * factors of the sum-factorized operator, the LOR matrix K_h as a 3^d-point
 * stencil, Galerkin level stencils of the element-structured hierarchy, the
 * lexicographic ILU(0) factors of every vertex patch at every level, and the
 * coarse-space hierarchy.  Allocates all device memory of the context and
 * uploads the mesh.  LOR_EINVAL if an element has det J <= 0 at a quadrature
 * point, LOR_EBREAKDOWN if any ILU(0) pivot is not positive.  A failed setup
 * is not retried: later lor_setup calls return LOR_ESTATE (destroy the
 * context). */
lor_status lor_setup(lor_ctx* ctx);

typedef struct {
  long long nvec;      /* length of an L-vector (all grid nodes)               */
  long long ndof;      /* unknowns: interior nodes (CG) or all DG nodes        */
  long long npatch;    /* vertex patches J                                     */
  long long ncoarse;   /* interior coarse-space unknowns                       */
  int levels;          /* patch hierarchy levels                               */
  int coarse_levels;   /* coarse-space V-cycle levels                          */
  long long factor_rows; /* sum of patch rows over all patches and levels     */
  size_t device_bytes; /* device memory held by the context                    */
} lor_info;

lor_status lor_get_info(const lor_ctx* ctx, lor_info* info);

/* b = M f for the Galerkin right-hand side of Eq. (system), integrated with
 * (p+1)^d Gauss-Legendre points: kind 0: f = 1; kind 1: f = d pi^2 prod_a
 * sin(pi x_a) (manufactured solution u = prod_a sin(pi x_a)).  d_b: device
 * float64 L-vector (or DG vector for DG contexts). */
lor_status lor_rhs(lor_ctx* ctx, int kind, double* d_b);

/* The load vector of the caller's right-hand side f (Eq. (system): f is an input
 * of the problem, b_i = integral of f phi_i), integrated with the (p+1)^d
 * Gauss-Legendre points of every element under the element map the operator
 * uses (multilinear, or the isoparametric interpolant of lor_set_node_coordinates).
 * lor_quadrature_points writes the physical coordinates of those points into the
 * caller's HOST array xq (nel (p+1)^d points x dim doubles, point-major; elements
 * x fastest, point q = qx + Q qy + Q^2 qz inside an element, Q = p+1); it makes no
 * CUDA call and works before lor_setup.  lor_rhs_f takes f at those points as a
 * DEVICE float64 array d_fq (same order) and writes b into d_b (an L-vector with
 * zero boundary entries, or a DG vector for DG contexts).  LOR_EINVAL for NULL
 * arrays, LOR_ESTATE before lor_setup. */
lor_status lor_quadrature_points(const lor_ctx* ctx, double* xq);
lor_status lor_rhs_f(lor_ctx* ctx, const double* d_fq, double* d_b);

/* y = A x, the matrix-free sum-factorized operator (Section 2; Eq. (ip)/(br2)
 * for DG contexts).  prec LOR_FP64: x, y float64; LOR_FP32: x, y float32. */
lor_status lor_apply_A(lor_ctx* ctx, const void* d_x, void* d_y, int prec);

/* z = B r, the additive-Schwarz LOR preconditioner of Eq. (as): coarse-space
 * correction plus one V(1,1) cycle with ordered ILU(0) smoothing on every
 * vertex patch (Sections 3.2-3.4); for DG contexts B_DG of Eq. (dg-as).
 * prec LOR_FP64: float64 vectors and factors; LOR_FP32: float32 vectors,
 * float32 stencils and float32/bf16 factors. */
lor_status lor_apply_P(lor_ctx* ctx, const void* d_r, void* d_z, int prec);

/* Solves A x = b by preconditioned CG from x0 = 0 to ||r|| <= rtol ||b||
 * (Section 4).  LOR_FP64: plain FP64 PCG.  LOR_MIXED: iterative refinement
 * with FP64 residuals b - A x and FP64 corrections; each correction is a PCG
 * solve with FP32 operator and preconditioner and FP64 inner products.
 * d_b, d_x: device float64 L-vectors.  iters: total (inner) iterations;
 * rel_res: final ||b - A x|| / ||b|| computed in FP64.  Either may be NULL. */
lor_status lor_pcg_solve(lor_ctx* ctx, const double* d_b, double* d_x,
                         int* iters, double* rel_res);

/* Same as lor_pcg_solve with HOST buffers (pageable or pinned): copies b to
 * the device, solves, copies x back, all on the context stream. */
lor_status lor_pcg_solve_host(lor_ctx* ctx, const double* h_b, double* h_x,
                              int* iters, double* rel_res);

/* Selects the precision lor_pcg_solve uses from now on (lor_prec); the context
 * keeps FP64 and FP32 (and, if requested, bf16) data, so no setup is redone. */
lor_status lor_set_prec(lor_ctx* ctx, int prec);

/* Checkpoint / resume of the FP64 PCG solve (an auxiliary service; not in the
 * paper).  After lor_pcg_solve with LOR_FP64 returned LOR_OK or LOR_ENOCONV on
 * this context (and before anything else uses its Krylov vectors: another
 * solve or a batch), lor_pcg_state_save copies the iteration state into a
 * caller-owned HOST buffer of lor_pcg_state_size bytes.  The state holds a
 * header (problem sizes, iteration count, ||b||, r.z, r.r), then x (from d_x,
 * the solve's solution), r = b - A x, z and the search direction p.
 * lor_pcg_resume continues PCG from such a state, on a context set up for the
 * same problem (dimension, degree, mesh sizes, discretization, learned
 * correction on or off), for up to max_it more iterations.  d_b is the
 * right-hand side and d_x receives the iterate.  *iters counts all iterations
 * since the original start.  LOR_ESTATE if there is no state to save;
 * LOR_EINVAL for a buffer that is too small, not a state, or a state of
 * another problem; LOR_ENOCONV as lor_pcg_solve. */
lor_status lor_pcg_state_size(const lor_ctx* ctx, size_t* bytes);
lor_status lor_pcg_state_save(lor_ctx* ctx, const double* d_x, void* host, size_t bytes);
lor_status lor_pcg_resume(lor_ctx* ctx, const void* host, size_t bytes, const double* d_b, double* d_x, int* iters,
                          double* rel_res);

/* Pointwise coefficients b(x) (Section 4.2, the coefficients b1-b3) in place of
 * the per-element kappa, for CG contexts.  The coefficient is sampled at two
 * point sets, both listed by lor_coefficient_points:
 *   - the (p+1)^d Gauss-Legendre points of every element, where K_p is
 *     integrated: nq = nel (p+1)^d points, element-major (elements x fastest),
 *     q = qx + Q qy + Q^2 qz inside an element;
 *   - the 2^d Gauss points of every sub-cell of the GLL-refined mesh, where K_h
 *     is integrated (Section 3.1): nh = cells 2^d points, cells x fastest on the
 *     (N-1)^d sub-cell grid, g = gx + 2 gy + 4 gz inside a cell.
 * lor_coefficient_sizes gives nq and nh.  lor_coefficient_points writes the
 * physical coordinates (dim doubles per point, point-major) into caller-owned
 * HOST arrays xq and xh (either may be NULL); it makes no CUDA call and works
 * before lor_setup.  lor_set_coefficient copies the HOST values b(xq) and b(xh);
 * it must precede lor_setup (LOR_ESTATE after), and it refuses DG contexts, NULL
 * arrays and values that are not positive and finite (LOR_EINVAL). */
lor_status lor_coefficient_sizes(const lor_ctx* ctx, long long* nq, long long* nh);
lor_status lor_coefficient_points(const lor_ctx* ctx, double* xq, double* xh);
lor_status lor_set_coefficient(lor_ctx* ctx, const double* bq, const double* bh);

/* Curved (isoparametric) elements, as in the curved meshes of Section 4.2, for CG
 * contexts.  X (HOST, copied) gives the physical coordinates of every level-0 GLL
 * node: X[a*ntot + (K*Ny+J)*Nx+I], ntot = Nx*Ny(*Nz), a < dim (the L-vector node
 * order).  K_p then uses the degree-p isoparametric map of each element's nodes
 * (its Jacobian at the Gauss points), and K_h the LOR sub-cells with these
 * corners.  The coarse space and the patch weights stay defined in reference
 * coordinates.  Must precede lor_setup (LOR_ESTATE after).  LOR_EINVAL for DG
 * contexts, with lor_set_coefficient, for a NULL array or a non-finite
 * coordinate; lor_setup reports a non-positive Jacobian as LOR_EINVAL.
 * lor_rhs then integrates on the isoparametric elements. */
lor_status lor_set_node_coordinates(lor_ctx* ctx, const double* X);

/* Selects the ILU(0) ordering of every patch level (Section 3.4): 0 =
 * lexicographic (x fastest; the default), 1 = reverse Cuthill-McKee of the
 * 3^d-point pattern of the patch box (breadth-first from the node of smallest
 * (degree, index), neighbours by increasing (degree, index), reversed), 2 =
 * minimum discarded fill of the patch matrix (the node whose elimination would
 * discard the smallest 2-norm of fill is ordered next, ties by smallest index;
 * the kept fill updates the remaining matrix).  Orderings 1 and 2 are computed
 * on the host during lor_setup together with the ILU(0) factors in that order,
 * one patch per host thread at a time (MDF costs about 26^2 operations per
 * remaining neighbour per elimination step, seconds per thousand patches at
 * p = 4); their sweeps follow the dependency levels of the order, in fronts of
 * at most 32 rows, with records that hold all 3^d - 1 couplings of a row.  Must
 * precede lor_setup (LOR_ESTATE after); LOR_EINVAL for other values.  A
 * non-positive pivot of the ordered factorization makes lor_setup return
 * LOR_EBREAKDOWN. */
lor_status lor_set_ordering(lor_ctx* ctx, int ordering);

/* Host-only utility (no context, no CUDA call): the ordering lor_set_ordering
 * uses, for one box of A x B x C nodes (C = 1 in 2D; at most 2^20 nodes) with the
 * 3^d-point pattern.  a27: per node (x fastest) its 3^d stencil values in
 * stencil-offset order ((dz+1)*9 + (dy+1)*3 + (dx+1); zero for neighbours
 * outside the box), read only for MDF (ordering 2).  perm (A*B*C ints, host):
 * perm[q] = box index of the q-th node.  LOR_EBREAKDOWN if MDF meets a
 * non-positive pivot, LOR_EINVAL for bad sizes or ordering. */
lor_status lor_box_ordering(int dim, int A, int B, int C, int ordering, const double* a27, int* perm);

/* Host-only utility (no context, no CUDA call): the ILU(0) factorization in a
 * given order (Section 3.4) that lor_setup applies to every RCM- or MDF-ordered
 * patch level, for one box laid out as in lor_box_ordering.  perm (A*B*C ints):
 * the elimination order, perm[q] = box index of the q-th node; it must be a
 * permutation.  lu (A*B*C x 3^d doubles, host, written): per node its factor
 * entries in stencil-offset order: at the offsets of neighbours eliminated
 * before it the multipliers of the unit lower factor, at the centre the pivot
 * u_ii, at the other in-box offsets the entries of the upper factor, 0 outside
 * the box.  level (A*B*C ints, host, written; may be NULL): the dependency level
 * of each node (0 without earlier neighbours, else one more than the largest
 * level among them), i.e. the wavefronts of the ordered sweeps.  LOR_EBREAKDOWN
 * on a non-positive pivot, LOR_EINVAL for bad sizes or a perm that is not a
 * permutation. */
lor_status lor_box_ilu0(int dim, int A, int B, int C, const double* a27, const int* perm, double* lu,
                        int* level);

/* Patches enlarged for isotropic overlap on anisotropic meshes (Section 4.5):
 * spans (host, npatch x dim x 2 ints, patch-major, per axis: lo then hi) lets the
 * patch of vertex v cover the elements v - lo .. v + hi - 1 along each axis
 * (clamped to the mesh) instead of v - 1 .. v; 1, 1 is the vertex patch.  The
 * element-structured V(1,1) cycle runs on each enlarged box unchanged; a box that
 * keeps several vertices on its coarsest level solves them with the inverse of its
 * box matrix, formed on the host in lor_setup.  Enlarged patches use host-built
 * factors, per-patch schedules and a node-by-node gather of the patch outputs (in
 * patch order).  NULL restores vertex patches.  Must precede lor_setup (LOR_ESTATE
 * after); CG only, unit patch weights, no learned correction; LOR_EINVAL for a
 * span outside 1..8. */
lor_status lor_set_patch_spans(lor_ctx* ctx, const int* spans);

/* The ILU(0) order of one patch level: perm[q] = box index (x fastest within the
 * patch box) of the q-th row, for level 0 <= level < levels - 1 (the vertex level
 * is solved exactly) and patch 0 <= patch < npatch (vertex (i,j,k) is patch
 * (k*(ny+1)+j)*(nx+1)+i).  *count = rows of the box; perm may be NULL to query
 * it, else cap >= *count (LOR_EINVAL otherwise).  Host memory, filled from the
 * context's host copy; the identity for the lexicographic ordering. */
lor_status lor_patch_ordering(lor_ctx* ctx, int level, long long patch, int* perm, int cap, int* count);

/* Switches the patch-sum weighting of lor_options.weighting (0 unit weights,
 * 1 counting matrix, 2 partition of unity) for later calls; the weights are evaluated inside the
 * patch kernel, so no setup is redone.  A batch (lor_batch_create) keeps the
 * setting its contexts had when its CUDA graph was captured (first
 * lor_batch_solve).  LOR_EINVAL for other values or if the learned correction
 * is enabled (it is trained for unit weights). */
lor_status lor_set_weighting(lor_ctx* ctx, int weighting);

/* Selects how apply_P combines the coarse space with the patches: 0 = additive,
 * B = P_0 R_0 P_0^T + sum_j R_j^T V_j R_j (Eq. (as), the default); 1 = hybrid,
 * the coarse correction multiplicative and the patches additive among
 * themselves (the variant Section 4.1 leaves to future work), in the symmetric
 * form B_hyb = B_0 + (I - B_0 K_h) B_loc (I - K_h B_0), B_0 = P_0 R_0 P_0^T,
 * B_loc the patch sum and K_h the LOR matrix on the interior nodes.  B_hyb is
 * B_0 plus a congruence of B_loc, so it is symmetric positive definite and PCG
 * applies.  An apply in hybrid form costs the additive one plus a second coarse
 * V-cycle and two K_h stencil products.  2 = B(1), the whole domain as one patch
 * (Section 4.1, Table 2): one V(1,1) cycle of the element-structured hierarchy
 * on the global level grids, one lexicographic ILU(0) smoothing before and one
 * after the coarse-level correction on every level above the vertex level, and
 * the coarse solver R_0 on the vertex level.  Its ILU(0) factors are computed
 * when the mode is first selected (hyperplane-parallel factorization on the
 * device; LOR_EBREAKDOWN on a non-positive pivot) and its sweeps run one launch
 * per hyperplane i + 2j + 4k of each level grid.  The first switch to 1 or 2
 * allocates that form's work space (three float64 vectors of nvec entries for
 * 1; factors of 3^d float64 and float32 values per level-grid node and six
 * vectors per level for 2; LOR_ENOMEM if that fails); the setting holds for
 * every later apply_P and solve, and for the DG preconditioner's conforming
 * part.  LOR_ESTATE before lor_setup; LOR_EINVAL for other values or with the
 * learned correction enabled (it is trained for the additive form). */
lor_status lor_set_schwarz(lor_ctx* ctx, int mode);

/* Number of kernels this context has launched so far (all entry points). */
lor_status lor_launch_count(const lor_ctx* ctx, long long* count);

/* Kernel timing with CUDA events recorded on the context stream around every
 * launch of the hot kernels while profiling is on (at most 8192 launches per
 * kernel are kept).  lor_profile(ctx, 1) clears and starts, 0 stops.
 * lor_profile_read sums the recorded durations of one kernel class:
 *   0 patch V-cycle FP64, 1 patch V-cycle FP32, 2 apply_A FP64, 3 apply_A FP32,
 *   4 coarse-space correction FP64, 5 coarse-space correction FP32.
 * It synchronises the stream. */
lor_status lor_profile(lor_ctx* ctx, int on);
lor_status lor_profile_read(lor_ctx* ctx, int kernel, double* total_ms, long long* launches);

/* Per-iteration residual norms ||r_k||_2 of the last solve (k = 0..count-1,
 * FP64 outer residuals and inner FP64-accumulated norms for LOR_MIXED). */
lor_status lor_residual_history(const lor_ctx* ctx, double* out, int cap, int* count);

/* ---- Batched solves (serving-shaped workloads; the paper solves one problem)
 * Many independent CG contexts (after lor_setup; uneven sizes and degrees) are
 * advanced together by flexible CG with FP64 vectors and inner products and
 * the FP32 LOR preconditioner of each context.  One iteration of all solves is
 * captured once into a CUDA graph with one branch per solve; the host launches
 * it until every solve has reached its rtol.  lor_batch_create also tunes the
 * operator's tile shape per polynomial degree by timing.  The batch borrows the
 * contexts (they must outlive it) and their work vectors; stream: cudaStream_t
 * or NULL.  d_b[s], d_x[s]: device float64 L-vectors of context s. */
typedef struct lor_batch lor_batch;
lor_status lor_batch_create(lor_batch** batch, int n, lor_ctx** ctxs, void* stream);
lor_status lor_batch_solve(lor_batch* batch, const double* const* d_b, double* const* d_x, int* iters,
                           double* rel_res);
/* Wall time of the last solve's iteration loop (ms) and nodes of its graph. */
lor_status lor_batch_stats(const lor_batch* batch, double* loop_ms, int* graph_nodes);
void lor_batch_destroy(lor_batch* batch);

/* ---- Learned per-patch correction (the learned form of the method)
 * After the V(1,1) cycle of every interior vertex patch, a 3-layer 3x3x3
 * convolutional network (2 -> 16 -> 16 -> 1 channels, ReLU, bf16 weights, FP32
 * accumulation) maps the remaining level-0 residual t to the correction
 * rho s N([s t / rho, log(diag/mean diag)]), s = diag(A_j)^(-1/2), rho = rms(s t).
 * It applies to the FP32 preconditioner (LOR_MIXED solves); with it on, the
 * Krylov iteration is flexible CG.  Parameters: one float array of
 * LOR_LEARNED_NPARAM values, W1[16][2][27] b1[16] W2[16][16][27] b2[16]
 * W3[1][16][27] b3[1], taps ordered (dz+1)*9+(dy+1)*3+(dx+1).
 * lor_learned_params: copy host parameters in (h_in) and/or out (h_out).
 * lor_learned_enable: switch the correction on (1) or off (0).
 * lor_learned_variant: 0 (default) = the correction is added after the whole
 *   V(1,1) cycle; 1 = it replaces the level-0 post-smoothing: the patch cycle
 *   returns after the coarse correction and the network sees the residual that
 *   leaves.  The variant applies to training (the pairs come from the cycle of
 *   the variant) and to inference, so parameters trained for one variant are
 *   not meant for the other.  LOR_EINVAL for other values.
 * lor_learned_train: `steps` Adam steps (learning rate lr) on batches of
 *   `batch` interior patches of this context; each step draws random errors e,
 *   runs the plain V-cycle x = V(A e) and minimises
 *   (delta - c)^T A_j (delta - c) / delta^T A_j delta, delta = e - x; h_loss
 *   (host, `steps` floats, may be NULL) receives the mean loss per step.
 * lor_learned_eval: forward (and, with d_delta, loss and gradient) on given
 *   patch data: d_ids (device, npatch interior patch ids), d_t / d_delta
 *   (device, npatch x (2p-1)^3 floats, lexicographic box order); outputs the
 *   correction d_c, per-patch loss d_loss (device) and the summed gradient
 *   h_grad (host, LOR_LEARNED_NPARAM floats).  Intended for checks. */
#define LOR_LEARNED_NPARAM 8241
lor_status lor_learned_params(lor_ctx* ctx, const float* h_in, float* h_out, int count);
lor_status lor_learned_enable(lor_ctx* ctx, int on);
lor_status lor_learned_variant(lor_ctx* ctx, int variant);
lor_status lor_learned_train(lor_ctx* ctx, int steps, int batch, float lr, unsigned long long seed, float* h_loss);
lor_status lor_learned_eval(lor_ctx* ctx, int npatch, const int* d_ids, const float* d_t, const float* d_delta,
                            float* d_c, float* d_loss, float* h_grad);

/* Allocation-free right-hand side (no counterpart in the paper; a service for
 * callers that may not call cudaMalloc).  Some callers cannot allocate device
 * memory: a host framework that hands all device memory to its own caching
 * pool and forbids raw cudaMalloc, or a process whose device-memory budget is
 * fixed at start-up.  They cannot build a lor_ctx either, so this entry point
 * needs none: given DEVICE vertex coordinates (layout as for lor_create), it
 * computes the same b = M f as lor_rhs (kinds 0 and 1, (p+1)^d Gauss points)
 * into the caller's DEVICE vector d_b (an L-vector, boundary entries 0), on
 * `stream` (a cudaStream_t or NULL).
 * Scratch: the per-point quadrature weights and the 1D basis tables live in
 * one file-scope static device array of LOR_RHS_STATIC_MAX_DOUBLES doubles
 * (16 MiB, held by every GPU that loads the library until the process exits);
 * problems with nel*(p+1)^d > LOR_RHS_STATIC_MAX_DOUBLES - 256 are rejected
 * with LOR_EINVAL.  The call allocates nothing and frees nothing.
 * The first call on a device looks up the device address of that array (with
 * the device current); make that first call before any stream capture.
 * Every call shares the one array and overwrites it, so calls that may run
 * concurrently on the GPU (other streams, other threads) race: serialise them.
 * Returns LOR_EINVAL for bad arguments, LOR_ECUDA if a CUDA call fails. */
#define LOR_RHS_STATIC_MAX_DOUBLES (1 << 21)
lor_status lor_rhs_static(int dim, int p, int nx, int ny, int nz, const double* d_vertices, int kind,
                          double* d_b, void* stream);

/* Device-side error check (no paper counterpart).  lor_apply_A/lor_apply_P
 * only enqueue work; a bounded device wait inside them that ran out (a factor
 * bulk copy of the patch kernel that did not complete within its poll limit;
 * the kernel then skips the rest of that warp's work and returns) is recorded
 * in the context's device status word.  This call synchronizes the context
 * stream, returns LOR_ETIMEOUT if such a wait ran out since the last check and
 * clears the record (the context stays usable), else LOR_OK.  lor_pcg_solve
 * performs the same check before it returns. */
lor_status lor_device_status(lor_ctx* ctx);

/* Self-test of the bounded device waits (no paper counterpart): launches one
 * warp that waits on an mbarrier at which nothing ever arrives, giving up after
 * `polls` polls (1 <= polls <= 2^24; 2^12 takes well under a millisecond).  The
 * expected result is LOR_ETIMEOUT, reported and cleared as by
 * lor_device_status; LOR_OK would mean the wait did not time out. */
lor_status lor_selftest_wait(lor_ctx* ctx, int polls);

/* FP64 FMA throughput of the current device (no paper counterpart; the
 * denominator of the FP64 operator's roofline): a kernel of independent FP64
 * FMA chains on every SM, best of three timed launches, in TFLOP/s (an FMA
 * counts 2 flops).  Needs no context; runs on the legacy default stream and
 * synchronizes it.  LOR_EINVAL for NULL, LOR_ECUDA if a CUDA call fails. */
lor_status lor_measure_fp64_peak(double* tflops);

const char* lor_last_error(const lor_ctx* ctx);
void lor_destroy(lor_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LOR_H */
