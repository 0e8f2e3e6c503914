// Internal declarations of the LOR solver library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lor.h"

#define LOR_MAXP 8
#define LOR_MAXSPAN 8     // elements an enlarged patch may take on each side of its vertex
#define LOR_MAXLEV 5      // p <= 8: at most 4 patch levels (8,4,2,1) + slack
#define LOR_MAXCLEV 8     // coarse-space V-cycle levels

// ------------------------------------------------------------------ host basis
namespace lorh {
// GLL points/weights of degree p on [0,1]; Gauss-Legendre with q points on [0,1].
void gll(int p, double* x, double* w);
void gauss(int q, double* x, double* w);
// Lagrange basis on `nodes` (m of them) at points t (nt): B[t*m+i], D[t*m+i].
void lagrange(int m, const double* nodes, int nt, const double* t, double* B, double* D);
// Element-structured hierarchy (Section 3.3): GLL-index subsets per level.
std::vector<std::vector<int>> level_selections(int p, int mg_levels);
// Orderings of a patch-level box (A x B x C nodes, 3^d-point pattern) for ILU(0)
// (Section 3.4), as permutations new position -> box index (orderings.cpp):
// reverse Cuthill-McKee of the pattern, and minimum discarded fill of the matrix
// a27 (per node its 3^d stencil values, zero outside the box; false on a
// non-positive pivot).
void rcm_box(int dim, int A, int B, int C, std::vector<int>& perm);
bool mdf_box(int dim, int A, int B, int C, const std::vector<double>& a27, std::vector<int>& perm);
// ILU(0) of a27 in the order perm, in place in box-index layout (lu: per node the
// multipliers at earlier neighbours, u_ij at later ones and u_ii at the centre),
// and the level of every node in the dependency schedule of the order (0 for
// nodes without earlier neighbours).  False on a non-positive pivot.
bool ilu0_ordered(int dim, int A, int B, int C, const std::vector<double>& a27, const std::vector<int>& perm,
                  std::vector<double>& lu, std::vector<int>& level);
}  // namespace lorh

// ---------------------------------------------------------- device-side tables
// 1D prolongation entry of a fine point: value = w0*coarse[c0] + w1*coarse[c1].
struct Prolong1D { int c0, c1; double w0, w1; };

// Patch 1D structure of one level and one axis type (0 interior, 1 boundary).
// Restriction entry of one coarse point: the fine points feeding it (a coarsening
// step may skip up to 2p-1 fine points per axis when the hierarchy is truncated).
#define LOR_MAXR (2 * LOR_MAXP)
struct RestrictEntry { int cnt; int f[LOR_MAXR]; double w[LOR_MAXR]; };

struct PatchAxis {
  int len;        // unknowns along the axis at this level
  int clen;       // unknowns at the next coarser level
};

struct LevelGrid {
  int m;                  // intervals per element
  int N[3];               // nodes per direction (1 for unused dims)
  long long ntot;
};

// Shape of a patch box at one level: wavefront schedule for lexicographic ILU(0).
// Factor storage of one patch level: front-major records of lor_rec(dim) values
// (16 in 3D, 8 in 2D).  L record of a row: its 13 (3D) / 4 (2D) strictly-lower
// ILU(0) multipliers in stencil-offset order; U record: its upper coefficients
// in stencil-offset order and 1/u_ii in slot rec-2.  Slot rec-1 of both holds
// the row's lexicographic index in the patch box as raw integer bits (low 16
// bits of a bf16 slot, the 32-bit pattern of a float slot, the low word of a
// double slot), so a sweep reads a row's position together with its factors.
// The records of each wavefront are padded to a multiple of 4 rows so every
// front block starts on a 16-byte boundary (bulk-copy alignment); a padding
// record is all zero except its index, which points at the first guard cell
// after the box (index = rows), so a sweep may process it like a real row.
__host__ __device__ constexpr int lor_rec(int dim) { return dim == 3 ? 16 : 8; }

// Records of an algebraically ordered patch level (RCM or MDF, Section 3.4): any
// neighbour may precede a row in the order, so a record holds all 26 (3D) / 8 (2D)
// couplings in stencil-offset order without the centre: the L record the
// multipliers of the earlier neighbours (0 at the later ones), the U record the
// coefficients of the later neighbours, and 1/u_ii in slot rec-2; slot rec-1 holds
// the row index as in the lexicographic records.  Rows are grouped by their level
// in the dependency schedule of the order, each level split into fronts of at most
// 32 rows (rows of one level never couple), fronts padded to 4 records.
__host__ __device__ constexpr int lor_rec_gen(int dim) { return dim == 3 ? 32 : 16; }

// Per-patch, per-level schedule of an ordered patch level: fronts and bulk-copy
// chunks as in BoxShape, offsets into ctx->d_gfpad / d_gchunk.
struct GenSched {
  int nfront, rpad, front_off;
  int nchunk[3], chunk_off[3];
  // box of this patch at this level (any patch span): extents, origin in the level
  // grid, rows, guard band; elements spanned per axis (selects the patch-local 1D
  // transfer tables); at the vertex level, the offset of the inverse of the box
  // matrix (when it has more than one row) in ctx->d_binv
  int dims[3], org[3], rows, guard, k[3];
  long long binv_off;
};

// Patch-local 1D transfer between level l and l+1 along an axis spanning k elements
// (fine and coarse unknowns: the open interiors of the span), in global memory:
// prolongation rows (fine -> <= 2 coarse; coarse index -1 or clen = the span's end,
// value 0) and the transposed restriction lists.  T = double or float.
template <typename T>
struct XferG {
  const int* c0;
  const int* c1;
  const T* w0;
  const T* w1;
  const int* rstart;
  const int* rf;
  const T* rw;
};
// row length of the row-major stencil copies: 3^dim padded to a multiple of 4
__host__ __device__ constexpr int lor_nsp(int dim) { return dim == 3 ? 28 : 12; }
struct BoxShape {
  int dims[3];            // box extents (x, y, z); 1 for unused dims
  int rows;
  int nfront;
  int front_off;          // offset into ctx->d_front / d_fpad (nfront+1 entries)
  int row_off;            // offset into the per-row tables (rows entries)
  int rpad;               // padded records of one part (L or U)
  int maxfront;           // largest padded front (records)
  int nchunk[3];          // groups of consecutive fronts streamed as one bulk copy,
  int chunk_off[3];       // per factor element size (index 0: 2, 1: 4, 2: 8 bytes);
  int maxchunk[3];        // offsets into ctx->d_chunk (nchunk+1 front indices); records
  int guard;              // largest |stencil offset| in the lexicographic box index
};

struct lor_ctx {
  lor_options opt;
  int dim, p;
  int n[3];
  int nel;
  cudaStream_t stream;
  std::string err;
  bool setup_done = false;
  bool setup_started = false;   // a failed lor_setup leaves partial state: no retry

  // mesh
  double* d_vert = nullptr;   // SoA dim x NV
  double* d_kappa = nullptr;
  std::vector<double> h_vert, h_kappa;
  // optional pointwise coefficient b(x) (lor_set_coefficient): values at the Gauss
  // points of K_p ([element][q]) and of the LOR sub-cells of K_h ([cell][g])
  std::vector<double> h_bq, h_bh;
  double* d_bq = nullptr;
  double* d_bh = nullptr;
  // optional GLL node coordinates of curved elements (lor_set_node_coordinates), SoA dim x ntot
  std::vector<double> h_nodes;

  // 1D basis (host copies, device constant tables are uploaded per launch)
  double gll_x[LOR_MAXP + 1], gll_w[LOR_MAXP + 1];
  double gl_x[LOR_MAXP + 2], gl_w[LOR_MAXP + 2];
  double B[(LOR_MAXP + 1) * (LOR_MAXP + 1)];   // B[q*(p+1)+i] = l_i(gl_q)
  double Dq[(LOR_MAXP + 1) * (LOR_MAXP + 1)];  // collocated derivative at GL points

  // operator data
  double* d_G64 = nullptr;    // [nel][ncomp][Q] geometric factors (kappa w detJ J^-1 J^-T)
  float* d_G32 = nullptr;
  double* d_X = nullptr;      // level-0 node coordinates SoA dim x ntot

  // level hierarchy
  int L = 0;
  std::vector<std::vector<int>> sel;
  LevelGrid lev[LOR_MAXLEV];
  double* d_S64[LOR_MAXLEV] = {};   // [NS][ntot_l] stencils
  float* d_S32[LOR_MAXLEV] = {};
  // row-major copies [ntot_l][lor_nsp(dim)] of the patch-level stencils (levels
  // 0..L-2), read by the patch residuals as whole rows
  double* d_SA64[LOR_MAXLEV] = {};
  float* d_SA32[LOR_MAXLEV] = {};
  Prolong1D* d_P1[LOR_MAXLEV][3] = {};    // global 1D prolongation level l+1 -> l (per axis)
  int* d_R1ptr[LOR_MAXLEV][3] = {};       // restriction CSR: coarse -> fine list
  int* d_R1idx[LOR_MAXLEV][3] = {};
  double* d_R1w[LOR_MAXLEV][3] = {};

  // patches
  int J = 0;                  // number of vertex patches
  int NS = 27;                // stencil size 3^dim
  std::vector<BoxShape> shapes;           // [level][8 shapes]
  BoxShape* d_shapes = nullptr;           // device copy of `shapes`
  int* d_poslex = nullptr;                // lexicographic index -> wavefront position
  int* d_front = nullptr;     // row position where each wavefront starts
  int* d_fpad = nullptr;      // record offset where each wavefront starts
  int* d_chunk = nullptr;     // first front of each bulk-copy chunk
  int* d_rowlex = nullptr;    // lexicographic index of the row at a wavefront position
  int* d_recof = nullptr;     // record index of the row at a wavefront position
  // per-level per-axis-type patch-local 1D prolongation (fine -> coarse, local idx)
  Prolong1D* d_pp[LOR_MAXLEV][2] = {};
  // per-level per-axis-type patch-local restriction: coarse local c -> 3 (fine local f, w), f = -1 unused
  struct RestrictEntry* d_rr[LOR_MAXLEV][2] = {};
  long long* d_facoff = nullptr;          // [level][J] record offsets into factor arrays
  int* d_porder = nullptr;                // patches grouped by box shape, interior first
  long long fac_rows = 0;
  double* d_F64 = nullptr;
  float* d_F32 = nullptr;
  __nv_bfloat16* d_F16 = nullptr;
  int smem_patch64 = 0, smem_patch32 = 0;
  // per-warp level-0 iterate of the patch kernel (one slot of x0_stride values per
  // resident warp; small enough to stay in L2)
  void* d_xs = nullptr;
  long long xs_bytes = 0;
  // per-patch outputs of the patch kernel (J slices of level-0 box rows, sized for
  // float64), summed node by node into z by a gather kernel
  void* d_zp = nullptr;
  // coarse-space combination of apply_P: 0 additive (Eq. (as)), 1 hybrid (coarse
  // multiplicative); the hybrid form's three level-0 work vectors (float64-sized)
  int schwarz = 0;
  void* d_hyb = nullptr;
  int maxfront = 0;           // largest padded front over all levels/shapes (records)
  // ILU(0) ordering of the patch levels: 0 lexicographic (wavefront records), 1 RCM,
  // 2 MDF (ordered records, per-patch schedules; host permutations kept for
  // lor_patch_ordering)
  int ordering = 0;
  // patch spans (lor_set_patch_spans): per patch and axis the elements on each side
  // of its vertex (1, 1 = the vertex patch); empty = vertex patches
  std::vector<int> h_spans;
  int span_kmax = 2;                       // most elements spanned along an axis
  bool gen = false;                        // ordered or enlarged patches: host-built factors and schedules
  void* d_xferg64 = nullptr;               // XferG<double>[level][kmax + 1] (device)
  void* d_xferg32 = nullptr;               // XferG<float>[level][kmax + 1]
  double* d_binv64 = nullptr;              // vertex-level inverses of enlarged patches
  float* d_binv32 = nullptr;
  long long* d_gather_ptr = nullptr;       // level-0 node -> its entries in the patch output slices
  long long* d_gather_idx = nullptr;
  int gen_rows0 = 0, gen_A0 = 0, gen_AB0 = 0, gen_rows1 = 0, gen_guard0 = 0;   // largest level-0/1 boxes
  long long gen_ovl = 0;                   // largest overlay of the coarse levels (values)
  GenSched* d_gsched = nullptr;            // [level][J]
  int* d_gfpad = nullptr;
  int* d_gchunk = nullptr;
  int gen_tab_ints = 0;                    // largest per-patch table (ints) over all levels
  int gen_maxchunk[3] = {0, 0, 0};
  std::vector<std::vector<int>> h_perm;    // [level * J + j] new position -> box index
  int maxchunk[3] = {0, 0, 0};   // largest chunk (records) for 2-, 4-, 8-byte factors
  int* d_status = nullptr;    // device error word

  // coarse space (vertex grid hierarchy)
  int CL = 0;
  int cN[LOR_MAXCLEV][3];
  long long cntot[LOR_MAXCLEV];
  double* d_cS64[LOR_MAXCLEV] = {};
  float* d_cS32[LOR_MAXCLEV] = {};
  double* d_cDinv64[LOR_MAXCLEV] = {};   // 1 / l1 row sums
  float* d_cDinv32[LOR_MAXCLEV] = {};
  Prolong1D* d_cP1[LOR_MAXCLEV][3] = {};
  int* d_cR1ptr[LOR_MAXCLEV][3] = {};
  int* d_cR1idx[LOR_MAXCLEV][3] = {};
  double* d_cR1w[LOR_MAXCLEV][3] = {};
  int ncoarse_direct = 0;
  int* d_cdirect_idx = nullptr;           // interior node index of each direct unknown
  // P_0 (vertex-grid multilinear basis at the level-0 nodes) in the path precisions:
  // [gllx (p+1) | 1D restriction weights by offset (2p-1)], and scratch for the
  // separable passes of P_0^T (x, then y, then z)
  double* d_p0w64 = nullptr;
  float* d_p0w32 = nullptr;
  double* d_p0t64[2] = {};
  float* d_p0t32[2] = {};
  double* d_cInv64 = nullptr;             // dense inverse at the coarsest level
  float* d_cInv32 = nullptr;
  // coarse work vectors per level: r, x, t (double and float)
  double* d_cw64[LOR_MAXCLEV][4] = {};
  float* d_cw32[LOR_MAXCLEV][4] = {};

  // Krylov work (double) and mixed inner (float)
  double* d_v64[8] = {};
  float* d_v32[8] = {};
  double* d_scal = nullptr;   // device scalars
  double* d_part = nullptr;   // reduction partials
  unsigned int* d_count = nullptr;
  double* h_scal = nullptr;   // pinned mirror
  std::vector<double> hist;

  // event timing of hot kernels (lor_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev[6];   // start/stop pairs per kernel class
  int nev[6] = {0, 0, 0, 0, 0, 0};
  // DG discretization data (dg.cu); nullptr for continuous contexts
  void* dg_state = nullptr;
  long long nv = 0;            // length of the solver's vectors (CG grid or DG blocks)
  // the last FP64 PCG solve left a resumable state in the Krylov vectors
  bool pcg_state_ok = false;
  double pcg_bnorm = 0.0;
  int pcg_iters = 0;
  int tune_ne = 1;             // apply_A tile variant (elements per CTA), set by the autotuner
  const double* conv_flag = nullptr;   // batched solves: patch kernel returns early when *conv_flag != 0
  // learned correction (learned.cu)
  // single-patch preconditioner B(1) (single.cu), built by lor_set_schwarz(ctx, 2)
  void* single = nullptr;
  void* learned = nullptr;
  bool learned_on = false;
  bool learned_replace = false;        // variant: the correction replaces the level-0 post-smoothing
  float* learned_tout = nullptr;       // level-0 residuals of interior patches after the cycle
  size_t bytes = 0;
  long long launches = 0;      // kernels launched by this context
  std::vector<void*> allocs;
};

// ---------------------------------------------------------------- error helpers
lor_status lor_fail(lor_ctx* c, lor_status s, const std::string& msg);
lor_status lor_cuda_check(lor_ctx* c, cudaError_t e, const char* what);
void* lor_alloc(lor_ctx* c, size_t bytes);   // tracked device allocation (nullptr on failure)

// -------------------------------------------------------------- kernel launchers
// setup.cu
lor_status lor_setup_geometry(lor_ctx* c);
lor_status lor_setup_stencils(lor_ctx* c);
lor_status lor_setup_patches(lor_ctx* c);
lor_status lor_setup_coarse(lor_ctx* c);
// apply_a.cu
lor_status lor_launch_apply_A64(lor_ctx* c, const double* x, double* y);
lor_status lor_launch_apply_A32(lor_ctx* c, const float* x, float* y);
// b = M f with f from `kind` (0: 1, 1: manufactured) or, when fq is given, the
// caller's values at the quadrature points (device, nel (p+1)^d, lor_quadrature_points order)
lor_status lor_launch_rhs(lor_ctx* c, int kind, double* b, const double* fq = nullptr);
lor_status lor_launch_rhs_weights(lor_ctx* c, int kind, double* W);
lor_status lor_launch_dgvol64(lor_ctx* c, const double* x, double* y);
lor_status lor_launch_dgvol32(lor_ctx* c, const float* x, float* y);
// dg.cu
lor_status lor_setup_dg(lor_ctx* c);
lor_status lor_launch_apply_A_dg64(lor_ctx* c, const double* x, double* y);
lor_status lor_launch_apply_A_dg32(lor_ctx* c, const float* x, float* y);
lor_status lor_launch_apply_P_dg64(lor_ctx* c, const double* r, double* z);
lor_status lor_launch_apply_P_dg32(lor_ctx* c, const float* r, float* z);
lor_status lor_launch_rhs_dg(lor_ctx* c, double* b, const double* W);
void lor_free_dg(lor_ctx* c);
void lor_free_learned(lor_ctx* c);
void lor_free_single(lor_ctx* c);
lor_status lor_single_prepare(lor_ctx* c);
template <typename T> lor_status lor_single_apply(lor_ctx* c, const T* r, T* z);
// coarse solver R_0: its right-hand side buffer (the full vertex grid) and one solve,
// returning the buffer that holds the result (apply_p.cu)
template <typename T> T* lor_coarse_rhs(lor_ctx* c);
template <typename T> T* lor_coarse_solve(lor_ctx* c);
lor_status lor_learned_apply(lor_ctx* c, float* z);
lor_status lor_patch_local32(lor_ctx* c, const int* plist, int nlist, const float* rloc, float* xloc, int vstride);
// operator / preconditioner of the context's discretization (CG or DG)
lor_status lor_opA64(lor_ctx* c, const double* x, double* y);
lor_status lor_opA32(lor_ctx* c, const float* x, float* y);
lor_status lor_opP64(lor_ctx* c, const double* r, double* z);
lor_status lor_opP32(lor_ctx* c, const float* r, float* z);
// apply_p.cu
lor_status lor_launch_apply_P64(lor_ctx* c, const double* r, double* z);
lor_status lor_launch_apply_P32(lor_ctx* c, const float* r, float* z);
lor_status lor_patch_prepare(lor_ctx* c);   // launch shapes, shared-memory fit, iterate slots
lor_status lor_launch_wait_selftest(lor_ctx* c, int polls);
// Synchronizes the context stream and reads the device status word: a bounded
// device wait that ran out since the last check -> LOR_ETIMEOUT (the word is
// cleared, so the context stays usable).
lor_status lor_take_device_status(lor_ctx* c);
// krylov.cu
lor_status lor_pcg64(lor_ctx* c, const double* b, double* x, int* iters, double* relres);
lor_status lor_pcg_mixed(lor_ctx* c, const double* b, double* x, int* iters, double* relres);
// checkpoint / resume of the FP64 PCG (lor_pcg_state_save, lor_pcg_resume)
size_t lor_pcg_state_bytes(const lor_ctx* c);
lor_status lor_pcg_save(lor_ctx* c, const double* x, void* host, size_t bytes);
lor_status lor_pcg_resume_impl(lor_ctx* c, const void* host, size_t bytes, const double* b, double* x, int* iters,
                               double* relres);
lor_status lor_setup_krylov(lor_ctx* c);
BoxShape* lor_dev_shapes(lor_ctx* c);
double* lor_basis64(lor_ctx* c, int which);
// sizes and physical coordinates of the coefficient sample points (host; no CUDA call)
void lor_coef_sizes(const lor_ctx* c, long long* nq, long long* nh);
void lor_coef_points(const lor_ctx* c, double* xq, double* xh);
// physical coordinates of the (p+1)^d Gauss points of every element under the
// element map the operator uses (multilinear, or the isoparametric interpolant of
// the given node coordinates); host only
void lor_quad_points(const lor_ctx* c, double* xq);
float* lor_basis32(lor_ctx* c, int which);

// event pair around a hot kernel launch (no-op unless profiling)
void lor_prof_begin(lor_ctx* c, int k);
void lor_prof_end(lor_ctx* c, int k);

// small device utilities shared by the .cu files
__host__ __device__ inline long long lor_ceil_div(long long a, long long b) { return (a + b - 1) / b; }
