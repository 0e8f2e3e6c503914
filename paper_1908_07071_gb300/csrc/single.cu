// B(1): the whole domain as one additive-Schwarz patch (Section 4.1, Table 2).
//
// One V(1,1) cycle of the element-structured hierarchy (Section 3.3) on the global
// LOR levels: on every level l below the vertex level, one ordered ILU(0) smoothing
// (forward and backward sweep) before and one after the correction from level l+1;
// restriction P_l^T and prolongation P_l are the tensor 1D linear interpolations
// between the level grids, the level operators the Galerkin stencils the patch
// cycle uses; the vertex level (the p = 1 problem on the coarse mesh) is solved by
// the coarse solver R_0 of the coarse space.  Unknowns are the interior nodes of
// each level grid (Dirichlet rows and columns dropped).
//
// ILU(0) is lexicographic (x fastest) on the 3^d-point pattern of each level grid.
// In that order every strictly lower neighbour of node (i, j, k) lies on an
// earlier hyperplane w = i + 2 j + 4 k, so the rows of one hyperplane are
// independent: the factorization and both sweeps run hyperplane by hyperplane,
// one launch per hyperplane, over row lists built on the host.  Factor record of
// a row: 3^d values in stencil-offset order, the ILU(0) multipliers l_ij at the
// lower offsets, 1/u_ii at the centre and u_ij at the upper offsets.
#include <algorithm>
#include <vector>

#include "lor_internal.h"

namespace {

__device__ __forceinline__ bool interior(int dim, const int* N, int I, int J, int K) {
  return I > 0 && I < N[0] - 1 && J > 0 && J < N[1] - 1 && (dim == 2 || (K > 0 && K < N[2] - 1));
}

struct GridArg {
  int dim;
  int N[3];
  long long ntot;
};

__device__ __forceinline__ void offs(int dim, int o, int& dx, int& dy, int& dz) {
  dx = o % 3 - 1;
  dy = (o / 3) % 3 - 1;
  dz = dim == 3 ? o / 9 - 1 : 0;
}

// ILU(0) of the rows of one hyperplane (IKJ form: for each lower neighbour k in
// increasing order, a_ik /= u_kk, then a_ij -= a_ik u_kj for the upper entries j of
// row k inside row i's pattern).  A non-positive pivot sets status bit 2.
__global__ void k_s_ilu(GridArg g, const double* __restrict__ S, const int* __restrict__ rows, int cnt,
                        double* __restrict__ F, int* status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int NS = g.dim == 3 ? 27 : 9, C = NS / 2;
  const long long G = rows[t];
  const int I = (int)(G % g.N[0]), J = (int)((G / g.N[0]) % g.N[1]), K = (int)(G / ((long long)g.N[0] * g.N[1]));
  double a[27];
  bool in[27];
  for (int o = 0; o < NS; ++o) {
    int dx, dy, dz;
    offs(g.dim, o, dx, dy, dz);
    in[o] = interior(g.dim, g.N, I + dx, J + dy, K + dz);
    a[o] = in[o] ? S[(long long)o * g.ntot + G] : 0.0;
  }
  for (int o = 0; o < C; ++o) {
    if (!in[o]) continue;
    int dx, dy, dz;
    offs(g.dim, o, dx, dy, dz);
    const long long Gk = G + ((long long)dz * g.N[1] + dy) * g.N[0] + dx;
    const double* Fk = F + Gk * NS;
    a[o] *= Fk[C];
    const double l = a[o];
    for (int o2 = C + 1; o2 < NS; ++o2) {
      int ex, ey, ez;
      offs(g.dim, o2, ex, ey, ez);
      const int fx = dx + ex, fy = dy + ey, fz = dz + ez;
      if (fx < -1 || fx > 1 || fy < -1 || fy > 1 || fz < -1 || fz > 1) continue;
      const int oj = g.dim == 3 ? (fz + 1) * 9 + (fy + 1) * 3 + (fx + 1) : (fy + 1) * 3 + (fx + 1);
      if (in[oj]) a[oj] -= l * Fk[o2];
    }
  }
  double* Fi = F + G * NS;
  if (!(a[C] > 0.0)) {
    atomicOr(status, 2);
    for (int o = 0; o < NS; ++o) Fi[o] = 0.0;
    return;
  }
  for (int o = 0; o < NS; ++o) Fi[o] = o == C ? 1.0 / a[C] : a[o];
}

__global__ void k_s_to32(const double* __restrict__ a, float* __restrict__ b, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// forward sweep on one hyperplane: y_i = b_i - sum_{j lower} l_ij y_j
template <typename T>
__global__ void k_s_fwd(GridArg g, const T* __restrict__ F, const int* __restrict__ rows, int cnt,
                        const T* __restrict__ b, T* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int NS = g.dim == 3 ? 27 : 9, C = NS / 2;
  const long long G = rows[t];
  const int I = (int)(G % g.N[0]), J = (int)((G / g.N[0]) % g.N[1]), K = (int)(G / ((long long)g.N[0] * g.N[1]));
  const T* Fi = F + G * NS;
  T s = b[G];
  for (int o = 0; o < C; ++o) {
    int dx, dy, dz;
    offs(g.dim, o, dx, dy, dz);
    if (interior(g.dim, g.N, I + dx, J + dy, K + dz)) s -= Fi[o] * y[G + ((long long)dz * g.N[1] + dy) * g.N[0] + dx];
  }
  y[G] = s;
}

// backward sweep on one hyperplane: x_i = (y_i - sum_{j upper} u_ij x_j) / u_ii
template <typename T>
__global__ void k_s_bwd(GridArg g, const T* __restrict__ F, const int* __restrict__ rows, int cnt,
                        const T* __restrict__ y, T* __restrict__ x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int NS = g.dim == 3 ? 27 : 9, C = NS / 2;
  const long long G = rows[t];
  const int I = (int)(G % g.N[0]), J = (int)((G / g.N[0]) % g.N[1]), K = (int)(G / ((long long)g.N[0] * g.N[1]));
  const T* Fi = F + G * NS;
  T s = y[G];
  for (int o = C + 1; o < NS; ++o) {
    int dx, dy, dz;
    offs(g.dim, o, dx, dy, dz);
    if (interior(g.dim, g.N, I + dx, J + dy, K + dz)) s -= Fi[o] * x[G + ((long long)dz * g.N[1] + dy) * g.N[0] + dx];
  }
  x[G] = Fi[C] * s;
}

// y = b - A x on the interior nodes of a level grid (A its stencil with the Dirichlet
// rows and columns dropped), 0 on the boundary
template <typename T>
__global__ void k_s_resid(GridArg g, const T* __restrict__ S, const T* __restrict__ b, const T* __restrict__ x,
                          T* __restrict__ y) {
  const long long G = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (G >= g.ntot) return;
  const int I = (int)(G % g.N[0]), J = (int)((G / g.N[0]) % g.N[1]), K = (int)(G / ((long long)g.N[0] * g.N[1]));
  if (!interior(g.dim, g.N, I, J, K)) {
    y[G] = T(0);
    return;
  }
  const int NS = g.dim == 3 ? 27 : 9;
  T s = 0;
  for (int o = 0; o < NS; ++o) {
    int dx, dy, dz;
    offs(g.dim, o, dx, dy, dz);
    if (interior(g.dim, g.N, I + dx, J + dy, K + dz))
      s += S[(long long)o * g.ntot + G] * x[G + ((long long)dz * g.N[1] + dy) * g.N[0] + dx];
  }
  y[G] = b[G] - s;
}

// one restriction pass along `axis`: out[.., c, ..] = sum_{f in R(c)} w_f in[.., f, ..];
// out has extents n (n[axis] = coarse length), in the same with nf along axis.
// mask: the last pass, zero on the boundary of the coarse grid g.
template <typename T>
__global__ void k_s_restrict(int axis, int n0, int n1, int n2, int nf, const int* __restrict__ ptr,
                             const int* __restrict__ idx, const double* __restrict__ w, const T* __restrict__ in,
                             T* __restrict__ out, int mask, GridArg g) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)n0 * n1 * n2;
  if (q >= nt) return;
  const int i0 = (int)(q % n0), i1 = (int)((q / n0) % n1), i2 = (int)(q / ((long long)n0 * n1));
  if (mask && !interior(g.dim, g.N, i0, i1, i2)) {
    out[q] = T(0);
    return;
  }
  const int c = axis == 0 ? i0 : axis == 1 ? i1 : i2;
  const int m0 = axis == 0 ? nf : n0, m1 = axis == 1 ? nf : n1;
  T s = 0;
  for (int e = ptr[c]; e < ptr[c + 1]; ++e) {
    const int f = idx[e];
    const long long src = axis == 0 ? ((long long)i2 * m1 + i1) * m0 + f
                        : axis == 1 ? ((long long)i2 * m1 + f) * m0 + i0
                                    : ((long long)f * m1 + i1) * m0 + i0;
    s += T(w[e]) * in[src];
  }
  out[q] = s;
}

// one prolongation pass along `axis`: out[.., f, ..] = w0 in[.., c0, ..] + w1 in[.., c1, ..];
// out has extents n (n[axis] = fine length), in the same with nc along axis.
// add: the last pass, x += out on the interior of the fine grid g.
template <typename T>
__global__ void k_s_prolong(int axis, int n0, int n1, int n2, int nc, const Prolong1D* __restrict__ P,
                            const T* __restrict__ in, T* __restrict__ out, int add, GridArg g) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)n0 * n1 * n2;
  if (q >= nt) return;
  const int i0 = (int)(q % n0), i1 = (int)((q / n0) % n1), i2 = (int)(q / ((long long)n0 * n1));
  const int f = axis == 0 ? i0 : axis == 1 ? i1 : i2;
  const int m0 = axis == 0 ? nc : n0, m1 = axis == 1 ? nc : n1;
  const Prolong1D pf = P[f];
  T s = 0;
  const int cs[2] = {pf.c0, pf.c1};
  const double ws[2] = {pf.w0, pf.w1};
  for (int u = 0; u < 2; ++u) {
    if (cs[u] < 0 || ws[u] == 0.0) continue;
    const int cc = cs[u];
    const long long src = axis == 0 ? ((long long)i2 * m1 + i1) * m0 + cc
                        : axis == 1 ? ((long long)i2 * m1 + cc) * m0 + i0
                                    : ((long long)cc * m1 + i1) * m0 + i0;
    s += T(ws[u]) * in[src];
  }
  if (add) {
    if (interior(g.dim, g.N, i0, i1, i2)) out[q] += s;
  } else {
    out[q] = s;
  }
}

template <typename T>
__global__ void k_s_add(T* __restrict__ x, const T* __restrict__ d, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += d[i];
}

template <typename T>
__global__ void k_s_copy_masked(GridArg g, const T* __restrict__ a, T* __restrict__ b) {
  const long long G = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (G >= g.ntot) return;
  const int I = (int)(G % g.N[0]), J = (int)((G / g.N[0]) % g.N[1]), K = (int)(G / ((long long)g.N[0] * g.N[1]));
  b[G] = interior(g.dim, g.N, I, J, K) ? a[G] : T(0);
}

GridArg grid_of(const lor_ctx* c, int l) {
  GridArg g;
  g.dim = c->dim;
  for (int a = 0; a < 3; ++a) g.N[a] = c->lev[l].N[a];
  g.ntot = c->lev[l].ntot;
  return g;
}

unsigned nblk(long long n) { return (unsigned)std::max<long long>(1, lor_ceil_div(n, 256)); }

long long interior_count(const lor_ctx* c, int l) {
  long long m = 1;
  for (int a = 0; a < c->dim; ++a) m *= std::max(c->lev[l].N[a] - 2, 0);
  return m;
}

}  // namespace

struct SingleState {
  int levels = 0;                           // smoothed levels (0 .. L-2)
  std::vector<int> front_off[LOR_MAXLEV];   // hyperplane offsets into the row list
  int* d_rows[LOR_MAXLEV] = {};
  double* F64[LOR_MAXLEV] = {};
  float* F32[LOR_MAXLEV] = {};
  // per level: r, x, t, w (float64-sized) and two transfer buffers
  double* vec[LOR_MAXLEV][6] = {};
  // the apply as a CUDA graph per precision (index 0 FP64, 1 FP32), for one (r, z) pair:
  // its thousands of hyperplane launches replay as one graph launch
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec[2] = {};
  const void* gr[2] = {};
  void* gz[2] = {};
  long long glaunches[2] = {};
  ~SingleState() {
    for (int q = 0; q < 2; ++q)
      if (exec[q]) cudaGraphExecDestroy(exec[q]);
    if (cap) cudaStreamDestroy(cap);
  }
};

static SingleState* SS(lor_ctx* c) { return (SingleState*)c->single; }

void lor_free_single(lor_ctx* c) {
  delete SS(c);
  c->single = nullptr;
}

lor_status lor_single_prepare(lor_ctx* c) {
  if (c->single) return LOR_OK;
  SingleState* s = new SingleState();
  c->single = s;
  s->levels = c->L - 1;
  const int NS = c->NS;
  for (int l = 0; l < s->levels; ++l) {
    const GridArg g = grid_of(c, l);
    const int M[3] = {std::max(g.N[0] - 2, 0), std::max(g.N[1] - 2, 0), c->dim == 3 ? std::max(g.N[2] - 2, 0) : 1};
    const int nfront = (M[0] > 0 && M[1] > 0 && M[2] > 0) ? (M[0] - 1) + 2 * (M[1] - 1) + 4 * (M[2] - 1) + 1 : 0;
    std::vector<int> cnt(nfront + 1, 0);
    for (int k = 0; k < M[2]; ++k)
      for (int j = 0; j < M[1]; ++j)
        for (int i = 0; i < M[0]; ++i) ++cnt[i + 2 * j + 4 * k + 1];
    for (int w = 0; w < nfront; ++w) cnt[w + 1] += cnt[w];
    s->front_off[l] = cnt;
    std::vector<int> rows(std::max<long long>((long long)M[0] * M[1] * M[2], 1));
    std::vector<int> pos(cnt.begin(), cnt.end() - (nfront > 0 ? 1 : 0));
    const int K0 = c->dim == 3 ? 1 : 0;
    for (int k = 0; k < M[2]; ++k)
      for (int j = 0; j < M[1]; ++j)
        for (int i = 0; i < M[0]; ++i)
          rows[pos[i + 2 * j + 4 * k]++] = (int)(((long long)(k + K0) * g.N[1] + (j + 1)) * g.N[0] + (i + 1));
    if (g.ntot > 0x7fffffffLL) return lor_fail(c, LOR_EINVAL, "single patch: level grid too large");
    s->d_rows[l] = (int*)lor_alloc(c, rows.size() * 4);
    s->F64[l] = (double*)lor_alloc(c, (size_t)g.ntot * NS * 8);
    s->F32[l] = (float*)lor_alloc(c, (size_t)g.ntot * NS * 4);
    for (int q = 0; q < 6; ++q) s->vec[l][q] = (double*)lor_alloc(c, (size_t)g.ntot * 8);
    bool ok = s->d_rows[l] && s->F64[l] && s->F32[l];
    for (int q = 0; q < 6; ++q) ok = ok && s->vec[l][q];
    if (!ok) return lor_fail(c, LOR_ENOMEM, "alloc single-patch factors");
    cudaMemcpyAsync(s->d_rows[l], rows.data(), rows.size() * 4, cudaMemcpyHostToDevice, c->stream);
    cudaMemsetAsync(s->F64[l], 0, (size_t)g.ntot * NS * 8, c->stream);
    for (int q = 0; q < 6; ++q) cudaMemsetAsync(s->vec[l][q], 0, (size_t)g.ntot * 8, c->stream);
    for (int w = 0; w < nfront; ++w) {
      const int n = cnt[w + 1] - cnt[w];
      k_s_ilu<<<nblk(n), 256, 0, c->stream>>>(g, c->d_S64[l], s->d_rows[l] + cnt[w], n, s->F64[l], c->d_status);
      ++c->launches;
    }
    const long long nf = g.ntot * NS;
    k_s_to32<<<nblk(nf), 256, 0, c->stream>>>(s->F64[l], s->F32[l], nf);
    ++c->launches;
    // the host row list must outlive the asynchronous copy
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return lor_cuda_check(c, e, "single-patch ILU(0)");
  }
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "single-patch ILU(0)");
  if (st & 2) return lor_fail(c, LOR_EBREAKDOWN, "single-patch ILU(0) breakdown: non-positive pivot");
  return LOR_OK;
}

namespace {

template <typename T> const T* factors(SingleState* s, int l);
template <> const double* factors<double>(SingleState* s, int l) { return s->F64[l]; }
template <> const float* factors<float>(SingleState* s, int l) { return s->F32[l]; }

template <typename T> const T* stencil(lor_ctx* c, int l);
template <> const double* stencil<double>(lor_ctx* c, int l) { return c->d_S64[l]; }
template <> const float* stencil<float>(lor_ctx* c, int l) { return c->d_S32[l]; }

// x = (L U)^{-1} b on level l; y: scratch
template <typename T>
void ilu_solve(lor_ctx* c, int l, const T* b, T* y, T* x) {
  SingleState* s = SS(c);
  const GridArg g = grid_of(c, l);
  const std::vector<int>& off = s->front_off[l];
  const int nfront = (int)off.size() - 1;
  const T* F = factors<T>(s, l);
  for (int w = 0; w < nfront; ++w) {
    const int n = off[w + 1] - off[w];
    k_s_fwd<T><<<nblk(n), 256, 0, c->stream>>>(g, F, s->d_rows[l] + off[w], n, b, y);
  }
  for (int w = nfront - 1; w >= 0; --w) {
    const int n = off[w + 1] - off[w];
    k_s_bwd<T><<<nblk(n), 256, 0, c->stream>>>(g, F, s->d_rows[l] + off[w], n, y, x);
  }
  c->launches += 2 * nfront;
}

// out (level l+1 grid, boundary 0) = P_l^T in (level l grid); t1, t2: scratch of the fine size
template <typename T>
void restrict_to(lor_ctx* c, int l, const T* in, T* out, T* t1, T* t2) {
  const GridArg gf = grid_of(c, l), gc = grid_of(c, l + 1);
  int n[3] = {gf.N[0], gf.N[1], gf.N[2]};
  const T* src = in;
  for (int a = 0; a < c->dim; ++a) {
    const int nf = n[a];
    n[a] = gc.N[a];
    const bool last = a == c->dim - 1;
    T* dst = last ? out : (a == 0 ? t1 : t2);
    const long long nt = (long long)n[0] * n[1] * n[2];
    k_s_restrict<T><<<nblk(nt), 256, 0, c->stream>>>(a, n[0], n[1], n[2], nf, c->d_R1ptr[l][a], c->d_R1idx[l][a],
                                                     c->d_R1w[l][a], src, dst, last ? 1 : 0, gc);
    ++c->launches;
    src = dst;
  }
}

// x (level l grid, interior) += P_l e (e on the level l+1 grid); t1, t2: scratch of the fine size
template <typename T>
void prolong_add(lor_ctx* c, int l, const T* e, T* x, T* t1, T* t2) {
  const GridArg gf = grid_of(c, l), gc = grid_of(c, l + 1);
  int n[3] = {gc.N[0], gc.N[1], gc.N[2]};
  const T* src = e;
  for (int a = c->dim - 1; a >= 0; --a) {
    const int nc = n[a];
    n[a] = gf.N[a];
    const bool last = a == 0;
    T* dst = last ? x : (a == c->dim - 1 ? t1 : t2);
    const long long nt = (long long)n[0] * n[1] * n[2];
    k_s_prolong<T><<<nblk(nt), 256, 0, c->stream>>>(a, n[0], n[1], n[2], nc, c->d_P1[l][a], src, dst, last ? 1 : 0,
                                                    gf);
    ++c->launches;
    src = dst;
  }
}

// x = V(1,1) r on level l (both on the level grid, boundary entries 0)
template <typename T>
lor_status vcycle(lor_ctx* c, int l, const T* r, T* x) {
  SingleState* s = SS(c);
  const GridArg g = grid_of(c, l);
  T* t = (T*)s->vec[l][2];
  T* w = (T*)s->vec[l][3];
  T* t1 = (T*)s->vec[l][4];
  T* t2 = (T*)s->vec[l][5];
  const T* S = stencil<T>(c, l);
  cudaMemsetAsync(x, 0, g.ntot * sizeof(T), c->stream);
  ilu_solve<T>(c, l, r, w, x);   // pre-smoothing from x = 0
  if (interior_count(c, l + 1) > 0) {   // the next level has unknowns
    k_s_resid<T><<<nblk(g.ntot), 256, 0, c->stream>>>(g, S, r, x, t);
    ++c->launches;
    T* rc;
    T* ec;
    if (l + 1 == c->L - 1) {     // vertex level: R_0 (the coarse space's V-cycle)
      rc = lor_coarse_rhs<T>(c);
      restrict_to<T>(c, l, t, rc, t1, t2);
      ec = lor_coarse_solve<T>(c);
    } else {
      rc = (T*)s->vec[l + 1][0];
      ec = (T*)s->vec[l + 1][1];
      restrict_to<T>(c, l, t, rc, t1, t2);
      if (vcycle<T>(c, l + 1, rc, ec)) return LOR_ECUDA;
    }
    prolong_add<T>(c, l, ec, x, t1, t2);
  }
  k_s_resid<T><<<nblk(g.ntot), 256, 0, c->stream>>>(g, S, r, x, t);
  ++c->launches;
  // post-smoothing: the backward sweep overwrites t (its forward sweep has read it),
  // whose boundary entries the residual left at 0
  ilu_solve<T>(c, l, t, w, t);
  k_s_add<T><<<nblk(g.ntot), 256, 0, c->stream>>>(x, t, g.ntot);
  ++c->launches;
  return lor_cuda_check(c, cudaGetLastError(), "single-patch V-cycle");
}

}  // namespace

namespace {

template <typename T>
lor_status single_apply_launches(lor_ctx* c, const T* r, T* z) {
  SingleState* s = SS(c);
  const GridArg g0 = grid_of(c, 0);
  if (s->levels == 0) {          // p = 1: the level grid is the vertex grid, B(1) = R_0
    if (interior_count(c, 0) == 0)
      return lor_cuda_check(c, cudaMemsetAsync(z, 0, g0.ntot * sizeof(T), c->stream), "B(1)");
    T* rc = lor_coarse_rhs<T>(c);
    k_s_copy_masked<T><<<nblk(g0.ntot), 256, 0, c->stream>>>(g0, r, rc);
    const T* ec = lor_coarse_solve<T>(c);
    k_s_copy_masked<T><<<nblk(g0.ntot), 256, 0, c->stream>>>(g0, ec, z);
    c->launches += 2;
    return lor_cuda_check(c, cudaGetLastError(), "B(1)");
  }
  // the caller's r may hold boundary values: take its interior part
  T* r0 = (T*)s->vec[0][0];
  k_s_copy_masked<T><<<nblk(g0.ntot), 256, 0, c->stream>>>(g0, r, r0);
  ++c->launches;
  return vcycle<T>(c, 0, r0, z);
}

}  // namespace

// The apply is captured once per (r, z, precision) into a CUDA graph on a private
// stream and replayed on the context's stream; inside an enclosing capture (a batch)
// its kernels are launched directly.
template <typename T>
lor_status lor_single_apply(lor_ctx* c, const T* r, T* z) {
  SingleState* s = SS(c);
  if (!s) return lor_fail(c, LOR_ESTATE, "single-patch preconditioner not prepared");
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c->stream, &cst) != cudaSuccess || cst != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return single_apply_launches<T>(c, r, z);
  }
  const int q = sizeof(T) == 8 ? 0 : 1;
  if (!(s->exec[q] && s->gr[q] == (const void*)r && s->gz[q] == (void*)z)) {
    if (s->exec[q]) { cudaGraphExecDestroy(s->exec[q]); s->exec[q] = nullptr; }
    if (!s->cap && cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking) != cudaSuccess)
      return lor_fail(c, LOR_ECUDA, "B(1): capture stream");
    const cudaStream_t keep = c->stream;
    const long long l0 = c->launches;
    c->stream = s->cap;
    if (cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      c->stream = keep;
      return lor_fail(c, LOR_ECUDA, "B(1): begin capture");
    }
    const lor_status st = single_apply_launches<T>(c, r, z);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s->cap, &g);
    c->stream = keep;
    if (st || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return st ? st : lor_fail(c, LOR_ECUDA, "B(1): capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(&s->exec[q], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      s->exec[q] = nullptr;
      cudaGetLastError();
      return lor_fail(c, LOR_ECUDA, "B(1): graph instantiate");
    }
    s->gr[q] = r;
    s->gz[q] = z;
    s->glaunches[q] = c->launches - l0;
    c->launches = l0;
  }
  c->launches += s->glaunches[q];
  return lor_cuda_check(c, cudaGraphLaunch(s->exec[q], c->stream), "B(1) graph launch");
}

template lor_status lor_single_apply<double>(lor_ctx*, const double*, double*);
template lor_status lor_single_apply<float>(lor_ctx*, const float*, float*);
