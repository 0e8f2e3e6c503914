// Matrix-free sum-factorized Q_p stiffness apply (Section 2; Section 3.6 Table 1:
// O(p^{d+1}) work per element).  y = sum_e E_e^T B^T G_e B E_e x with
//   B      : interpolation from the (p+1) GLL nodes to the q = p+1 Gauss points,
//            followed by the collocated Gauss-point derivative Dq (so that
//            grad = (Dq x B) u needs 2d instead of d^2 1D contractions),
//   G_e(q) : kappa_e w_q det J_q J_q^{-1} J_q^{-T}  (symmetric, precomputed),
//   E_e    : gather of the element's nodes from the structured node grid.
// One thread per (x,y) node column of an element (3D: the z column lives in
// registers, x/y contractions go through shared memory); several elements per
// CTA for small p.  The elements run in 2^d colour classes (element index parity
// per axis), one launch per class in a fixed order: elements of one class share
// no node, so element-interior outputs are stored and shared ones added without
// atomics, and y is the same bit for bit on every run.  Global boundary
// (Dirichlet) nodes read as 0 and are never written.
#include <mutex>

#include "lor_internal.h"
#include "geom.cuh"

namespace {

template <int P>
struct ElemsPerBlock {
  static constexpr int Q = P + 1;
  static constexpr int v2 = (256 / (Q * Q)) > 0 ? (256 / (Q * Q)) : 1;
};

// Elements per CTA of the 3D kernel for tile variant V (0: ~128, 1: ~256,
// 2: ~512 threads), capped so that the two shared tiles fit in 48 KB.
template <int P, typename T, int V>
struct TileNE {
  static constexpr int Q = P + 1;
  static constexpr int want = ((128 << V) / (Q * Q)) > 0 ? ((128 << V) / (Q * Q)) : 1;
  static constexpr int cap = (48 * 1024) / (2 * Q * Q * Q * (int)sizeof(T) + 1);
  static constexpr int v = want < cap ? want : (cap > 0 ? cap : 1);
};

// DGM = false: continuous Q_p on the structured node grid (gather/scatter,
// Dirichlet nodes masked).  DGM = true: element-local DG blocks of (p+1)^3
// values (element e at e*(p+1)^3), no masking, outputs stored (not added).
// color >= 0: the elements of colour class color (bit a = element index parity
// along axis a); color < 0: all elements (DG blocks, which share no node).
template <int P, typename T, bool DGM, int NE>
__global__ void __launch_bounds__(1024) k_apply3d(int nx, int ny, int nz, int color, const T* __restrict__ Bg,
                                                  const T* __restrict__ Dg, const T* __restrict__ G,
                                                  const T* __restrict__ x, T* __restrict__ y,
                                                  const double* __restrict__ conv) {
  if (conv && *conv != 0.0) return;   // converged member of a batched solve: nothing to do
  constexpr int Q = P + 1;
  constexpr int Q2 = Q * Q, Q3 = Q * Q * Q;
  __shared__ T sB[Q2], sD[Q2];
  __shared__ T s1[NE][Q3], s2[NE][Q3];
  const int tid = threadIdx.x;
  const int el = tid / Q2, rem = tid - el * Q2;
  const int tx = rem % Q, ty = rem / Q;
  for (int i = tid; i < Q2; i += blockDim.x) { sB[i] = Bg[i]; sD[i] = Dg[i]; }
  const long long ie = (long long)blockIdx.x * NE + el;
  const int Nx = nx * P + 1, Ny = ny * P + 1, Nz = nz * P + 1;
  int ex = 0, ey = 0, ez = 0;
  bool live;
  if (color < 0) {
    live = (el < NE) && (ie < (long long)nx * ny * nz);
    if (live) { ex = (int)(ie % nx); ey = (int)((ie / nx) % ny); ez = (int)(ie / ((long long)nx * ny)); }
  } else {
    const int cx = color & 1, cy = (color >> 1) & 1, cz = (color >> 2) & 1;
    const int mx = (nx - cx + 1) / 2, my = (ny - cy + 1) / 2, mz = (nz - cz + 1) / 2;
    live = (el < NE) && (ie < (long long)mx * my * mz);
    if (live) {
      ex = 2 * (int)(ie % mx) + cx; ey = 2 * (int)((ie / mx) % my) + cy; ez = 2 * (int)(ie / ((long long)mx * my)) + cz;
    }
  }
  const long long e = ((long long)ez * ny + ey) * nx + ex;
  const int I = ex * P + tx, Jn = ey * P + ty;
  const bool bxy = !DGM && (I == 0 || I == Nx - 1 || Jn == 0 || Jn == Ny - 1);
  T u[Q], v[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    const int K = ez * P + k;
    const bool bnd = bxy || (!DGM && (K == 0 || K == Nz - 1));
    if (DGM)
      u[k] = live ? x[e * Q3 + (k * Q + ty) * Q + tx] : T(0);
    else
      u[k] = (live && !bnd) ? x[((long long)K * Ny + Jn) * Nx + I] : T(0);
  }
  __syncthreads();
  T* S1 = s1[el < NE ? el : 0];
  T* S2 = s2[el < NE ? el : 0];
  // z: nodes -> Gauss points (registers)
#pragma unroll
  for (int qz = 0; qz < Q; ++qz) {
    T a = 0;
#pragma unroll
    for (int k = 0; k < Q; ++k) a += sB[qz * Q + k] * u[k];
    v[qz] = a;
  }
  if (el < NE) {
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) S1[(qz * Q + ty) * Q + tx] = v[qz];
  }
  __syncthreads();
  // y: (thread ty acts as qy)
#pragma unroll
  for (int qz = 0; qz < Q; ++qz) {
    T a = 0;
#pragma unroll
    for (int j = 0; j < Q; ++j) a += sB[ty * Q + j] * S1[(qz * Q + j) * Q + tx];
    u[qz] = a;
  }
  __syncthreads();
  if (el < NE) {
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) S1[(qz * Q + ty) * Q + tx] = u[qz];
  }
  __syncthreads();
  // x: (thread tx acts as qx) -> v = u at Gauss point (tx, ty, qz)
#pragma unroll
  for (int qz = 0; qz < Q; ++qz) {
    T a = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) a += sB[tx * Q + i] * S1[(qz * Q + ty) * Q + i];
    v[qz] = a;
  }
  __syncthreads();
  if (el < NE) {
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) S1[(qz * Q + ty) * Q + tx] = v[qz];
  }
  __syncthreads();
  // reference gradient at Gauss points, then G * grad
  T gx[Q], gy[Q], gz[Q];
#pragma unroll
  for (int qz = 0; qz < Q; ++qz) {
    T a = 0, b = 0, c = 0;
#pragma unroll
    for (int k = 0; k < Q; ++k) c += sD[qz * Q + k] * v[k];
#pragma unroll
    for (int j = 0; j < Q; ++j) b += sD[ty * Q + j] * S1[(qz * Q + j) * Q + tx];
#pragma unroll
    for (int i = 0; i < Q; ++i) a += sD[tx * Q + i] * S1[(qz * Q + ty) * Q + i];
    T g00 = 0, g01 = 0, g02 = 0, g11 = 0, g12 = 0, g22 = 0;
    if (live) {
      const T* Ge = G + e * 6 * Q3 + (qz * Q + ty) * Q + tx;
      g00 = Ge[0]; g01 = Ge[Q3]; g02 = Ge[2 * Q3]; g11 = Ge[3 * Q3]; g12 = Ge[4 * Q3]; g22 = Ge[5 * Q3];
    }
    gx[qz] = g00 * a + g01 * b + g02 * c;
    gy[qz] = g01 * a + g11 * b + g12 * c;
    gz[qz] = g02 * a + g12 * b + g22 * c;
  }
  __syncthreads();
  if (el < NE) {
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) {
      S1[(qz * Q + ty) * Q + tx] = gx[qz];
      S2[(qz * Q + ty) * Q + tx] = gy[qz];
    }
  }
  __syncthreads();
  // transposed derivative: w = Dq_x^T gx + Dq_y^T gy + Dq_z^T gz
#pragma unroll
  for (int qz = 0; qz < Q; ++qz) {
    T a = 0;
#pragma unroll
    for (int k = 0; k < Q; ++k) a += sD[k * Q + qz] * gz[k];
#pragma unroll
    for (int j = 0; j < Q; ++j) a += sD[j * Q + ty] * S2[(qz * Q + j) * Q + tx];
#pragma unroll
    for (int i = 0; i < Q; ++i) a += sD[i * Q + tx] * S1[(qz * Q + ty) * Q + i];
    v[qz] = a;
  }
  __syncthreads();
  if (el < NE) {
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) S1[(qz * Q + ty) * Q + tx] = v[qz];
  }
  __syncthreads();
  // transposed interpolation: x (tx = node i), y (ty = node j), z (registers)
#pragma unroll
  for (int qz = 0; qz < Q; ++qz) {
    T a = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) a += sB[i * Q + tx] * S1[(qz * Q + ty) * Q + i];
    u[qz] = a;
  }
  __syncthreads();
  if (el < NE) {
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) S1[(qz * Q + ty) * Q + tx] = u[qz];
  }
  __syncthreads();
#pragma unroll
  for (int qz = 0; qz < Q; ++qz) {
    T a = 0;
#pragma unroll
    for (int j = 0; j < Q; ++j) a += sB[j * Q + ty] * S1[(qz * Q + j) * Q + tx];
    v[qz] = a;
  }
  if (!live) return;
  const bool inx = (tx > 0 && tx < P), iny = (ty > 0 && ty < P);
#pragma unroll
  for (int k = 0; k < Q; ++k) {
    T a = 0;
#pragma unroll
    for (int qz = 0; qz < Q; ++qz) a += sB[qz * Q + k] * v[qz];
    if (DGM) {
      y[e * Q3 + (k * Q + ty) * Q + tx] = a;
      continue;
    }
    const int K = ez * P + k;
    if (bxy || K == 0 || K == Nz - 1) continue;
    T* dst = y + ((long long)K * Ny + Jn) * Nx + I;
    if (inx && iny && k > 0 && k < P) *dst = a;
    else *dst += a;   // no other element of this colour class touches the node
  }
}

template <int P, typename T>
__global__ void __launch_bounds__(256) k_apply2d(int nx, int ny, int color, const T* __restrict__ Bg,
                                                 const T* __restrict__ Dg, const T* __restrict__ G,
                                                 const T* __restrict__ x, T* __restrict__ y,
                                                 const double* __restrict__ conv) {
  if (conv && *conv != 0.0) return;   // converged member of a batched solve: nothing to do
  constexpr int Q = P + 1;
  constexpr int Q2 = Q * Q;
  constexpr int NE = ElemsPerBlock<P>::v2;
  __shared__ T sB[Q2], sD[Q2];
  __shared__ T s1[NE][Q2], s2[NE][Q2];
  const int tid = threadIdx.x;
  const int el = tid / Q2, rem = tid - el * Q2;
  const int tx = rem % Q, ty = rem / Q;
  for (int i = tid; i < Q2; i += blockDim.x) { sB[i] = Bg[i]; sD[i] = Dg[i]; }
  const long long ie = (long long)blockIdx.x * NE + el;
  const int cx = color & 1, cy = (color >> 1) & 1;
  const int mx = (nx - cx + 1) / 2, my = (ny - cy + 1) / 2;
  const bool live = (el < NE) && (ie < (long long)mx * my);
  const int Nx = nx * P + 1, Ny = ny * P + 1;
  int ex = 0, ey = 0;
  if (live) { ex = 2 * (int)(ie % mx) + cx; ey = 2 * (int)(ie / mx) + cy; }
  const long long e = (long long)ey * nx + ex;
  const int I = ex * P + tx, Jn = ey * P + ty;
  const bool bnd = (I == 0 || I == Nx - 1 || Jn == 0 || Jn == Ny - 1);
  T* S1 = s1[el < NE ? el : 0];
  T* S2 = s2[el < NE ? el : 0];
  T u = (live && !bnd) ? x[(long long)Jn * Nx + I] : T(0);
  __syncthreads();
  if (el < NE) S1[ty * Q + tx] = u;
  __syncthreads();
  T a = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) a += sB[tx * Q + i] * S1[ty * Q + i];      // (qx, node j)
  __syncthreads();
  if (el < NE) S2[ty * Q + tx] = a;
  __syncthreads();
  T v = 0;
#pragma unroll
  for (int j = 0; j < Q; ++j) v += sB[ty * Q + j] * S2[j * Q + tx];      // (qx, qy)
  __syncthreads();
  if (el < NE) S1[ty * Q + tx] = v;
  __syncthreads();
  T ga = 0, gb = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) ga += sD[tx * Q + i] * S1[ty * Q + i];
#pragma unroll
  for (int j = 0; j < Q; ++j) gb += sD[ty * Q + j] * S1[j * Q + tx];
  T g00 = 0, g01 = 0, g11 = 0;
  if (live) {
    const T* Ge = G + e * 3 * Q2 + ty * Q + tx;
    g00 = Ge[0]; g01 = Ge[Q2]; g11 = Ge[2 * Q2];
  }
  const T gx = g00 * ga + g01 * gb, gy = g01 * ga + g11 * gb;
  __syncthreads();
  if (el < NE) { S1[ty * Q + tx] = gx; S2[ty * Q + tx] = gy; }
  __syncthreads();
  T w = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) w += sD[i * Q + tx] * S1[ty * Q + i];
#pragma unroll
  for (int j = 0; j < Q; ++j) w += sD[j * Q + ty] * S2[j * Q + tx];
  __syncthreads();
  if (el < NE) S1[ty * Q + tx] = w;
  __syncthreads();
  a = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) a += sB[i * Q + tx] * S1[ty * Q + i];      // (node i, qy)
  __syncthreads();
  if (el < NE) S2[ty * Q + tx] = a;
  __syncthreads();
  T out = 0;
#pragma unroll
  for (int j = 0; j < Q; ++j) out += sB[j * Q + ty] * S2[j * Q + tx];
  if (!live || bnd) return;
  T* dst = y + (long long)Jn * Nx + I;
  if (tx > 0 && tx < P && ty > 0 && ty < P) *dst = out;
  else *dst += out;   // no other element of this colour class touches the node
}

template <typename T>
struct BasisDev {
  const T* B;
  const T* D;
};

template <typename T>
lor_status launch_apply(lor_ctx* c, const T* B, const T* D, const T* G, const T* x, T* y) {
  const long long nvec = c->lev[0].ntot;
  cudaError_t e = cudaMemsetAsync(y, 0, sizeof(T) * nvec, c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "apply_A memset");
  const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
  const int pk = sizeof(T) == 8 ? 2 : 3;
  lor_prof_begin(c, pk);
  const int ncolor = c->dim == 3 ? 8 : 4;
  for (int color = 0; color < ncolor; ++color) {
    const int cx = color & 1, cy = (color >> 1) & 1, cz = (color >> 2) & 1;
    const long long ncls = (long long)((nx - cx + 1) / 2) * ((ny - cy + 1) / 2) * (c->dim == 3 ? (nz - cz + 1) / 2 : 1);
    if (ncls == 0) continue;
#define LOR_VAR3(PP, V)                                                                     \
  {                                                                                         \
    constexpr int NE = TileNE<PP, T, V>::v;                                                 \
    const int threads = NE * (PP + 1) * (PP + 1);                                           \
    const long long blocks = lor_ceil_div(ncls, NE);                                        \
    k_apply3d<PP, T, false, NE><<<(unsigned)blocks, threads, 0, c->stream>>>(nx, ny, nz, color, B, D, G, x, y, c->conv_flag); \
  }
#define LOR_CASE3(PP)                                                                       \
  case PP: {                                                                                \
    if (c->dim == 3) {                                                                      \
      if (c->tune_ne == 0) LOR_VAR3(PP, 0)                                                  \
      else if (c->tune_ne == 2) LOR_VAR3(PP, 2)                                             \
      else LOR_VAR3(PP, 1)                                                                  \
    } else {                                                                                \
      constexpr int NE = ElemsPerBlock<PP>::v2;                                             \
      const int threads = NE * (PP + 1) * (PP + 1);                                         \
      const long long blocks = lor_ceil_div(ncls, NE);                                      \
      k_apply2d<PP, T><<<(unsigned)blocks, threads, 0, c->stream>>>(nx, ny, color, B, D, G, x, y, c->conv_flag); \
    }                                                                                       \
  } break;
    switch (c->p) {
      LOR_CASE3(1) LOR_CASE3(2) LOR_CASE3(3) LOR_CASE3(4)
      LOR_CASE3(5) LOR_CASE3(6) LOR_CASE3(7) LOR_CASE3(8)
      default: return lor_fail(c, LOR_EINVAL, "unsupported p");
    }
#undef LOR_CASE3
#undef LOR_VAR3
    ++c->launches;
  }
  lor_prof_end(c, pk);
  return lor_cuda_check(c, cudaGetLastError(), "apply_A launch");
}

template <typename T>
lor_status launch_apply_dgvol(lor_ctx* c, const T* B, const T* D, const T* G, const T* x, T* y) {
  const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
#define LOR_VARDG(PP, V)                                                                      \
  {                                                                                           \
    constexpr int NE = TileNE<PP, T, V>::v;                                                   \
    const int threads = NE * (PP + 1) * (PP + 1);                                             \
    const long long blocks = lor_ceil_div((long long)c->nel, NE);                             \
    k_apply3d<PP, T, true, NE><<<(unsigned)blocks, threads, 0, c->stream>>>(nx, ny, nz, -1, B, D, G, x, y, nullptr); \
  }
#define LOR_CASEDG(PP)                                                                        \
  case PP: {                                                                                  \
    if (c->tune_ne == 0) LOR_VARDG(PP, 0)                                                     \
    else if (c->tune_ne == 2) LOR_VARDG(PP, 2)                                                \
    else LOR_VARDG(PP, 1)                                                                     \
  } break;
  switch (c->p) {
    LOR_CASEDG(1) LOR_CASEDG(2) LOR_CASEDG(3) LOR_CASEDG(4)
    LOR_CASEDG(5) LOR_CASEDG(6) LOR_CASEDG(7) LOR_CASEDG(8)
    default: return lor_fail(c, LOR_EINVAL, "unsupported p");
  }
#undef LOR_CASEDG
#undef LOR_VARDG
  ++c->launches;
  return lor_cuda_check(c, cudaGetLastError(), "DG volume launch");
}

// ---------------------------------------------------------------- right-hand side
// W[e][q] = w_q det J_q f(X_q) at the (p+1)^d Gauss points; then b = sum_e E^T B^T W.
__global__ void k_rhs_weights(int dim, int p, int nx, int ny, int nz, const double* __restrict__ vert,
                              const double* __restrict__ glx, const double* __restrict__ glw, int kind,
                              double* __restrict__ W) {
  const int Q = p + 1;
  const int Qd = dim == 3 ? Q * Q * Q : Q * Q;
  const long long nel = (long long)nx * ny * (dim == 3 ? nz : 1);
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nel * Qd) return;
  const long long e = gid / Qd;
  const int q = (int)(gid - e * Qd);
  const int qx = q % Q, qy = (q / Q) % Q, qz = dim == 3 ? q / (Q * Q) : 0;
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = dim == 3 ? (int)(e / ((long long)nx * ny)) : 0;
  const double xi[3] = {glx[qx], glx[qy], glx[qz]};
  const long long NV = (long long)(nx + 1) * (ny + 1) * (dim == 3 ? (nz + 1) : 1);
  double X[3] = {0, 0, 0}, J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  const int nc = 1 << dim;
  for (int cc = 0; cc < nc; ++cc) {
    const int b[3] = {cc & 1, (cc >> 1) & 1, (cc >> 2) & 1};
    const long long vid = ((long long)(ez + b[2]) * (ny + 1) + (ey + b[1])) * (nx + 1) + (ex + b[0]);
    double f[3], df[3];
    for (int a = 0; a < 3; ++a) { f[a] = b[a] ? xi[a] : 1.0 - xi[a]; df[a] = b[a] ? 1.0 : -1.0; }
    for (int a = 0; a < dim; ++a) {
      const double V = vert[a * NV + vid];
      double N = 1.0;
      for (int t = 0; t < dim; ++t) N *= f[t];
      X[a] += N * V;
      for (int bb = 0; bb < dim; ++bb) {
        double g = 1.0;
        for (int t = 0; t < dim; ++t) g *= (t == bb) ? df[t] : f[t];
        J[a][bb] += g * V;
      }
    }
  }
  double det;
  if (dim == 3)
    det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
          J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  else
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  double fval = 1.0;
  if (kind == 1) {
    const double pi = 3.14159265358979323846;
    fval = dim * pi * pi;
    for (int a = 0; a < dim; ++a) fval *= sin(pi * X[a]);
  }
  double w = glw[qx] * glw[qy] * (dim == 3 ? glw[qz] : 1.0);
  W[gid] = w * fabs(det) * fval;
}

// Curved (isoparametric) elements: the same weights with the point and the Jacobian
// from the degree-p interpolant of the element's GLL node coordinates X (SoA dim x
// ntot); B, D: the 1D GLL basis and its derivative at the Gauss points ([q][i]).
__global__ void k_rhs_weights_iso(int dim, int p, int nx, int ny, int nz, const double* __restrict__ Xn,
                                  const double* __restrict__ B, const double* __restrict__ D,
                                  const double* __restrict__ glw, int kind, double* __restrict__ W) {
  const int Q = p + 1;
  const int Qd = dim == 3 ? Q * Q * Q : Q * Q;
  const long long nel = (long long)nx * ny * (dim == 3 ? nz : 1);
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nel * Qd) return;
  const long long e = gid / Qd;
  const int q = (int)(gid - e * Qd);
  const int qx = q % Q, qy = (q / Q) % Q, qz = dim == 3 ? q / (Q * Q) : 0;
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = dim == 3 ? (int)(e / ((long long)nx * ny)) : 0;
  const int Nx = nx * p + 1, Ny = ny * p + 1;
  const long long ntot = (long long)Nx * Ny * (dim == 3 ? nz * p + 1 : 1);
  double X[3], J[3][3];
  lorg::iso_map(dim, p, ex, ey, ez, qx, qy, qz, Nx, Ny, ntot, Xn, B, D, X, J);
  double det;
  if (dim == 3)
    det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
          J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  else
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  double fval = 1.0;
  if (kind == 1) {
    const double pi = 3.14159265358979323846;
    fval = dim * pi * pi;
    for (int a = 0; a < dim; ++a) fval *= sin(pi * X[a]);
  }
  const double w = glw[qx] * glw[qy] * (dim == 3 ? glw[qz] : 1.0);
  W[gid] = w * fabs(det) * fval;
}

// b += sum over the elements of colour class `color` (element index parity per
// axis, as in the operator kernels): elements of one class share no node, so the
// node sums are plain adds, and the classes run in a fixed order.
__global__ void k_rhs_scatter(int dim, int p, int nx, int ny, int nz, int color, const double* __restrict__ Bm,
                              const double* __restrict__ W, double* __restrict__ b) {
  const int Q = p + 1;
  const int Qd = dim == 3 ? Q * Q * Q : Q * Q;
  const int cx = color & 1, cy = (color >> 1) & 1, cz = (color >> 2) & 1;
  const int mx = (nx - cx + 1) / 2, my = (ny - cy + 1) / 2, mz = dim == 3 ? (nz - cz + 1) / 2 : 1;
  const long long ncls = (long long)mx * my * mz;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= ncls * Qd) return;
  const long long ie = gid / Qd;
  const int a = (int)(gid - ie * Qd);
  const long long e = ((long long)(dim == 3 ? 2 * (int)(ie / ((long long)mx * my)) + cz : 0) * ny +
                       (2 * (int)((ie / mx) % my) + cy)) * nx + (2 * (int)(ie % mx) + cx);
  const int i = a % Q, j = (a / Q) % Q, k = dim == 3 ? a / (Q * Q) : 0;
  double s = 0.0;
  const double* We = W + e * Qd;
  for (int q = 0; q < Qd; ++q) {
    const int qx = q % Q, qy = (q / Q) % Q, qz = dim == 3 ? q / (Q * Q) : 0;
    double phi = Bm[qx * Q + i] * Bm[qy * Q + j];
    if (dim == 3) phi *= Bm[qz * Q + k];
    s += phi * We[q];
  }
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = dim == 3 ? (int)(e / ((long long)nx * ny)) : 0;
  const int Nx = nx * p + 1, Ny = ny * p + 1, Nz = dim == 3 ? nz * p + 1 : 1;
  const int I = ex * p + i, Jn = ey * p + j, K = ez * p + k;
  if (I == 0 || I == Nx - 1 || Jn == 0 || Jn == Ny - 1) return;
  if (dim == 3 && (K == 0 || K == Nz - 1)) return;
  b[((long long)K * Ny + Jn) * Nx + I] += s;
}

// W[q] *= f[q]: the caller's f at the quadrature points times the f = 1 weights
__global__ void k_scale_by(double* __restrict__ W, const double* __restrict__ f, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) W[i] *= f[i];
}

}  // namespace

// Basis tables live in a small device block allocated in lor_setup_geometry:
// [B64 | D64 | B32 | D32 | glx | glw], see lor_setup_geometry.

lor_status lor_launch_apply_A64(lor_ctx* c, const double* x, double* y) {
  return launch_apply<double>(c, lor_basis64(c, 0), lor_basis64(c, 1), c->d_G64, x, y);
}

lor_status lor_launch_apply_A32(lor_ctx* c, const float* x, float* y) {
  return launch_apply<float>(c, lor_basis32(c, 0), lor_basis32(c, 1), c->d_G32, x, y);
}

lor_status lor_launch_dgvol64(lor_ctx* c, const double* x, double* y) {
  return launch_apply_dgvol<double>(c, lor_basis64(c, 0), lor_basis64(c, 1), c->d_G64, x, y);
}

lor_status lor_launch_dgvol32(lor_ctx* c, const float* x, float* y) {
  return launch_apply_dgvol<float>(c, lor_basis32(c, 0), lor_basis32(c, 1), c->d_G32, x, y);
}

lor_status lor_launch_rhs_weights(lor_ctx* c, int kind, double* W) {
  const int Q = c->p + 1;
  const long long Qd = c->dim == 3 ? (long long)Q * Q * Q : (long long)Q * Q;
  const long long tot = (long long)c->nel * Qd;
  if (!c->h_nodes.empty())   // curved elements (lor_set_node_coordinates)
    k_rhs_weights_iso<<<(unsigned)lor_ceil_div(tot, 256), 256, 0, c->stream>>>(
        c->dim, c->p, c->n[0], c->n[1], c->n[2], c->d_X, lor_basis64(c, 0), lor_basis64(c, 5), lor_basis64(c, 3),
        kind, W);
  else
    k_rhs_weights<<<(unsigned)lor_ceil_div(tot, 256), 256, 0, c->stream>>>(
        c->dim, c->p, c->n[0], c->n[1], c->n[2], c->d_vert, lor_basis64(c, 2), lor_basis64(c, 3), kind, W);
  ++c->launches;
  return lor_cuda_check(c, cudaGetLastError(), "rhs weights");
}

lor_status lor_launch_rhs(lor_ctx* c, int kind, double* b, const double* fq) {
  const int Q = c->p + 1;
  const long long Qd = c->dim == 3 ? (long long)Q * Q * Q : (long long)Q * Q;
  const long long tot = (long long)c->nel * Qd;
  double* W = (double*)c->d_v64[7];   // scratch: Krylov vector 7 holds >= nel*(p+1)^d (lor_setup_krylov)
  // quadrature weights w_q det J_q f(x_q): f from the kind, or the caller's values
  if (lor_launch_rhs_weights(c, fq ? 0 : kind, W)) return LOR_ECUDA;
  if (fq) {
    k_scale_by<<<(unsigned)lor_ceil_div(tot, 256), 256, 0, c->stream>>>(W, fq, tot);
    ++c->launches;
  }
  if (c->dg_state) return lor_launch_rhs_dg(c, b, W);
  cudaError_t e = cudaMemsetAsync(b, 0, sizeof(double) * c->lev[0].ntot, c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "rhs memset");
  for (int color = 0; color < (c->dim == 3 ? 8 : 4); ++color) {
    k_rhs_scatter<<<(unsigned)lor_ceil_div(tot, 256), 256, 0, c->stream>>>(c->dim, c->p, c->n[0], c->n[1], c->n[2],
                                                                          color, lor_basis64(c, 0), W, b);
    ++c->launches;
  }
  return lor_cuda_check(c, cudaGetLastError(), "rhs launch");
}

// ---------------------------------------------------------- allocation-free rhs
// One file-scope device array serves every call of lor_rhs_static: the first
// 256 doubles hold the 1D tables (B at Gauss points, Gauss nodes and weights),
// the rest the per-point weights W.  Host code must not use the symbol itself
// as an address: the device address is looked up once per device.
static __device__ __align__(256) double g_rhs_static[LOR_RHS_STATIC_MAX_DOUBLES];

namespace {
const int kStaticTables = 256;
std::mutex g_rhs_static_mu;
double* g_rhs_static_ptr[128] = {};

double* rhs_static_scratch(cudaError_t* err) {
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
  std::lock_guard<std::mutex> lk(g_rhs_static_mu);
  if (!g_rhs_static_ptr[dev]) {
    void* ptr = nullptr;
    *err = cudaGetSymbolAddress(&ptr, g_rhs_static);
    if (*err != cudaSuccess) return nullptr;
    g_rhs_static_ptr[dev] = (double*)ptr;
  }
  return g_rhs_static_ptr[dev];
}

// The 1D tables of one call, passed by value as a kernel argument (so no host
// buffer is copied): B at the Gauss points [q][i], Gauss nodes and weights.
struct RhsTables { double B[(LOR_MAXP + 1) * (LOR_MAXP + 1)]; double x[LOR_MAXP + 1]; double w[LOR_MAXP + 1]; };

// Writes the tables into the head of the static array: B at 0, nodes at 128,
// weights at 192 (the offsets the weight and scatter kernels are given).
__global__ void k_rhs_tables(RhsTables t, int Q, double* __restrict__ head) {
  for (int i = threadIdx.x; i < kStaticTables; i += blockDim.x) {
    double v = 0.0;
    if (i < Q * Q) v = t.B[i];
    else if (i >= 128 && i < 128 + Q) v = t.x[i - 128];
    else if (i >= 192 && i < 192 + Q) v = t.w[i - 192];
    head[i] = v;
  }
}
}  // namespace

extern "C" lor_status lor_rhs_static(int dim, int p, int nx, int ny, int nz, const double* d_vertices, int kind,
                                     double* d_b, void* stream) {
  if ((dim != 2 && dim != 3) || p < 1 || p > LOR_MAXP || nx < 1 || ny < 1 || (dim == 3 && nz < 1)) return LOR_EINVAL;
  if (!d_vertices || !d_b || kind < 0 || kind > 1) return LOR_EINVAL;
  const int Q = p + 1;
  const int zz = dim == 3 ? nz : 1;
  const long long nel = (long long)nx * ny * zz;
  const long long Qd = dim == 3 ? (long long)Q * Q * Q : (long long)Q * Q;
  if (nel * Qd > (long long)LOR_RHS_STATIC_MAX_DOUBLES - kStaticTables) return LOR_EINVAL;
  cudaError_t e;
  double* base = rhs_static_scratch(&e);
  if (!base) return LOR_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // 1D tables on the host, written into the head of the static array by a kernel
  RhsTables tab;
  double gll_x[LOR_MAXP + 1], gll_w[LOR_MAXP + 1], Dn[(LOR_MAXP + 1) * (LOR_MAXP + 1)];
  lorh::gll(p, gll_x, gll_w);
  lorh::gauss(Q, tab.x, tab.w);
  lorh::lagrange(Q, gll_x, Q, tab.x, tab.B, Dn);
  k_rhs_tables<<<1, 128, 0, st>>>(tab, Q, base);
  const long long nvec = (long long)(nx * p + 1) * (ny * p + 1) * (dim == 3 ? (nz * p + 1) : 1);
  if ((e = cudaMemsetAsync(d_b, 0, sizeof(double) * nvec, st)) != cudaSuccess) return LOR_ECUDA;
  double* W = base + kStaticTables;
  const unsigned blocks = (unsigned)lor_ceil_div(nel * Qd, 256);
  k_rhs_weights<<<blocks, 256, 0, st>>>(dim, p, nx, ny, zz, d_vertices, base + 128, base + 192, kind, W);
  for (int color = 0; color < (dim == 3 ? 8 : 4); ++color)
    k_rhs_scatter<<<blocks, 256, 0, st>>>(dim, p, nx, ny, zz, color, base, W, d_b);
  return cudaGetLastError() == cudaSuccess ? LOR_OK : LOR_ECUDA;
}
