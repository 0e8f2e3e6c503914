// Additive-Schwarz LOR preconditioner z = B r (Section 3.2, Eq. (as)):
//   B = P_0 R_0 P_0^T + sum_j R_j^T V_j R_j,
// with one vertex patch per coarse vertex (Eq. (patch)) and V_j one V(1,1) cycle
// of the element-structured hierarchy (Section 3.3) smoothed by lexicographic
// ILU(0) (Section 3.4).
//
// Patch kernel: one CTA per patch runs the whole V-cycle in shared memory:
// gather R_j r, per level ILU(0) pre-smoothing (wavefront-scheduled forward and
// backward sweeps), 3^d-point residual with the level's Galerkin LOR stencil,
// tensor restriction, exact solve on the vertex level (<= 1 unknown), then
// prolongation, residual and post-smoothing on the way up, and a scatter-add of
// x_j into z.  Vectors live in zero-padded boxes so that stencil and factor
// reads need no bounds checks (factors of out-of-box couplings are stored as 0).
//
// Coarse space: P_0^T r at the interior vertices, one V-cycle on the vertex grid
// (l1-Jacobi smoothing, Galerkin levels, dense inverse on the coarsest grid),
// z += P_0 e.
#include "lor_internal.h"

namespace {

template <typename FT> __device__ __forceinline__ float tofl(FT v);
template <> __device__ __forceinline__ float tofl<float>(float v) { return v; }
template <> __device__ __forceinline__ float tofl<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T, typename FT> __device__ __forceinline__ T fac(const FT* p) { return (T)tofl<FT>(*p); }
template <> __device__ __forceinline__ double fac<double, double>(const double* p) { return *p; }

struct PLevel {
  const void* S;          // [NS][ntot] stencil of this level (T)
  long long ntot;
  int N[3];
  int m;
  const Prolong1D* pp[2];       // this level -> next coarser, patch-local, per axis type
  const RestrictEntry* rr[2];   // next coarser <- this level, patch-local, per axis type
};

struct PatchArgs {
  int dim, NS, L, J;
  int n[3];
  PLevel lv[LOR_MAXLEV];
  const BoxShape* shapes;       // [L][8]
  const int* front;
  const int* rowpad;
  const int* rowlex;
  const long long* facoff;      // [L][J]
  const void* F;
  const void* r;
  void* z;
};

struct Box {
  int A, B, C;       // extents
  int rows;
  int pa, pb;        // padded extents (A+2, B+2)
  int pz;            // 1 if the z axis is padded (3D)
  int org[3];        // global level index of local (0,0,0)
  int type[3];       // axis type (0 interior, 1 boundary)
};

__device__ __forceinline__ int pad_of(const Box& b, int i, int j, int k) {
  return ((k + b.pz) * b.pb + (j + 1)) * b.pa + (i + 1);
}

template <int DIM>
__device__ __forceinline__ void off_table(const Box& b, int* off) {
  constexpr int NS = DIM == 3 ? 27 : 9;
#pragma unroll
  for (int o = 0; o < NS; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = DIM == 3 ? o / 9 - 1 : 0;
    off[o] = (dz * b.pb + dy) * b.pa + dx;
  }
}

// in-place (L U)^{-1} on the padded vector t of one level
template <int DIM, typename T, typename FT>
__device__ void ilu_solve(const Box& b, const BoxShape& bs, const int* front, const int* rowpad, const FT* F, T* t) {
  constexpr int NS = DIM == 3 ? 27 : 9;
  constexpr int C = NS / 2;
  int off[NS];
  off_table<DIM>(b, off);
  const int rows = bs.rows;
  const int* fr = front + bs.front_off;
  const int* rp = rowpad + bs.row_off;
  for (int f = 0; f < bs.nfront; ++f) {
    const int e = fr[f + 1];
    for (int pos = fr[f] + threadIdx.x; pos < e; pos += blockDim.x) {
      const int pi = rp[pos];
      T s = t[pi];
#pragma unroll
      for (int o = 0; o < C; ++o) s -= fac<T, FT>(F + (long long)o * rows + pos) * t[pi + off[o]];
      t[pi] = s;
    }
    __syncthreads();
  }
  for (int f = bs.nfront - 1; f >= 0; --f) {
    const int e = fr[f + 1];
    for (int pos = fr[f] + threadIdx.x; pos < e; pos += blockDim.x) {
      const int pi = rp[pos];
      T s = t[pi];
#pragma unroll
      for (int o = C + 1; o < NS; ++o) s -= fac<T, FT>(F + (long long)o * rows + pos) * t[pi + off[o]];
      t[pi] = s * fac<T, FT>(F + (long long)C * rows + pos);
    }
    __syncthreads();
  }
}

// t = rhs - A x on one level; rhs from global r (level 0) or from rs
template <int DIM, typename T>
__device__ void residual(const Box& b, const PLevel& lv, const T* rglob, const T* rs, const T* x, T* t) {
  constexpr int NS = DIM == 3 ? 27 : 9;
  int off[NS];
  off_table<DIM>(b, off);
  const T* S = (const T*)lv.S;
  for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
    const int i = lex % b.A, j = (lex / b.A) % b.B, k = lex / (b.A * b.B);
    const long long G = ((long long)(b.org[2] + k) * lv.N[1] + (b.org[1] + j)) * lv.N[0] + (b.org[0] + i);
    const int pi = pad_of(b, i, j, k);
    T s = rglob ? rglob[G] : rs[lex];
#pragma unroll
    for (int o = 0; o < NS; ++o) s -= S[(long long)o * lv.ntot + G] * x[pi + off[o]];
    t[pi] = s;
  }
}

template <int DIM, typename T, typename FT>
__global__ void __launch_bounds__(128) k_patch_vcycle(PatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = (T*)smem_raw;
  const int j = blockIdx.x;
  int v[3];
  v[0] = j % (a.n[0] + 1);
  v[1] = (j / (a.n[0] + 1)) % (a.n[1] + 1);
  v[2] = DIM == 3 ? j / ((a.n[0] + 1) * (a.n[1] + 1)) : 0;
  int sh = 0, type[3] = {0, 0, 0};
  for (int t = 0; t < DIM; ++t) {
    type[t] = (v[t] == 0 || v[t] == a.n[t]) ? 1 : 0;
    sh |= type[t] << t;
  }
  Box bx[LOR_MAXLEV];
  BoxShape bsh[LOR_MAXLEV];
  T* xs[LOR_MAXLEV];
  T* ts[LOR_MAXLEV];
  T* rs[LOR_MAXLEV];
  long long offset = 0;
  for (int l = 0; l < a.L; ++l) {
    BoxShape bs = a.shapes[l * 8 + sh];
    bsh[l] = bs;
    Box& b = bx[l];
    b.A = bs.dims[0]; b.B = bs.dims[1]; b.C = bs.dims[2];
    b.rows = bs.rows;
    b.pa = b.A + 2; b.pb = b.B + 2; b.pz = DIM == 3 ? 1 : 0;
    const int pc = DIM == 3 ? b.C + 2 : 1;
    for (int t = 0; t < 3; ++t) {
      b.type[t] = type[t];
      b.org[t] = t < DIM ? (v[t] > 0 ? v[t] - 1 : 0) * a.lv[l].m + 1 : 0;
    }
    const int padn = b.pa * b.pb * pc;
    xs[l] = sm + offset; offset += padn;
    ts[l] = sm + offset; offset += padn;
    rs[l] = sm + offset; offset += (l > 0 ? b.rows : 0);
  }
  if (bx[0].rows == 0) return;
  for (long long i = threadIdx.x; i < offset; i += blockDim.x) sm[i] = T(0);
  __syncthreads();
  const T* rg = (const T*)a.r;
  const FT* F = (const FT*)a.F;
  // deepest level with unknowns
  int bottom = 0;
  while (bottom + 1 < a.L && bx[bottom + 1].rows > 0) ++bottom;
  // ---- down
  for (int l = 0; l < bottom; ++l) {
    const Box& b = bx[l];
    const PLevel& lv = a.lv[l];
    const FT* Fl = F + a.facoff[(long long)l * a.J + j];
    for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
      const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
      const long long G = ((long long)(b.org[2] + k) * lv.N[1] + (b.org[1] + jj)) * lv.N[0] + (b.org[0] + i);
      ts[l][pad_of(b, i, jj, k)] = l == 0 ? rg[G] : rs[l][lex];
    }
    __syncthreads();
    ilu_solve<DIM, T, FT>(b, bsh[l], a.front, a.rowpad, Fl, ts[l]);
    for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
      const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
      const int pi = pad_of(b, i, jj, k);
      xs[l][pi] = ts[l][pi];
    }
    __syncthreads();
    residual<DIM, T>(b, lv, l == 0 ? rg : nullptr, rs[l], xs[l], ts[l]);
    __syncthreads();
    // restriction to level l+1
    const Box& bc = bx[l + 1];
    for (int lex = threadIdx.x; lex < bc.rows; lex += blockDim.x) {
      const int ci = lex % bc.A, cj = (lex / bc.A) % bc.B, ck = lex / (bc.A * bc.B);
      const RestrictEntry& ex = lv.rr[b.type[0]][ci];
      const RestrictEntry& ey = lv.rr[b.type[1]][cj];
      const RestrictEntry* ez = DIM == 3 ? &lv.rr[b.type[2]][ck] : nullptr;
      T s = 0;
      const int nz = DIM == 3 ? ez->cnt : 1;
      for (int tz = 0; tz < nz; ++tz) {
        const int fz = DIM == 3 ? ez->f[tz] : 0;
        const T wz = DIM == 3 ? (T)ez->w[tz] : T(1);
        for (int ty = 0; ty < ey.cnt; ++ty) {
          const T wy = (T)ey.w[ty] * wz;
          const int fy = ey.f[ty];
          for (int tx = 0; tx < ex.cnt; ++tx) s += (T)ex.w[tx] * wy * ts[l][pad_of(b, ex.f[tx], fy, fz)];
        }
      }
      rs[l + 1][lex] = s;
    }
    __syncthreads();
  }
  // ---- coarsest level with unknowns: exact solve.  The vertex level of a patch
  // has a single unknown; a truncated hierarchy may stop above it, in which case
  // the bottom level is smoothed twice by ILU(0) (pre and post, no coarse solve).
  {
    const int l = bottom;
    const Box& b = bx[l];
    const PLevel& lv = a.lv[l];
    if (l == a.L - 1) {
      const T* S = (const T*)lv.S;
      for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
        const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
        const long long G = ((long long)(b.org[2] + k) * lv.N[1] + (b.org[1] + jj)) * lv.N[0] + (b.org[0] + i);
        const T rhs = l == 0 ? rg[G] : rs[l][lex];
        xs[l][pad_of(b, i, jj, k)] = rhs / S[(long long)(a.NS / 2) * lv.ntot + G];   // rows <= 1
      }
      __syncthreads();
    } else {
      const FT* Fl = F + a.facoff[(long long)l * a.J + j];
      for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
        const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
        const long long G = ((long long)(b.org[2] + k) * lv.N[1] + (b.org[1] + jj)) * lv.N[0] + (b.org[0] + i);
        ts[l][pad_of(b, i, jj, k)] = l == 0 ? rg[G] : rs[l][lex];
      }
      __syncthreads();
      ilu_solve<DIM, T, FT>(b, bsh[l], a.front, a.rowpad, Fl, ts[l]);
      for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
        const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
        const int pi = pad_of(b, i, jj, k);
        xs[l][pi] = ts[l][pi];
      }
      __syncthreads();
      residual<DIM, T>(b, lv, l == 0 ? rg : nullptr, rs[l], xs[l], ts[l]);
      __syncthreads();
      ilu_solve<DIM, T, FT>(b, bsh[l], a.front, a.rowpad, Fl, ts[l]);
      for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
        const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
        const int pi = pad_of(b, i, jj, k);
        xs[l][pi] += ts[l][pi];
      }
      __syncthreads();
    }
  }
  // ---- up
  for (int l = bottom - 1; l >= 0; --l) {
    const Box& b = bx[l];
    const Box& bc = bx[l + 1];
    const PLevel& lv = a.lv[l];
    const FT* Fl = F + a.facoff[(long long)l * a.J + j];
    for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
      const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
      const Prolong1D px = lv.pp[b.type[0]][i], py = lv.pp[b.type[1]][jj];
      Prolong1D pz;
      if (DIM == 3) pz = lv.pp[b.type[2]][k]; else { pz.c0 = 0; pz.w0 = 1.0; pz.c1 = -2; pz.w1 = 0.0; }
      T s = 0;
      const int nzz = DIM == 3 ? 2 : 1;
      for (int sz = 0; sz < nzz; ++sz) {
        const int cz = sz ? pz.c1 : pz.c0;
        if (cz < -1) continue;
        const T wz = (T)(sz ? pz.w1 : pz.w0);
        for (int sy = 0; sy < 2; ++sy) {
          const int cy = sy ? py.c1 : py.c0;
          if (cy < -1) continue;
          const T wy = (T)(sy ? py.w1 : py.w0) * wz;
          for (int sx = 0; sx < 2; ++sx) {
            const int cx = sx ? px.c1 : px.c0;
            if (cx < -1) continue;
            s += (T)(sx ? px.w1 : px.w0) * wy * xs[l + 1][pad_of(bc, cx, cy, DIM == 3 ? cz : 0)];
          }
        }
      }
      xs[l][pad_of(b, i, jj, k)] += s;
    }
    __syncthreads();
    residual<DIM, T>(b, lv, l == 0 ? rg : nullptr, rs[l], xs[l], ts[l]);
    __syncthreads();
    ilu_solve<DIM, T, FT>(b, bsh[l], a.front, a.rowpad, Fl, ts[l]);
    for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
      const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
      const int pi = pad_of(b, i, jj, k);
      xs[l][pi] += ts[l][pi];
    }
    __syncthreads();
  }
  // ---- scatter-add R_j^T x_j
  T* z = (T*)a.z;
  const Box& b = bx[0];
  const PLevel& lv = a.lv[0];
  for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
    const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
    const long long G = ((long long)(b.org[2] + k) * lv.N[1] + (b.org[1] + jj)) * lv.N[0] + (b.org[0] + i);
    atomicAdd(z + G, xs[0][pad_of(b, i, jj, k)]);
  }
}

// ------------------------------------------------------------------ coarse space
// rc[V] = sum_F P0[F][V] r[F] for interior vertices V (P0: Q1 interpolation at GLL nodes)
template <typename T>
__global__ void k_coarse_restrict0(int dim, int p, int nx, int ny, int nz, const double* __restrict__ gllx,
                                   const T* __restrict__ r, T* __restrict__ rc) {
  const int Vx = nx + 1, Vy = ny + 1, Vz = dim == 3 ? nz + 1 : 1;
  const long long nv = (long long)Vx * Vy * Vz;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nv) return;
  const int V[3] = {(int)(gid % Vx), (int)((gid / Vx) % Vy), (int)(gid / ((long long)Vx * Vy))};
  const bool bnd = V[0] == 0 || V[0] == nx || V[1] == 0 || V[1] == ny || (dim == 3 && (V[2] == 0 || V[2] == nz));
  if (bnd) { rc[gid] = T(0); return; }
  const int Nx = nx * p + 1, Ny = ny * p + 1;
  // 1D weights of the fine indices (V-1)p+1 .. (V+1)p-1
  T s = 0;
  const int len = 2 * p - 1;
  const int kz = dim == 3 ? len : 1;
  for (int c = 0; c < kz; ++c) {
    T wz = 1;
    int Kf = 0;
    if (dim == 3) {
      Kf = (V[2] - 1) * p + 1 + c;
      const int t = c + 1;   // position within [ (V-1)p, (V+1)p ]
      wz = (T)(t <= p ? gllx[t] : 1.0 - gllx[t - p]);
    }
    for (int b = 0; b < len; ++b) {
      const int Jf = (V[1] - 1) * p + 1 + b;
      const int tb = b + 1;
      const T wy = (T)(tb <= p ? gllx[tb] : 1.0 - gllx[tb - p]) * wz;
      const T* row = r + ((long long)Kf * Ny + Jf) * Nx + (V[0] - 1) * p + 1;
      for (int a = 0; a < len; ++a) {
        const int ta = a + 1;
        s += (T)(ta <= p ? gllx[ta] : 1.0 - gllx[ta - p]) * wy * row[a];
      }
    }
  }
  rc[gid] = s;
}

// z[F] += sum_V P0[F][V] e[V] for interior fine nodes
template <typename T>
__global__ void k_coarse_prolong0(int dim, int p, int nx, int ny, int nz, const double* __restrict__ gllx,
                                  const T* __restrict__ e, T* __restrict__ z) {
  const int Nx = nx * p + 1, Ny = ny * p + 1, Nz = dim == 3 ? nz * p + 1 : 1;
  const long long nt = (long long)Nx * Ny * Nz;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nt) return;
  const int I = (int)(gid % Nx), Jn = (int)((gid / Nx) % Ny), K = (int)(gid / ((long long)Nx * Ny));
  if (I == 0 || I == Nx - 1 || Jn == 0 || Jn == Ny - 1 || (dim == 3 && (K == 0 || K == Nz - 1))) return;
  const int ex = min(I / p, nx - 1), ey = min(Jn / p, ny - 1), ez = dim == 3 ? min(K / p, nz - 1) : 0;
  const double xi[3] = {gllx[I - ex * p], gllx[Jn - ey * p], dim == 3 ? gllx[K - ez * p] : 0.0};
  const int Vx = nx + 1, Vy = ny + 1;
  T s = 0;
  const int nc = 1 << dim;
  for (int cc = 0; cc < nc; ++cc) {
    const int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
    double w = (bx ? xi[0] : 1.0 - xi[0]) * (by ? xi[1] : 1.0 - xi[1]);
    if (dim == 3) w *= bz ? xi[2] : 1.0 - xi[2];
    s += (T)w * e[((long long)(ez + bz) * Vy + (ey + by)) * Vx + (ex + bx)];
  }
  z[gid] += s;
}

__device__ __forceinline__ bool grid_bnd(int dim, const int* N, int I, int J, int K) {
  return I == 0 || I == N[0] - 1 || J == 0 || J == N[1] - 1 || (dim == 3 && (K == 0 || K == N[2] - 1));
}

struct CGrid { int dim; int N[3]; };

// xout = xin + Dinv (r - A xin) on interior nodes (xin == nullptr: xin = 0)
template <typename T>
__global__ void k_cjacobi(CGrid g, const T* __restrict__ S, const T* __restrict__ Dinv, const T* __restrict__ r,
                          const T* __restrict__ xin, T* __restrict__ xout) {
  const long long nt = (long long)g.N[0] * g.N[1] * g.N[2];
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nt) return;
  const int I = (int)(gid % g.N[0]), Jn = (int)((gid / g.N[0]) % g.N[1]), K = (int)(gid / ((long long)g.N[0] * g.N[1]));
  if (grid_bnd(g.dim, g.N, I, Jn, K)) { xout[gid] = T(0); return; }
  T s = r[gid];
  T x0 = 0;
  if (xin) {
    const int NS = g.dim == 3 ? 27 : 9;
    for (int o = 0; o < NS; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = g.dim == 3 ? o / 9 - 1 : 0;
      const long long h = gid + ((long long)dz * g.N[1] + dy) * g.N[0] + dx;
      s -= S[(long long)o * nt + gid] * xin[h];
    }
    x0 = xin[gid];
  }
  xout[gid] = x0 + Dinv[gid] * s;
}

template <typename T>
__global__ void k_cresid(CGrid g, const T* __restrict__ S, const T* __restrict__ r, const T* __restrict__ x,
                         T* __restrict__ t) {
  const long long nt = (long long)g.N[0] * g.N[1] * g.N[2];
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nt) return;
  const int I = (int)(gid % g.N[0]), Jn = (int)((gid / g.N[0]) % g.N[1]), K = (int)(gid / ((long long)g.N[0] * g.N[1]));
  if (grid_bnd(g.dim, g.N, I, Jn, K)) { t[gid] = T(0); return; }
  T s = r[gid];
  const int NS = g.dim == 3 ? 27 : 9;
  for (int o = 0; o < NS; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = g.dim == 3 ? o / 9 - 1 : 0;
    const long long h = gid + ((long long)dz * g.N[1] + dy) * g.N[0] + dx;
    s -= S[(long long)o * nt + gid] * x[h];
  }
  t[gid] = s;
}

struct CTransfer {
  int dim;
  int Nf[3], Nc[3];
  const Prolong1D* P[3];
  const int* Rptr[3];
  const int* Ridx[3];
  const double* Rw[3];
};

template <typename T>
__global__ void k_crestrict(CTransfer g, const T* __restrict__ t, T* __restrict__ rc) {
  const long long ntc = (long long)g.Nc[0] * g.Nc[1] * g.Nc[2];
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= ntc) return;
  const int C[3] = {(int)(gid % g.Nc[0]), (int)((gid / g.Nc[0]) % g.Nc[1]), (int)(gid / ((long long)g.Nc[0] * g.Nc[1]))};
  if (grid_bnd(g.dim, g.Nc, C[0], C[1], C[2])) { rc[gid] = T(0); return; }
  T s = 0;
  const int zlo = g.dim == 3 ? g.Rptr[2][C[2]] : 0, zhi = g.dim == 3 ? g.Rptr[2][C[2] + 1] : 1;
  for (int iz = zlo; iz < zhi; ++iz) {
    const int fz = g.dim == 3 ? g.Ridx[2][iz] : 0;
    const T wz = g.dim == 3 ? (T)g.Rw[2][iz] : T(1);
    for (int iy = g.Rptr[1][C[1]]; iy < g.Rptr[1][C[1] + 1]; ++iy) {
      const int fy = g.Ridx[1][iy];
      const T wy = (T)g.Rw[1][iy] * wz;
      for (int ix = g.Rptr[0][C[0]]; ix < g.Rptr[0][C[0] + 1]; ++ix)
        s += (T)g.Rw[0][ix] * wy * t[((long long)fz * g.Nf[1] + fy) * g.Nf[0] + g.Ridx[0][ix]];
    }
  }
  rc[gid] = s;
}

template <typename T>
__global__ void k_cprolong_add(CTransfer g, const T* __restrict__ xc, T* __restrict__ x) {
  const long long ntf = (long long)g.Nf[0] * g.Nf[1] * g.Nf[2];
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= ntf) return;
  const int I = (int)(gid % g.Nf[0]), Jn = (int)((gid / g.Nf[0]) % g.Nf[1]), K = (int)(gid / ((long long)g.Nf[0] * g.Nf[1]));
  if (grid_bnd(g.dim, g.Nf, I, Jn, K)) return;
  const Prolong1D px = g.P[0][I], py = g.P[1][Jn];
  Prolong1D pz;
  if (g.dim == 3) pz = g.P[2][K]; else { pz.c0 = 0; pz.w0 = 1.0; pz.c1 = -1; pz.w1 = 0.0; }
  T s = 0;
  for (int sz = 0; sz < 2; ++sz) {
    const int cz = sz ? pz.c1 : pz.c0;
    if (cz < 0) continue;
    for (int sy = 0; sy < 2; ++sy) {
      const int cy = sy ? py.c1 : py.c0;
      if (cy < 0) continue;
      for (int sx = 0; sx < 2; ++sx) {
        const int cx = sx ? px.c1 : px.c0;
        if (cx < 0) continue;
        const double w = (sx ? px.w1 : px.w0) * (sy ? py.w1 : py.w0) * (sz ? pz.w1 : pz.w0);
        s += (T)w * xc[((long long)cz * g.Nc[1] + cy) * g.Nc[0] + cx];
      }
    }
  }
  x[gid] += s;
}

// x[idx[a]] = sum_b Inv[a][b] r[idx[b]]: one warp per row
template <typename T>
__global__ void k_cdense(int nd, const int* __restrict__ idx, const T* __restrict__ Inv, const T* __restrict__ r,
                         T* __restrict__ x) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nd) return;
  T s = 0;
  for (int b = lane; b < nd; b += 32) s += Inv[(long long)warp * nd + b] * r[idx[b]];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[idx[warp]] = s;
}

template <typename T> struct Sel;
template <> struct Sel<double> {
  static double* cw(lor_ctx* c, int l, int k) { return c->d_cw64[l][k]; }
  static const double* cS(lor_ctx* c, int l) { return c->d_cS64[l]; }
  static const double* cD(lor_ctx* c, int l) { return c->d_cDinv64[l]; }
  static const double* inv(lor_ctx* c) { return c->d_cInv64; }
  static const void* S(lor_ctx* c, int l) { return c->d_S64[l]; }
};
template <> struct Sel<float> {
  static float* cw(lor_ctx* c, int l, int k) { return c->d_cw32[l][k]; }
  static const float* cS(lor_ctx* c, int l) { return c->d_cS32[l]; }
  static const float* cD(lor_ctx* c, int l) { return c->d_cDinv32[l]; }
  static const float* inv(lor_ctx* c) { return c->d_cInv32; }
  static const void* S(lor_ctx* c, int l) { return c->d_S32[l]; }
};

static const int kCoarseSweeps = 2;

// one V-cycle on coarse level l: rhs in cw[l][0]; returns the buffer holding x
template <typename T>
T* coarse_vcycle(lor_ctx* c, int l) {
  T* r = Sel<T>::cw(c, l, 0);
  T* xa = Sel<T>::cw(c, l, 1);
  T* xb = Sel<T>::cw(c, l, 2);
  T* t = Sel<T>::cw(c, l, 3);
  const long long nt = c->cntot[l];
  const unsigned nb = (unsigned)lor_ceil_div(nt, 128);
  CGrid g;
  g.dim = c->dim;
  for (int a = 0; a < 3; ++a) g.N[a] = c->cN[l][a];
  if (l == c->CL - 1) {
    if (c->ncoarse_direct > 0) {
      const int nd = c->ncoarse_direct;
      k_cdense<T><<<(unsigned)lor_ceil_div((long long)nd * 32, 128), 128, 0, c->stream>>>(
          nd, c->d_cdirect_idx, Sel<T>::inv(c), r, xa);
      ++c->launches;
    }
    return xa;
  }
  const T* S = Sel<T>::cS(c, l);
  const T* D = Sel<T>::cD(c, l);
  T* cur = xa;
  T* oth = xb;
  k_cjacobi<T><<<nb, 128, 0, c->stream>>>(g, S, D, r, (const T*)nullptr, cur);
  ++c->launches;
  for (int s = 1; s < kCoarseSweeps; ++s) {
    k_cjacobi<T><<<nb, 128, 0, c->stream>>>(g, S, D, r, cur, oth);
    ++c->launches;
    T* tmp = cur; cur = oth; oth = tmp;
  }
  k_cresid<T><<<nb, 128, 0, c->stream>>>(g, S, r, cur, t);
  ++c->launches;
  CTransfer tr;
  tr.dim = c->dim;
  for (int a = 0; a < 3; ++a) {
    tr.Nf[a] = c->cN[l][a]; tr.Nc[a] = c->cN[l + 1][a];
    tr.P[a] = c->d_cP1[l][a]; tr.Rptr[a] = c->d_cR1ptr[l][a]; tr.Ridx[a] = c->d_cR1idx[l][a]; tr.Rw[a] = c->d_cR1w[l][a];
  }
  const long long ntc = c->cntot[l + 1];
  k_crestrict<T><<<(unsigned)lor_ceil_div(ntc, 128), 128, 0, c->stream>>>(tr, t, Sel<T>::cw(c, l + 1, 0));
  ++c->launches;
  T* xc = coarse_vcycle<T>(c, l + 1);
  k_cprolong_add<T><<<nb, 128, 0, c->stream>>>(tr, xc, cur);
  ++c->launches;
  for (int s = 0; s < kCoarseSweeps; ++s) {
    k_cjacobi<T><<<nb, 128, 0, c->stream>>>(g, S, D, r, cur, oth);
    ++c->launches;
    T* tmp = cur; cur = oth; oth = tmp;
  }
  return cur;
}

template <typename T, typename FT>
lor_status launch_apply_P(lor_ctx* c, const T* r, T* z, const FT* F, size_t smem) {
  const long long nvec = c->lev[0].ntot;
  cudaError_t e = cudaMemsetAsync(z, 0, sizeof(T) * nvec, c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "apply_P memset");
  PatchArgs a;
  a.dim = c->dim; a.NS = c->NS; a.L = c->L; a.J = c->J;
  for (int t = 0; t < 3; ++t) a.n[t] = c->n[t];
  for (int l = 0; l < c->L; ++l) {
    PLevel& lv = a.lv[l];
    lv.S = Sel<T>::S(c, l);
    lv.ntot = c->lev[l].ntot;
    for (int t = 0; t < 3; ++t) lv.N[t] = c->lev[l].N[t];
    lv.m = c->lev[l].m;
    for (int t = 0; t < 2; ++t) { lv.pp[t] = c->d_pp[l][t]; lv.rr[t] = c->d_rr[l][t]; }
  }
  a.shapes = lor_dev_shapes(c);
  a.front = c->d_front; a.rowpad = c->d_rowpad; a.rowlex = c->d_rowlex;
  a.facoff = c->d_facoff;
  a.F = F; a.r = r; a.z = z;
  const int pk = sizeof(T) == 8 ? 0 : 1;
  lor_prof_begin(c, pk);
  if (c->dim == 3) {
    auto kern = k_patch_vcycle<3, T, FT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<c->J, 128, smem, c->stream>>>(a);
    ++c->launches;
  } else {
    auto kern = k_patch_vcycle<2, T, FT>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<c->J, 128, smem, c->stream>>>(a);
    ++c->launches;
  }
  lor_prof_end(c, pk);
  if (lor_cuda_check(c, cudaGetLastError(), "patch vcycle")) return LOR_ECUDA;
  lor_prof_begin(c, pk + 4);
  // coarse space
  const double* gllx = lor_basis64(c, 4);
  const long long nv = c->cntot[0];
  k_coarse_restrict0<T><<<(unsigned)lor_ceil_div(nv, 128), 128, 0, c->stream>>>(c->dim, c->p, c->n[0], c->n[1],
                                                                                   c->n[2], gllx, r, Sel<T>::cw(c, 0, 0));
  ++c->launches;
  T* ec = coarse_vcycle<T>(c, 0);
  k_coarse_prolong0<T><<<(unsigned)lor_ceil_div(nvec, 128), 128, 0, c->stream>>>(c->dim, c->p, c->n[0], c->n[1],
                                                                                   c->n[2], gllx, ec, z);
  ++c->launches;
  lor_prof_end(c, pk + 4);
  return lor_cuda_check(c, cudaGetLastError(), "coarse space");
}

}  // namespace

lor_status lor_launch_apply_P64(lor_ctx* c, const double* r, double* z) {
  return launch_apply_P<double, double>(c, r, z, c->d_F64, (size_t)c->smem_patch64);
}

lor_status lor_launch_apply_P32(lor_ctx* c, const float* r, float* z) {
  if (c->d_F16) return launch_apply_P<float, __nv_bfloat16>(c, r, z, c->d_F16, (size_t)c->smem_patch32);
  return launch_apply_P<float, float>(c, r, z, c->d_F32, (size_t)c->smem_patch32);
}
