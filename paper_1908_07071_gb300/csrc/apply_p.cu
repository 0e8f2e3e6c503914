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
#include <algorithm>

#include "lor_internal.h"

namespace {

template <typename FT> __device__ __forceinline__ float tofl(FT v);
template <> __device__ __forceinline__ float tofl<float>(float v) { return v; }
template <> __device__ __forceinline__ float tofl<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T, typename FT> __device__ __forceinline__ T fac(FT v) { return (T)tofl<FT>(v); }
template <> __device__ __forceinline__ double fac<double, double>(double v) { return v; }

struct PLevel {
  const void* S;          // [NS][ntot] stencil of this level (T)
  long long ntot;
  int N[3];
  int m;
  const Prolong1D* pp[2];       // this level -> next coarser, patch-local, per axis type
  const RestrictEntry* rr[2];   // next coarser <- this level, patch-local, per axis type
  int len[2], clen[2];          // fine / coarse unknowns along an axis of each type
};

// Shared-memory copy of one 1D patch-local transfer (one level, one axis type):
// prolongation rows (fine -> <= 2 coarse) and the transposed restriction lists.
template <typename T>
struct Xfer1D {
  int c0[2 * LOR_MAXP], c1[2 * LOR_MAXP];
  T w0[2 * LOR_MAXP], w1[2 * LOR_MAXP];
  int rstart[2 * LOR_MAXP + 1];
  int rf[4 * LOR_MAXP];
  T rw[4 * LOR_MAXP];
};

struct PatchArgs {
  int dim, NS, L, J;
  int n[3];
  PLevel lv[LOR_MAXLEV];
  const BoxShape* shapes;       // [L][8]
  const int* front;
  const int* fpad;
  const int* chunk;
  const int* rowlex;
  const int* recof;
  const unsigned* nbmask;
  const long long* facoff;      // [L][J] record offsets
  const void* F;
  const void* r;
  void* z;
  int* status;
  int slot_bytes;               // ring slot size (bytes, multiple of 16)
  int tab_ints;                 // shared-memory ints reserved for wavefront tables
  const int* porder;            // patch visiting order (grouped by box shape)
  const double* conv;           // optional: skip all work when *conv != 0 (converged batched solve)
  // patch-local mode (learned-correction training data): patches plist[0..nlist)
  // take their level-0 right-hand side from rloc and write x to xloc (lexicographic
  // box order, stride vstride per listed patch) instead of gathering / scattering
  const int* plist;
  int nlist;
  const void* rloc;
  void* xloc;
  int vstride;
  // residual capture (learned-correction inference): the level-0 residual left by
  // the cycle on every interior patch is written to tout + visiting position * vstride
  void* tout;
};

struct Box {
  int A, B, C;       // extents
  int rows;
  int org[3];        // global level index of local (0,0,0)
  int type[3];       // axis type (0 interior, 1 boundary)
};

// ---- TMA bulk-copy ring (one elected producer thread, mbarrier completion) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  // order earlier generic-proxy reads of this slot before the async-proxy write
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Waits for the phase `parity` of `bar`; gives up after a bounded number of
// polls (returns false) so that a lost copy cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned addr = smem_u32(bar);
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <typename FT, int NBUF>
struct Ring {
  unsigned char* base;   // slot s starts at base + s * bytes
  int bytes;
  __device__ __forceinline__ FT* slot(int s) const { return (FT*)(base + (size_t)s * bytes); }
  unsigned long long* bar;
  unsigned phase;     // bit s: parity expected next on slot s
  unsigned inflight;  // producer view: bit s set while a copy into slot s is pending
};

// Shared-memory copies of one level's wavefront tables.
struct LevelTables {
  const unsigned short* rowlex;   // lexicographic row index per wavefront position
  const int* front;               // nfront+1 row positions
  const int* fpad;                // nfront+1 record offsets
  const int* chunk;               // nchunk+1 front indices
};

// One triangular sweep over a level, run by ONE warp.  Factor blocks stream
// through the ring in chunks of whole fronts: lane 0 issues the bulk copies and
// observes their completion, __syncwarp publishes them to the other lanes.
// Inside a chunk, lanes loop over the rows of a front and __syncwarp separates
// fronts.  t has a zero guard band, so neighbour reads need no clamping
// (multipliers of out-of-box neighbours are stored as 0).  BACK selects the
// backward sweep (U part, fronts in reverse, scaled by 1/u_ii).
template <int DIM, bool BACK, typename T, typename FT, int NBUF>
__device__ __forceinline__ bool sweep(const FT* __restrict__ part, const int* __restrict__ fr,
                                      const int* __restrict__ fp, const int* __restrict__ ch,
                                      const unsigned short* __restrict__ rl, int nc, int A, int AB, T* t,
                                      Ring<FT, NBUF>& rg) {
  constexpr int NS = DIM == 3 ? 27 : 9;
  constexpr int C = NS / 2;
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    for (int c = 0; c < NBUF - 1 && c < nc; ++c) {
      const int k = BACK ? nc - 1 - c : c;
      bulk_load(rg.slot(c % NBUF), part + (long long)fp[ch[k]] * LOR_REC,
                (unsigned)((fp[ch[k + 1]] - fp[ch[k]]) * LOR_REC * sizeof(FT)), rg.bar + (c % NBUF));
      rg.inflight |= 1u << (c % NBUF);
    }
  }
  for (int c = 0; c < nc; ++c) {
    const int sl = c % NBUF;
    int ok = 1;
    if (lane == 0) ok = mbar_wait(rg.bar + sl, (rg.phase >> sl) & 1u) ? 1 : 0;
    rg.phase ^= 1u << sl;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return false;
    if (lane == 0) {
      rg.inflight &= ~(1u << sl);
      const int cn = c + NBUF - 1;
      if (cn < nc) {
        const int k = BACK ? nc - 1 - cn : cn;
        bulk_load(rg.slot(cn % NBUF), part + (long long)fp[ch[k]] * LOR_REC,
                  (unsigned)((fp[ch[k + 1]] - fp[ch[k]]) * LOR_REC * sizeof(FT)), rg.bar + (cn % NBUF));
        rg.inflight |= 1u << (cn % NBUF);
      }
    }
    __syncwarp();
    const FT* blk = rg.slot(sl);
    const int k = BACK ? nc - 1 - c : c;
    const int fa = ch[k], fb = ch[k + 1];
    const int r0 = fp[fa];
    for (int q = 0; q < fb - fa; ++q) {
      const int f = BACK ? fb - 1 - q : fa + q;
      const int p0 = fr[f], p1 = fr[f + 1];
      const FT* fbk = blk + (fp[f] - r0) * LOR_REC;
      for (int pos = p0 + lane; pos < p1; pos += 32) {
        const int li = rl[pos];
        const FT* rec = fbk + (pos - p0) * LOR_REC;
        T s0 = t[li], s1 = T(0);
#pragma unroll
        for (int o = 0; o < C; ++o) {
          const int so = BACK ? C + 1 + o : o;                 // stencil offset index
          const int dx = so % 3 - 1, dy = (so / 3) % 3 - 1, dz = DIM == 3 ? so / 9 - 1 : 0;
          const T v = fac<T, FT>(rec[o]) * t[li + dz * AB + dy * A + dx];
          if (o & 1) s1 -= v; else s0 -= v;
        }
        t[li] = BACK ? (s0 + s1) * fac<T, FT>(rec[LOR_REC - 1]) : s0 + s1;
      }
      __syncwarp();
    }
  }
  return true;
}

// in-place (L U)^{-1} t on one level: warp 0 runs the forward and backward
// sweeps, the other warps wait at the closing __syncthreads.  Returns false on
// all threads if a bulk copy timed out.
template <typename FT>
constexpr int elem_class() { return sizeof(FT) == 2 ? 0 : (sizeof(FT) == 4 ? 1 : 2); }

template <int DIM, typename T, typename FT, int NBUF>
__device__ bool ilu_solve(const BoxShape& bs, const LevelTables& tb, const FT* FL, T* t, Ring<FT, NBUF>& rg,
                          int* abort) {
  constexpr int ES = elem_class<FT>();
  if (threadIdx.x < 32) {
    const int A = bs.dims[0], AB = bs.dims[0] * bs.dims[1];
    bool ok = sweep<DIM, false, T, FT, NBUF>(FL, tb.front, tb.fpad, tb.chunk, tb.rowlex, bs.nchunk[ES], A, AB, t, rg);
    if (ok)
      ok = sweep<DIM, true, T, FT, NBUF>(FL + (long long)bs.rpad * LOR_REC, tb.front, tb.fpad, tb.chunk, tb.rowlex,
                                          bs.nchunk[ES], A, AB, t, rg);
    if (!ok && threadIdx.x == 0) *abort = 1;
  }
  __syncthreads();
  return *abort == 0;
}

// t = rhs - A x on one level (rhs from global r on level 0, else from rs).
template <int DIM, typename T>
__device__ __forceinline__ void residual(int A, int B, int Cz, int ox, int oy, int oz, int Nx, int Ny, long long ntot,
                                         const T* __restrict__ S, const T* __restrict__ rglob,
                                         const T* __restrict__ rs, const T* x, T* t) {
  constexpr int NS = DIM == 3 ? 27 : 9;
  const int rows = A * B * Cz;
  for (int lex = threadIdx.x; lex < rows; lex += blockDim.x) {
    const int i = lex % A, j = (lex / A) % B, k = lex / (A * B);
    const long long G = ((long long)(oz + k) * Ny + (oy + j)) * Nx + (ox + i);
    T s = rglob ? rglob[G] : rs[lex];
#pragma unroll
    for (int o = 0; o < NS; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = DIM == 3 ? o / 9 - 1 : 0;
      const T sv = S[(long long)o * ntot + G];   // the row's own coefficient: always in range
      const bool in = (unsigned)(i + dx) < (unsigned)A && (unsigned)(j + dy) < (unsigned)B &&
                      (unsigned)(k + dz) < (unsigned)Cz;
      const T xv = in ? x[lex + (dz * B + dy) * A + dx] : T(0);
      s -= sv * xv;
    }
    t[lex] = s;
  }
}

#define LOR_RESID(l_, rglob_) \
  residual<DIM, T>(bx[l_].A, bx[l_].B, bx[l_].C, bx[l_].org[0], bx[l_].org[1], bx[l_].org[2], a.lv[l_].N[0], \
                   a.lv[l_].N[1], a.lv[l_].ntot, (const T*)a.lv[l_].S, rglob_, rs[l_], xs[l_], ts[l_])

template <int DIM, typename T, typename FT, int NBUF>
__global__ void __launch_bounds__(256) k_patch_vcycle(PatchArgs a) {
  constexpr int ES = elem_class<FT>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int abort_flag;
  if (a.conv && *a.conv != 0.0) return;
  // shared memory: [NBUF mbarriers | pad][ring][transfer tables][wavefront tables][vectors]
  Ring<FT, NBUF> rg;
  rg.bar = (unsigned long long*)smem_raw;
  unsigned char* ring0 = smem_raw + 128;
  rg.base = ring0;
  rg.bytes = a.slot_bytes;
  rg.phase = 0;
  rg.inflight = 0;
  Xfer1D<T>* xf = (Xfer1D<T>*)(ring0 + (size_t)NBUF * a.slot_bytes);   // [level][type]
  int* ip = (int*)(xf + 2 * (a.L > 1 ? a.L - 1 : 1));
  int* ip_end = ip + a.tab_ints;
  T* sm = (T*)ip_end;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < NBUF; ++s) mbar_init(rg.bar + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // 1D transfer tables of every level (independent of the patch)
  for (int l = 0; l + 1 < a.L; ++l)
    for (int ty = 0; ty < 2; ++ty) {
      Xfer1D<T>& X = xf[l * 2 + ty];
      const int len = a.lv[l].len[ty], clen = a.lv[l].clen[ty];
      for (int f = threadIdx.x; f < len; f += blockDim.x) {
        const Prolong1D pr = a.lv[l].pp[ty][f];
        X.c0[f] = pr.c0; X.c1[f] = pr.c1; X.w0[f] = (T)pr.w0; X.w1[f] = (T)pr.w1;
      }
      if (threadIdx.x == 0) {
        int q = 0;
        for (int cc = 0; cc < clen; ++cc) {
          X.rstart[cc] = q;
          const RestrictEntry& e = a.lv[l].rr[ty][cc];
          for (int t = 0; t < e.cnt; ++t) { X.rf[q] = e.f[t]; X.rw[q] = (T)e.w[t]; ++q; }
        }
        X.rstart[clen] = q;
      }
    }
  int cur_sh = -1;
  // per-level state of the current patch: one shared copy (thread 0 writes it)
  __shared__ LevelTables tb[LOR_MAXLEV];
  __shared__ BoxShape bsh[LOR_MAXLEV];
  __shared__ Box bx[LOR_MAXLEV];
  __shared__ T* xs[LOR_MAXLEV];
  __shared__ T* ts[LOR_MAXLEV];
  __shared__ T* rs[LOR_MAXLEV];
  __shared__ long long s_offset;
  const int nwork = a.plist ? a.nlist : a.J;
  for (int jo = blockIdx.x; jo < nwork; jo += gridDim.x) {
    const int j = a.plist ? a.plist[jo] : a.porder[jo];
    int v[3];
    v[0] = j % (a.n[0] + 1);
    v[1] = (j / (a.n[0] + 1)) % (a.n[1] + 1);
    v[2] = DIM == 3 ? j / ((a.n[0] + 1) * (a.n[1] + 1)) : 0;
    int sh = 0, type[3] = {0, 0, 0};
    for (int t = 0; t < DIM; ++t) {
      type[t] = (v[t] == 0 || v[t] == a.n[t]) ? 1 : 0;
      sh |= type[t] << t;
    }
    __syncthreads();   // previous patch done with shared memory
    if (sh != cur_sh) {
      // wavefront tables of every level of this shape
      if (threadIdx.x == 0) {
        int ioff = 0;
        for (int l = 0; l < a.L; ++l) {
          bsh[l] = a.shapes[l * 8 + sh];
          tb[l].front = ip + ioff; ioff += bsh[l].nfront + 1;
          tb[l].fpad = ip + ioff; ioff += bsh[l].nfront + 1;
          tb[l].chunk = ip + ioff; ioff += bsh[l].nchunk[ES] + 1;
        }
        unsigned short* up = (unsigned short*)(ip + ioff);
        int uoff = 0;
        for (int l = 0; l < a.L; ++l) { tb[l].rowlex = up + uoff; uoff += bsh[l].rows; }
      }
      __syncthreads();
      for (int l = 0; l < a.L; ++l) {
        const int nf1 = bsh[l].nfront + 1;
        for (int i = threadIdx.x; i < nf1; i += blockDim.x) {
          ((int*)tb[l].front)[i] = a.front[bsh[l].front_off + i];
          ((int*)tb[l].fpad)[i] = a.fpad[bsh[l].front_off + i];
        }
        for (int i = threadIdx.x; i <= bsh[l].nchunk[ES]; i += blockDim.x)
          ((int*)tb[l].chunk)[i] = a.chunk[bsh[l].chunk_off[ES] + i];
        for (int i = threadIdx.x; i < bsh[l].rows; i += blockDim.x)
          ((unsigned short*)tb[l].rowlex)[i] = (unsigned short)a.rowlex[bsh[l].row_off + i];
      }
      cur_sh = sh;
    }
    if (bsh[0].rows == 0) continue;
    if (threadIdx.x == 0) {
      long long offset = 0;
      for (int l = 0; l < a.L; ++l) {
        const BoxShape& bs = bsh[l];
        Box& b = bx[l];
        b.A = bs.dims[0]; b.B = bs.dims[1]; b.C = bs.dims[2];
        b.rows = bs.rows;
        for (int t = 0; t < 3; ++t) {
          b.type[t] = type[t];
          b.org[t] = t < DIM ? (v[t] > 0 ? v[t] - 1 : 0) * a.lv[l].m + 1 : 0;
        }
        xs[l] = sm + offset; offset += b.rows;
        ts[l] = sm + offset + bs.guard; offset += b.rows + 2 * bs.guard;
        rs[l] = sm + offset; offset += (l > 0 || a.plist ? b.rows : 0);
      }
      s_offset = offset;
    }
    __syncthreads();
    for (long long i = threadIdx.x; i < s_offset; i += blockDim.x) sm[i] = T(0);
    __syncthreads();
    // level-0 right-hand side: the global vector, or the listed patch's own data
    const T* rg0 = a.plist ? nullptr : (const T*)a.r;
    if (a.plist) {
      const T* src = (const T*)a.rloc + (long long)jo * a.vstride;
      for (int lex = threadIdx.x; lex < bx[0].rows; lex += blockDim.x) rs[0][lex] = src[lex];
      __syncthreads();
    }
    const FT* F = (const FT*)a.F;
    int bottom = 0;
    while (bottom + 1 < a.L && bx[bottom + 1].rows > 0) ++bottom;
    bool ok = true;
    // ---- down
    for (int l = 0; l < bottom && ok; ++l) {
      const Box& b = bx[l];
      const PLevel& lv = a.lv[l];
      const FT* FL = F + a.facoff[(long long)l * a.J + j] * LOR_REC;
      for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
        const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
        const long long G = ((long long)(b.org[2] + k) * lv.N[1] + (b.org[1] + jj)) * lv.N[0] + (b.org[0] + i);
        ts[l][lex] = (l == 0 && rg0) ? rg0[G] : rs[l][lex];
      }
      __syncthreads();
      ok = ilu_solve<DIM, T, FT, NBUF>(bsh[l], tb[l], FL, ts[l], rg, &abort_flag);
      if (!ok) break;
      for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) xs[l][lex] = ts[l][lex];
      __syncthreads();
      LOR_RESID(l, l == 0 ? rg0 : nullptr);
      __syncthreads();
      const Xfer1D<T>& X0 = xf[l * 2 + type[0]];
      const Xfer1D<T>& X1 = xf[l * 2 + type[1]];
      const Xfer1D<T>& X2 = xf[l * 2 + type[2]];
      const int fA = b.A, fB = b.B;
      const int cA = bx[l + 1].A, cB = bx[l + 1].B, crows = bx[l + 1].rows;
      const T* tl = ts[l];
      T* rn = rs[l + 1];
      for (int lex = threadIdx.x; lex < crows; lex += blockDim.x) {
        const int ci = lex % cA, cj = (lex / cA) % cB, ck = lex / (cA * cB);
        T s = 0;
        const int z0 = DIM == 3 ? X2.rstart[ck] : 0, z1 = DIM == 3 ? X2.rstart[ck + 1] : 1;
        for (int tz = z0; tz < z1; ++tz) {
          const int fz = DIM == 3 ? X2.rf[tz] : 0;
          const T wz = DIM == 3 ? X2.rw[tz] : T(1);
          for (int ty = X1.rstart[cj]; ty < X1.rstart[cj + 1]; ++ty) {
            const T wy = X1.rw[ty] * wz;
            const int rowb = (fz * fB + X1.rf[ty]) * fA;
            for (int tx = X0.rstart[ci]; tx < X0.rstart[ci + 1]; ++tx) s += X0.rw[tx] * wy * tl[rowb + X0.rf[tx]];
          }
        }
        rn[lex] = s;
      }
      __syncthreads();
    }
    // ---- bottom level: exact solve on the vertex level (<= 1 unknown); a
    // truncated box (boundary patch whose vertex level is empty) is smoothed by
    // ILU(0) twice instead (pre and post, no coarser correction)
    if (ok) {
      const int l = bottom;
      const Box& b = bx[l];
      const PLevel& lv = a.lv[l];
      if (l == a.L - 1) {
        const T* S = (const T*)lv.S;
        for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
          const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
          const long long G = ((long long)(b.org[2] + k) * lv.N[1] + (b.org[1] + jj)) * lv.N[0] + (b.org[0] + i);
          const T rhs = (l == 0 && rg0) ? rg0[G] : rs[l][lex];
          xs[l][lex] = rhs / S[(long long)(a.NS / 2) * lv.ntot + G];
        }
        __syncthreads();
      } else {
        const FT* FL = F + a.facoff[(long long)l * a.J + j] * LOR_REC;
        for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
          const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
          const long long G = ((long long)(b.org[2] + k) * lv.N[1] + (b.org[1] + jj)) * lv.N[0] + (b.org[0] + i);
          ts[l][lex] = (l == 0 && rg0) ? rg0[G] : rs[l][lex];
        }
        __syncthreads();
        ok = ilu_solve<DIM, T, FT, NBUF>(bsh[l], tb[l], FL, ts[l], rg, &abort_flag);
        if (ok) {
          for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) xs[l][lex] = ts[l][lex];
          __syncthreads();
          LOR_RESID(l, l == 0 ? rg0 : nullptr);
          __syncthreads();
          ok = ilu_solve<DIM, T, FT, NBUF>(bsh[l], tb[l], FL, ts[l], rg, &abort_flag);
        }
        if (ok) {
          for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) xs[l][lex] += ts[l][lex];
          __syncthreads();
        }
      }
    }
    // ---- up
    for (int l = bottom - 1; l >= 0 && ok; --l) {
      const Box& b = bx[l];
      const Box& bc = bx[l + 1];
      const PLevel& lv = a.lv[l];
      const FT* FL = F + a.facoff[(long long)l * a.J + j] * LOR_REC;
      const Xfer1D<T>& X0 = xf[l * 2 + type[0]];
      const Xfer1D<T>& X1 = xf[l * 2 + type[1]];
      const Xfer1D<T>& X2 = xf[l * 2 + type[2]];
      const int fA = b.A, fB = b.B, frows = b.rows;
      const int cA = bc.A, cB = bc.B, cC = bc.C;
      const T* xc = xs[l + 1];
      T* xl = xs[l];
      for (int lex = threadIdx.x; lex < frows; lex += blockDim.x) {
        const int i = lex % fA, jj = (lex / fA) % fB, k = lex / (fA * fB);
        T s = 0;
        const int nzz = DIM == 3 ? 2 : 1;
        for (int sz = 0; sz < nzz; ++sz) {
          const int cz = DIM == 3 ? (sz ? X2.c1[k] : X2.c0[k]) : 0;
          if (cz < 0 || cz >= cC) continue;
          const T wz = DIM == 3 ? (sz ? X2.w1[k] : X2.w0[k]) : T(1);
          for (int sy = 0; sy < 2; ++sy) {
            const int cy = sy ? X1.c1[jj] : X1.c0[jj];
            if (cy < 0 || cy >= cB) continue;
            const T wy = (sy ? X1.w1[jj] : X1.w0[jj]) * wz;
            for (int sx = 0; sx < 2; ++sx) {
              const int cx = sx ? X0.c1[i] : X0.c0[i];
              if (cx < 0 || cx >= cA) continue;
              s += (sx ? X0.w1[i] : X0.w0[i]) * wy * xc[(cz * cB + cy) * cA + cx];
            }
          }
        }
        xl[lex] += s;
      }
      __syncthreads();
      LOR_RESID(l, l == 0 ? rg0 : nullptr);
      __syncthreads();
      ok = ilu_solve<DIM, T, FT, NBUF>(bsh[l], tb[l], FL, ts[l], rg, &abort_flag);
      if (!ok) break;
      for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) xs[l][lex] += ts[l][lex];
      __syncthreads();
    }
    if (!ok) {
      // a bulk copy did not arrive in time: report, drain what is still in flight, leave
      if (threadIdx.x == 0) {
        atomicOr(a.status, 4);
        for (int s = 0; s < NBUF; ++s)
          if (rg.inflight & (1u << s)) mbar_wait(rg.bar + s, (rg.phase >> s) & 1u);
      }
      return;
    }
    const Box& b = bx[0];
    const PLevel& lv = a.lv[0];
    if (a.plist) {     // patch-local output
      T* dst = (T*)a.xloc + (long long)jo * a.vstride;
      for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) dst[lex] = xs[0][lex];
      continue;
    }
    // ---- scatter-add R_j^T x_j
    T* z = (T*)a.z;
    for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) {
      const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
      const long long G = ((long long)(b.org[2] + k) * lv.N[1] + (b.org[1] + jj)) * lv.N[0] + (b.org[0] + i);
      atomicAdd(z + G, xs[0][lex]);
    }
    if (a.tout && sh == 0) {   // residual left on an interior patch, for the learned correction
      LOR_RESID(0, rg0);
      __syncthreads();
      T* dst = (T*)a.tout + (long long)jo * a.vstride;
      for (int lex = threadIdx.x; lex < b.rows; lex += blockDim.x) dst[lex] = ts[0][lex];
    }
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

const int kPatchThreads = 256;

template <typename FT>
constexpr int ring_depth() { return sizeof(FT) == 2 ? 3 : 2; }

template <typename T, typename FT>
size_t patch_smem_bytes(const lor_ctx* c, int* tab_ints = nullptr, bool local = false) {
  size_t vec = 0, tab = 0;
  for (int l = 0; l < c->L; ++l) {
    const BoxShape& bs = c->shapes[l * 8 + 0];   // interior shape is the largest
    vec += (size_t)bs.rows * (l > 0 || local ? 3 : 2) + 2 * (size_t)bs.guard;   // x, t (+guards), r
    tab += 2 * (size_t)(bs.nfront + 1) + (size_t)(bs.nchunk[elem_class<FT>()] + 1) + ((size_t)bs.rows + 1) / 2;
  }
  tab = (tab + 3) / 4 * 4;   // ints, keeps the vectors 16-byte aligned
  if (tab_ints) *tab_ints = (int)tab;
  const size_t slot = (size_t)c->maxchunk[elem_class<FT>()] * LOR_REC * sizeof(FT);
  return 128 + ring_depth<FT>() * slot + 2 * (c->L > 1 ? c->L - 1 : 1) * sizeof(Xfer1D<T>) + 4 * tab + vec * sizeof(T);
}

template <typename T, typename FT>
void fill_patch_args(lor_ctx* c, PatchArgs& a, const FT* F) {
  a.dim = c->dim; a.NS = c->NS; a.L = c->L; a.J = c->J;
  for (int t = 0; t < 3; ++t) a.n[t] = c->n[t];
  for (int l = 0; l < c->L; ++l) {
    PLevel& lv = a.lv[l];
    lv.S = Sel<T>::S(c, l);
    lv.ntot = c->lev[l].ntot;
    for (int t = 0; t < 3; ++t) lv.N[t] = c->lev[l].N[t];
    lv.m = c->lev[l].m;
    for (int t = 0; t < 2; ++t) { lv.pp[t] = c->d_pp[l][t]; lv.rr[t] = c->d_rr[l][t]; }
    for (int t = 0; t < 2; ++t) {
      const int m = c->lev[l].m, mc = l + 1 < c->L ? c->lev[l + 1].m : 1;
      lv.len[t] = t == 0 ? 2 * m - 1 : m - 1;
      lv.clen[t] = t == 0 ? 2 * mc - 1 : mc - 1;
    }
  }
  a.shapes = lor_dev_shapes(c);
  a.front = c->d_front; a.fpad = c->d_fpad; a.chunk = c->d_chunk; a.rowlex = c->d_rowlex; a.recof = c->d_recof;
  a.nbmask = c->d_nbmask;
  a.facoff = c->d_facoff;
  a.F = F; a.r = nullptr; a.z = nullptr;
  a.status = c->d_status;
  a.porder = c->d_porder;
  a.conv = c->conv_flag;
  a.plist = nullptr; a.nlist = 0; a.rloc = nullptr; a.xloc = nullptr; a.vstride = 0; a.tout = nullptr;
  a.slot_bytes = c->maxchunk[elem_class<FT>()] * LOR_REC * (int)sizeof(FT);
}

template <typename T, typename FT>
lor_status launch_patch_kernel(lor_ctx* c, PatchArgs& a, bool local) {
  const size_t smem = patch_smem_bytes<T, FT>(c, &a.tab_ints, local);
  constexpr int NB = ring_depth<FT>();
  // persistent CTAs: as many as fit on the device, each walking patches j, j+grid, ...
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long work = a.plist ? a.nlist : c->J;
  if (work <= 0) return LOR_OK;
  if (c->dim == 3) {
    auto kern = k_patch_vcycle<3, T, FT, NB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPatchThreads, smem);
    const int grid = (int)std::min<long long>(work, (long long)std::max(per_sm, 1) * nsm);
    kern<<<grid, kPatchThreads, smem, c->stream>>>(a);
  } else {
    auto kern = k_patch_vcycle<2, T, FT, NB>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPatchThreads, smem);
    const int grid = (int)std::min<long long>(work, (long long)std::max(per_sm, 1) * nsm);
    kern<<<grid, kPatchThreads, smem, c->stream>>>(a);
  }
  ++c->launches;
  return lor_cuda_check(c, cudaGetLastError(), "patch vcycle");
}

template <typename T, typename FT>
lor_status launch_apply_P(lor_ctx* c, const T* r, T* z, const FT* F) {
  const long long nvec = c->lev[0].ntot;
  cudaError_t e = cudaMemsetAsync(z, 0, sizeof(T) * nvec, c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "apply_P memset");
  PatchArgs a;
  fill_patch_args<T, FT>(c, a, F);
  a.r = r; a.z = z;
  if (c->learned_on && sizeof(T) == 4) {
    a.tout = c->learned_tout;
    a.vstride = c->shapes[0].rows;
  }
  const int pk = sizeof(T) == 8 ? 0 : 1;
  lor_prof_begin(c, pk);
  if (launch_patch_kernel<T, FT>(c, a, false)) return LOR_ECUDA;
  lor_prof_end(c, pk);
  if (c->learned_on && sizeof(T) == 4) {
    if (lor_learned_apply(c, (float*)z)) return LOR_ECUDA;
  }
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
  return launch_apply_P<double, double>(c, r, z, c->d_F64);
}

lor_status lor_launch_apply_P32(lor_ctx* c, const float* r, float* z) {
  if (c->d_F16) return launch_apply_P<float, __nv_bfloat16>(c, r, z, c->d_F16);
  return launch_apply_P<float, float>(c, r, z, c->d_F32);
}

// Patch-local V-cycles (FP32 vectors) of the listed patches: rhs rloc -> x xloc.
lor_status lor_patch_local32(lor_ctx* c, const int* plist, int nlist, const float* rloc, float* xloc, int vstride) {
  PatchArgs a;
  if (c->d_F16) {
    fill_patch_args<float, __nv_bfloat16>(c, a, c->d_F16);
    a.plist = plist; a.nlist = nlist; a.rloc = rloc; a.xloc = xloc; a.vstride = vstride;
    return launch_patch_kernel<float, __nv_bfloat16>(c, a, true);
  }
  fill_patch_args<float, float>(c, a, c->d_F32);
  a.plist = plist; a.nlist = nlist; a.rloc = rloc; a.xloc = xloc; a.vstride = vstride;
  return launch_patch_kernel<float, float>(c, a, true);
}

size_t lor_patch_smem(const lor_ctx* c, int which) {
  if (which == 0) return patch_smem_bytes<double, double>(c);
  if (which == 1) return patch_smem_bytes<float, float>(c);
  return patch_smem_bytes<float, __nv_bfloat16>(c);
}
