// Additive-Schwarz LOR preconditioner z = B r (Section 3.2, Eq. (as)):
//   B = P_0 R_0 P_0^T + sum_j R_j^T V_j R_j,
// with one vertex patch per coarse vertex (Eq. (patch)) and V_j one V(1,1) cycle
// of the element-structured hierarchy (Section 3.3) smoothed by lexicographic
// ILU(0) (Section 3.4).
//
// Patch kernel: each patch group (one warp, or two warps when shared memory
// holds at most 8 patches per SM) runs the whole V-cycle of one patch at a time:
// gather R_j r, per level ILU(0) pre-smoothing (wavefront-scheduled forward and
// backward sweeps over factor records streamed by bulk copies), 3^d-point
// residual with the level's Galerkin LOR stencil, tensor restriction, exact
// solve on the vertex level (<= 1 unknown), then prolongation, residual and
// post-smoothing on the way up; x_j goes to the patch's own slice of a
// per-patch buffer, and a gather kernel sums the slices of the (at most 2^d)
// patches containing each node in a fixed order, so z is reproducible bit for
// bit.  Many patches
// are in flight per SM (one per group), so the latency-bound sweeps of one patch
// overlap those of the others; a two-warp group splits the rows of every loop
// and of every wavefront between its warps.  Vectors live in zero-padded boxes
// so that factor reads need no bounds checks (factors of out-of-box couplings
// are stored as 0); the level-0 iterate is kept in a per-group global slot (L2) and
// the level-0 residual is formed in place, which keeps a patch's shared-memory
// footprint to the level-0 work vector, the coarse levels and the copy ring.
//
// Coarse space: P_0^T r at the interior vertices, one V-cycle on the vertex grid
// (l1-Jacobi smoothing, Galerkin levels, dense inverse on the coarsest grid),
// z += P_0 e.
#include <algorithm>

#include "lor_internal.h"

namespace {

struct PLevel {
  const void* S;          // [NS][ntot] stencil of this level (T)
  const void* Sa;         // [ntot][nsp] row-major copy (T)
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
  const int* fpad;
  const int* chunk;
  const GenSched* gsched;       // ordered or enlarged patches: per-patch schedules and boxes [L][J] (else null)
  const void* xferg;            //   patch-local transfers XferG<T>[level][kmax1] (span of k elements)
  int kmax1;
  const void* binv;             //   vertex-level inverses (T), offsets in gsched[L-1][j].binv_off
  const long long* facoff;      // [L][J] record offsets
  const void* F;
  const void* r;
  void* zp;                     // per-patch outputs (T): patch j at zp + j * zstride, lexicographic box order
  long long zstride;
  int* status;
  int slot_bytes;               // ring slot size (bytes, multiple of 16)
  int tab_ints;                 // per-group shared-memory ints reserved for wavefront tables
  int xf_bytes;                 // shared transfer tables at the start of dynamic shared memory
  int warp_bytes;               // per-group block size (bytes, multiple of 128)
  int aux_n;                    // per-group vector layout: auxiliary buffers (plane buffers / r1)
  int ovl_n;                    //   then level-0 t with guards, overlaid by the coarse levels
  void* xs;                     // per-group level-0 iterate slots (T), x0_stride values each
  long long x0_stride;
  const int* porder;            // patch visiting order (grouped by box shape)
  const double* conv;           // optional: skip all work when *conv != 0 (converged batched solve)
  int wp;                       // > 0: patch sum weighted on both sides (wp = p), 0: unit weights
  int wmode;                    //   1: counting matrix D^{-1/2}, 2: partition of unity sqrt(theta_v)
  const void* hat;              //   vertex hat table of the coarse space (T), used by mode 2
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
  // the learned correction's replace variant: the level-0 post-smoothing is left out
  // (the cycle returns x0 after the coarse correction; the residual r - A x0 it
  // leaves is what the correction sees)
  int skip_post0;
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
  // factor records are read once per smoothing: evict them from L2 first, so that
  // the stencil rows shared by neighbouring patches stay resident
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}

// Waits for the phase `parity` of `bar`; gives up after `limit` polls (returns
// false) so that a lost copy cannot hang the GPU.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int limit = 1 << 22) {
  const unsigned addr = smem_u32(bar);
  for (int it = 0; it < limit; ++it) {
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


// The threads that run one patch: one warp (WG = 1) or two warps (WG = 2, named
// barrier 1 + group index over their 64 threads).  Every branch that a group
// takes around a sync() depends only on values the whole group holds alike.
template <int WG>
struct Grp {
  static constexpr int NT = 32 * WG;
  int gl;   // thread index in the group
  int id;   // group index in the CTA
  __device__ __forceinline__ void sync() const {
    if constexpr (WG == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + id), "r"(NT) : "memory");
  }
};

// One factor record held in registers: R values of type FT as 32-bit words.
template <int R, typename FT>
struct RecRegs {
  static constexpr int NW = R * (int)sizeof(FT) / 4;
  unsigned w[NW];
  __device__ __forceinline__ void load(const FT* rec) {
    const uint4* q = (const uint4*)rec;
#pragma unroll
    for (int v = 0; v < NW / 4; ++v) {
      const uint4 u = q[v];
      w[4 * v] = u.x; w[4 * v + 1] = u.y; w[4 * v + 2] = u.z; w[4 * v + 3] = u.w;
    }
  }
  // value of slot o (o a compile-time constant after unrolling)
  template <typename T>
  __device__ __forceinline__ T val(int o) const {
    if constexpr (sizeof(FT) == 2) {
      const unsigned x = w[o >> 1];
      return (T)__uint_as_float((o & 1) ? (x & 0xffff0000u) : (x << 16));
    } else if constexpr (sizeof(FT) == 4) {
      return (T)__uint_as_float(w[o]);
    } else {
      return (T)__hiloint2double((int)w[2 * o + 1], (int)w[2 * o]);
    }
  }
};

// Row index (slot R-1, raw integer bits) of the record at rec.
template <int R, typename FT>
__device__ __forceinline__ int rec_index(const FT* rec) {
  if constexpr (sizeof(FT) == 2) return ((const unsigned short*)rec)[R - 1];
  else if constexpr (sizeof(FT) == 4) return ((const int*)rec)[R - 1];
  else return ((const int*)rec)[2 * (R - 1)];
}

// NR rows of one front of a sweep (row u: record rec[u], box index li[u]):
// t[li] -= sum of the row's strictly lower (forward) or upper (backward, then
// scaled by 1/u_ii) couplings.  Rows of one front never couple, so every load
// of the front is issued before its first store; the row indices of the next
// front (records nrec[u], read only if nxt) are loaded in the same round.
// Value of slot o of a record in shared memory (ordered records are read in place).
template <typename T, typename FT>
__device__ __forceinline__ T rec_val(const FT* rec, int o) {
  if constexpr (sizeof(FT) == 2) return (T)__bfloat162float(rec[o]);
  else return (T)rec[o];
}

template <int DIM, bool BACK, typename T, typename FT, int NR, bool GEN>
__device__ __forceinline__ void sweep_front(const FT* const* rec, int* li, const FT* const* nrec, bool nxt, int A,
                                            int AB, T* t) {
  constexpr int NS = DIM == 3 ? 27 : 9;
  constexpr int C = NS / 2;
  // lexicographic records: the 13 (4) lower or upper couplings; ordered records:
  // all 26 (8) couplings, zero where the neighbour is on the other side of the row
  constexpr int NC = GEN ? NS - 1 : C;
  constexpr int R = GEN ? lor_rec_gen(DIM) : lor_rec(DIM);
  RecRegs<GEN ? 4 : R, FT> rr[NR];
  T tv[NR][NC + 1];
#pragma unroll
  for (int u = 0; u < NR; ++u) {
    if constexpr (!GEN) rr[u].load(rec[u]);
    tv[u][NC] = t[li[u]];
#pragma unroll
    for (int o = 0; o < NC; ++o) {
      const int so = GEN ? (o < C ? o : o + 1) : (BACK ? C + 1 + o : o);   // stencil offset index
      const int dx = so % 3 - 1, dy = (so / 3) % 3 - 1, dz = DIM == 3 ? so / 9 - 1 : 0;
      tv[u][o] = t[li[u] + dz * AB + dy * A + dx];
    }
  }
  int ln[NR];
#pragma unroll
  for (int u = 0; u < NR; ++u) ln[u] = nxt ? rec_index<R, FT>(nrec[u]) : 0;
#pragma unroll
  for (int u = 0; u < NR; ++u) {
    T s0 = tv[u][NC], s1 = T(0);
#pragma unroll
    for (int o = 0; o < NC; ++o) {
      T w;
      if constexpr (GEN) w = rec_val<T, FT>(rec[u], o);
      else w = rr[u].template val<T>(o);
      const T v = w * tv[u][o];
      if (o & 1) s1 -= v; else s0 -= v;
    }
    T dinv;
    if constexpr (GEN) dinv = rec_val<T, FT>(rec[u], R - 2);
    else dinv = rr[u].template val<T>(R - 2);
    t[li[u]] = BACK ? (s0 + s1) * dinv : s0 + s1;
  }
#pragma unroll
  for (int u = 0; u < NR; ++u) li[u] = ln[u];
}

// One triangular sweep over a level, run by one patch group.  Factor blocks
// stream through the ring in chunks of whole fronts: thread 0 of the group issues
// the bulk copies and observes their completion, then publishes it (and whether
// the copy arrived in time) to the group.  Inside a chunk, a one-warp group takes
// records q and q+32 of a front in lane q (fronts hold at most 64 records; the
// second row only when the front is wider than 32); a two-warp group takes record
// q in thread q, and its second warp sits out fronts of at most 32 rows.  A thread
// without a row reads the all-zero record zrec, whose row index `dummy` is the
// first guard cell after the box, and writes 0 there, like a padding record.  The
// row indices of the next front are read ahead so that a front's critical path is
// one round of shared-memory loads of t.  The group synchronizes between fronts.
// t has a zero guard band, so neighbour reads need no clamping (multipliers of
// out-of-box neighbours are stored as 0).  BACK selects the backward sweep (U
// part, fronts in reverse, scaled by 1/u_ii).  okf: a shared word of the group.
template <int DIM, bool BACK, typename T, typename FT, int NBUF, bool GEN, int WG>
__device__ __forceinline__ bool sweep(const FT* __restrict__ part, const int* __restrict__ fp,
                                      const int* __restrict__ ch, int nc, int A, int AB, int dummy,
                                      const FT* zrec, T* t, Ring<FT, NBUF>& rg, const Grp<WG>& g, int* okf) {
  constexpr int R = GEN ? lor_rec_gen(DIM) : lor_rec(DIM);
  const int gl = g.gl;
  // chunk c of the sweep (fronts in reverse order when BACK): its records
  auto chunk_src = [&](int c) { return part + (long long)fp[ch[BACK ? nc - 1 - c : c]] * R; };
  auto chunk_bytes = [&](int c) {
    const int k = BACK ? nc - 1 - c : c;
    return (unsigned)((fp[ch[k + 1]] - fp[ch[k]]) * R * sizeof(FT));
  };
  if (gl == 0) {
    for (int c = 0; c < NBUF - 1 && c < nc; ++c) {
      bulk_load(rg.slot(c % NBUF), chunk_src(c), chunk_bytes(c), rg.bar + (c % NBUF));
      rg.inflight |= 1u << (c % NBUF);
    }
  }
  for (int c = 0; c < nc; ++c) {
    const int sl = c % NBUF;
    int ok = 1;
    if (gl == 0) ok = mbar_wait(rg.bar + sl, (rg.phase >> sl) & 1u) ? 1 : 0;
    rg.phase ^= 1u << sl;
    if constexpr (WG == 1) {
      ok = __shfl_sync(0xffffffffu, ok, 0);
    } else {
      if (gl == 0) *okf = ok;
      g.sync();
      ok = *okf;
    }
    if (!ok) return false;
    if (gl == 0) {
      rg.inflight &= ~(1u << sl);
      const int cn = c + NBUF - 1;
      if (cn < nc) {
        bulk_load(rg.slot(cn % NBUF), chunk_src(cn), chunk_bytes(cn), rg.bar + (cn % NBUF));
        rg.inflight |= 1u << (cn % NBUF);
      }
    }
    if constexpr (WG == 1) __syncwarp();
    const FT* blk = rg.slot(sl);
    const int k = BACK ? nc - 1 - c : c;
    const int fa = ch[k], fb = ch[k + 1], nf = fb - fa;
    const int r0 = fp[fa];
    // records [b, e) of the block for the current front, and their row indices
    int f = BACK ? fb - 1 : fa;
    int b = fp[f] - r0, e = fp[f + 1] - r0;
    if constexpr (WG == 1) {
      const int lane = gl;
      int li[2];
      li[0] = lane < e - b ? rec_index<R, FT>(blk + (b + lane) * R) : dummy;
      li[1] = lane + 32 < e - b ? rec_index<R, FT>(blk + (b + lane + 32) * R) : dummy;
      for (int q = 0; q < nf; ++q) {
        const int n = e - b;
        const bool more = q + 1 < nf;
        // the next front shares one bound with this one
        int bn = b, en = e;
        if (more) {
          if (BACK) { en = b; bn = fp[f - 1] - r0; }
          else { bn = e; en = fp[f + 2] - r0; }
        }
        const FT* rec[2] = {lane < n ? blk + (b + lane) * R : zrec, lane + 32 < n ? blk + (b + lane + 32) * R : zrec};
        const FT* nrec[2] = {lane < en - bn ? blk + (bn + lane) * R : zrec,
                             lane + 32 < en - bn ? blk + (bn + lane + 32) * R : zrec};
        if (n > 32) {   // warp-uniform
          sweep_front<DIM, BACK, T, FT, 2, GEN>(rec, li, nrec, more, A, AB, t);
        } else {
          sweep_front<DIM, BACK, T, FT, 1, GEN>(rec, li, nrec, more, A, AB, t);
          li[1] = more ? rec_index<R, FT>(nrec[1]) : dummy;
        }
        if (more) {
          // lanes past the next front's rows take the zero record (index dummy)
          if (!(lane < en - bn)) li[0] = dummy;
          if (!(lane + 32 < en - bn)) li[1] = dummy;
        }
        f = BACK ? f - 1 : f + 1; b = bn; e = en;
        __syncwarp();
      }
    } else {
      const int w32 = gl & ~31;   // first record of this warp
      int li[1];
      li[0] = gl < e - b ? rec_index<R, FT>(blk + (b + gl) * R) : dummy;
      for (int q = 0; q < nf; ++q) {
        const int n = e - b;
        const bool more = q + 1 < nf;
        int bn = b, en = e;
        if (more) {
          if (BACK) { en = b; bn = fp[f - 1] - r0; }
          else { bn = e; en = fp[f + 2] - r0; }
        }
        const FT* rec[1] = {gl < n ? blk + (b + gl) * R : zrec};
        const FT* nrec[1] = {gl < en - bn ? blk + (bn + gl) * R : zrec};
        if (n > w32) sweep_front<DIM, BACK, T, FT, 1, GEN>(rec, li, nrec, more, A, AB, t);   // warp-uniform
        else li[0] = more ? rec_index<R, FT>(nrec[0]) : dummy;
        if (more && !(gl < en - bn)) li[0] = dummy;
        f = BACK ? f - 1 : f + 1; b = bn; e = en;
        g.sync();
      }
    }
  }
  return true;
}

// in-place (L U)^{-1} t on one level, run by the calling group (forward then
// backward sweep).  Returns false if a bulk copy timed out (the whole group
// returns false).
template <typename FT>
constexpr int elem_class() { return sizeof(FT) == 2 ? 0 : (sizeof(FT) == 4 ? 1 : 2); }

template <int DIM, typename T, typename FT, int NBUF, bool GEN, int WG>
__device__ __forceinline__ bool ilu_solve(const BoxShape& bs, const int* fp, const int* ch, const FT* FL, T* t,
                                          Ring<FT, NBUF>& rg, const FT* zrec, const Grp<WG>& g, int* okf) {
  constexpr int ES = elem_class<FT>();
  constexpr int R = GEN ? lor_rec_gen(DIM) : lor_rec(DIM);
  const int A = bs.dims[0], AB = bs.dims[0] * bs.dims[1];
  bool ok = sweep<DIM, false, T, FT, NBUF, GEN, WG>(FL, fp, ch, bs.nchunk[ES], A, AB, bs.rows, zrec, t, rg, g, okf);
  if (ok)
    ok = sweep<DIM, true, T, FT, NBUF, GEN, WG>(FL + (long long)bs.rpad * R, fp, ch, bs.nchunk[ES], A, AB, bs.rows,
                                                 zrec, t, rg, g, okf);
  g.sync();
  return ok;
}

// Strided walk over the rows of a box in lexicographic order: the thread starts
// at row lex0 and advances by `stride` rows per step (the threads of its patch
// group), tracking (i, j, k).
struct BoxIter {
  int i, j, k;
  int si, sj, sk;   // stride = sk*A*B + sj*A + si
  int A, B;
  __device__ __forceinline__ void init(int lex0, int A_, int B_, int stride) {
    A = A_; B = B_;
    i = lex0 % A; j = (lex0 / A) % B; k = lex0 / (A * B);
    si = stride % A; sj = (stride / A) % B; sk = stride / (A * B);
  }
  __device__ __forceinline__ void next() {
    i += si;
    int c = i >= A;
    i -= c ? A : 0;
    j += sj + c;
    c = j >= B;
    j -= c ? B : 0;
    k += sk + c;
  }
};

// One patch level as seen by a warp: box extents, origin in the level grid, and
// the shared-memory vectors (offsets from the warp's vector base; -1: absent).
struct WLevel {
  int A, B, C, rows;
  int org[3];
  int xo, to, ro;   // x (with guards), t (with guards), rhs
};

// Row s of the row-major stencil (nsp values) into registers.
template <int DIM, typename T>
__device__ __forceinline__ void load_row(const T* __restrict__ Sa, int G, T* s) {
  constexpr int NSP = lor_nsp(DIM);
  const uint4* q = (const uint4*)(Sa + (size_t)G * NSP);
  constexpr int NV = NSP * (int)sizeof(T) / 16;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const uint4 u = __ldg(q + v);
    if constexpr (sizeof(T) == 4) {
      s[4 * v] = __uint_as_float(u.x); s[4 * v + 1] = __uint_as_float(u.y);
      s[4 * v + 2] = __uint_as_float(u.z); s[4 * v + 3] = __uint_as_float(u.w);
    } else {
      s[2 * v] = __hiloint2double((int)u.y, (int)u.x);
      s[2 * v + 1] = __hiloint2double((int)u.w, (int)u.z);
    }
  }
}

// rhs - sum_o S_o x(nbr_o) for the row (i, j, k) of a box (A, B, C): out-of-box
// neighbours contribute nothing (the patch operator R_j A R_j^T keeps only
// couplings inside the box).  xv(o) returns the neighbour value; its index is
// always inside a guarded array, so reads are safe before masking.
template <int DIM, typename T, typename XV>
__device__ __forceinline__ T row_residual(const T* s, T rhs, int i, int j, int k, int A, int B, int C, XV xv) {
  constexpr int NS = DIM == 3 ? 27 : 9;
  T acc0 = rhs, acc1 = T(0);
#pragma unroll
  for (int o = 0; o < NS; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = DIM == 3 ? o / 9 - 1 : 0;
    const bool in = (unsigned)(i + dx) < (unsigned)A && (unsigned)(j + dy) < (unsigned)B &&
                    (DIM == 2 || (unsigned)(k + dz) < (unsigned)C);
    const T v = in ? xv(o, dx, dy, dz) : T(0);
    if (o & 1) acc1 -= s[o] * v;
    else acc0 -= s[o] * v;
  }
  return acc0 + acc1;
}

// Counting-matrix weight D^{-1/2} of a level-0 node (I, J, K): D is the number of
// vertex patches containing it, 2 per axis along which the node lies strictly
// inside an element (both vertices of that element edge carry a patch) and 1
// where it lies on a vertex plane.
template <int DIM, typename T>
__device__ __forceinline__ T count_weight(int I, int J, int K, int p) {
  const int c = (I % p != 0) + (J % p != 0) + (DIM == 3 ? (K % p != 0) : 0);
  return T(1) / sqrt(T(1 << c));
}

// Weight of level-0 node (I, J, K) in the patch sum.  mode 1: the counting-matrix
// weight above.  mode 2: the partition of unity sqrt(theta_v), theta_v the Q1
// function of the patch's vertex v in the element reference coordinates.  Along
// axis a it is the vertex hat, which the coarse-space table holds at positions
// p + t, t = I - (v_a - 1) p in [1, 2p - 1] for every node of the patch; ho_a =
// (2 - v_a) p turns the global index into that position.
template <int DIM, typename T>
__device__ __forceinline__ T node_weight(int mode, int I, int J, int K, int p, int ho0, int ho1, int ho2,
                                         const T* __restrict__ hat) {
  if (mode == 1) return count_weight<DIM, T>(I, J, K, p);
  T h = hat[ho0 + I] * hat[ho1 + J];
  if (DIM == 3) h *= hat[ho2 + K];
  return sqrt(h);
}

// ho_a = (2 - v_a) p for the vertex v of patch j on an n0 x n1 (x n2) element grid
// (vertices numbered x fastest).
template <int DIM>
__device__ __forceinline__ void hat_offsets(int j, int n0, int n1, int p, int* ho) {
  const int v0 = j % (n0 + 1), v1 = (j / (n0 + 1)) % (n1 + 1);
  ho[0] = (2 - v0) * p;
  ho[1] = (2 - v1) * p;
  ho[2] = DIM == 3 ? (2 - j / ((n0 + 1) * (n1 + 1))) * p : 0;
}

// Level-0 residual in place: t holds x on entry (rows of the box, zero guard
// bands) and rhs - A x on exit.  Planes are done in order; plane k is computed
// into tmp from prev (x of plane k-1, guarded) and t (planes k, k+1 still x),
// then plane k's x moves to prev (and to xout, when given) and tmp into t.
// wp > 0: the global right-hand side is weighted (node_weight with mode wmode).
template <int DIM, typename T, int WG>
__device__ void resid0_inplace(const WLevel& b, const PLevel& lv, const T* __restrict__ rg0,
                               const T* __restrict__ rloc, T* t, T* prev, T* tmp, T* xout, int wp, int wmode,
                               int jp, int n0, int n1, const T* __restrict__ hat, const Grp<WG>& g) {
  constexpr int NSP = lor_nsp(DIM);
  constexpr int NT = Grp<WG>::NT;
  const int gl = g.gl;
  const int A = b.A, B = b.B, C = b.C, AB = A * B;
  const T* Sa = (const T*)lv.Sa;
  const int N0 = lv.N[0], N1 = lv.N[1];
  int ho[3] = {0, 0, 0};
  if (wmode == 2) hat_offsets<DIM>(jp, n0, n1, wp, ho);
  for (int k = 0; k < C; ++k) {
    BoxIter it;
    it.init(gl, A, B, NT);   // walks plane-local rows (k component unused)
    for (int p = gl; p < AB; p += NT, it.next()) {
      const int i = it.i, j = it.j;
      const int lex = k * AB + p;
      const int G = ((b.org[2] + k) * N1 + (b.org[1] + j)) * N0 + (b.org[0] + i);
      T s[NSP];
      load_row<DIM, T>(Sa, G, s);
      T rhs = rloc ? rloc[lex] : rg0[G];
      if (wp) rhs *= node_weight<DIM, T>(wmode, b.org[0] + i, b.org[1] + j, b.org[2] + k, wp, ho[0], ho[1], ho[2], hat);
      tmp[p] = row_residual<DIM, T>(s, rhs, i, j, k, A, B, C, [&](int o, int dx, int dy, int dz) -> T {
        return dz < 0 ? prev[p + dy * A + dx] : t[lex + dz * AB + dy * A + dx];
      });
    }
    g.sync();
    for (int p = gl; p < AB; p += NT) {
      const T xv = t[k * AB + p];
      prev[p] = xv;
      if (xout) xout[k * AB + p] = xv;
      t[k * AB + p] = tmp[p];
    }
    g.sync();
  }
}

// t = r - A x on a level l >= 1 (separate guarded arrays).
template <int DIM, typename T, int WG>
__device__ void resid_level(const WLevel& b, const PLevel& lv, const T* r, const T* x, T* t, const Grp<WG>& g) {
  constexpr int NSP = lor_nsp(DIM);
  constexpr int NT = Grp<WG>::NT;
  const int A = b.A, B = b.B, C = b.C, AB = A * B;
  const T* Sa = (const T*)lv.Sa;
  const int N0 = lv.N[0], N1 = lv.N[1];
  BoxIter it;
  it.init(g.gl, A, B, NT);
  for (int lex = g.gl; lex < b.rows; lex += NT, it.next()) {
    const int G = ((b.org[2] + it.k) * N1 + (b.org[1] + it.j)) * N0 + (b.org[0] + it.i);
    T s[NSP];
    load_row<DIM, T>(Sa, G, s);
    t[lex] = row_residual<DIM, T>(s, r[lex], it.i, it.j, it.k, A, B, C, [&](int o, int dx, int dy, int dz) -> T {
      return x[lex + dz * AB + dy * A + dx];
    });
  }
  g.sync();
}

// r_c = R t: tensor restriction of a level-l vector to level l+1 (patch-local).
template <int DIM, typename T, typename X, int WG>
__device__ void restrict_level(const WLevel& bf, const WLevel& bc, const X& X0, const X& X1, const X& X2, const T* tl,
                               T* rn, const Grp<WG>& g) {
  constexpr int NT = Grp<WG>::NT;
  const int fA = bf.A, fB = bf.B, cA = bc.A, cB = bc.B;
  BoxIter it;
  it.init(g.gl, cA, cB, NT);
  for (int lex = g.gl; lex < bc.rows; lex += NT, it.next()) {
    const int ci = it.i, cj = it.j, ck = it.k;
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
  g.sync();
}

// (P x_c)(row) for a fine row (i, j, k) of level l (patch-local tensor prolongation).
template <int DIM, typename T, typename X>
__device__ __forceinline__ T prolong_row(const WLevel& bc, const X& X0, const X& X1, const X& X2, const T* xc, int i,
                                         int j, int k) {
  const int cA = bc.A, cB = bc.B, cC = bc.C;
  T s = 0;
  const int nzz = DIM == 3 ? 2 : 1;
  for (int sz = 0; sz < nzz; ++sz) {
    const int cz = DIM == 3 ? (sz ? X2.c1[k] : X2.c0[k]) : 0;
    if (cz < 0 || cz >= cC) continue;
    const T wz = DIM == 3 ? (sz ? X2.w1[k] : X2.w0[k]) : T(1);
    for (int sy = 0; sy < 2; ++sy) {
      const int cy = sy ? X1.c1[j] : X1.c0[j];
      if (cy < 0 || cy >= cB) continue;
      const T wy = (sy ? X1.w1[j] : X1.w0[j]) * wz;
      for (int sx = 0; sx < 2; ++sx) {
        const int cx = sx ? X0.c1[i] : X0.c0[i];
        if (cx < 0 || cx >= cA) continue;
        s += (sx ? X0.w1[i] : X0.w0[i]) * wy * xc[(cz * cB + cy) * cA + cx];
      }
    }
  }
  return s;
}

// Rows a lane keeps in flight in the simple global-memory loops of the patch
// kernel (gather, slot updates, scatter): their loads are issued together, so one
// latency covers all of them.
constexpr int kRowsInFlight = 4;

// Per-group shared-memory block (byte offsets): mbarriers, the group's
// copy-arrival flag, a zero factor record, level metadata of the current box
// shape, the bulk-copy ring, the wavefront tables of the shape, and the vectors.
// The zero record spans the widest record (32 doubles of an ordered FP64 level).
constexpr int kWarpBars = 0, kWarpZrec = 32, kWarpMeta = 288, kWarpShape = 352, kWarpRing = 768;
constexpr int kWarpOk = 24;   // after the ring mbarriers
static_assert(kWarpBars + 2 * 8 <= kWarpOk && kWarpOk + 4 <= kWarpZrec, "group flag overlaps the mbarriers");
static_assert(kWarpMeta - kWarpZrec >= 32 * 8, "zero record smaller than an ordered FP64 record");
static_assert(kWarpShape - kWarpMeta >= 2 * LOR_MAXLEV * 4, "level metadata does not fit");
static_assert(kWarpRing - kWarpShape >= LOR_MAXLEV * (int)sizeof(BoxShape), "box shapes do not fit");
// ordered/enlarged patches: per level the box origin and the elements spanned per axis
// (6 ints), then the ring
constexpr int kWarpGeo = 736, kWarpRingGen = 896;
static_assert(kWarpGeo >= kWarpShape + LOR_MAXLEV * (int)sizeof(BoxShape), "geometry overlaps the box shapes");
static_assert(kWarpRingGen - kWarpGeo >= LOR_MAXLEV * 6 * 4, "geometry does not fit");
__host__ __device__ constexpr int warp_ring_offset(bool gen) { return gen ? kWarpRingGen : kWarpRing; }

// The patch kernel.  Each group of WG warps runs whole V-cycles for its own
// patches (one after another; no block barriers, only the group's own):
//   t0 <- R_j r; t0 <- ILU(t0) (= x0); x0 -> its global slot, t0 <- r - A x0
//   (in place); r1 <- R t0; levels 1..bottom as below; x0 += P x1 (global
//   slot); t0 <- x0; t0 <- r - A x0; t0 <- ILU(t0); z += R_j^T (x0 + t0).
// Levels l >= 1 live in shared memory over t0's space: down: t <- r,
// ILU, x <- t, t <- r - A x, r_{l+1} <- R t; the vertex level is solved exactly
// (<= 1 unknown), a truncated box (boundary patch whose vertex level is empty)
// is smoothed by ILU twice instead; up: x += P x_{l+1}, t <- r - A x, ILU, x += t.
template <int DIM, typename T, typename FT, int NBUF, bool GEN, int WG>
__global__ void __launch_bounds__(WG == 2 ? 512 : 384, 1) k_patch_warp(PatchArgs a) {
  constexpr int ES = elem_class<FT>();
  constexpr int R = GEN ? lor_rec_gen(DIM) : lor_rec(DIM);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (a.conv && *a.conv != 0.0) return;
  static_assert(NBUF * 8 <= kWarpOk, "ring mbarriers overlap the group flag");
  constexpr int NT = Grp<WG>::NT;
  const Grp<WG> g{(int)(threadIdx.x % NT), (int)(threadIdx.x / NT)};
  const int gl = g.gl, ng = blockDim.x / NT;
  // CTA-wide: 1D transfer tables of every level (independent of the patch)
  Xfer1D<T>* xf = (Xfer1D<T>*)smem_raw;   // [level][axis type]
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
  __syncthreads();
  // per-group block
  unsigned char* wb = smem_raw + a.xf_bytes + (size_t)g.id * a.warp_bytes;
  Ring<FT, NBUF> rg;
  rg.bar = (unsigned long long*)(wb + kWarpBars);
  rg.base = wb + warp_ring_offset(GEN);
  rg.bytes = a.slot_bytes;
  rg.phase = 0;
  rg.inflight = 0;
  const FT* zrec = (const FT*)(wb + kWarpZrec);
  int* okf = (int*)(wb + kWarpOk);   // copy-arrival flag published to the group
  int* meta = (int*)(wb + kWarpMeta);   // tbf[LOR_MAXLEV] | tbc[LOR_MAXLEV]
  BoxShape* bsh = (BoxShape*)(wb + kWarpShape);
  int* ip = (int*)(wb + warp_ring_offset(GEN) + (size_t)NBUF * a.slot_bytes);
  int* geo = (int*)(wb + kWarpGeo);     // GEN: [level][org x3, k x3]
  T* vec = (T*)(ip + a.tab_ints);
  for (int q = gl; q < 64; q += NT) ((unsigned*)(wb + kWarpZrec))[q] = 0u;
  if (gl == 0) {
    for (int s = 0; s < NBUF; ++s) mbar_init(rg.bar + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  g.sync();
  const long long gw = (long long)blockIdx.x * ng + g.id;
  T* xslot = (T*)a.xs + gw * a.x0_stride;       // this group's level-0 iterate
  const int nwork = a.plist ? a.nlist : a.J;
  const long long step = (long long)gridDim.x * ng;
  int cur_sh = -1;
  const FT* F = (const FT*)a.F;
  const T* hat = (const T*)a.hat;
  for (long long jo = gw; jo < nwork; jo += step) {
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
    if (GEN || sh != cur_sh) {
      // wavefront tables of every level of this shape (ordered levels: of this patch)
      g.sync();
      if (gl == 0) {
        int ioff = 0;
        for (int l = 0; l < a.L; ++l) {
          bsh[l] = a.shapes[l * 8 + sh];
          if (GEN) {
            const GenSched gs = a.gsched[(long long)l * a.J + j];
            bsh[l].nfront = gs.nfront;
            bsh[l].rpad = gs.rpad;
            bsh[l].front_off = gs.front_off;
            for (int e = 0; e < 3; ++e) { bsh[l].nchunk[e] = gs.nchunk[e]; bsh[l].chunk_off[e] = gs.chunk_off[e]; }
            for (int e = 0; e < 3; ++e) { bsh[l].dims[e] = gs.dims[e]; geo[l * 6 + e] = gs.org[e]; geo[l * 6 + 3 + e] = gs.k[e]; }
            bsh[l].rows = gs.rows;
            bsh[l].guard = gs.guard;
          }
          meta[l] = ioff; ioff += bsh[l].nfront + 1;
          meta[LOR_MAXLEV + l] = ioff; ioff += bsh[l].nchunk[ES] + 1;
        }
      }
      g.sync();
      for (int l = 0; l < a.L; ++l) {
        const int nf1 = bsh[l].nfront + 1;
        for (int i = gl; i < nf1; i += NT) ip[meta[l] + i] = a.fpad[bsh[l].front_off + i];
        for (int i = gl; i <= bsh[l].nchunk[ES]; i += NT) ip[meta[LOR_MAXLEV + l] + i] = a.chunk[bsh[l].chunk_off[ES] + i];
      }
      g.sync();
      cur_sh = sh;
    }
    if (bsh[0].rows == 0) continue;
    // level boxes and their vectors: level 0 keeps t0 after the auxiliary
    // buffers; levels >= 1 overlay t0's space (x, t with guards, r)
    WLevel bx[LOR_MAXLEV];
    int bottom = 0;
    {
      long long off = a.aux_n;
      for (int l = 0; l < a.L; ++l) {
        const BoxShape& bs = bsh[l];
        WLevel& b = bx[l];
        b.A = bs.dims[0]; b.B = bs.dims[1]; b.C = bs.dims[2];
        b.rows = bs.rows;
        for (int t = 0; t < 3; ++t)
          b.org[t] = GEN ? geo[l * 6 + t] : (t < DIM ? (v[t] > 0 ? v[t] - 1 : 0) * a.lv[l].m + 1 : 0);
        if (l == 0) {
          b.xo = -1; b.to = a.aux_n + bs.guard; b.ro = -1;
        } else {
          b.xo = (int)off + bs.guard; off += b.rows + 2 * bs.guard + 1;
          b.to = (int)off + bs.guard; off += b.rows + 2 * bs.guard + 1;
          if (l == 1) { b.ro = 0; } else { b.ro = (int)off; off += b.rows; }
        }
      }
      while (bottom + 1 < a.L && bx[bottom + 1].rows > 0) ++bottom;
    }
    const T* rg0 = a.plist ? nullptr : (const T*)a.r;
    const T* rloc = a.plist ? (const T*)a.rloc + jo * a.vstride : nullptr;
    const WLevel& b0 = bx[0];
    const PLevel& lv0 = a.lv[0];
    T* t0 = vec + b0.to;
    const int guard0 = bsh[0].guard;
    const int AB0 = b0.A * b0.B;
    bool ok = true;
    if (a.L == 1) {
      // the level-0 box is the vertex level: exact solve
      const T* S = (const T*)lv0.S;
      BoxIter it;
      it.init(gl, b0.A, b0.B, NT);
      int ho[3] = {0, 0, 0};
      if (a.wmode == 2) hat_offsets<DIM>(j, a.n[0], a.n[1], a.wp, ho);
      for (int lex = gl; lex < b0.rows; lex += NT, it.next()) {
        const int G = ((b0.org[2] + it.k) * lv0.N[1] + (b0.org[1] + it.j)) * lv0.N[0] + (b0.org[0] + it.i);
        T rhs = rloc ? rloc[lex] : rg0[G];
        if (a.wp)
          rhs *= node_weight<DIM, T>(a.wmode, b0.org[0] + it.i, b0.org[1] + it.j, b0.org[2] + it.k, a.wp, ho[0], ho[1],
                                     ho[2], hat);
        if (GEN && b0.rows > 1) t0[lex] = rhs;
        else xslot[lex] = rhs / S[(long long)(a.NS / 2) * lv0.ntot + G];
        if (!(GEN && b0.rows > 1)) t0[lex] = T(0);
      }
      g.sync();
      if (GEN && b0.rows > 1) {   // several vertices in the box: the stored inverse
        const T* Bi = (const T*)a.binv + a.gsched[j].binv_off;
        for (int lex = gl; lex < b0.rows; lex += NT) {
          T acc = 0;
          for (int q = 0; q < b0.rows; ++q) acc += Bi[(long long)lex * b0.rows + q] * t0[q];
          xslot[lex] = acc;
        }
        g.sync();
        for (int lex = gl; lex < b0.rows; lex += NT) t0[lex] = T(0);
        g.sync();
      }
    } else {
      // ---- level 0 down: t0 <- rhs (zero guards), ILU, residual in place (x0 -> slot)
      for (int q = gl; q < b0.rows + 2 * guard0 + 1; q += NT) t0[q - guard0] = T(0);
      g.sync();
      {
        constexpr int U = kRowsInFlight;
        BoxIter it;
        it.init(gl, b0.A, b0.B, NT);
        int ho[3] = {0, 0, 0};
        if (a.wmode == 2) hat_offsets<DIM>(j, a.n[0], a.n[1], a.wp, ho);
        for (int l0 = gl; l0 < b0.rows; l0 += NT * U) {
          T v[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int lex = l0 + NT * u;
            const int G = ((b0.org[2] + it.k) * lv0.N[1] + (b0.org[1] + it.j)) * lv0.N[0] + (b0.org[0] + it.i);
            const T w = a.wp ? node_weight<DIM, T>(a.wmode, b0.org[0] + it.i, b0.org[1] + it.j, b0.org[2] + it.k, a.wp,
                                                   ho[0], ho[1], ho[2], hat)
                             : T(1);
            it.next();
            if (lex < b0.rows) v[u] = (rloc ? rloc[lex] : rg0[G]) * w;
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (l0 + NT * u < b0.rows) t0[l0 + NT * u] = v[u];
        }
      }
      g.sync();
      const FT* FL0 = F + a.facoff[j] * R;
      ok = ilu_solve<DIM, T, FT, NBUF, GEN, WG>(bsh[0], ip + meta[0], ip + meta[LOR_MAXLEV],
                                                FL0, t0, rg, zrec, g, okf);
      T* prev = vec + (b0.A + 1);                 // guarded plane buffers
      T* tmp = prev + AB0 + (b0.A + 1);
      if (ok) resid0_inplace<DIM, T, WG>(b0, lv0, rg0, rloc, t0, prev, tmp, xslot,
                                         a.wp, a.wmode, j, a.n[0], a.n[1], hat, g);
      if (ok && bottom > 0) {
        // ---- coarse levels
        if constexpr (GEN) {
          const XferG<T>* xg = (const XferG<T>*)a.xferg;
          restrict_level<DIM, T>(bx[0], bx[1], xg[geo[3]], xg[geo[4]], xg[geo[5]], t0, vec + bx[1].ro, g);
        } else {
          restrict_level<DIM, T>(bx[0], bx[1], xf[type[0]], xf[type[1]], xf[type[2]], t0, vec + bx[1].ro, g);
        }
        for (int q = gl; q < a.ovl_n; q += NT) vec[a.aux_n + q] = T(0);
        g.sync();
        for (int l = 1; l < bottom && ok; ++l) {
          const WLevel& b = bx[l];
          T* x = vec + b.xo; T* t = vec + b.to; T* r = vec + b.ro;
          const FT* FL = F + a.facoff[(long long)l * a.J + j] * R;
          for (int q = gl; q < b.rows; q += NT) t[q] = r[q];
          g.sync();
          ok = ilu_solve<DIM, T, FT, NBUF, GEN, WG>(bsh[l], ip + meta[l], ip + meta[LOR_MAXLEV + l],
                                                    FL, t, rg, zrec, g, okf);
          if (!ok) break;
          for (int q = gl; q < b.rows; q += NT) x[q] = t[q];
          g.sync();
          resid_level<DIM, T, WG>(b, a.lv[l], r, x, t, g);
          if constexpr (GEN) {
            const XferG<T>* xg = (const XferG<T>*)a.xferg + l * a.kmax1;
            restrict_level<DIM, T>(b, bx[l + 1], xg[geo[l * 6 + 3]], xg[geo[l * 6 + 4]], xg[geo[l * 6 + 5]], t,
                                   vec + bx[l + 1].ro, g);
          } else {
            restrict_level<DIM, T>(b, bx[l + 1], xf[l * 2 + type[0]], xf[l * 2 + type[1]], xf[l * 2 + type[2]], t,
                                   vec + bx[l + 1].ro, g);
          }
        }
        if (ok) {
          const int l = bottom;
          const WLevel& b = bx[l];
          const PLevel& lv = a.lv[l];
          T* x = vec + b.xo; T* t = vec + b.to; T* r = vec + b.ro;
          if (l == a.L - 1 && GEN && b.rows > 1) {
            // an enlarged patch keeps several vertices: x = A_box^{-1} r with the stored inverse
            const T* Bi = (const T*)a.binv + a.gsched[(long long)l * a.J + j].binv_off;
            for (int lex = gl; lex < b.rows; lex += NT) {
              T acc = 0;
              for (int q = 0; q < b.rows; ++q) acc += Bi[(long long)lex * b.rows + q] * r[q];
              x[lex] = acc;
            }
            g.sync();
          } else if (l == a.L - 1) {
            const T* S = (const T*)lv.S;
            BoxIter it;
            it.init(gl, b.A, b.B, NT);
            for (int lex = gl; lex < b.rows; lex += NT, it.next()) {
              const int G = ((b.org[2] + it.k) * lv.N[1] + (b.org[1] + it.j)) * lv.N[0] + (b.org[0] + it.i);
              x[lex] = r[lex] / S[(long long)(a.NS / 2) * lv.ntot + G];
            }
            g.sync();
          } else {
            const FT* FL = F + a.facoff[(long long)l * a.J + j] * R;
            for (int q = gl; q < b.rows; q += NT) t[q] = r[q];
            g.sync();
            ok = ilu_solve<DIM, T, FT, NBUF, GEN, WG>(bsh[l], ip + meta[l], ip + meta[LOR_MAXLEV + l],
                                                      FL, t, rg, zrec, g, okf);
            if (ok) {
              for (int q = gl; q < b.rows; q += NT) x[q] = t[q];
              g.sync();
              resid_level<DIM, T, WG>(b, lv, r, x, t, g);
              ok = ilu_solve<DIM, T, FT, NBUF, GEN, WG>(bsh[l], ip + meta[l], ip + meta[LOR_MAXLEV + l],
                                                        FL, t, rg, zrec, g, okf);
            }
            if (ok) {
              for (int q = gl; q < b.rows; q += NT) x[q] += t[q];
              g.sync();
            }
          }
        }
        for (int l = bottom - 1; l >= 1 && ok; --l) {
          const WLevel& b = bx[l];
          T* x = vec + b.xo; T* t = vec + b.to; T* r = vec + b.ro;
          const T* xc = vec + bx[l + 1].xo;
          const FT* FL = F + a.facoff[(long long)l * a.J + j] * R;
          BoxIter it;
          it.init(gl, b.A, b.B, NT);
          for (int lex = gl; lex < b.rows; lex += NT, it.next()) {
            if constexpr (GEN) {
              const XferG<T>* xg = (const XferG<T>*)a.xferg + l * a.kmax1;
              x[lex] += prolong_row<DIM, T>(bx[l + 1], xg[geo[l * 6 + 3]], xg[geo[l * 6 + 4]], xg[geo[l * 6 + 5]], xc,
                                            it.i, it.j, it.k);
            } else {
              x[lex] += prolong_row<DIM, T>(bx[l + 1], xf[l * 2 + type[0]], xf[l * 2 + type[1]], xf[l * 2 + type[2]],
                                            xc, it.i, it.j, it.k);
            }
          }
          g.sync();
          resid_level<DIM, T, WG>(b, a.lv[l], r, x, t, g);
          ok = ilu_solve<DIM, T, FT, NBUF, GEN, WG>(bsh[l], ip + meta[l], ip + meta[LOR_MAXLEV + l],
                                                    FL, t, rg, zrec, g, okf);
          if (!ok) break;
          for (int q = gl; q < b.rows; q += NT) x[q] += t[q];
          g.sync();
        }
        if (ok) {
          // ---- level 0 up: x0 += P x1 in the slot, t0 <- x0, residual in place
          const T* x1 = vec + bx[1].xo;
          constexpr int U = kRowsInFlight;
          BoxIter it;
          it.init(gl, b0.A, b0.B, NT);
          for (int l0 = gl; l0 < b0.rows; l0 += NT * U) {
            T xv[U];
            int iu[U], ju[U], ku[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              iu[u] = it.i; ju[u] = it.j; ku[u] = it.k;
              it.next();
              if (l0 + NT * u < b0.rows) xv[u] = xslot[l0 + NT * u];
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
              if (l0 + NT * u < b0.rows)
                if constexpr (GEN) {
                  const XferG<T>* xg = (const XferG<T>*)a.xferg;
                  xslot[l0 + NT * u] = xv[u] + prolong_row<DIM, T>(bx[1], xg[geo[3]], xg[geo[4]], xg[geo[5]], x1,
                                                                   iu[u], ju[u], ku[u]);
                } else {
                  xslot[l0 + NT * u] = xv[u] + prolong_row<DIM, T>(bx[1], xf[type[0]], xf[type[1]], xf[type[2]], x1,
                                                                   iu[u], ju[u], ku[u]);
                }
          }
          g.sync();
          // t0 <- x0 (x1 lived over t0's space; every thread is done with it now)
          for (int q = gl; q < guard0; q += NT) { t0[q - guard0] = T(0); t0[b0.rows + q] = T(0); }
          if (gl == 0) t0[b0.rows + guard0] = T(0);
          for (int l0 = gl; l0 < b0.rows; l0 += NT * U) {
            T xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
              if (l0 + NT * u < b0.rows) xv[u] = xslot[l0 + NT * u];
#pragma unroll
            for (int u = 0; u < U; ++u)
              if (l0 + NT * u < b0.rows) t0[l0 + NT * u] = xv[u];
          }
          g.sync();
          resid0_inplace<DIM, T, WG>(b0, lv0, rg0, rloc, t0, prev, tmp, nullptr,
                                     a.wp, a.wmode, j, a.n[0], a.n[1], hat, g);
        }
      }
      if (ok && !a.skip_post0)
        ok = ilu_solve<DIM, T, FT, NBUF, GEN, WG>(bsh[0], ip + meta[0], ip + meta[LOR_MAXLEV],
                                                  FL0, t0, rg, zrec, g, okf);
    }
    if (!ok) {
      // a bulk copy did not arrive in time: report, drain what is still in flight, leave
      if (gl == 0) {
        atomicOr(a.status, 4);
        for (int s = 0; s < NBUF; ++s)
          if (rg.inflight & (1u << s)) mbar_wait(rg.bar + s, (rg.phase >> s) & 1u);
      }
      return;
    }
    // ---- x_j = x0 + t0: patch-local output, or scatter-add R_j^T x_j
    if (a.plist) {
      T* dst = (T*)a.xloc + jo * a.vstride;
      for (int lex = gl; lex < b0.rows; lex += NT) dst[lex] = xslot[lex] + (a.skip_post0 ? T(0) : t0[lex]);
      g.sync();   // the next patch overwrites t0 and the slot
      continue;
    }
    // the weighted R_j^T x_j goes to the patch's own output slice (lexicographic
    // box order); k_patch_sum adds the slices node by node in a fixed order
    T* zj = (T*)a.zp + (long long)j * a.zstride;
    {
      constexpr int U = kRowsInFlight;
      BoxIter it;
      it.init(gl, b0.A, b0.B, NT);
      int ho[3] = {0, 0, 0};
      if (a.wmode == 2) hat_offsets<DIM>(j, a.n[0], a.n[1], a.wp, ho);
      for (int l0 = gl; l0 < b0.rows; l0 += NT * U) {
        T xv[U], w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          w[u] = a.wp && l0 + NT * u < b0.rows
                     ? node_weight<DIM, T>(a.wmode, b0.org[0] + it.i, b0.org[1] + it.j, b0.org[2] + it.k, a.wp, ho[0],
                                           ho[1], ho[2], hat)
                     : T(1);
          it.next();
          if (l0 + NT * u < b0.rows) xv[u] = xslot[l0 + NT * u];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int lex = l0 + NT * u;
          if (lex < b0.rows) {
            const T xj = a.skip_post0 ? xv[u] : xv[u] + t0[lex];
            zj[lex] = w[u] * xj;
            if (a.tout && sh == 0 && !a.skip_post0) t0[lex] = xj;
          }
        }
      }
    }
    g.sync();
    if (a.tout && sh == 0) {   // residual left on an interior patch, for the learned correction
      T* prev = vec + (b0.A + 1);
      T* tmp = prev + AB0 + (b0.A + 1);
      // (without the post-smoothing t0 already holds r - A x0)
      if (!a.skip_post0)
        resid0_inplace<DIM, T, WG>(b0, lv0, rg0, nullptr, t0, prev, tmp, nullptr,
                                   a.wp, a.wmode, j, a.n[0], a.n[1], hat, g);
      T* dst = (T*)a.tout + jo * a.vstride;
      for (int lex = gl; lex < b0.rows; lex += NT) dst[lex] = t0[lex];
      g.sync();
    }
  }
}

// z[node] = sum over the (at most 2^d) vertex patches containing the interior node
// of their output slices, in a fixed order (vertex index ascending along x, then
// y, then z); boundary nodes get 0.  Patch j covers, along each axis, the nodes
// org + [0, len) of its box: org = (v-1) p + 1 and len = 2p - 1 for an interior
// vertex v, org = 1, len = p - 1 at v = 0 and org = (n-1) p + 1, len = p - 1 at v = n.
// z[node] = sum of the node's entries in the patch output slices, listed per node in
// patch order (enlarged patches, whose overlap has no closed form); 0 if none.
template <typename T>
__global__ void k_patch_gather(long long nt, const long long* __restrict__ ptr, const long long* __restrict__ idx,
                               const T* __restrict__ zp, const double* __restrict__ conv, T* __restrict__ z) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nt) return;
  if (conv && *conv != 0.0) { z[gid] = T(0); return; }
  T s = 0;
  for (long long q = ptr[gid]; q < ptr[gid + 1]; ++q) s += zp[idx[q]];
  z[gid] = s;
}

template <typename T>
__global__ void k_patch_sum(int dim, int p, int nx, int ny, int nz, const T* __restrict__ zp, long long zstride,
                            const double* __restrict__ conv, T* __restrict__ z) {
  const int Nx = nx * p + 1, Ny = ny * p + 1, Nz = dim == 3 ? nz * p + 1 : 1;
  const long long nt = (long long)Nx * Ny * Nz;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nt) return;
  if (conv && *conv != 0.0) { z[gid] = T(0); return; }   // converged batched solve: the patch kernel did nothing
  const int I[3] = {(int)(gid % Nx), (int)((gid / Nx) % Ny), (int)(gid / ((long long)Nx * Ny))};
  const int n[3] = {nx, ny, nz};
  const int N[3] = {Nx, Ny, Nz};
  for (int a = 0; a < dim; ++a)
    if (I[a] == 0 || I[a] == N[a] - 1) { z[gid] = T(0); return; }
  // per axis: candidate vertices, the node's local index in each, and the box length
  int cv[3][2], cl[3][2], cn[3][2], cnt[3] = {1, 1, 1};
  for (int a = 0; a < 3; ++a) { cv[a][0] = 0; cl[a][0] = 0; cn[a][0] = 1; }
  for (int a = 0; a < dim; ++a) {
    const int q = I[a] / p, rem = I[a] - q * p;
    const int v0 = rem == 0 ? q : q, v1 = q + 1;
    cnt[a] = rem == 0 ? 1 : 2;
    const int vs[2] = {v0, v1};
    for (int s = 0; s < cnt[a]; ++s) {
      const int v = vs[s];
      const int org = (v > 0 ? (v - 1) * p : 0) + 1;
      cv[a][s] = v;
      cl[a][s] = I[a] - org;
      cn[a][s] = (v == 0 || v == n[a]) ? p - 1 : 2 * p - 1;
    }
  }
  T s = T(0);
  for (int c2 = 0; c2 < cnt[2]; ++c2)
    for (int c1 = 0; c1 < cnt[1]; ++c1)
      for (int c0 = 0; c0 < cnt[0]; ++c0) {
        const long long jp = ((long long)cv[2][c2] * (ny + 1) + cv[1][c1]) * (nx + 1) + cv[0][c0];
        const long long lex = ((long long)cl[2][c2] * cn[1][c1] + cl[1][c1]) * cn[0][c0] + cl[0][c0];
        s += zp[jp * zstride + lex];
      }
  z[gid] = s;
}

// ------------------------------------------------------------------ coarse space
// rc[V] = sum_F P0[F][V] r[F] for interior vertices V (P0: Q1 interpolation at GLL nodes)
// One separable pass of P_0^T = (R_z x R_y x R_x) r: contracts axis `ax` of a
// d0 x d1 x d2 array (x fastest) to the vertex grid along that axis (Vn vertices):
//   out[.., v, ..] = sum_{a < 2p-1} w[a] in[.., (v-1)p+1+a, ..]  for interior v, 0 on the boundary,
// where w are the 1D values of the vertex hat function at the GLL-refined nodes of
// the two elements around the vertex.
template <typename T>
__global__ void k_p0t_pass(const T* __restrict__ in, T* __restrict__ out, int d0, int d1, int d2, int ax, int p,
                           int Vn, const T* __restrict__ w, const double* __restrict__ conv) {
  if (conv && *conv != 0.0) return;   // converged batched solve
  const int o0 = ax == 0 ? Vn : d0, o1 = ax == 1 ? Vn : d1, o2 = ax == 2 ? Vn : d2;
  const long long no = (long long)o0 * o1 * o2;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= no) return;
  const int i = (int)(gid % o0), j = (int)((gid / o0) % o1), k = (int)(gid / ((long long)o0 * o1));
  const int v = ax == 0 ? i : (ax == 1 ? j : k);
  if (v == 0 || v == Vn - 1) { out[gid] = T(0); return; }
  const long long st = ax == 0 ? 1 : (ax == 1 ? (long long)d0 : (long long)d0 * d1);
  const long long base = ((long long)(ax == 2 ? (v - 1) * p + 1 : k) * d1 + (ax == 1 ? (v - 1) * p + 1 : j)) * d0 +
                         (ax == 0 ? (v - 1) * p + 1 : i);
  T s = 0;
  for (int a = 0; a < 2 * p - 1; ++a) s += w[a] * in[base + a * st];
  out[gid] = s;
}

// z[F] += sum_V P0[F][V] e[V] for interior fine nodes (weights in the path precision)
template <typename T>
__global__ void k_coarse_prolong0(int dim, int p, int nx, int ny, int nz, const T* __restrict__ gllx,
                                  const T* __restrict__ e, T sgn, T* __restrict__ z, const double* __restrict__ conv) {
  if (conv && *conv != 0.0) return;   // converged batched solve: z stays 0
  const int Nx = nx * p + 1, Ny = ny * p + 1, Nz = dim == 3 ? nz * p + 1 : 1;
  const long long nt = (long long)Nx * Ny * Nz;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nt) return;
  const int I = (int)(gid % Nx), Jn = (int)((gid / Nx) % Ny), K = (int)(gid / ((long long)Nx * Ny));
  if (I == 0 || I == Nx - 1 || Jn == 0 || Jn == Ny - 1 || (dim == 3 && (K == 0 || K == Nz - 1))) return;
  const int ex = min(I / p, nx - 1), ey = min(Jn / p, ny - 1), ez = dim == 3 ? min(K / p, nz - 1) : 0;
  const T xi[3] = {gllx[I - ex * p], gllx[Jn - ey * p], dim == 3 ? gllx[K - ez * p] : T(0)};
  const int Vx = nx + 1, Vy = ny + 1;
  T s = 0;
  const int nc = 1 << dim;
  for (int cc = 0; cc < nc; ++cc) {
    const int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
    T w = (bx ? xi[0] : T(1) - xi[0]) * (by ? xi[1] : T(1) - xi[1]);
    if (dim == 3) w *= bz ? xi[2] : T(1) - xi[2];
    s += w * e[((long long)(ez + bz) * Vy + (ey + by)) * Vx + (ex + bx)];
  }
  z[gid] += sgn * s;
}

// y = b - K_h x (or y = K_h x when b is null) on the interior level-0 nodes, K_h the
// LOR stencil with the Dirichlet rows and columns dropped; y = 0 on the boundary.
template <typename T>
__global__ void k_kh_apply(int dim, int Nx, int Ny, int Nz, const T* __restrict__ S, const T* __restrict__ x,
                           const T* __restrict__ b, T* __restrict__ y) {
  const long long nt = (long long)Nx * Ny * Nz;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nt) return;
  const int I = (int)(gid % Nx), Jn = (int)((gid / Nx) % Ny), K = (int)(gid / ((long long)Nx * Ny));
  if (I == 0 || I == Nx - 1 || Jn == 0 || Jn == Ny - 1 || (dim == 3 && (K == 0 || K == Nz - 1))) {
    y[gid] = T(0);
    return;
  }
  const int NS = dim == 3 ? 27 : 9;
  T s = 0;
  for (int o = 0; o < NS; ++o) {
    const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = dim == 3 ? o / 9 - 1 : 0;
    const int I2 = I + dx, J2 = Jn + dy, K2 = K + dz;
    if (I2 == 0 || I2 == Nx - 1 || J2 == 0 || J2 == Ny - 1 || (dim == 3 && (K2 == 0 || K2 == Nz - 1))) continue;
    s += S[(long long)o * nt + gid] * x[gid + ((long long)dz * Ny + dy) * Nx + dx];
  }
  y[gid] = b ? b[gid] - s : s;
}

template <typename T>
__global__ void k_add2(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ z, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = a[i] + b[i];
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
  static const double* p0w(lor_ctx* c) { return c->d_p0w64; }
  static double* p0t(lor_ctx* c, int k) { return c->d_p0t64[k]; }
};
template <> struct Sel<float> {
  static float* cw(lor_ctx* c, int l, int k) { return c->d_cw32[l][k]; }
  static const float* cS(lor_ctx* c, int l) { return c->d_cS32[l]; }
  static const float* cD(lor_ctx* c, int l) { return c->d_cDinv32[l]; }
  static const float* inv(lor_ctx* c) { return c->d_cInv32; }
  static const void* S(lor_ctx* c, int l) { return c->d_S32[l]; }
  static const float* p0w(lor_ctx* c) { return c->d_p0w32; }
  static float* p0t(lor_ctx* c, int k) { return c->d_p0t32[k]; }
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

// Patch groups per CTA (one CTA per SM when shared memory allows): up to 12
// one-warp groups, or up to 8 two-warp groups (512 threads, at most 128 registers
// each).  Two warps per patch are used for 3D boxes in FP32 when shared memory
// holds at most 8 patches per SM anyway (large boxes, wide wavefronts), so the
// second warp costs no patch in flight; FP64 (more registers), 2D and smaller
// boxes run one warp per patch.  Each group owns a named barrier 1 + index
// (ids 1..15).
const int kMaxGroups1 = 12, kMaxGroups2 = 8;
static_assert(kMaxGroups1 <= 15 && kMaxGroups2 <= 15, "named barrier ids 1..15");

template <typename FT>
constexpr int ring_depth() { return 2; }

// Per-group shared-memory layout of the patch kernel (sizes for the largest,
// interior, box shape; other shapes fit inside).
struct WarpLayout {
  int slot_bytes, tab_ints, aux_n, ovl_n, warp_bytes, xf_bytes;
  long long x0_stride;
};

template <typename T, typename FT>
WarpLayout warp_layout(const lor_ctx* c) {
  WarpLayout w;
  const int es = elem_class<FT>();
  w.slot_bytes = c->maxchunk[es] * lor_rec(c->dim) * (int)sizeof(FT);
  int tab = 0;
  for (int s = 0; s < 8; ++s) {
    int t = 0;
    for (int l = 0; l < c->L; ++l) t += c->shapes[l * 8 + s].nfront + 1 + c->shapes[l * 8 + s].nchunk[es] + 1;
    tab = std::max(tab, t);
  }
  if (c->gen) {   // ordered records and per-patch schedules
    w.slot_bytes = std::max(c->gen_maxchunk[es], 1) * lor_rec_gen(c->dim) * (int)sizeof(FT);
    tab = std::max(tab, c->gen_tab_ints);
  }
  w.tab_ints = (tab + 3) / 4 * 4;
  const BoxShape& b0 = c->shapes[0];
  const int A = b0.dims[0], B = b0.dims[1];
  w.aux_n = 2 * A * B + 2 * (A + 1);
  if (c->L > 1) w.aux_n = std::max(w.aux_n, c->shapes[8].rows);
  w.aux_n = (w.aux_n + 3) / 4 * 4;
  long long ovl = 0;
  for (int l = 1; l < c->L; ++l) {
    const BoxShape& bs = c->shapes[l * 8];
    ovl += 2LL * (bs.rows + 2 * bs.guard + 1) + (l >= 2 ? bs.rows : 0);
  }
  w.ovl_n = (int)std::max<long long>(b0.rows + 2LL * b0.guard + 1, ovl);
  w.x0_stride = (b0.rows + 31) / 32 * 32;
  if (c->gen) {   // per-patch boxes: the largest of every buffer
    w.aux_n = std::max(2 * c->gen_AB0 + 2 * (c->gen_A0 + 1), c->L > 1 ? c->gen_rows1 : 0);
    w.aux_n = std::max(w.aux_n, 4);
    w.aux_n = (w.aux_n + 3) / 4 * 4;
    w.ovl_n = (int)std::max<long long>(c->gen_ovl, 4);
    w.x0_stride = (std::max(c->gen_rows0, 1) + 31) / 32 * 32;
  }
  const size_t bytes = (size_t)warp_ring_offset(c->gen) + (size_t)ring_depth<FT>() * w.slot_bytes +
                       4 * (size_t)w.tab_ints + (size_t)(w.aux_n + w.ovl_n) * sizeof(T);
  w.warp_bytes = (int)((bytes + 127) / 128 * 128);
  w.xf_bytes = (int)((2 * (c->L > 1 ? c->L - 1 : 1) * sizeof(Xfer1D<T>) + 127) / 128 * 128);
  return w;
}

template <typename T, typename FT>
void fill_patch_args(lor_ctx* c, PatchArgs& a, const FT* F) {
  a.dim = c->dim; a.NS = c->NS; a.L = c->L; a.J = c->J;
  for (int t = 0; t < 3; ++t) a.n[t] = c->n[t];
  for (int l = 0; l < c->L; ++l) {
    PLevel& lv = a.lv[l];
    lv.S = Sel<T>::S(c, l);
    lv.Sa = sizeof(T) == 8 ? (const void*)c->d_SA64[l] : (const void*)c->d_SA32[l];
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
  a.fpad = c->d_fpad; a.chunk = c->d_chunk;
  a.gsched = nullptr;
  a.xferg = nullptr;
  a.kmax1 = 0;
  a.binv = nullptr;
  if (c->gen) {
    a.fpad = c->d_gfpad; a.chunk = c->d_gchunk; a.gsched = c->d_gsched;
    a.xferg = sizeof(T) == 8 ? c->d_xferg64 : c->d_xferg32;
    a.kmax1 = c->span_kmax + 1;
    a.binv = sizeof(T) == 8 ? (const void*)c->d_binv64 : (const void*)c->d_binv32;
  }
  a.facoff = c->d_facoff;
  a.F = F; a.r = nullptr;
  a.zp = c->d_zp;
  a.status = c->d_status;
  a.porder = c->d_porder;
  a.conv = c->conv_flag;
  a.plist = nullptr; a.nlist = 0; a.rloc = nullptr; a.xloc = nullptr; a.vstride = 0; a.tout = nullptr;
  a.skip_post0 = 0;
  a.wp = c->opt.weighting ? c->p : 0;
  a.wmode = c->opt.weighting;
  a.hat = Sel<T>::p0w(c);
  const WarpLayout w = warp_layout<T, FT>(c);
  a.slot_bytes = w.slot_bytes;
  a.tab_ints = w.tab_ints;
  a.xf_bytes = w.xf_bytes;
  a.warp_bytes = w.warp_bytes;
  a.aux_n = w.aux_n;
  a.ovl_n = w.ovl_n;
  a.xs = c->d_xs;
  a.x0_stride = w.x0_stride;
  a.zstride = w.x0_stride;
}

// Launch shape of the patch kernel: warps per CTA (shared memory) and resident
// CTAs per SM; returns false if not even one warp fits.
// The kernel instantiation for a context; two-warp groups exist in 3D only.
template <typename T, typename FT, int WG>
auto patch_kernel(const lor_ctx* c) {
  constexpr int NB = ring_depth<FT>();
  if constexpr (WG == 2)
    return c->gen ? k_patch_warp<3, T, FT, NB, true, 2> : k_patch_warp<3, T, FT, NB, false, 2>;
  else
    return c->dim == 3 ? (c->gen ? k_patch_warp<3, T, FT, NB, true, 1> : k_patch_warp<3, T, FT, NB, false, 1>)
                       : (c->gen ? k_patch_warp<2, T, FT, NB, true, 1> : k_patch_warp<2, T, FT, NB, false, 1>);
}

template <typename T, typename FT>
bool patch_launch_shape(const lor_ctx* c, int* ng, int* wg, int* grid, size_t* smem) {
  const WarpLayout w = warp_layout<T, FT>(c);
  int dev = 0, nsm = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int fit = (maxsm - w.xf_bytes) / w.warp_bytes;
  if (fit < 1) return false;
  *wg = sizeof(T) == 4 && c->dim == 3 && fit <= kMaxGroups2 ? 2 : 1;
  *ng = std::min(*wg == 2 ? kMaxGroups2 : kMaxGroups1, fit);
  *smem = (size_t)w.xf_bytes + (size_t)*ng * w.warp_bytes;
  int per_sm = 0;
  if constexpr (sizeof(T) == 4) {
    if (*wg == 2) {
      auto kern = patch_kernel<T, FT, 2>(c);
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64 * *ng, *smem);
    }
  }
  if (*wg == 1) {
    auto kern = patch_kernel<T, FT, 1>(c);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * *ng, *smem);
  }
  *grid = std::max(per_sm, 1) * nsm;
  return true;
}

template <typename T, typename FT>
lor_status launch_patch_kernel(lor_ctx* c, PatchArgs& a) {
  const long long work = a.plist ? a.nlist : c->J;
  if (work <= 0) return LOR_OK;
  int ng = 0, wg = 1, grid = 0;
  size_t smem = 0;
  if (!patch_launch_shape<T, FT>(c, &ng, &wg, &grid, &smem)) return lor_fail(c, LOR_EINVAL, "patch does not fit");
  // persistent groups: as many as fit, each walking patches g, g + (all groups), ...
  grid = (int)std::min<long long>(grid, (work + ng - 1) / ng);
  if ((long long)grid * ng * a.x0_stride * (long long)sizeof(T) > c->xs_bytes)
    return lor_fail(c, LOR_ESTATE, "patch iterate slots too small");
  if constexpr (sizeof(T) == 4) {
    if (wg == 2) patch_kernel<T, FT, 2>(c)<<<grid, 64 * ng, smem, c->stream>>>(a);
  }
  if (wg == 1) patch_kernel<T, FT, 1>(c)<<<grid, 32 * ng, smem, c->stream>>>(a);
  ++c->launches;
  return lor_cuda_check(c, cudaGetLastError(), "patch vcycle");
}

// z = sum_j R_j^T V_j(R_j r) (plus the learned correction when it is on)
template <typename T, typename FT>
lor_status patch_part(lor_ctx* c, const T* r, T* z, const FT* F) {
  const long long nvec = c->lev[0].ntot;
  PatchArgs a;
  fill_patch_args<T, FT>(c, a, F);
  a.r = r;
  if (c->learned_on && sizeof(T) == 4) {
    a.tout = c->learned_tout;
    a.vstride = c->shapes[0].rows;
    a.skip_post0 = c->learned_replace ? 1 : 0;
  }
  const int pk = sizeof(T) == 8 ? 0 : 1;
  lor_prof_begin(c, pk);
  if (launch_patch_kernel<T, FT>(c, a)) return LOR_ECUDA;
  lor_prof_end(c, pk);
  // z = sum_j R_j^T x_j, node by node in a fixed order
  if (c->d_gather_ptr)
    k_patch_gather<T><<<(unsigned)lor_ceil_div(nvec, 256), 256, 0, c->stream>>>(
        nvec, c->d_gather_ptr, c->d_gather_idx, (const T*)c->d_zp, c->conv_flag, z);
  else
    k_patch_sum<T><<<(unsigned)lor_ceil_div(nvec, 256), 256, 0, c->stream>>>(
        c->dim, c->p, c->n[0], c->n[1], c->n[2], (const T*)c->d_zp, a.zstride, c->conv_flag, z);
  ++c->launches;
  if (c->learned_on && sizeof(T) == 4) {
    if (lor_learned_apply(c, (float*)z)) return LOR_ECUDA;
  }
  return LOR_OK;
}

// z += sgn P_0 R_0 P_0^T r (the coarse space of Eq. (as))
template <typename T>
lor_status coarse_part(lor_ctx* c, const T* r, T* z, T sgn) {
  const long long nvec = c->lev[0].ntot;
  const int pk = sizeof(T) == 8 ? 0 : 1;
  lor_prof_begin(c, pk + 4);
  // coarse space: rc = P_0^T r by separable passes (x, y[, z])
  {
    const LevelGrid& g0 = c->lev[0];
    const int p = c->p, V0 = c->n[0] + 1, V1 = c->n[1] + 1, V2 = c->dim == 3 ? c->n[2] + 1 : 1;
    const T* w = Sel<T>::p0w(c) + p + 1;
    T* t1 = Sel<T>::p0t(c, 0);
    T* t2 = Sel<T>::p0t(c, 1);
    T* rc = Sel<T>::cw(c, 0, 0);
    long long m = (long long)g0.N[2] * g0.N[1] * V0;
    k_p0t_pass<T><<<(unsigned)lor_ceil_div(m, 256), 256, 0, c->stream>>>(r, t1, g0.N[0], g0.N[1], g0.N[2], 0, p, V0, w, c->conv_flag);
    m = (long long)g0.N[2] * V1 * V0;
    k_p0t_pass<T><<<(unsigned)lor_ceil_div(m, 256), 256, 0, c->stream>>>(t1, c->dim == 3 ? t2 : rc, V0, g0.N[1], g0.N[2], 1,
                                                                          p, V1, w, c->conv_flag);
    c->launches += 2;
    if (c->dim == 3) {
      m = (long long)V2 * V1 * V0;
      k_p0t_pass<T><<<(unsigned)lor_ceil_div(m, 256), 256, 0, c->stream>>>(t2, rc, V0, V1, g0.N[2], 2, p, V2, w, c->conv_flag);
      ++c->launches;
    }
  }
  T* ec = coarse_vcycle<T>(c, 0);
  k_coarse_prolong0<T><<<(unsigned)lor_ceil_div(nvec, 256), 256, 0, c->stream>>>(c->dim, c->p, c->n[0], c->n[1],
                                                                                   c->n[2], Sel<T>::p0w(c), ec, sgn, z,
                                                                                   c->conv_flag);
  ++c->launches;
  lor_prof_end(c, pk + 4);
  return lor_cuda_check(c, cudaGetLastError(), "coarse space");
}

// B r with the coarse space additive (Eq. (as)), or hybrid: the coarse correction
// multiplicative and the patches additive among themselves, in the symmetric form
//   B_hyb = B_0 + (I - B_0 K_h) B_loc (I - K_h B_0),
// B_0 = P_0 R_0 P_0^T, B_loc the patch sum, K_h the LOR matrix on the interior nodes
// (the variant Section 4.1 leaves to future work).  Hybrid steps: z0 = B_0 r,
// t = r - K_h z0, z1 = B_loc t, z = z0 + z1 - B_0 (K_h z1).
template <typename T, typename FT>
lor_status launch_apply_P(lor_ctx* c, const T* r, T* z, const FT* F) {
  if (c->schwarz == 2) return lor_single_apply<T>(c, r, z);
  if (c->schwarz == 0) {
    if (patch_part<T, FT>(c, r, z, F)) return LOR_ECUDA;
    return coarse_part<T>(c, r, z, T(1));
  }
  const LevelGrid& g0 = c->lev[0];
  const long long nvec = g0.ntot;
  if (!c->d_hyb) return lor_fail(c, LOR_ESTATE, "hybrid Schwarz workspace missing");
  T* z0 = (T*)c->d_hyb;
  T* t = z0 + nvec;
  T* z1 = t + nvec;
  const T* S = (const T*)Sel<T>::S(c, 0);
  const unsigned nb = (unsigned)lor_ceil_div(nvec, 256);
  const int Nz = c->dim == 3 ? g0.N[2] : 1;
  cudaMemsetAsync(z0, 0, nvec * sizeof(T), c->stream);
  if (coarse_part<T>(c, r, z0, T(1))) return LOR_ECUDA;
  k_kh_apply<T><<<nb, 256, 0, c->stream>>>(c->dim, g0.N[0], g0.N[1], Nz, S, z0, r, t);
  ++c->launches;
  if (patch_part<T, FT>(c, t, z1, F)) return LOR_ECUDA;
  k_kh_apply<T><<<nb, 256, 0, c->stream>>>(c->dim, g0.N[0], g0.N[1], Nz, S, z1, nullptr, t);
  k_add2<T><<<nb, 256, 0, c->stream>>>(z0, z1, z, nvec);
  c->launches += 2;
  return coarse_part<T>(c, t, z, T(-1));
}

// Self-test of the bounded waits: one warp waits on an mbarrier at which nothing
// arrives; the wait gives up after `polls` polls and the kernel reports it in the
// context status word (bit 4, the same bit as a bulk-copy timeout of the patch
// kernel), then invalidates the barrier and returns.
__global__ void k_wait_selftest(int polls, int* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0u, polls)) atomicOr(status, 4);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
  }
}

}  // namespace

template <typename T>
T* lor_coarse_rhs(lor_ctx* c) {
  return Sel<T>::cw(c, 0, 0);
}

template <typename T>
T* lor_coarse_solve(lor_ctx* c) {
  return coarse_vcycle<T>(c, 0);
}

template double* lor_coarse_rhs<double>(lor_ctx*);
template float* lor_coarse_rhs<float>(lor_ctx*);
template double* lor_coarse_solve<double>(lor_ctx*);
template float* lor_coarse_solve<float>(lor_ctx*);

lor_status lor_launch_wait_selftest(lor_ctx* c, int polls) {
  k_wait_selftest<<<1, 32, 0, c->stream>>>(polls, c->d_status);
  ++c->launches;
  return lor_cuda_check(c, cudaGetLastError(), "wait self-test");
}

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
    a.wp = 0;   // patch-local problems: unit weights
    a.skip_post0 = c->learned_replace ? 1 : 0;
    return launch_patch_kernel<float, __nv_bfloat16>(c, a);
  }
  fill_patch_args<float, float>(c, a, c->d_F32);
  a.plist = plist; a.nlist = nlist; a.rloc = rloc; a.xloc = xloc; a.vstride = vstride;
  a.wp = 0;   // patch-local problems: unit weights
  a.skip_post0 = c->learned_replace ? 1 : 0;
  return launch_patch_kernel<float, float>(c, a);
}

// Checks that the patch kernel fits (every precision this context can run) and
// allocates the per-group level-0 iterate slots for the largest launch and the
// per-patch output slices (J slices of x0_stride values, float64-sized).
lor_status lor_patch_prepare(lor_ctx* c) {
  long long need = 0;
  int ng = 0, wg = 1, grid = 0;
  size_t smem = 0;
  if (!patch_launch_shape<double, double>(c, &ng, &wg, &grid, &smem))
    return lor_fail(c, LOR_EINVAL, "patch does not fit in shared memory");
  need = std::max(need, (long long)grid * ng * warp_layout<double, double>(c).x0_stride * 8);
  c->smem_patch64 = (int)smem;
  const bool bf = c->d_F16 != nullptr;
  const bool ok32 = bf ? patch_launch_shape<float, __nv_bfloat16>(c, &ng, &wg, &grid, &smem)
                       : patch_launch_shape<float, float>(c, &ng, &wg, &grid, &smem);
  if (!ok32) return lor_fail(c, LOR_EINVAL, "patch does not fit in shared memory");
  need = std::max(need, (long long)grid * ng * warp_layout<float, float>(c).x0_stride * 4);
  c->smem_patch32 = (int)smem;
  c->xs_bytes = need;
  c->d_xs = lor_alloc(c, (size_t)std::max<long long>(need, 8));
  if (!c->d_xs) return lor_fail(c, LOR_ENOMEM, "alloc patch iterate slots");
  const long long zbytes = (long long)c->J * warp_layout<double, double>(c).x0_stride * 8;
  c->d_zp = lor_alloc(c, (size_t)std::max<long long>(zbytes, 8));
  if (!c->d_zp) return lor_fail(c, LOR_ENOMEM, "alloc patch outputs");
  return LOR_OK;
}
