// Learned per-patch correction of the LOR V-cycle (the learned form).
//
// On every interior vertex patch, after the V(1,1) cycle (Section 3.3) leaves a
// level-0 residual t, a 3-layer convolutional network adds the correction
//   c = rho * s * N([s * t / rho, log(diag / mean diag)]),  s = diag^(-1/2),
//   N = conv3^3(2->16) - ReLU - conv3^3(16->16) - ReLU - conv3^3(16->1),
// zero padding at the patch boundary, rho = rms(s * t).  Weights are stored in
// bf16; every convolution, forward and backward, runs on the BF16 tensor cores
// with FP32 accumulation, on bf16 activations and gradients (channel-last rows of
// 16 channels).  Training minimises the normalised
// energy of the error left after the correction, on pairs made by the plain
// V-cycle from random errors e: delta = e - V(A e), t = A delta,
//   L = (delta - c)^T A (delta - c) / (delta^T A delta),
// with hand-written backward kernels and Adam.  Since N is nonlinear the outer
// Krylov method switches to flexible CG when the correction is on.
// Kernels work on batches of S interior patches; a patch box holds V = (2p-1)^3
// values in lexicographic order (x fastest).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lor_internal.h"

namespace {

const int CH = 16;
const int NW1 = CH * 2 * 27, NW2 = CH * CH * 27, NW3 = CH * 27;
const int OFF_W1 = 0, OFF_B1 = NW1, OFF_W2 = OFF_B1 + CH, OFF_B2 = OFF_W2 + NW2, OFF_W3 = OFF_B2 + CH,
          OFF_B3 = OFF_W3 + NW3, NPARAM = OFF_B3 + 1;

struct PBox {
  int A, B, C, V;
  int n[3];        // elements per direction (patch vertex from id)
  int m;           // level-0 intervals per element (p)
  int N[3];        // level-0 grid
  long long ntot;
};

__device__ __forceinline__ long long box_global(const PBox& b, int j, int lex) {
  const int vx = j % (b.n[0] + 1), vy = (j / (b.n[0] + 1)) % (b.n[1] + 1), vz = j / ((b.n[0] + 1) * (b.n[1] + 1));
  const int i = lex % b.A, jj = (lex / b.A) % b.B, k = lex / (b.A * b.B);
  const int ox = (vx - 1) * b.m + 1, oy = (vy - 1) * b.m + 1, oz = (vz - 1) * b.m + 1;   // interior patch
  return ((long long)(oz + k) * b.N[1] + (oy + jj)) * b.N[0] + (ox + i);
}

__device__ __forceinline__ float block_sum_f(float v, float* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  float s = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
  return s;
}

// out = A_j in on each listed patch (box-restricted level-0 LOR stencil), optionally out = base - A in
__global__ void k_lrn_stencil(PBox b, const int* ids, const float* __restrict__ S, const float* __restrict__ in,
                              const float* __restrict__ base, float* __restrict__ out) {
  const int k = blockIdx.x;
  const int j = ids[k];
  const float* x = in + (long long)k * b.V;
  for (int lex = threadIdx.x; lex < b.V; lex += blockDim.x) {
    const int i = lex % b.A, jj = (lex / b.A) % b.B, kk = lex / (b.A * b.B);
    const long long G = box_global(b, j, lex);
    float s = 0;
    for (int o = 0; o < 27; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
      if ((unsigned)(i + dx) < (unsigned)b.A && (unsigned)(jj + dy) < (unsigned)b.B && (unsigned)(kk + dz) < (unsigned)b.C)
        s += S[(long long)o * b.ntot + G] * x[lex + (dz * b.B + dy) * b.A + dx];
    }
    out[(long long)k * b.V + lex] = base ? base[(long long)k * b.V + lex] - s : s;
  }
}

__global__ void k_lrn_diag(PBox b, const int* ids, const float* __restrict__ S, float* __restrict__ diag) {
  const int k = blockIdx.x;
  for (int lex = threadIdx.x; lex < b.V; lex += blockDim.x)
    diag[(long long)k * b.V + lex] = S[(long long)13 * b.ntot + box_global(b, ids[k], lex)];
}

// random errors e (counter-based: SplitMix64 of (seed, patch slot, voxel), Box-Muller)
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_lrn_noise(int V, int S, unsigned long long seed, float* e) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)S * V) return;
  const unsigned long long a = mix64(seed + 0x9E3779B97F4A7C15ull * (2 * i + 1));
  const unsigned long long c = mix64(seed + 0x9E3779B97F4A7C15ull * (2 * i + 2));
  const double u1 = 1.0 - (double)(a >> 11) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(c >> 11) * (1.0 / 9007199254740992.0);
  e[i] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
}

__global__ void k_sub(const float* a, const float* b, float* c, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) c[i] = a[i] - b[i];
}

// features: x0 = [s t / rho, log(diag / mean diag)], s = diag^-1/2; per patch rho
__global__ void k_lrn_feat(int V, const float* __restrict__ t, const float* __restrict__ diag, float* __restrict__ x0,
                           float* __restrict__ sc, float* __restrict__ rho) {
  __shared__ float sh[32];
  const int k = blockIdx.x;
  const float* tk = t + (long long)k * V;
  const float* dk = diag + (long long)k * V;
  float s2 = 0, sd = 0;
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    const float st = tk[v] * rsqrtf(dk[v]);
    s2 += st * st;
    sd += dk[v];
  }
  const float tot2 = block_sum_f(s2, sh);
  const float totd = block_sum_f(sd, sh);
  const float r = sqrtf(tot2 / V);
  const float rinv = r > 0 ? 1.0f / r : 0.0f;
  const float mean = totd / V;
  if (threadIdx.x == 0) rho[k] = r;
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    const float s = rsqrtf(dk[v]);
    sc[(long long)k * V + v] = s;
    x0[((long long)k * 2 + 0) * V + v] = tk[v] * s * rinv;
    x0[((long long)k * 2 + 1) * V + v] = logf(dk[v] / mean);
  }
}

// ---------------------------------------------------------------------------
// Tensor-core convolutions.  Every 3x3x3 convolution of the network, forward and
// backward, is an implicit GEMM on the BF16 tensor cores (mma.sync m16n8k16, FP32
// accumulation).  Activations and gradients live channel-last in bf16, 16 channels
// (32 bytes) per voxel; layers with fewer channels are zero padded to 16.
//   forward / backward data: out[v][n] = sum_tap sum_k Wt[tap][n][k] in[v + tap][k]
//     (M = 16 voxels of a tile, N = 16 channels, K = 16 channels per tap),
//   weight gradient: dW[tap][o][ci] = sum_v g[v][o] act[v + tap][ci]
//     (M = 16 output channels, N = 16 input channels, K = voxels).
// A CTA takes one patch: its input box goes to shared memory with a one-voxel zero
// halo (the zero padding of the convolution), rows of 32 bytes whose two 16-byte
// halves are swapped on every other group of four rows, so that ldmatrix reads of
// eight consecutive rows hit distinct banks.  The A fragments gather the rows of
// 16 voxels shifted by the tap; ldmatrix takes one row address per lane.

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned swz(unsigned base, int row, int half) {
  return base + (unsigned)row * 32u + ((unsigned)(half ^ ((row >> 2) & 1)) << 4);
}

__device__ __forceinline__ void ldsm4(unsigned addr, unsigned* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}

__device__ __forceinline__ void ldsm2(unsigned addr, unsigned* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}

__device__ __forceinline__ void ldsm4t(unsigned addr, unsigned* r) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}

// d += a b for one m16n8k16 tile (bf16 inputs, fp32 accumulators)
__device__ __forceinline__ void mma16816(float* d, const unsigned* a, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *(const unsigned*)&v;
}

__device__ __forceinline__ unsigned relu_bf16x2(unsigned x) {
  __nv_bfloat162 v = *(const __nv_bfloat162*)&x;
  v = __hmax2(v, __float2bfloat162_rn(0.0f));
  return *(const unsigned*)&v;
}

__device__ __forceinline__ void sts128(unsigned addr, uint4 v) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// Padded input box of patch k in shared memory (rows of 16 bf16 channels, zero
// halo).  IN 0: bf16 rows with ReLU applied (a = max(z, 0)); IN 1: bf16 rows as
// they are; IN 2: fp32 channel-planar [nin][V] (nin <= 2), rounded to bf16 and
// packed along x: the row of voxel (i, j, k) holds the nin channels of voxels
// i-1, i, i+1 (columns 2 dxi + c, zero outside the box), so that a convolution
// takes the three x-taps in one K = 16 step and loops over 9 (dy, dz) groups.
template <int IN>
__device__ __forceinline__ void load_box(const PBox& b, int k, int nin, const void* __restrict__ in, unsigned char* box) {
  const int P0 = b.A + 2, P1 = b.B + 2, P2 = b.C + 2;
  const int rows = P0 * P1 * P2;
  const unsigned base = smem_addr(box);
  for (int idx = threadIdx.x; idx < rows * 2; idx += blockDim.x) {
    const int row = idx >> 1, h = idx & 1;
    const int pi = row % P0, pj = (row / P0) % P1, pk = row / (P0 * P1);
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (pi >= 1 && pi <= b.A && pj >= 1 && pj <= b.B && pk >= 1 && pk <= b.C) {
      const long long v = ((long long)(pk - 1) * b.B + (pj - 1)) * b.A + (pi - 1);
      if constexpr (IN == 2) {
        if (h == 0) {
          const float* f = (const float*)in + (long long)k * nin * b.V;
          unsigned w3[3];
          for (int dxi = 0; dxi < 3; ++dxi) {
            const int ii = pi - 1 + dxi - 1;
            w3[dxi] = 0u;
            if (ii >= 0 && ii < b.A) w3[dxi] = pack_bf16(f[v + dxi - 1], nin > 1 ? f[b.V + v + dxi - 1] : 0.0f);
          }
          val.x = w3[0]; val.y = w3[1]; val.z = w3[2];
        }
      } else {
        val = ((const uint4*)in)[((long long)k * b.V + v) * 2 + h];
        if constexpr (IN == 0) {
          val.x = relu_bf16x2(val.x); val.y = relu_bf16x2(val.y);
          val.z = relu_bf16x2(val.z); val.w = relu_bf16x2(val.w);
        }
      }
    }
    sts128(swz(base, row, h), val);
  }
}

// Implicit-GEMM convolution of one patch per CTA (256 threads, 8 warps, tiles of
// 16 voxels).  Wt: [27][16 n][16 k] bf16 (IN 2: [9 (dy, dz) groups][16 n][16 packed k]).  OUT 0: bf16 rows out[v][n] = acc + bias[n]
// (pre-activation); OUT 1: bf16 rows masked, out[v][n] = zmask[v][n] > 0 ? acc : 0
// (a backward-data step through a ReLU); OUT 2: fp32 out[v] = acc[v][0] + bias[0].
template <int IN, int OUT>
__global__ void __launch_bounds__(256) k_tc_conv(PBox b, int nin, const void* __restrict__ in,
                                                 const __nv_bfloat16* __restrict__ Wt, const float* __restrict__ bias,
                                                 const __nv_bfloat16* __restrict__ zmask, void* __restrict__ out) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int k = blockIdx.x;
  const int P0 = b.A + 2, P1 = b.B + 2, P2 = b.C + 2;
  unsigned char* box = sm;
  unsigned char* wsm = sm + (size_t)P0 * P1 * P2 * 32;
  const unsigned bbase = smem_addr(box), wbase = smem_addr(wsm);
  for (int idx = threadIdx.x; idx < 27 * 16 * 2; idx += blockDim.x)
    sts128(swz(wbase, idx >> 1, idx & 1), ((const uint4*)Wt)[idx]);
  load_box<IN>(b, k, nin, in, box);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int V = b.V, ntile = (V + 15) / 16;
  const int rl = (lane & 7) + ((lane >> 3) & 1) * 8, hl = lane >> 4;     // A rows (voxels) / k half
  const int on = (lane & 7) + (lane >> 4) * 8, wh = (lane >> 3) & 1;     // B rows (n) / k half
  const int g = lane >> 2, t2 = (lane & 3) * 2;                          // accumulator row / column pair
  for (int tile = warp; tile < ntile; tile += 8) {
    const int v = min(tile * 16 + rl, V - 1);
    const int i = v % b.A, j = (v / b.A) % b.B, kk = v / (b.A * b.B);
    const int prow = ((kk + 1) * P1 + (j + 1)) * P0 + (i + 1);
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    constexpr int NT = IN == 2 ? 9 : 27;   // x-packed input: one step per (dy, dz)
#pragma unroll 3
    for (int tap = 0; tap < NT; ++tap) {
      const int dx = IN == 2 ? 0 : tap % 3 - 1;
      const int dy = IN == 2 ? tap % 3 - 1 : (tap / 3) % 3 - 1, dz = IN == 2 ? tap / 3 - 1 : tap / 9 - 1;
      const int r = prow + (dz * P1 + dy) * P0 + dx;
      unsigned a[4], bq[4];
      ldsm4(swz(bbase, r, hl), a);
      if constexpr (OUT == 2) {   // one output channel: the n 0-7 half only
        ldsm2(swz(wbase, tap * 16 + on, wh), bq);
        mma16816(acc[0], a, bq[0], bq[1]);
      } else {
        ldsm4(swz(wbase, tap * 16 + on, wh), bq);
        mma16816(acc[0], a, bq[0], bq[1]);
        mma16816(acc[1], a, bq[2], bq[3]);
      }
    }
    const long long v0 = (long long)tile * 16 + g, v1 = v0 + 8;
#pragma unroll
    for (int nh = 0; nh < 2; ++nh) {
      const int n = nh * 8 + t2;
      if constexpr (OUT == 2) {
        if (nh == 0 && t2 == 0) {
          float* y = (float*)out + (long long)k * V;
          if (v0 < V) y[v0] = acc[0][0] + bias[0];
          if (v1 < V) y[v1] = acc[0][2] + bias[0];
        }
      } else {
        unsigned* o = (unsigned*)out;
        const long long q0 = ((long long)k * V + v0) * 8 + (n >> 1), q1 = ((long long)k * V + v1) * 8 + (n >> 1);
        if constexpr (OUT == 0) {
          if (v0 < V) o[q0] = pack_bf16(acc[nh][0] + bias[n], acc[nh][1] + bias[n + 1]);
          if (v1 < V) o[q1] = pack_bf16(acc[nh][2] + bias[n], acc[nh][3] + bias[n + 1]);
        } else {
          const unsigned* zm = (const unsigned*)zmask;
          if (v0 < V) {
            const unsigned zr = zm[q0];
            const __nv_bfloat162 z = *(const __nv_bfloat162*)&zr;
            o[q0] = pack_bf16(__low2float(z) > 0.f ? acc[nh][0] : 0.f, __high2float(z) > 0.f ? acc[nh][1] : 0.f);
          }
          if (v1 < V) {
            const unsigned zr = zm[q1];
            const __nv_bfloat162 z = *(const __nv_bfloat162*)&zr;
            o[q1] = pack_bf16(__low2float(z) > 0.f ? acc[nh][2] : 0.f, __high2float(z) > 0.f ? acc[nh][3] : 0.f);
          }
        }
      }
    }
  }
}

// Weight gradient of one patch per CTA: dWp[k][tap][o][ci] = sum_v g[v][o] act[v + tap][ci]
// and dbp[k][o] = sum_v g[v][o].  GIN 0: g as bf16 rows; GIN 1: g fp32 [V] (one
// channel), rounded to bf16.  AIN: the activation box as in load_box (0: bf16 rows
// + ReLU, 2: fp32 planar x0, packed along x: the tap slots are then the 9 (dy, dz)
// groups and the columns 2 dxi + ci).  The voxels stream through shared memory 64
// at a time; warp w accumulates the tap slots w, w+8, w+16, w+24.
template <int GIN, int AIN>
__global__ void __launch_bounds__(256) k_tc_wgrad(PBox b, int nin, const void* __restrict__ gin,
                                                  const void* __restrict__ act, float* __restrict__ dWp,
                                                  float* __restrict__ dbp) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int k = blockIdx.x;
  const int P0 = b.A + 2, P1 = b.B + 2, P2 = b.C + 2;
  unsigned char* box = sm;
  unsigned char* gsm = sm + (size_t)P0 * P1 * P2 * 32;
  const unsigned bbase = smem_addr(box), gbase = smem_addr(gsm);
  load_box<AIN>(b, k, nin, act, box);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int V = b.V;
  float acc[4][2][4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int nh = 0; nh < 2; ++nh)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[m][nh][q] = 0.f;
  const int ar = (lane & 7) + (lane >> 4) * 8, ah = (lane >> 3) & 1;       // A (g^T) rows: voxels / o half
  const int br = (lane & 7) + ((lane >> 3) & 1) * 8, bh = lane >> 4;       // B (act) rows: voxels / ci half
  float bsum = 0.f;   // threads 0..15: bias gradient of channel threadIdx.x
  for (int v0 = 0; v0 < V; v0 += 64) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < 64 * 2; idx += blockDim.x) {
      const int row = idx >> 1, h = idx & 1;
      const long long v = v0 + row;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (v < V) {
        if constexpr (GIN == 1) {
          if (h == 0) val.x = pack_bf16(((const float*)gin)[(long long)k * V + v], 0.0f);
        } else {
          val = ((const uint4*)gin)[((long long)k * V + v) * 2 + h];
        }
      }
      sts128(swz(gbase, row, h), val);
    }
    __syncthreads();
    if (threadIdx.x < 16) {   // bias gradient from the same bf16 values, voxel order fixed
      const int o = threadIdx.x;
      for (int row = 0; row < 64 && v0 + row < V; ++row) {
        const unsigned short* hrow = (const unsigned short*)(gsm + row * 32 + (((o >> 3) ^ ((row >> 2) & 1)) << 4));
        bsum += __bfloat162float(__ushort_as_bfloat16(hrow[o & 7]));
      }
    }
    for (int sub = 0; sub < 4 && v0 + sub * 16 < V; ++sub) {
      unsigned a[4];
      ldsm4t(swz(gbase, sub * 16 + ar, ah), a);
      const int v = min(v0 + sub * 16 + br, V - 1);   // rows past V meet zero g rows
      const int i = v % b.A, j = (v / b.A) % b.B, kk = v / (b.A * b.B);
      const int prow = ((kk + 1) * P1 + (j + 1)) * P0 + (i + 1);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int tap = warp + 8 * m;
        if (tap < (AIN == 2 ? 9 : 27)) {
          const int dx = AIN == 2 ? 0 : tap % 3 - 1;
          const int dy = AIN == 2 ? tap % 3 - 1 : (tap / 3) % 3 - 1, dz = AIN == 2 ? tap / 3 - 1 : tap / 9 - 1;
          unsigned bq[4];
          ldsm4t(swz(bbase, prow + (dz * P1 + dy) * P0 + dx, bh), bq);
          mma16816(acc[m][0], a, bq[0], bq[1]);
          mma16816(acc[m][1], a, bq[2], bq[3]);
        }
      }
    }
  }
  const int g = lane >> 2, t2 = (lane & 3) * 2;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int tap = warp + 8 * m;
    if (tap >= (AIN == 2 ? 9 : 27)) continue;
    float* d = dWp + ((long long)k * 27 + tap) * 256;
#pragma unroll
    for (int nh = 0; nh < 2; ++nh) {
      const int ci = nh * 8 + t2;
      d[g * 16 + ci] = acc[m][nh][0];
      d[g * 16 + ci + 1] = acc[m][nh][1];
      d[(g + 8) * 16 + ci] = acc[m][nh][2];
      d[(g + 8) * 16 + ci + 1] = acc[m][nh][3];
    }
  }
  if (threadIdx.x < 16) dbp[(long long)k * 16 + threadIdx.x] = bsum;
}

// G[W][o][ci][tap] = sum over the S patches (in order) of dWp[k][tap][o][ci], for
// o < cout, ci < cin (packed: dWp[k][tap / 3][o][2 (tap % 3) + ci], the x-packed
// layout); G[b][o] likewise from dbp.
__global__ void k_tc_wreduce(int S, int cin, int cout, int packed, const float* __restrict__ dWp,
                             const float* __restrict__ dbp, float* __restrict__ GW, float* __restrict__ Gb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nw = cout * cin * 27;
  if (idx < nw) {
    const int tap = idx % 27, ci = (idx / 27) % cin, o = idx / (27 * cin);
    const int slot = packed ? tap / 3 : tap, col = packed ? 2 * (tap % 3) + ci : ci;
    float s = 0.f;
    for (int k = 0; k < S; ++k) s += dWp[((long long)k * 27 + slot) * 256 + o * 16 + col];
    GW[idx] = s;
  } else if (idx < nw + cout) {
    const int o = idx - nw;
    float s = 0.f;
    for (int k = 0; k < S; ++k) s += dbp[(long long)k * 16 + o];
    Gb[o] = s;
  }
}

// Tensor-core weight sets from the bf16 parameters W[o][ci][tap] (cout x cin):
// forward Wt[tap][n = o][k = ci]; backward data (the transposed convolution, taps
// mirrored) Wt[tap][n = ci][k = o] = W[o][ci][26 - tap]; zero outside the layer's
// channels.  packed (for an x-packed input, at most 2 input channels): slot g =
// (dz+1) 3 + (dy+1) and column 2 dxi + c hold the entry of tap 3 g + dxi, channel c.
// Padded biases: bias16[n] = b[n] for n < cout, else 0.
__global__ void k_tc_prep(const __nv_bfloat16* __restrict__ Wb, const float* __restrict__ bias, int cin, int cout,
                          int transpose, int packed, __nv_bfloat16* __restrict__ Wt, float* __restrict__ bias16) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < 27 * 256) {
    const int slot = idx / 256, n = (idx / 16) % 16, col = idx % 16;
    // the tap and the input channel (k) of this entry
    int tap = slot, kk = col;
    bool live = true;
    if (packed) {
      tap = 3 * slot + col / 2;
      kk = col % 2;
      live = slot < 9 && col < 6;
    }
    __nv_bfloat16 w = __float2bfloat16(0.0f);
    if (live) {
      if (!transpose) {
        if (n < cout && kk < cin) w = Wb[(n * cin + kk) * 27 + tap];
      } else {
        if (kk < cout && n < cin) w = Wb[(kk * cin + n) * 27 + (26 - tap)];
      }
    }
    Wt[idx] = w;
  }
  if (bias16 && idx < 16) bias16[idx] = idx < cout ? bias[idx] : 0.0f;
}

// c = rho s y, and optionally z[G] += c on the listed patches of colour class cls
// (vertex index parity per axis): patches of one class do not overlap, so the adds
// need no atomics, and the classes run one after another in a fixed order.
__global__ void k_lrn_out(PBox b, const int* ids, const float* __restrict__ y, const float* __restrict__ sc,
                          const float* __restrict__ rho, float* __restrict__ cout, float* z, int cls) {
  const int k = blockIdx.y;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.V) return;
  const long long q = (long long)k * b.V + v;
  const float c = rho[k] * sc[q] * y[q];
  if (cout) cout[q] = c;
  if (z) {
    const int j = ids[k];
    const int vx = j % (b.n[0] + 1), vy = (j / (b.n[0] + 1)) % (b.n[1] + 1), vz = j / ((b.n[0] + 1) * (b.n[1] + 1));
    if (((vx & 1) | ((vy & 1) << 1) | ((vz & 1) << 2)) == cls) z[box_global(b, j, v)] += c;
  }
}

// loss and dL/dy per patch: d = delta - c, Ad = A_j d, L = d.Ad / delta.t, gy = -2 rho s Ad / norm
__global__ void k_lrn_loss(PBox b, const int* ids, const float* __restrict__ S, const float* __restrict__ delta,
                           const float* __restrict__ t, const float* __restrict__ c, const float* __restrict__ sc,
                           const float* __restrict__ rho, float* __restrict__ gy, float* __restrict__ loss) {
  extern __shared__ float d[];
  __shared__ float sh[32];
  const int k = blockIdx.x;
  const int j = ids[k];
  const long long base = (long long)k * b.V;
  float nrm = 0;
  for (int v = threadIdx.x; v < b.V; v += blockDim.x) {
    d[v] = delta[base + v] - c[base + v];
    nrm += delta[base + v] * t[base + v];
  }
  __syncthreads();
  float num = 0;
  const float norm = block_sum_f(nrm, sh);
  for (int lex = threadIdx.x; lex < b.V; lex += blockDim.x) {
    const int i = lex % b.A, jj = (lex / b.A) % b.B, kk = lex / (b.A * b.B);
    const long long G = box_global(b, j, lex);
    float s = 0;
    for (int o = 0; o < 27; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
      if ((unsigned)(i + dx) < (unsigned)b.A && (unsigned)(jj + dy) < (unsigned)b.B && (unsigned)(kk + dz) < (unsigned)b.C)
        s += S[(long long)o * b.ntot + G] * d[lex + (dz * b.B + dy) * b.A + dx];
    }
    num += d[lex] * s;
    gy[base + lex] = -2.0f * rho[k] * sc[base + lex] * s / norm;
  }
  const float tot = block_sum_f(num, sh);
  if (threadIdx.x == 0) loss[k] = tot / norm;
}

__global__ void k_lrn_adam(int n, float* P, const float* G, float* m, float* v, float lr, float b1t, float b2t,
                           float scale, __nv_bfloat16* Pb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i] * scale;
  m[i] = 0.9f * m[i] + 0.1f * g;
  v[i] = 0.999f * v[i] + 0.001f * g * g;
  const float mh = m[i] / (1.0f - b1t), vh = v[i] / (1.0f - b2t);
  P[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
  Pb[i] = __float2bfloat16(P[i]);
}

__global__ void k_f2bf(int n, const float* P, __nv_bfloat16* Pb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Pb[i] = __float2bfloat16(P[i]);
}

}  // namespace

struct LearnState {
  PBox box;
  int nint = 0;          // interior patches (the first nint entries of the visiting order)
  int S = 0;             // batch (patches per chunk)
  float* P = nullptr;    // FP32 master parameters [NPARAM]
  __nv_bfloat16* Pb = nullptr;
  float *G = nullptr, *m = nullptr, *v = nullptr;
  int adam_t = 0;
  float *x0, *z1, *z2, *y, *g2, *g1, *gy, *sc, *rho, *loss, *cc;
  float *e, *r, *x, *t, *delta, *diag;
  // tensor-core weight sets ([27][16][16] bf16): forward layers 1-3, backward data of
  // layers 3 and 2; padded biases of the forward layers; per-patch weight-gradient
  // partials (summed in patch order by k_tc_wreduce)
  __nv_bfloat16* Wt[5] = {};
  float* bias16[3] = {};
  float *dWp = nullptr, *dbp = nullptr;
  int smem_conv = 0, smem_wgrad = 0;
  float* diag_all = nullptr;   // diag of every interior patch (inference)
  int* ids = nullptr;          // interior patch ids in visiting order
  int* bids = nullptr;         // patch ids of the current training batch
};

static LearnState* LS(lor_ctx* c) { return (LearnState*)c->learned; }

static lor_status learned_init(lor_ctx* c) {
  if (c->learned) return LOR_OK;
  if (c->dim != 3 || c->dg_state) return lor_fail(c, LOR_EINVAL, "learned correction: 3D CG contexts only");
  if (!c->h_spans.empty()) return lor_fail(c, LOR_EINVAL, "learned correction: vertex patches only");
  LearnState* s = new LearnState();
  c->learned = s;
  const BoxShape& bs = c->shapes[0];
  s->box.A = bs.dims[0]; s->box.B = bs.dims[1]; s->box.C = bs.dims[2]; s->box.V = bs.rows;
  for (int a = 0; a < 3; ++a) { s->box.n[a] = c->n[a]; s->box.N[a] = c->lev[0].N[a]; }
  s->box.m = c->lev[0].m;
  s->box.ntot = c->lev[0].ntot;
  s->nint = 1;
  for (int a = 0; a < 3; ++a) s->nint *= std::max(c->n[a] - 1, 0);
  s->S = std::max(1, std::min(s->nint, 2048));
  const long long SV = (long long)s->S * s->box.V;
  auto F = [&](long long k) { return (float*)lor_alloc(c, std::max<long long>(k, 1) * 4); };
  s->P = F(NPARAM); s->G = F(NPARAM); s->m = F(NPARAM); s->v = F(NPARAM);
  s->Pb = (__nv_bfloat16*)lor_alloc(c, NPARAM * 2);
  s->x0 = F(2 * SV); s->z1 = F(CH * SV); s->z2 = F(CH * SV); s->y = F(SV);
  s->g2 = F(CH * SV); s->g1 = F(CH * SV); s->gy = F(SV); s->sc = F(SV); s->rho = F(s->S); s->loss = F(s->S);
  s->cc = F(SV);
  s->e = F(SV); s->r = F(SV); s->x = F(SV); s->t = F(SV); s->delta = F(SV); s->diag = F(SV);
  s->diag_all = F((long long)s->nint * s->box.V);
  for (int q = 0; q < 5; ++q) s->Wt[q] = (__nv_bfloat16*)lor_alloc(c, 27 * 256 * 2);
  for (int q = 0; q < 3; ++q) s->bias16[q] = F(16);
  s->dWp = F((long long)s->S * 27 * 256);
  s->dbp = F((long long)s->S * 16);
  s->ids = c->d_porder;   // interior patches come first in the visiting order
  s->bids = (int*)lor_alloc(c, (size_t)s->S * 4);
  c->learned_tout = F((long long)s->nint * s->box.V);
  if (!s->P || !s->G || !s->m || !s->v || !s->Pb || !s->x0 || !s->z1 || !s->z2 || !s->y || !s->g2 || !s->g1 ||
      !s->gy || !s->sc || !s->rho || !s->loss || !s->cc || !s->e || !s->r || !s->x || !s->t || !s->delta ||
      !s->diag || !s->diag_all || !c->learned_tout || !s->bids || !s->Wt[0] || !s->Wt[1] || !s->Wt[2] ||
      !s->Wt[3] || !s->Wt[4] || !s->bias16[0] || !s->bias16[1] || !s->bias16[2] || !s->dWp || !s->dbp)
    return lor_fail(c, LOR_ENOMEM, "alloc learned-correction buffers");
  {
    const long long rows = (long long)(s->box.A + 2) * (s->box.B + 2) * (s->box.C + 2);
    s->smem_conv = (int)(rows * 32 + 27 * 16 * 32);
    s->smem_wgrad = (int)(rows * 32 + 64 * 32);
    int dev = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (s->smem_conv > maxsm || s->smem_wgrad > maxsm) return lor_fail(c, LOR_EINVAL, "learned correction: patch too large");
    cudaFuncSetAttribute(k_tc_conv<2, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_conv);
    cudaFuncSetAttribute(k_tc_conv<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_conv);
    cudaFuncSetAttribute(k_tc_conv<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_conv);
    cudaFuncSetAttribute(k_tc_conv<2, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_conv);
    cudaFuncSetAttribute(k_tc_conv<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_conv);
    cudaFuncSetAttribute(k_tc_wgrad<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_wgrad);
    cudaFuncSetAttribute(k_tc_wgrad<0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_wgrad);
    cudaFuncSetAttribute(k_tc_wgrad<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s->smem_wgrad);
  }
  if (s->nint > 0) {
    k_lrn_diag<<<s->nint, 128, 0, c->stream>>>(s->box, s->ids, c->d_S32[0], s->diag_all);
    ++c->launches;
  }
  return lor_cuda_check(c, cudaGetLastError(), "learned init");
}

// tensor-core weight sets and padded biases from the current parameters
static void prep_weights(lor_ctx* c) {
  LearnState* s = LS(c);
  const unsigned g = (27 * 256 + 255) / 256;
  // layer 1 reads the x-packed features, the layer-3 backward-data step the x-packed gy
  k_tc_prep<<<g, 256, 0, c->stream>>>(s->Pb + OFF_W1, s->P + OFF_B1, 2, CH, 0, 1, s->Wt[0], s->bias16[0]);
  k_tc_prep<<<g, 256, 0, c->stream>>>(s->Pb + OFF_W2, s->P + OFF_B2, CH, CH, 0, 0, s->Wt[1], s->bias16[1]);
  k_tc_prep<<<g, 256, 0, c->stream>>>(s->Pb + OFF_W3, s->P + OFF_B3, CH, 1, 0, 0, s->Wt[2], s->bias16[2]);
  k_tc_prep<<<g, 256, 0, c->stream>>>(s->Pb + OFF_W3, nullptr, CH, 1, 1, 1, s->Wt[3], nullptr);
  k_tc_prep<<<g, 256, 0, c->stream>>>(s->Pb + OFF_W2, nullptr, CH, CH, 1, 0, s->Wt[4], nullptr);
  c->launches += 5;
}

// forward of S patches: t, diag -> y (and the cache: features x0, pre-activations
// z1, z2 as bf16 rows)
static void forward(lor_ctx* c, int S, const float* t, const float* diag) {
  LearnState* s = LS(c);
  const PBox& b = s->box;
  k_lrn_feat<<<S, 256, 0, c->stream>>>(b.V, t, diag, s->x0, s->sc, s->rho);
  k_tc_conv<2, 0><<<S, 256, s->smem_conv, c->stream>>>(b, 2, s->x0, s->Wt[0], s->bias16[0], nullptr, s->z1);
  k_tc_conv<0, 0><<<S, 256, s->smem_conv, c->stream>>>(b, 0, s->z1, s->Wt[1], s->bias16[1], nullptr, s->z2);
  k_tc_conv<0, 2><<<S, 256, s->smem_conv, c->stream>>>(b, 0, s->z2, s->Wt[2], s->bias16[2], nullptr, s->y);
  c->launches += 4;
}

// gradients of the summed loss of S patches into s->G (overwritten)
static void backward(lor_ctx* c, int S, const int* ids, const float* t, const float* delta) {
  LearnState* s = LS(c);
  const PBox& b = s->box;
  const dim3 grid((unsigned)lor_ceil_div(b.V, 256), S);
  k_lrn_out<<<grid, 256, 0, c->stream>>>(b, ids, s->y, s->sc, s->rho, s->cc, nullptr, 0);
  k_lrn_loss<<<S, 256, b.V * sizeof(float), c->stream>>>(b, ids, c->d_S32[0], delta, t, s->cc, s->sc, s->rho, s->gy,
                                                          s->loss);
  const unsigned gw3 = (unsigned)lor_ceil_div(1 * CH * 27 + 1, 256), gw2 = (unsigned)lor_ceil_div(CH * CH * 27 + CH, 256),
                 gw1 = (unsigned)lor_ceil_div(CH * 2 * 27 + CH, 256);
  // layer 3: weight gradient from gy and a2 = relu(z2); data gradient g2 = (W3^T gy) relu'(z2)
  k_tc_wgrad<1, 0><<<S, 256, s->smem_wgrad, c->stream>>>(b, 0, s->gy, s->z2, s->dWp, s->dbp);
  k_tc_wreduce<<<gw3, 256, 0, c->stream>>>(S, CH, 1, 0, s->dWp, s->dbp, s->G + OFF_W3, s->G + OFF_B3);
  k_tc_conv<2, 1><<<S, 256, s->smem_conv, c->stream>>>(b, 1, s->gy, s->Wt[3], nullptr, (const __nv_bfloat16*)s->z2,
                                                        s->g2);
  // layer 2: weight gradient from g2 and a1 = relu(z1); g1 = (W2^T g2) relu'(z1)
  k_tc_wgrad<0, 0><<<S, 256, s->smem_wgrad, c->stream>>>(b, 0, s->g2, s->z1, s->dWp, s->dbp);
  k_tc_wreduce<<<gw2, 256, 0, c->stream>>>(S, CH, CH, 0, s->dWp, s->dbp, s->G + OFF_W2, s->G + OFF_B2);
  k_tc_conv<1, 1><<<S, 256, s->smem_conv, c->stream>>>(b, 0, s->g2, s->Wt[4], nullptr, (const __nv_bfloat16*)s->z1,
                                                        s->g1);
  // layer 1: weight gradient from g1 and the features x0
  k_tc_wgrad<0, 2><<<S, 256, s->smem_wgrad, c->stream>>>(b, 2, s->g1, s->x0, s->dWp, s->dbp);
  k_tc_wreduce<<<gw1, 256, 0, c->stream>>>(S, 2, CH, 1, s->dWp, s->dbp, s->G + OFF_W1, s->G + OFF_B1);
  c->launches += 10;
}

lor_status lor_learned_apply(lor_ctx* c, float* z) {
  LearnState* s = LS(c);
  const PBox& b = s->box;
  for (int k0 = 0; k0 < s->nint; k0 += s->S) {
    const int S = std::min(s->S, s->nint - k0);
    const float* t = c->learned_tout + (long long)k0 * b.V;
    forward(c, S, t, s->diag_all + (long long)k0 * b.V);
    const dim3 grid((unsigned)lor_ceil_div(b.V, 256), S);
    for (int cls = 0; cls < 8; ++cls) {   // overlapping patches add in a fixed class order
      k_lrn_out<<<grid, 256, 0, c->stream>>>(b, s->ids + k0, s->y, s->sc, s->rho, nullptr, z, cls);
      ++c->launches;
    }
  }
  return lor_cuda_check(c, cudaGetLastError(), "learned apply");
}


extern "C" {

lor_status lor_learned_params(lor_ctx* c, const float* h_in, float* h_out, int count) {
  if (!c || !c->setup_done) return LOR_EINVAL;
  if (count != NPARAM) return lor_fail(c, LOR_EINVAL, "learned parameters: wrong count");
  lor_status st = learned_init(c);
  if (st) return st;
  LearnState* s = LS(c);
  cudaError_t e = cudaSuccess;
  if (h_in) {
    e = cudaMemcpyAsync(s->P, h_in, NPARAM * 4, cudaMemcpyHostToDevice, c->stream);
    k_f2bf<<<(NPARAM + 255) / 256, 256, 0, c->stream>>>(NPARAM, s->P, s->Pb);
    ++c->launches;
    prep_weights(c);
    cudaMemsetAsync(s->m, 0, NPARAM * 4, c->stream);
    cudaMemsetAsync(s->v, 0, NPARAM * 4, c->stream);
    s->adam_t = 0;
  }
  if (h_out && e == cudaSuccess) e = cudaMemcpyAsync(h_out, s->P, NPARAM * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return lor_cuda_check(c, e, "learned parameters");
}

lor_status lor_learned_enable(lor_ctx* c, int on) {
  if (!c || !c->setup_done) return LOR_EINVAL;
  // the correction is trained on the residuals of the unit-weight patch cycle
  if (on && c->opt.weighting) return lor_fail(c, LOR_EINVAL, "learned correction needs unit patch weights");
  if (on && c->schwarz) return lor_fail(c, LOR_EINVAL, "learned correction needs the additive form");
  lor_status st = learned_init(c);
  if (st) return st;
  c->learned_on = on != 0 && LS(c)->nint > 0;
  return LOR_OK;
}

lor_status lor_learned_variant(lor_ctx* c, int variant) {
  if (!c || !c->setup_done) return LOR_EINVAL;
  if (variant < 0 || variant > 1) return lor_fail(c, LOR_EINVAL, "learned variant: 0 (add) or 1 (replace)");
  c->learned_replace = variant == 1;
  return LOR_OK;
}

lor_status lor_learned_eval(lor_ctx* c, int npatch, const int* d_ids, const float* d_t, const float* d_delta,
                            float* d_c, float* d_loss, float* h_grad) {
  if (!c || !c->learned || npatch < 1 || npatch > LS(c)->S || !d_ids || !d_t) return LOR_EINVAL;
  LearnState* s = LS(c);
  const PBox& b = s->box;
  k_lrn_diag<<<npatch, 128, 0, c->stream>>>(b, d_ids, c->d_S32[0], s->diag);
  ++c->launches;
  forward(c, npatch, d_t, s->diag);
  if (d_delta) {
    backward(c, npatch, d_ids, d_t, d_delta);
    if (d_loss) cudaMemcpyAsync(d_loss, s->loss, npatch * 4, cudaMemcpyDeviceToDevice, c->stream);
    if (h_grad) cudaMemcpyAsync(h_grad, s->G, NPARAM * 4, cudaMemcpyDeviceToHost, c->stream);
  } else {
    const dim3 grid((unsigned)lor_ceil_div(b.V, 256), npatch);
    k_lrn_out<<<grid, 256, 0, c->stream>>>(b, d_ids, s->y, s->sc, s->rho, s->cc, nullptr, 0);
    ++c->launches;
  }
  if (d_c) cudaMemcpyAsync(d_c, s->cc, (size_t)npatch * b.V * 4, cudaMemcpyDeviceToDevice, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  return lor_cuda_check(c, e, "learned eval");
}

lor_status lor_learned_train(lor_ctx* c, int steps, int batch, float lr, unsigned long long seed, float* h_loss) {
  if (!c || !c->setup_done || steps < 0 || !(lr > 0)) return LOR_EINVAL;
  lor_status st = learned_init(c);
  if (st) return st;
  LearnState* s = LS(c);
  if (s->nint == 0) return lor_fail(c, LOR_EINVAL, "no interior patch to train on");
  const PBox& b = s->box;
  const int S = std::max(1, std::min({batch, s->S, s->nint}));
  std::vector<int> order(s->nint), hid(S);
  std::vector<float> hl(S);
  cudaMemcpy(order.data(), s->ids, s->nint * 4, cudaMemcpyDeviceToHost);
  const long long SV = (long long)S * b.V;
  for (int it = 0; it < steps; ++it) {
    // batch: S patches spread over the interior, rotating with the step
    for (int k = 0; k < S; ++k) hid[k] = order[(size_t)((it * 7919ull + (unsigned long long)k * s->nint / S) % s->nint)];
    cudaMemcpyAsync(s->bids, hid.data(), S * 4, cudaMemcpyHostToDevice, c->stream);
    // data: e random, r = A e, x = V(r), t = r - A x = A delta, delta = e - x
    k_lrn_noise<<<(unsigned)lor_ceil_div(SV, 256), 256, 0, c->stream>>>(b.V, S, seed + 0x1000193ull * (it + 1), s->e);
    k_lrn_stencil<<<S, 128, 0, c->stream>>>(b, s->bids, c->d_S32[0], s->e, nullptr, s->r);
    c->launches += 2;
    if ((st = lor_patch_local32(c, s->bids, S, s->r, s->x, b.V))) return st;
    k_lrn_stencil<<<S, 128, 0, c->stream>>>(b, s->bids, c->d_S32[0], s->x, s->r, s->t);
    k_sub<<<(unsigned)lor_ceil_div(SV, 256), 256, 0, c->stream>>>(s->e, s->x, s->delta, SV);
    k_lrn_diag<<<S, 128, 0, c->stream>>>(b, s->bids, c->d_S32[0], s->diag);
    c->launches += 3;
    forward(c, S, s->t, s->diag);
    backward(c, S, s->bids, s->t, s->delta);
    s->adam_t += 1;
    const float b1t = powf(0.9f, (float)s->adam_t), b2t = powf(0.999f, (float)s->adam_t);
    k_lrn_adam<<<(NPARAM + 255) / 256, 256, 0, c->stream>>>(NPARAM, s->P, s->G, s->m, s->v, lr, b1t, b2t,
                                                            1.0f / S, s->Pb);
    ++c->launches;
    prep_weights(c);
    if (h_loss) {
      cudaMemcpyAsync(hl.data(), s->loss, S * 4, cudaMemcpyDeviceToHost, c->stream);
      cudaError_t e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) return lor_cuda_check(c, e, "learned train");
      double m = 0;
      for (float v : hl) m += v;
      h_loss[it] = (float)(m / S);
    }
  }
  return lor_cuda_check(c, cudaStreamSynchronize(c->stream), "learned train");
}

}  // extern "C"

void lor_free_learned(lor_ctx* c) {
  delete LS(c);
  c->learned = nullptr;
}
