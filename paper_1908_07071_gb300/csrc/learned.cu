// Learned per-patch correction of the LOR V-cycle (the learned form).
//
// On every interior vertex patch, after the V(1,1) cycle (Section 3.3) leaves a
// level-0 residual t, a 3-layer convolutional network adds the correction
//   c = rho * s * N([s * t / rho, log(diag / mean diag)]),  s = diag^(-1/2),
//   N = conv3^3(2->16) - ReLU - conv3^3(16->16) - ReLU - conv3^3(16->1),
// zero padding at the patch boundary, rho = rms(s * t).  Weights are stored in
// bf16 and applied with FP32 accumulation.  Training minimises the normalised
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

// z_out[o][v] = b[o] + sum_{i,tap} W[o][i][tap] * act(in[i][v + tap]); act = ReLU if RELU_IN
template <int CIN, int COUT, bool RELU_IN>
__global__ void __launch_bounds__(256) k_lrn_conv(PBox b, const __nv_bfloat16* __restrict__ Wb,
                                                  const float* __restrict__ bias, const float* __restrict__ in,
                                                  float* __restrict__ out) {
  __shared__ float W[COUT * CIN * 27];
  for (int i = threadIdx.x; i < COUT * CIN * 27; i += blockDim.x) W[i] = __bfloat162float(Wb[i]);
  __syncthreads();
  const int k = blockIdx.y;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.V) return;
  const int i = v % b.A, j = (v / b.A) % b.B, kk = v / (b.A * b.B);
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = bias[o];
  const float* ink = in + (long long)k * CIN * b.V;
  for (int tap = 0; tap < 27; ++tap) {
    const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
    if (!((unsigned)(i + dx) < (unsigned)b.A && (unsigned)(j + dy) < (unsigned)b.B && (unsigned)(kk + dz) < (unsigned)b.C))
      continue;
    const int vn = v + (dz * b.B + dy) * b.A + dx;
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) {
      float a = ink[(long long)ci * b.V + vn];
      if (RELU_IN) a = fmaxf(a, 0.0f);
#pragma unroll
      for (int o = 0; o < COUT; ++o) acc[o] += W[(o * CIN + ci) * 27 + tap] * a;
    }
  }
  float* ok = out + (long long)k * COUT * b.V;
#pragma unroll
  for (int o = 0; o < COUT; ++o) ok[(long long)o * b.V + v] = acc[o];
}

// c = rho s y, and optionally z[G] += c on the listed patches
__global__ void k_lrn_out(PBox b, const int* ids, const float* __restrict__ y, const float* __restrict__ sc,
                          const float* __restrict__ rho, float* __restrict__ cout, float* z) {
  const int k = blockIdx.y;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.V) return;
  const long long q = (long long)k * b.V + v;
  const float c = rho[k] * sc[q] * y[q];
  if (cout) cout[q] = c;
  if (z) atomicAdd(z + box_global(b, ids[k], v), c);
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

// g_in[i][v] = relu'(z_in[i][v]) * sum_{o,tap} W[o][i][tap] g_out[o][v - tap]
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_lrn_bwd_data(PBox b, const __nv_bfloat16* __restrict__ Wb,
                                                      const float* __restrict__ gout, const float* __restrict__ zin,
                                                      float* __restrict__ gin) {
  __shared__ float W[COUT * CIN * 27];
  for (int i = threadIdx.x; i < COUT * CIN * 27; i += blockDim.x) W[i] = __bfloat162float(Wb[i]);
  __syncthreads();
  const int k = blockIdx.y;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= b.V) return;
  const int i = v % b.A, j = (v / b.A) % b.B, kk = v / (b.A * b.B);
  float acc[CIN];
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.0f;
  const float* gk = gout + (long long)k * COUT * b.V;
  for (int tap = 0; tap < 27; ++tap) {
    const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
    // output voxel u with u + tap = v
    if (!((unsigned)(i - dx) < (unsigned)b.A && (unsigned)(j - dy) < (unsigned)b.B && (unsigned)(kk - dz) < (unsigned)b.C))
      continue;
    const int u = v - ((dz * b.B + dy) * b.A + dx);
#pragma unroll
    for (int o = 0; o < COUT; ++o) {
      const float g = gk[(long long)o * b.V + u];
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) acc[ci] += W[(o * CIN + ci) * 27 + tap] * g;
    }
  }
  const float* zk = zin + (long long)k * CIN * b.V;
  float* out = gin + (long long)k * CIN * b.V;
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci) out[(long long)ci * b.V + v] = zk[(long long)ci * b.V + v] > 0.0f ? acc[ci] : 0.0f;
}

// dW[o][i][tap] += sum_v g[o][v] act(in[i][v + tap]); db[o] += sum_v g[o][v]  (one CTA per patch)
template <int CIN, int COUT, bool RELU_IN>
__global__ void __launch_bounds__(256) k_lrn_bwd_w(PBox b, const float* __restrict__ gout, const float* __restrict__ in,
                                                   float* __restrict__ dW, float* __restrict__ db) {
  const int k = blockIdx.x;
  const float* gk = gout + (long long)k * COUT * b.V;
  const float* ik = in + (long long)k * CIN * b.V;
  for (int w = threadIdx.x; w < COUT * CIN * 27; w += blockDim.x) {
    const int tap = w % 27, ci = (w / 27) % CIN, o = w / (27 * CIN);
    const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
    const int off = (dz * b.B + dy) * b.A + dx;
    float acc = 0;
    for (int v = 0; v < b.V; ++v) {
      const int i = v % b.A, j = (v / b.A) % b.B, kk = v / (b.A * b.B);
      if (!((unsigned)(i + dx) < (unsigned)b.A && (unsigned)(j + dy) < (unsigned)b.B && (unsigned)(kk + dz) < (unsigned)b.C))
        continue;
      float a = ik[(long long)ci * b.V + v + off];
      if (RELU_IN) a = fmaxf(a, 0.0f);
      acc += gk[(long long)o * b.V + v] * a;
    }
    atomicAdd(dW + w, acc);
  }
  for (int o = threadIdx.x; o < COUT; o += blockDim.x) {
    float s = 0;
    for (int v = 0; v < b.V; ++v) s += gk[(long long)o * b.V + v];
    atomicAdd(db + o, s);
  }
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
  float* diag_all = nullptr;   // diag of every interior patch (inference)
  int* ids = nullptr;          // interior patch ids in visiting order
  int* bids = nullptr;         // patch ids of the current training batch
};

static LearnState* LS(lor_ctx* c) { return (LearnState*)c->learned; }

static lor_status learned_init(lor_ctx* c) {
  if (c->learned) return LOR_OK;
  if (c->dim != 3 || c->dg_state) return lor_fail(c, LOR_EINVAL, "learned correction: 3D CG contexts only");
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
  s->ids = c->d_porder;   // interior patches come first in the visiting order
  s->bids = (int*)lor_alloc(c, (size_t)s->S * 4);
  c->learned_tout = F((long long)s->nint * s->box.V);
  if (!s->P || !s->G || !s->m || !s->v || !s->Pb || !s->x0 || !s->z1 || !s->z2 || !s->y || !s->g2 || !s->g1 ||
      !s->gy || !s->sc || !s->rho || !s->loss || !s->cc || !s->e || !s->r || !s->x || !s->t || !s->delta ||
      !s->diag || !s->diag_all || !c->learned_tout || !s->bids)
    return lor_fail(c, LOR_ENOMEM, "alloc learned-correction buffers");
  if (s->nint > 0) {
    k_lrn_diag<<<s->nint, 128, 0, c->stream>>>(s->box, s->ids, c->d_S32[0], s->diag_all);
    ++c->launches;
  }
  return lor_cuda_check(c, cudaGetLastError(), "learned init");
}

// forward of S patches: t, diag -> y (and the cache)
static void forward(lor_ctx* c, int S, const float* t, const float* diag) {
  LearnState* s = LS(c);
  const PBox& b = s->box;
  const dim3 grid((unsigned)lor_ceil_div(b.V, 256), S);
  k_lrn_feat<<<S, 256, 0, c->stream>>>(b.V, t, diag, s->x0, s->sc, s->rho);
  k_lrn_conv<2, CH, false><<<grid, 256, 0, c->stream>>>(b, s->Pb + OFF_W1, s->P + OFF_B1, s->x0, s->z1);
  k_lrn_conv<CH, CH, true><<<grid, 256, 0, c->stream>>>(b, s->Pb + OFF_W2, s->P + OFF_B2, s->z1, s->z2);
  k_lrn_conv<CH, 1, true><<<grid, 256, 0, c->stream>>>(b, s->Pb + OFF_W3, s->P + OFF_B3, s->z2, s->y);
  c->launches += 4;
}

// gradients of the mean loss of S patches into s->G (zeroed here)
static void backward(lor_ctx* c, int S, const int* ids, const float* t, const float* delta) {
  LearnState* s = LS(c);
  const PBox& b = s->box;
  const dim3 grid((unsigned)lor_ceil_div(b.V, 256), S);
  k_lrn_out<<<grid, 256, 0, c->stream>>>(b, ids, s->y, s->sc, s->rho, s->cc, nullptr);
  k_lrn_loss<<<S, 256, b.V * sizeof(float), c->stream>>>(b, ids, c->d_S32[0], delta, t, s->cc, s->sc, s->rho, s->gy,
                                                          s->loss);
  cudaMemsetAsync(s->G, 0, NPARAM * 4, c->stream);
  k_lrn_bwd_w<CH, 1, true><<<S, 256, 0, c->stream>>>(b, s->gy, s->z2, s->G + OFF_W3, s->G + OFF_B3);
  k_lrn_bwd_data<CH, 1><<<grid, 256, 0, c->stream>>>(b, s->Pb + OFF_W3, s->gy, s->z2, s->g2);
  k_lrn_bwd_w<CH, CH, true><<<S, 256, 0, c->stream>>>(b, s->g2, s->z1, s->G + OFF_W2, s->G + OFF_B2);
  k_lrn_bwd_data<CH, CH><<<grid, 256, 0, c->stream>>>(b, s->Pb + OFF_W2, s->g2, s->z1, s->g1);
  k_lrn_bwd_w<2, CH, false><<<S, 256, 0, c->stream>>>(b, s->g1, s->x0, s->G + OFF_W1, s->G + OFF_B1);
  c->launches += 7;
}

lor_status lor_learned_apply(lor_ctx* c, float* z) {
  LearnState* s = LS(c);
  const PBox& b = s->box;
  for (int k0 = 0; k0 < s->nint; k0 += s->S) {
    const int S = std::min(s->S, s->nint - k0);
    const float* t = c->learned_tout + (long long)k0 * b.V;
    forward(c, S, t, s->diag_all + (long long)k0 * b.V);
    const dim3 grid((unsigned)lor_ceil_div(b.V, 256), S);
    k_lrn_out<<<grid, 256, 0, c->stream>>>(b, s->ids + k0, s->y, s->sc, s->rho, nullptr, z);
    ++c->launches;
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
  lor_status st = learned_init(c);
  if (st) return st;
  c->learned_on = on != 0 && LS(c)->nint > 0;
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
    k_lrn_out<<<grid, 256, 0, c->stream>>>(b, d_ids, s->y, s->sc, s->rho, s->cc, nullptr);
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
