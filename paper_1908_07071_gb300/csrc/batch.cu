// Batched serving: many independent LOR-preconditioned solves of uneven mesh
// size and degree advanced together.
//
// Each solve keeps its own context (operator, LOR factors, Krylov vectors).  One
// iteration of flexible CG (Polak-Ribiere beta; Notay, SIAM J. Sci. Comput.
// 22(4), 2000) for ALL solves is captured once into a CUDA graph: every solve
// runs on its own branch (forked stream), so the GPU executes the branches
// concurrently, and the whole iteration is one graph launch.  Vectors and inner
// products are FP64; the preconditioner runs in FP32 (bf16/fp32 factors).  All
// scalars live on the device; a solve whose residual reaches rtol sets a
// converged flag that freezes it (alpha = 0) and makes its patch kernel exit at
// once.  The host reads the converged flags after each launch.
// Before the first solve, apply_A's tile shape (elements per CTA) is chosen per
// polynomial degree by timing the three compiled variants (autotuner).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lor_internal.h"

namespace {

enum { B_RZ = 0, B_PAP = 1, B_RR = 2, B_ALPHA = 4, B_BETA = 5, B_BB = 6, B_FLAG = 7, B_CONV = 9, B_TOL2 = 10,
       B_ITERS = 11, B_RZN = 12 };
enum { F_STORE_RR = 0, F_ALPHA = 1, F_UPDATE = 2, F_BETA = 3, F_RZ = 4 };

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Two-stage deterministic reduction of (v0, v1); the last block applies `op`.
__device__ void finish2(double v0, double v1, double* part, unsigned* count, double* scal, int op) {
  __shared__ double sh0[32], sh1[32];
  __shared__ bool last;
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh0[w] = v0; sh1[w] = v1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += sh0[k]; b += sh1[k]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
    __threadfence();
    last = atomicInc(count, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double a = 0, b = 0;
  for (int k = 0; k < (int)gridDim.x; ++k) {
    a += ((volatile double*)part)[2 * k];
    b += ((volatile double*)part)[2 * k + 1];
  }
  const bool conv = scal[B_CONV] != 0.0;
  if (op == F_STORE_RR) {
    scal[B_RR] = a;
  } else if (op == F_ALPHA) {              // a = p.Ap
    scal[B_PAP] = a;
    if (!conv && !(a > 0.0)) { scal[B_FLAG] = 1.0; scal[B_CONV] = 1.0; }
    scal[B_ALPHA] = (conv || !(a > 0.0)) ? 0.0 : scal[B_RZ] / a;
  } else if (op == F_UPDATE) {             // a = r.r after the update
    scal[B_RR] = a;
    if (!conv) scal[B_ITERS] += 1.0;
    if (a <= scal[B_TOL2]) scal[B_CONV] = 1.0;
  } else if (op == F_BETA) {               // a = r.z_new, b = r.z_old
    scal[B_BETA] = conv ? 0.0 : (a - b) / scal[B_RZ];
    scal[B_RZ] = a;
  } else {                                 // F_RZ: a = r.z
    scal[B_RZ] = a;
  }
}

const int kRB = 1024, kRT = 256;

unsigned rblocks(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>(kRB, lor_ceil_div(n, kRT * 4)));
}

#define GRID_STRIDE(i, n) for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

__global__ void __launch_bounds__(256) k_b_init(double* x, double* r, const double* b, const unsigned char* bm,
                                                long long n, double* part, unsigned* count, double* scal) {
  double s = 0;
  GRID_STRIDE(i, n) {
    const double v = bm[i] ? 0.0 : b[i];
    r[i] = v;
    x[i] = 0.0;
    s += v * v;
  }
  finish2(s, 0.0, part, count, scal, F_STORE_RR);
}

__global__ void k_b_setconv(double* scal, double rtol) {
  scal[B_BB] = scal[B_RR];
  scal[B_TOL2] = rtol * rtol * scal[B_RR];
  scal[B_CONV] = scal[B_RR] == 0.0 ? 1.0 : 0.0;
  scal[B_ITERS] = 0.0;
  scal[B_FLAG] = 0.0;
}

// Every kernel of the captured iteration skips its vector work once the solve has
// converged (scal[B_CONV] != 0, set at the end of the update that reached rtol);
// the reductions still finish, with zero sums, so the scalars stay frozen.
__global__ void __launch_bounds__(256) k_b_dot(const double* a, const double* b, long long n, double* part,
                                               unsigned* count, double* scal, int op) {
  double s = 0;
  if (scal[B_CONV] == 0.0) GRID_STRIDE(i, n) s += a[i] * b[i];
  finish2(s, 0.0, part, count, scal, op);
}

__global__ void __launch_bounds__(256) k_b_update(double* x, double* r, const double* p, const double* Ap,
                                                  long long n, double* part, unsigned* count, double* scal) {
  const double al = scal[B_ALPHA];
  double s = 0;
  if (scal[B_CONV] == 0.0) GRID_STRIDE(i, n) {
    x[i] += al * p[i];
    const double ri = r[i] - al * Ap[i];
    r[i] = ri;
    s += ri * ri;
  }
  finish2(s, 0.0, part, count, scal, F_UPDATE);
}

__global__ void k_b_down(float* d, const double* s, long long n, const double* scal) {
  if (scal && scal[B_CONV] != 0.0) return;
  GRID_STRIDE(i, n) d[i] = (float)s[i];
}

// z_new = (double) z32; dots r.z_new and r.z_old; z = z_new
__global__ void __launch_bounds__(256) k_b_up_dots(double* z, const float* z32, const double* r, long long n,
                                                   double* part, unsigned* count, double* scal, int op) {
  double a = 0, b = 0;
  if (scal[B_CONV] == 0.0) GRID_STRIDE(i, n) {
    const double zn = (double)z32[i];
    a += r[i] * zn;
    b += r[i] * z[i];
    z[i] = zn;
  }
  finish2(a, b, part, count, scal, op);
}

__global__ void k_b_xpay(double* p, const double* z, long long n, const double* scal, int copy) {
  if (!copy && scal[B_CONV] != 0.0) return;
  const double be = copy ? 0.0 : scal[B_BETA];
  GRID_STRIDE(i, n) p[i] = z[i] + be * p[i];
}

__global__ void k_b_gather(double* const* scals, int n, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) {
    out[2 * s] = scals[s][B_CONV];
    out[2 * s + 1] = scals[s][B_FLAG];
  }
}

__global__ void __launch_bounds__(256) k_b_resid(const double* b, const double* Ax, const unsigned char* bm,
                                                 long long n, double* part, unsigned* count, double* scal) {
  double s = 0;
  GRID_STRIDE(i, n) {
    const double v = bm[i] ? 0.0 : b[i] - Ax[i];
    s += v * v;
  }
  finish2(s, 0.0, part, count, scal, F_STORE_RR);
}

}  // namespace

struct lor_batch {
  int n = 0;
  std::vector<lor_ctx*> c;
  cudaStream_t main = nullptr;
  std::vector<cudaStream_t> st;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<double*> xs;
  double** d_scals = nullptr;
  double* d_flags = nullptr;
  double* h_flags = nullptr;
  std::string err;
  double graph_ms = 0;
  int graph_nodes = 0;
};

static double* scal_of(lor_ctx* c) { return c->d_scal; }
static unsigned char* bmask(lor_ctx* c) { return (unsigned char*)c->d_v32[7]; }

// one FCG iteration of solve s on stream st (captured)
static lor_status enqueue_iteration(lor_ctx* c, double* x, cudaStream_t st) {
  const cudaStream_t keep = c->stream;
  c->stream = st;
  const long long n = c->nv;
  double *r = c->d_v64[0], *z = c->d_v64[1], *p = c->d_v64[2], *Ap = c->d_v64[3];
  float *r32 = c->d_v32[1], *z32 = c->d_v32[2];
  double* sc = scal_of(c);
  c->conv_flag = sc + B_CONV;   // a converged solve's operator kernels return at once
  lor_status s = lor_opA64(c, p, Ap);
  if (!s) {
    k_b_dot<<<rblocks(n), kRT, 0, st>>>(p, Ap, n, c->d_part, c->d_count, sc, F_ALPHA);
    k_b_update<<<rblocks(n), kRT, 0, st>>>(x, r, p, Ap, n, c->d_part, c->d_count, sc);
    k_b_down<<<rblocks(n), kRT, 0, st>>>(r32, r, n, sc);
    c->launches += 3;
    s = lor_opP32(c, r32, z32);
  }
  c->conv_flag = nullptr;
  if (!s) {
    k_b_up_dots<<<rblocks(n), kRT, 0, st>>>(z, z32, r, n, c->d_part, c->d_count, sc, F_BETA);
    k_b_xpay<<<rblocks(n), kRT, 0, st>>>(p, z, n, sc, 0);
    c->launches += 2;
  }
  c->stream = keep;
  return s;
}

static lor_status tune(lor_batch* b) {
  // autotuner: per degree, time the three tile variants of apply_A on one solve
  for (int p = 1; p <= LOR_MAXP; ++p) {
    lor_ctx* rep = nullptr;
    for (lor_ctx* c : b->c)
      if (c->p == p && c->dim == 3 && (!rep || c->nel > rep->nel)) rep = c;
    if (!rep) continue;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double* x = rep->d_v64[2];
    double* y = rep->d_v64[3];
    float best = 1e30f;
    int bestv = 1;
    for (int v = 0; v < 3; ++v) {
      rep->tune_ne = v;
      lor_opA64(rep, x, y);
      cudaEventRecord(e0, rep->stream);
      for (int k = 0; k < 5; ++k) lor_opA64(rep, x, y);
      cudaEventRecord(e1, rep->stream);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bestv = v; }
    }
    for (lor_ctx* c : b->c)
      if (c->p == p) c->tune_ne = bestv;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  return cudaGetLastError() == cudaSuccess ? LOR_OK : LOR_ECUDA;
}

extern "C" {

lor_status lor_batch_create(lor_batch** out, int n, lor_ctx** ctxs, void* stream) {
  if (!out || n < 1 || !ctxs) return LOR_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i] || !ctxs[i]->setup_done || ctxs[i]->dg_state) return LOR_EINVAL;
  for (int i = 0; i < n; ++i) ctxs[i]->pcg_state_ok = false;   // the batch reuses their Krylov vectors
  lor_batch* b = new lor_batch();
  b->n = n;
  b->c.assign(ctxs, ctxs + n);
  b->main = (cudaStream_t)stream;
  b->st.resize(n);
  b->join.resize(n);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < n && ok; ++i) {
    ok = cudaStreamCreateWithFlags(&b->st[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
  }
  std::vector<double*> sc(n);
  for (int i = 0; i < n; ++i) sc[i] = scal_of(ctxs[i]);
  ok = ok && cudaMalloc(&b->d_scals, n * sizeof(double*)) == cudaSuccess &&
       cudaMalloc(&b->d_flags, 2 * n * sizeof(double)) == cudaSuccess &&
       cudaMallocHost(&b->h_flags, 2 * n * sizeof(double)) == cudaSuccess;
  if (ok) ok = cudaMemcpy(b->d_scals, sc.data(), n * sizeof(double*), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    lor_batch_destroy(b);
    return LOR_ECUDA;
  }
  if (tune(b) != LOR_OK) {
    lor_batch_destroy(b);
    return LOR_ECUDA;
  }
  *out = b;
  return LOR_OK;
}

lor_status lor_batch_solve(lor_batch* b, const double* const* d_b, double* const* d_x, int* iters,
                           double* rel_res) {
  if (!b || !d_b || !d_x) return LOR_EINVAL;
  const int n = b->n;
  for (lor_ctx* c : b->c) c->pcg_state_ok = false;   // the batch reuses their Krylov vectors
  // per-solve start: r = b, x = 0, z = P r, p = z (on the main stream)
  for (int s = 0; s < n; ++s) {
    lor_ctx* c = b->c[s];
    const cudaStream_t keep = c->stream;
    c->stream = b->main;
    const long long nv = c->nv;
    double *r = c->d_v64[0], *z = c->d_v64[1], *p = c->d_v64[2];
    float *r32 = c->d_v32[1], *z32 = c->d_v32[2];
    double* sc = scal_of(c);
    cudaMemsetAsync(sc, 0, 16 * 8, b->main);
    k_b_init<<<rblocks(nv), kRT, 0, b->main>>>(d_x[s], r, d_b[s], bmask(c), nv, c->d_part, c->d_count, sc);
    k_b_setconv<<<1, 1, 0, b->main>>>(sc, c->opt.rtol);
    k_b_down<<<rblocks(nv), kRT, 0, b->main>>>(r32, r, nv, nullptr);
    lor_status st = lor_opP32(c, r32, z32);
    cudaMemsetAsync(z, 0, nv * 8, b->main);
    k_b_up_dots<<<rblocks(nv), kRT, 0, b->main>>>(z, z32, r, nv, c->d_part, c->d_count, sc, F_RZ);
    k_b_xpay<<<rblocks(nv), kRT, 0, b->main>>>(p, z, nv, sc, 1);
    c->launches += 5;
    c->stream = keep;
    if (st) return st;
  }
  // capture one iteration of every solve into a graph (once per set of x pointers)
  bool recapture = !b->exec || b->xs.size() != (size_t)n;
  for (int s = 0; s < n && !recapture; ++s) recapture = b->xs[s] != d_x[s];
  if (recapture) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->xs.assign(d_x, d_x + n);
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return LOR_ECUDA;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaStreamDestroy(cs);
      return LOR_ECUDA;
    }
    cudaEventRecord(b->fork, cs);
    lor_status st = LOR_OK;
    for (int s = 0; s < n && !st; ++s) {
      cudaStreamWaitEvent(b->st[s], b->fork, 0);
      st = enqueue_iteration(b->c[s], d_x[s], b->st[s]);
      cudaEventRecord(b->join[s], b->st[s]);
      cudaStreamWaitEvent(cs, b->join[s], 0);
    }
    k_b_gather<<<(unsigned)lor_ceil_div(n, 128), 128, 0, cs>>>(b->d_scals, n, b->d_flags);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) { cudaGetLastError(); b->err = cudaGetErrorString(e); }
      return st ? st : LOR_ECUDA;
    }
    b->graph = g;
    size_t nodes = 0;
    cudaGraphGetNodes(g, nullptr, &nodes);
    b->graph_nodes = (int)nodes;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) { cudaGetLastError(); return LOR_ECUDA; }
  }
  int maxit = 0;
  for (lor_ctx* c : b->c) maxit = std::max(maxit, c->opt.max_it);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, b->main);
  int it = 0;
  bool any_flag = false;
  for (; it < maxit; ++it) {
    if (cudaGraphLaunch(b->exec, b->main) != cudaSuccess ||
        cudaMemcpyAsync(b->h_flags, b->d_flags, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, b->main) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->main) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return LOR_ECUDA;
    }
    bool all = true;
    for (int s = 0; s < n; ++s) {
      all = all && b->h_flags[2 * s] != 0.0;
      any_flag = any_flag || b->h_flags[2 * s + 1] != 0.0;
    }
    if (all) break;
  }
  cudaEventRecord(e1, b->main);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  b->graph_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // per-solve iterations and FP64 relative residuals
  lor_status ret = LOR_OK;
  for (int s = 0; s < n; ++s) {
    lor_ctx* c = b->c[s];
    const cudaStream_t keep = c->stream;
    c->stream = b->main;
    double* sc = scal_of(c);
    double h[16];
    cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, b->main);
    cudaStreamSynchronize(b->main);
    const double bb = h[B_BB];
    const long long nv = c->nv;
    lor_opA64(c, d_x[s], c->d_v64[3]);
    k_b_resid<<<rblocks(nv), kRT, 0, b->main>>>(d_b[s], c->d_v64[3], bmask(c), nv, c->d_part, c->d_count, sc);
    ++c->launches;
    double rr = 0;
    cudaMemcpyAsync(&rr, sc + B_RR, 8, cudaMemcpyDeviceToHost, b->main);
    cudaStreamSynchronize(b->main);
    const lor_status ds = lor_take_device_status(c);   // a timed-out patch V-cycle invalidates this solve
    c->stream = keep;
    if (iters) iters[s] = (int)h[B_ITERS];
    if (rel_res) rel_res[s] = bb > 0 ? sqrt(rr / bb) : 0.0;
    if (h[B_CONV] == 0.0) ret = LOR_ENOCONV;
    if (h[B_FLAG] != 0.0) ret = LOR_ENAN;
    if (ds != LOR_OK) ret = ds;
  }
  (void)any_flag;
  return ret;
}

lor_status lor_batch_stats(const lor_batch* b, double* loop_ms, int* graph_nodes) {
  if (!b) return LOR_EINVAL;
  if (loop_ms) *loop_ms = b->graph_ms;
  if (graph_nodes) *graph_nodes = b->graph_nodes;
  return LOR_OK;
}

void lor_batch_destroy(lor_batch* b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  else cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->st)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_scals) cudaFree(b->d_scals);
  if (b->d_flags) cudaFree(b->d_flags);
  if (b->h_flags) cudaFreeHost(b->h_flags);
  delete b;
}

}  // extern "C"
