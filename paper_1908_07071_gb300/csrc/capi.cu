// C ABI of the LOR solver (declared in include/lor.h).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "lor_internal.h"

lor_status lor_fail(lor_ctx* c, lor_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

lor_status lor_cuda_check(lor_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LOR_OK;
  return lor_fail(c, e == cudaErrorMemoryAllocation ? LOR_ENOMEM : LOR_ECUDA,
                  std::string(what) + ": " + cudaGetErrorString(e));
}

void* lor_alloc(lor_ctx* c, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (cudaMemsetAsync(p, 0, bytes, c->stream) != cudaSuccess) {
    cudaFree(p);
    return nullptr;
  }
  c->allocs.push_back(p);
  c->bytes += bytes;
  return p;
}

static const int kMaxProf = 8192;

void lor_prof_begin(lor_ctx* c, int k) {
  if (!c->prof || c->nev[k] >= kMaxProf) return;
  std::vector<cudaEvent_t>& v = c->ev[k];
  const int i = c->nev[k];
  while ((int)v.size() < 2 * (i + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    v.push_back(e);
  }
  cudaEventRecord(v[2 * i], c->stream);
}

void lor_prof_end(lor_ctx* c, int k) {
  if (!c->prof || c->nev[k] >= kMaxProf) return;
  if ((int)c->ev[k].size() < 2 * (c->nev[k] + 1)) return;
  cudaEventRecord(c->ev[k][2 * c->nev[k] + 1], c->stream);
  c->nev[k]++;
}

lor_status lor_opA64(lor_ctx* c, const double* x, double* y) {
  return c->dg_state ? lor_launch_apply_A_dg64(c, x, y) : lor_launch_apply_A64(c, x, y);
}
lor_status lor_opA32(lor_ctx* c, const float* x, float* y) {
  return c->dg_state ? lor_launch_apply_A_dg32(c, x, y) : lor_launch_apply_A32(c, x, y);
}
lor_status lor_opP64(lor_ctx* c, const double* r, double* z) {
  return c->dg_state ? lor_launch_apply_P_dg64(c, r, z) : lor_launch_apply_P64(c, r, z);
}
lor_status lor_opP32(lor_ctx* c, const float* r, float* z) {
  return c->dg_state ? lor_launch_apply_P_dg32(c, r, z) : lor_launch_apply_P32(c, r, z);
}

lor_status lor_take_device_status(lor_ctx* c) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "device status");
  if (st & 4) {
    e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return lor_cuda_check(c, e, "device status reset");
    return lor_fail(c, LOR_ETIMEOUT, "a bounded device wait ran out (factor bulk copy not completed)");
  }
  return LOR_OK;
}

extern "C" {

lor_status lor_profile(lor_ctx* c, int on) {
  if (!c) return LOR_EINVAL;
  c->prof = on != 0;
  if (on)
    for (int k = 0; k < 6; ++k) c->nev[k] = 0;
  return LOR_OK;
}

lor_status lor_profile_read(lor_ctx* c, int kernel, double* total_ms, long long* launches) {
  if (!c || kernel < 0 || kernel >= 6 || !total_ms || !launches) return LOR_EINVAL;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "profile read");
  double tot = 0;
  for (int i = 0; i < c->nev[kernel]; ++i) {
    float ms = 0;
    e = cudaEventElapsedTime(&ms, c->ev[kernel][2 * i], c->ev[kernel][2 * i + 1]);
    if (e != cudaSuccess) return lor_cuda_check(c, e, "event elapsed");
    tot += ms;
  }
  *total_ms = tot;
  *launches = c->nev[kernel];
  return LOR_OK;
}

void lor_default_options(lor_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->dim = 3;
  o->p = 4;
  o->nx = o->ny = o->nz = 8;
  o->disc = LOR_CG;
  o->eta = 1.0;
  o->mg_levels = 0;
  o->prec = LOR_FP64;
  o->rtol = 1e-8;
  o->max_it = 1000;
  o->inner_rtol = 1e-3;
  o->factor_bf16 = 0;
  o->weighting = 0;
}

// Copies n doubles at src into dst: through the copy engine when the CUDA runtime
// reports src as device or managed memory, else (host memory, or no device at
// all) directly.  False if a device copy fails.
static bool read_mesh_array(const double* src, size_t n, std::vector<double>& dst, cudaStream_t st) {
  dst.resize(n);
  cudaPointerAttributes at;
  const cudaError_t e = cudaPointerGetAttributes(&at, src);
  if (e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
    if (cudaMemcpyAsync(dst.data(), src, n * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  }
  if (e != cudaSuccess) cudaGetLastError();   // no device, or memory the runtime does not track
  std::copy(src, src + n, dst.begin());
  return true;
}

lor_status lor_create(lor_ctx** out, const lor_options* opt, const double* vertices, const double* kappa,
                      void* stream) {
  if (!out || !opt || !vertices || !kappa) return LOR_EINVAL;
  *out = nullptr;
  if (opt->dim != 2 && opt->dim != 3) return LOR_EINVAL;
  if (opt->p < 1 || opt->p > LOR_MAXP) return LOR_EINVAL;
  if (opt->nx < 1 || opt->ny < 1 || (opt->dim == 3 && opt->nz < 1)) return LOR_EINVAL;
  if (opt->disc != LOR_CG && opt->disc != LOR_DG_IP && opt->disc != LOR_DG_BR2) return LOR_EINVAL;
  if (opt->disc != LOR_CG && (opt->dim != 3 || !(opt->eta > 0))) return LOR_EINVAL;
  if (!(opt->rtol > 0) || opt->max_it < 1) return LOR_EINVAL;
  if (opt->weighting < 0 || opt->weighting > 2) return LOR_EINVAL;
  // element and vertex counts are ints in the kernels' index arithmetic
  const long long nel_ll = (long long)opt->nx * opt->ny * (opt->dim == 3 ? opt->nz : 1);
  const long long nv_ll = (long long)(opt->nx + 1) * (opt->ny + 1) * (opt->dim == 3 ? opt->nz + 1 : 1);
  if (nel_ll > INT_MAX || nv_ll * opt->dim > INT_MAX) return LOR_EINVAL;
  lor_ctx* c = new (std::nothrow) lor_ctx();
  if (!c) return LOR_ENOMEM;
  c->opt = *opt;
  c->dim = opt->dim;
  c->p = opt->p;
  c->n[0] = opt->nx;
  c->n[1] = opt->ny;
  c->n[2] = opt->dim == 3 ? opt->nz : 1;
  c->nel = c->n[0] * c->n[1] * c->n[2];
  c->stream = (cudaStream_t)stream;
  try {
    if (!read_mesh_array(vertices, (size_t)nv_ll * c->dim, c->h_vert, c->stream) ||
        !read_mesh_array(kappa, (size_t)c->nel, c->h_kappa, c->stream)) {
      delete c;
      return LOR_ECUDA;
    }
  } catch (const std::bad_alloc&) {
    delete c;
    return LOR_ENOMEM;
  }
  for (double k : c->h_kappa)
    if (!(k > 0) || !std::isfinite(k)) {
      delete c;
      return LOR_EINVAL;
    }
  for (double v : c->h_vert)
    if (!std::isfinite(v)) {
      delete c;
      return LOR_EINVAL;
    }
  *out = c;
  return LOR_OK;
}

lor_status lor_setup(lor_ctx* c) {
  if (!c) return LOR_EINVAL;
  if (c->setup_done) return lor_fail(c, LOR_ESTATE, "lor_setup called twice");
  if (c->setup_started)
    return lor_fail(c, LOR_ESTATE, "an earlier lor_setup failed; destroy the context and create a new one");
  c->setup_started = true;
  lor_status s;
  if ((s = lor_setup_geometry(c))) return s;
  if ((s = lor_setup_stencils(c))) return s;
  if ((s = lor_setup_patches(c))) return s;
  if ((s = lor_setup_coarse(c))) return s;
  c->nv = c->lev[0].ntot;
  if (c->opt.disc != LOR_CG) {
    if ((s = lor_setup_dg(c))) return s;
    c->nv = (long long)c->nel * (c->p + 1) * (c->p + 1) * (c->p + 1);
  }
  if ((s = lor_setup_krylov(c))) return s;
  if ((s = lor_patch_prepare(c))) return s;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "setup");
  c->setup_done = true;
  return LOR_OK;
}

lor_status lor_get_info(const lor_ctx* c, lor_info* info) {
  if (!c || !info) return LOR_EINVAL;
  std::memset(info, 0, sizeof(*info));
  long long nvec = 1, ndof = 1;
  for (int a = 0; a < c->dim; ++a) {
    nvec *= (long long)c->n[a] * c->p + 1;
    ndof *= (long long)c->n[a] * c->p - 1;
  }
  info->nvec = nvec;
  info->ndof = ndof;
  if (c->opt.disc != LOR_CG) {
    long long q = 1;
    for (int a = 0; a < c->dim; ++a) q *= c->p + 1;
    info->nvec = info->ndof = (long long)c->nel * q;
  }
  long long J = 1, nc = 1;
  for (int a = 0; a < c->dim; ++a) { J *= c->n[a] + 1; nc *= c->n[a] - 1; }
  info->npatch = J;
  info->ncoarse = nc;
  info->levels = c->L;
  info->coarse_levels = c->CL;
  info->factor_rows = c->fac_rows;
  info->device_bytes = c->bytes;
  return LOR_OK;
}

static lor_status ready(lor_ctx* c) {
  if (!c) return LOR_EINVAL;
  if (!c->setup_done) return lor_fail(c, LOR_ESTATE, "lor_setup has not completed");
  return LOR_OK;
}

lor_status lor_rhs(lor_ctx* c, int kind, double* d_b) {
  lor_status s = ready(c);
  if (s) return s;
  if (!d_b || kind < 0 || kind > 1) return lor_fail(c, LOR_EINVAL, "lor_rhs: bad argument");
  return lor_launch_rhs(c, kind, d_b);
}

lor_status lor_quadrature_points(const lor_ctx* c, double* xq) {
  if (!c || !xq) return LOR_EINVAL;
  lor_quad_points(c, xq);
  return LOR_OK;
}

lor_status lor_rhs_f(lor_ctx* c, const double* d_fq, double* d_b) {
  lor_status s = ready(c);
  if (s) return s;
  if (!d_fq || !d_b) return lor_fail(c, LOR_EINVAL, "lor_rhs_f: null vector");
  return lor_launch_rhs(c, 0, d_b, d_fq);
}

lor_status lor_apply_A(lor_ctx* c, const void* x, void* y, int prec) {
  lor_status s = ready(c);
  if (s) return s;
  if (!x || !y) return lor_fail(c, LOR_EINVAL, "lor_apply_A: null vector");
  if (prec == LOR_FP64) return lor_opA64(c, (const double*)x, (double*)y);
  if (prec == LOR_FP32) return lor_opA32(c, (const float*)x, (float*)y);
  return lor_fail(c, LOR_EINVAL, "lor_apply_A: prec must be LOR_FP64 or LOR_FP32");
}

lor_status lor_apply_P(lor_ctx* c, const void* r, void* z, int prec) {
  lor_status s = ready(c);
  if (s) return s;
  if (!r || !z) return lor_fail(c, LOR_EINVAL, "lor_apply_P: null vector");
  if (prec == LOR_FP64) return lor_opP64(c, (const double*)r, (double*)z);
  if (prec == LOR_FP32) return lor_opP32(c, (const float*)r, (float*)z);
  return lor_fail(c, LOR_EINVAL, "lor_apply_P: prec must be LOR_FP64 or LOR_FP32");
}

lor_status lor_device_status(lor_ctx* c) {
  lor_status s = ready(c);
  if (s) return s;
  return lor_take_device_status(c);
}

lor_status lor_selftest_wait(lor_ctx* c, int polls) {
  lor_status s = ready(c);
  if (s) return s;
  if (polls < 1 || polls > (1 << 24)) return lor_fail(c, LOR_EINVAL, "lor_selftest_wait: polls in [1, 2^24]");
  if ((s = lor_launch_wait_selftest(c, polls))) return s;
  return lor_take_device_status(c);
}

lor_status lor_pcg_solve(lor_ctx* c, const double* b, double* x, int* iters, double* rel_res) {
  lor_status s = ready(c);
  if (s) return s;
  if (!b || !x) return lor_fail(c, LOR_EINVAL, "lor_pcg_solve: null vector");
  c->pcg_state_ok = false;   // an FP64 solve leaves a new resumable state
  s = c->opt.prec == LOR_MIXED ? lor_pcg_mixed(c, b, x, iters, rel_res) : lor_pcg64(c, b, x, iters, rel_res);
  if (s != LOR_OK && s != LOR_ENOCONV) return s;
  const lor_status d = lor_take_device_status(c);   // a timed-out patch V-cycle invalidates the result
  return d != LOR_OK ? d : s;
}

lor_status lor_pcg_state_size(const lor_ctx* c, size_t* bytes) {
  if (!c || !bytes) return LOR_EINVAL;
  if (!c->setup_done) return LOR_ESTATE;
  *bytes = lor_pcg_state_bytes(c);
  return LOR_OK;
}

lor_status lor_pcg_state_save(lor_ctx* c, const double* d_x, void* host, size_t bytes) {
  lor_status s = ready(c);
  if (s) return s;
  if (!d_x || !host) return lor_fail(c, LOR_EINVAL, "lor_pcg_state_save: null pointer");
  return lor_pcg_save(c, d_x, host, bytes);
}

lor_status lor_pcg_resume(lor_ctx* c, const void* host, size_t bytes, const double* d_b, double* d_x, int* iters,
                          double* rel_res) {
  lor_status s = ready(c);
  if (s) return s;
  if (!host || !d_b || !d_x) return lor_fail(c, LOR_EINVAL, "lor_pcg_resume: null pointer");
  c->pcg_state_ok = false;
  s = lor_pcg_resume_impl(c, host, bytes, d_b, d_x, iters, rel_res);
  if (s != LOR_OK && s != LOR_ENOCONV) return s;
  const lor_status d = lor_take_device_status(c);
  return d != LOR_OK ? d : s;
}

lor_status lor_pcg_solve_host(lor_ctx* c, const double* hb, double* hx, int* iters, double* rel_res) {
  lor_status s = ready(c);
  if (s) return s;
  if (!hb || !hx) return lor_fail(c, LOR_EINVAL, "lor_pcg_solve_host: null vector");
  const long long n = c->nv;
  double* db = c->d_v64[5];
  double* dx = c->d_v64[6];
  cudaError_t e = cudaMemcpyAsync(db, hb, n * 8, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "copy b");
  s = lor_pcg_solve(c, db, dx, iters, rel_res);
  if (s != LOR_OK && s != LOR_ENOCONV) return s;
  e = cudaMemcpyAsync(hx, dx, n * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "copy x");
  return s;
}

lor_status lor_coefficient_sizes(const lor_ctx* c, long long* nq, long long* nh) {
  if (!c || !nq || !nh) return LOR_EINVAL;
  lor_coef_sizes(c, nq, nh);
  return LOR_OK;
}

lor_status lor_coefficient_points(const lor_ctx* c, double* xq, double* xh) {
  if (!c) return LOR_EINVAL;
  lor_coef_points(c, xq, xh);
  return LOR_OK;
}

lor_status lor_set_coefficient(lor_ctx* c, const double* bq, const double* bh) {
  if (!c) return LOR_EINVAL;
  if (c->setup_started) return lor_fail(c, LOR_ESTATE, "lor_set_coefficient must precede lor_setup");
  if (c->opt.disc != LOR_CG)
    return lor_fail(c, LOR_EINVAL, "pointwise coefficients: CG only (the DG penalty takes kappa per element)");
  if (!bq || !bh) return lor_fail(c, LOR_EINVAL, "lor_set_coefficient: null array");
  if (!c->h_nodes.empty())
    return lor_fail(c, LOR_EINVAL, "pointwise coefficients are sampled on multilinear elements, not curved ones");
  long long nq = 0, nh = 0;
  lor_coef_sizes(c, &nq, &nh);
  try {
    c->h_bq.assign(bq, bq + nq);
    c->h_bh.assign(bh, bh + nh);
  } catch (const std::bad_alloc&) {
    c->h_bq.clear();
    c->h_bh.clear();
    return lor_fail(c, LOR_ENOMEM, "lor_set_coefficient: host copy");
  }
  for (const std::vector<double>* v : {&c->h_bq, &c->h_bh})
    for (double x : *v)
      if (!(x > 0) || !std::isfinite(x)) {
        c->h_bq.clear();
        c->h_bh.clear();
        return lor_fail(c, LOR_EINVAL, "lor_set_coefficient: values must be positive and finite");
      }
  return LOR_OK;
}

lor_status lor_set_ordering(lor_ctx* c, int ordering) {
  if (!c) return LOR_EINVAL;
  if (c->setup_started) return lor_fail(c, LOR_ESTATE, "lor_set_ordering must precede lor_setup");
  if (ordering < 0 || ordering > 2) return lor_fail(c, LOR_EINVAL, "lor_set_ordering: 0 (lexicographic), 1 (RCM) or 2 (MDF)");
  c->ordering = ordering;
  c->gen = c->ordering != 0 || !c->h_spans.empty();
  return LOR_OK;
}

lor_status lor_set_patch_spans(lor_ctx* c, const int* spans) {
  if (!c) return LOR_EINVAL;
  if (c->setup_started) return lor_fail(c, LOR_ESTATE, "lor_set_patch_spans must precede lor_setup");
  if (c->opt.disc != LOR_CG) return lor_fail(c, LOR_EINVAL, "enlarged patches: CG only");
  if (c->opt.weighting) return lor_fail(c, LOR_EINVAL, "enlarged patches take unit patch weights");
  if (!spans) {
    c->h_spans.clear();
  } else {
    long long J = 1;
    for (int a = 0; a < c->dim; ++a) J *= c->n[a] + 1;
    for (long long q = 0; q < J * c->dim * 2; ++q)
      if (spans[q] < 1 || spans[q] > LOR_MAXSPAN) return lor_fail(c, LOR_EINVAL, "patch span out of range");
    c->h_spans.assign(spans, spans + J * c->dim * 2);
  }
  c->gen = c->ordering != 0 || !c->h_spans.empty();
  return LOR_OK;
}

lor_status lor_box_ordering(int dim, int A, int B, int C, int ordering, const double* a27, int* perm) {
  if ((dim != 2 && dim != 3) || A < 1 || B < 1 || C < 1 || (dim == 2 && C != 1) || !perm) return LOR_EINVAL;
  if (ordering < 0 || ordering > 2 || (ordering == 2 && !a27)) return LOR_EINVAL;
  const long long n = (long long)A * B * C;
  if (n > (1 << 20)) return LOR_EINVAL;
  std::vector<int> out;
  try {
    if (ordering == 0) {
      out.resize(n);
      for (long long q = 0; q < n; ++q) out[q] = (int)q;
    } else if (ordering == 1) {
      lorh::rcm_box(dim, A, B, C, out);
    } else {
      const int NS = dim == 3 ? 27 : 9;
      std::vector<double> a(a27, a27 + n * NS);
      if (!lorh::mdf_box(dim, A, B, C, a, out)) return LOR_EBREAKDOWN;
    }
  } catch (const std::bad_alloc&) {
    return LOR_ENOMEM;
  }
  for (long long q = 0; q < n; ++q) perm[q] = out[q];
  return LOR_OK;
}

lor_status lor_box_ilu0(int dim, int A, int B, int C, const double* a27, const int* perm, double* lu, int* level) {
  if ((dim != 2 && dim != 3) || A < 1 || B < 1 || C < 1 || (dim == 2 && C != 1) || !a27 || !perm || !lu)
    return LOR_EINVAL;
  const long long n = (long long)A * B * C;
  if (n > (1 << 20)) return LOR_EINVAL;
  const int NS = dim == 3 ? 27 : 9;
  try {
    std::vector<char> seen(n, 0);
    for (long long q = 0; q < n; ++q) {
      if (perm[q] < 0 || perm[q] >= n || seen[perm[q]]) return LOR_EINVAL;
      seen[perm[q]] = 1;
    }
    std::vector<double> a(a27, a27 + n * NS), out;
    std::vector<int> p(perm, perm + n), lev;
    if (!lorh::ilu0_ordered(dim, A, B, C, a, p, out, lev)) return LOR_EBREAKDOWN;
    std::copy(out.begin(), out.end(), lu);
    if (level) std::copy(lev.begin(), lev.end(), level);
  } catch (const std::bad_alloc&) {
    return LOR_ENOMEM;
  }
  return LOR_OK;
}

lor_status lor_patch_ordering(lor_ctx* c, int level, long long patch, int* perm, int cap, int* count) {
  if (!c || !count) return LOR_EINVAL;
  if (!c->setup_done) return lor_fail(c, LOR_ESTATE, "lor_patch_ordering: call lor_setup first");
  if (level < 0 || level + 1 >= c->L || patch < 0 || patch >= c->J)
    return lor_fail(c, LOR_EINVAL, "lor_patch_ordering: level or patch out of range");
  const int n0 = c->n[0] + 1, n1 = c->n[1] + 1;
  const int v[3] = {(int)(patch % n0), (int)((patch / n0) % n1), c->dim == 3 ? (int)(patch / ((long long)n0 * n1)) : 0};
  int sh = 0;
  for (int a = 0; a < c->dim; ++a) sh |= ((v[a] == 0 || v[a] == c->n[a]) ? 1 : 0) << a;
  const int rows = c->gen ? (int)c->h_perm[(size_t)level * c->J + patch].size() : c->shapes[level * 8 + sh].rows;
  *count = rows;
  if (!perm) return LOR_OK;
  if (cap < rows) return lor_fail(c, LOR_EINVAL, "lor_patch_ordering: buffer too small");
  if (!c->gen) {
    for (int q = 0; q < rows; ++q) perm[q] = q;
  } else {
    const std::vector<int>& h = c->h_perm[(size_t)level * c->J + patch];
    for (int q = 0; q < rows; ++q) perm[q] = h[q];
  }
  return LOR_OK;
}

lor_status lor_set_node_coordinates(lor_ctx* c, const double* X) {
  if (!c) return LOR_EINVAL;
  if (c->setup_started) return lor_fail(c, LOR_ESTATE, "lor_set_node_coordinates must precede lor_setup");
  if (c->opt.disc != LOR_CG) return lor_fail(c, LOR_EINVAL, "curved elements: CG only");
  if (!c->h_bq.empty()) return lor_fail(c, LOR_EINVAL, "curved elements do not combine with lor_set_coefficient");
  if (!X) return lor_fail(c, LOR_EINVAL, "lor_set_node_coordinates: null array");
  long long ntot = 1;
  for (int a = 0; a < c->dim; ++a) ntot *= (long long)c->n[a] * c->p + 1;
  try {
    c->h_nodes.assign(X, X + ntot * c->dim);
  } catch (const std::bad_alloc&) {
    c->h_nodes.clear();
    return lor_fail(c, LOR_ENOMEM, "lor_set_node_coordinates: host copy");
  }
  for (double x : c->h_nodes)
    if (!std::isfinite(x)) {
      c->h_nodes.clear();
      return lor_fail(c, LOR_EINVAL, "lor_set_node_coordinates: non-finite coordinate");
    }
  return LOR_OK;
}

lor_status lor_set_schwarz(lor_ctx* c, int mode) {
  if (!c || !c->setup_done) return LOR_ESTATE;
  if (mode < 0 || mode > 2)
    return lor_fail(c, LOR_EINVAL, "lor_set_schwarz: 0 (additive), 1 (hybrid) or 2 (single patch)");
  if (mode != 0 && c->learned_on) return lor_fail(c, LOR_EINVAL, "learned correction needs the additive form");
  if (mode == 2) {
    const lor_status st = lor_single_prepare(c);
    if (st) return st;
  }
  if (mode == 1 && !c->d_hyb) {
    c->d_hyb = lor_alloc(c, (size_t)3 * c->lev[0].ntot * sizeof(double));
    if (!c->d_hyb) return lor_fail(c, LOR_ENOMEM, "alloc hybrid Schwarz work vectors");
  }
  c->schwarz = mode;
  c->pcg_state_ok = false;
  return LOR_OK;
}

lor_status lor_set_weighting(lor_ctx* c, int weighting) {
  if (!c) return LOR_EINVAL;
  if (weighting < 0 || weighting > 2) return lor_fail(c, LOR_EINVAL, "lor_set_weighting: 0, 1 or 2");
  if (weighting && c->learned_on) return lor_fail(c, LOR_EINVAL, "learned correction needs unit patch weights");
  if (weighting && !c->h_spans.empty()) return lor_fail(c, LOR_EINVAL, "enlarged patches take unit patch weights");
  c->opt.weighting = weighting;
  return LOR_OK;
}

lor_status lor_set_prec(lor_ctx* c, int prec) {
  if (!c) return LOR_EINVAL;
  if (prec != LOR_FP64 && prec != LOR_MIXED) return lor_fail(c, LOR_EINVAL, "lor_set_prec: LOR_FP64 or LOR_MIXED");
  c->opt.prec = prec;
  return LOR_OK;
}

lor_status lor_launch_count(const lor_ctx* c, long long* count) {
  if (!c || !count) return LOR_EINVAL;
  *count = c->launches;
  return LOR_OK;
}

lor_status lor_residual_history(const lor_ctx* c, double* out, int cap, int* count) {
  if (!c || !count) return LOR_EINVAL;
  *count = (int)c->hist.size();
  if (out)
    for (int i = 0; i < cap && i < (int)c->hist.size(); ++i) out[i] = c->hist[i];
  return LOR_OK;
}

const char* lor_last_error(const lor_ctx* c) { return c ? c->err.c_str() : "null context"; }

void lor_destroy(lor_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  if (c->dg_state) lor_free_dg(c);
  if (c->learned) lor_free_learned(c);
  if (c->single) lor_free_single(c);
  for (void* p : c->allocs) cudaFree(p);
  for (int k = 0; k < 6; ++k)
    for (cudaEvent_t e : c->ev[k]) cudaEventDestroy(e);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  delete c;
}

}  // extern "C"
