// Interior-penalty and BR2 DG operators and the DG preconditioner (3D).
//
// Section 2.1, Eq. (ip)/(br2): a(u,v) = sum_D (b grad u, grad v)_D
//   - <{b grad u}, [[v]]> - <[[u]], {b grad v}> + penalty, with
//   IP  penalty <sigma [[u]], [[v]]>, sigma = eta p^2 b_F / h_F (b_F = max(b-,b+),
//       h_F = min|D-|,|D+| / |F|), face integrals with (p+1)^2 Gauss points;
//   BR2 penalty sum_e eta (b r_e[[u]], r_e[[v]]) with the GLL-lumped lifting, which
//       is nodal at the GLL face nodes: eta b_K (w_f|J_f|)^2 / (c w_f w_end |J_K|)
//       per side K (c = 4 on interior faces, 1 on Dirichlet faces).
// Section 3.5, Eq. (dg-as): B_DG = R_B Q_B + R_p Q_p, R_B point Jacobi on the
//   element-boundary nodes, R_p = the conforming LOR preconditioner B through the
//   injection E of H^1_0 into the DG space: z = D_B^{-1} r + E B E^T r.
//
// Volume term: the element-local sum-factorized kernel.  Face terms: one
// thread per (face, Gauss point) forms the averaged flux and the jump into a
// small face buffer; one thread per (face, side, element node) applies the
// transposed trace and normal-derivative evaluation and adds into y.
// Faces: for axis a, (n_a+1) n_b n_c faces (b < c the other axes), face id
// off_a + (tc*n_b + tb)*(n_a+1) + ia; the "first" side is the element below the
// face (ia-1, node index p along a) if it exists, else the element above (index
// 0); the normal n points out of the first side.
#include <algorithm>
#include <cmath>
#include <vector>

#include "geom.cuh"
#include "lor_internal.h"

namespace {

struct FaceTopo {
  int eF, eS;      // first / second element (eS = -1 on Dirichlet faces)
  int a;           // normal axis
  int endF, endS;  // node index of the face along a in each element (0 or p)
};

__device__ __forceinline__ void face_decode(int f, const int* n, int* a, int* ia, int* tb, int* tc) {
  int off = 0;
  for (int ax = 0; ax < 3; ++ax) {
    const int b = ax == 0 ? 1 : 0, c = ax == 2 ? 1 : 2;
    const int cnt = (n[ax] + 1) * n[b] * n[c];
    if (f < off + cnt) {
      const int r = f - off;
      *a = ax;
      *ia = r % (n[ax] + 1);
      *tb = (r / (n[ax] + 1)) % n[b];
      *tc = r / ((n[ax] + 1) * n[b]);
      return;
    }
    off += cnt;
  }
}

// Face colour classes: faces with normal axis a whose position ia along a has the
// parity par.  Two faces of one class never touch the same element (face ia lies
// between elements ia-1 and ia along a), so a kernel over one class may add into
// element nodes without atomics; the 6 classes run one after another in a fixed
// order, which makes the sums the same bit for bit on every run.
struct FaceClass { int a, par, m; long long count; int off; };

__host__ __device__ inline FaceClass face_class(const int* n, int a, int par) {
  FaceClass k;
  k.a = a; k.par = par;
  const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  k.m = (n[a] + 1 - par + 1) / 2;                   // positions ia = par, par + 2, ... <= n[a]
  k.count = (long long)k.m * n[b] * n[c];
  k.off = 0;
  for (int ax = 0; ax < a; ++ax) {
    const int bb = ax == 0 ? 1 : 0, cc = ax == 2 ? 1 : 2;
    k.off += (n[ax] + 1) * n[bb] * n[cc];
  }
  return k;
}

// face index (face_decode numbering) of the idx-th face of class k
__device__ __forceinline__ int class_face(const FaceClass& k, const int* n, long long idx) {
  const int ia = k.par + 2 * (int)(idx % k.m);
  return k.off + ia + (n[k.a] + 1) * (int)(idx / k.m);
}

__device__ __forceinline__ int elem_id(const int* n, int a, int ia, int tb, int tc) {
  int e3[3];
  const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  e3[a] = ia; e3[b] = tb; e3[c] = tc;
  return (e3[2] * n[1] + e3[1]) * n[0] + e3[0];
}

// element-local index of the node with coordinate i along a, j along b, k along c
__device__ __forceinline__ int loc3(int Q, int a, int i, int j, int k) {
  int x[3];
  const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  x[a] = i; x[b] = j; x[c] = k;
  return (x[2] * Q + x[1]) * Q + x[0];
}

struct DGGeomArgs {
  int p, n[3], nface;
  double eta;
  int br2;
  const double* vert;
  const double* kappa;
  const double* vol;
  const double* glx;   // Gauss points
  const double* glw;
  const double* gllx;
  const double* gllw;
  FaceTopo* topo;
  double* cF;          // [f][3][Q2]
  double* cS;
  double* W;           // [f][Q2]
  double* sigma;       // [f]
  double* beta;        // [f][Q2] (GLL face nodes)
  int* status;
};

__global__ void k_elem_volume(int p, int nx, int ny, int nz, const double* __restrict__ vert,
                              const double* __restrict__ glx, const double* __restrict__ glw, double* vol) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)nx * ny * nz) return;
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((long long)nx * ny));
  const long long NV = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  double Pc[8][3];
  lorg::element_corners(3, nx, ny, ex, ey, ez, vert, NV, Pc);
  const int Q = p + 1;
  double s = 0;
  for (int q = 0; q < Q * Q * Q; ++q) {
    const double xi[3] = {glx[q % Q], glx[(q / Q) % Q], glx[q / (Q * Q)]};
    double X[3], J[3][3];
    lorg::multilinear(3, Pc, xi, X, J);
    s += glw[q % Q] * glw[(q / Q) % Q] * glw[q / (Q * Q)] * fabs(lorg::det3(J));
  }
  vol[e] = s;
}

// one thread per face: topology, flux coefficients c = b W J^{-1} n, area weights,
// sigma, and the nodal BR2 penalty
__global__ void k_face_geom(DGGeomArgs g) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= g.nface) return;
  int a, ia, tb, tc;
  face_decode(f, g.n, &a, &ia, &tb, &tc);
  const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  const int p = g.p, Q = p + 1, Q2 = Q * Q;
  FaceTopo t;
  t.a = a;
  if (ia > 0) {
    t.eF = elem_id(g.n, a, ia - 1, tb, tc);
    t.endF = p;
    t.eS = ia < g.n[a] ? elem_id(g.n, a, ia, tb, tc) : -1;
    t.endS = 0;
  } else {
    t.eF = elem_id(g.n, a, 0, tb, tc);
    t.endF = 0;
    t.eS = -1;
    t.endS = 0;
  }
  g.topo[f] = t;
  const long long NV = (long long)(g.n[0] + 1) * (g.n[1] + 1) * (g.n[2] + 1);
  double PF[8][3], PS[8][3];
  {
    const int e = t.eF;
    lorg::element_corners(3, g.n[0], g.n[1], e % g.n[0], (e / g.n[0]) % g.n[1], e / (g.n[0] * g.n[1]), g.vert, NV, PF);
  }
  if (t.eS >= 0) {
    const int e = t.eS;
    lorg::element_corners(3, g.n[0], g.n[1], e % g.n[0], (e / g.n[0]) % g.n[1], e / (g.n[0] * g.n[1]), g.vert, NV, PS);
  }
  const double kF = g.kappa[t.eF], kS = t.eS >= 0 ? g.kappa[t.eS] : 0.0;
  const double sgn = t.endF == p ? 1.0 : -1.0;
  double area = 0;
  for (int q = 0; q < Q2; ++q) {
    const int q1 = q % Q, q2 = q / Q;
    double xi[3];
    xi[a] = t.endF == p ? 1.0 : 0.0;
    xi[b] = g.glx[q1];
    xi[c] = g.glx[q2];
    double X[3], J[3][3], Ji[3][3];
    lorg::multilinear(3, PF, xi, X, J);
    const double det = lorg::det3(J);
    if (!(det > 0)) atomicOr(g.status, 1);
    lorg::inv_dd(3, J, det, Ji);
    // J^{-T} e_a = row a of J^{-1}
    double gv[3] = {sgn * Ji[a][0], sgn * Ji[a][1], sgn * Ji[a][2]};
    const double gn = sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
    const double nrm[3] = {gv[0] / gn, gv[1] / gn, gv[2] / gn};
    const double W = g.glw[q1] * g.glw[q2] * det * gn;
    area += W;
    g.W[(long long)f * Q2 + q] = W;
    for (int r = 0; r < 3; ++r) {
      double s = 0;
      for (int t2 = 0; t2 < 3; ++t2) s += Ji[r][t2] * nrm[t2];
      g.cF[((long long)f * 3 + r) * Q2 + q] = kF * W * s;
    }
    if (t.eS >= 0) {
      double xs[3];
      xs[a] = 0.0; xs[b] = xi[b]; xs[c] = xi[c];
      double X2[3], J2[3][3], Ji2[3][3];
      lorg::multilinear(3, PS, xs, X2, J2);
      const double det2 = lorg::det3(J2);
      lorg::inv_dd(3, J2, det2, Ji2);
      for (int r = 0; r < 3; ++r) {
        double s = 0;
        for (int t2 = 0; t2 < 3; ++t2) s += Ji2[r][t2] * nrm[t2];
        g.cS[((long long)f * 3 + r) * Q2 + q] = kS * W * s;
      }
    } else {
      for (int r = 0; r < 3; ++r) g.cS[((long long)f * 3 + r) * Q2 + q] = 0.0;
    }
  }
  const double kmax = t.eS >= 0 ? fmax(kF, kS) : kF;
  const double hF = (t.eS >= 0 ? fmin(g.vol[t.eF], g.vol[t.eS]) : g.vol[t.eF]) / area;
  g.sigma[f] = g.eta * p * p * kmax / hF;
  // BR2 nodal penalty at the GLL face nodes
  const double wend = g.gllw[0];
  for (int q = 0; q < Q2; ++q) {
    const int j = q % Q, k = q / Q;
    double xi[3];
    xi[a] = t.endF == p ? 1.0 : 0.0;
    xi[b] = g.gllx[j];
    xi[c] = g.gllx[k];
    double X[3], J[3][3], Ji[3][3];
    lorg::multilinear(3, PF, xi, X, J);
    const double det = lorg::det3(J);
    lorg::inv_dd(3, J, det, Ji);
    const double gn = sqrt(Ji[a][0] * Ji[a][0] + Ji[a][1] * Ji[a][1] + Ji[a][2] * Ji[a][2]);
    const double wf = g.gllw[j] * g.gllw[k];
    const double dA = wf * det * gn;
    const double cc = t.eS >= 0 ? 4.0 : 1.0;
    double be = g.eta * kF * dA * dA / (cc * wf * wend * det);
    if (t.eS >= 0) {
      double xs[3];
      xs[a] = 0.0; xs[b] = xi[b]; xs[c] = xi[c];
      double X2[3], J2[3][3];
      lorg::multilinear(3, PS, xs, X2, J2);
      be += g.eta * kS * dA * dA / (cc * wf * wend * lorg::det3(J2));
    }
    g.beta[(long long)f * Q2 + q] = be;
  }
}

template <typename T>
struct FaceData {
  const FaceTopo* topo;
  const T* cF;
  const T* cS;
  const T* W;
  const T* sigma;
  const T* beta;
};

struct Tab {     // 1D tables (precision T): B/D at Gauss points, GLL nodal derivative row data
  const void* B;    // [Q][Q]  l_j(gl_q)
  const void* D;    // [Q][Q]  l_j'(gl_q)
  const void* Dn;   // [Q][Q]  l_j'(gll_i) (nodal differentiation matrix)
};

// All face terms of the faces of class k, one CTA per face, sum-factorized in shared
// memory (O(Q^3) work per face and side):
//  1. per side, the trace x(end, j, k) and the nodal normal derivative
//     sum_i Dn[end][i] x(i, j, k) at the face's GLL nodes;
//  2. both interpolated to the Gauss points (contractions along j, then k): u,
//     the tangential derivatives and the normal derivative, combined with the
//     side's geometric coefficients into c . grad u;
//  3. per point the averaged flux, the jump and the penalty (IP; BR2 adds its
//     nodal penalty in step 5): value-test weights of each side and the
//     gradient-test weight;
//  4. per side the transposed interpolation of those weights back to the face
//     nodes (contractions along q2, then q1): G1 (times the normal derivative of
//     the test function) and G2 (value and tangential-derivative tests);
//  5. every element node (i, j, k) of each side: y += Dn[end][i] G1(j, k), plus
//     G2(j, k) and the BR2 penalty at i = end.
// No two faces of a class share an element, so the adds need no atomics.
template <typename T>
__global__ void __launch_bounds__(128) k_face_sf(int p, FaceClass fk, int n0, int n1, int n2, int br2,
                                                 FaceData<T> fd, Tab tb, const T* __restrict__ x, T* y) {
  constexpr int MQ2 = (LOR_MAXP + 1) * (LOR_MAXP + 1);
  const int Q = p + 1, Q2 = Q * Q, Q3 = Q2 * Q;
  __shared__ T sB[MQ2], sD[MQ2], sDn[MQ2];
  __shared__ T tr[2][MQ2], nd[2][MQ2];            // [side][j + Q k]
  __shared__ T c1[2][MQ2], c2[2][MQ2], c3[2][MQ2];  // [side][q1 + Q k] partial contractions
  __shared__ T uv[2][MQ2], fl[2][MQ2];            // [side][q]: u and c . grad u at the Gauss points
  __shared__ T wv[3][MQ2];                        // [q]: value test of side 0, of side 1, gradient test
  __shared__ T m1[2][MQ2], m2[2][MQ2], m3[2][MQ2], m4[2][MQ2];
  __shared__ T g1[2][MQ2], g2[2][MQ2];            // [side][j + Q k]
  const int n[3] = {n0, n1, n2};
  const int f = class_face(fk, n, blockIdx.x);
  const FaceTopo t = fd.topo[f];
  const int ns = t.eS >= 0 ? 2 : 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int b = t.a == 0 ? 1 : 0, c = t.a == 2 ? 1 : 2;
  for (int i = tid; i < Q2; i += nt) {
    sB[i] = ((const T*)tb.B)[i];
    sD[i] = ((const T*)tb.D)[i];
    sDn[i] = ((const T*)tb.Dn)[i];
  }
  __syncthreads();
  // 1. traces and nodal normal derivatives
  for (int idx = tid; idx < ns * Q2; idx += nt) {
    const int s = idx / Q2, jk = idx - s * Q2, j = jk % Q, k = jk / Q;
    const int e = s ? t.eS : t.eF, end = s ? t.endS : t.endF;
    const T* xe = x + (long long)e * Q3;
    tr[s][jk] = xe[loc3(Q, t.a, end, j, k)];
    T ln = 0;
    for (int i = 0; i < Q; ++i) ln += sDn[end * Q + i] * xe[loc3(Q, t.a, i, j, k)];
    nd[s][jk] = ln;
  }
  __syncthreads();
  // 2a. along j
  for (int idx = tid; idx < ns * Q2; idx += nt) {
    const int s = idx / Q2, r = idx - s * Q2, q1 = r % Q, k = r / Q;
    T a1 = 0, a2 = 0, a3 = 0;
    for (int j = 0; j < Q; ++j) {
      const T v = tr[s][j + Q * k];
      a1 += sB[q1 * Q + j] * v;
      a2 += sD[q1 * Q + j] * v;
      a3 += sB[q1 * Q + j] * nd[s][j + Q * k];
    }
    c1[s][r] = a1; c2[s][r] = a2; c3[s][r] = a3;
  }
  __syncthreads();
  // 2b. along k: u and c . grad u at every Gauss point
  for (int idx = tid; idx < ns * Q2; idx += nt) {
    const int s = idx / Q2, q = idx - s * Q2, q1 = q % Q, q2 = q / Q;
    T u = 0, db = 0, dc = 0, da = 0;
    for (int k = 0; k < Q; ++k) {
      const T bk = sB[q2 * Q + k];
      u += bk * c1[s][q1 + Q * k];
      db += bk * c2[s][q1 + Q * k];
      dc += sD[q2 * Q + k] * c1[s][q1 + Q * k];
      da += bk * c3[s][q1 + Q * k];
    }
    T g[3];
    g[t.a] = da; g[b] = db; g[c] = dc;
    const T* cv = (s ? fd.cS : fd.cF) + (long long)f * 3 * Q2;
    uv[s][q] = u;
    fl[s][q] = cv[q] * g[0] + cv[Q2 + q] * g[1] + cv[2 * Q2 + q] * g[2];
  }
  __syncthreads();
  // 3. flux, jump and penalty per point
  for (int q = tid; q < Q2; q += nt) {
    const T half = ns == 2 ? T(0.5) : T(1);
    const T jump = ns == 2 ? uv[0][q] - uv[1][q] : uv[0][q];
    const T avg = half * (ns == 2 ? fl[0][q] + fl[1][q] : fl[0][q]);
    const T pen = br2 ? T(0) : fd.sigma[f] * fd.W[(long long)f * Q2 + q] * jump;
    wv[0][q] = -avg + pen;
    wv[1][q] = avg - pen;
    wv[2][q] = -half * jump;
  }
  __syncthreads();
  // 4a. per side and point the four weight fields, contracted along q2
  for (int idx = tid; idx < ns * Q2; idx += nt) {
    const int s = idx / Q2, r = idx - s * Q2, q1 = r % Q, k = r / Q;
    const T* cv = (s ? fd.cS : fd.cF) + (long long)f * 3 * Q2;
    const T* ca = cv + t.a * Q2;
    const T* cb = cv + b * Q2;
    const T* cc = cv + c * Q2;
    T h1 = 0, h2 = 0, h3 = 0, h4 = 0;
    for (int q2 = 0; q2 < Q; ++q2) {
      const int q = q2 * Q + q1;
      const T bk = sB[q2 * Q + k];
      const T sg = wv[2][q];
      h1 += bk * sg * ca[q];
      h2 += bk * wv[s][q];
      h3 += bk * sg * cb[q];
      h4 += sD[q2 * Q + k] * sg * cc[q];
    }
    m1[s][r] = h1; m2[s][r] = h2; m3[s][r] = h3; m4[s][r] = h4;
  }
  __syncthreads();
  // 4b. along q1: G1 and G2 at the face nodes (j, k)
  for (int idx = tid; idx < ns * Q2; idx += nt) {
    const int s = idx / Q2, jk = idx - s * Q2, j = jk % Q, k = jk / Q;
    T a1 = 0, a2 = 0;
    for (int q1 = 0; q1 < Q; ++q1) {
      const T bj = sB[q1 * Q + j];
      a1 += bj * m1[s][q1 + Q * k];
      a2 += bj * (m2[s][q1 + Q * k] + m4[s][q1 + Q * k]) + sD[q1 * Q + j] * m3[s][q1 + Q * k];
    }
    g1[s][jk] = a1;
    g2[s][jk] = a2;
  }
  __syncthreads();
  // 5. element nodes of both sides
  for (int idx = tid; idx < ns * Q3; idx += nt) {
    const int s = idx / Q3, node = idx - s * Q3;
    const int i = node % Q, jk = node / Q, j = jk % Q, k = jk / Q;
    const int e = s ? t.eS : t.eF, end = s ? t.endS : t.endF;
    T v = sDn[end * Q + i] * g1[s][jk];
    if (i == end) {
      v += g2[s][jk];
      if (br2) {
        const T jump = ns == 2 ? tr[0][jk] - tr[1][jk] : tr[0][jk];
        const T pb = fd.beta[(long long)f * Q2 + jk] * jump;
        v += s ? -pb : pb;
      }
    }
    y[(long long)e * Q3 + loc3(Q, t.a, i, j, k)] += v;
  }
}

// diagonal of A_DG: volume part per node, face part per (face, side, face node)
__global__ void k_diag_volume(int p, int nel, const double* __restrict__ B, const double* __restrict__ D,
                              const double* __restrict__ G, double* diag) {
  const int Q = p + 1, Q3 = Q * Q * Q;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)nel * Q3) return;
  const long long e = gid / Q3;
  const int n = (int)(gid - e * Q3);
  const int i = n % Q, j = (n / Q) % Q, k = n / (Q * Q);
  const double* Ge = G + e * 6 * Q3;
  double s = 0;
  for (int q = 0; q < Q3; ++q) {
    const int qx = q % Q, qy = (q / Q) % Q, qz = q / (Q * Q);
    const double bx = B[qx * Q + i], by = B[qy * Q + j], bz = B[qz * Q + k];
    const double g0 = D[qx * Q + i] * by * bz, g1 = bx * D[qy * Q + j] * bz, g2 = bx * by * D[qz * Q + k];
    s += Ge[q] * g0 * g0 + Ge[3 * Q3 + q] * g1 * g1 + Ge[5 * Q3 + q] * g2 * g2 +
         2.0 * (Ge[Q3 + q] * g0 * g1 + Ge[2 * Q3 + q] * g0 * g2 + Ge[4 * Q3 + q] * g1 * g2);
  }
  diag[gid] = s;
}

__global__ void k_diag_face(int p, FaceClass fk, int n0, int n1, int n2, int br2, FaceData<double> fd,
                            const double* __restrict__ B, const double* __restrict__ D, const double* __restrict__ Dn,
                            double* diag) {
  const int Q = p + 1, Q2 = Q * Q, Q3 = Q2 * Q;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= fk.count * 2 * Q2) return;
  const int n[3] = {n0, n1, n2};
  const long long fi = gid / (2 * Q2);
  const int f = class_face(fk, n, fi);
  const int r = (int)(gid - fi * 2 * Q2);
  const int s = r / Q2, jk = r % Q2;
  const FaceTopo t = fd.topo[f];
  if (s == 1 && t.eS < 0) return;
  const int j = jk % Q, k = jk / Q;
  const int e = s ? t.eS : t.eF;
  const int end = s ? t.endS : t.endF;
  const double sign = s ? -1.0 : 1.0;
  const double half = t.eS >= 0 ? 0.5 : 1.0;
  const double* cv = (s ? fd.cS : fd.cF) + (long long)f * 3 * Q2;
  const int b = t.a == 0 ? 1 : 0, c = t.a == 2 ? 1 : 2;
  double acc = 0;
  for (int q2 = 0; q2 < Q; ++q2)
    for (int q1 = 0; q1 < Q; ++q1) {
      const int q = q2 * Q + q1;
      const double phi = B[q1 * Q + j] * B[q2 * Q + k];
      const double ga = Dn[end * Q + end] * phi, gb = D[q1 * Q + j] * B[q2 * Q + k], gc = B[q1 * Q + j] * D[q2 * Q + k];
      const double cgrad = cv[t.a * Q2 + q] * ga + cv[b * Q2 + q] * gb + cv[c * Q2 + q] * gc;
      acc += -2.0 * half * sign * phi * cgrad;
      if (!br2) acc += fd.sigma[f] * fd.W[(long long)f * Q2 + q] * phi * phi;
    }
  if (br2) acc += fd.beta[(long long)f * Q2 + jk];
  diag[(long long)e * Q3 + loc3(Q, t.a, end, j, k)] += acc;
}

// E^T: DG block values summed into the conforming node grid.  One thread per
// grid node adds the block values of the (at most 8) elements sharing it, in a
// fixed order (element index ascending along x, then y, then z).
template <typename T>
__global__ void k_dg_to_cg(int p, int nx, int ny, int nz, const T* __restrict__ xd, T* xc) {
  const int Q = p + 1, Q3 = Q * Q * Q;
  const int Nx = nx * p + 1, Ny = ny * p + 1, Nz = nz * p + 1;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)Nx * Ny * Nz) return;
  const int I = (int)(gid % Nx), Jn = (int)((gid / Nx) % Ny), K = (int)(gid / ((long long)Nx * Ny));
  // per axis: the elements containing the node (the one before a shared plane first)
  const int e0x = I % p == 0 && I > 0 ? I / p - 1 : min(I / p, nx - 1);
  const int e1x = I % p == 0 && I > 0 && I / p < nx ? I / p : -1;
  const int e0y = Jn % p == 0 && Jn > 0 ? Jn / p - 1 : min(Jn / p, ny - 1);
  const int e1y = Jn % p == 0 && Jn > 0 && Jn / p < ny ? Jn / p : -1;
  const int e0z = K % p == 0 && K > 0 ? K / p - 1 : min(K / p, nz - 1);
  const int e1z = K % p == 0 && K > 0 && K / p < nz ? K / p : -1;
  T s = T(0);
  for (int cz = 0; cz < 2; ++cz) {
    const int ez = cz ? e1z : e0z;
    if (ez < 0) continue;
    for (int cy = 0; cy < 2; ++cy) {
      const int ey = cy ? e1y : e0y;
      if (ey < 0) continue;
      for (int cx = 0; cx < 2; ++cx) {
        const int ex = cx ? e1x : e0x;
        if (ex < 0) continue;
        const long long e = ((long long)ez * ny + ey) * nx + ex;
        const int li = I - ex * p, lj = Jn - ey * p, lk = K - ez * p;
        s += xd[e * Q3 + (lk * Q + lj) * Q + li];
      }
    }
  }
  xc[gid] = s;
}

// z_dg = [element-boundary node] r / diag + E zc
template <typename T>
__global__ void k_dg_combine(int p, int nx, int ny, int nz, const T* __restrict__ r, const T* __restrict__ dinv,
                             const T* __restrict__ zc, T* z) {
  const int Q = p + 1, Q3 = Q * Q * Q;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long long)nx * ny * nz * Q3) return;
  const long long e = gid / Q3;
  const int n = (int)(gid - e * Q3);
  const int i = n % Q, j = (n / Q) % Q, k = n / (Q * Q);
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = (int)(e / ((long long)nx * ny));
  const int Nx = nx * p + 1, Ny = ny * p + 1;
  const long long g = ((long long)(ez * p + k) * Ny + (ey * p + j)) * Nx + (ex * p + i);
  const bool vb = i == 0 || i == p || j == 0 || j == p || k == 0 || k == p;
  z[gid] = (vb ? r[gid] * dinv[gid] : T(0)) + zc[g];
}

__global__ void k_inv_to(const double* __restrict__ d, double* d64, float* d32, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    d64[i] = 1.0 / d[i];
    d32[i] = (float)(1.0 / d[i]);
  }
}

__global__ void k_d2f(const double* __restrict__ a, float* b, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// element-local right-hand side b_e = B^T W_e
__global__ void k_rhs_dg(int p, long long nel, const double* __restrict__ Bm, const double* __restrict__ W,
                         double* __restrict__ b) {
  const int Q = p + 1, Q3 = Q * Q * Q;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nel * Q3) return;
  const long long e = gid / Q3;
  const int n = (int)(gid - e * Q3);
  const int i = n % Q, j = (n / Q) % Q, k = n / (Q * Q);
  const double* We = W + e * Q3;
  double s = 0;
  for (int q = 0; q < Q3; ++q)
    s += Bm[(q % Q) * Q + i] * Bm[((q / Q) % Q) * Q + j] * Bm[(q / (Q * Q)) * Q + k] * We[q];
  b[gid] = s;
}

}  // namespace

// ================================================================== host side
struct DGState {
  int nface = 0;
  FaceTopo* topo = nullptr;
  double *cF64, *cS64, *W64, *sig64, *beta64;
  float *cF32, *cS32, *W32, *sig32, *beta32;
  double* dinv64;
  float* dinv32;
  double *tab64;   // B | D | Dn  (Q*Q each)
  float *tab32;
  double *cgin64, *cgout64;
  float *cgin32, *cgout32;
};

static DGState* dgs(lor_ctx* c) { return (DGState*)c->dg_state; }

template <typename T> static FaceData<T> face_data(lor_ctx* c);
template <> FaceData<double> face_data<double>(lor_ctx* c) {
  DGState* s = dgs(c);
  return FaceData<double>{s->topo, s->cF64, s->cS64, s->W64, s->sig64, s->beta64};
}
template <> FaceData<float> face_data<float>(lor_ctx* c) {
  DGState* s = dgs(c);
  return FaceData<float>{s->topo, s->cF32, s->cS32, s->W32, s->sig32, s->beta32};
}
template <typename T> static Tab tabs(lor_ctx* c, int Q);
template <> Tab tabs<double>(lor_ctx* c, int Q) {
  double* t = dgs(c)->tab64;
  return Tab{t, t + Q * Q, t + 2 * Q * Q};
}
template <> Tab tabs<float>(lor_ctx* c, int Q) {
  float* t = dgs(c)->tab32;
  return Tab{t, t + Q * Q, t + 2 * Q * Q};
}

lor_status lor_setup_dg(lor_ctx* c) {
  if (c->dim != 3) return lor_fail(c, LOR_EINVAL, "DG discretizations are implemented for dim = 3");
  DGState* s = new DGState();
  c->dg_state = s;
  const int p = c->p, Q = p + 1, Q2 = Q * Q, Q3 = Q2 * Q;
  const int* n = c->n;
  s->nface = (n[0] + 1) * n[1] * n[2] + n[0] * (n[1] + 1) * n[2] + n[0] * n[1] * (n[2] + 1);
  const long long nf = s->nface, nel = c->nel, ndg = nel * Q3;
  auto A64 = [&](long long k) { return (double*)lor_alloc(c, k * 8); };
  auto A32 = [&](long long k) { return (float*)lor_alloc(c, k * 4); };
  s->topo = (FaceTopo*)lor_alloc(c, nf * sizeof(FaceTopo));
  s->cF64 = A64(nf * 3 * Q2); s->cS64 = A64(nf * 3 * Q2); s->W64 = A64(nf * Q2);
  s->sig64 = A64(nf); s->beta64 = A64(nf * Q2);
  s->cF32 = A32(nf * 3 * Q2); s->cS32 = A32(nf * 3 * Q2); s->W32 = A32(nf * Q2);
  s->sig32 = A32(nf); s->beta32 = A32(nf * Q2);

  s->dinv64 = A64(ndg); s->dinv32 = A32(ndg);
  s->tab64 = A64(3 * Q2); s->tab32 = A32(3 * Q2);
  s->cgin64 = A64(c->lev[0].ntot); s->cgout64 = A64(c->lev[0].ntot);
  s->cgin32 = A32(c->lev[0].ntot); s->cgout32 = A32(c->lev[0].ntot);
  double* vol = A64(nel);
  double* diag = A64(ndg);
  if (!s->topo || !s->cF64 || !s->cS64 || !s->W64 || !s->sig64 || !s->beta64 || !s->cF32 || !s->cS32 || !s->W32 ||
      !s->sig32 || !s->beta32 || !s->dinv64 || !s->dinv32 || !s->tab64 || !s->tab32 ||
      !s->cgin64 || !s->cgout64 || !s->cgin32 || !s->cgout32 || !vol || !diag)
    return lor_fail(c, LOR_ENOMEM, "alloc DG data");
  // 1D tables: B, D at Gauss points (as in the volume kernel) and the nodal GLL derivative
  std::vector<double> t64(3 * Q2);
  double Bn[(LOR_MAXP + 1) * (LOR_MAXP + 1)], Dn[(LOR_MAXP + 1) * (LOR_MAXP + 1)], Dq[(LOR_MAXP + 1) * (LOR_MAXP + 1)];
  lorh::lagrange(Q, c->gll_x, Q, c->gl_x, t64.data(), Dq);          // B and D at Gauss points
  for (int i = 0; i < Q2; ++i) t64[Q2 + i] = Dq[i];
  lorh::lagrange(Q, c->gll_x, Q, c->gll_x, Bn, Dn);                  // nodal derivative matrix
  for (int i = 0; i < Q2; ++i) t64[2 * Q2 + i] = Dn[i];
  std::vector<float> t32(t64.begin(), t64.end());
  cudaMemcpyAsync(s->tab64, t64.data(), t64.size() * 8, cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(s->tab32, t32.data(), t32.size() * 4, cudaMemcpyHostToDevice, c->stream);
  k_elem_volume<<<(unsigned)lor_ceil_div(nel, 128), 128, 0, c->stream>>>(p, n[0], n[1], n[2], c->d_vert,
                                                                           lor_basis64(c, 2), lor_basis64(c, 3), vol);
  ++c->launches;
  DGGeomArgs g;
  g.p = p; g.n[0] = n[0]; g.n[1] = n[1]; g.n[2] = n[2]; g.nface = (int)nf;
  g.eta = c->opt.eta; g.br2 = c->opt.disc == LOR_DG_BR2;
  g.vert = c->d_vert; g.kappa = c->d_kappa; g.vol = vol;
  g.glx = lor_basis64(c, 2); g.glw = lor_basis64(c, 3); g.gllx = lor_basis64(c, 4);
  double* gllw = A64(Q);
  if (!gllw) return lor_fail(c, LOR_ENOMEM, "alloc");
  cudaMemcpyAsync(gllw, c->gll_w, Q * 8, cudaMemcpyHostToDevice, c->stream);
  g.gllw = gllw;
  g.topo = s->topo; g.cF = s->cF64; g.cS = s->cS64; g.W = s->W64; g.sigma = s->sig64; g.beta = s->beta64;
  g.status = c->d_status;
  k_face_geom<<<(unsigned)lor_ceil_div(nf, 64), 64, 0, c->stream>>>(g);
  ++c->launches;
  auto conv = [&](const double* a, float* b, long long k) {
    k_d2f<<<(unsigned)lor_ceil_div(k, 256), 256, 0, c->stream>>>(a, b, k);
    ++c->launches;
  };
  conv(s->cF64, s->cF32, nf * 3 * Q2);
  conv(s->cS64, s->cS32, nf * 3 * Q2);
  conv(s->W64, s->W32, nf * Q2);
  conv(s->sig64, s->sig32, nf);
  conv(s->beta64, s->beta32, nf * Q2);
  // diagonal
  k_diag_volume<<<(unsigned)lor_ceil_div(ndg, 128), 128, 0, c->stream>>>(p, c->nel, s->tab64, s->tab64 + Q2,
                                                                          c->d_G64, diag);
  ++c->launches;
  for (int a = 0; a < 3; ++a)
    for (int par = 0; par < 2; ++par) {
      const FaceClass fk = face_class(c->n, a, par);
      if (fk.count == 0) continue;
      k_diag_face<<<(unsigned)lor_ceil_div(fk.count * 2 * Q2, 128), 128, 0, c->stream>>>(
          p, fk, c->n[0], c->n[1], c->n[2], c->opt.disc == LOR_DG_BR2, face_data<double>(c), s->tab64, s->tab64 + Q2,
          s->tab64 + 2 * Q2, diag);
      ++c->launches;
    }
  k_inv_to<<<(unsigned)lor_ceil_div(ndg, 256), 256, 0, c->stream>>>(diag, s->dinv64, s->dinv32, ndg);
  ++c->launches;
  return lor_cuda_check(c, cudaGetLastError(), "DG setup");
}


template <typename T>
static lor_status apply_A_dg(lor_ctx* c, const T* x, T* y) {
  extern lor_status lor_launch_dgvol64(lor_ctx*, const double*, double*);
  extern lor_status lor_launch_dgvol32(lor_ctx*, const float*, float*);
  lor_status st = sizeof(T) == 8 ? lor_launch_dgvol64(c, (const double*)x, (double*)y)
                                 : lor_launch_dgvol32(c, (const float*)x, (float*)y);
  if (st) return st;
  const int p = c->p, Q = p + 1;
  const bool br2 = c->opt.disc == LOR_DG_BR2;
  // face classes one after another (no two faces of a class share an element)
  for (int a = 0; a < 3; ++a)
    for (int par = 0; par < 2; ++par) {
      const FaceClass fk = face_class(c->n, a, par);
      if (fk.count == 0) continue;
      k_face_sf<T><<<(unsigned)fk.count, 128, 0, c->stream>>>(p, fk, c->n[0], c->n[1], c->n[2], br2 ? 1 : 0,
                                                              face_data<T>(c), tabs<T>(c, Q), x, y);
      ++c->launches;
    }
  return lor_cuda_check(c, cudaGetLastError(), "DG apply");
}

lor_status lor_launch_apply_A_dg64(lor_ctx* c, const double* x, double* y) { return apply_A_dg<double>(c, x, y); }
lor_status lor_launch_apply_A_dg32(lor_ctx* c, const float* x, float* y) { return apply_A_dg<float>(c, x, y); }

template <typename T>
static lor_status apply_P_dg(lor_ctx* c, const T* r, T* z, T* cgin, T* cgout, const T* dinv) {
  const int p = c->p, Q = p + 1;
  const long long ndg = (long long)c->nel * Q * Q * Q;
  k_dg_to_cg<T><<<(unsigned)lor_ceil_div(c->lev[0].ntot, 256), 256, 0, c->stream>>>(p, c->n[0], c->n[1], c->n[2], r,
                                                                                      cgin);
  ++c->launches;
  lor_status st = sizeof(T) == 8 ? lor_launch_apply_P64(c, (const double*)cgin, (double*)cgout)
                                 : lor_launch_apply_P32(c, (const float*)cgin, (float*)cgout);
  if (st) return st;
  k_dg_combine<T><<<(unsigned)lor_ceil_div(ndg, 256), 256, 0, c->stream>>>(p, c->n[0], c->n[1], c->n[2], r, dinv,
                                                                            cgout, z);
  ++c->launches;
  return lor_cuda_check(c, cudaGetLastError(), "DG precond");
}

lor_status lor_launch_apply_P_dg64(lor_ctx* c, const double* r, double* z) {
  DGState* s = dgs(c);
  return apply_P_dg<double>(c, r, z, s->cgin64, s->cgout64, s->dinv64);
}
lor_status lor_launch_apply_P_dg32(lor_ctx* c, const float* r, float* z) {
  DGState* s = dgs(c);
  return apply_P_dg<float>(c, r, z, s->cgin32, s->cgout32, s->dinv32);
}

lor_status lor_launch_rhs_dg(lor_ctx* c, double* b, const double* W) {
  const int Q = c->p + 1;
  const long long ndg = (long long)c->nel * Q * Q * Q;
  k_rhs_dg<<<(unsigned)lor_ceil_div(ndg, 128), 128, 0, c->stream>>>(c->p, c->nel, lor_basis64(c, 0), W, b);
  ++c->launches;
  return lor_cuda_check(c, cudaGetLastError(), "DG rhs");
}

void lor_free_dg(lor_ctx* c) {
  delete dgs(c);
  c->dg_state = nullptr;
}
