// Setup of the LOR preconditioner and the operator data (Section 3, Table 1).
//  * geometric factors of the sum-factorized operator (Section 2)
//  * K_h: multilinear stiffness on the GLL-refined mesh T_h as a 3^d-point stencil
//    per node (Section 3.1), 2-point Gauss per direction on every sub-element
//  * Galerkin level stencils A_{l+1} = P^T A_l P of the element-structured
//    hierarchy (Section 3.3), P = tensor 1D linear interpolation in reference
//    coordinates
//  * lexicographic ILU(0) of every vertex patch at every level (Section 3.4),
//    one CTA per patch, rows level-scheduled by wavefront i + 2j + 4k
//  * coarse-space hierarchy on the vertex grid (Section 3.2, R_0)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <array>
#include <atomic>
#include <map>
#include <cstring>
#include <thread>

#include "lor_internal.h"
#include "geom.cuh"

// ------------------------------------------------------------------ basis block
// Device layout of the small basis block: for precision 64: [B | Dq | glx | glw |
// gllx | Dn], each (LOR_MAXP+2)^2 doubles (Dn: derivative of the GLL Lagrange basis at
// the Gauss points, [q][i]); for 32: [B | Dq] floats.
static const int kBlk = (LOR_MAXP + 2) * (LOR_MAXP + 2);

// The two blocks are the first two allocations of the context (lor_setup_geometry).
double* lor_basis64(lor_ctx* c, int which) { return (double*)c->allocs[0] + which * kBlk; }
float* lor_basis32(lor_ctx* c, int which) { return (float*)c->allocs[1] + which * kBlk; }
BoxShape* lor_dev_shapes(lor_ctx* c) { return c->d_shapes; }

// Sample points of a pointwise coefficient (Section 4.2), in the layouts k_geom and
// k_lor_stencil read: K_p Gauss points [element][q] (elements x fastest, q = qx +
// Q qy + Q^2 qz, Q = p + 1 Gauss-Legendre points per axis) and the 2-point Gauss
// points of the LOR sub-cells [cell][g] (cells x fastest on the GLL-refined grid,
// g = gx + 2 gy + 4 gz), each as dim coordinates.
void lor_coef_sizes(const lor_ctx* c, long long* nq, long long* nh) {
  const int dim = c->dim, p = c->p;
  long long q = 1, cells = 1;
  for (int a = 0; a < dim; ++a) { q *= p + 1; cells *= (long long)c->n[a] * p; }
  *nq = (long long)c->nel * q;
  *nh = cells * (1LL << dim);
}

void lor_coef_points(const lor_ctx* c, double* xq, double* xh) {
  const int dim = c->dim, p = c->p, Q = p + 1, nx = c->n[0], ny = c->n[1], nz = c->n[2];
  double gllx[LOR_MAXP + 1], gllw[LOR_MAXP + 1], glx[LOR_MAXP + 2], glw[LOR_MAXP + 2];
  lorh::gll(p, gllx, gllw);
  lorh::gauss(Q, glx, glw);
  const long long NV = (long long)(nx + 1) * (ny + 1) * (dim == 3 ? nz + 1 : 1);
  const double* vert = c->h_vert.data();
  const int Qd = dim == 3 ? Q * Q * Q : Q * Q;
  double Pc[8][3], X[3], J[3][3];
  if (xq) {
    for (long long e = 0; e < c->nel; ++e) {
      const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = dim == 3 ? (int)(e / ((long long)nx * ny)) : 0;
      lorg::element_corners(dim, nx, ny, ex, ey, ez, vert, NV, Pc);
      for (int q = 0; q < Qd; ++q) {
        const double xi[3] = {glx[q % Q], glx[(q / Q) % Q], dim == 3 ? glx[q / (Q * Q)] : 0.0};
        lorg::multilinear(dim, Pc, xi, X, J);
        for (int a = 0; a < dim; ++a) xq[(e * Qd + q) * dim + a] = X[a];
      }
    }
  }
  if (xh) {
    const int Nx = nx * p + 1, Ny = ny * p + 1, Nz = dim == 3 ? nz * p + 1 : 1;
    const double gq = 0.5 - 0.5 / sqrt(3.0);
    const double g1[2] = {gq, 1.0 - gq};
    const int nc = 1 << dim;
    // node position: the element map at the node's GLL point (as k_nodes)
    auto node = [&](int I, int Jn, int K, double* out) {
      const int ex = std::min(I / p, nx - 1), ey = std::min(Jn / p, ny - 1), ez = dim == 3 ? std::min(K / p, nz - 1) : 0;
      const double xi[3] = {gllx[I - ex * p], gllx[Jn - ey * p], dim == 3 ? gllx[K - ez * p] : 0.0};
      double P[8][3], JJ[3][3];
      lorg::element_corners(dim, nx, ny, ex, ey, ez, vert, NV, P);
      lorg::multilinear(dim, P, xi, out, JJ);
    };
    long long cidx = 0;
    for (int oz = 0; oz < (dim == 3 ? Nz - 1 : 1); ++oz)
      for (int oy = 0; oy < Ny - 1; ++oy)
        for (int ox = 0; ox < Nx - 1; ++ox, ++cidx) {
          double Cc[8][3] = {};
          for (int t = 0; t < nc; ++t) node(ox + (t & 1), oy + ((t >> 1) & 1), oz + ((t >> 2) & 1), Cc[t]);
          for (int g = 0; g < nc; ++g) {
            const double xi[3] = {g1[g & 1], g1[(g >> 1) & 1], dim == 3 ? g1[(g >> 2) & 1] : 0.0};
            lorg::multilinear(dim, Cc, xi, X, J);
            for (int a = 0; a < dim; ++a) xh[(cidx * nc + g) * dim + a] = X[a];
          }
        }
  }
}

void lor_quad_points(const lor_ctx* c, double* xq) {
  if (c->h_nodes.empty()) {   // multilinear elements: the K_p sample points
    lor_coef_points(c, xq, nullptr);
    return;
  }
  // curved elements: the degree-p interpolant of the GLL node coordinates
  const int dim = c->dim, p = c->p, Q = p + 1, nx = c->n[0], ny = c->n[1];
  double gllx[LOR_MAXP + 1], gllw[LOR_MAXP + 1], glx[LOR_MAXP + 2], glw[LOR_MAXP + 2];
  double Bq[(LOR_MAXP + 1) * (LOR_MAXP + 1)], Dq[(LOR_MAXP + 1) * (LOR_MAXP + 1)];
  lorh::gll(p, gllx, gllw);
  lorh::gauss(Q, glx, glw);
  lorh::lagrange(Q, gllx, Q, glx, Bq, Dq);   // Bq[q * Q + i] = l_i(gl_q)
  const int Nx = nx * p + 1, Ny = ny * p + 1;
  const long long ntot = (long long)Nx * Ny * (dim == 3 ? (long long)c->n[2] * p + 1 : 1);
  const int Qd = dim == 3 ? Q * Q * Q : Q * Q;
  const double* X = c->h_nodes.data();
  for (long long e = 0; e < c->nel; ++e) {
    const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = dim == 3 ? (int)(e / ((long long)nx * ny)) : 0;
    for (int q = 0; q < Qd; ++q) {
      const int qx = q % Q, qy = (q / Q) % Q, qz = dim == 3 ? q / (Q * Q) : 0;
      double acc[3] = {0.0, 0.0, 0.0};
      for (int k = 0; k < (dim == 3 ? Q : 1); ++k)
        for (int j = 0; j < Q; ++j)
          for (int i = 0; i < Q; ++i) {
            const double phi = Bq[qx * Q + i] * Bq[qy * Q + j] * (dim == 3 ? Bq[qz * Q + k] : 1.0);
            const long long node = ((long long)(ez * p + k) * Ny + (ey * p + j)) * Nx + (ex * p + i);
            for (int a = 0; a < dim; ++a) acc[a] += phi * X[a * ntot + node];
          }
      for (int a = 0; a < dim; ++a) xq[(e * Qd + q) * dim + a] = acc[a];
    }
  }
}

namespace {

// G[e][comp][q] = kappa_e w_q det J (J^{-1} J^{-T})_{ab}, comps (00,01,02,11,12,22) / (00,01,11)
// bq (optional): the coefficient at every Gauss point ([e][q]) in place of kappa_e.
__global__ void k_geom(int dim, int p, int nx, int ny, int nz, const double* __restrict__ vert,
                       const double* __restrict__ kappa, const double* __restrict__ bq,
                       const double* __restrict__ glx, const double* __restrict__ glw, double* __restrict__ G64,
                       float* __restrict__ G32, int* status) {
  const int Q = p + 1;
  const int Qd = dim == 3 ? Q * Q * Q : Q * Q;
  const long long nel = (long long)nx * ny * (dim == 3 ? nz : 1);
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= nel * Qd) return;
  const long long e = gid / Qd;
  const int q = (int)(gid - e * Qd);
  const int qx = q % Q, qy = (q / Q) % Q, qz = dim == 3 ? q / (Q * Q) : 0;
  const int ex = (int)(e % nx), ey = (int)((e / nx) % ny), ez = dim == 3 ? (int)(e / ((long long)nx * ny)) : 0;
  const long long NV = (long long)(nx + 1) * (ny + 1) * (dim == 3 ? (nz + 1) : 1);
  double Pc[8][3];
  lorg::element_corners(dim, nx, ny, ex, ey, ez, vert, NV, Pc);
  const double xi[3] = {glx[qx], glx[qy], dim == 3 ? glx[qz] : 0.0};
  double X[3], J[3][3];
  lorg::multilinear(dim, Pc, xi, X, J);
  const double det = dim == 3 ? lorg::det3(J) : (J[0][0] * J[1][1] - J[0][1] * J[1][0]);
  if (!(det > 0)) { atomicOr(status, 1); return; }
  double Ji[3][3];
  lorg::inv_dd(dim, J, det, Ji);
  const double w = glw[qx] * glw[qy] * (dim == 3 ? glw[qz] : 1.0);
  const double s = (bq ? bq[gid] : kappa[e]) * w * det;
  const int ncomp = dim == 3 ? 6 : 3;
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  const int ja[3] = {0, 0, 1}, jb[3] = {0, 1, 1};
  for (int cpt = 0; cpt < ncomp; ++cpt) {
    const int a = dim == 3 ? ia[cpt] : ja[cpt], b = dim == 3 ? ib[cpt] : jb[cpt];
    double g = 0;
    for (int t = 0; t < dim; ++t) g += Ji[a][t] * Ji[b][t];
    const long long o = e * ncomp * Qd + (long long)cpt * Qd + q;
    G64[o] = s * g;
    G32[o] = (float)(s * g);
  }
}

// Curved (isoparametric) elements: G as k_geom, with J at each Gauss point from the
// degree-p interpolant of the element's GLL node coordinates X (SoA dim x ntot):
// J[a][b] = sum_n X_a(n) d(phi_n)/d(xi_b), phi_n the tensor GLL Lagrange basis.
// B, D: the 1D basis and its derivative at the Gauss points ([q][i], Q x Q).
__global__ void k_geom_iso(int dim, int p, int nx, int ny, int nz, const double* __restrict__ X,
                           const double* __restrict__ kappa, const double* __restrict__ B,
                           const double* __restrict__ D, const double* __restrict__ glw, double* __restrict__ G64,
                           float* __restrict__ G32, int* status) {
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
  double Xq[3], J[3][3];
  lorg::iso_map(dim, p, ex, ey, ez, qx, qy, qz, Nx, Ny, ntot, X, B, D, Xq, J);
  const double det = dim == 3 ? lorg::det3(J) : (J[0][0] * J[1][1] - J[0][1] * J[1][0]);
  if (!(det > 0)) { atomicOr(status, 1); return; }
  double Ji[3][3];
  lorg::inv_dd(dim, J, det, Ji);
  const double w = glw[qx] * glw[qy] * (dim == 3 ? glw[qz] : 1.0);
  const double s = kappa[e] * w * det;
  const int ncomp = dim == 3 ? 6 : 3;
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  const int ja[3] = {0, 0, 1}, jb[3] = {0, 1, 1};
  for (int cpt = 0; cpt < ncomp; ++cpt) {
    const int a = dim == 3 ? ia[cpt] : ja[cpt], b = dim == 3 ? ib[cpt] : jb[cpt];
    double gsum = 0;
    for (int t = 0; t < dim; ++t) gsum += Ji[a][t] * Ji[b][t];
    const long long o = e * ncomp * Qd + (long long)cpt * Qd + q;
    G64[o] = s * gsum;
    G32[o] = (float)(s * gsum);
  }
}

// physical coordinates of every level-0 node: element map at the GLL point
__global__ void k_nodes(int dim, int p, int nx, int ny, int nz, const double* __restrict__ vert,
                        const double* __restrict__ gllx, double* __restrict__ X) {
  const int Nx = nx * p + 1, Ny = ny * p + 1, Nz = dim == 3 ? nz * p + 1 : 1;
  const long long ntot = (long long)Nx * Ny * Nz;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= ntot) return;
  const int I = (int)(gid % Nx), Jn = (int)((gid / Nx) % Ny), K = (int)(gid / ((long long)Nx * Ny));
  const int ex = min(I / p, nx - 1), ey = min(Jn / p, ny - 1), ez = dim == 3 ? min(K / p, nz - 1) : 0;
  const double xi[3] = {gllx[I - ex * p], gllx[Jn - ey * p], dim == 3 ? gllx[K - ez * p] : 0.0};
  const long long NV = (long long)(nx + 1) * (ny + 1) * (dim == 3 ? (nz + 1) : 1);
  double Pc[8][3];
  lorg::element_corners(dim, nx, ny, ex, ey, ez, vert, NV, Pc);
  double Xp[3], J[3][3];
  lorg::multilinear(dim, Pc, xi, Xp, J);
  for (int a = 0; a < dim; ++a) X[a * ntot + gid] = Xp[a];
}

// K_h stencil row of every level-0 node (all 2^d sub-cells around it).
// bh (optional): the coefficient at the 2^d Gauss points of every sub-cell
// ([cell][g], cells x fastest, g = gx + 2 gy + 4 gz) in place of the parent's kappa.
__global__ void k_lor_stencil(int dim, int p, int nx, int ny, int nz, const double* __restrict__ X,
                              const double* __restrict__ kappa, const double* __restrict__ bh,
                              double* __restrict__ S) {
  const int Nx = nx * p + 1, Ny = ny * p + 1, Nz = dim == 3 ? nz * p + 1 : 1;
  const long long ntot = (long long)Nx * Ny * Nz;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= ntot) return;
  const int NS = dim == 3 ? 27 : 9;
  const int I = (int)(gid % Nx), Jn = (int)((gid / Nx) % Ny), K = (int)(gid / ((long long)Nx * Ny));
  double acc[27];
  for (int o = 0; o < 27; ++o) acc[o] = 0.0;
  const double gq = 0.5 - 0.5 / sqrt(3.0);
  const double g1[2] = {gq, 1.0 - gq};
  const int ncz = dim == 3 ? 2 : 1;
  for (int cz = 0; cz < ncz; ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        // cell with origin (I-1+cx, Jn-1+cy, K-1+cz); this node is its corner (1-cx, 1-cy, 1-cz)
        const int ox = I - 1 + cx, oy = Jn - 1 + cy, oz = dim == 3 ? K - 1 + cz : 0;
        if (ox < 0 || ox > Nx - 2 || oy < 0 || oy > Ny - 2) continue;
        if (dim == 3 && (oz < 0 || oz > Nz - 2)) continue;
        const int me = (1 - cx) + 2 * (1 - cy) + (dim == 3 ? 4 * (1 - cz) : 0);
        double Pc[8][3];
        const int nc = 1 << dim;
        for (int t = 0; t < nc; ++t) {
          const long long nid = ((long long)(oz + ((t >> 2) & 1)) * Ny + (oy + ((t >> 1) & 1))) * Nx + (ox + (t & 1));
          for (int a = 0; a < 3; ++a) Pc[t][a] = a < dim ? X[a * ntot + nid] : 0.0;
        }
        const long long e = dim == 3 ? ((long long)(oz / p) * ny + oy / p) * nx + ox / p : (long long)(oy / p) * nx + ox / p;
        const double kap = kappa[e];
        const int ngz = dim == 3 ? 2 : 1;
        for (int gz = 0; gz < ngz; ++gz)
          for (int gy = 0; gy < 2; ++gy)
            for (int gx = 0; gx < 2; ++gx) {
              const double xi[3] = {g1[gx], g1[gy], dim == 3 ? g1[gz] : 0.0};
              double Xq[3], J[3][3];
              lorg::multilinear(dim, Pc, xi, Xq, J);
              const double det = dim == 3 ? lorg::det3(J) : (J[0][0] * J[1][1] - J[0][1] * J[1][0]);
              double Ji[3][3];
              lorg::inv_dd(dim, J, det, Ji);
              const double bv =
                  bh ? bh[(((long long)oz * (Ny - 1) + oy) * (Nx - 1) + ox) * nc + (gz * 4 + gy * 2 + gx)] : kap;
              const double wq = (dim == 3 ? 0.125 : 0.25) * fabs(det) * bv;
              // reference gradients of the corner functions
              double gme[3];
              double gref[8][3];
              for (int t = 0; t < nc; ++t) {
                double f[3], df[3];
                for (int a = 0; a < 3; ++a) {
                  const int bit = (t >> a) & 1;
                  f[a] = bit ? xi[a] : 1.0 - xi[a];
                  df[a] = bit ? 1.0 : -1.0;
                }
                for (int bb = 0; bb < dim; ++bb) {
                  double g = 1.0;
                  for (int a = 0; a < dim; ++a) g *= (a == bb) ? df[a] : f[a];
                  gref[t][bb] = g;
                }
              }
              // physical gradient J^{-T} gref
              double gph[8][3];
              for (int t = 0; t < nc; ++t)
                for (int a = 0; a < dim; ++a) {
                  double s = 0;
                  for (int bb = 0; bb < dim; ++bb) s += Ji[bb][a] * gref[t][bb];
                  gph[t][a] = s;
                }
              for (int a = 0; a < dim; ++a) gme[a] = gph[me][a];
              for (int t = 0; t < nc; ++t) {
                double d = 0;
                for (int a = 0; a < dim; ++a) d += gme[a] * gph[t][a];
                const int dx = ox + (t & 1) - I, dy = oy + ((t >> 1) & 1) - Jn, dz = dim == 3 ? oz + ((t >> 2) & 1) - K : 0;
                const int o = dim == 3 ? (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1) : (dy + 1) * 3 + (dx + 1);
                acc[o] += wq * d;
              }
            }
      }
  for (int o = 0; o < NS; ++o) S[(long long)o * ntot + gid] = acc[o];
}

// Galerkin coarse stencil A_c = P^T A_f P on structured grids with tensor 1D P.
// Pf: per axis, per fine index: coarse (c0,w0,c1,w1); R: per axis CSR coarse -> fine.
struct GalerkinArgs {
  int dim;
  int Nf[3], Nc[3];
  const Prolong1D* Pf[3];
  const int* Rptr[3];
  const int* Ridx[3];
  const double* Rw[3];
};

__global__ void k_galerkin(GalerkinArgs g, const double* __restrict__ Sf, double* __restrict__ Sc) {
  const long long ntc = (long long)g.Nc[0] * g.Nc[1] * g.Nc[2];
  const long long ntf = (long long)g.Nf[0] * g.Nf[1] * g.Nf[2];
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= ntc) return;
  const int dim = g.dim;
  const int NS = dim == 3 ? 27 : 9;
  const int C[3] = {(int)(gid % g.Nc[0]), (int)((gid / g.Nc[0]) % g.Nc[1]), (int)(gid / ((long long)g.Nc[0] * g.Nc[1]))};
  double acc[27];
  for (int o = 0; o < 27; ++o) acc[o] = 0.0;
  const int zlo = dim == 3 ? g.Rptr[2][C[2]] : 0, zhi = dim == 3 ? g.Rptr[2][C[2] + 1] : 1;
  for (int iz = zlo; iz < zhi; ++iz) {
    const int fz = dim == 3 ? g.Ridx[2][iz] : 0;
    const double wz = dim == 3 ? g.Rw[2][iz] : 1.0;
    for (int iy = g.Rptr[1][C[1]]; iy < g.Rptr[1][C[1] + 1]; ++iy) {
      const int fy = g.Ridx[1][iy];
      const double wy = g.Rw[1][iy];
      for (int ix = g.Rptr[0][C[0]]; ix < g.Rptr[0][C[0] + 1]; ++ix) {
        const int fx = g.Ridx[0][ix];
        const double wi = g.Rw[0][ix] * wy * wz;
        const long long fi = ((long long)fz * g.Nf[1] + fy) * g.Nf[0] + fx;
        for (int o = 0; o < NS; ++o) {
          const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = dim == 3 ? o / 9 - 1 : 0;
          const int jx = fx + dx, jy = fy + dy, jz = fz + dz;
          if (jx < 0 || jx >= g.Nf[0] || jy < 0 || jy >= g.Nf[1]) continue;
          if (dim == 3 && (jz < 0 || jz >= g.Nf[2])) continue;
          const double a = Sf[(long long)o * ntf + fi];
          if (a == 0.0) continue;
          const Prolong1D px = g.Pf[0][jx], py = g.Pf[1][jy];
          Prolong1D pz;
          if (dim == 3) pz = g.Pf[2][jz]; else { pz.c0 = 0; pz.w0 = 1.0; pz.c1 = -1; pz.w1 = 0.0; }
          for (int sz = 0; sz < 2; ++sz) {
            const int cz = sz ? pz.c1 : pz.c0;
            const double vz = sz ? pz.w1 : pz.w0;
            if (cz < 0) continue;
            for (int sy = 0; sy < 2; ++sy) {
              const int cy = sy ? py.c1 : py.c0;
              const double vy = sy ? py.w1 : py.w0;
              if (cy < 0) continue;
              for (int sx = 0; sx < 2; ++sx) {
                const int cx = sx ? px.c1 : px.c0;
                const double vx = sx ? px.w1 : px.w0;
                if (cx < 0) continue;
                const int ox = cx - C[0], oy = cy - C[1], oz = dim == 3 ? cz - C[2] : 0;
                const int oc = dim == 3 ? (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1) : (oy + 1) * 3 + (ox + 1);
                acc[oc] += wi * a * vx * vy * vz;
              }
            }
          }
        }
      }
    }
  }
  for (int o = 0; o < NS; ++o) Sc[(long long)o * ntc + gid] = acc[o];
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// Row-major copy of a stencil: Sa[g * nsp + o] = S[o * ntot + g], zero padded.
template <typename T>
__global__ void k_stencil_rows(const T* __restrict__ S, T* __restrict__ Sa, long long ntot, int NS, int nsp) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ntot) return;
  for (int o = 0; o < nsp; ++o) Sa[g * nsp + o] = o < NS ? S[(long long)o * ntot + g] : T(0);
}

// Factor records to FP32 / bf16: values rounded, the index slot (rec-1) copied
// as raw integer bits.
__global__ void k_fac_to32(const double* __restrict__ a, float* __restrict__ b, long long n, int rec) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  b[i] = (i % rec == rec - 1) ? __int_as_float((int)__double_as_longlong(a[i])) : (float)a[i];
}

__global__ void k_fac_to16(const double* __restrict__ a, __nv_bfloat16* __restrict__ b, long long n, int rec) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i % rec == rec - 1) {
    __nv_bfloat16_raw raw;
    raw.x = (unsigned short)__double_as_longlong(a[i]);
    b[i] = __nv_bfloat16(raw);
  } else {
    b[i] = __double2bfloat16(a[i]);
  }
}

// ILU(0) of every patch at one level.  One CTA per patch; rows in wavefront order.
struct IluArgs {
  int dim, NS;
  int n[3];            // elements per direction
  int m;               // intervals per element at this level
  int N[3];            // level grid
  const BoxShape* shapes;   // 8 shapes of this level
  const int* rowlex;
  const int* recof;
  const int* front;
  const int* poslex;   // lex -> pos, per shape (offset = shape.row_off)
  const long long* facoff;  // this level's record offsets [J]
  const double* S;
  double* F;
  int* status;
};

__device__ inline void patch_vertex(int j, const int* n, int dim, int* v) {
  v[0] = j % (n[0] + 1);
  v[1] = (j / (n[0] + 1)) % (n[1] + 1);
  v[2] = dim == 3 ? j / ((n[0] + 1) * (n[1] + 1)) : 0;
}

__global__ void k_ilu0(IluArgs a) {
  const int j = blockIdx.x;
  int v[3];
  patch_vertex(j, a.n, a.dim, v);
  int sh = 0;
  for (int t = 0; t < a.dim; ++t) sh |= ((v[t] == 0 || v[t] == a.n[t]) ? 1 : 0) << t;
  const BoxShape bs = a.shapes[sh];
  if (bs.rows == 0) return;
  const int dx0 = bs.dims[0], dy0 = bs.dims[1], dz0 = bs.dims[2];
  int org[3];
  for (int t = 0; t < 3; ++t) org[t] = (t < a.dim) ? (v[t] > 0 ? v[t] - 1 : 0) * a.m + 1 : 0;
  const long long ntot = (long long)a.N[0] * a.N[1] * a.N[2];
  const int R = lor_rec(a.dim);
  double* FL = a.F + a.facoff[j] * R;           // L records
  double* FU = FL + (long long)bs.rpad * R;      // U records
  // index slot of every record: padding records point at the guard cell after the box
  for (int q = threadIdx.x; q < bs.rpad; q += blockDim.x) {
    FL[(long long)q * R + R - 1] = __longlong_as_double((long long)bs.rows);
    FU[(long long)q * R + R - 1] = __longlong_as_double((long long)bs.rows);
  }
  __syncthreads();
  const int* rowlex = a.rowlex + bs.row_off;
  const int* recof = a.recof + bs.row_off;
  const int* poslex = a.poslex + bs.row_off;
  const int* front = a.front + bs.front_off;
  const int NS = a.NS, C = NS / 2;
  for (int f = 0; f < bs.nfront; ++f) {
    for (int pos = front[f] + threadIdx.x; pos < front[f + 1]; pos += blockDim.x) {
      const int lex = rowlex[pos];
      const int i = lex % dx0, jj = (lex / dx0) % dy0, k = lex / (dx0 * dy0);
      const long long G = ((long long)(org[2] + k) * a.N[1] + (org[1] + jj)) * a.N[0] + (org[0] + i);
      double r[27];
      for (int o = 0; o < NS; ++o) {
        const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = a.dim == 3 ? o / 9 - 1 : 0;
        const int ni = i + ox, nj = jj + oy, nk = k + oz;
        const bool in = ni >= 0 && ni < dx0 && nj >= 0 && nj < dy0 && nk >= 0 && nk < dz0;
        r[o] = in ? a.S[(long long)o * ntot + G] : 0.0;
      }
      for (int o = 0; o < C; ++o) {            // lower neighbours, ascending column order
        const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = a.dim == 3 ? o / 9 - 1 : 0;
        const int ni = i + ox, nj = jj + oy, nk = k + oz;
        if (!(ni >= 0 && ni < dx0 && nj >= 0 && nj < dy0 && nk >= 0 && nk < dz0)) continue;
        const double* Uk = FU + (long long)recof[poslex[(nk * dy0 + nj) * dx0 + ni]] * R;
        const double l = r[o] * Uk[R - 2];   // a_ik / u_kk
        r[o] = l;
        for (int o2 = C + 1; o2 < NS; ++o2) {   // upper part of row k
          const int px = ox + (o2 % 3 - 1), py = oy + ((o2 / 3) % 3 - 1), pz = oz + (a.dim == 3 ? o2 / 9 - 1 : 0);
          if (px < -1 || px > 1 || py < -1 || py > 1 || pz < -1 || pz > 1) continue;
          const int ot = a.dim == 3 ? (pz + 1) * 9 + (py + 1) * 3 + (px + 1) : (py + 1) * 3 + (px + 1);
          r[ot] -= l * Uk[o2 - C - 1];
        }
      }
      if (!(r[C] > 0.0)) atomicOr(a.status, 2);
      double* Li = FL + (long long)recof[pos] * R;
      double* Ui = FU + (long long)recof[pos] * R;
      for (int o = 0; o < R - 1; ++o) {
        Li[o] = o < C ? r[o] : 0.0;
        Ui[o] = o < C ? r[C + 1 + o] : 0.0;
      }
      Ui[R - 2] = 1.0 / r[C];
      Li[R - 1] = __longlong_as_double((long long)lex);
      Ui[R - 1] = __longlong_as_double((long long)lex);
    }
    __syncthreads();
  }
}

// l1 row sums over interior neighbours, inverted; boundary rows get 0.
__global__ void k_l1_dinv(int dim, int Nx, int Ny, int Nz, const double* __restrict__ S, double* __restrict__ D64,
                          float* __restrict__ D32) {
  const long long ntot = (long long)Nx * Ny * Nz;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= ntot) return;
  const int I = (int)(gid % Nx), Jn = (int)((gid / Nx) % Ny), K = (int)(gid / ((long long)Nx * Ny));
  const bool bnd = I == 0 || I == Nx - 1 || Jn == 0 || Jn == Ny - 1 || (dim == 3 && (K == 0 || K == Nz - 1));
  double s = 0;
  const int NS = dim == 3 ? 27 : 9;
  if (!bnd) {
    for (int o = 0; o < NS; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = dim == 3 ? o / 9 - 1 : 0;
      const int a = I + dx, b = Jn + dy, c = K + dz;
      const bool nb = a == 0 || a == Nx - 1 || b == 0 || b == Ny - 1 || (dim == 3 && (c == 0 || c == Nz - 1));
      if (!nb) s += fabs(S[(long long)o * ntot + gid]);
    }
  }
  const double di = bnd ? 0.0 : 1.0 / s;
  D64[gid] = di;
  D32[gid] = (float)di;
}

}  // namespace

// ============================================================== host-side setup
static lor_status upload(lor_ctx* c, void** dst, const void* src, size_t bytes) {
  *dst = lor_alloc(c, bytes);
  if (!*dst) return lor_fail(c, LOR_ENOMEM, "device allocation failed");
  return lor_cuda_check(c, cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, c->stream), "upload");
}

static lor_status check_status(lor_ctx* c, const char* what) {
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, what);
  if (st & 1) return lor_fail(c, LOR_EINVAL, "inverted element: det J <= 0 at a quadrature point");
  if (st & 2) return lor_fail(c, LOR_EBREAKDOWN, "ILU(0) breakdown: non-positive pivot");
  return LOR_OK;
}

lor_status lor_setup_geometry(lor_ctx* c) {
  const int p = c->p, Q = p + 1;
  // basis block (allocation 0: doubles, allocation 1: floats)
  std::vector<double> h64(6 * kBlk, 0.0);
  std::vector<float> h32(2 * kBlk, 0.0f);
  lorh::gll(p, c->gll_x, c->gll_w);
  lorh::gauss(Q, c->gl_x, c->gl_w);
  double Dn[(LOR_MAXP + 2) * (LOR_MAXP + 2)];
  lorh::lagrange(Q, c->gll_x, Q, c->gl_x, c->B, Dn);          // B[q][i] at Gauss points
  double Bg[(LOR_MAXP + 2) * (LOR_MAXP + 2)];
  lorh::lagrange(Q, c->gl_x, Q, c->gl_x, Bg, c->Dq);          // Gauss-nodal differentiation
  for (int i = 0; i < Q * Q; ++i) {
    h64[0 * kBlk + i] = c->B[i];
    h64[1 * kBlk + i] = c->Dq[i];
    h64[5 * kBlk + i] = Dn[i];
    h32[0 * kBlk + i] = (float)c->B[i];
    h32[1 * kBlk + i] = (float)c->Dq[i];
  }
  for (int i = 0; i < Q; ++i) {
    h64[2 * kBlk + i] = c->gl_x[i];
    h64[3 * kBlk + i] = c->gl_w[i];
    h64[4 * kBlk + i] = c->gll_x[i];
  }
  void* d;
  if (upload(c, &d, h64.data(), h64.size() * 8)) return LOR_ENOMEM;
  if (upload(c, &d, h32.data(), h32.size() * 4)) return LOR_ENOMEM;
  c->d_status = (int*)lor_alloc(c, 64);
  if (!c->d_status) return lor_fail(c, LOR_ENOMEM, "alloc status");
  cudaMemsetAsync(c->d_status, 0, 64, c->stream);
  // mesh
  if (upload(c, (void**)&c->d_vert, c->h_vert.data(), c->h_vert.size() * 8)) return LOR_ENOMEM;
  if (upload(c, (void**)&c->d_kappa, c->h_kappa.data(), c->h_kappa.size() * 8)) return LOR_ENOMEM;
  if (!c->h_bq.empty()) {   // pointwise coefficient (lor_set_coefficient)
    if (upload(c, (void**)&c->d_bq, c->h_bq.data(), c->h_bq.size() * 8)) return LOR_ENOMEM;
    if (upload(c, (void**)&c->d_bh, c->h_bh.data(), c->h_bh.size() * 8)) return LOR_ENOMEM;
  }
  // geometric factors
  const int Qd = c->dim == 3 ? Q * Q * Q : Q * Q;
  const int ncomp = c->dim == 3 ? 6 : 3;
  const long long ng = (long long)c->nel * ncomp * Qd;
  c->d_G64 = (double*)lor_alloc(c, ng * 8);
  c->d_G32 = (float*)lor_alloc(c, ng * 4);
  if (!c->d_G64 || !c->d_G32) return lor_fail(c, LOR_ENOMEM, "alloc geometric factors");
  const long long tot = (long long)c->nel * Qd;
  if (!c->h_nodes.empty()) {
    // curved elements (lor_set_node_coordinates): the GLL node coordinates are given;
    // the stencil setup uses them as they are, and K_p takes its isoparametric map
    if (upload(c, (void**)&c->d_X, c->h_nodes.data(), c->h_nodes.size() * 8)) return LOR_ENOMEM;
    k_geom_iso<<<(unsigned)lor_ceil_div(tot, 128), 128, 0, c->stream>>>(
        c->dim, p, c->n[0], c->n[1], c->n[2], c->d_X, c->d_kappa, lor_basis64(c, 0), lor_basis64(c, 5),
        lor_basis64(c, 3), c->d_G64, c->d_G32, c->d_status);
  } else {
    k_geom<<<(unsigned)lor_ceil_div(tot, 128), 128, 0, c->stream>>>(
        c->dim, p, c->n[0], c->n[1], c->n[2], c->d_vert, c->d_kappa, c->d_bq, lor_basis64(c, 2),
        lor_basis64(c, 3), c->d_G64, c->d_G32, c->d_status);
  }
  ++c->launches;
  if (lor_cuda_check(c, cudaGetLastError(), "geometry")) return LOR_ECUDA;
  return check_status(c, "geometry");
}

// 1D global prolongation (level l+1 -> l) of one axis with nel elements:
// linear interpolation in the element reference coordinate (GLL positions).
static std::vector<Prolong1D> prolong_axis(int nel, const double* gllx, const std::vector<int>& sf,
                                           const std::vector<int>& sc) {
  const int mf = (int)sf.size() - 1, mc = (int)sc.size() - 1;
  std::vector<Prolong1D> P(nel * mf + 1);
  for (int e = 0; e < nel; ++e)
    for (int t = 0; t <= mf; ++t) {
      const int g = sf[t];
      int a = 0;
      while (a + 1 <= mc && sc[a + 1] <= g) ++a;
      Prolong1D pr;
      if (sc[a] == g) { pr.c0 = e * mc + a; pr.w0 = 1.0; pr.c1 = -1; pr.w1 = 0.0; }
      else {
        const double w = (gllx[g] - gllx[sc[a]]) / (gllx[sc[a + 1]] - gllx[sc[a]]);
        pr.c0 = e * mc + a; pr.w0 = 1.0 - w; pr.c1 = e * mc + a + 1; pr.w1 = w;
      }
      P[e * mf + t] = pr;
    }
  return P;
}

// coarse-vertex-grid 1D coarsening (keep even positions + last), index-space weights
static std::vector<Prolong1D> prolong_index(int nf, int* nc_out) {
  std::vector<int> keep;
  for (int i = 0; i < nf; i += 2) keep.push_back(i);
  if (keep.back() != nf - 1) keep.push_back(nf - 1);
  *nc_out = (int)keep.size();
  std::vector<Prolong1D> P(nf);
  for (int i = 0; i < nf; ++i) {
    int b = 0;
    while (keep[b] < i) ++b;
    Prolong1D pr;
    if (keep[b] == i) { pr.c0 = b; pr.w0 = 1.0; pr.c1 = -1; pr.w1 = 0.0; }
    else {
      const double w = double(i - keep[b - 1]) / double(keep[b] - keep[b - 1]);
      pr.c0 = b - 1; pr.w0 = 1.0 - w; pr.c1 = b; pr.w1 = w;
    }
    P[i] = pr;
  }
  return P;
}

// transpose of a 1D prolongation as CSR (coarse -> list of fine with weights)
static void restrict_csr(const std::vector<Prolong1D>& P, int nc, std::vector<int>& ptr, std::vector<int>& idx,
                         std::vector<double>& w) {
  std::vector<std::vector<std::pair<int, double>>> rows(nc);
  for (int f = 0; f < (int)P.size(); ++f) {
    if (P[f].c0 >= 0 && P[f].w0 != 0.0) rows[P[f].c0].push_back({f, P[f].w0});
    if (P[f].c1 >= 0 && P[f].w1 != 0.0) rows[P[f].c1].push_back({f, P[f].w1});
  }
  ptr.assign(nc + 1, 0);
  idx.clear();
  w.clear();
  for (int cidx = 0; cidx < nc; ++cidx) {
    for (auto& pr : rows[cidx]) { idx.push_back(pr.first); w.push_back(pr.second); }
    ptr[cidx + 1] = (int)idx.size();
  }
}

static lor_status upload_prolong(lor_ctx* c, const std::vector<Prolong1D>& P, int nc, Prolong1D** dP, int** dptr,
                                 int** didx, double** dw) {
  std::vector<int> ptr, idx;
  std::vector<double> w;
  restrict_csr(P, nc, ptr, idx, w);
  if (upload(c, (void**)dP, P.data(), P.size() * sizeof(Prolong1D))) return LOR_ENOMEM;
  if (upload(c, (void**)dptr, ptr.data(), ptr.size() * 4)) return LOR_ENOMEM;
  if (upload(c, (void**)didx, idx.data(), std::max<size_t>(1, idx.size()) * 4)) return LOR_ENOMEM;
  if (upload(c, (void**)dw, w.data(), std::max<size_t>(1, w.size()) * 8)) return LOR_ENOMEM;
  return LOR_OK;
}

static lor_status galerkin(lor_ctx* c, int dim, const int* Nf, const int* Nc, Prolong1D* const* P,
                           int* const* Rptr, int* const* Ridx, double* const* Rw, const double* Sf, double* Sc) {
  GalerkinArgs g;
  g.dim = dim;
  for (int a = 0; a < 3; ++a) {
    g.Nf[a] = Nf[a]; g.Nc[a] = Nc[a];
    g.Pf[a] = P[a]; g.Rptr[a] = Rptr[a]; g.Ridx[a] = Ridx[a]; g.Rw[a] = Rw[a];
  }
  const long long ntc = (long long)Nc[0] * Nc[1] * Nc[2];
  k_galerkin<<<(unsigned)lor_ceil_div(ntc, 128), 128, 0, c->stream>>>(g, Sf, Sc);
  ++c->launches;
  return lor_cuda_check(c, cudaGetLastError(), "galerkin");
}

lor_status lor_setup_stencils(lor_ctx* c) {
  const int dim = c->dim, p = c->p;
  c->NS = dim == 3 ? 27 : 9;
  c->sel = lorh::level_selections(p, c->opt.mg_levels);
  c->L = (int)c->sel.size();
  if (c->L > LOR_MAXLEV) return lor_fail(c, LOR_EINVAL, "too many levels");
  for (int l = 0; l < c->L; ++l) {
    LevelGrid& g = c->lev[l];
    g.m = (int)c->sel[l].size() - 1;
    for (int a = 0; a < 3; ++a) g.N[a] = a < dim ? c->n[a] * g.m + 1 : 1;
    g.ntot = (long long)g.N[0] * g.N[1] * g.N[2];
  }
  const long long nt0 = c->lev[0].ntot;
  if (!c->d_X) {   // multilinear elements: the element map at the GLL points (curved: given)
    c->d_X = (double*)lor_alloc(c, nt0 * dim * 8);
    if (!c->d_X) return lor_fail(c, LOR_ENOMEM, "alloc coordinates");
    k_nodes<<<(unsigned)lor_ceil_div(nt0, 128), 128, 0, c->stream>>>(dim, p, c->n[0], c->n[1], c->n[2], c->d_vert,
                                                                       lor_basis64(c, 4), c->d_X);
    ++c->launches;
  }
  for (int l = 0; l < c->L; ++l) {
    const long long nt = c->lev[l].ntot;
    c->d_S64[l] = (double*)lor_alloc(c, nt * c->NS * 8);
    c->d_S32[l] = (float*)lor_alloc(c, nt * c->NS * 4);
    if (!c->d_S64[l] || !c->d_S32[l]) return lor_fail(c, LOR_ENOMEM, "alloc stencils");
  }
  k_lor_stencil<<<(unsigned)lor_ceil_div(nt0, 128), 128, 0, c->stream>>>(dim, p, c->n[0], c->n[1], c->n[2], c->d_X,
                                                                           c->d_kappa, c->d_bh, c->d_S64[0]);
  ++c->launches;
  if (lor_cuda_check(c, cudaGetLastError(), "lor stencil")) return LOR_ECUDA;
  for (int l = 0; l + 1 < c->L; ++l) {
    for (int a = 0; a < dim; ++a) {
      std::vector<Prolong1D> P = prolong_axis(c->n[a], c->gll_x, c->sel[l], c->sel[l + 1]);
      if (upload_prolong(c, P, c->lev[l + 1].N[a], &c->d_P1[l][a], &c->d_R1ptr[l][a], &c->d_R1idx[l][a],
                         &c->d_R1w[l][a]))
        return LOR_ENOMEM;
    }
    if (galerkin(c, dim, c->lev[l].N, c->lev[l + 1].N, c->d_P1[l], c->d_R1ptr[l], c->d_R1idx[l], c->d_R1w[l],
                 c->d_S64[l], c->d_S64[l + 1]))
      return LOR_ECUDA;
  }
  for (int l = 0; l < c->L; ++l) {
    const long long n = c->lev[l].ntot * c->NS;
    k_to_float<<<(unsigned)lor_ceil_div(n, 256), 256, 0, c->stream>>>(c->d_S64[l], c->d_S32[l], n);
    ++c->launches;
  }
  // row-major copies for the patch residuals
  if (c->lev[0].ntot >= (1LL << 31)) return lor_fail(c, LOR_EINVAL, "level-0 grid too large");
  for (int l = 0; l < c->L; ++l) {
    const long long nt = c->lev[l].ntot;
    c->d_SA64[l] = (double*)lor_alloc(c, nt * lor_nsp(dim) * 8);
    c->d_SA32[l] = (float*)lor_alloc(c, nt * lor_nsp(dim) * 4);
    if (!c->d_SA64[l] || !c->d_SA32[l]) return lor_fail(c, LOR_ENOMEM, "alloc row stencils");
    k_stencil_rows<double><<<(unsigned)lor_ceil_div(nt, 256), 256, 0, c->stream>>>(c->d_S64[l], c->d_SA64[l], nt,
                                                                                    c->NS, lor_nsp(dim));
    k_stencil_rows<float><<<(unsigned)lor_ceil_div(nt, 256), 256, 0, c->stream>>>(c->d_S32[l], c->d_SA32[l], nt,
                                                                                   c->NS, lor_nsp(dim));
    c->launches += 2;
  }
  return lor_cuda_check(c, cudaGetLastError(), "stencil conversion");
}

// ------------------------------------------------------------ patch structures
static int axis_len(int type, int m) { return type == 0 ? 2 * m - 1 : m - 1; }
// bulk-copy chunk of factor records per element size (2, 4, 8 bytes); a wider
// front is a chunk of its own
static const int kChunkBytes[3] = {4096, 4096, 8192};

// Factors of algebraically ordered patch levels (RCM or MDF, Section 3.4), built on
// the host: per patch and level the box matrix from the level stencil, the
// ordering, ILU(0) in that order, the dependency levels of the order (fronts of at
// most 32 rows) and the records (lor_rec_gen layout).  Patches are spread over the
// host threads; the permutations are kept for lor_patch_ordering.
static lor_status setup_ordered_factors(lor_ctx* c) {
  const int dim = c->dim, NS = c->NS, C = NS / 2, R = lor_rec_gen(dim), L = c->L, J = c->J;
  std::vector<std::vector<double>> hS(L);
  for (int l = 0; l < L; ++l) {
    hS[l].resize((size_t)NS * c->lev[l].ntot);
    cudaError_t e = cudaMemcpyAsync(hS[l].data(), c->d_S64[l], hS[l].size() * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return lor_cuda_check(c, e, "ordered factors: stencil copy");
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "ordered factors: stencil copy");
  struct Out {
    std::vector<double> rec;             // 2 * rpad records (L part, then U part)
    std::vector<int> fpad;               // record offset of every front (nfront + 1)
    std::vector<int> chunk[3];           // front index of every chunk start (nchunk + 1)
    int nfront = 0, rpad = 0, rows = 0;
    bool ok = true;
  };
  std::vector<Out> out((size_t)L * J);
  c->h_perm.assign((size_t)L * J, std::vector<int>());
  // box of every patch at every level: the elements e0 .. e1-1 of its span along
  // each axis (the vertex patch: one element on each side of the vertex), the open
  // interior of those elements at the level's resolution
  std::vector<GenSched> gs((size_t)L * J);
  for (int l = 0; l < L; ++l)
    for (int j = 0; j < J; ++j) {
      GenSched& g = gs[(size_t)l * J + j];
      std::memset(&g, 0, sizeof(g));
      const int v[3] = {j % (c->n[0] + 1), (j / (c->n[0] + 1)) % (c->n[1] + 1),
                        dim == 3 ? j / ((c->n[0] + 1) * (c->n[1] + 1)) : 0};
      const int m = c->lev[l].m;
      g.rows = 1;
      for (int a = 0; a < 3; ++a) {
        if (a >= dim) { g.dims[a] = 1; g.org[a] = 0; g.k[a] = 1; continue; }
        const int lo = c->h_spans.empty() ? 1 : c->h_spans[((size_t)j * dim + a) * 2];
        const int hi = c->h_spans.empty() ? 1 : c->h_spans[((size_t)j * dim + a) * 2 + 1];
        const int e0 = std::max(v[a] - lo, 0), e1 = std::min(v[a] + hi, c->n[a]);
        g.k[a] = e1 - e0;
        g.dims[a] = std::max(g.k[a] * m - 1, 0);
        g.org[a] = e0 * m + 1;
        g.rows *= g.dims[a];
      }
      g.guard = g.dims[0] * g.dims[1] + g.dims[0] + 1;
    }
  // RCM depends on the pattern only: one permutation per box extent
  std::map<std::array<int, 3>, std::vector<int>> rcm;
  if (c->ordering == 1)
    for (int l = 0; l + 1 < L; ++l)
      for (int j = 0; j < J; ++j) {
        const GenSched& g = gs[(size_t)l * J + j];
        const std::array<int, 3> key = {g.dims[0], g.dims[1], g.dims[2]};
        if (g.rows && !rcm.count(key)) lorh::rcm_box(dim, key[0], key[1], key[2], rcm[key]);
      }
  // vertex level: the inverse of the box matrix of every patch with more than one row
  // there (an enlarged patch keeps several vertices on its coarsest level)
  std::vector<std::vector<double>> binv(J);
  std::atomic<long long> next(0);
  const long long ntask = (long long)L * J;
  auto work = [&]() {
    for (;;) {
      const long long task = next++;
      if (task >= ntask) return;
      const int l = (int)(task / J), j = (int)(task % J);
      const GenSched& gb = gs[(size_t)l * J + j];
      Out& o = out[(size_t)l * J + j];
      o.rows = gb.rows;
      o.fpad.assign(1, 0);
      for (int es = 0; es < 3; ++es) o.chunk[es].assign(1, 0);
      if (gb.rows == 0) continue;
      const int A = gb.dims[0], B = gb.dims[1], Cd = gb.dims[2], n = gb.rows;
      const LevelGrid& g = c->lev[l];
      const int* org = gb.org;
      std::vector<double> a27((size_t)n * NS, 0.0);
      for (int lex = 0; lex < n; ++lex) {
        const int i = lex % A, jj = (lex / A) % B, k = lex / (A * B);
        const long long G = ((long long)(org[2] + k) * g.N[1] + (org[1] + jj)) * g.N[0] + (org[0] + i);
        for (int q = 0; q < NS; ++q) {
          const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = dim == 3 ? q / 9 - 1 : 0;
          const int ni = i + dx, nj = jj + dy, nk = k + dz;
          if (ni >= 0 && ni < A && nj >= 0 && nj < B && nk >= 0 && nk < Cd)
            a27[(size_t)lex * NS + q] = hS[l][(size_t)q * g.ntot + G];
        }
      }
      if (l == L - 1) {   // vertex level: exact solve
        if (n > 1) {
          std::vector<double> M((size_t)n * n, 0.0), I((size_t)n * n, 0.0);
          for (int r = 0; r < n; ++r) {
            I[(size_t)r * n + r] = 1.0;
            const int x = r % A, y = (r / A) % B, z = r / (A * B);
            for (int q = 0; q < NS; ++q) {
              const double val = a27[(size_t)r * NS + q];
              if (val == 0.0) continue;
              const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = dim == 3 ? q / 9 - 1 : 0;
              M[(size_t)r * n + ((z + dz) * B + (y + dy)) * A + (x + dx)] = val;
            }
          }
          // Gauss-Jordan with partial pivoting (the box matrix is SPD)
          for (int col = 0; col < n && o.ok; ++col) {
            int piv = col;
            for (int r = col + 1; r < n; ++r)
              if (std::fabs(M[(size_t)r * n + col]) > std::fabs(M[(size_t)piv * n + col])) piv = r;
            if (!(std::fabs(M[(size_t)piv * n + col]) > 0.0)) { o.ok = false; break; }
            if (piv != col)
              for (int q = 0; q < n; ++q) {
                std::swap(M[(size_t)piv * n + q], M[(size_t)col * n + q]);
                std::swap(I[(size_t)piv * n + q], I[(size_t)col * n + q]);
              }
            const double d = 1.0 / M[(size_t)col * n + col];
            for (int q = 0; q < n; ++q) { M[(size_t)col * n + q] *= d; I[(size_t)col * n + q] *= d; }
            for (int r = 0; r < n; ++r) {
              if (r == col) continue;
              const double f = M[(size_t)r * n + col];
              if (f == 0.0) continue;
              for (int q = 0; q < n; ++q) {
                M[(size_t)r * n + q] -= f * M[(size_t)col * n + q];
                I[(size_t)r * n + q] -= f * I[(size_t)col * n + q];
              }
            }
          }
          binv[j] = I;
        }
        continue;
      }
      std::vector<int>& perm = c->h_perm[(size_t)l * J + j];
      if (c->ordering == 1) perm = rcm[{A, B, Cd}];
      else if (c->ordering == 0) { perm.resize(n); for (int q = 0; q < n; ++q) perm[q] = q; }
      else if (!lorh::mdf_box(dim, A, B, Cd, a27, perm)) { o.ok = false; continue; }
      std::vector<double> lu;
      std::vector<int> level;
      if (!lorh::ilu0_ordered(dim, A, B, Cd, a27, perm, lu, level)) { o.ok = false; continue; }
      std::vector<int> pos(n);
      for (int q = 0; q < n; ++q) pos[perm[q]] = q;
      int nlev = 0;
      for (int q = 0; q < n; ++q) nlev = std::max(nlev, level[q] + 1);
      std::vector<std::vector<int>> bylev(nlev);
      for (int q = 0; q < n; ++q) bylev[level[perm[q]]].push_back(perm[q]);
      std::vector<std::vector<int>> fronts;
      for (auto& lv : bylev)
        for (size_t s0 = 0; s0 < lv.size(); s0 += 32)
          fronts.emplace_back(lv.begin() + s0, lv.begin() + std::min(lv.size(), s0 + 32));
      int rec = 0;
      for (auto& f : fronts) { rec += (int)((f.size() + 3) / 4 * 4); o.fpad.push_back(rec); }
      o.nfront = (int)fronts.size();
      o.rpad = rec;
      o.rec.assign((size_t)2 * rec * R, 0.0);
      for (int q = 0; q < 2 * rec; ++q) {   // padding records: index = the guard cell after the box
        long long idx = n;
        std::memcpy(&o.rec[(size_t)q * R + R - 1], &idx, 8);
      }
      int q = 0;
      for (size_t fi = 0; fi < fronts.size(); ++fi) {
        q = o.fpad[fi];
        for (int i : fronts[fi]) {
          double* Lr = &o.rec[(size_t)q * R];
          double* Ur = &o.rec[(size_t)(rec + q) * R];
          const int x = i % A, y = (i / A) % B, z = i / (A * B);
          for (int s2 = 0; s2 < NS - 1; ++s2) {
            const int so = s2 < C ? s2 : s2 + 1;
            const int dx = so % 3 - 1, dy = (so / 3) % 3 - 1, dz = dim == 3 ? so / 9 - 1 : 0;
            const int X = x + dx, Y = y + dy, Z = z + dz;
            if (X < 0 || X >= A || Y < 0 || Y >= B || Z < 0 || Z >= Cd) continue;
            const int nbi = (Z * B + Y) * A + X;
            const double val = lu[(size_t)i * NS + so];
            if (pos[nbi] < pos[i]) Lr[s2] = val;
            else Ur[s2] = val;
          }
          Ur[R - 2] = 1.0 / lu[(size_t)i * NS + C];
          const long long idx = i;
          std::memcpy(&Lr[R - 1], &idx, 8);
          std::memcpy(&Ur[R - 1], &idx, 8);
          ++q;
        }
      }
      for (int es = 0; es < 3; ++es) {   // chunks of whole fronts, as for the wavefront records
        const int cap = kChunkBytes[es] / (R * (2 << es));
        int fa = 0;
        while (fa < o.nfront) {
          int fb = fa + 1;
          while (fb < o.nfront && o.fpad[fb + 1] - o.fpad[fa] <= cap) ++fb;
          o.chunk[es].push_back(fb);
          fa = fb;
        }
      }
    }
  };
  {
    const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int t = 0; t < nth; ++t) pool.emplace_back(work);
    for (auto& th : pool) th.join();
  }
  for (const Out& o : out)
    if (!o.ok) return lor_fail(c, LOR_EBREAKDOWN, "ordered ILU(0) breakdown: non-positive pivot");
  // concatenate: record offsets, schedules, front and chunk tables
  std::vector<long long> off((size_t)L * J);
  std::vector<int> gfpad, gchunk;
  long long tot = 0;
  c->gen_tab_ints = 0;
  for (int es = 0; es < 3; ++es) c->gen_maxchunk[es] = 0;
  std::vector<int> tab(J, 0);
  for (int l = 0; l < L; ++l)
    for (int j = 0; j < J; ++j) {
      const size_t t = (size_t)l * J + j;
      const Out& o = out[t];
      GenSched& g = gs[t];
      off[t] = tot;
      g.nfront = o.nfront;
      g.rpad = o.rpad;
      g.front_off = (int)gfpad.size();
      if (o.fpad.empty()) gfpad.push_back(0);
      else gfpad.insert(gfpad.end(), o.fpad.begin(), o.fpad.end());
      int maxc = 0;
      for (int es = 0; es < 3; ++es) {
        g.chunk_off[es] = (int)gchunk.size();
        if (o.chunk[es].empty()) { gchunk.push_back(0); g.nchunk[es] = 0; continue; }
        g.nchunk[es] = (int)o.chunk[es].size() - 1;
        gchunk.insert(gchunk.end(), o.chunk[es].begin(), o.chunk[es].end());
        for (int k = 0; k < g.nchunk[es]; ++k)
          c->gen_maxchunk[es] = std::max(c->gen_maxchunk[es], o.fpad[o.chunk[es][k + 1]] - o.fpad[o.chunk[es][k]]);
        maxc = std::max(maxc, g.nchunk[es]);
      }
      tab[j] += g.nfront + 1 + maxc + 1;
      tot += 2LL * o.rpad;
      if (l + 1 < L) c->fac_rows += o.rows;
    }
  for (int j = 0; j < J; ++j) c->gen_tab_ints = std::max(c->gen_tab_ints, tab[j]);
  // vertex-level inverses
  std::vector<double> hb;
  for (int j = 0; j < J; ++j) {
    GenSched& g = gs[(size_t)(L - 1) * J + j];
    g.binv_off = (long long)hb.size();
    hb.insert(hb.end(), binv[j].begin(), binv[j].end());
  }
  if (hb.empty()) hb.push_back(0.0);
  {
    std::vector<float> hb32(hb.begin(), hb.end());
    if (upload(c, (void**)&c->d_binv64, hb.data(), hb.size() * 8)) return LOR_ENOMEM;
    if (upload(c, (void**)&c->d_binv32, hb32.data(), hb32.size() * 4)) return LOR_ENOMEM;
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return lor_cuda_check(c, e, "vertex-level inverses");
  }
  // largest boxes (shared-memory layout of the patch kernel)
  c->gen_rows0 = c->gen_A0 = c->gen_AB0 = c->gen_rows1 = c->gen_guard0 = 0;
  c->gen_ovl = 0;
  c->span_kmax = 2;
  for (int j = 0; j < J; ++j) {
    const GenSched& g0 = gs[j];
    c->gen_rows0 = std::max(c->gen_rows0, g0.rows);
    c->gen_A0 = std::max(c->gen_A0, g0.dims[0]);
    c->gen_AB0 = std::max(c->gen_AB0, g0.dims[0] * g0.dims[1]);
    c->gen_guard0 = std::max(c->gen_guard0, g0.guard);
    if (L > 1) c->gen_rows1 = std::max(c->gen_rows1, gs[(size_t)J + j].rows);
    long long ovl = 0;
    for (int l = 1; l < L; ++l) {
      const GenSched& g = gs[(size_t)l * J + j];
      ovl += 2LL * (g.rows + 2 * g.guard + 1) + (l >= 2 ? g.rows : 0);
    }
    c->gen_ovl = std::max(c->gen_ovl, std::max<long long>(ovl, g0.rows + 2LL * g0.guard + 1));
    for (int a = 0; a < dim; ++a) c->span_kmax = std::max(c->span_kmax, g0.k[a]);
  }
  // patch-local 1D transfers for every level and span length k (1 .. kmax elements)
  {
    const int K1 = c->span_kmax + 1;
    std::vector<int> ib;              // int pool: c0 | c1 | rstart | rf per (l, k)
    std::vector<double> wb;           // weight pool: w0 | w1 | rw per (l, k)
    struct Off { size_t c0, c1, rs, rf, w0, w1, rw; };
    std::vector<Off> offs((size_t)L * K1, Off{0, 0, 0, 0, 0, 0, 0});
    for (int l = 0; l + 1 < L; ++l)
      for (int k = 1; k <= c->span_kmax; ++k) {
        const int m = c->lev[l].m, mc = c->lev[l + 1].m;
        std::vector<Prolong1D> P = prolong_axis(k, c->gll_x, c->sel[l], c->sel[l + 1]);
        const int len = std::max(k * m - 1, 0), clen = std::max(k * mc - 1, 0);
        Off& o = offs[(size_t)l * K1 + k];
        o.c0 = ib.size(); for (int f = 0; f < len; ++f) ib.push_back(P[f + 1].c0 >= 0 ? P[f + 1].c0 - 1 : -2);
        o.c1 = ib.size(); for (int f = 0; f < len; ++f) ib.push_back(P[f + 1].c1 >= 0 ? P[f + 1].c1 - 1 : -2);
        o.w0 = wb.size(); for (int f = 0; f < len; ++f) wb.push_back(P[f + 1].w0);
        o.w1 = wb.size(); for (int f = 0; f < len; ++f) wb.push_back(P[f + 1].w1);
        // transpose: coarse local index -> the fine local indices feeding it
        std::vector<std::vector<std::pair<int, double>>> rows(std::max(clen, 1));
        for (int f = 0; f < len; ++f) {
          const int cs[2] = {ib[o.c0 + f], ib[o.c1 + f]};
          const double ws[2] = {wb[o.w0 + f], wb[o.w1 + f]};
          for (int s2 = 0; s2 < 2; ++s2)
            if (cs[s2] >= 0 && cs[s2] < clen && ws[s2] != 0.0) rows[cs[s2]].push_back({f, ws[s2]});
        }
        o.rs = ib.size();
        int q = 0;
        std::vector<int> rf;
        std::vector<double> rw;
        for (int cc = 0; cc < clen; ++cc) {
          ib.push_back(q);
          for (auto& pr : rows[cc]) { rf.push_back(pr.first); rw.push_back(pr.second); ++q; }
        }
        ib.push_back(q);
        o.rf = ib.size(); ib.insert(ib.end(), rf.begin(), rf.end());
        o.rw = wb.size(); wb.insert(wb.end(), rw.begin(), rw.end());
      }
    if (ib.empty()) ib.push_back(0);
    if (wb.empty()) wb.push_back(0.0);
    std::vector<float> wb32(wb.begin(), wb.end());
    int* d_ib = nullptr;
    double* d_wb64 = nullptr;
    float* d_wb32 = nullptr;
    if (upload(c, (void**)&d_ib, ib.data(), ib.size() * 4)) return LOR_ENOMEM;
    if (upload(c, (void**)&d_wb64, wb.data(), wb.size() * 8)) return LOR_ENOMEM;
    if (upload(c, (void**)&d_wb32, wb32.data(), wb32.size() * 4)) return LOR_ENOMEM;
    std::vector<XferG<double>> x64((size_t)L * K1);
    std::vector<XferG<float>> x32((size_t)L * K1);
    for (size_t t = 0; t < offs.size(); ++t) {
      const Off& o = offs[t];
      x64[t] = {d_ib + o.c0, d_ib + o.c1, d_wb64 + o.w0, d_wb64 + o.w1, d_ib + o.rs, d_ib + o.rf, d_wb64 + o.rw};
      x32[t] = {d_ib + o.c0, d_ib + o.c1, d_wb32 + o.w0, d_wb32 + o.w1, d_ib + o.rs, d_ib + o.rf, d_wb32 + o.rw};
    }
    if (upload(c, &c->d_xferg64, x64.data(), x64.size() * sizeof(XferG<double>))) return LOR_ENOMEM;
    if (upload(c, &c->d_xferg32, x32.data(), x32.size() * sizeof(XferG<float>))) return LOR_ENOMEM;
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return lor_cuda_check(c, e, "patch transfer tables");
  }
  // enlarged patches: every level-0 node's entries in the patch output slices (patches in
  // index order), summed by k_patch_gather in place of the closed-form vertex-patch sum
  if (!c->h_spans.empty()) {
    const long long nt = c->lev[0].ntot;
    const long long zstride = (c->gen_rows0 + 31) / 32 * 32;
    std::vector<long long> cnt(nt + 1, 0);
    const LevelGrid& g0l = c->lev[0];
    auto each = [&](auto&& fn) {
      for (int j = 0; j < J; ++j) {
        const GenSched& g = gs[j];
        for (int lex = 0; lex < g.rows; ++lex) {
          const int i = lex % g.dims[0], jj = (lex / g.dims[0]) % g.dims[1], k = lex / (g.dims[0] * g.dims[1]);
          const long long G = ((long long)(g.org[2] + k) * g0l.N[1] + (g.org[1] + jj)) * g0l.N[0] + (g.org[0] + i);
          fn(G, (long long)j * zstride + lex);
        }
      }
    };
    each([&](long long G, long long) { ++cnt[G + 1]; });
    for (long long q = 0; q < nt; ++q) cnt[q + 1] += cnt[q];
    std::vector<long long> idx(std::max<long long>(cnt[nt], 1)), pos(cnt.begin(), cnt.end() - 1);
    each([&](long long G, long long z) { idx[pos[G]++] = z; });
    if (upload(c, (void**)&c->d_gather_ptr, cnt.data(), cnt.size() * 8)) return LOR_ENOMEM;
    if (upload(c, (void**)&c->d_gather_idx, idx.data(), idx.size() * 8)) return LOR_ENOMEM;
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return lor_cuda_check(c, e, "patch gather list");
  }
  const long long nval = tot * R;
  std::vector<double> all((size_t)std::max<long long>(nval, 1), 0.0);
  for (size_t t = 0; t < out.size(); ++t)
    if (!out[t].rec.empty()) std::memcpy(&all[(size_t)off[t] * R], out[t].rec.data(), out[t].rec.size() * 8);
  if (upload(c, (void**)&c->d_facoff, off.data(), off.size() * 8)) return LOR_ENOMEM;
  if (upload(c, (void**)&c->d_gsched, gs.data(), gs.size() * sizeof(GenSched))) return LOR_ENOMEM;
  if (upload(c, (void**)&c->d_gfpad, gfpad.data(), gfpad.size() * 4)) return LOR_ENOMEM;
  if (upload(c, (void**)&c->d_gchunk, gchunk.data(), gchunk.size() * 4)) return LOR_ENOMEM;
  if (upload(c, (void**)&c->d_F64, all.data(), all.size() * 8)) return LOR_ENOMEM;
  if (c->opt.factor_bf16) c->d_F16 = (__nv_bfloat16*)lor_alloc(c, all.size() * 2);
  else c->d_F32 = (float*)lor_alloc(c, all.size() * 4);
  if (!(c->d_F16 || c->d_F32)) return lor_fail(c, LOR_ENOMEM, "alloc factors");
  if (nval > 0) {
    if (c->d_F32) k_fac_to32<<<(unsigned)lor_ceil_div(nval, 256), 256, 0, c->stream>>>(c->d_F64, c->d_F32, nval, R);
    else k_fac_to16<<<(unsigned)lor_ceil_div(nval, 256), 256, 0, c->stream>>>(c->d_F64, c->d_F16, nval, R);
    ++c->launches;
  }
  // the upload's host buffers go out of scope here: finish the copies first
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "ordered factors");
  return lor_cuda_check(c, cudaGetLastError(), "ordered factors");
}

lor_status lor_setup_patches(lor_ctx* c) {
  const int dim = c->dim;
  c->J = 1;
  for (int a = 0; a < dim; ++a) c->J *= (c->n[a] + 1);
  const int nshape = 1 << dim;
  std::vector<int> front, fpad, rowlex, recof, poslex, chunk;
  c->shapes.assign(c->L * 8, BoxShape());
  c->maxfront = 0;
  for (int l = 0; l < c->L; ++l) {
    const int m = c->lev[l].m;
    for (int s = 0; s < nshape; ++s) {
      BoxShape bs;
      for (int a = 0; a < 3; ++a) bs.dims[a] = a < dim ? axis_len((s >> a) & 1, m) : 1;
      bs.rows = bs.dims[0] * bs.dims[1] * bs.dims[2];
      const int A = bs.dims[0], Bd = bs.dims[1], Cd = bs.dims[2];
      const int nfront = bs.rows ? (A - 1) + 2 * (Bd - 1) + (dim == 3 ? 4 * (Cd - 1) : 0) + 1 : 0;
      bs.nfront = nfront;
      bs.front_off = (int)front.size();
      bs.row_off = (int)rowlex.size();
      std::vector<std::vector<int>> byf(std::max(nfront, 0));
      for (int k = 0; k < Cd; ++k)
        for (int j = 0; j < Bd; ++j)
          for (int i = 0; i < A; ++i) byf[i + 2 * j + 4 * k].push_back((k * Bd + j) * A + i);
      std::vector<int> pl(bs.rows);
      front.push_back(0);
      fpad.push_back(0);
      int pos = 0, rec = 0, mf = 0;
      for (int f = 0; f < nfront; ++f) {
        int q = 0;
        for (int lex : byf[f]) {
          rowlex.push_back(lex);
          recof.push_back(rec + q++);
          pl[lex] = pos++;
        }
        const int padlen = (int)((byf[f].size() + 3) / 4 * 4);
        rec += padlen;
        mf = std::max(mf, padlen);
        front.push_back(pos);
        fpad.push_back(rec);
      }
      bs.rpad = rec;
      bs.maxfront = mf;
      if (mf > 64) return lor_fail(c, LOR_EINVAL, "wavefront wider than 64 rows");
      c->maxfront = std::max(c->maxfront, mf);
      // chunks of whole fronts of at most kChunkBytes per factor element size; a
      // front larger than that is a chunk of its own
      for (int es = 0; es < 3; ++es) {
        const int cap = kChunkBytes[es] / (lor_rec(dim) * (2 << es));
        bs.chunk_off[es] = (int)chunk.size();
        bs.nchunk[es] = 0;
        bs.maxchunk[es] = 0;
        int fa = 0;
        chunk.push_back(0);
        const int base = bs.front_off;
        while (fa < nfront) {
          int fb = fa + 1;
          while (fb < nfront && (fpad[base + fb + 1] - fpad[base + fa]) <= cap) ++fb;
          chunk.push_back(fb);
          bs.maxchunk[es] = std::max(bs.maxchunk[es], fpad[base + fb] - fpad[base + fa]);
          ++bs.nchunk[es];
          fa = fb;
        }
      }
      bs.guard = A * Bd + A + 1;
      for (int t = 0; t < bs.rows; ++t) poslex.push_back(pl[t]);
      c->shapes[l * 8 + s] = bs;
    }
  }
  if (upload(c, (void**)&c->d_front, front.data(), front.size() * 4)) return LOR_ENOMEM;
  if (upload(c, (void**)&c->d_fpad, fpad.data(), fpad.size() * 4)) return LOR_ENOMEM;
  if (upload(c, (void**)&c->d_chunk, chunk.data(), chunk.size() * 4)) return LOR_ENOMEM;
  for (auto& bs : c->shapes)
    for (int es = 0; es < 3; ++es) c->maxchunk[es] = std::max(c->maxchunk[es], bs.maxchunk[es]);
  if (upload(c, (void**)&c->d_rowlex, rowlex.data(), std::max<size_t>(1, rowlex.size()) * 4)) return LOR_ENOMEM;
  if (upload(c, (void**)&c->d_recof, recof.data(), std::max<size_t>(1, recof.size()) * 4)) return LOR_ENOMEM;
  if (upload(c, (void**)&c->d_poslex, poslex.data(), std::max<size_t>(1, poslex.size()) * 4)) return LOR_ENOMEM;
  if (upload(c, (void**)&c->d_shapes, c->shapes.data(), c->shapes.size() * sizeof(BoxShape))) return LOR_ENOMEM;
  int* d_poslex = c->d_poslex;
  BoxShape* d_shapes = c->d_shapes;

  // patch-local 1D prolongation per level and axis type (fine local -> coarse local)
  for (int l = 0; l + 1 < c->L; ++l) {
    const int m = c->lev[l].m, mc = c->lev[l + 1].m;
    for (int type = 0; type < 2; ++type) {
      // model axis: interior type = vertex 1 of 2 elements; boundary type = vertex 0
      const int v = type == 0 ? 1 : 0, nel = type == 0 ? 2 : 1;
      std::vector<Prolong1D> P = prolong_axis(nel, c->gll_x, c->sel[l], c->sel[l + 1]);
      const int len = axis_len(type, m);
      const int of = (v > 0 ? v - 1 : 0) * m + 1, oc = (v > 0 ? v - 1 : 0) * mc + 1;
      std::vector<Prolong1D> loc(std::max(len, 1));
      for (int f = 0; f < len; ++f) {
        Prolong1D pr = P[of + f];
        pr.c0 = pr.c0 >= 0 ? pr.c0 - oc : -2;
        pr.c1 = pr.c1 >= 0 ? pr.c1 - oc : -2;
        loc[f] = pr;   // local coarse index in [-1, clen]; -1 / clen are the patch boundary
      }
      if (upload(c, (void**)&c->d_pp[l][type], loc.data(), loc.size() * sizeof(Prolong1D))) return LOR_ENOMEM;
      // transpose: for every coarse local index the (<= 3) fine local indices feeding it
      const int clen = axis_len(type, mc);
      std::vector<RestrictEntry> rr(std::max(clen, 1));
      for (auto& e : rr) { e.cnt = 0; for (int t = 0; t < LOR_MAXR; ++t) { e.f[t] = 0; e.w[t] = 0.0; } }
      for (int f = 0; f < len; ++f) {
        const int cs[2] = {loc[f].c0, loc[f].c1};
        const double ws[2] = {loc[f].w0, loc[f].w1};
        for (int s2 = 0; s2 < 2; ++s2) {
          if (cs[s2] < 0 || cs[s2] >= clen || ws[s2] == 0.0) continue;
          RestrictEntry& e = rr[cs[s2]];
          if (e.cnt == LOR_MAXR) return lor_fail(c, LOR_EINVAL, "restriction stencil too wide");
          e.f[e.cnt] = f; e.w[e.cnt] = ws[s2]; ++e.cnt;
        }
      }
      if (upload(c, (void**)&c->d_rr[l][type], rr.data(), rr.size() * sizeof(RestrictEntry))) return LOR_ENOMEM;
    }
  }

  // visiting order of the patch kernel: patches grouped by box shape, interior
  // patches first and in blocks of kOrderBlock^dim vertices (blocks and the
  // vertices inside them in lexicographic order), so that the patches in flight
  // at one time cover a compact set of elements and share stencil rows in L2
  {
    const int kOrderBlock = 8;
    std::vector<int> order;
    const int n0 = c->n[0] + 1, n1 = c->n[1] + 1;
    auto shape_of = [&](int j) {
      int v[3] = {j % n0, (j / n0) % n1, dim == 3 ? j / (n0 * n1) : 0};
      int sh = 0;
      for (int a = 0; a < dim; ++a) sh |= ((v[a] == 0 || v[a] == c->n[a]) ? 1 : 0) << a;
      return sh;
    };
    const int nb[3] = {(c->n[0] + kOrderBlock - 1) / kOrderBlock, (c->n[1] + kOrderBlock - 1) / kOrderBlock,
                       dim == 3 ? (c->n[2] + kOrderBlock - 1) / kOrderBlock : 1};
    for (int bz = 0; bz < nb[2]; ++bz)
      for (int by = 0; by < nb[1]; ++by)
        for (int bxi = 0; bxi < nb[0]; ++bxi)
          for (int z = 0; z < (dim == 3 ? kOrderBlock : 1); ++z)
            for (int y = 0; y < kOrderBlock; ++y)
              for (int x = 0; x < kOrderBlock; ++x) {
                const int v0 = 1 + bxi * kOrderBlock + x, v1 = 1 + by * kOrderBlock + y;
                const int v2 = dim == 3 ? 1 + bz * kOrderBlock + z : 0;
                if (v0 >= c->n[0] || v1 >= c->n[1] || (dim == 3 && v2 >= c->n[2])) continue;
                order.push_back((v2 * n1 + v1) * n0 + v0);
              }
    for (int want = 1; want < 8; ++want)
      for (int j = 0; j < c->J; ++j)
        if (shape_of(j) == want) order.push_back(j);
    if ((long long)order.size() != c->J) return lor_fail(c, LOR_EINVAL, "patch order incomplete");
    if (upload(c, (void**)&c->d_porder, order.data(), order.size() * 4)) return LOR_ENOMEM;
  }
  if (c->gen) return setup_ordered_factors(c);
  // factor storage offsets (records; a patch level holds 2*rpad records)
  std::vector<long long> off((size_t)c->L * c->J);
  long long tot = 0;
  for (int l = 0; l < c->L; ++l)
    for (int j = 0; j < c->J; ++j) {
      int v[3] = {j % (c->n[0] + 1), (j / (c->n[0] + 1)) % (c->n[1] + 1), dim == 3 ? j / ((c->n[0] + 1) * (c->n[1] + 1)) : 0};
      int sh = 0;
      for (int a = 0; a < dim; ++a) sh |= ((v[a] == 0 || v[a] == c->n[a]) ? 1 : 0) << a;
      off[(size_t)l * c->J + j] = tot;
      if (l + 1 < c->L) {   // the vertex level is solved exactly and has no factors
        tot += 2LL * c->shapes[l * 8 + sh].rpad;
        c->fac_rows += c->shapes[l * 8 + sh].rows;
      }
    }
  tot *= lor_rec(dim);   // values
  if (upload(c, (void**)&c->d_facoff, off.data(), off.size() * 8)) return LOR_ENOMEM;
  // FP64 records for the FP64 path, and the one reduced-precision copy the FP32
  // path reads (bf16 if requested, else FP32)
  c->d_F64 = (double*)lor_alloc(c, std::max<long long>(tot, 1) * 8);
  if (c->opt.factor_bf16) c->d_F16 = (__nv_bfloat16*)lor_alloc(c, std::max<long long>(tot, 1) * 2);
  else c->d_F32 = (float*)lor_alloc(c, std::max<long long>(tot, 1) * 4);
  if (!c->d_F64 || !(c->d_F16 || c->d_F32)) return lor_fail(c, LOR_ENOMEM, "alloc factors");
  // ILU(0) per level (the last level is solved exactly and needs no factors)
  for (int l = 0; l + 1 < c->L; ++l) {
    IluArgs a;
    a.dim = dim; a.NS = c->NS;
    for (int t = 0; t < 3; ++t) { a.n[t] = c->n[t]; a.N[t] = c->lev[l].N[t]; }
    a.m = c->lev[l].m;
    a.shapes = d_shapes + l * 8;
    a.rowlex = c->d_rowlex; a.recof = c->d_recof; a.front = c->d_front; a.poslex = d_poslex;
    a.facoff = c->d_facoff + (size_t)l * c->J;
    a.S = c->d_S64[l];
    a.F = c->d_F64;
    a.status = c->d_status;
    k_ilu0<<<c->J, 128, 0, c->stream>>>(a);
    ++c->launches;
    if (lor_cuda_check(c, cudaGetLastError(), "ilu0")) return LOR_ECUDA;
  }
  if (tot > 0) {   // p = 1: the patch box is the vertex level, solved exactly, no factors
    if (c->d_F32)
      k_fac_to32<<<(unsigned)lor_ceil_div(tot, 256), 256, 0, c->stream>>>(c->d_F64, c->d_F32, tot, lor_rec(dim));
    else
      k_fac_to16<<<(unsigned)lor_ceil_div(tot, 256), 256, 0, c->stream>>>(c->d_F64, c->d_F16, tot, lor_rec(dim));
    ++c->launches;
    if (lor_cuda_check(c, cudaGetLastError(), "factor conversion")) return LOR_ECUDA;
  }
  return check_status(c, "ilu0");
}

// ------------------------------------------------------------------ coarse space
lor_status lor_setup_coarse(lor_ctx* c) {
  const int dim = c->dim;
  // level 0 of the coarse hierarchy = the vertex level of the patch hierarchy
  const LevelGrid& lv = c->lev[c->L - 1];
  for (int a = 0; a < 3; ++a) c->cN[0][a] = lv.N[a];
  c->cntot[0] = lv.ntot;
  c->d_cS64[0] = c->d_S64[c->L - 1];
  c->d_cS32[0] = c->d_S32[c->L - 1];
  auto interior = [&](int l) {
    long long s = 1;
    for (int a = 0; a < dim; ++a) s *= std::max(c->cN[l][a] - 2, 0);
    return s;
  };
  int l = 0;
  while (interior(l) > 343 && l + 1 < LOR_MAXCLEV) {
    int Nc[3] = {1, 1, 1};
    for (int a = 0; a < dim; ++a) {
      int ncn;
      std::vector<Prolong1D> P = prolong_index(c->cN[l][a], &ncn);
      Nc[a] = ncn;
      if (upload_prolong(c, P, ncn, &c->d_cP1[l][a], &c->d_cR1ptr[l][a], &c->d_cR1idx[l][a], &c->d_cR1w[l][a]))
        return LOR_ENOMEM;
    }
    for (int a = 0; a < 3; ++a) c->cN[l + 1][a] = Nc[a];
    c->cntot[l + 1] = (long long)Nc[0] * Nc[1] * Nc[2];
    c->d_cS64[l + 1] = (double*)lor_alloc(c, c->cntot[l + 1] * c->NS * 8);
    c->d_cS32[l + 1] = (float*)lor_alloc(c, c->cntot[l + 1] * c->NS * 4);
    if (!c->d_cS64[l + 1] || !c->d_cS32[l + 1]) return lor_fail(c, LOR_ENOMEM, "alloc coarse stencils");
    if (galerkin(c, dim, c->cN[l], c->cN[l + 1], c->d_cP1[l], c->d_cR1ptr[l], c->d_cR1idx[l], c->d_cR1w[l],
                 c->d_cS64[l], c->d_cS64[l + 1]))
      return LOR_ECUDA;
    const long long n = c->cntot[l + 1] * c->NS;
    k_to_float<<<(unsigned)lor_ceil_div(n, 256), 256, 0, c->stream>>>(c->d_cS64[l + 1], c->d_cS32[l + 1], n);
    ++c->launches;
    ++l;
  }
  c->CL = l + 1;
  for (int t = 0; t < c->CL; ++t) {
    const long long nt = c->cntot[t];
    c->d_cDinv64[t] = (double*)lor_alloc(c, nt * 8);
    c->d_cDinv32[t] = (float*)lor_alloc(c, nt * 4);
    for (int k = 0; k < 4; ++k) {
      c->d_cw64[t][k] = (double*)lor_alloc(c, nt * 8);
      c->d_cw32[t][k] = (float*)lor_alloc(c, nt * 4);
      if (!c->d_cw64[t][k] || !c->d_cw32[t][k]) return lor_fail(c, LOR_ENOMEM, "alloc coarse vectors");
    }
    if (!c->d_cDinv64[t] || !c->d_cDinv32[t]) return lor_fail(c, LOR_ENOMEM, "alloc coarse diag");
    k_l1_dinv<<<(unsigned)lor_ceil_div(nt, 128), 128, 0, c->stream>>>(dim, c->cN[t][0], c->cN[t][1], c->cN[t][2],
                                                                        c->d_cS64[t], c->d_cDinv64[t], c->d_cDinv32[t]);
    ++c->launches;
  }
  if (lor_cuda_check(c, cudaGetLastError(), "coarse setup")) return LOR_ECUDA;
  // P_0 tables and P_0^T scratch (x-pass: Nz*Ny*Vx, y-pass: Nz*Vy*Vx)
  {
    const int p = c->p;
    std::vector<double> w64(3 * p, 0.0);
    for (int i = 0; i <= p; ++i) w64[i] = c->gll_x[i];
    for (int a = 0; a < 2 * p - 1; ++a) {
      const int t = a + 1;   // position in [(V-1)p, (V+1)p]
      w64[p + 1 + a] = t <= p ? c->gll_x[t] : 1.0 - c->gll_x[t - p];
    }
    std::vector<float> w32(w64.begin(), w64.end());
    if (upload(c, (void**)&c->d_p0w64, w64.data(), w64.size() * 8)) return LOR_ENOMEM;
    if (upload(c, (void**)&c->d_p0w32, w32.data(), w32.size() * 4)) return LOR_ENOMEM;
    const LevelGrid& g0 = c->lev[0];
    const long long V0 = c->n[0] + 1, V1 = c->n[1] + 1;
    const long long n1 = (long long)g0.N[2] * g0.N[1] * V0, n2 = (long long)g0.N[2] * V1 * V0;
    for (int k = 0; k < 2; ++k) {
      const long long nn = k == 0 ? n1 : n2;
      c->d_p0t64[k] = (double*)lor_alloc(c, nn * 8);
      c->d_p0t32[k] = (float*)lor_alloc(c, nn * 4);
      if (!c->d_p0t64[k] || !c->d_p0t32[k]) return lor_fail(c, LOR_ENOMEM, "alloc P0 scratch");
    }
  }
  // dense inverse of the coarsest operator (interior unknowns) on the host
  const int t = c->CL - 1;
  const long long nt = c->cntot[t];
  std::vector<double> S(nt * c->NS);
  cudaError_t e = cudaMemcpyAsync(S.data(), c->d_cS64[t], S.size() * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return lor_cuda_check(c, e, "coarse copy");
  const int* N = c->cN[t];
  std::vector<int> idx;
  std::vector<long long> where(nt, -1);
  for (long long g = 0; g < nt; ++g) {
    const int I = (int)(g % N[0]), Jn = (int)((g / N[0]) % N[1]), K = (int)(g / ((long long)N[0] * N[1]));
    const bool bnd = I == 0 || I == N[0] - 1 || Jn == 0 || Jn == N[1] - 1 || (dim == 3 && (K == 0 || K == N[2] - 1));
    if (!bnd) { where[g] = (long long)idx.size(); idx.push_back((int)g); }
  }
  const int nd = (int)idx.size();
  c->ncoarse_direct = nd;
  std::vector<double> A((size_t)nd * nd, 0.0), Inv((size_t)nd * nd, 0.0);
  for (int r = 0; r < nd; ++r) {
    const long long g = idx[r];
    const int I = (int)(g % N[0]), Jn = (int)((g / N[0]) % N[1]), K = (int)(g / ((long long)N[0] * N[1]));
    for (int o = 0; o < c->NS; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = dim == 3 ? o / 9 - 1 : 0;
      const long long h = ((long long)(K + dz) * N[1] + (Jn + dy)) * N[0] + (I + dx);
      if (h < 0 || h >= nt || where[h] < 0) continue;
      A[(size_t)r * nd + where[h]] = S[(size_t)o * nt + g];
    }
  }
  // Cholesky A = L L^T, then columns of A^{-1}
  std::vector<double> Lc((size_t)nd * nd, 0.0);
  for (int j = 0; j < nd; ++j) {
    double s = A[(size_t)j * nd + j];
    for (int k = 0; k < j; ++k) s -= Lc[(size_t)j * nd + k] * Lc[(size_t)j * nd + k];
    if (!(s > 0)) return lor_fail(c, LOR_EBREAKDOWN, "coarse Cholesky: matrix not positive definite");
    const double d = sqrt(s);
    Lc[(size_t)j * nd + j] = d;
    for (int i = j + 1; i < nd; ++i) {
      double t2 = A[(size_t)i * nd + j];
      for (int k = 0; k < j; ++k) t2 -= Lc[(size_t)i * nd + k] * Lc[(size_t)j * nd + k];
      Lc[(size_t)i * nd + j] = t2 / d;
    }
  }
  std::vector<double> y(nd);
  for (int col = 0; col < nd; ++col) {
    for (int i = 0; i < nd; ++i) {
      double s = (i == col) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= Lc[(size_t)i * nd + k] * y[k];
      y[i] = s / Lc[(size_t)i * nd + i];
    }
    for (int i = nd - 1; i >= 0; --i) {
      double s = y[i];
      for (int k = i + 1; k < nd; ++k) s -= Lc[(size_t)k * nd + i] * Inv[(size_t)k * nd + col];
      Inv[(size_t)i * nd + col] = s / Lc[(size_t)i * nd + i];
    }
  }
  std::vector<float> Inv32(Inv.begin(), Inv.end());
  if (nd > 0) {
    if (upload(c, (void**)&c->d_cdirect_idx, idx.data(), idx.size() * 4)) return LOR_ENOMEM;
    if (upload(c, (void**)&c->d_cInv64, Inv.data(), Inv.size() * 8)) return LOR_ENOMEM;
    if (upload(c, (void**)&c->d_cInv32, Inv32.data(), Inv32.size() * 4)) return LOR_ENOMEM;
  }
  e = cudaStreamSynchronize(c->stream);
  return lor_cuda_check(c, e, "coarse setup");
}
