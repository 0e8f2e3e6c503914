// Host and device helpers for multilinear element maps (Section 2: every element is the
// image of the unit cube under the multilinear interpolation of its vertices).
#pragma once

namespace lorg {

__host__ __device__ __forceinline__ double det3(const double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

// inverse of a dim x dim matrix (dim 2 or 3) by the adjugate
__host__ __device__ __forceinline__ void inv_dd(int dim, const double J[3][3], double det, double Ji[3][3]) {
  if (dim == 3) {
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  } else {
    Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
  }
}

// Multilinear map of the 2^dim points P[c][a] (corner c = cx + 2cy + 4cz) at xi:
// X and J[a][b] = dX_a/dxi_b.
__host__ __device__ __forceinline__ void multilinear(int dim, const double (*Pc)[3], const double* xi, double* X, double J[3][3]) {
  for (int a = 0; a < 3; ++a) { X[a] = 0; for (int b = 0; b < 3; ++b) J[a][b] = 0; }
  const int nc = 1 << dim;
  for (int cc = 0; cc < nc; ++cc) {
    double f[3], df[3];
    for (int a = 0; a < 3; ++a) {
      const int bit = (cc >> a) & 1;
      f[a] = bit ? xi[a] : 1.0 - xi[a];
      df[a] = bit ? 1.0 : -1.0;
    }
    double N = 1.0;
    for (int t = 0; t < dim; ++t) N *= f[t];
    for (int bb = 0; bb < dim; ++bb) {
      double g = 1.0;
      for (int t = 0; t < dim; ++t) g *= (t == bb) ? df[t] : f[t];
      for (int a = 0; a < dim; ++a) J[a][bb] += g * Pc[cc][a];
    }
    for (int a = 0; a < dim; ++a) X[a] += N * Pc[cc][a];
  }
}

__host__ __device__ __forceinline__ void element_corners(int dim, int nx, int ny, int ex, int ey, int ez, const double* vert,
                                       long long NV, double (*Pc)[3]) {
  const int nc = 1 << dim;
  for (int cc = 0; cc < nc; ++cc) {
    const int bx = cc & 1, by = (cc >> 1) & 1, bz = (cc >> 2) & 1;
    const long long vid = ((long long)(ez + bz) * (ny + 1) + (ey + by)) * (nx + 1) + (ex + bx);
    for (int a = 0; a < 3; ++a) Pc[cc][a] = a < dim ? vert[a * NV + vid] : 0.0;
  }
}


// Isoparametric (curved) element map: the degree-p interpolant of the element's GLL
// node coordinates Xn (SoA dim x ntot on the Nx x Ny (x Nz) node grid) at the Gauss
// point (qx, qy, qz) of element (ex, ey, ez).  B, D: the 1D GLL basis and its
// derivative at the Gauss points ([q][i], Q = p + 1).  Returns X and J[a][b] = dX_a/dxi_b.
__device__ __forceinline__ void iso_map(int dim, int p, int ex, int ey, int ez, int qx, int qy, int qz, int Nx,
                                        int Ny, long long ntot, const double* Xn, const double* B,
                                        const double* D, double* X, double J[3][3]) {
  const int Q = p + 1;
  for (int a = 0; a < 3; ++a) { X[a] = 0; for (int b = 0; b < 3; ++b) J[a][b] = 0; }
  const int nk = dim == 3 ? Q : 1;
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < Q; ++j)
      for (int i = 0; i < Q; ++i) {
        const long long node = ((long long)(ez * p + k) * Ny + (ey * p + j)) * Nx + (ex * p + i);
        const double bx = B[qx * Q + i], by = B[qy * Q + j], bz = dim == 3 ? B[qz * Q + k] : 1.0;
        const double g[3] = {D[qx * Q + i] * by * bz, bx * D[qy * Q + j] * bz,
                             dim == 3 ? bx * by * D[qz * Q + k] : 0.0};
        const double phi = bx * by * bz;
        for (int a = 0; a < dim; ++a) {
          const double xa = Xn[a * ntot + node];
          X[a] += phi * xa;
          for (int b = 0; b < dim; ++b) J[a][b] += xa * g[b];
        }
      }
}

}  // namespace lorg
