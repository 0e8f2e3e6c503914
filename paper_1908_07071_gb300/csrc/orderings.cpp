// Algebraic orderings of the patch-level ILU(0) smoothers (Section 3.4) and the
// ILU(0) factorization in such an order, on the host.
//
// A patch level is a box of A x B x C nodes (x fastest; C = 1 in 2D) whose matrix
// couples nodes at distance at most one along every axis (the 3^d-point LOR
// pattern).  The matrix arrives as `a27`: for every node, its 27 (3D) or 9 (2D)
// stencil values in stencil-offset order ((dz+1)*9 + (dy+1)*3 + (dx+1)), zero for
// neighbours outside the box.
//
// RCM (Cuthill and McKee 1969, reversed): breadth-first search from the unvisited
// node of smallest (degree, index), each node's unvisited neighbours taken by
// increasing (degree, index), the whole sequence reversed.
//
// MDF (minimum discarded fill; D'Azevedo, Forsyth and Tang 1992): eliminating node
// i next would create a_ji a_ik / a_ii for every pair j != k of its remaining
// neighbours; ILU(0) keeps the entries that fall on the pattern and discards the
// others.  The node whose discarded entries have the smallest 2-norm is ordered
// next (ties: the smallest index), the kept part of its elimination updates the
// remaining matrix, and the discarded fill of its remaining neighbours (the only
// nodes whose rows, columns or neighbour sets change) is recomputed.  This file is
// compiled without floating-point contraction, so every product and sum rounds
// on its own, as in a plain evaluation of the definition.
#include <algorithm>
#include <cmath>
#include <set>
#include <utility>
#include <vector>

#include "lor_internal.h"

namespace {

struct Box {
  int dim, A, B, C, n;
  int coord(int i, int a) const { return a == 0 ? i % A : a == 1 ? (i / A) % B : i / (A * B); }
  // stencil-offset index of node k seen from node i (both in the box, adjacent)
  int off(int i, int k) const {
    const int dx = coord(k, 0) - coord(i, 0), dy = coord(k, 1) - coord(i, 1), dz = coord(k, 2) - coord(i, 2);
    return dim == 3 ? (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1) : (dy + 1) * 3 + (dx + 1);
  }
  bool adjacent(int i, int k) const {
    for (int a = 0; a < 3; ++a)
      if (std::abs(coord(k, a) - coord(i, a)) > 1) return false;
    return true;
  }
  // neighbours (other than i) in increasing index order
  std::vector<int> nbrs(int i) const {
    std::vector<int> out;
    const int x = coord(i, 0), y = coord(i, 1), z = coord(i, 2);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (!dx && !dy && !dz) continue;
          const int X = x + dx, Y = y + dy, Z = z + dz;
          if (X < 0 || X >= A || Y < 0 || Y >= B || Z < 0 || Z >= C) continue;
          out.push_back((Z * B + Y) * A + X);
        }
    std::sort(out.begin(), out.end());
    return out;
  }
};

Box make_box(int dim, int A, int B, int C) {
  Box b;
  b.dim = dim; b.A = A; b.B = B; b.C = dim == 3 ? C : 1;
  b.n = b.A * b.B * b.C;
  return b;
}

}  // namespace

namespace lorh {

void rcm_box(int dim, int A, int B, int C, std::vector<int>& perm) {
  const Box b = make_box(dim, A, B, C);
  std::vector<std::vector<int>> nb(b.n);
  for (int i = 0; i < b.n; ++i) nb[i] = b.nbrs(i);
  std::vector<char> seen(b.n, 0);
  std::vector<int> order;
  order.reserve(b.n);
  auto less = [&](int u, int v) {
    return nb[u].size() != nb[v].size() ? nb[u].size() < nb[v].size() : u < v;
  };
  while ((int)order.size() < b.n) {
    int s = -1;
    for (int i = 0; i < b.n; ++i)
      if (!seen[i] && (s < 0 || less(i, s))) s = i;
    size_t head = order.size();
    order.push_back(s);
    seen[s] = 1;
    while (head < order.size()) {
      const int u = order[head++];
      std::vector<int> next;
      for (int v : nb[u])
        if (!seen[v]) next.push_back(v);
      std::sort(next.begin(), next.end(), less);
      for (int v : next) {
        seen[v] = 1;
        order.push_back(v);
      }
    }
  }
  perm.assign(order.rbegin(), order.rend());
}

bool mdf_box(int dim, int A, int B, int C, const std::vector<double>& a27, std::vector<int>& perm) {
  const Box b = make_box(dim, A, B, C);
  const int NS = dim == 3 ? 27 : 9, D = NS / 2;
  std::vector<double> a(a27);
  std::vector<std::vector<int>> nb(b.n);
  for (int i = 0; i < b.n; ++i) nb[i] = b.nbrs(i);
  std::vector<char> alive(b.n, 1);
  auto at = [&](int i, int k) -> double& { return a[(size_t)i * NS + (i == k ? D : b.off(i, k))]; };
  auto fill = [&](int i) {
    std::vector<int> live;
    for (int j : nb[i])
      if (alive[j]) live.push_back(j);
    if (live.size() < 2) return 0.0;
    const double piv = at(i, i);
    std::vector<double> col(live.size()), row(live.size());
    for (size_t x = 0; x < live.size(); ++x) {
      col[x] = at(live[x], i) / piv;
      row[x] = at(i, live[x]);
    }
    double s = 0.0;
    for (size_t x = 0; x < live.size(); ++x)
      for (size_t y = 0; y < live.size(); ++y) {
        if (live[x] == live[y] || b.adjacent(live[x], live[y])) continue;
        const double v = col[x] * row[y];
        s += v * v;
      }
    return std::sqrt(s);
  };
  std::vector<double> df(b.n);
  std::set<std::pair<double, int>> queue;
  for (int i = 0; i < b.n; ++i) {
    df[i] = fill(i);
    queue.insert({df[i], i});
  }
  perm.clear();
  perm.reserve(b.n);
  while (!queue.empty()) {
    const int i = queue.begin()->second;
    queue.erase(queue.begin());
    perm.push_back(i);
    alive[i] = 0;
    const double piv = at(i, i);
    if (!(piv > 0.0)) return false;
    std::vector<int> live;
    for (int j : nb[i])
      if (alive[j]) live.push_back(j);
    for (int j : live) {
      const double lj = at(j, i) / piv;
      for (int k : live)
        if (j == k || b.adjacent(j, k)) at(j, k) = at(j, k) - lj * at(i, k);
    }
    for (int u : live) {
      queue.erase({df[u], u});
      df[u] = fill(u);
      queue.insert({df[u], u});
    }
  }
  return true;
}

bool ilu0_ordered(int dim, int A, int B, int C, const std::vector<double>& a27, const std::vector<int>& perm,
                  std::vector<double>& lu, std::vector<int>& level) {
  const Box b = make_box(dim, A, B, C);
  const int NS = dim == 3 ? 27 : 9, D = NS / 2;
  std::vector<int> pos(b.n);
  for (int q = 0; q < b.n; ++q) pos[perm[q]] = q;
  lu = a27;
  level.assign(b.n, 0);
  auto at = [&](int i, int k) -> double& { return lu[(size_t)i * NS + (i == k ? D : b.off(i, k))]; };
  for (int q = 0; q < b.n; ++q) {
    const int i = perm[q];
    std::vector<int> nb = b.nbrs(i);
    std::vector<int> lower;
    for (int k : nb)
      if (pos[k] < q) lower.push_back(k);
    std::sort(lower.begin(), lower.end(), [&](int u, int v) { return pos[u] < pos[v]; });
    int lev = 0;
    for (int k : lower) {
      double& aik = at(i, k);
      aik = aik / at(k, k);
      const double l = aik;
      // entries j of row i's pattern that come after k in the order: a_ij -= l a_kj
      for (int j : nb) {
        if (pos[j] <= pos[k] || !b.adjacent(k, j)) continue;
        at(i, j) = at(i, j) - l * at(k, j);
      }
      if (pos[i] > pos[k] && b.adjacent(k, i)) at(i, i) = at(i, i) - l * at(k, i);
      lev = std::max(lev, level[k] + 1);
    }
    level[i] = lev;
    if (!(at(i, i) > 0.0)) return false;
  }
  return true;
}

}  // namespace lorh
