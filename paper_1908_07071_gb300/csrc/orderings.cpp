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
#include <functional>
#include <cmath>
#include <set>
#include <utility>
#include <vector>

#include "lor_internal.h"

namespace {

struct Box {
  int dim, A, B, C, n;
  int coord(int i, int a) const { return a == 0 ? i % A : a == 1 ? (i / A) % B : i / (A * B); }
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
  // Stencil offsets o (o = (dz+1)*9 + (dy+1)*3 + (dx+1), 2D without dz) relative
  // to the node being eliminated.  Two neighbours at offsets o1, o2 are adjacent
  // (or equal) when their coordinates differ by at most one along every axis;
  // rel[o1][o2] is then the offset of the second seen from the first, and bit o2
  // of far[o1] is set when they are not.  A node's in-box neighbours by increasing
  // offset are its neighbours by increasing index (the box is numbered x fastest),
  // so walking set bits upwards visits nodes in index order.
  int rel[27][27];
  unsigned far[27];
  for (int o1 = 0; o1 < NS; ++o1) {
    far[o1] = 0;
    for (int o2 = 0; o2 < NS; ++o2) {
      const int dx = o2 % 3 - o1 % 3, dy = (o2 / 3) % 3 - (o1 / 3) % 3, dz = dim == 3 ? o2 / 9 - o1 / 9 : 0;
      const bool adj = std::abs(dx) <= 1 && std::abs(dy) <= 1 && std::abs(dz) <= 1;
      rel[o1][o2] = adj ? (dim == 3 ? (dz + 1) * 9 : 0) + (dy + 1) * 3 + (dx + 1) : -1;
      if (!adj) far[o1] |= 1u << o2;
    }
  }
  int step[27];   // index step of offset o
  for (int o = 0; o < NS; ++o)
    step[o] = (o % 3 - 1) + ((o / 3) % 3 - 1) * A + (dim == 3 ? (o / 9 - 1) * A * B : 0);
  std::vector<unsigned> inbox(b.n);   // bit o: the neighbour at offset o lies in the box
  for (int i = 0; i < b.n; ++i) {
    const int x = b.coord(i, 0), y = b.coord(i, 1), z = b.coord(i, 2);
    unsigned m = 0;
    for (int o = 0; o < NS; ++o) {
      const int X = x + o % 3 - 1, Y = y + (o / 3) % 3 - 1, Z = z + (dim == 3 ? o / 9 - 1 : 0);
      if (o != D && X >= 0 && X < A && Y >= 0 && Y < B && Z >= 0 && Z < C) m |= 1u << o;
    }
    inbox[i] = m;
  }
  std::vector<double> a(a27);
  std::vector<char> alive(b.n, 1);
  auto live_mask = [&](int i) {   // offsets of the remaining neighbours of i
    unsigned m = 0;
    for (unsigned r = inbox[i]; r; r &= r - 1) {
      const int o = __builtin_ctz(r);
      if (alive[i + step[o]]) m |= 1u << o;
    }
    return m;
  };
  // 2-norm of the fill that eliminating i would discard: the products
  // (a_ji / a_ii) a_ik over ordered pairs (j, k) of distinct, non-adjacent
  // remaining neighbours, summed j-major in index order
  auto fill = [&](int i) {
    const unsigned lm = live_mask(i);
    if (__builtin_popcount(lm) < 2) return 0.0;
    const double* ai = &a[(size_t)i * NS];
    const double piv = ai[D];
    double col[27];
    for (unsigned r = lm; r; r &= r - 1) {
      const int o = __builtin_ctz(r);
      col[o] = a[(size_t)(i + step[o]) * NS + (NS - 1 - o)] / piv;   // a_{j i} / a_ii, j at offset o
    }
    double s = 0.0;
    for (unsigned r = lm; r; r &= r - 1) {
      const int ox = __builtin_ctz(r);
      const double cx = col[ox];
      for (unsigned q = lm & far[ox]; q; q &= q - 1) {
        const double v = cx * ai[__builtin_ctz(q)];
        s += v * v;
      }
    }
    return std::sqrt(s);
  };
  // next node: smallest (discarded fill, index) among the remaining ones, from a
  // binary min-heap (Section 3.6: O(n log n) per patch); entries whose stamp is out
  // of date are skipped
  struct Entry {
    double df;
    int i;
    unsigned stamp;
    bool operator>(const Entry& o) const { return df != o.df ? df > o.df : i > o.i; }
  };
  std::vector<Entry> heap;
  heap.reserve((size_t)b.n * 4);
  std::vector<unsigned> stamp(b.n, 0);
  auto push = [&](double df, int i) {
    heap.push_back({df, i, stamp[i]});
    std::push_heap(heap.begin(), heap.end(), std::greater<Entry>());
  };
  for (int i = 0; i < b.n; ++i) push(fill(i), i);
  perm.clear();
  perm.reserve(b.n);
  while (!heap.empty()) {
    std::pop_heap(heap.begin(), heap.end(), std::greater<Entry>());
    const Entry e = heap.back();
    heap.pop_back();
    if (!alive[e.i] || e.stamp != stamp[e.i]) continue;
    const int i = e.i;
    perm.push_back(i);
    alive[i] = 0;
    const double* ai = &a[(size_t)i * NS];
    const double piv = ai[D];
    if (!(piv > 0.0)) return false;
    const unsigned lm = live_mask(i);
    // kept part of the elimination: a_jk -= (a_ji / a_ii) a_ik for adjacent or equal j, k
    for (unsigned r = lm; r; r &= r - 1) {
      const int ox = __builtin_ctz(r);
      double* aj = &a[(size_t)(i + step[ox]) * NS];
      const double lj = aj[NS - 1 - ox] / piv;
      for (unsigned q = lm & ~far[ox]; q; q &= q - 1) {
        const int oy = __builtin_ctz(q);
        const int t = rel[ox][oy];
        aj[t] = aj[t] - lj * ai[oy];
      }
    }
    for (unsigned r = lm; r; r &= r - 1) {
      const int u = i + step[__builtin_ctz(r)];
      ++stamp[u];
      push(fill(u), u);
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
  // offset tables as in mdf_box: rel[o1][o2] is the offset of the neighbour at o2
  // seen from the neighbour at o1 when the two are adjacent, else -1
  int rel[27][27], step[27];
  for (int o1 = 0; o1 < NS; ++o1)
    for (int o2 = 0; o2 < NS; ++o2) {
      const int dx = o2 % 3 - o1 % 3, dy = (o2 / 3) % 3 - (o1 / 3) % 3, dz = dim == 3 ? o2 / 9 - o1 / 9 : 0;
      rel[o1][o2] = (std::abs(dx) <= 1 && std::abs(dy) <= 1 && std::abs(dz) <= 1)
                        ? (dim == 3 ? (dz + 1) * 9 : 0) + (dy + 1) * 3 + (dx + 1)
                        : -1;
    }
  for (int o = 0; o < NS; ++o)
    step[o] = (o % 3 - 1) + ((o / 3) % 3 - 1) * A + (dim == 3 ? (o / 9 - 1) * A * B : 0);
  lu = a27;
  level.assign(b.n, 0);
  for (int q = 0; q < b.n; ++q) {
    const int i = perm[q];
    const int x = b.coord(i, 0), y = b.coord(i, 1), z = b.coord(i, 2);
    // the in-box neighbours of i (offsets, increasing = increasing index), and
    // those ordered before i, sorted by their position in the order
    int nbo[26], low[26];
    int nn = 0, nl = 0;
    for (int o = 0; o < NS; ++o) {
      const int X = x + o % 3 - 1, Y = y + (o / 3) % 3 - 1, Z = z + (dim == 3 ? o / 9 - 1 : 0);
      if (o == D || X < 0 || X >= A || Y < 0 || Y >= B || Z < 0 || Z >= C) continue;
      nbo[nn++] = o;
      if (pos[i + step[o]] < q) low[nl++] = o;
    }
    for (int u = 1; u < nl; ++u)   // insertion sort by position (positions are distinct)
      for (int v = u; v > 0 && pos[i + step[low[v - 1]]] > pos[i + step[low[v]]]; --v) std::swap(low[v - 1], low[v]);
    double* li = &lu[(size_t)i * NS];
    int lev = 0;
    for (int u = 0; u < nl; ++u) {
      const int ok = low[u];
      const int k = i + step[ok];
      const double* lk = &lu[(size_t)k * NS];
      li[ok] = li[ok] / lk[D];
      const double l = li[ok];
      // entries j of row i's pattern that come after k in the order: a_ij -= l a_kj
      for (int w = 0; w < nn; ++w) {
        const int oj = nbo[w];
        const int t = rel[ok][oj];
        if (t < 0 || pos[i + step[oj]] <= pos[k]) continue;
        li[oj] = li[oj] - l * lk[t];
      }
      li[D] = li[D] - l * lk[NS - 1 - ok];
      lev = std::max(lev, level[k] + 1);
    }
    level[i] = lev;
    if (!(li[D] > 0.0)) return false;
  }
  return true;
}

}  // namespace lorh
