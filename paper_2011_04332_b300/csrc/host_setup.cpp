// Per-cell-type setup on the host, once per type: topology, rest geometry, lumped
// masses, the projective-dynamics matrix, a fill-reducing ordering, the FP64
// Cholesky (LDL^T) factor and the chunked tables the GPU triangular solves read.
//
// The global matrix is A = M/dt^2 + sum_t w_t G_t^T G_t + sum_e w_e c_e c_e^T
// (projective dynamics of Bouaziz et al. 2014, reused as the initial Hessian of the
// quasi-Newton iteration of Liu et al. 2017; both named in the paper's
// Implementation and architecture section); with Rayleigh damping C = c_alpha M +
// c_beta L (L the sum over elements) it is (1/dt^2 + c_alpha/dt) M + (1 + c_beta/dt) L.  It depends only on the rest mesh,
// the weights and dt, so it is factored once per cell type.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <numeric>
#include <functional>
#include <iterator>
#include <set>
#include <utility>

#include "npfem_internal.h"
#include "../../include/npfem.h"

namespace npfem {
namespace {

struct V3 {
  double x, y, z;
};
inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline double cotangent(V3 a, V3 b) { return dot(a, b) / norm(cross(a, b)); }

// ---------------------------------------------------------------- element colours
// Colour elements of k vertices each so that no two elements of a colour share a vertex,
// and store them colour by colour (stable within a colour): the CTA iteration kernels add
// one colour's gradient contributions to the shared-memory gradient at a time, without
// conflicts and in a fixed order, with a barrier after each colour.  A CTA of nt threads
// takes ceil(size / nt) passes over a colour, so the colouring minimises the passes
// sum_c ceil(|c| / nt) and then the colours:
//  1. DSatur (Brélaz 1979): the uncoloured element whose neighbours (elements sharing a
//     vertex with it) show the most distinct colours goes next (ties: more neighbours,
//     then the lower index), into the least-filled colour none of them has (a new colour
//     only when every existing one is taken);
//  2. balancing: an element moves from a colour whose last pass is partly filled to one
//     whose last pass has room and that no neighbour has, when that takes a pass away
//     and adds none — first out of the colours that spill over into an extra pass (the
//     emptiest last pass first), then out of the smallest colours until they are empty;
//  3. within each colour, an order for the shared-memory banks (below).
// Returns false (and leaves the elements as they were) if more than kMaxColours colours
// would be needed.
bool colour_elements(int n, int k, int nt, std::vector<int32_t>* elems, std::vector<int32_t>* cptr) {
  const int m = (int)elems->size() / k;
  // neighbours: elements sharing a vertex
  std::vector<std::vector<int>> inc(n);
  for (int e = 0; e < m; ++e)
    for (int j = 0; j < k; ++j) inc[(*elems)[(size_t)k * e + j]].push_back(e);
  std::vector<std::vector<int>> nb(m);
  for (int e = 0; e < m; ++e) {
    for (int j = 0; j < k; ++j)
      for (int f : inc[(*elems)[(size_t)k * e + j]])
        if (f != e) nb[e].push_back(f);
    std::sort(nb[e].begin(), nb[e].end());
    nb[e].erase(std::unique(nb[e].begin(), nb[e].end()), nb[e].end());
  }
  // 1. DSatur
  std::vector<int> colour(m, -1), count;
  std::vector<uint64_t> seen(m, 0);  // colours among the coloured neighbours
  std::set<std::array<int, 3>> queue;  // (-saturation, -degree, e): first is next
  for (int e = 0; e < m; ++e) queue.insert({0, -(int)nb[e].size(), e});
  while (!queue.empty()) {
    const int e = (*queue.begin())[2];
    queue.erase(queue.begin());
    int best = -1;
    for (int c = 0; c < (int)count.size(); ++c)
      if (!((seen[e] >> c) & 1u) && (best < 0 || count[c] < count[best])) best = c;
    if (best < 0) {
      if ((int)count.size() == kMaxColours) return false;
      best = (int)count.size();
      count.push_back(0);
    }
    colour[e] = best;
    ++count[best];
    for (int f : nb[e]) {
      if (colour[f] >= 0 || ((seen[f] >> best) & 1u)) continue;
      queue.erase({-__builtin_popcountll(seen[f]), -(int)nb[f].size(), f});
      seen[f] |= uint64_t(1) << best;
      queue.insert({-__builtin_popcountll(seen[f]), -(int)nb[f].size(), f});
    }
  }
  // 2. balancing
  const int nc = (int)count.size();
  auto passes = [&](int size) { return (size + nt - 1) / nt; };
  auto room = [&](int c) { return passes(count[c] + 1) == passes(count[c]) && count[c] > 0; };
  auto move_one = [&](int from) {  // one element of `from` to the fullest colour with room
    for (int e = 0; e < m; ++e) {
      if (colour[e] != from) continue;
      uint64_t taken = 0;
      for (int f : nb[e]) taken |= uint64_t(1) << colour[f];
      int to = -1;
      for (int c = 0; c < nc; ++c)
        if (c != from && !((taken >> c) & 1u) && room(c) && (to < 0 || count[c] % nt > count[to] % nt)) to = c;
      if (to >= 0) {
        colour[e] = to;
        --count[from];
        ++count[to];
        return true;
      }
    }
    return false;
  };
  std::vector<char> stuck(nc, 0);
  for (;;) {  // colours spilling into an extra pass, emptiest last pass first
    int c = -1;
    for (int d = 0; d < nc; ++d)
      if (!stuck[d] && count[d] > nt && count[d] % nt != 0 && (c < 0 || count[d] % nt < count[c] % nt)) c = d;
    if (c < 0) break;
    const int target = count[c] - count[c] % nt;
    while (count[c] > target && move_one(c)) {
    }
    if (count[c] > target) stuck[c] = 1;
  }
  std::fill(stuck.begin(), stuck.end(), 0);
  for (;;) {  // the smallest colours, emptied if they can be
    int c = -1;
    for (int d = 0; d < nc; ++d)
      if (!stuck[d] && count[d] > 0 && count[d] < nt && (c < 0 || count[d] < count[c])) c = d;
    if (c < 0) break;
    const std::vector<int> save = colour, save_count = count;
    while (count[c] > 0 && move_one(c)) {
    }
    if (count[c] > 0) {  // partly emptied: no pass saved, undo
      colour = save;
      count = save_count;
      stuck[c] = 1;
    }
  }
  // renumber the non-empty colours in order, and lay the elements out colour by colour
  std::vector<int> renum(nc, -1);
  int used = 0;
  for (int c = 0; c < nc; ++c)
    if (count[c] > 0) renum[c] = used++;
  cptr->assign(used + 1, 0);
  for (int e = 0; e < m; ++e) ++(*cptr)[renum[colour[e]] + 1];
  for (int c = 0; c < used; ++c) (*cptr)[c + 1] += (*cptr)[c];
  std::vector<int32_t> next(cptr->begin(), cptr->end() - 1), out(elems->size());
  for (int e = 0; e < m; ++e) {
    const int p = next[renum[colour[e]]]++;
    for (int j = 0; j < k; ++j) out[(size_t)k * p + j] = (*elems)[(size_t)k * e + j];
  }
  // 3. shared-memory banks: a warp of the CTA kernels takes 32 consecutive elements of a
  // class, and its loads of the elements' j-th vertices (x_v at word 3v of the shared
  // arrays, bank 3v mod 32) are conflict-free when those vertices differ mod 32.  Within
  // each class, elements are dealt to warps greedily, each slot taking the element (and,
  // for triangles, the cyclic rotation of its vertices, which keeps its orientation) that
  // adds the fewest repeats of a residue at any vertex position.
  {
    std::vector<int32_t> dealt(out.size());
    std::vector<int> pool;
    for (size_t c = 0; c + 1 < cptr->size(); ++c) {
      const int lo = (*cptr)[c], hi = (*cptr)[c + 1];
      pool.clear();
      for (int e = lo; e < hi; ++e) pool.push_back(e);
      int slot = lo;
      while (!pool.empty()) {
        int cnt[4][32] = {};
        for (int w = 0; w < 32 && !pool.empty(); ++w, ++slot) {
          int best = -1, best_rot = 0, best_cost = 1 << 30;
          for (int q = 0; q < (int)pool.size(); ++q) {
            const int32_t* el = &out[(size_t)k * pool[q]];
            for (int r = 0; r < (k == 3 ? 3 : 1); ++r) {
              int cost = 0;
              for (int j = 0; j < k; ++j) cost += cnt[j][el[(j + r) % k] & 31];
              if (cost < best_cost) {
                best_cost = cost;
                best = q;
                best_rot = r;
              }
            }
            if (best_cost == 0) break;
          }
          const int32_t* el = &out[(size_t)k * pool[best]];
          for (int j = 0; j < k; ++j) {
            const int32_t vj = el[(j + best_rot) % k];
            dealt[(size_t)k * slot + j] = vj;
            ++cnt[j][vj & 31];
          }
          pool.erase(pool.begin() + best);
        }
      }
      // then pairwise exchanges between the class's warps (with re-rotation of
      // triangles) while they lower the number of same-residue pairs in some warp
      const int nwarps = (hi - lo + 31) / 32;
      if (nwarps < 2) continue;
      std::vector<std::array<std::array<int, 32>, 4>> hist(nwarps);
      for (auto& hw : hist)
        for (auto& hp : hw) hp.fill(0);
      for (int e = lo; e < hi; ++e)
        for (int j = 0; j < k; ++j) ++hist[(e - lo) / 32][j][dealt[(size_t)k * e + j] & 31];
      for (int sweep = 0; sweep < 4; ++sweep) {
        bool improved = false;
        for (int a = lo; a < hi; ++a)
          for (int b = a + 1; b < hi; ++b) {
            const int wa = (a - lo) / 32, wb = (b - lo) / 32;
            if (wa == wb) continue;
            int32_t* ea = &dealt[(size_t)k * a];
            int32_t* eb = &dealt[(size_t)k * b];
            // gain of moving b's vertices into warp a (rotation rb) and a's into warp b (ra)
            int delta_best = 0, rab = 0, rbb = 0;
            for (int ra = 0; ra < (k == 3 ? 3 : 1); ++ra)
              for (int rb = 0; rb < (k == 3 ? 3 : 1); ++rb) {
                int delta = 0;
                for (int j = 0; j < k; ++j) {
                  const int xa = ea[j] & 31, xb = eb[j] & 31;            // current residues
                  const int na = ea[(j + ra) % k] & 31, nb = eb[(j + rb) % k] & 31;  // new
                  // warp a loses xa, gains nb; warp b loses xb, gains na (pair counts)
                  int ca = hist[wa][j][xa] - 1, cb = hist[wb][j][xb] - 1;
                  delta -= ca + cb;
                  delta += (nb == xa ? ca : hist[wa][j][nb]) + (na == xb ? cb : hist[wb][j][na]);
                }
                if (delta < delta_best) {
                  delta_best = delta;
                  rab = ra;
                  rbb = rb;
                }
              }
            if (delta_best < 0) {
              int32_t na[4], nb[4];
              for (int j = 0; j < k; ++j) {
                na[j] = ea[(j + rab) % k];
                nb[j] = eb[(j + rbb) % k];
              }
              for (int j = 0; j < k; ++j) {
                --hist[wa][j][ea[j] & 31];
                --hist[wb][j][eb[j] & 31];
                ea[j] = nb[j];
                eb[j] = na[j];
                ++hist[wa][j][ea[j] & 31];
                ++hist[wb][j][eb[j] & 31];
              }
              improved = true;
            }
          }
        if (!improved) break;
      }
    }
    out.swap(dealt);
  }
  // the invariant the CTA kernels rely on, checked as built: within a class, every vertex
  // occurs at most once
  std::vector<int> vseen(n, -1);
  for (size_t c = 0; c + 1 < cptr->size(); ++c)
    for (int e = (*cptr)[c]; e < (*cptr)[c + 1]; ++e)
      for (int j = 0; j < k; ++j) {
        const int v = out[(size_t)k * e + j];
        if (vseen[v] == (int)c) return false;
        vseen[v] = (int)c;
      }
  elems->swap(out);
  return true;
}

// ---------------------------------------------------------------- orderings
using Graph = std::vector<std::vector<int>>;

// Geometric nested dissection: split along the longest axis at the median; the
// separator is the set of left-side vertices with a neighbour on the right side.
void nested_dissection(const Graph& g, const std::vector<V3>& p, std::vector<int> idx,
                       std::vector<int>* order, int leaf) {
  if ((int)idx.size() <= leaf) {
    order->insert(order->end(), idx.begin(), idx.end());
    return;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v : idx) {
    const double c[3] = {p[v].x, p[v].y, p[v].z};
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], c[k]);
      hi[k] = std::max(hi[k], c[k]);
    }
  }
  int ax = 0;
  for (int k = 1; k < 3; ++k)
    if (hi[k] - lo[k] > hi[ax] - lo[ax]) ax = k;
  auto coord = [&](int v) { return ax == 0 ? p[v].x : (ax == 1 ? p[v].y : p[v].z); };
  std::vector<int> sorted = idx;
  std::sort(sorted.begin(), sorted.end(), [&](int a, int b) {
    double ca = coord(a), cb = coord(b);
    return ca < cb || (ca == cb && a < b);
  });
  size_t half = sorted.size() / 2;
  std::vector<char> side(p.size(), 2);  // 0 left, 1 right, 2 outside this subproblem
  for (size_t i = 0; i < sorted.size(); ++i) side[sorted[i]] = i < half ? 0 : 1;
  std::vector<int> left, right, sep;
  for (int v : sorted) {
    if (side[v] == 1) {
      right.push_back(v);
      continue;
    }
    bool touches = false;
    for (int u : g[v])
      if (side[u] == 1) {
        touches = true;
        break;
      }
    (touches ? sep : left).push_back(v);
  }
  if (left.empty() || right.empty()) {  // cannot split further
    order->insert(order->end(), idx.begin(), idx.end());
    return;
  }
  std::sort(left.begin(), left.end());
  std::sort(right.begin(), right.end());
  nested_dissection(g, p, left, order, leaf);
  nested_dissection(g, p, right, order, leaf);
  order->insert(order->end(), sep.begin(), sep.end());
}

// Nested dissection with a searched separator: at every level, try cut planes of several
// directions (given unit vectors) at several quantile positions, take the vertices on one
// side that touch the other side as the separator (either side), and keep the smallest
// separator.  Subproblems of at most `leaf` vertices are ordered as they stand.
void searched_dissection(const Graph& g, const std::vector<V3>& p, const std::vector<V3>& dirs,
                         std::vector<int> idx, std::vector<int>* order, int leaf) {
  if ((int)idx.size() <= leaf) {
    order->insert(order->end(), idx.begin(), idx.end());
    return;
  }
  static const double kFractions[] = {0.4, 0.45, 0.5, 0.55, 0.6};
  std::vector<char> side(p.size(), 2);  // 0 lower, 1 upper, 2 outside this subproblem
  std::vector<int> best_lo, best_hi, best_sep;
  size_t best = SIZE_MAX;
  std::vector<int> sorted;
  for (const V3& d : dirs) {
    sorted = idx;
    std::sort(sorted.begin(), sorted.end(), [&](int a, int b) {
      const double ca = dot(p[a], d), cb = dot(p[b], d);
      return ca < cb || (ca == cb && a < b);
    });
    for (double fr : kFractions) {
      const size_t cut = (size_t)(fr * (double)sorted.size());
      for (size_t i = 0; i < sorted.size(); ++i) side[sorted[i]] = i < cut ? 0 : 1;
      for (char sep_side = 0; sep_side < 2; ++sep_side) {
        std::vector<int> lo, hi, sep;
        for (int v : sorted) {
          bool on_sep = false;
          if (side[v] == sep_side)
            for (int u : g[v])
              if (side[u] == 1 - sep_side) {
                on_sep = true;
                break;
              }
          (on_sep ? sep : (side[v] == 0 ? lo : hi)).push_back(v);
        }
        if (!lo.empty() && !hi.empty() && sep.size() < best) {
          best = sep.size();
          best_lo.swap(lo);
          best_hi.swap(hi);
          best_sep.swap(sep);
        }
      }
    }
    for (int v : idx) side[v] = 2;
  }
  if (best == SIZE_MAX) {  // cannot split further
    order->insert(order->end(), idx.begin(), idx.end());
    return;
  }
  std::sort(best_lo.begin(), best_lo.end());
  std::sort(best_hi.begin(), best_hi.end());
  searched_dissection(g, p, dirs, best_lo, order, leaf);
  searched_dissection(g, p, dirs, best_hi, order, leaf);
  order->insert(order->end(), best_sep.begin(), best_sep.end());
}

// Cut directions for searched_dissection: the three axes, the ten face and space
// diagonals of a cube (up to sign), and 30 points of a Fibonacci lattice on the upper
// hemisphere (deterministic).
std::vector<V3> cut_directions() {
  std::vector<V3> d = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1},
                       {0, 1, -1}, {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {-1, 1, 1}};
  const double golden = 3.14159265358979323846 * (3.0 - std::sqrt(5.0));
  const int m = 30;
  for (int k = 0; k < m; ++k) {
    const double z = 1.0 - (k + 0.5) / m;  // (0, 1): upper hemisphere
    const double r = std::sqrt(1.0 - z * z);
    d.push_back({r * std::cos(golden * k), r * std::sin(golden * k), z});
  }
  for (V3& v : d) {
    const double l = norm(v);
    v = {v.x / l, v.y / l, v.z / l};
  }
  return d;
}

// Smallest vertex separator along the cut edges of a two-sided split: a minimum vertex
// cover of the bipartite graph of cut edges.  By König's theorem, with a maximum matching
// M and Z the vertices reachable from unmatched lower-side vertices by alternating paths,
// the cover is (lower \ Z) ∪ (upper ∩ Z).  side[v]: 0 lower, 1 upper, 2 outside this
// subproblem; `pos` is scratch of size n, all -1 on entry and on return.
std::vector<int> cut_cover(const Graph& g, const std::vector<char>& side, const std::vector<int>& idx,
                           std::vector<int>& pos) {
  std::vector<int> A, B;
  for (int v : idx) {
    bool cut = false;
    for (int u : g[v])
      if (side[u] == 1 - side[v]) {
        cut = true;
        break;
      }
    if (cut) {
      std::vector<int>& s = side[v] == 0 ? A : B;
      pos[v] = (int)s.size();
      s.push_back(v);
    }
  }
  std::vector<int> aptr(A.size() + 1, 0), adj;
  for (size_t a = 0; a < A.size(); ++a) {
    for (int u : g[A[a]])
      if (side[u] == 1) adj.push_back(pos[u]);
    aptr[a + 1] = (int)adj.size();
  }
  std::vector<int> mate_a(A.size(), -1), mate_b(B.size(), -1);
  std::vector<char> seen;
  // Kuhn's augmenting-path search from lower vertex a.
  std::function<bool(int)> augment = [&](int a) -> bool {
    for (int q = aptr[a]; q < aptr[a + 1]; ++q) {
      const int b = adj[q];
      if (seen[b]) continue;
      seen[b] = 1;
      if (mate_b[b] < 0 || augment(mate_b[b])) {
        mate_a[a] = b;
        mate_b[b] = a;
        return true;
      }
    }
    return false;
  };
  for (size_t a = 0; a < A.size(); ++a) {
    seen.assign(B.size(), 0);
    augment((int)a);
  }
  std::vector<char> za(A.size(), 0), zb(B.size(), 0);
  std::vector<int> stack;
  for (size_t a = 0; a < A.size(); ++a)
    if (mate_a[a] < 0) {
      za[a] = 1;
      stack.push_back((int)a);
    }
  while (!stack.empty()) {
    const int a = stack.back();
    stack.pop_back();
    for (int q = aptr[a]; q < aptr[a + 1]; ++q) {
      const int b = adj[q];
      if (!zb[b]) {
        zb[b] = 1;
        const int a2 = mate_b[b];
        if (a2 >= 0 && !za[a2]) {
          za[a2] = 1;
          stack.push_back(a2);
        }
      }
    }
  }
  std::vector<int> cover;
  for (size_t a = 0; a < A.size(); ++a)
    if (!za[a]) cover.push_back(A[a]);
  for (size_t b = 0; b < B.size(); ++b)
    if (zb[b]) cover.push_back(B[b]);
  for (int v : A) pos[v] = -1;
  for (int v : B) pos[v] = -1;
  return cover;
}

// Nested dissection with searched cut planes and cut-cover separators: at every level, for
// cut planes of the given directions at the 35–65 % quantiles, the separator is the
// minimum cover of the cut edges; the kept split minimises |S| (1 + bal (max(|L|,|U|) /
// (|L| + |U|) − 1/2)).  Every leaf and separator is one block; stage[v] numbers the blocks
// in elimination order.
void covered_dissection(const Graph& g, const std::vector<V3>& p, const std::vector<V3>& dirs,
                        std::vector<int> idx, std::vector<int>* order, std::vector<int>* stage, int* nstage,
                        int leaf, double bal, std::vector<char>& side, std::vector<int>& pos) {
  auto emit = [&](const std::vector<int>& block) {
    for (int v : block) (*stage)[v] = *nstage;
    ++*nstage;
    order->insert(order->end(), block.begin(), block.end());
  };
  if ((int)idx.size() <= leaf) {
    emit(idx);
    return;
  }
  static const double kFractions[] = {0.35, 0.4, 0.45, 0.5, 0.55, 0.6, 0.65};
  std::vector<int> sorted, best_sep;
  size_t best_dir = 0, best_cut = 0;
  double best = 1e300;
  for (size_t di = 0; di < dirs.size(); ++di) {
    const V3 d = dirs[di];
    sorted = idx;
    std::sort(sorted.begin(), sorted.end(), [&](int a, int b) {
      const double ca = dot(p[a], d), cb = dot(p[b], d);
      return ca < cb || (ca == cb && a < b);
    });
    for (double fr : kFractions) {
      const size_t cut = (size_t)(fr * (double)sorted.size());
      for (size_t i = 0; i < sorted.size(); ++i) side[sorted[i]] = i < cut ? 0 : 1;
      std::vector<int> sep = cut_cover(g, side, idx, pos);
      size_t nlo = cut, nhi = sorted.size() - cut;
      for (int v : sep) --(side[v] == 0 ? nlo : nhi);
      if (nlo > 0 && nhi > 0) {
        const double big = (double)std::max(nlo, nhi), both = (double)(nlo + nhi);
        const double score = (double)sep.size() * (1.0 + bal * (big / both - 0.5));
        if (score < best) {
          best = score;
          best_dir = di;
          best_cut = cut;
          best_sep.swap(sep);
        }
      }
    }
  }
  if (best > 1e299) {  // cannot split further
    for (int v : idx) side[v] = 2;
    emit(idx);
    return;
  }
  // rebuild the kept split
  const V3 d = dirs[best_dir];
  sorted = idx;
  std::sort(sorted.begin(), sorted.end(), [&](int a, int b) {
    const double ca = dot(p[a], d), cb = dot(p[b], d);
    return ca < cb || (ca == cb && a < b);
  });
  for (size_t i = 0; i < sorted.size(); ++i) side[sorted[i]] = i < best_cut ? 0 : 1;
  for (int v : best_sep) side[v] = 3;
  std::vector<int> best_lo, best_hi;
  for (int v : sorted)
    if (side[v] != 3) (side[v] == 0 ? best_lo : best_hi).push_back(v);
  for (int v : idx) side[v] = 2;
  std::sort(best_lo.begin(), best_lo.end());
  std::sort(best_hi.begin(), best_hi.end());
  covered_dissection(g, p, dirs, best_lo, order, stage, nstage, leaf, bal, side, pos);
  covered_dissection(g, p, dirs, best_hi, order, stage, nstage, leaf, bal, side, pos);
  emit(best_sep);
}

// Minimum degree constrained to a block order: the elimination graph is that of the whole
// pattern, and the next vertex is one of least degree among the earliest block not yet
// eliminated (reorders the vertices inside every leaf and separator of a dissection; the
// last block, the top separator, keeps its order: its fill is dense whatever the order).
std::vector<int> constrained_minimum_degree(const Graph& g, const std::vector<int>& stage, int nstage) {
  const int n = (int)g.size();
  std::vector<std::vector<int>> nb(n);  // sorted neighbour lists of the elimination graph
  for (int v = 0; v < n; ++v) {
    for (int u : g[v])
      if (u != v) nb[v].push_back(u);
    std::sort(nb[v].begin(), nb[v].end());
    nb[v].erase(std::unique(nb[v].begin(), nb[v].end()), nb[v].end());
  }
  std::set<std::array<int, 3>> pq;
  for (int v = 0; v < n; ++v) pq.insert({stage[v], (int)nb[v].size(), v});
  std::vector<int> order, merged;
  order.reserve(n);
  while (!pq.empty()) {
    if ((*pq.begin())[0] == nstage - 1) {
      for (int v = 0; v < n; ++v)
        if (stage[v] == nstage - 1) order.push_back(v);
      break;
    }
    const int v = (*pq.begin())[2];
    pq.erase(pq.begin());
    order.push_back(v);
    const std::vector<int> N = nb[v];
    for (int a : N) {  // eliminating v joins its neighbours into a clique
      pq.erase({stage[a], (int)nb[a].size(), a});
      merged.clear();
      std::set_union(nb[a].begin(), nb[a].end(), N.begin(), N.end(), std::back_inserter(merged));
      merged.erase(std::remove_if(merged.begin(), merged.end(), [&](int x) { return x == a || x == v; }),
                   merged.end());
      nb[a].swap(merged);
      pq.insert({stage[a], (int)nb[a].size(), a});
    }
  }
  return order;
}

// Exact minimum degree on the elimination graph (small n only).
std::vector<int> minimum_degree(const Graph& g) {
  int n = (int)g.size();
  std::vector<std::set<int>> nb(n);
  for (int v = 0; v < n; ++v)
    for (int u : g[v])
      if (u != v) nb[v].insert(u);
  std::vector<char> alive(n, 1);
  std::set<std::pair<int, int>> pq;
  for (int v = 0; v < n; ++v) pq.insert({(int)nb[v].size(), v});
  std::vector<int> order;
  order.reserve(n);
  while (!pq.empty()) {
    int v = pq.begin()->second;
    pq.erase(pq.begin());
    alive[v] = 0;
    order.push_back(v);
    std::vector<int> N(nb[v].begin(), nb[v].end());
    for (int a : N) {
      pq.erase({(int)nb[a].size(), a});
      nb[a].erase(v);
      for (int b : N)
        if (b != a) nb[a].insert(b);
      pq.insert({(int)nb[a].size(), a});
    }
  }
  return order;
}

// Symbolic factorisation of the permuted pattern: column structures (rows > j).
int64_t symbolic(const Graph& g, const std::vector<int>& order, std::vector<std::vector<int>>* cols) {
  int n = (int)g.size();
  std::vector<int> inv(n);
  for (int i = 0; i < n; ++i) inv[order[i]] = i;
  std::vector<std::vector<int>> children(n);
  cols->assign(n, {});
  int64_t nnz = 0;
  for (int j = 0; j < n; ++j) {
    std::set<int> s;
    for (int u : g[order[j]]) {
      int r = inv[u];
      if (r > j) s.insert(r);
    }
    for (int c : children[j])
      for (int r : (*cols)[c])
        if (r > j) s.insert(r);
    (*cols)[j].assign(s.begin(), s.end());
    nnz += (int64_t)s.size();
    if (!s.empty()) children[*s.begin()].push_back(j);
  }
  return nnz;
}

}  // namespace

// Pack the updates of one sweep into levels of W sub-chunks of kChunk updates (one per
// lane; W = 1: one warp's chunks): every level's sources are final before it starts,
// its targets are distinct, and in each sub-chunk at most kBankCap targets share a
// shared-memory bank class (t mod 16; a row of three doubles starts at bank 6t mod 32).
// Greedy list scheduling, sources with the longest remaining dependency chain first;
// sub-chunks fill in order.  A level that reads or writes a row written since the last
// synchronisation gets bit 0 (synchronise first), so the levels between two
// synchronisations commute.  `relabel` maps r -> n-1-r when emitting indices.
void pack_sweep(int n, const std::vector<SweepOp>& ops, bool relabel, int W, std::vector<int32_t>* meta,
                std::vector<uint32_t>* rc, std::vector<double>* val) {
  constexpr int kBankCap = 3;
  const int width = W * kChunk;
  std::vector<std::vector<int>> by_src(n);
  std::vector<int> remaining(n, 0);
  for (int k = 0; k < (int)ops.size(); ++k) {
    by_src[ops[k].s].push_back(k);
    remaining[ops[k].t]++;
  }
  std::vector<int> dist(n, 0);
  for (int s = n - 1; s >= 0; --s) {
    int d = 0;
    for (int k : by_src[s]) d = std::max(d, 1 + dist[ops[k].t]);
    dist[s] = d;
  }
  std::set<std::pair<int, int>> ready;  // (-dist, source) with pending updates
  std::vector<size_t> next(n, 0);       // next pending update of each source
  for (int s = 0; s < n; ++s)
    if (remaining[s] == 0 && !by_src[s].empty()) ready.insert({-dist[s], s});
  auto emit_index = [&](int r) { return relabel ? n - 1 - r : r; };
  std::vector<char> dirty(n + 1, 0), in_level(n + 1, 0);
  std::vector<int> dirty_list;
  size_t done = 0;
  while (done < ops.size()) {
    std::vector<std::vector<int>> sub(W);
    std::vector<std::array<int, 16>> cls(W);
    for (auto& c : cls) c.fill(0);
    int count = 0;
    std::vector<std::pair<int, int>> revisit;
    while (!ready.empty() && count < width) {
      auto it = ready.begin();
      auto key = *it;
      ready.erase(it);
      int s = key.second;
      std::vector<int>& lst = by_src[s];
      std::vector<int> keep;
      for (size_t q = next[s]; q < lst.size(); ++q) {
        int k = lst[q];
        int t = ops[k].t;
        const int b = emit_index(t) & 15;
        int w = 0;
        while (w < W && ((int)sub[w].size() >= kChunk || cls[w][b] >= kBankCap)) ++w;
        if (count < width && !in_level[t] && w < W) {
          sub[w].push_back(k);
          in_level[t] = 1;
          cls[w][b]++;
          ++count;
        } else {
          keep.push_back(k);
        }
      }
      if (!keep.empty()) {
        lst.assign(keep.begin(), keep.end());
        next[s] = 0;
        revisit.push_back(key);
      } else {
        next[s] = lst.size();
      }
    }
    for (auto& key : revisit) ready.insert(key);
    // hazard with rows written since the last synchronisation
    bool hazard = false;
    for (auto& sc : sub)
      for (int k : sc)
        if (dirty[ops[k].t] || dirty[ops[k].s]) hazard = true;
    if (hazard) {
      for (int r : dirty_list) dirty[r] = 0;
      dirty_list.clear();
    }
    for (int w = 0; w < W; ++w) {
      meta->push_back((hazard ? 1 : 0) | (sub[w].empty() && W > 1 ? 2 : 0));
      for (int l = 0; l < kChunk; ++l) {
        if (l < (int)sub[w].size()) {
          const SweepOp& op = ops[sub[w][l]];
          rc->push_back((uint32_t)emit_index(op.t) | ((uint32_t)emit_index(op.s) << 16));
          val->push_back(op.v);
        } else {
          rc->push_back((uint32_t)n | ((uint32_t)n << 16));
          val->push_back(0.0);
        }
      }
    }
    for (auto& sc : sub)
      for (int k : sc) {
        int t = ops[k].t;
        in_level[t] = 0;
        if (!dirty[t]) {
          dirty[t] = 1;
          dirty_list.push_back(t);
        }
      }
    done += count;
    for (auto& sc : sub)
      for (int k : sc) {
        int t = ops[k].t;
        if (--remaining[t] == 0 && !by_src[t].empty()) ready.insert({-dist[t], t});
      }
  }
}

int build_host_type(int n, int T, const double* xyz, const int32_t* tris, double w_strain,
                    double w_bend, double w_area, double w_vol, double density, double dt,
                    double c_alpha, double c_beta, HostType* out, std::string* err) {
  if (n < 4 || T < 4 || !xyz || !tris || !(dt > 0) || !(density > 0)) {
    *err = "create_cell_type: need n >= 4, T >= 4, dt > 0, density > 0 and non-null arrays";
    return NPFEM_ERR_INVALID_ARG;
  }
  if (!(c_alpha >= 0) || !(c_beta >= 0) || std::isinf(c_alpha) || std::isinf(c_beta)) {
    *err = "create_cell_type: damping c_alpha and c_beta must be finite and >= 0";
    return NPFEM_ERR_INVALID_ARG;
  }
  if (n > 65535) {
    *err = "create_cell_type: at most 65535 vertices per cell type";
    return NPFEM_ERR_UNSUPPORTED;
  }
  HostType& H = *out;
  H.n = n;
  H.T = T;
  H.dt = dt;
  H.c_alpha = c_alpha;
  H.c_beta = c_beta;
  H.w_area = w_area;
  H.w_vol = w_vol;
  H.tris.assign(tris, tris + 3 * T);
  std::vector<V3> X(n);
  for (int i = 0; i < n; ++i) X[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
  for (int k = 0; k < 3 * T; ++k)
    if (tris[k] < 0 || tris[k] >= n) {
      *err = "create_cell_type: triangle index out of range";
      return NPFEM_ERR_BAD_MESH;
    }

  // ---- topology: each directed edge once, each undirected edge in both directions
  std::map<std::pair<int, int>, int> directed;  // (a,b) -> opposite vertex
  for (int t = 0; t < T; ++t) {
    const int* v = &tris[3 * t];
    for (int k = 0; k < 3; ++k) {
      int a = v[k], b = v[(k + 1) % 3], c = v[(k + 2) % 3];
      if (a == b || b == c || a == c) {
        *err = "create_cell_type: triangle with repeated vertex";
        return NPFEM_ERR_BAD_MESH;
      }
      if (!directed.emplace(std::make_pair(a, b), c).second) {
        *err = "create_cell_type: edge traversed twice in one direction (non-manifold or inconsistent orientation)";
        return NPFEM_ERR_BAD_MESH;
      }
    }
  }
  for (auto& kv : directed) {
    int a = kv.first.first, b = kv.first.second;
    if (a < b) {
      auto it = directed.find({b, a});
      if (it == directed.end()) {
        *err = "create_cell_type: open edge (mesh is not closed)";
        return NPFEM_ERR_BAD_MESH;
      }
      H.hinges.insert(H.hinges.end(), {a, b, kv.second, it->second});
    }
  }
  H.E = (int)H.hinges.size() / 4;
  if (2 * H.E != 3 * T) {
    *err = "create_cell_type: mesh is not a closed manifold";
    return NPFEM_ERR_BAD_MESH;
  }
  // ---- elements in colour order (each triangle keeps its vertex order, hence its
  // orientation); every per-element table below follows this order
  const int nt = 32 * default_cta_warps(n);
  if (!colour_elements(n, 3, nt, &H.tris, &H.tri_cptr) || !colour_elements(n, 4, nt, &H.hinges, &H.hinge_cptr)) {
    H.tri_cptr.clear();
    H.hinge_cptr.clear();
  }
  tris = H.tris.data();

  // ---- per-triangle rest frame: Dm = [[|e1|, e2.u], [0, e2.w]], F = [e1 e2] Dm^-1
  H.Dinv.resize(3 * T);
  H.w_tri.resize(T);
  std::vector<double> area(T);
  std::vector<double> vert_area(n, 0.0);
  double A0 = 0.0;
  for (int t = 0; t < T; ++t) {
    V3 x0 = X[tris[3 * t]], x1 = X[tris[3 * t + 1]], x2 = X[tris[3 * t + 2]];
    V3 e1 = sub(x1, x0), e2 = sub(x2, x0);
    V3 cr = cross(e1, e2);
    double crn = norm(cr);
    if (!(crn > 0.0)) {
      *err = "create_cell_type: degenerate rest triangle";
      return NPFEM_ERR_BAD_MESH;
    }
    double l1 = norm(e1);
    double a01 = dot(e2, e1) / l1;  // e2 . u
    double a11 = crn / l1;          // e2 . w  (w = n x u)
    // inverse of [[l1, a01], [0, a11]]
    H.Dinv[3 * t + 0] = 1.0 / l1;
    H.Dinv[3 * t + 1] = -a01 / (l1 * a11);
    H.Dinv[3 * t + 2] = 1.0 / a11;
    area[t] = 0.5 * crn;
    H.w_tri[t] = w_strain * area[t];
    A0 += area[t];
    for (int k = 0; k < 3; ++k) vert_area[tris[3 * t + k]] += area[t] / 3.0;
  }
  H.A0 = A0;
  H.area = area;
  V3 ctr{0, 0, 0};
  for (auto& p : X) ctr = {ctr.x + p.x / n, ctr.y + p.y / n, ctr.z + p.z / n};
  double V0 = 0.0;
  for (int t = 0; t < T; ++t) {
    V3 a = sub(X[tris[3 * t]], ctr), b = sub(X[tris[3 * t + 1]], ctr), c = sub(X[tris[3 * t + 2]], ctr);
    V0 += dot(a, cross(b, c)) / 6.0;
  }
  if (!(V0 > 0.0)) {
    *err = "create_cell_type: non-positive rest volume (mesh must be oriented outward)";
    return NPFEM_ERR_BAD_MESH;
  }
  H.V0 = V0;
  H.mass.resize(n);
  H.total_mass = density * V0;
  for (int i = 0; i < n; ++i) H.mass[i] = density * V0 * vert_area[i] / A0;

  // ---- hinges: cotangent stencil with rest cotangents, |K0|, weight
  int E = H.E;
  H.c_hinge.resize(4 * E);
  H.K0.resize(4 * E);
  H.w_hinge.resize(E);
  H.hinge_unit.resize(E);
  for (int e = 0; e < E; ++e) {
    const int* h = &H.hinges[4 * e];
    V3 p0 = X[h[0]], p1 = X[h[1]], p2 = X[h[2]], p3 = X[h[3]];
    double cA0 = cotangent(sub(p1, p0), sub(p2, p0));
    double cA1 = cotangent(sub(p0, p1), sub(p2, p1));
    double cB0 = cotangent(sub(p1, p0), sub(p3, p0));
    double cB1 = cotangent(sub(p0, p1), sub(p3, p1));
    double c[4] = {cA1 + cB1, cA0 + cB0, -(cA0 + cA1), -(cB0 + cB1)};
    V3 K{0, 0, 0};
    const V3 d[3] = {sub(p1, p0), sub(p2, p0), sub(p3, p0)};
    for (int k = 0; k < 3; ++k) K = {K.x + c[k + 1] * d[k].x, K.y + c[k + 1] * d[k].y, K.z + c[k + 1] * d[k].z};
    for (int k = 0; k < 4; ++k) H.c_hinge[4 * e + k] = c[k];
    H.K0[4 * e + 0] = K.x;
    H.K0[4 * e + 1] = K.y;
    H.K0[4 * e + 2] = K.z;
    H.K0[4 * e + 3] = norm(K);
    double aA = 0.5 * norm(cross(sub(p1, p0), sub(p2, p0)));
    double aB = 0.5 * norm(cross(sub(p1, p0), sub(p3, p0)));
    H.hinge_unit[e] = 3.0 / (aA + aB);
    H.w_hinge[e] = w_bend * H.hinge_unit[e];
  }

  // ---- gradient gather lists
  {
    std::vector<std::vector<std::pair<int32_t, double>>> inc(n);
    for (int t = 0; t < T; ++t)
      for (int k = 0; k < 3; ++k) inc[tris[3 * t + k]].push_back({t * 3 + k, 0.0});
    for (int e = 0; e < E; ++e)
      for (int k = 0; k < 4; ++k) inc[H.hinges[4 * e + k]].push_back({-(e * 4 + k) - 1, H.c_hinge[4 * e + k]});
    H.inc_ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
      H.inc_ptr[i + 1] = H.inc_ptr[i] + (int)inc[i].size();
      for (auto& pr : inc[i]) {
        H.inc_code.push_back(pr.first);
        H.inc_coef.push_back(pr.second);
      }
    }
  }

  // ---- assemble A (sparse, symmetric): (1/dt^2 + c_alpha/dt) M + (1 + c_beta/dt) L,
  // the elastic part L scaled by ls (1 without damping)
  std::map<std::pair<int, int>, double> Aij;
  const double ls = 1.0 + c_beta / dt;
  for (int i = 0; i < n; ++i) Aij[{i, i}] += H.mass[i] * (1.0 / (dt * dt) + c_alpha / dt);
  for (int t = 0; t < T; ++t) {
    // G = Dm^-T S, S = [[-1,1,0],[-1,0,1]];  Dm^-1 = [[d00, d01], [0, d11]]
    double d00 = H.Dinv[3 * t], d01 = H.Dinv[3 * t + 1], d11 = H.Dinv[3 * t + 2];
    double G[2][3] = {{-d00, d00, 0.0}, {-(d01 + d11), d01, d11}};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double s = G[0][a] * G[0][b] + G[1][a] * G[1][b];
        Aij[{tris[3 * t + a], tris[3 * t + b]}] += ls * (H.w_tri[t] * s);
      }
  }
  for (int e = 0; e < E; ++e)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        Aij[{H.hinges[4 * e + a], H.hinges[4 * e + b]}] +=
            ls * (H.w_hinge[e] * H.c_hinge[4 * e + a] * H.c_hinge[4 * e + b]);
  Graph g(n);
  for (auto& kv : Aij)
    if (kv.first.first != kv.first.second) g[kv.first.first].push_back(kv.first.second);

  // ---- ordering: least fill among geometric nested dissections (longest axis at the
  // median; searched cut planes with one-sided or cut-cover separators, the latter also
  // reordered by constrained minimum degree) and minimum degree
  std::vector<int> best;
  std::vector<std::vector<int>> best_cols;
  int64_t best_nnz = -1;
  {
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::vector<std::vector<int>> orders;
    for (int leaf : {16, 32, 64}) {
      std::vector<int> o;
      nested_dissection(g, X, idx, &o, leaf);
      orders.push_back(o);
    }
    const std::vector<V3> dirs = cut_directions();
    for (int leaf : {4, 8}) {
      std::vector<int> o;
      searched_dissection(g, X, dirs, idx, &o, leaf);
      orders.push_back(o);
    }
    {
      std::vector<char> side(n, 2);
      std::vector<int> pos(n, -1);
      for (double bal : {0.3, 0.7}) {
        std::vector<int> o, stage(n, 0);
        int nstage = 0;
        covered_dissection(g, X, dirs, idx, &o, &stage, &nstage, 4, bal, side, pos);
        orders.push_back(constrained_minimum_degree(g, stage, nstage));
      }
    }
    if (n <= 1500) orders.push_back(minimum_degree(g));  // exact, quadratic-ish: small meshes only
    for (auto& o : orders) {
      std::vector<std::vector<int>> cols;
      int64_t nz = symbolic(g, o, &cols);
      if (best_nnz < 0 || nz < best_nnz) {
        best_nnz = nz;
        best = o;
        best_cols = std::move(cols);
      }
    }
  }
  H.perm.assign(best.begin(), best.end());
  H.nnz_factor = best_nnz;
  std::vector<int> inv(n);
  for (int i = 0; i < n; ++i) inv[best[i]] = i;

  // ---- numeric left-looking Cholesky on the symbolic pattern
  std::vector<std::vector<double>> Lval(n);
  std::vector<double> Ldiag(n);
  std::vector<std::vector<std::pair<int, int>>> rowlist(n);  // row r -> (col k, position in col k)
  for (int j = 0; j < n; ++j)
    for (size_t q = 0; q < best_cols[j].size(); ++q) rowlist[best_cols[j][q]].push_back({j, (int)q});
  std::vector<double> work(n, 0.0);
  for (int j = 0; j < n; ++j) {
    // scatter A(j:n, j) in permuted numbering
    int vj = best[j];
    work[j] = Aij[{vj, vj}];
    for (int u : g[vj]) {
      int r = inv[u];
      if (r > j) work[r] = Aij[{u, vj}];
    }
    // subtract sum_k L(j:n,k) L(j,k) over k with L(j,k) != 0
    for (auto& kq : rowlist[j]) {
      int k = kq.first;
      double ljk = Lval[k][kq.second];
      work[j] -= ljk * ljk;
      for (size_t q = kq.second + 1; q < best_cols[k].size(); ++q) work[best_cols[k][q]] -= Lval[k][q] * ljk;
    }
    double piv = work[j];
    if (!(piv > 0.0) || !std::isfinite(piv)) {
      char buf[160];
      std::snprintf(buf, sizeof buf, "create_cell_type: global matrix not positive definite (pivot %g at %d)", piv, j);
      *err = buf;
      return NPFEM_ERR_NOT_SPD;
    }
    double d = std::sqrt(piv);
    Ldiag[j] = d;
    work[j] = 0.0;
    Lval[j].resize(best_cols[j].size());
    for (size_t q = 0; q < best_cols[j].size(); ++q) {
      int r = best_cols[j][q];
      Lval[j][q] = work[r] / d;
      work[r] = 0.0;
    }
  }

  // ---- LDL^T form: Lt(i,j) = L(i,j)/L(j,j), D = L(j,j)^2
  H.dinv.resize(n);
  for (int j = 0; j < n; ++j) {
    H.dinv[j] = 1.0 / (Ldiag[j] * Ldiag[j]);
    for (auto& v : Lval[j]) v /= Ldiag[j];
  }
  // forward sweep (Lt y = z): z[i] -= Lt(i,j) z[j] for i > j; backward sweep
  // (Lt^T w = y): z[j] -= Lt(i,j) z[i], relabelled r -> n-1-r so that in both sweeps a
  // target index exceeds its source index
  std::vector<SweepOp> fwd, bwd;
  for (int j = 0; j < n; ++j)
    for (size_t q = 0; q < best_cols[j].size(); ++q) {
      int i = best_cols[j][q];
      fwd.push_back({i, j, Lval[j][q]});
      bwd.push_back({n - 1 - j, n - 1 - i, Lval[j][q]});
    }
  pack_sweep(n, fwd, false, 1, &H.fwd_meta, &H.fwd_rc, &H.fwd_val);
  pack_sweep(n, bwd, true, 1, &H.bwd_meta, &H.bwd_rc, &H.bwd_val);
  for (int i = 0; i < kCtaPacks; ++i) {
    HostType::LevelPack& P = H.cta[i];
    P.W = kCtaWarps[i];
    pack_sweep(n, fwd, false, P.W, &P.fwd_meta, &P.fwd_rc, &P.fwd_val);
    pack_sweep(n, bwd, true, P.W, &P.bwd_meta, &P.bwd_rc, &P.bwd_val);
  }
  return NPFEM_OK;
}

}  // namespace npfem
