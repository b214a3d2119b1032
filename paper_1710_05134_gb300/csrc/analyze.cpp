// Host symbolic phase of the sparse LDL^T (Section 3.3; task (i) of Section 4.3).
//
// The ordering Q and the symbolic factorization depend only on the common sparsity pattern of
// A and B, so they are computed once here and reused for every shift sigma.
//
//  1. Quotient graph: rows with identical off-diagonal adjacency (the orbitals of one atom) are
//     merged into one ordering vertex.
//  2. Nested dissection on the quotient graph: each piece is split at the weighted median of a
//     sort key (the coordinate of its widest axis when coordinates are given, else the
//     breadth-first level from a pseudo-peripheral vertex); the vertex separator is the lighter
//     of the two one-sided boundaries of that cut.  Periodic boundaries need no special case:
//     the wrap-around edges are part of the cut, so their boundary joins the separator.
//     Refined variant (option): several balanced cut positions on every long axis are tried, and
//     each cut's separator is a minimum-weight vertex cover of the bipartite graph of cut edges
//     (by Koenig's theorem a minimum cut of the unit-network src -> side 1 -> side 2 -> sink,
//     found with Dinic's max-flow algorithm); the cut with the lightest separator, weighted by
//     its imbalance, is taken.
//  3. Assembly tree: every ND node is one front whose fully-summed variables are the node's
//     variables; its contribution-block rows are its later neighbours plus its children's
//     contribution rows; its parent is the front owning the smallest of those rows.
//  4. Index maps: child contribution rows -> parent positions, original lower entries ->
//     (front, row, col), level schedule (tree height), device memory plan with slack rows for
//     pivots delayed from the children.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>

#include "kep_internal.h"

namespace kep {
namespace {

struct Quotient {
  int32_t ns = 0;
  std::vector<int32_t> sn_of;                 // row -> supernode
  std::vector<int64_t> mem_ptr;               // members of each supernode
  std::vector<int32_t> mem;
  std::vector<int64_t> qrp;                   // quotient adjacency
  std::vector<int32_t> qci;
  std::vector<int32_t> w;                     // weight = member count
};

uint64_t adj_hash(const int32_t* a, int64_t len, int32_t self) {
  uint64_t h = 1469598103934665603ull;
  for (int64_t i = 0; i < len; ++i) {
    if (a[i] == self) continue;
    h ^= static_cast<uint64_t>(a[i]) + 0x9e3779b97f4a7c15ull;
    h *= 1099511628211ull;
  }
  return h;
}

bool same_open_adj(const std::vector<int64_t>& rp, const std::vector<int32_t>& ci, int32_t x,
                   int32_t y) {
  int64_t i = rp[x], ie = rp[x + 1], j = rp[y], je = rp[y + 1];
  while (true) {
    while (i < ie && ci[i] == x) ++i;
    while (j < je && ci[j] == y) ++j;
    if (i == ie || j == je) return i == ie && j == je;
    if (ci[i] != ci[j]) return false;
    ++i; ++j;
  }
}

Quotient build_quotient(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci) {
  Quotient q;
  std::vector<uint64_t> h(n);
  for (int64_t i = 0; i < n; ++i)
    h[i] = adj_hash(ci.data() + rp[i], rp[i + 1] - rp[i], static_cast<int32_t>(i));
  std::vector<int32_t> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
    return h[a] != h[b] ? h[a] < h[b] : a < b;
  });
  q.sn_of.assign(n, -1);
  std::vector<int32_t> leaders;
  int64_t g0 = 0;
  while (g0 < n) {
    int64_t g1 = g0;
    while (g1 < n && h[ord[g1]] == h[ord[g0]]) ++g1;
    // within one hash group, compare exactly against the group's leaders
    std::vector<int32_t> group_leaders;
    for (int64_t t = g0; t < g1; ++t) {
      int32_t r = ord[t];
      int32_t found = -1;
      for (int32_t L : group_leaders)
        if (same_open_adj(rp, ci, L, r)) { found = q.sn_of[L]; break; }
      if (found < 0) {
        found = q.ns++;
        group_leaders.push_back(r);
        leaders.push_back(r);
      }
      q.sn_of[r] = found;
    }
    g0 = g1;
  }
  // members, ordered by row index inside each supernode
  q.w.assign(q.ns, 0);
  for (int64_t i = 0; i < n; ++i) q.w[q.sn_of[i]]++;
  q.mem_ptr.assign(q.ns + 1, 0);
  for (int32_t s = 0; s < q.ns; ++s) q.mem_ptr[s + 1] = q.mem_ptr[s] + q.w[s];
  q.mem.resize(n);
  {
    std::vector<int64_t> fill(q.mem_ptr.begin(), q.mem_ptr.end() - 1);
    for (int64_t i = 0; i < n; ++i) q.mem[fill[q.sn_of[i]]++] = static_cast<int32_t>(i);
  }
  // renumber supernodes by their smallest row so the quotient keeps the input's locality
  std::vector<int32_t> first_row(q.ns);
  for (int32_t s = 0; s < q.ns; ++s) first_row[s] = q.mem[q.mem_ptr[s]];
  std::vector<int32_t> sord(q.ns);
  std::iota(sord.begin(), sord.end(), 0);
  std::sort(sord.begin(), sord.end(), [&](int32_t a, int32_t b) { return first_row[a] < first_row[b]; });
  std::vector<int32_t> newid(q.ns);
  for (int32_t s = 0; s < q.ns; ++s) newid[sord[s]] = s;
  for (int64_t i = 0; i < n; ++i) q.sn_of[i] = newid[q.sn_of[i]];
  std::vector<int32_t> w2(q.ns);
  for (int32_t s = 0; s < q.ns; ++s) w2[newid[s]] = q.w[s];
  q.w.swap(w2);
  q.mem_ptr.assign(q.ns + 1, 0);
  for (int32_t s = 0; s < q.ns; ++s) q.mem_ptr[s + 1] = q.mem_ptr[s] + q.w[s];
  {
    std::vector<int64_t> fill(q.mem_ptr.begin(), q.mem_ptr.end() - 1);
    for (int64_t i = 0; i < n; ++i) q.mem[fill[q.sn_of[i]]++] = static_cast<int32_t>(i);
  }
  // quotient adjacency from each supernode's first member
  q.qrp.assign(q.ns + 1, 0);
  std::vector<int32_t> tmp;
  std::vector<std::vector<int32_t>> adjs(q.ns);
  for (int32_t s = 0; s < q.ns; ++s) {
    int32_t r = q.mem[q.mem_ptr[s]];
    tmp.clear();
    for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
      int32_t t = q.sn_of[ci[e]];
      if (t != s) tmp.push_back(t);
    }
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    adjs[s] = tmp;
    q.qrp[s + 1] = q.qrp[s] + static_cast<int64_t>(tmp.size());
  }
  q.qci.resize(q.qrp[q.ns]);
  for (int32_t s = 0; s < q.ns; ++s)
    std::copy(adjs[s].begin(), adjs[s].end(), q.qci.begin() + q.qrp[s]);
  return q;
}

// Quotient of a complex Hermitian pencil's real embedding (order n = 2 h, rows r and r + h the
// real and imaginary parts of one complex variable, with equal closed neighbourhoods by
// construction): supernode s = {s, s + h}, weight 2, adjacency that of row s folded onto the pairs.
// The ordering then sees the complex pattern, and each complex variable's two rows stay together.
Quotient build_pair_quotient(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci) {
  Quotient q;
  const int32_t h = static_cast<int32_t>(n / 2);
  q.ns = h;
  q.sn_of.resize(n);
  for (int64_t i = 0; i < n; ++i) q.sn_of[i] = static_cast<int32_t>(i % h);
  q.w.assign(h, 2);
  q.mem_ptr.resize(h + 1);
  q.mem.resize(n);
  for (int32_t s = 0; s < h; ++s) {
    q.mem_ptr[s] = 2 * static_cast<int64_t>(s);
    q.mem[2 * s] = s;
    q.mem[2 * s + 1] = s + h;
  }
  q.mem_ptr[h] = n;
  q.qrp.assign(h + 1, 0);
  std::vector<int32_t> tmp;
  for (int32_t s = 0; s < h; ++s) {
    tmp.clear();
    for (int64_t e = rp[s]; e < rp[s + 1]; ++e) {
      const int32_t t = ci[e] % h;
      if (t != s) tmp.push_back(t);
    }
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    q.qci.insert(q.qci.end(), tmp.begin(), tmp.end());
    q.qrp[s + 1] = static_cast<int64_t>(q.qci.size());
  }
  return q;
}

struct ND {
  const Quotient& q;
  const double* coords;          // per row (n x 3) or null
  int64_t leaf_weight;
  bool refined = false;          // cut search and minimum-vertex-cover separators
  std::vector<std::vector<int32_t>> nodes;   // supernodes of each ND node, post-order
  std::vector<int32_t> tag, side, level, queue;
  int32_t gen = 0;

  ND(const Quotient& qq, const double* c, int64_t leaf) : q(qq), coords(c), leaf_weight(leaf) {
    tag.assign(q.ns, 0); side.assign(q.ns, 0); level.assign(q.ns, -1); queue.resize(q.ns);
  }

  double coord(int32_t s, int axis) const {
    return coords[3 * static_cast<int64_t>(q.mem[q.mem_ptr[s]]) + axis];
  }

  // breadth-first levels inside S (marked with g); unreached vertices keep level -1
  int32_t bfs(const std::vector<int32_t>& S, int32_t root, int32_t g) {
    for (int32_t s : S) level[s] = -1;
    int64_t head = 0, tail = 0;
    level[root] = 0; queue[tail++] = root;
    int32_t depth = 0;
    while (head < tail) {
      int32_t v = queue[head++];
      depth = std::max(depth, level[v]);
      for (int64_t e = q.qrp[v]; e < q.qrp[v + 1]; ++e) {
        int32_t u = q.qci[e];
        if (tag[u] == g && level[u] < 0) { level[u] = level[v] + 1; queue[tail++] = u; }
      }
    }
    return depth;
  }

  int64_t weight(const std::vector<int32_t>& S) const {
    int64_t W = 0;
    for (int32_t s : S) W += q.w[s];
    return W;
  }

  void emit_leaf(std::vector<int32_t>& S, std::vector<int32_t>& tops) {
    tops.push_back(static_cast<int32_t>(nodes.size()));
    nodes.push_back(S);
  }

  // Minimum-weight vertex cover of the bipartite graph of cut edges between X (side 1) and Y
  // (side 2) inside the piece marked g: max flow from src through x (capacity w_x), x -> y for
  // every cut edge (unbounded), y (capacity w_y) to sink; the cover is the set of X vertices not
  // reachable from src in the residual graph plus the Y vertices that are.
  std::vector<int32_t> min_cover(const std::vector<int32_t>& X, const std::vector<int32_t>& Y, int32_t g) {
    const int32_t nx = static_cast<int32_t>(X.size()), ny = static_cast<int32_t>(Y.size());
    const int32_t src = nx + ny, snk = nx + ny + 1, N = nx + ny + 2;
    std::vector<int32_t>& pos = level;               // scratch: position of each Y vertex
    for (int32_t i = 0; i < ny; ++i) pos[Y[i]] = nx + i;
    struct Edge { int32_t to; int64_t cap; };
    std::vector<Edge> es;
    std::vector<std::vector<int32_t>> adj(N);
    auto add = [&](int32_t a, int32_t b, int64_t cap) {
      adj[a].push_back(static_cast<int32_t>(es.size())); es.push_back({b, cap});
      adj[b].push_back(static_cast<int32_t>(es.size())); es.push_back({a, 0});
    };
    const int64_t kInf = int64_t(1) << 40;
    for (int32_t i = 0; i < nx; ++i) add(src, i, q.w[X[i]]);
    for (int32_t i = 0; i < ny; ++i) add(nx + i, snk, q.w[Y[i]]);
    for (int32_t i = 0; i < nx; ++i)
      for (int64_t e = q.qrp[X[i]]; e < q.qrp[X[i] + 1]; ++e) {
        const int32_t u = q.qci[e];
        if (tag[u] == g && side[u] == 2) add(i, pos[u], kInf);
      }
    std::vector<int32_t> dist(N), it(N), bq;
    auto layer = [&]() {
      std::fill(dist.begin(), dist.end(), -1);
      bq.assign(1, src); dist[src] = 0;
      for (size_t h = 0; h < bq.size(); ++h)
        for (int32_t ei : adj[bq[h]])
          if (es[ei].cap > 0 && dist[es[ei].to] < 0) { dist[es[ei].to] = dist[bq[h]] + 1; bq.push_back(es[ei].to); }
      return dist[snk] >= 0;
    };
    // augmenting paths are src -> x -> y -> sink: the recursion is at most three deep
    std::function<int64_t(int32_t, int64_t)> push = [&](int32_t v, int64_t f) -> int64_t {
      if (v == snk) return f;
      for (int32_t& i = it[v]; i < static_cast<int32_t>(adj[v].size()); ++i) {
        Edge& e = es[adj[v][i]];
        if (e.cap > 0 && dist[e.to] == dist[v] + 1) {
          const int64_t d = push(e.to, std::min(f, e.cap));
          if (d > 0) { e.cap -= d; es[adj[v][i] ^ 1].cap += d; return d; }
        }
      }
      return 0;
    };
    while (layer()) {
      std::fill(it.begin(), it.end(), 0);
      while (push(src, kInf) > 0) {}
    }
    std::vector<char> reach(N, 0);
    bq.assign(1, src); reach[src] = 1;
    for (size_t h = 0; h < bq.size(); ++h)
      for (int32_t ei : adj[bq[h]])
        if (es[ei].cap > 0 && !reach[es[ei].to]) { reach[es[ei].to] = 1; bq.push_back(es[ei].to); }
    std::vector<int32_t> cover;
    for (int32_t i = 0; i < nx; ++i) if (!reach[i]) cover.push_back(X[i]);
    for (int32_t i = 0; i < ny; ++i) if (reach[nx + i]) cover.push_back(Y[i]);
    return cover;
  }

  // the one-sided boundaries of the cut S1 | S2 (side[] set) inside the piece marked g
  void boundaries(const std::vector<int32_t>& S1, const std::vector<int32_t>& S2, int32_t g,
                  std::vector<int32_t>& B1, std::vector<int32_t>& B2) {
    B1.clear(); B2.clear();
    for (int32_t s : S1)
      for (int64_t e = q.qrp[s]; e < q.qrp[s + 1]; ++e) {
        int32_t u = q.qci[e];
        if (tag[u] == g && side[u] == 2) { B1.push_back(s); break; }
      }
    for (int32_t s : S2)
      for (int64_t e = q.qrp[s]; e < q.qrp[s + 1]; ++e) {
        int32_t u = q.qci[e];
        if (tag[u] == g && side[u] == 1) { B2.push_back(s); break; }
      }
  }

  // Refined split of S (marked g, weight W): sort keys of every axis at least half as long as the
  // longest (or the breadth-first levels), cut positions with 42-58 % of the weight on the first
  // side, minimum-vertex-cover separators; the cut minimising w(sep) (1 + 2 |W1 - W2| / W).
  void split_refined(const std::vector<int32_t>& S, int32_t g, int64_t W, std::vector<int32_t>& S1,
                     std::vector<int32_t>& S2, std::vector<int32_t>& sep) {
    std::vector<std::vector<double>> keys;
    if (coords) {
      double ext[3], emax = 0;
      for (int ax = 0; ax < 3; ++ax) {
        double lo = 1e300, hi = -1e300;
        for (int32_t s : S) { double c = coord(s, ax); lo = std::min(lo, c); hi = std::max(hi, c); }
        ext[ax] = hi - lo;
        emax = std::max(emax, ext[ax]);
      }
      for (int ax = 0; ax < 3; ++ax) {
        if (ext[ax] < 0.5 * emax) continue;
        keys.emplace_back(S.size());
        for (size_t i = 0; i < S.size(); ++i) keys.back()[i] = coord(S[i], ax);
      }
    } else {
      int32_t root = S[0];
      int32_t d = bfs(S, root, g);
      for (int it = 0; it < 4; ++it) {
        int32_t far = root, best = -1;
        for (int32_t s : S) if (level[s] > best) { best = level[s]; far = s; }
        int32_t d2 = bfs(S, far, g);
        if (d2 <= d) { bfs(S, root, g); break; }
        d = d2; root = far;
      }
      keys.emplace_back(S.size());
      for (size_t i = 0; i < S.size(); ++i)
        keys.back()[i] = level[S[i]] < 0 ? 1e30 : static_cast<double>(level[S[i]]);
    }
    double best_score = 1e300;
    std::vector<int32_t> idx(S.size()), T1, T2, B1, B2;
    std::vector<int64_t> pre(S.size() + 1);
    for (const std::vector<double>& key : keys) {
      std::iota(idx.begin(), idx.end(), 0);
      std::sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
        return key[a] != key[b] ? key[a] < key[b] : S[a] < S[b];
      });
      pre[0] = 0;
      for (size_t i = 0; i < idx.size(); ++i) pre[i + 1] = pre[i] + q.w[S[idx[i]]];
      std::vector<size_t> cuts;
      size_t med = 0;
      while (med < idx.size() && 2 * pre[med + 1] <= W) ++med;
      cuts.push_back(std::min(std::max<size_t>(med, 1), idx.size() - 1));
      size_t a = 0, b = idx.size() - 1;
      while (a < idx.size() && 100 * pre[a] < 42 * W) ++a;
      while (b > 0 && 100 * pre[b] > 58 * W) --b;
      if (a >= 1 && b > a)
        for (size_t t = 0; t <= 12; ++t) cuts.push_back(a + (b - a) * t / 12);
      for (size_t cut : cuts) {
        T1.clear(); T2.clear();
        for (size_t i = 0; i < idx.size(); ++i) {
          const int32_t s = S[idx[i]];
          if (i < cut) { T1.push_back(s); side[s] = 1; } else { T2.push_back(s); side[s] = 2; }
        }
        boundaries(T1, T2, g, B1, B2);
        std::vector<int32_t> cand = weight(B1) <= weight(B2) ? B1 : B2;
        if (!B1.empty()) {
          std::vector<int32_t> cover = min_cover(B1, B2, g);
          if (weight(cover) < weight(cand)) cand.swap(cover);
        }
        const double w1 = static_cast<double>(pre[cut]), w2 = static_cast<double>(W - pre[cut]);
        const double score = static_cast<double>(weight(cand)) * (1.0 + 2.0 * std::fabs(w1 - w2) / W);
        if (score < best_score) { best_score = score; S1 = T1; S2 = T2; sep.swap(cand); }
      }
    }
    for (int32_t s : S1) side[s] = 1;
    for (int32_t s : S2) side[s] = 2;
  }

  // Split S; appends the ids of the resulting top nodes to tops.
  void run(std::vector<int32_t> S, std::vector<int32_t>& tops) {
    if (S.empty()) return;
    if (refined) { run_refined(std::move(S), tops); return; }
    int64_t W = weight(S);
    if (W <= leaf_weight || S.size() < 4) { emit_leaf(S, tops); return; }
    int32_t g = ++gen;
    for (int32_t s : S) tag[s] = g;
    std::vector<double> key(S.size());
    if (coords) {
      int best = 0; double ext = -1;
      for (int ax = 0; ax < 3; ++ax) {
        double lo = 1e300, hi = -1e300;
        for (int32_t s : S) { double c = coord(s, ax); lo = std::min(lo, c); hi = std::max(hi, c); }
        if (hi - lo > ext) { ext = hi - lo; best = ax; }
      }
      for (size_t i = 0; i < S.size(); ++i) key[i] = coord(S[i], best);
    } else {
      int32_t root = S[0];
      int32_t d = bfs(S, root, g);
      for (int it = 0; it < 4; ++it) {
        int32_t far = root, best = -1;
        for (int32_t s : S) if (level[s] > best) { best = level[s]; far = s; }
        int32_t d2 = bfs(S, far, g);
        if (d2 <= d) { bfs(S, root, g); break; }
        d = d2; root = far;
      }
      for (size_t i = 0; i < S.size(); ++i)
        key[i] = level[S[i]] < 0 ? 1e30 : static_cast<double>(level[S[i]]);
    }
    std::vector<int32_t> idx(S.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
      return key[a] != key[b] ? key[a] < key[b] : S[a] < S[b];
    });
    int64_t acc = 0;
    size_t cut = 0;
    while (cut < idx.size() && 2 * (acc + q.w[S[idx[cut]]]) <= W) { acc += q.w[S[idx[cut]]]; ++cut; }
    if (cut == 0) cut = 1;
    if (cut >= idx.size()) cut = idx.size() - 1;
    std::vector<int32_t> S1, S2;
    for (size_t i = 0; i < idx.size(); ++i) {
      int32_t s = S[idx[i]];
      if (i < cut) { S1.push_back(s); side[s] = 1; } else { S2.push_back(s); side[s] = 2; }
    }
    // one-sided boundaries of the cut
    std::vector<int32_t> B1, B2;
    for (int32_t s : S1)
      for (int64_t e = q.qrp[s]; e < q.qrp[s + 1]; ++e) {
        int32_t u = q.qci[e];
        if (tag[u] == g && side[u] == 2) { B1.push_back(s); break; }
      }
    for (int32_t s : S2)
      for (int64_t e = q.qrp[s]; e < q.qrp[s + 1]; ++e) {
        int32_t u = q.qci[e];
        if (tag[u] == g && side[u] == 1) { B2.push_back(s); break; }
      }
    std::vector<int32_t>& sep = weight(B1) <= weight(B2) ? B1 : B2;
    int64_t wsep = weight(sep);
    if (10 * wsep > 6 * W) { emit_leaf(S, tops); return; }
    int32_t gs = ++gen;                       // mark separator members
    for (int32_t s : sep) tag[s] = gs;
    std::vector<int32_t> R1, R2;
    for (int32_t s : S1) if (tag[s] != gs) R1.push_back(s);
    for (int32_t s : S2) if (tag[s] != gs) R2.push_back(s);
    std::vector<int32_t> kids;
    run(std::move(R1), kids);
    run(std::move(R2), kids);
    if (sep.empty()) {
      tops.insert(tops.end(), kids.begin(), kids.end());
      return;
    }
    // separator vertices ordered by the sort key so neighbouring rows stay close
    tops.push_back(static_cast<int32_t>(nodes.size()));
    nodes.push_back(sep);
  }

  void run_refined(std::vector<int32_t> S, std::vector<int32_t>& tops) {
    int64_t W = weight(S);
    if (W <= leaf_weight || S.size() < 4) { emit_leaf(S, tops); return; }
    int32_t g = ++gen;
    for (int32_t s : S) tag[s] = g;
    std::vector<int32_t> S1, S2, sep;
    split_refined(S, g, W, S1, S2, sep);
    if (10 * weight(sep) > 6 * W) { emit_leaf(S, tops); return; }
    int32_t gs = ++gen;
    for (int32_t s : sep) tag[s] = gs;
    std::vector<int32_t> R1, R2;
    for (int32_t s : S1) if (tag[s] != gs) R1.push_back(s);
    for (int32_t s : S2) if (tag[s] != gs) R2.push_back(s);
    std::vector<int32_t> kids;
    run_refined(std::move(R1), kids);
    run_refined(std::move(R2), kids);
    if (sep.empty()) {
      tops.insert(tops.end(), kids.begin(), kids.end());
      return;
    }
    tops.push_back(static_cast<int32_t>(nodes.size()));
    nodes.push_back(sep);
  }
};

}  // namespace

// Device memory plan for a given slack: L storage and D storage offsets per front, solve vectors,
// and the per-level L21 panel workspace.  Leaves never receive delayed columns (no slack).
void plan_memory(Plan& P, int32_t slack_base) {
  const int32_t nt = P.nfronts;
  P.slack.resize(nt);
  for (int32_t t = 0; t < nt; ++t) {
    const bool leaf = P.child_ptr[t + 1] == P.child_ptr[t];
    P.slack[t] = leaf ? 0 : slack_base + static_cast<int32_t>(static_cast<int64_t>(P.m_sym[t]) * slack_base / 128);
  }
  P.slack_base = slack_base;
  layout_memory(P);
}

void layout_memory(Plan& P) {
  const int32_t nt = P.nfronts;
  P.m_alloc.resize(nt); P.p_alloc.resize(nt);
  P.front_off.assign(nt + 1, 0); P.vec_off.assign(nt + 1, 0); P.piv_off.assign(nt + 1, 0);
  for (int32_t t = 0; t < nt; ++t) {
    const int32_t s = P.slack[t];
    P.m_alloc[t] = P.m_sym[t] + s;
    P.p_alloc[t] = P.p_sym[t] + s;
    int64_t sz = static_cast<int64_t>(P.m_alloc[t]) * P.p_alloc[t];
    sz = (sz + 31) / 32 * 32;
    P.front_off[t + 1] = P.front_off[t] + sz;
    P.vec_off[t + 1] = P.vec_off[t] + P.m_alloc[t];
    P.piv_off[t + 1] = P.piv_off[t] + P.p_alloc[t];
  }
  P.front_total = P.front_off[nt];
  P.vec_total = P.vec_off[nt];
  P.piv_total = P.piv_off[nt];
  P.p21_off.assign(nt, 0);
  P.max_large_rows = 0;
  if (P.level_ptr.size() != static_cast<size_t>(P.nlevels) + 1) return;
  for (int32_t l = 0; l < P.nlevels; ++l) {
    int64_t off = 0;
    for (int64_t i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
      int32_t t = P.level_fronts[i];
      P.p21_off[t] = off;
      off += static_cast<int64_t>(P.m_alloc[t]) * kPanel;
    }
    P.max_large_rows = std::max(P.max_large_rows, off / kPanel);
  }
}

kep_status build_plan(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                      const std::vector<double>& av, const std::vector<double>& bv,
                      const double* coords, bool graph_order, bool refined, bool pairs, int32_t slack_base,
                      Plan& P, std::string& err) {
  P = Plan();
  P.n = n;
  P.nnz = rp[n];
  // ||A||_inf
  for (int64_t i = 0; i < n; ++i) {
    double s = 0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += std::fabs(av[e]);
    P.norm_a_inf = std::max(P.norm_a_inf, s);
  }
  if (pairs && (n % 2 != 0)) { err = "paired ordering needs an even order"; return KEP_ERR_INVALID; }
  Quotient q = pairs ? build_pair_quotient(n, rp, ci) : build_quotient(n, rp, ci);
  ND nd(q, graph_order ? nullptr : coords, /*leaf rows*/ 64);
  nd.refined = refined;
  std::vector<int32_t> all(q.ns);
  std::iota(all.begin(), all.end(), 0);
  // each connected piece of the graph is split on its own (disconnected pieces share no separator)
  std::vector<int32_t> tops;
  nd.run(std::move(all), tops);
  const int32_t nt = static_cast<int32_t>(nd.nodes.size());
  // ordering: nodes in post-order, supernodes expanded to rows
  P.perm.resize(n);
  P.iperm.resize(n);
  P.first.resize(nt);
  P.p_sym.resize(nt);
  {
    int64_t pos = 0;
    for (int32_t t = 0; t < nt; ++t) {
      P.first[t] = static_cast<int32_t>(pos);
      for (int32_t s : nd.nodes[t])
        for (int64_t m = q.mem_ptr[s]; m < q.mem_ptr[s + 1]; ++m) P.perm[pos++] = q.mem[m];
      P.p_sym[t] = static_cast<int32_t>(pos - P.first[t]);
    }
    if (pos != n) { err = "ordering lost variables"; return KEP_ERR_INVALID; }
  }
  for (int64_t i = 0; i < n; ++i) P.iperm[P.perm[i]] = static_cast<int32_t>(i);
  std::vector<int32_t> var_node(n);
  for (int32_t t = 0; t < nt; ++t)
    for (int32_t v = P.first[t]; v < P.first[t] + P.p_sym[t]; ++v) var_node[v] = t;
  // assembly tree and contribution-block rows
  std::vector<std::vector<int32_t>> cb(nt), kids(nt);
  P.parent.assign(nt, -1);
  std::vector<int32_t> cand;
  for (int32_t t = 0; t < nt; ++t) {
    int32_t f = P.first[t], last = f + P.p_sym[t] - 1;
    cand.clear();
    for (int32_t v = f; v <= last; ++v) {
      int32_t old = P.perm[v];
      for (int64_t e = rp[old]; e < rp[old + 1]; ++e) {
        int32_t u = P.iperm[ci[e]];
        if (u > last) cand.push_back(u);
      }
    }
    for (int32_t c : kids[t])
      for (int32_t u : cb[c])
        if (u > last) cand.push_back(u);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    cb[t] = cand;
    if (!cand.empty()) {
      P.parent[t] = var_node[cand[0]];
      kids[P.parent[t]].push_back(t);
    }
  }
  P.nfronts = nt;
  P.m_sym.resize(nt);
  P.child_ptr.assign(nt + 1, 0);
  for (int32_t t = 0; t < nt; ++t) {
    P.m_sym[t] = P.p_sym[t] + static_cast<int32_t>(cb[t].size());
    P.child_ptr[t + 1] = P.child_ptr[t] + static_cast<int32_t>(kids[t].size());
    P.max_children = std::max<int32_t>(P.max_children, static_cast<int32_t>(kids[t].size()));
  }
  P.child_idx.resize(P.child_ptr[nt]);
  for (int32_t t = 0; t < nt; ++t)
    std::copy(kids[t].begin(), kids[t].end(), P.child_idx.begin() + P.child_ptr[t]);
  P.struct_ptr.assign(nt + 1, 0);
  for (int32_t t = 0; t < nt; ++t) P.struct_ptr[t + 1] = P.struct_ptr[t] + P.m_sym[t];
  P.struct_var.resize(P.struct_ptr[nt]);
  for (int32_t t = 0; t < nt; ++t) {
    int64_t o = P.struct_ptr[t];
    for (int32_t i = 0; i < P.p_sym[t]; ++i) P.struct_var[o + i] = P.first[t] + i;
    std::copy(cb[t].begin(), cb[t].end(), P.struct_var.begin() + o + P.p_sym[t]);
  }
  // child CB rows -> parent symbolic positions
  P.relmap_ptr.assign(nt + 1, 0);
  for (int32_t t = 0; t < nt; ++t) P.relmap_ptr[t + 1] = P.relmap_ptr[t] + static_cast<int64_t>(cb[t].size());
  P.relmap.resize(P.relmap_ptr[nt]);
  for (int32_t t = 0; t < nt; ++t) {
    int32_t par = P.parent[t];
    if (par < 0) continue;
    const std::vector<int32_t>& pc = cb[par];
    int32_t pf = P.first[par], pp = P.p_sym[par];
    for (size_t i = 0; i < cb[t].size(); ++i) {
      int32_t u = cb[t][i];
      int32_t pos;
      if (u >= pf && u < pf + pp) pos = u - pf;
      else {
        auto it = std::lower_bound(pc.begin(), pc.end(), u);
        if (it == pc.end() || *it != u) { err = "contribution row missing in parent"; return KEP_ERR_INVALID; }
        pos = pp + static_cast<int32_t>(it - pc.begin());
      }
      P.relmap[P.relmap_ptr[t] + static_cast<int64_t>(i)] = pos;
    }
  }
  // original lower entries (new numbering, row >= col) -> owning front, symbolic (row, col)
  {
    std::vector<int64_t> cnt(nt + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
      int32_t I = P.iperm[i];
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        int32_t J = P.iperm[ci[e]];
        if (J <= I) cnt[var_node[J] + 1]++;
      }
    }
    for (int32_t t = 0; t < nt; ++t) cnt[t + 1] += cnt[t];
    P.ent_ptr = cnt;
    int64_t ne = cnt[nt];
    P.ent_r.resize(ne); P.ent_c.resize(ne); P.ent_a.resize(ne); P.ent_b.resize(ne); P.ent_src.resize(ne);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < n; ++i) {
      int32_t I = P.iperm[i];
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        int32_t J = P.iperm[ci[e]];
        if (J > I) continue;
        int32_t t = var_node[J];
        int32_t pf = P.first[t], pp = P.p_sym[t];
        int32_t r;
        if (I < pf + pp) r = I - pf;
        else {
          const std::vector<int32_t>& pc = cb[t];
          auto it = std::lower_bound(pc.begin(), pc.end(), I);
          if (it == pc.end() || *it != I) { err = "entry outside its front"; return KEP_ERR_INVALID; }
          r = pp + static_cast<int32_t>(it - pc.begin());
        }
        int64_t o = fill[t]++;
        P.ent_r[o] = r; P.ent_c[o] = J - pf; P.ent_a[o] = av[e]; P.ent_b[o] = bv[e]; P.ent_src[o] = e;
      }
    }
  }
  // level schedule: height above the leaves
  P.height.assign(nt, 0);
  for (int32_t t = 0; t < nt; ++t)
    for (int32_t c : kids[t]) P.height[t] = std::max(P.height[t], P.height[c] + 1);
  P.nlevels = 0;
  for (int32_t t = 0; t < nt; ++t) P.nlevels = std::max(P.nlevels, P.height[t] + 1);
  plan_memory(P, slack_base);
  P.level_ptr.assign(P.nlevels + 1, 0);
  for (int32_t t = 0; t < nt; ++t) P.level_ptr[P.height[t] + 1]++;
  for (int32_t l = 0; l < P.nlevels; ++l) P.level_ptr[l + 1] += P.level_ptr[l];
  P.level_fronts.resize(nt);
  P.level_nsmall.assign(P.nlevels, 0);
  P.level_nbig_solve.assign(P.nlevels, 0);
  {
    // every level's fronts in decreasing order: the largest ones (factored alone, solved by the
    // multi-block path) lead, the rest form one batch
    std::vector<std::vector<int32_t>> lv(P.nlevels);
    for (int32_t t = 0; t < nt; ++t) lv[P.height[t]].push_back(t);
    for (int32_t l = 0; l < P.nlevels; ++l) {
      std::stable_sort(lv[l].begin(), lv[l].end(),
                       [&](int32_t a, int32_t b) { return P.m_sym[a] > P.m_sym[b]; });
      int64_t o = P.level_ptr[l];
      for (int32_t t : lv[l]) {
        P.level_fronts[o++] = t;
        if (P.m_sym[t] <= kSmallMax) P.level_nsmall[l]++;
        if (P.m_sym[t] >= kSolveBigM && P.p_sym[t] >= kSolveBigP &&
            P.level_nbig_solve[l] == static_cast<int32_t>(o - 1 - P.level_ptr[l]))
          P.level_nbig_solve[l]++;
      }
      P.max_level_width = std::max<int32_t>(P.max_level_width, P.level_ptr[l + 1] - P.level_ptr[l]);
    }
  }
  // contribution-block pool: levels run bottom-up; a block is allocated when its front is
  // factored and released once its parent's level has assembled it (first fit, merged holes)
  {
    P.cb_off.assign(nt, -1);
    std::vector<std::pair<int64_t, int64_t>> holes;   // (offset, size), sorted by offset
    int64_t top = 0;
    auto alloc = [&](int64_t sz) -> int64_t {
      for (size_t h = 0; h < holes.size(); ++h)
        if (holes[h].second >= sz) {
          int64_t o = holes[h].first;
          holes[h].first += sz; holes[h].second -= sz;
          if (holes[h].second == 0) holes.erase(holes.begin() + h);
          return o;
        }
      int64_t o = top; top += sz; return o;
    };
    auto release = [&](int64_t o, int64_t sz) {
      auto it = std::lower_bound(holes.begin(), holes.end(), std::make_pair(o, int64_t(0)));
      it = holes.insert(it, {o, sz});
      size_t h = it - holes.begin();
      if (h + 1 < holes.size() && holes[h].first + holes[h].second == holes[h + 1].first) {
        holes[h].second += holes[h + 1].second; holes.erase(holes.begin() + h + 1);
      }
      if (h > 0 && holes[h - 1].first + holes[h - 1].second == holes[h].first) {
        holes[h - 1].second += holes[h].second; holes.erase(holes.begin() + h);
      }
      if (!holes.empty() && holes.back().first + holes.back().second == top) {
        top = holes.back().first; holes.pop_back();
      }
    };
    int64_t peak = 0;
    for (int32_t l = 0; l < P.nlevels; ++l) {
      for (int64_t i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
        int32_t t = P.level_fronts[i];
        int64_t c = P.m_sym[t] - P.p_sym[t];
        if (c > 0 && P.parent[t] >= 0) P.cb_off[t] = alloc((c * c + 31) / 32 * 32);
      }
      peak = std::max(peak, top);
      for (int64_t i = P.level_ptr[l]; i < P.level_ptr[l + 1]; ++i) {
        int32_t t = P.level_fronts[i];
        for (int32_t ch : kids[t])
          if (P.cb_off[ch] >= 0) {
            int64_t c = P.m_sym[ch] - P.p_sym[ch];
            release(P.cb_off[ch], (c * c + 31) / 32 * 32);
          }
      }
    }
    P.cb_total = std::max<int64_t>(peak, 32);
  }
  plan_memory(P, slack_base);   // again: level order is now known (panel workspace offsets)
  // statistics: #nzf and flops of the symbolic factorization
  for (int32_t t = 0; t < nt; ++t) {
    int64_t m = P.m_sym[t], p = P.p_sym[t];
    P.max_front = std::max(P.max_front, m);
    P.nnz_factor += p * m - p * (p - 1) / 2;
    for (int64_t i = 0; i < p; ++i) {
      double r = static_cast<double>(m - i - 1);
      P.flops += r * r + r;
    }
  }
  return KEP_OK;
}

}  // namespace kep
