// Nested-dissection symbolic analysis of one domain matrix (host only).
//
// Section II factors every domain with a sparse direct solver; this library
// factors domains of up to a few thousand unknowns as single dense fronts.
// For larger domains the analysis below splits the domain into a tree of
// fronts: the interface unknowns (the rows that B couples to the duals) are
// eliminated last, in the domain's root front, and the interior unknowns are
// ordered by nested dissection (George 1973), each separator a middle level
// of a breadth-first level structure rooted at a pseudo-peripheral vertex
// (George and Liu 1979), recursively down to leaves of at most leaf_max
// unknowns.  A front's update rows are the later-eliminated unknowns
// reachable from its own unknowns through itself and its subtree.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "../../include/dd.h"
#include "../../include/dd_diag.h"

namespace {

struct DomainNd {
  const std::vector<std::vector<int32_t>>& adj;
  int32_t leaf_max;
  std::vector<int32_t> stamp;   // vertex -> id of the set it currently belongs to
  int32_t next_stamp = 0;
  std::vector<int32_t> level;   // scratch: BFS level of each vertex
  std::vector<int32_t> parent;  // per tree node
  std::vector<std::vector<int32_t>> elim;

  DomainNd(const std::vector<std::vector<int32_t>>& a, int32_t lm)
      : adj(a), leaf_max(lm), stamp(a.size(), -1), level(a.size(), -1) {}

  int32_t new_node(std::vector<int32_t> verts) {
    std::sort(verts.begin(), verts.end());
    elim.push_back(std::move(verts));
    parent.push_back(-1);
    return (int32_t)elim.size() - 1;
  }

  int32_t mark(const std::vector<int32_t>& s) {
    const int32_t t = next_stamp++;
    for (int32_t v : s) stamp[v] = t;
    return t;
  }

  int32_t degree_in(int32_t v, int32_t t) const {
    int32_t d = 0;
    for (int32_t w : adj[v])
      if (stamp[w] == t) ++d;
    return d;
  }

  // breadth-first levels of the vertices stamped t reachable from r
  std::vector<std::vector<int32_t>> levels_from(int32_t r, int32_t t) {
    std::vector<std::vector<int32_t>> L;
    std::vector<int32_t> seen;
    L.push_back({r});
    level[r] = 0;
    seen.push_back(r);
    while (true) {
      std::vector<int32_t> nxt;
      for (int32_t v : L.back())
        for (int32_t w : adj[v])
          if (stamp[w] == t && level[w] < 0) {
            level[w] = (int32_t)L.size();
            nxt.push_back(w);
            seen.push_back(w);
          }
      if (nxt.empty()) break;
      std::sort(nxt.begin(), nxt.end());
      L.push_back(std::move(nxt));
    }
    for (int32_t v : seen) level[v] = -1;
    return L;
  }

  // connected components of the vertex set s (stamped t), each sorted
  std::vector<std::vector<int32_t>> components(const std::vector<int32_t>& s, int32_t t) {
    std::vector<std::vector<int32_t>> comps;
    const int32_t done = next_stamp++;
    for (int32_t v0 : s) {
      if (stamp[v0] != t) continue;
      std::vector<int32_t> c{v0}, stack{v0};
      stamp[v0] = done;
      while (!stack.empty()) {
        const int32_t v = stack.back();
        stack.pop_back();
        for (int32_t w : adj[v])
          if (stamp[w] == t) {
            stamp[w] = done;
            c.push_back(w);
            stack.push_back(w);
          }
      }
      std::sort(c.begin(), c.end());
      comps.push_back(std::move(c));
    }
    return comps;
  }

  // tree of the vertex set s; returns its root node
  int32_t dissect(std::vector<int32_t> s) {
    std::sort(s.begin(), s.end());
    if ((int32_t)s.size() <= leaf_max) return new_node(s);
    int32_t t = mark(s);
    std::vector<std::vector<int32_t>> comps = components(s, t);
    if (comps.size() > 1) {
      // no separator needed: two groups of whole components, largest first
      std::stable_sort(comps.begin(), comps.end(),
                       [](const std::vector<int32_t>& a, const std::vector<int32_t>& b) { return a.size() > b.size(); });
      std::vector<int32_t> ga, gb;
      for (const auto& c : comps) {
        std::vector<int32_t>& g = ga.size() <= gb.size() ? ga : gb;
        g.insert(g.end(), c.begin(), c.end());
      }
      const int32_t ca = dissect(ga), cb = dissect(gb);
      const int32_t node = new_node({});
      parent[ca] = parent[cb] = node;
      return node;
    }
    t = mark(s);
    // pseudo-peripheral vertex: start at a vertex of least degree, move to a
    // least-degree vertex of the last level while the eccentricity grows
    int32_t r = s[0], best = degree_in(s[0], t);
    for (int32_t v : s) {
      const int32_t d = degree_in(v, t);
      if (d < best) best = d, r = v;
    }
    std::vector<std::vector<int32_t>> L = levels_from(r, t);
    for (int it = 0; it < 8; ++it) {
      int32_t x = L.back()[0], dx = degree_in(x, t);
      for (int32_t v : L.back()) {
        const int32_t d = degree_in(v, t);
        if (d < dx) dx = d, x = v;
      }
      std::vector<std::vector<int32_t>> L2 = levels_from(x, t);
      if (L2.size() <= L.size()) break;
      L = std::move(L2);
    }
    if (L.size() < 3) return new_node(s);
    // separator: the level where half of the vertices have been passed
    size_t m = 1, cum = 0;
    for (size_t l = 0; l < L.size(); ++l) {
      cum += L[l].size();
      if (2 * cum >= s.size()) {
        m = l;
        break;
      }
    }
    m = std::min(std::max(m, (size_t)1), L.size() - 2);
    std::vector<int32_t> a, b;
    for (size_t l = 0; l < m; ++l) a.insert(a.end(), L[l].begin(), L[l].end());
    for (size_t l = m + 1; l < L.size(); ++l) b.insert(b.end(), L[l].begin(), L[l].end());
    const std::vector<int32_t> sep = L[m];
    const int32_t ca = dissect(a), cb = dissect(b);
    const int32_t node = new_node(sep);
    parent[ca] = parent[cb] = node;
    return node;
  }
};

// The analysis of one domain: its dissection tree and every front's rows.
struct DomainFronts {
  int32_t nf = 0;
  std::vector<int32_t> parent, fof, pos;          // per front; per row: front, elimination position
  std::vector<std::vector<int32_t>> elim, upd;    // per front: own rows (by position), update rows (by index)
  int64_t stored = 0;
};

int analyse_domain(int32_t n, const int32_t* rowptr, const int32_t* colind, const int8_t* is_last, int32_t leaf_max,
                   DomainFronts& out) {
  if (n < 0 || leaf_max < 1) return DD_ERR_INVALID_ARG;
  if (n > 0 && (!rowptr || !colind)) return DD_ERR_INVALID_ARG;
  if (n > 0 && rowptr[0] != 0) return DD_ERR_INVALID_ARG;
  std::vector<std::vector<int32_t>> adj(n);
  for (int32_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return DD_ERR_INVALID_ARG;
    for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
      const int32_t j = colind[q];
      if (j < 0 || j >= n) return DD_ERR_INVALID_ARG;
      if (j != i) adj[i].push_back(j);
    }
    std::sort(adj[i].begin(), adj[i].end());
    adj[i].erase(std::unique(adj[i].begin(), adj[i].end()), adj[i].end());
  }
  for (int32_t i = 0; i < n; ++i)
    for (int32_t j : adj[i])
      if (!std::binary_search(adj[j].begin(), adj[j].end(), i)) return DD_ERR_NOT_SYMMETRIC;

  DomainNd nd(adj, leaf_max);
  std::vector<int32_t> interior, iface;
  for (int32_t v = 0; v < n; ++v) (is_last && is_last[v] ? iface : interior).push_back(v);
  // the interface block is eliminated last, in the root; the interior below it
  if (!interior.empty()) {
    const int32_t c = nd.dissect(interior);
    const int32_t root = nd.new_node(iface);   // grows nd.parent: index it afterwards
    nd.parent[c] = root;
  } else {
    nd.new_node(iface);
  }
  const int32_t nf = (int32_t)nd.elim.size();
  // elimination order (nodes in creation order: children before parents) and
  // the depth of every node, for the ancestor test
  std::vector<int32_t> fof(n, -1), pos(n, -1), depth(nf, 0);
  int32_t k = 0;
  for (int32_t x = 0; x < nf; ++x)
    for (int32_t v : nd.elim[x]) {
      pos[v] = k++;
      fof[v] = x;
    }
  for (int32_t x = nf - 1; x >= 0; --x) depth[x] = nd.parent[x] < 0 ? 0 : depth[nd.parent[x]] + 1;
  auto ancestor = [&](int32_t a, int32_t x) {   // is a an ancestor of x (or x itself)
    while (depth[x] > depth[a]) x = nd.parent[x];
    return x == a;
  };
  // update rows: unknowns of proper ancestors adjacent to this front's own
  // unknowns, or passed up by its children
  std::vector<std::vector<int32_t>> upd(nf), children(nf);
  for (int32_t x = 0; x < nf; ++x)
    if (nd.parent[x] >= 0) children[nd.parent[x]].push_back(x);
  int64_t st = 0;
  for (int32_t x = 0; x < nf; ++x) {
    std::vector<int32_t> u;
    for (int32_t v : nd.elim[x])
      for (int32_t w : adj[v])
        if (fof[w] != x && ancestor(fof[w], x)) u.push_back(w);
    for (int32_t c : children[x])
      for (int32_t w : upd[c])
        if (fof[w] != x) u.push_back(w);
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    upd[x] = std::move(u);
    const int64_t e = (int64_t)nd.elim[x].size(), a = (int64_t)upd[x].size();
    st += e * (e - 1) / 2 + e * a;
  }
  out.nf = nf;
  out.parent = nd.parent;
  out.fof = std::move(fof);
  out.pos = std::move(pos);
  out.elim = std::move(nd.elim);
  out.upd = std::move(upd);
  out.stored = st;
  return DD_OK;
}

}  // namespace

extern "C" int dd_domain_symbolic(int32_t n, const int32_t* rowptr, const int32_t* colind, const int8_t* is_last,
                                  int32_t leaf_max, int32_t max_fronts, int32_t* n_front, int32_t* parent,
                                  int32_t* ne, int32_t* nu, int32_t* order, int32_t* front_of, int64_t* stored,
                                  int64_t upd_cap, int64_t* upd_ptr, int32_t* upd_idx) {
  if (!n_front || !parent || !ne || !nu || !stored || (upd_idx && !upd_ptr)) return DD_ERR_INVALID_ARG;
  if (n > 0 && (!order || !front_of)) return DD_ERR_INVALID_ARG;
  DomainFronts d;
  const int status = analyse_domain(n, rowptr, colind, is_last, leaf_max, d);
  if (status != DD_OK) return status;
  *n_front = d.nf;
  if (max_fronts < d.nf) return DD_ERR_INVALID_ARG;
  int64_t total = 0;
  for (int32_t x = 0; x < d.nf; ++x) {
    parent[x] = d.parent[x];
    ne[x] = (int32_t)d.elim[x].size();
    nu[x] = (int32_t)d.upd[x].size();
    total += nu[x];
  }
  for (int32_t v = 0; v < n; ++v) {
    order[d.pos[v]] = v;
    front_of[v] = d.fof[v];
  }
  *stored = d.stored;
  if (upd_ptr) {
    int64_t q = 0;
    for (int32_t x = 0; x < d.nf; ++x) {
      upd_ptr[x] = q;
      q += (int64_t)d.upd[x].size();
    }
    upd_ptr[d.nf] = q;
    if (upd_idx) {
      if (upd_cap < total) return DD_ERR_INVALID_ARG;
      q = 0;
      for (int32_t x = 0; x < d.nf; ++x)
        for (int32_t w : d.upd[x]) upd_idx[q++] = w;
    }
  }
  return DD_OK;
}

extern "C" int dd_domain_assembly(int32_t n, const int32_t* rowptr, const int32_t* colind, const int8_t* is_last,
                                  int32_t leaf_max, int32_t max_fronts, int32_t* n_front, int32_t* parent,
                                  int32_t* ne, int64_t rows_cap, int64_t* rows_ptr, int32_t* rows,
                                  int32_t* ea_map, int32_t* a_front, int32_t* a_row, int32_t* a_col) {
  if (!n_front || !parent || !ne || !rows_ptr) return DD_ERR_INVALID_ARG;
  DomainFronts d;
  const int status = analyse_domain(n, rowptr, colind, is_last, leaf_max, d);
  if (status != DD_OK) return status;
  *n_front = d.nf;
  if (max_fronts < d.nf) return DD_ERR_INVALID_ARG;
  // a front's rows: its own rows, then its update rows, both in elimination
  // order (so every child's update rows land in increasing parent rows)
  for (auto& u : d.upd) std::sort(u.begin(), u.end(), [&](int32_t a, int32_t b) { return d.pos[a] < d.pos[b]; });
  int64_t q = 0;
  for (int32_t x = 0; x < d.nf; ++x) {
    parent[x] = d.parent[x];
    ne[x] = (int32_t)d.elim[x].size();
    rows_ptr[x] = q;
    q += (int64_t)(d.elim[x].size() + d.upd[x].size());
  }
  rows_ptr[d.nf] = q;
  if (!rows) return DD_OK;   // sizes only
  if (rows_cap < q || !ea_map || (n > 0 && (!a_front || !a_row || !a_col))) return DD_ERR_INVALID_ARG;
  std::vector<int32_t> loc(n, -1);   // row -> index in the front being filled
  for (int32_t x = 0; x < d.nf; ++x) {
    int32_t* rx = rows + rows_ptr[x];
    int32_t r = 0;
    for (int32_t v : d.elim[x]) rx[r++] = v;
    for (int32_t v : d.upd[x]) rx[r++] = v;
  }
  // extend-add: each update row of a front, its row in the parent front
  for (int32_t x = 0; x < d.nf; ++x) {
    const int32_t p = d.parent[x];
    const int64_t b = rows_ptr[x];
    const int32_t e = (int32_t)d.elim[x].size(), m = (int32_t)(rows_ptr[x + 1] - b);
    for (int32_t r = 0; r < m; ++r) ea_map[b + r] = -1;
    if (p < 0) continue;
    const int64_t bp = rows_ptr[p];
    for (int32_t r = 0; r < (int32_t)(rows_ptr[p + 1] - bp); ++r) loc[rows[bp + r]] = r;
    for (int32_t r = e; r < m; ++r) ea_map[b + r] = loc[rows[b + r]];
    for (int32_t r = 0; r < (int32_t)(rows_ptr[p + 1] - bp); ++r) loc[rows[bp + r]] = -1;
  }
  // entries of A (symmetric): CSR row r supplies column r of its front; the
  // entry (r, c) with c eliminated no earlier than r goes to r's front at
  // (row of c, row of r), the other entries of the row are left to their
  // mirrors (a_front = -1)
  for (int32_t x = 0; x < d.nf; ++x) {
    const int64_t b = rows_ptr[x];
    for (int64_t r = b; r < rows_ptr[x + 1]; ++r) loc[rows[r]] = (int32_t)(r - b);
    int bad = 0;
    for (int32_t r : d.elim[x])
      for (int32_t qq = rowptr[r]; qq < rowptr[r + 1]; ++qq) {
        const int32_t c = colind[qq];
        if (d.pos[c] < d.pos[r]) {
          a_front[qq] = a_row[qq] = a_col[qq] = -1;
        } else {
          a_front[qq] = x;
          a_row[qq] = loc[c];
          a_col[qq] = loc[r];
          bad |= loc[c] < 0;
        }
      }
    for (int64_t r = b; r < rows_ptr[x + 1]; ++r) loc[rows[r]] = -1;
    if (bad) return DD_ERR_INVALID_ARG;   // not reached for a valid analysis
  }
  return DD_OK;
}
