// Shard plan of the front tree over several ranks (host only): dd_shard_plan,
// declared in include/dd_diag.h.
//
// Section II eliminates the primal unknowns by independent domain
// factorizations and factors the auxiliary matrix over a tree of dense
// blocks; both parallelise along subtrees of that tree.  The plan cuts the
// front tree into n_ranks subtrees of about equal algorithmic work, greedily
// splitting the subtree of largest work into its children; each rank owns one
// subtree (its domains and the fronts below the cut) and rank 0 also owns the
// fronts above the cuts.  The only exchange the plan implies is the block
// each cut subtree passes up (its root's Schur complement on the root's
// update duals) to the owner of the parent front, and in a solve the
// right-hand side of those duals up and their solved values down.
#include <algorithm>
#include <vector>

#include "../../include/dd.h"
#include "../../include/dd_diag.h"

extern "C" int dd_shard_plan(int32_t n_sub, const dd_subdomain* subs, int32_t n_dual, const dd_options* opt,
                             int32_t n_ranks, int32_t max_fronts, int32_t* n_front, int32_t* front_rank,
                             int32_t* rank_root) {
  if (n_ranks < 1 || max_fronts < 1 || !n_front || !front_rank || !rank_root) return DD_ERR_INVALID_ARG;
  std::vector<int32_t> parent(max_fronts), ne(max_fronts), nu(max_fronts), df(std::max(n_dual, 1));
  int st = dd_symbolic(n_sub, subs, n_dual, opt, max_fronts, n_front, parent.data(), ne.data(), nu.data(), df.data(),
                       0, nullptr, nullptr);
  if (st != DD_OK) return st;
  const int nf = *n_front;
  std::vector<std::vector<int32_t>> children(nf);
  std::vector<int32_t> roots;
  for (int x = 0; x < nf; ++x) {
    if (parent[x] >= 0) children[parent[x]].push_back(x);
    else roots.push_back(x);
  }
  if (roots.size() != 1) return DD_ERR_INVALID_ARG;
  // algorithmic work of every front, 3x its real flops at 8 real flops per
  // complex multiply-add (an integer, so that equal subtrees tie exactly and
  // the first one in the cut list wins), and of every subtree, children
  // before parents
  std::vector<long long> work(nf, 0);
  std::vector<int32_t> order, stack{roots[0]};
  while (!stack.empty()) {
    const int x = stack.back();
    stack.pop_back();
    order.push_back(x);
    for (int c : children[x]) stack.push_back(c);
  }
  for (auto it = order.rbegin(); it != order.rend(); ++it) {
    const int x = *it;
    const long long e = ne[x], u = nu[x];
    work[x] += 4 * e * e * e + 12 * e * e * u + 12 * e * u * u;
    if (parent[x] >= 0) work[parent[x]] += work[x];
  }
  // greedy cut: split the subtree of largest work into its children until
  // there are n_ranks subtrees
  std::vector<int32_t> cut{roots[0]};
  while ((int)cut.size() < n_ranks) {
    int best = -1;
    for (int q = 0; q < (int)cut.size(); ++q)
      if (!children[cut[q]].empty() && (best < 0 || work[cut[q]] > work[cut[best]])) best = q;
    if (best < 0) return DD_ERR_INVALID_ARG;   // fewer subtrees than ranks
    const int x = cut[best];
    cut.erase(cut.begin() + best);
    for (int c : children[x]) cut.push_back(c);
  }
  if ((int)cut.size() != n_ranks) return DD_ERR_INVALID_ARG;   // a split added more subtrees than ranks left
  std::sort(cut.begin(), cut.end());
  // every front: the rank of the cut subtree holding it, rank 0 above the cuts
  std::fill(front_rank, front_rank + nf, 0);
  for (int r = 0; r < n_ranks; ++r) {
    rank_root[r] = cut[r];
    std::vector<int32_t> s{cut[r]};
    while (!s.empty()) {
      const int x = s.back();
      s.pop_back();
      front_rank[x] = r;
      for (int c : children[x]) s.push_back(c);
    }
  }
  return DD_OK;
}
