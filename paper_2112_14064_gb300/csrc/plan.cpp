// Host planning for the rIGA multifrontal solver (integer only).
//
// Univariate spaces follow the paper's Section 3.1 (open knot vectors) and
// Section 3.3 (rIGA: knots on macroelement boundaries repeated p times, which
// makes those lines C^0 and turns them into one-DOF-thick separators).
// The ordering is the canonical separator nested dissection:
//   - a direction with a C^0 DOF line strictly inside the box is cut there,
//     at the line nearest the box centre (lower one on ties); with both
//     directions cuttable the longer one (x on ties) is cut;
//   - otherwise the longer direction (x on ties) of extent E is cut by a
//     p-wide band starting at lo + (E-p)/2 while E > leaf_min and E >= p+2;
//   - boxes list their DOFs x-fastest; post-order: low child, high child,
//     separator.
// Supernode structures are the exact symbolic unions (later-ordered
// neighbours of the pivots plus the children's structures); the parent of a
// supernode owns the first entry of its structure.
#include "plan.h"

#include <algorithm>
#include <array>
#include <atomic>
#include <iterator>
#include <map>
#include <mutex>
#include <stdexcept>
#include <thread>

namespace rq {
namespace {
// f(lo, hi) over [0, n) in contiguous chunks on up to 16 host threads (one
// chunk when n is small); f must not throw.
template <class F>
void parallel_ranges(int64_t n, int64_t min_chunk, F f) {
  int64_t hw = std::max(1u, std::thread::hardware_concurrency());
  int64_t T = std::min<int64_t>(std::min<int64_t>(hw, 16), std::max<int64_t>(1, n / min_chunk));
  if (T <= 1) {
    f(int64_t(0), n);
    return;
  }
  std::vector<std::thread> th;
  for (int64_t t = 1; t < T; ++t) th.emplace_back(f, n * t / T, n * (t + 1) / T);
  f(int64_t(0), n / T);
  for (auto& x : th) x.join();
}
}  // namespace

void Space1D::build(int ne_, int p_, int block_) {
  ne = ne_; p = p_; block = block_;
  knots.assign(p + 1, 0);
  for (int k = 1; k < ne; ++k) {
    int mult = (block > 0 && k % block == 0) ? p : 1;
    for (int r = 0; r < mult; ++r) knots.push_back(k);
  }
  for (int r = 0; r <= p; ++r) knots.push_back(ne);
  n_full = (int)knots.size() - p - 1;
  n = n_full - 2;
  c0.clear();
  for (int i = 1; i <= n_full - 2; ++i) {
    bool same = true;
    for (int r = i + 1; r <= i + p; ++r) same = same && knots[r] == knots[i + 1];
    if (p >= 2 && same && knots[i + 1] > 0 && knots[i + 1] < ne) c0.push_back(i - 1);
  }
  elo.resize(n);
  ehi.resize(n);
  for (int d = 0; d < n; ++d) {
    elo[d] = knots[d + 1];
    ehi[d] = knots[d + 1 + p + 1];
  }
  // element ex = [ex, ex+1]: the span s with knots[s] <= ex < knots[s+1]
  first_fn.resize(ne);
  for (int ex = 0; ex < ne; ++ex) {
    int s = p;
    while (!(knots[s] <= ex && ex < knots[s + 1])) ++s;
    first_fn[ex] = s - p;
  }
}

bool Space1D::coupled(int a, int b) const {
  int lo = std::max(elo[a], elo[b]);
  int hi = std::min(ehi[a], ehi[b]);
  return lo < hi;
}

void Plan::build_pattern(int ne_, int p_, int block_, int nq_, int leaf_min_) {
  ne = ne_; p = p_; block = block_; nq = nq_ > 0 ? nq_ : p_ + 1;
  leaf_min = leaf_min_ > 0 ? leaf_min_ : 8;
  if (p < 2 || p > 8) throw std::invalid_argument("p must be in [2, 8]");
  if (ne < 2) throw std::invalid_argument("ne must be >= 2");
  if (block < 0 || (block > 0 && ne % block)) throw std::invalid_argument("block must divide ne");
  if (nq < 1 || nq > 10) throw std::invalid_argument("n_quad must be in [1, 10]");
  sp.build(ne, p, block);
  n1 = sp.n;
  N = (int64_t)n1 * n1;
  // univariate coupling lists (ascending)
  std::vector<std::vector<int>> cpl(n1);
  for (int a = 0; a < n1; ++a)
    for (int b = std::max(0, a - 2 * p - 2); b < std::min(n1, a + 2 * p + 3); ++b)
      if (sp.coupled(a, b)) cpl[a].push_back(b);
  rowptr.assign(N + 1, 0);
  int64_t total = 0;
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n1; ++i) {
      total += (int64_t)cpl[i].size() * cpl[j].size();
      rowptr[i + (int64_t)n1 * j + 1] = (int32_t)total;
      if (total > INT32_MAX) throw std::invalid_argument("pattern too large for int32");
    }
  nnz = total;
  col.resize(nnz);
  parallel_ranges(n1, 64, [&](int64_t j0, int64_t j1) {
    for (int64_t j = j0; j < j1; ++j)
      for (int i = 0; i < n1; ++i) {
        int64_t o = rowptr[i + (int64_t)n1 * j];
        for (int bj : cpl[j])
          for (int bi : cpl[i]) col[o++] = (int32_t)(bi + n1 * bj);
      }
  });
}

namespace {
struct Box { int x0, x1, y0, y1; };

void nd_rec(int x0, int x1, int y0, int y1, const std::vector<int>& c0, int p, int leaf_min,
            std::vector<Box>& out) {
  if (x1 <= x0 || y1 <= y0) return;
  auto pick = [&](int lo, int hi, int& c) {
    bool found = false;
    long best = 0;
    for (int v : c0) {
      if (lo < v && v < hi - 1) {
        long d = std::labs(2L * v - (lo + hi - 1));
        if (!found || d < best) { best = d; c = v; found = true; }
      }
    }
    return found;
  };
  int cx = -1, cy = -1;
  bool hx = pick(x0, x1, cx), hy = pick(y0, y1, cy);
  int ex = x1 - x0, ey = y1 - y0;
  bool cut_x;
  int s0, s1;
  if (hx || hy) {
    cut_x = (hx && hy) ? (ex >= ey) : hx;
    s0 = cut_x ? cx : cy;
    s1 = s0 + 1;
  } else {
    cut_x = ex >= ey;
    int lo = cut_x ? x0 : y0, E = cut_x ? ex : ey;
    if (!(E > leaf_min && E >= p + 2)) { out.push_back({x0, x1, y0, y1}); return; }
    s0 = lo + (E - p) / 2;
    s1 = s0 + p;
  }
  if (cut_x) {
    nd_rec(x0, s0, y0, y1, c0, p, leaf_min, out);
    nd_rec(s1, x1, y0, y1, c0, p, leaf_min, out);
    out.push_back({s0, s1, y0, y1});
  } else {
    nd_rec(x0, x1, y0, s0, c0, p, leaf_min, out);
    nd_rec(x0, x1, s1, y1, c0, p, leaf_min, out);
    out.push_back({x0, x1, s0, s1});
  }
}
}  // namespace

void Plan::build_symbolic() {
  std::vector<Box> boxes;
  std::vector<int> c0 = sp.c0;
  std::sort(c0.begin(), c0.end());
  nd_rec(0, n1, 0, n1, c0, p, leaf_min, boxes);
  nsuper = (int)boxes.size();
  perm.clear();
  perm.reserve(N);
  sptr.assign(1, 0);
  for (const Box& b : boxes) {
    for (int y = b.y0; y < b.y1; ++y)
      for (int x = b.x0; x < b.x1; ++x) perm.push_back(x + n1 * y);
    sptr.push_back((int32_t)perm.size());
  }
  if ((int64_t)perm.size() != N) throw std::logic_error("boxes do not partition the DOFs");
  iperm.assign(N, -1);
  for (int64_t j = 0; j < N; ++j) iperm[perm[j]] = (int32_t)j;
  owner.resize(N);
  for (int s = 0; s < nsuper; ++s)
    for (int j = sptr[s]; j < sptr[s + 1]; ++j) owner[j] = s;

  // exact supernodal structures: the later-ordered neighbours of each
  // supernode's own rows (independent per supernode, host threads), then in
  // post-order the union with the children's structures (sorted merges)
  parent.assign(nsuper, -1);
  level.assign(nsuper, 0);
  std::vector<std::vector<int32_t>> kids(nsuper);
  std::vector<std::vector<int32_t>> st(nsuper);
  parallel_ranges(nsuper, 64, [&](int64_t s0, int64_t s1) {
    // stamp[i] = the last supernode that listed i: each neighbour is kept
    // once, so only the distinct entries are sorted
    std::vector<int32_t> stamp(N, -1);
    for (int64_t s = s0; s < s1; ++s) {
      int a = sptr[s], e = sptr[s + 1];
      std::vector<int32_t>& S = st[s];
      for (int j = a; j < e; ++j) {
        int32_t o = perm[j];
        for (int32_t q = rowptr[o]; q < rowptr[o + 1]; ++q) {
          int32_t i = iperm[col[q]];
          if (i >= e && stamp[i] != (int32_t)s) {
            stamp[i] = (int32_t)s;
            S.push_back(i);
          }
        }
      }
      std::sort(S.begin(), S.end());
    }
  });
  std::vector<int32_t> merged;
  for (int s = 0; s < nsuper; ++s) {
    int e = sptr[s + 1];
    int lv = 0;
    for (int32_t c : kids[s]) {
      const std::vector<int32_t>& C = st[c];
      auto from = std::lower_bound(C.begin(), C.end(), e);
      merged.clear();
      std::set_union(st[s].begin(), st[s].end(), from, C.end(), std::back_inserter(merged));
      st[s].swap(merged);
      lv = std::max(lv, level[c] + 1);
    }
    level[s] = lv;
    if (!st[s].empty()) {
      parent[s] = owner[st[s][0]];
      kids[parent[s]].push_back(s);
    }
  }
  upd_ptr.assign(nsuper + 1, 0);
  for (int s = 0; s < nsuper; ++s) upd_ptr[s + 1] = upd_ptr[s] + (int32_t)st[s].size();
  upd_idx.resize(upd_ptr[nsuper]);
  for (int s = 0; s < nsuper; ++s) std::copy(st[s].begin(), st[s].end(), upd_idx.begin() + upd_ptr[s]);
  child_ptr.assign(nsuper + 1, 0);
  for (int s = 0; s < nsuper; ++s) child_ptr[s + 1] = child_ptr[s] + (int32_t)kids[s].size();
  child_idx.resize(child_ptr[nsuper]);
  for (int s = 0; s < nsuper; ++s) std::copy(kids[s].begin(), kids[s].end(), child_idx.begin() + child_ptr[s]);
  nlevels = 0;
  for (int s = 0; s < nsuper; ++s) nlevels = std::max(nlevels, level[s] + 1);

  // factor storage, counts
  loff.assign(nsuper + 1, 0);
  uoff.assign(nsuper + 1, 0);
  nnz_L = 0; flops = 0; max_front = 0;
  for (int s = 0; s < nsuper; ++s) {
    int64_t k = sptr[s + 1] - sptr[s], u = upd_ptr[s + 1] - upd_ptr[s];
    loff[s + 1] = loff[s] + (k + u) * k;
    uoff[s + 1] = uoff[s] + u * u;
    nnz_L += k * (k + 1) / 2 + k * u;
    for (int64_t t = 0; t < k; ++t) {
      int64_t c = (k - 1 - t) + u;
      flops += c * c + 2 * c;
    }
    max_front = std::max(max_front, k + u);
  }
  l_total = loff[nsuper];
  u_total = uoff[nsuper];

  // extend-add maps: struct(s) -> rows of the parent's front
  // (independent per supernode: host threads)
  relmap.assign(upd_idx.size(), -1);
  std::atomic<int> outside{0};
  parallel_ranges(nsuper, 64, [&](int64_t s0, int64_t s1) {
    for (int64_t s = s0; s < s1; ++s) {
      int pa = parent[s];
      if (pa < 0) continue;
      int a = sptr[pa], e = sptr[pa + 1], k = e - a;
      const int32_t* ps = upd_idx.data() + upd_ptr[pa];
      int pu = upd_ptr[pa + 1] - upd_ptr[pa];
      int w = 0;
      for (int32_t q = upd_ptr[s]; q < upd_ptr[s + 1]; ++q) {
        int32_t i = upd_idx[q];
        if (i < e) { relmap[q] = i - a; continue; }
        while (w < pu && ps[w] < i) ++w;
        if (w >= pu || ps[w] != i) {
          outside = 1;
          break;
        }
        relmap[q] = k + w;
      }
    }
  });
  if (outside) throw std::logic_error("child structure not in parent front");

  // row pointers of the ND-ordered CSR (row j is the original row perm[j])
  rowptr_n.assign(N + 1, 0);
  for (int64_t j = 0; j < N; ++j) {
    int32_t o = perm[j];
    rowptr_n[j + 1] = rowptr_n[j] + (rowptr[o + 1] - rowptr[o]);
  }

  // level sets
  lvl_ptr.assign(nlevels + 1, 0);
  for (int s = 0; s < nsuper; ++s) lvl_ptr[level[s] + 1]++;
  for (int l = 0; l < nlevels; ++l) lvl_ptr[l + 1] += lvl_ptr[l];
  lvl_nodes.resize(nsuper);
  std::vector<int32_t> fill(lvl_ptr.begin(), lvl_ptr.end() - 1);
  for (int s = 0; s < nsuper; ++s) lvl_nodes[fill[level[s]]++] = s;
}

// Exact column structures of L in the ND order (no supernodal amalgamation):
// struct(j) = {i > j : Q_ij != 0} united with the structures of j's
// elimination-tree children, less j; the parent of j is the first entry of
// struct(j).  Each structure is merged once into its parent and released.
// The counts depend only on the mesh, so they are computed once per mesh in
// the process and cached: later handles of the same mesh (repeated solves)
// pay nothing.
void Plan::exact_counts() {
  if (nnz_L_exact >= 0) return;
  static std::mutex mu;
  static std::map<std::array<int, 5>, std::pair<int64_t, int64_t>> cache;
  const std::array<int, 5> key{ne, p, block, nq, leaf_min};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      nnz_L_exact = it->second.first;
      flops_exact = it->second.second;
      return;
    }
  }
  std::vector<std::vector<int32_t>> st(N);
  std::vector<int32_t> head(N, -1), next(N, -1);
  std::vector<int32_t> buf, tmp;
  int64_t nnz = 0, fl = 0;
  for (int64_t j = 0; j < N; ++j) {
    const int32_t o = perm[j];
    buf.clear();
    for (int32_t q = rowptr[o]; q < rowptr[o + 1]; ++q) {
      const int32_t i = iperm[col[q]];
      if (i > j) buf.push_back(i);
    }
    std::sort(buf.begin(), buf.end());
    for (int32_t c = head[j]; c >= 0; c = next[c]) {
      tmp.clear();
      std::set_union(buf.begin(), buf.end(), st[c].begin(), st[c].end(), std::back_inserter(tmp));
      buf.swap(tmp);
      std::vector<int32_t>().swap(st[c]);
    }
    auto it = std::lower_bound(buf.begin(), buf.end(), (int32_t)j);
    if (it != buf.end() && *it == (int32_t)j) buf.erase(it);
    const int64_t c = (int64_t)buf.size();
    nnz += 1 + c;
    fl += c * c + 2 * c;
    if (!buf.empty()) {
      const int32_t p = buf[0];
      next[j] = head[p];
      head[p] = (int32_t)j;
      st[j] = buf;
    }
  }
  nnz_L_exact = nnz;
  flops_exact = fl;
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = {nnz, fl};
}

}  // namespace rq
