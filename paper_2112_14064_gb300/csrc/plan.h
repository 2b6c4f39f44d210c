// Host-side integer planning: univariate spaces, CSR pattern, separator
// nested dissection, supernodal symbolic factorisation and front maps.
// No CUDA dependency: everything here is plain C++ on int32/int64.
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

namespace rq {

// Allocator that leaves elements default-initialised (uninitialised for
// integers) on resize, so that arrays of nnz entries are first touched by the
// host threads that fill them instead of by one sequential memset.
template <class T>
struct NoInit : std::allocator<T> {
  template <class U>
  struct rebind { using other = NoInit<U>; };
  NoInit() = default;
  template <class U>
  NoInit(const NoInit<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept { ::new ((void*)p) U; }
  template <class U, class... A>
  void construct(U* p, A&&... a) { ::new ((void*)p) U(std::forward<A>(a)...); }
};
using ivec = std::vector<int32_t, NoInit<int32_t>>;

struct Space1D {
  int ne = 0, p = 0, block = 0;
  std::vector<int> knots;   // knot numerators over ne (exact)
  int n_full = 0;           // B-splines on the open knot vector
  int n = 0;                // DOFs after the two Dirichlet functions are dropped
  std::vector<int> c0;      // DOF indices of the C^0 separator functions
  std::vector<int> elo, ehi;  // DOF d lives on elements [elo[d], ehi[d])
  std::vector<int> first_fn;  // element ex carries full functions first_fn[ex]..+p
  void build(int ne_, int p_, int block_);
  bool coupled(int a, int b) const;  // DOFs a, b share an open interval
};

struct Plan {
  // mesh
  int ne = 0, p = 0, block = 0, nq = 0, leaf_min = 8;
  Space1D sp;
  int n1 = 0;
  int64_t N = 0, nnz = 0;
  // original-order CSR pattern (columns ascending)
  std::vector<int32_t> rowptr;
  ivec col;
  // ordering and supernodes
  std::vector<int32_t> perm, iperm, sptr, owner;
  int nsuper = 0;
  std::vector<int32_t> parent, level, upd_ptr, upd_idx;
  int nlevels = 0;
  std::vector<int32_t> child_ptr, child_idx;  // children of each supernode
  // row pointers of the ND-ordered CSR (its columns, original slots and front
  // rows are formed on the device when the problem is analysed)
  std::vector<int32_t> rowptr_n;
  // front storage layout
  std::vector<int64_t> loff;       // factor panel of s: (k+u) x k, column-major
  std::vector<int64_t> uoff;       // update block of s: u x u, column-major
  std::vector<int32_t> relmap;     // for each s: struct(s) -> position in parent's front
  int64_t l_total = 0, u_total = 0;
  std::vector<int32_t> lvl_ptr, lvl_nodes;  // supernodes of each level, ascending
  int64_t nnz_L = 0, flops = 0, max_front = 0;
  // exact (scalar) counts: structurally non-zero entries of L and
  // sum_j (c_j^2 + 2 c_j) with the exact column counts c_j (exact_counts())
  int64_t nnz_L_exact = -1, flops_exact = -1;

  // build the pattern only (assemble) and the symbolic phase (analyze)
  void build_pattern(int ne_, int p_, int block_, int nq_, int leaf_min_);
  void build_symbolic();
  // exact column counts of L by the elimination tree (after build_symbolic)
  void exact_counts();
};

}  // namespace rq
