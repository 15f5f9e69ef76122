// Octree plan for a fast-multipole far field (host only; no device work).
//
// The paper evaluates its layer potentials with a fast multipole method
// (Section 4.1) and leaves the method's internals to its library.  This file
// builds the combinatorial part of the classical uniform-depth scheme
// (Greengard and Rokhlin 1987): a sparse octree of depth L over the nodes,
// the neighbour lists of the leaves (near interactions) and the interaction
// lists of every level (far interactions translated between expansions).
//
// Boxes at level l are the cells of a 2^l x 2^l x 2^l grid over a cube that
// holds every node; only cells containing nodes are kept.  Two boxes of one
// level are adjacent when their integer coordinates differ by at most 1 in
// each direction.  The lists are
//   U(leaf b)  = the leaves adjacent to b, b included;
//   V(box b)   = the children of the boxes adjacent to parent(b) that are not
//                adjacent to b (levels >= 2).
// Adjacency of two boxes implies adjacency of their parents, so for two
// leaves a, b exactly one of these holds: b is in U(a), or at exactly one
// level l the ancestors satisfy A_l(b) in V(A_l(a)).  Every ordered pair of
// nodes is therefore covered exactly once.  When the leaf side is at least
// (eta + 1) max_P R_P, every node of a patch near a target (|x - c_P| <
// eta R_P) lies in a leaf of U(leaf of the target), so the near-field
// corrections stay inside the leaf-to-leaf interactions.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <new>
#include <vector>

#include "internal.cuh"

struct lb_fmm_plan {
  int depth = 0;
  int64_t n = 0;
  double lo[3] = {0, 0, 0};
  double side = 0;
  std::vector<int64_t> perm;        // [n] node ids in Morton order
  std::vector<int64_t> level_ptr;   // [depth + 2] box ranges per level
  std::vector<uint64_t> key;        // [nbox] Morton key at its level, ascending per level
  std::vector<int64_t> parent;      // [nbox] -1 at level 0
  std::vector<int64_t> node_ptr;    // [nleaf + 1] ranges of perm per leaf
  std::vector<int64_t> u_ptr, u_idx;  // leaf-local indices
  std::vector<int64_t> v_ptr, v_idx;  // global box indices
};

namespace {

uint64_t spread3(uint64_t v) {  // 21 bits -> every third bit
  v &= 0x1fffffull;
  v = (v | v << 32) & 0x1f00000000ffffull;
  v = (v | v << 16) & 0x1f0000ff0000ffull;
  v = (v | v << 8) & 0x100f00f00f00f00full;
  v = (v | v << 4) & 0x10c30c30c30c30c3ull;
  v = (v | v << 2) & 0x1249249249249249ull;
  return v;
}

uint64_t compact3(uint64_t v) {
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
  v = (v ^ (v >> 32)) & 0x1fffffull;
  return v;
}

uint64_t morton(uint64_t x, uint64_t y, uint64_t z) { return spread3(x) | spread3(y) << 1 | spread3(z) << 2; }

void coords(uint64_t k, int64_t* c) {
  c[0] = (int64_t)compact3(k);
  c[1] = (int64_t)compact3(k >> 1);
  c[2] = (int64_t)compact3(k >> 2);
}

bool adjacent(uint64_t a, uint64_t b) {
  int64_t ca[3], cb[3];
  coords(a, ca);
  coords(b, cb);
  for (int k = 0; k < 3; ++k)
    if (std::llabs(ca[k] - cb[k]) > 1) return false;
  return true;
}

// index of key k among the boxes [b, e) of one level, or -1
int64_t find_box(const lb_fmm_plan* p, int64_t b, int64_t e, uint64_t k) {
  auto it = std::lower_bound(p->key.begin() + b, p->key.begin() + e, k);
  if (it == p->key.begin() + e || *it != k) return -1;
  return it - p->key.begin();
}

// boxes of level l adjacent to box index bi (same level), bi included
void neighbours(const lb_fmm_plan* p, int l, int64_t bi, std::vector<int64_t>& out) {
  out.clear();
  const int64_t b = p->level_ptr[l], e = p->level_ptr[l + 1];
  const int64_t m = (int64_t)1 << l;
  int64_t c[3];
  coords(p->key[bi], c);
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int64_t x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
        if (x < 0 || y < 0 || z < 0 || x >= m || y >= m || z >= m) continue;
        const int64_t j = find_box(p, b, e, morton((uint64_t)x, (uint64_t)y, (uint64_t)z));
        if (j >= 0) out.push_back(j);
      }
  std::sort(out.begin(), out.end());
}

int build(lb_fmm_plan* p, int64_t n, const double* X, double min_leaf_side, int max_depth) {
  double lo[3], hi[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = X[k];
    hi[k] = X[k];
  }
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      const double v = X[3 * i + k];
      if (!std::isfinite(v)) return lb_fail(nullptr, LB_EINVAL, "node %lld has a non-finite coordinate", (long long)i);
      lo[k] = std::min(lo[k], v);
      hi[k] = std::max(hi[k], v);
    }
  double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]});
  if (ext <= 0) ext = 1.0;
  const double side = ext * (1.0 + 1e-9);  // every node strictly inside the cube
  int depth = 0;
  while (depth < max_depth && side / (double)((int64_t)1 << (depth + 1)) >= min_leaf_side) ++depth;
  p->depth = depth;
  p->n = n;
  p->side = side;
  for (int k = 0; k < 3; ++k) p->lo[k] = lo[k];
  // leaf keys and the Morton order of the nodes (ties by node id)
  const int64_t m = (int64_t)1 << depth;
  std::vector<uint64_t> nk(n);
  for (int64_t i = 0; i < n; ++i) {
    uint64_t c[3];
    for (int k = 0; k < 3; ++k) {
      int64_t q = (int64_t)std::floor((X[3 * i + k] - lo[k]) / side * (double)m);
      c[k] = (uint64_t)std::min<int64_t>(std::max<int64_t>(q, 0), m - 1);
    }
    nk[i] = morton(c[0], c[1], c[2]);
  }
  p->perm.resize(n);
  for (int64_t i = 0; i < n; ++i) p->perm[i] = i;
  std::stable_sort(p->perm.begin(), p->perm.end(), [&](int64_t a, int64_t b) { return nk[a] < nk[b]; });
  // boxes level by level, coarsest first
  std::vector<std::vector<uint64_t>> lev(depth + 1);
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t k = nk[p->perm[i]];
    if (lev[depth].empty() || lev[depth].back() != k) lev[depth].push_back(k);
  }
  for (int l = depth - 1; l >= 0; --l)
    for (uint64_t k : lev[l + 1]) {
      const uint64_t pk = k >> 3;
      if (lev[l].empty() || lev[l].back() != pk) lev[l].push_back(pk);
    }
  p->level_ptr.assign(depth + 2, 0);
  for (int l = 0; l <= depth; ++l) p->level_ptr[l + 1] = p->level_ptr[l] + (int64_t)lev[l].size();
  p->key.clear();
  for (int l = 0; l <= depth; ++l) p->key.insert(p->key.end(), lev[l].begin(), lev[l].end());
  const int64_t nbox = p->level_ptr[depth + 1];
  p->parent.assign(nbox, -1);
  for (int l = 1; l <= depth; ++l)
    for (int64_t bi = p->level_ptr[l]; bi < p->level_ptr[l + 1]; ++bi)
      p->parent[bi] = find_box(p, p->level_ptr[l - 1], p->level_ptr[l], p->key[bi] >> 3);
  // node ranges of the leaves
  const int64_t L0 = p->level_ptr[depth], nleaf = nbox - L0;
  p->node_ptr.assign(nleaf + 1, 0);
  {
    int64_t leaf = 0;
    for (int64_t i = 0; i < n; ++i) {
      while (p->key[L0 + leaf] != nk[p->perm[i]]) ++leaf;
      ++p->node_ptr[leaf + 1];
    }
    for (int64_t b = 0; b < nleaf; ++b) p->node_ptr[b + 1] += p->node_ptr[b];
  }
  // U lists of the leaves (leaf-local indices)
  std::vector<int64_t> nb;
  p->u_ptr.assign(nleaf + 1, 0);
  p->u_idx.clear();
  for (int64_t b = 0; b < nleaf; ++b) {
    neighbours(p, depth, L0 + b, nb);
    for (int64_t j : nb) p->u_idx.push_back(j - L0);
    p->u_ptr[b + 1] = (int64_t)p->u_idx.size();
  }
  // V lists, every level from 2 down
  p->v_ptr.assign(nbox + 1, 0);
  p->v_idx.clear();
  std::vector<int64_t> pn, row;
  for (int64_t bi = 0; bi < nbox; ++bi) {
    int l = 0;
    while (bi >= p->level_ptr[l + 1]) ++l;
    row.clear();
    if (l >= 2) {
      neighbours(p, l - 1, p->parent[bi], pn);
      for (int64_t q : pn) {
        const uint64_t base = p->key[q] << 3;
        for (uint64_t ch = 0; ch < 8; ++ch) {
          const int64_t c = find_box(p, p->level_ptr[l], p->level_ptr[l + 1], base | ch);
          if (c >= 0 && !adjacent(p->key[c], p->key[bi])) row.push_back(c);
        }
      }
      std::sort(row.begin(), row.end());
    }
    p->v_idx.insert(p->v_idx.end(), row.begin(), row.end());
    p->v_ptr[bi + 1] = (int64_t)p->v_idx.size();
  }
  return LB_OK;
}

}  // namespace

extern "C" int lb_fmm_plan_create(int64_t n, const double* X, double min_leaf_side, int max_depth,
                                  lb_fmm_plan** out) {
  if (!out) return lb_fail(nullptr, LB_EINVAL, "null output pointer");
  *out = nullptr;
  if (n < 1 || !X) return lb_fail(nullptr, LB_EINVAL, "need n >= 1 nodes");
  if (max_depth < 0 || max_depth > 20) return lb_fail(nullptr, LB_EINVAL, "max_depth must be in [0, 20]");
  if (!(min_leaf_side > 0)) return lb_fail(nullptr, LB_EINVAL, "min_leaf_side must be positive");
  lb_fmm_plan* p = new (std::nothrow) lb_fmm_plan;
  if (!p) return lb_fail(nullptr, LB_ENOMEM, "host allocation failed");
  int rc;
  try {
    rc = build(p, n, X, min_leaf_side, max_depth);
  } catch (const std::bad_alloc&) {
    rc = lb_fail(nullptr, LB_ENOMEM, "host allocation failed");
  }
  if (rc != LB_OK) {
    delete p;
    return rc;
  }
  *out = p;
  return LB_OK;
}

extern "C" int lb_fmm_plan_info(const lb_fmm_plan* p, lb_fmm_info* info) {
  if (!p || !info) return lb_fail(nullptr, LB_EINVAL, "null argument");
  info->depth = p->depth;
  info->n = p->n;
  info->nbox = p->level_ptr.back();
  info->nleaf = p->level_ptr.back() - p->level_ptr[p->depth];
  info->nu = (int64_t)p->u_idx.size();
  info->nv = (int64_t)p->v_idx.size();
  for (int k = 0; k < 3; ++k) info->lo[k] = p->lo[k];
  info->side = p->side;
  return LB_OK;
}

extern "C" int lb_fmm_plan_arrays(const lb_fmm_plan* p, int64_t* perm, int64_t* level_ptr, int64_t* box_key,
                                  int64_t* box_parent, int64_t* node_ptr, int64_t* u_ptr, int64_t* u_idx,
                                  int64_t* v_ptr, int64_t* v_idx) {
  if (!p) return lb_fail(nullptr, LB_EINVAL, "null plan");
  auto put = [](int64_t* dst, const std::vector<int64_t>& src) {
    if (dst) std::copy(src.begin(), src.end(), dst);
  };
  put(perm, p->perm);
  put(level_ptr, p->level_ptr);
  if (box_key)
    for (size_t i = 0; i < p->key.size(); ++i) box_key[i] = (int64_t)p->key[i];
  put(box_parent, p->parent);
  put(node_ptr, p->node_ptr);
  put(u_ptr, p->u_ptr);
  put(u_idx, p->u_idx);
  put(v_ptr, p->v_ptr);
  put(v_idx, p->v_idx);
  return LB_OK;
}

extern "C" int lb_fmm_plan_destroy(lb_fmm_plan* p) {
  delete p;
  return LB_OK;
}
