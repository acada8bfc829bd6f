// fmm_oracle.cpp -- the CPU oracle for the FMM data-structure build.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
// definition of what the GPU library computes, written from the paper
// (Q. Hu, N. A. Gumerov, R. Duraiswami, "Parallel algorithms for constructing
// data structures for fast multipole methods", arXiv:1301.1704).  Only the
// tests, __graft_entry__.smoke() and the cpu_baseline leg of bench.py may load
// it.  It shares no code, header, table or helper with the CUDA path.
// Built a second time with OpenMP (for the timed CPU baseline only), the key
// loop and the per-box list loop run on all cores; the test
// test_parallel_build_equals_serial pins that build to this one.
//
// What it computes, in the paper's order:
//   * box index of a point at the finest grid and its Morton key
//     (Sec. 2, "BoxIndex(P[i])" in Alg. 1; Sec. 1.4 Morton indices);
//   * the order of the points (Alg. 1 pseudo-sort, made deterministic:
//     ascending (Morton key, original index), done with std::sort);
//   * per level 0..L: the Morton keys of the non-empty boxes
//     ("NonEmptyBoxIndex"), the bookmarks ("Bookmark", first sorted point of
//     each non-empty box, plus a final entry n), parent ranks and child ranges
//     (Alg. 3, Sec. 2.2);
//   * per level 2..L and per non-empty receiver box: the E2 neighbour list
//     (Alg. 4; Sec. 1.4 item 2) and the E4 interaction list
//     (Sec. 1.4 item 4: E4(n,l) = E2(Parent(n), l-1) \ E2(n,l)), both as
//     ascending ranks of non-empty source boxes, in CSR form;
//   * cluster-size mode (Sec. 2.1): the smallest level L >= 2 at which no
//     finest box of either set holds more than s points.
//
// Lists come from two independent routes: "stencil" (decode the box, step
// to each neighbouring cell, binary-search its key among the non-empty source
// boxes, sort the hits) and "brute" (test every (receiver, source) box pair
// against the definition).  Neither uses the identity that the children of a
// parent's neighbours are exactly E2 + E4; the tests check that identity.
//
// Readings where the paper is silent (the same readings the library takes):
//   * 21 bits per dimension, 63-bit keys; x -> bit 3k, y -> 3k+1, z -> 3k+2;
//   * domain [0,1] inclusive; 1.0 goes to the last cell; < 0, > 1, NaN are
//     errors;
//   * order inside a box: (full key, original index);
//   * E2 includes the box itself when it is a non-empty source box;
//   * lists at every level 2..L, none at levels 0 and 1; no periodicity.
//
// Parity pins (tests/): geometric bisection of the cube for the keys,
// numpy's stable sort for the order, invariants of the bookmarks, all-pairs
// brute force for the lists, the parent-neighbourhood identity, symmetry for
// src == recv, and the closed-form list counts of a full lattice.

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

namespace {

const int kMaxLevel = 21;                 // 21 bits per dimension
const uint32_t kGrid = 1u << kMaxLevel;   // cells per dimension at level 21

enum {
  ORC_OK = 0,
  ORC_ERR_ARG = 1,
  ORC_ERR_DOMAIN = 2,
  ORC_ERR_LEVEL = 3,
};

// Sec. 2 "BoxIndex": the level-21 cell of one coordinate.  x * 2^21 is exact in
// float32 (power-of-two scale) and truncation is floor for x >= 0.
int quantize(float x, uint32_t* q) {
  if (!(x >= 0.0f && x <= 1.0f)) return ORC_ERR_DOMAIN;  // NaN fails too
  uint32_t v = (uint32_t)(x * 2097152.0f);
  if (v == kGrid) v = kGrid - 1;  // x == 1.0 belongs to the last cell
  *q = v;
  return ORC_OK;
}

// Sec. 1.4 / Sec. 2.3: Morton index by bit interleaving, one bit at a time.
uint64_t interleave(uint32_t qx, uint32_t qy, uint32_t qz, int bits) {
  uint64_t key = 0;
  for (int k = 0; k < bits; ++k) {
    key |= (uint64_t)((qx >> k) & 1u) << (3 * k);
    key |= (uint64_t)((qy >> k) & 1u) << (3 * k + 1);
    key |= (uint64_t)((qz >> k) & 1u) << (3 * k + 2);
  }
  return key;
}

// Sec. 2.3 deinterleave: Morton index -> integer box coordinates.
void deinterleave(uint64_t key, int bits, int64_t c[3]) {
  c[0] = c[1] = c[2] = 0;
  for (int k = 0; k < bits; ++k) {
    c[0] |= (int64_t)((key >> (3 * k)) & 1u) << k;
    c[1] |= (int64_t)((key >> (3 * k + 1)) & 1u) << k;
    c[2] |= (int64_t)((key >> (3 * k + 2)) & 1u) << k;
  }
}

int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

// Chebyshev (max-norm) distance between two boxes of one level.
int64_t cheb(const int64_t a[3], const int64_t b[3]) {
  int64_t d = 0;
  for (int i = 0; i < 3; ++i) d = std::max(d, iabs64(a[i] - b[i]));
  return d;
}

struct Side {
  uint32_t n = 0;
  std::vector<uint64_t> point_key;           // per input point, original order
  std::vector<uint32_t> perm;                // sorted position -> original index
  std::vector<uint64_t> sorted_key;          // keys in sorted order
  std::vector<std::vector<uint64_t>> key;    // per level: box Morton keys
  std::vector<std::vector<uint32_t>> off;    // per level: bookmarks (nbox+1)
  std::vector<std::vector<uint32_t>> parent; // per level >= 1: rank at l-1
  std::vector<std::vector<uint32_t>> child;  // per level < L: ranges at l+1
};

struct Tree {
  int L = 0;
  int s_unmet = 0;
  Side side[2];  // 0 = sources, 1 = receivers
  std::vector<std::vector<uint32_t>> e2_off, e2_idx, e4_off, e4_idx;
};

// Keys of every point of one set, in input order.  (Compiled with OpenMP,
// the loop runs on all cores; the first error of any point is returned.)
int make_keys(const float* xyz, uint32_t n, std::vector<uint64_t>* keys) {
  keys->assign(n, 0);
  int err = ORC_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < (int64_t)n; ++i) {
    uint32_t q[3];
    int st = ORC_OK;
    for (int d = 0; d < 3 && st == ORC_OK; ++d) st = quantize(xyz[3 * (size_t)i + d], &q[d]);
    if (st != ORC_OK) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      err = st;
      continue;
    }
    (*keys)[i] = interleave(q[0], q[1], q[2], kMaxLevel);
  }
  return err;
}

// Alg. 1, deterministic: ascending (key, original index).
void sort_points(Side* s) {
  std::vector<std::pair<uint64_t, uint32_t>> pairs(s->n);
  for (uint32_t i = 0; i < s->n; ++i) pairs[i] = std::make_pair(s->point_key[i], i);
  std::sort(pairs.begin(), pairs.end());
  s->perm.resize(s->n);
  s->sorted_key.resize(s->n);
  for (uint32_t j = 0; j < s->n; ++j) {
    s->sorted_key[j] = pairs[j].first;
    s->perm[j] = pairs[j].second;
  }
}

// The order variant that sorts only by the box (Sec. 2.1: the order of the
// points inside a box is irrelevant): ascending (level-L key, original
// index).  The boxes of levels 0..L are the same as in the full-key order.
void box_key_order(Side* s, int L) {
  const int shift = 3 * (kMaxLevel - L);
  std::vector<std::pair<uint64_t, uint32_t>> pairs(s->n);
  for (uint32_t i = 0; i < s->n; ++i) pairs[i] = std::make_pair(s->point_key[i] >> shift, i);
  std::sort(pairs.begin(), pairs.end());
  for (uint32_t j = 0; j < s->n; ++j) s->perm[j] = pairs[j].second;
}

// Alg. 3 for every level 0..Lmax: the distinct level-l keys along the sorted
// order are the non-empty boxes; the first occurrence is the bookmark.
void make_boxes(Side* s, int Lmax) {
  s->key.assign(Lmax + 1, {});
  s->off.assign(Lmax + 1, {});
  s->parent.assign(Lmax + 1, {});
  s->child.assign(Lmax + 1, {});
  for (int l = 0; l <= Lmax; ++l) {
    const int shift = 3 * (kMaxLevel - l);
    for (uint32_t j = 0; j < s->n; ++j) {
      uint64_t kl = s->sorted_key[j] >> shift;
      if (j == 0 || kl != (s->sorted_key[j - 1] >> shift)) {
        s->key[l].push_back(kl);
        s->off[l].push_back(j);
      }
    }
    s->off[l].push_back(s->n);
  }
  // Parent rank: where the parent's key sits among the level l-1 keys.
  for (int l = 1; l <= Lmax; ++l) {
    const std::vector<uint64_t>& up = s->key[l - 1];
    for (uint64_t kl : s->key[l]) {
      uint64_t pk = kl >> 3;
      auto it = std::lower_bound(up.begin(), up.end(), pk);
      s->parent[l].push_back((uint32_t)(it - up.begin()));
    }
  }
  // Child range of box b at level l: the level l+1 boxes whose parent is b.
  for (int l = 0; l < Lmax; ++l) {
    const std::vector<uint32_t>& par = s->parent[l + 1];
    for (uint32_t b = 0; b <= (uint32_t)s->key[l].size(); ++b) {
      auto it = std::lower_bound(par.begin(), par.end(), b);
      s->child[l].push_back((uint32_t)(it - par.begin()));
    }
  }
}

// Largest box occupancy at level l.
uint32_t max_occupancy(const Side& s, int l) {
  uint32_t m = 0;
  for (size_t b = 0; b + 1 < s.off[l].size(); ++b)
    m = std::max(m, s.off[l][b + 1] - s.off[l][b]);
  return m;
}

// Ascending level-l keys of the non-empty source boxes (not owned).
struct KeyView {
  const uint64_t* p;
  size_t n;
};

KeyView view_of(const std::vector<uint64_t>& v) { return KeyView{v.data(), v.size()}; }

// Rank of a level-l key among the non-empty source boxes, or -1.
int64_t find_rank(KeyView keys, uint64_t k) {
  const uint64_t* it = std::lower_bound(keys.p, keys.p + keys.n, k);
  if (it == keys.p + keys.n || *it != k) return -1;
  return (int64_t)(it - keys.p);
}

// Stencil route for one receiver box (key rk at level l >= 2).
//   E2: the 27 cells at Chebyshev distance <= 1 inside the cube.
//   E4: the children of the 27 cells around the parent (Sec. 1.4 item 4),
//       minus E2.
void stencil_lists(KeyView src_keys, int l, uint64_t rk,
                   std::vector<uint32_t>* e2, std::vector<uint32_t>* e4) {
  e2->clear();
  e4->clear();
  const int64_t side = (int64_t)1 << l;
  int64_t c[3];
  deinterleave(rk, l, c);
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t n[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
        if (n[0] < 0 || n[1] < 0 || n[2] < 0 || n[0] >= side || n[1] >= side || n[2] >= side)
          continue;
        int64_t r = find_rank(src_keys, interleave((uint32_t)n[0], (uint32_t)n[1], (uint32_t)n[2], l));
        if (r >= 0) e2->push_back((uint32_t)r);
      }
  const int64_t pside = side >> 1;
  const int64_t p[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t q[3] = {p[0] + dx, p[1] + dy, p[2] + dz};
        if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= pside || q[1] >= pside || q[2] >= pside)
          continue;
        for (int o = 0; o < 8; ++o) {
          int64_t t[3] = {2 * q[0] + (o & 1), 2 * q[1] + ((o >> 1) & 1), 2 * q[2] + ((o >> 2) & 1)};
          if (cheb(t, c) <= 1) continue;  // belongs to E2(n, l)
          int64_t r = find_rank(src_keys, interleave((uint32_t)t[0], (uint32_t)t[1], (uint32_t)t[2], l));
          if (r >= 0) e4->push_back((uint32_t)r);
        }
      }
  std::sort(e2->begin(), e2->end());
  std::sort(e4->begin(), e4->end());
}

// Brute-force route for one receiver box: every source box of the level is
// tested against the definitions of E2 and E4.
void brute_lists(KeyView src_keys, int l, uint64_t rk,
                 std::vector<uint32_t>* e2, std::vector<uint32_t>* e4) {
  e2->clear();
  e4->clear();
  int64_t c[3], pc[3];
  deinterleave(rk, l, c);
  for (int d = 0; d < 3; ++d) pc[d] = c[d] >> 1;
  for (uint32_t t = 0; t < (uint32_t)src_keys.n; ++t) {
    int64_t s[3], ps[3];
    deinterleave(src_keys.p[t], l, s);
    for (int d = 0; d < 3; ++d) ps[d] = s[d] >> 1;
    if (cheb(c, s) <= 1)
      e2->push_back(t);
    else if (cheb(pc, ps) <= 1)
      e4->push_back(t);
  }
}

void make_lists(Tree* t, int mode) {
  const int L = t->L;
  t->e2_off.assign(L + 1, {});
  t->e2_idx.assign(L + 1, {});
  t->e4_off.assign(L + 1, {});
  t->e4_idx.assign(L + 1, {});
  const Side& src = t->side[0];
  const Side& recv = t->side[1];
  for (int l = 2; l <= L; ++l) {
    t->e2_off[l].push_back(0);
    t->e4_off[l].push_back(0);
    // Receiver boxes in blocks; each block's lists are appended in box order.
    // (Compiled with OpenMP, the blocks of a round run on all cores.)
    const std::vector<uint64_t>& rkeys = recv.key[l];
    const int64_t nr = (int64_t)rkeys.size(), blk = 4096;
    const int64_t nblk = (nr + blk - 1) / blk, round = 64;
    for (int64_t b0 = 0; b0 < nblk; b0 += round) {
      const int64_t b1 = std::min(nblk, b0 + round);
      std::vector<std::vector<uint32_t>> e2b(b1 - b0), e4b(b1 - b0), c2b(b1 - b0), c4b(b1 - b0);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
      for (int64_t b = b0; b < b1; ++b) {
        std::vector<uint32_t> e2, e4;
        for (int64_t r = b * blk; r < std::min(nr, (b + 1) * blk); ++r) {
          if (mode == 1)
            brute_lists(view_of(src.key[l]), l, rkeys[r], &e2, &e4);
          else
            stencil_lists(view_of(src.key[l]), l, rkeys[r], &e2, &e4);
          e2b[b - b0].insert(e2b[b - b0].end(), e2.begin(), e2.end());
          e4b[b - b0].insert(e4b[b - b0].end(), e4.begin(), e4.end());
          c2b[b - b0].push_back((uint32_t)e2.size());
          c4b[b - b0].push_back((uint32_t)e4.size());
        }
      }
      for (int64_t b = b0; b < b1; ++b) {
        t->e2_idx[l].insert(t->e2_idx[l].end(), e2b[b - b0].begin(), e2b[b - b0].end());
        t->e4_idx[l].insert(t->e4_idx[l].end(), e4b[b - b0].begin(), e4b[b - b0].end());
        for (size_t k = 0; k < c2b[b - b0].size(); ++k) {
          t->e2_off[l].push_back(t->e2_off[l].back() + c2b[b - b0][k]);
          t->e4_off[l].push_back(t->e4_off[l].back() + c4b[b - b0][k]);
        }
      }
    }
  }
}

void truncate_levels(Side* s, int L) {
  s->key.resize(L + 1);
  s->off.resize(L + 1);
  s->parent.resize(L + 1);
  s->child.resize(L + 1);
  s->child[L].clear();  // no level L+1
}

}  // namespace

extern "C" {

// Morton keys of n points (xyz float32 [n][3]) in input order.
int orc_keys(const float* xyz, uint32_t n, uint64_t* keys) {
  if (n > 0 && (!xyz || !keys)) return ORC_ERR_ARG;
  std::vector<uint64_t> k;
  int st = make_keys(xyz, n, &k);
  if (st != ORC_OK) return st;
  if (n) std::memcpy(keys, k.data(), sizeof(uint64_t) * n);
  return ORC_OK;
}

uint64_t orc_encode(uint32_t qx, uint32_t qy, uint32_t qz, int bits) {
  return interleave(qx, qy, qz, bits);
}

void orc_decode(uint64_t key, int bits, int64_t* c3) { deinterleave(key, bits, c3); }

// Builds the whole structure.  L in [0, 21] (L mode) or L = -1 and s >= 1
// (cluster-size mode).  mode: 0 = stencil lists, 1 = brute-force lists,
// 2 = no lists (keys, order and boxes only); plus 16 for the box-key order
// of the points.
int orc_build(const float* src, uint32_t N, const float* recv, uint32_t M, int L,
              uint32_t s, int mode, void** out) {
  if (!out) return ORC_ERR_ARG;
  *out = nullptr;
  const bool box_order = (mode & 16) != 0;
  mode &= ~16;
  if ((N > 0 && !src) || (M > 0 && !recv) || mode < 0 || mode > 2) return ORC_ERR_ARG;
  if (L > kMaxLevel || L < -1 || (L == -1 && s == 0)) return ORC_ERR_LEVEL;
  Tree* t = new Tree();
  const float* in[2] = {src, recv};
  const uint32_t cnt[2] = {N, M};
  for (int k = 0; k < 2; ++k) {
    Side& sd = t->side[k];
    sd.n = cnt[k];
    int st = make_keys(in[k], sd.n, &sd.point_key);
    if (st != ORC_OK) {
      delete t;
      return st;
    }
    sort_points(&sd);
  }
  const int Lbox = (L >= 0) ? L : kMaxLevel;
  for (int k = 0; k < 2; ++k) make_boxes(&t->side[k], Lbox);
  if (L >= 0) {
    t->L = L;
  } else {
    // Sec. 2.1 cluster size: smallest level >= 2 where both sets fit.
    t->L = kMaxLevel;
    t->s_unmet = 1;
    for (int l = 2; l <= kMaxLevel; ++l) {
      if (max_occupancy(t->side[0], l) <= s && max_occupancy(t->side[1], l) <= s) {
        t->L = l;
        t->s_unmet = 0;
        break;
      }
    }
    for (int k = 0; k < 2; ++k) truncate_levels(&t->side[k], t->L);
  }
  if (box_order)
    for (int k = 0; k < 2; ++k) box_key_order(&t->side[k], t->L);
  if (mode != 2) make_lists(t, mode);
  *out = t;
  return ORC_OK;
}

void orc_free(void* h) { delete static_cast<Tree*>(h); }

int orc_level(void* h) { return static_cast<Tree*>(h)->L; }
int orc_s_unmet(void* h) { return static_cast<Tree*>(h)->s_unmet; }

// side: 0 = sources, 1 = receivers.
const uint32_t* orc_perm(void* h, int side) { return static_cast<Tree*>(h)->side[side].perm.data(); }
const uint64_t* orc_sorted_keys(void* h, int side) {
  return static_cast<Tree*>(h)->side[side].sorted_key.data();
}

uint32_t orc_nbox(void* h, int side, int l) {
  return (uint32_t) static_cast<Tree*>(h)->side[side].key[l].size();
}
const uint64_t* orc_box_keys(void* h, int side, int l) {
  return static_cast<Tree*>(h)->side[side].key[l].data();
}
const uint32_t* orc_box_off(void* h, int side, int l) {
  return static_cast<Tree*>(h)->side[side].off[l].data();
}
const uint32_t* orc_box_parent(void* h, int side, int l) {
  return static_cast<Tree*>(h)->side[side].parent[l].data();
}
uint32_t orc_box_child_len(void* h, int side, int l) {
  return (uint32_t) static_cast<Tree*>(h)->side[side].child[l].size();
}
const uint32_t* orc_box_child(void* h, int side, int l) {
  return static_cast<Tree*>(h)->side[side].child[l].data();
}

// which: 0 = E2, 1 = E4.  Valid for levels 2..L when lists were built.
uint64_t orc_nnz(void* h, int which, int l) {
  Tree* t = static_cast<Tree*>(h);
  return which == 0 ? t->e2_idx[l].size() : t->e4_idx[l].size();
}
const uint32_t* orc_list_off(void* h, int which, int l) {
  Tree* t = static_cast<Tree*>(h);
  return which == 0 ? t->e2_off[l].data() : t->e4_off[l].data();
}
const uint32_t* orc_list_idx(void* h, int which, int l) {
  Tree* t = static_cast<Tree*>(h);
  return which == 0 ? t->e2_idx[l].data() : t->e4_idx[l].data();
}

// Lists of one receiver box, for sampled checks at sizes where the whole
// list build is too slow.  src_keys: the nsrc ascending level-l source box
// keys.  mode 0 = stencil, 1 = brute.  e2 needs room for 27, e4 for 189.
int orc_box_lists(const uint64_t* src_keys, uint32_t nsrc, int l, uint64_t rkey, int mode,
                  uint32_t* e2, uint32_t* n2, uint32_t* e4, uint32_t* n4) {
  if (l < 2 || l > kMaxLevel || (nsrc && !src_keys)) return ORC_ERR_ARG;
  const KeyView keys{src_keys, nsrc};
  std::vector<uint32_t> a, b;
  if (mode == 1)
    brute_lists(keys, l, rkey, &a, &b);
  else
    stencil_lists(keys, l, rkey, &a, &b);
  *n2 = (uint32_t)a.size();
  *n4 = (uint32_t)b.size();
  if (a.size() > 27 || b.size() > 189) return ORC_ERR_ARG;  // impossible by definition
  std::copy(a.begin(), a.end(), e2);
  std::copy(b.begin(), b.end(), e4);
  return ORC_OK;
}

}  // extern "C"
