// Host-side block tree of libacm (see forest.hpp).
#include "forest.hpp"

#include <algorithm>

namespace acm {

Directions::Directions() {
  int nf = 0, ne = 6, nc = 18;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int n = (dx != 0) + (dy != 0) + (dz != 0);
        int* slot = nullptr;
        if (n == 1) slot = d[nf++];
        else if (n == 2) slot = d[ne++];
        else if (n == 3) slot = d[nc++];
        if (slot) { slot[0] = dx; slot[1] = dy; slot[2] = dz; }
      }
}
const Directions kDirs;

size_t LeafMap::capacity_for(int64_t max_entries) {
  size_t cap = 16;
  while (cap < (size_t)(2 * max_entries + 16)) cap <<= 1;
  return cap;
}

void LeafMap::init(int64_t max_entries, Entry* storage) {
  const size_t cap = capacity_for(max_entries);
  if (storage) {
    own_.clear();
    tab_ = storage;
  } else {
    own_.assign(cap, Entry{BoxKey{0, 0, 0, 0}, -1});
    tab_ = own_.data();
  }
  for (size_t i = 0; i < cap; ++i) tab_[i] = Entry{BoxKey{0, 0, 0, 0}, -1};
  mask_ = cap - 1;
  n_ = 0;
}

void LeafMap::clear() {
  for (size_t i = 0; i <= mask_; ++i) tab_[i].slot = -1;
  n_ = 0;
}

void LeafMap::put(const BoxKey& k, int32_t slot) {
  size_t i = hash(k) & mask_;
  while (true) {
    Entry& e = tab_[i];
    if (e.slot < 0) {
      e.k = k;
      e.slot = slot;
      ++n_;
      return;
    }
    if (e.k == k) {
      e.slot = slot;
      return;
    }
    i = (i + 1) & mask_;
  }
}

bool LeafMap::erase(const BoxKey& k) {
  size_t i = hash(k) & mask_;
  while (true) {
    if (tab_[i].slot < 0) return false;
    if (tab_[i].k == k) break;
    i = (i + 1) & mask_;
  }
  // backward-shift deletion keeps every probe chain unbroken
  size_t j = i;
  while (true) {
    j = (j + 1) & mask_;
    if (tab_[j].slot < 0) break;
    const size_t home = hash(tab_[j].k) & mask_;
    // move entry j into the hole at i unless its home lies cyclically in (i, j]
    const bool in_range = (i <= j) ? (home > i && home <= j) : (home > i || home <= j);
    if (!in_range) {
      tab_[i] = tab_[j];
      i = j;
    }
  }
  tab_[i].slot = -1;
  --n_;
  return true;
}

Forest::Forest(const int nr[3], int bs, int jmin, int jmax, int64_t maxb, LeafMap::Entry* leaf_storage)
    : Bs(bs), M(bs - 1), Jmin(jmin), Jmax(jmax), max_blocks(maxb) {
  for (int a = 0; a < 3; ++a) nroot[a] = nr[a];
  leaves.init(maxb, leaf_storage);
  clear();
}

void Forest::clear() {
  leaves.clear();
  free_.assign((size_t)((max_blocks + 63) / 64), ~0ull);
  if (max_blocks % 64) free_.back() = (1ull << (max_blocks % 64)) - 1;
  nfree_ = max_blocks;
}

BoxKey Forest::wrap(int J, int64_t x, int64_t y, int64_t z) const {
  int64_t v[3] = {x, y, z};
  for (int a = 0; a < 3; ++a) {
    int64_t n = nblocks_axis(J, a);
    v[a] %= n;
    if (v[a] < 0) v[a] += n;
  }
  return BoxKey{J, (int32_t)v[0], (int32_t)v[1], (int32_t)v[2]};
}

// Spread the low 21 bits of v to every third bit (bit i -> bit 3i).
static inline uint64_t spread3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | v << 32) & 0x1f00000000ffffull;
  v = (v | v << 16) & 0x1f0000ff0000ffull;
  v = (v | v << 8) & 0x100f00f00f00f00full;
  v = (v | v << 4) & 0x10c30c30c30c30c3ull;
  v = (v | v << 2) & 0x1249249249249249ull;
  return v;
}

uint64_t Forest::treecode(const BoxKey& k) const {
  const int J = k.J;
  const uint64_t rx = (uint64_t)k.x >> J, ry = (uint64_t)k.y >> J, rz = (uint64_t)k.z >> J;
  const uint64_t root = rx + (uint64_t)nroot[0] * (ry + (uint64_t)nroot[1] * rz);
  const uint64_t m = (1ull << J) - 1;
  // digit of level l (bx + 2 by + 4 bz from bit J-l of the in-root coordinates) at bits 3(18-l)
  const uint64_t il = spread3(k.x & m) | (spread3(k.y & m) << 1) | (spread3(k.z & m) << 2);
  return (root << 56) | (J ? il << (3 * (18 - J)) : 0ull);
}

bool Forest::key_less(const BoxKey& a, const BoxKey& b) const {
  const uint64_t ta = treecode(a), tb = treecode(b);
  if (ta != tb) return ta < tb;
  return a.J < b.J;
}

std::vector<BoxKey> Forest::sorted() const {
  std::vector<std::pair<std::pair<uint64_t, int>, BoxKey>> tmp;
  tmp.reserve(leaves.size());
  leaves.for_each([&](const BoxKey& k, int32_t) { tmp.push_back({{treecode(k), k.J}, k}); });
  std::sort(tmp.begin(), tmp.end(),
            [](const auto& a, const auto& b) { return a.first < b.first; });
  std::vector<BoxKey> out;
  out.reserve(tmp.size());
  for (auto& t : tmp) out.push_back(t.second);
  return out;
}

bool Forest::apply_pass(const std::vector<BoxKey>& removed, const std::vector<BoxKey>& created,
                        std::vector<int32_t>* created_slots, bool created_sorted) {
  if ((int64_t)created.size() - (int64_t)removed.size() > nfree_) return false;
  for (const BoxKey& k : removed) {
    const int32_t s = leaves.get(k);
    if (s < 0) continue;
    free_[s >> 6] |= 1ull << (s & 63);
    ++nfree_;
    leaves.erase(k);
  }
  std::vector<size_t> idx(created.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
  if (!created_sorted) {
    std::vector<std::pair<uint64_t, int>> keys(created.size());
    for (size_t i = 0; i < created.size(); ++i) keys[i] = {treecode(created[i]), created[i].J};
    std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return keys[a] < keys[b]; });
  }
  if (created_slots) created_slots->assign(created.size(), -1);
  // ascending key order takes ascending free slots: one forward sweep over the bitmap
  size_t w = 0;
  for (size_t i : idx) {
    while (free_[w] == 0) ++w;
    const int b = __builtin_ctzll(free_[w]);
    free_[w] &= free_[w] - 1;
    --nfree_;
    const int32_t s = (int32_t)(w * 64 + b);
    leaves.put(created[i], s);
    if (created_slots) (*created_slots)[i] = s;
  }
  return true;
}

bool Forest::take_slots(const std::vector<int32_t>& freed, size_t n, std::vector<int32_t>* slots) {
  if ((int64_t)n - (int64_t)freed.size() > nfree_) return false;
  for (int32_t s : freed) {
    free_[s >> 6] |= 1ull << (s & 63);
    ++nfree_;
  }
  slots->resize(n);
  size_t w = 0;
  for (size_t i = 0; i < n; ++i) {
    while (free_[w] == 0) ++w;
    const int b = __builtin_ctzll(free_[w]);
    free_[w] &= free_[w] - 1;
    --nfree_;
    (*slots)[i] = (int32_t)(w * 64 + b);
  }
  return true;
}

void Forest::update_leaves(const std::vector<BoxKey>& removed, const std::vector<BoxKey>& created,
                           const std::vector<int32_t>& slots) {
  for (const BoxKey& k : removed) leaves.erase(k);
  for (size_t i = 0; i < created.size(); ++i) leaves.put(created[i], slots[i]);
}

BoxStatus Forest::box_status(int J, int64_t x, int64_t y, int64_t z) const {
  BoxStatus st;
  st.type = BOX_NONE;
  st.octant = 0;
  for (int c = 0; c < 8; ++c) st.slot[c] = -1;
  const BoxKey k = wrap(J, x, y, z);
  const int32_t s = leaves.get(k);
  if (s >= 0) {
    st.type = BOX_LEAF;
    st.slot[0] = s;
    return st;
  }
  if (J > 0) {
    const int32_t sp = leaves.get(BoxKey{J - 1, k.x >> 1, k.y >> 1, k.z >> 1});
    if (sp >= 0) {
      st.type = BOX_COARSER;
      st.slot[0] = sp;
      st.octant = (k.x & 1) | ((k.y & 1) << 1) | ((k.z & 1) << 2);
      return st;
    }
  }
  bool any = false;
  for (int c = 0; c < 8; ++c) {
    const int32_t sc = leaves.get(child(k, c));
    if (sc >= 0) {
      st.slot[c] = sc;
      any = true;
    }
  }
  if (any) st.type = BOX_REFINED;
  return st;
}

// Children of the box at offset d that touch the block (ascending child number).
static int touching_children(const int d[3], int out[8]) {
  int n = 0;
  for (int c = 0; c < 8; ++c) {
    const int cc[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
      if (d[a] == 1 && cc[a] != 0) ok = false;
      if (d[a] == -1 && cc[a] != 1) ok = false;
    }
    if (ok) out[n++] = c;
  }
  return n;
}

bool Forest::is_graded() const {
  bool ok = true;
  leaves.for_each([&](const BoxKey& b, int32_t) {
    for (int k = 0; k < 26 && ok; ++k) {
      const int* d = kDirs.d[k];
      BoxStatus st = box_status(b.J, (int64_t)b.x + d[0], (int64_t)b.y + d[1], (int64_t)b.z + d[2]);
      if (st.type == BOX_NONE) ok = false;
      if (st.type == BOX_REFINED) {
        int tc[8];
        const int n = touching_children(d, tc);
        for (int i = 0; i < n; ++i)
          if (st.slot[tc[i]] < 0) ok = false;
      }
    }
  });
  return ok;
}

bool Forest::tiles_domain() const {
  if (leaves.empty()) return false;
  int Jref = 0;
  leaves.for_each([&](const BoxKey& k, int32_t) { Jref = std::max(Jref, k.J); });
  // volume count in units of level-Jref boxes, then no overlap via the parent chain
  __int128 vol = 0;
  leaves.for_each([&](const BoxKey& k, int32_t) { vol += (__int128)1 << (3 * (Jref - k.J)); });
  __int128 total = (__int128)nblocks_axis(Jref, 0) * nblocks_axis(Jref, 1) * nblocks_axis(Jref, 2);
  if (vol != total) return false;
  bool ok = true;
  leaves.for_each([&](const BoxKey& b, int32_t) {
    for (int L = b.J - 1; L >= 0 && ok; --L) {
      const int s = b.J - L;
      if (leaves.contains(BoxKey{L, b.x >> s, b.y >> s, b.z >> s})) ok = false;
    }
  });
  return ok;
}

void Forest::neighbour_table(const std::vector<BoxKey>& order, int32_t* nbr, int8_t* rel) const {
  for (size_t i = 0; i < order.size(); ++i) {
    const BoxKey& b = order[i];
    int32_t* row = nbr + 56 * i;
    for (int e = 0; e < 56; ++e) row[e] = -1;
    for (int k = 0; k < 26; ++k) {
      const int* d = kDirs.d[k];
      const BoxStatus st =
          box_status(b.J, (int64_t)b.x + d[0], (int64_t)b.y + d[1], (int64_t)b.z + d[2]);
      int s0, n;
      group_of(k, &s0, &n);
      if (st.type == BOX_LEAF) {
        row[s0] = st.slot[0];
        rel[26 * i + k] = 0;
      } else if (st.type == BOX_COARSER) {
        row[s0] = st.slot[0];
        rel[26 * i + k] = -1;
      } else if (st.type == BOX_REFINED) {
        int tc[8];
        const int nt = touching_children(d, tc);
        for (int j = 0; j < nt && j < n; ++j) row[s0 + j] = st.slot[tc[j]];
        rel[26 * i + k] = 1;
      } else {
        rel[26 * i + k] = 0;
      }
    }
  }
}

}  // namespace acm
