// Host-side block tree of libacm: leaves, octal treecodes, slot pool, neighbour queries.
//
// Paper, Sec. 4.1: equal-size Bs^3 blocks held in one preallocated array, positioned by
// octal (Gargantini) treecodes from which level, position and neighbours are computed; the
// tree metadata lives apart from the block data.  Sec. 3.5: refinement of all blocks and
// coarsening of sister groups, keeping the grid graded.  The rules fixed here (treecode bit
// layout, slot assignment, table layout, 26-neighbour 2:1 grading) are the ones documented in
// include/acm.h.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "leafhash.hpp"

namespace acm {

struct BoxKey {
  int32_t J, x, y, z;
  bool operator==(const BoxKey& o) const { return J == o.J && x == o.x && y == o.y && z == o.z; }
};

struct BoxKeyHash {
  size_t operator()(const BoxKey& k) const { return (size_t)leaf_hash(k.J, k.x, k.y, k.z); }
};

enum BoxType : uint8_t { BOX_LEAF = 0, BOX_COARSER = 1, BOX_REFINED = 2, BOX_NONE = 3 };

// Open-addressing hash table (linear probing, backward-shift deletion) from a box to the slot
// of the leaf occupying it.  Capacity is a power of two at least twice the block pool, so a
// probe always meets an empty entry.  The table may live in caller-provided storage (pinned
// host memory, copied byte for byte to the device, which probes it with the same hash).
class LeafMap {
 public:
  struct Entry {
    BoxKey k;
    int32_t slot;     // -1: empty
  };
  static size_t capacity_for(int64_t max_entries);
  // storage: capacity_for(max_entries) entries owned by the caller, or nullptr (owned here)
  void init(int64_t max_entries, Entry* storage = nullptr);
  const Entry* data() const { return tab_; }
  size_t capacity() const { return mask_ + 1; }
  void clear();
  int32_t get(const BoxKey& k) const {
    size_t i = hash(k) & mask_;
    while (true) {
      const Entry& e = tab_[i];
      if (e.slot < 0) return -1;
      if (e.k == k) return e.slot;
      i = (i + 1) & mask_;
    }
  }
  bool contains(const BoxKey& k) const { return get(k) >= 0; }
  void put(const BoxKey& k, int32_t slot);
  bool erase(const BoxKey& k);
  size_t size() const { return n_; }
  bool empty() const { return n_ == 0; }
  template <typename F>
  void for_each(F&& fn) const {
    for (size_t i = 0; i <= mask_; ++i)
      if (tab_[i].slot >= 0) fn(tab_[i].k, tab_[i].slot);
  }

 private:
  static size_t hash(const BoxKey& k) { return BoxKeyHash()(k); }
  std::vector<Entry> own_;
  Entry* tab_ = nullptr;
  size_t mask_ = 0, n_ = 0;
};
static_assert(sizeof(LeafMap::Entry) == sizeof(LeafEntry), "leaf map entries are copied to the device");

// Status of a level-J box as seen from a neighbour: a leaf itself, covered by a leaf one
// level coarser (slot[0], octant = which half per axis), or refined into level J+1 leaves
// (slot[c] for child c = cx + 2cy + 4cz, -1 where the child is not a leaf).
struct BoxStatus {
  BoxType type;
  int32_t slot[8];
  int octant;
};

// 26 neighbour directions: iterate dz, dy, dx over -1, 0, 1 (x fastest); faces, then edges,
// then corners.
struct Directions {
  int d[26][3];
  Directions();
};
extern const Directions kDirs;

// First table entry of direction k in the 56-entry layout and the group size.
inline void group_of(int k, int* start, int* n) {
  if (k < 6) { *start = 4 * k; *n = 4; }
  else if (k < 18) { *start = 24 + 2 * (k - 6); *n = 2; }
  else { *start = 48 + (k - 18); *n = 1; }
}

class Forest {
 public:
  // leaf_storage: LeafMap::capacity_for(max_blocks) entries owned by the caller, or nullptr
  Forest(const int nroot[3], int Bs, int Jmin, int Jmax, int64_t max_blocks,
         LeafMap::Entry* leaf_storage = nullptr);

  int nroot[3];
  int Bs, M, Jmin, Jmax;
  int64_t max_blocks;
  LeafMap leaves;

  int64_t nblocks_axis(int J, int a) const { return (int64_t)nroot[a] << J; }
  BoxKey wrap(int J, int64_t x, int64_t y, int64_t z) const;
  uint64_t treecode(const BoxKey& k) const;
  bool key_less(const BoxKey& a, const BoxKey& b) const;
  std::vector<BoxKey> sorted() const;
  int64_t n_free() const { return nfree_; }

  void clear();
  // One adaptation pass: release the slots of `removed`, then give `created` (any order)
  // the lowest free slots in ascending key order.  Returns false (and changes nothing) if
  // the pool is too small.  created_slots[i] is the slot of created[i].
  bool apply_pass(const std::vector<BoxKey>& removed, const std::vector<BoxKey>& created,
                  std::vector<int32_t>* created_slots, bool created_sorted = false);
  // The same pass in two halves, for callers that know the removed leaves' slots and hold the
  // created boxes in ascending key order: take_slots releases `freed` and assigns the n lowest
  // free slots in ascending order (false, and nothing changed, if the pool is too small);
  // update_leaves then records the pass in the leaf map.
  bool take_slots(const std::vector<int32_t>& freed, size_t n, std::vector<int32_t>* slots);
  void update_leaves(const std::vector<BoxKey>& removed, const std::vector<BoxKey>& created,
                     const std::vector<int32_t>& slots);

  BoxStatus box_status(int J, int64_t x, int64_t y, int64_t z) const;
  bool is_graded() const;
  bool tiles_domain() const;

  // Children of a box, child c = cx + 2cy + 4cz.
  static BoxKey child(const BoxKey& p, int c) {
    return BoxKey{p.J + 1, 2 * p.x + (c & 1), 2 * p.y + ((c >> 1) & 1), 2 * p.z + ((c >> 2) & 1)};
  }

  // 56-entry neighbour slots and 26 relative levels of each block of `order`.
  void neighbour_table(const std::vector<BoxKey>& order, int32_t* nbr, int8_t* rel) const;

 private:
  std::vector<uint64_t> free_;    // bit set = slot free
  int64_t nfree_ = 0;
};

}  // namespace acm
