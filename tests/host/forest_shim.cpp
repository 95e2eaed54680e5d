// C entry points over the library's host block tree (forest.cpp), so that the CPU test suite can
// exercise the host logic without a GPU: built with g++ by tests/test_host_forest.py.
#include <cstdint>
#include <vector>

#include "forest.hpp"

using acm::BoxKey;
using acm::Forest;

extern "C" {

void* hf_create(int nx, int ny, int nz, int Bs, int Jmin, int Jmax, int64_t max_blocks) {
  const int nr[3] = {nx, ny, nz};
  return new Forest(nr, Bs, Jmin, Jmax, max_blocks);
}

void hf_destroy(void* h) { delete static_cast<Forest*>(h); }

static std::vector<BoxKey> keys(int n, const int32_t* J, const int32_t* x, const int32_t* y, const int32_t* z) {
  std::vector<BoxKey> v(n);
  for (int i = 0; i < n; ++i) v[i] = BoxKey{J[i], x[i], y[i], z[i]};
  return v;
}

// One adaptation pass; created_slots[i] receives the slot of created box i.  1 on success.
int hf_apply_pass(void* h, int nr, const int32_t* rJ, const int32_t* rx, const int32_t* ry, const int32_t* rz,
                  int nc, const int32_t* cJ, const int32_t* cx, const int32_t* cy, const int32_t* cz,
                  int32_t* created_slots) {
  Forest* f = static_cast<Forest*>(h);
  std::vector<int32_t> slots;
  if (!f->apply_pass(keys(nr, rJ, rx, ry, rz), keys(nc, cJ, cx, cy, cz), &slots)) return 0;
  for (int i = 0; i < nc; ++i) created_slots[i] = slots[i];
  return 1;
}

// take_slots: the n lowest free slots after releasing `freed`, in ascending order.  1 on success.
int hf_take_slots(void* h, int nfreed, const int32_t* freed, int n, int32_t* out) {
  Forest* f = static_cast<Forest*>(h);
  std::vector<int32_t> s;
  if (!f->take_slots(std::vector<int32_t>(freed, freed + nfreed), (size_t)n, &s)) return 0;
  for (int i = 0; i < n; ++i) out[i] = s[i];
  return 1;
}

int64_t hf_n(void* h) { return (int64_t)static_cast<Forest*>(h)->leaves.size(); }

// Leaves in ascending key order: level, coordinates, slot and treecode of each.
void hf_sorted(void* h, int32_t* J, int32_t* x, int32_t* y, int32_t* z, int32_t* slot, uint64_t* code) {
  Forest* f = static_cast<Forest*>(h);
  const std::vector<BoxKey> o = f->sorted();
  for (size_t i = 0; i < o.size(); ++i) {
    J[i] = o[i].J;
    x[i] = o[i].x;
    y[i] = o[i].y;
    z[i] = o[i].z;
    slot[i] = f->leaves.get(o[i]);
    code[i] = f->treecode(o[i]);
  }
}

int hf_is_graded(void* h) { return static_cast<Forest*>(h)->is_graded() ? 1 : 0; }
int hf_tiles_domain(void* h) { return static_cast<Forest*>(h)->tiles_domain() ? 1 : 0; }

// 56 neighbour slots and 26 relative levels of every leaf, in ascending key order.
void hf_neighbour_table(void* h, int32_t* nbr, int8_t* rel) {
  Forest* f = static_cast<Forest*>(h);
  f->neighbour_table(f->sorted(), nbr, rel);
}

// A standalone leaf map: put / erase / get, for the map's own checks.
void* hm_create(int64_t max_entries) {
  acm::LeafMap* m = new acm::LeafMap();
  m->init(max_entries);
  return m;
}
void hm_destroy(void* h) { delete static_cast<acm::LeafMap*>(h); }
void hm_put(void* h, int32_t J, int32_t x, int32_t y, int32_t z, int32_t s) {
  static_cast<acm::LeafMap*>(h)->put(BoxKey{J, x, y, z}, s);
}
int hm_erase(void* h, int32_t J, int32_t x, int32_t y, int32_t z) {
  return static_cast<acm::LeafMap*>(h)->erase(BoxKey{J, x, y, z}) ? 1 : 0;
}
int32_t hm_get(void* h, int32_t J, int32_t x, int32_t y, int32_t z) {
  return static_cast<acm::LeafMap*>(h)->get(BoxKey{J, x, y, z});
}
int64_t hm_size(void* h) { return (int64_t)static_cast<acm::LeafMap*>(h)->size(); }

}  // extern "C"
