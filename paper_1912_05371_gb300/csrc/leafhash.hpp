// Leaf-map entry and box hash, shared by the host tree (forest.cpp) and the device leaf table of
// the topology kernels (topo.cu).
#pragma once

#include <cstdint>
#include <cstddef>

#if defined(__CUDACC__)
#define ACM_HD __host__ __device__ __forceinline__
#else
#define ACM_HD inline
#endif

namespace acm {

// Box (J, x, y, z) -> slot of the leaf occupying it; slot -1 marks an empty table entry.
struct LeafEntry {
  int32_t J, x, y, z;
  int32_t slot;
};
static_assert(sizeof(LeafEntry) == 20, "LeafEntry must be 5 packed int32");

// Combine the four coordinates, then mix all bits into the low ones (the 64-bit finaliser of
// MurmurHash3): tables index with the low bits, and without the final mixing neighbouring boxes
// fall into long runs of occupied entries under linear probing.
ACM_HD uint64_t leaf_hash(int32_t J, int32_t x, int32_t y, int32_t z) {
  uint64_t h = (uint64_t)(uint32_t)J * 0x9E3779B97F4A7C15ull;
  h ^= (uint64_t)(uint32_t)x + 0x7F4A7C159E3779B9ull + (h << 6) + (h >> 2);
  h ^= (uint64_t)(uint32_t)y + 0x94D049BB133111EBull + (h << 6) + (h >> 2);
  h ^= (uint64_t)(uint32_t)z + 0xBF58476D1CE4E5B9ull + (h << 6) + (h >> 2);
  h ^= h >> 33;
  h *= 0xff51afd7ed558ccdull;
  h ^= h >> 33;
  h *= 0xc4ceb9fe1a85ec53ull;
  h ^= h >> 33;
  return h;
}

}  // namespace acm
