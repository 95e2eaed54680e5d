// Device-side topology of libacm: the neighbourhood table of every block, the fine-wins task
// list and the coarse-face slab list, built on the GPU from the block list alone.
//
// Paper, Sec. 4.1: blocks are located through their treecodes and the neighbours of a block are
// found from its own coordinates (no pointers between blocks).  Here the leaves are first put
// into a device hash table (box -> slot; the table stores slots and keys are read back through
// a slot-indexed box array), then every (block, neighbour box) pair is one thread that resolves
// the box the way the host tree does (leaf, else coarser leaf, else refined into leaves).
#include "common.cuh"
#include "kernels.hpp"

namespace acm {

namespace {

__constant__ int kFaceBoxT[6] = {12, 14, 10, 16, 4, 22};

// Insert every leaf (rank r: box binfo[r], slot blist[r]) into the table (all entries -1 before)
// and record its box by slot.  Linear probing with compare-and-swap on the slot word.
__global__ void __launch_bounds__(256) k_index(TreeK t, const int4* binfo, const int32_t* blist, int64_t n,
                                               int* tab, int4* box, int* err) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int4 b = binfo[r];
  const int s = blist[r];
  box[s] = b;
  size_t i = (size_t)(leaf_hash(b.x, b.y, b.z, b.w) & t.mask);
  for (unsigned long long k = 0; k <= t.mask; ++k) {
    if (atomicCAS(tab + i, -1, s) == -1) return;
    i = (i + 1) & (size_t)t.mask;
  }
  atomicOr(err, 4);
}

// Periodic wrap of a neighbour coordinate (within one box of the range: no division).
__device__ __forceinline__ int wrap_axis(long long v, long long n) {
  if (v < 0) v += n;
  else if (v >= n) v -= n;
  return (int)v;
}

// Status of the level-J box (x, y, z) (unwrapped) as seen from a neighbour: a leaf, covered by a
// leaf one level coarser (octant = which half per axis), or refined into level J+1 leaves.
struct DevStatus {
  int type;          // kTypeLeaf, kTypeCoarser, kTypeRefined, kTypeNone
  int octant;
  int slot[8];
};

// The box itself, its parent and its 8 children are looked up together: the first probe of each
// of the 10 keys is issued at once (independent loads), and only a key whose first table entry
// belongs to another box continues probing.  The answer is the host tree's: leaf, else coarser
// leaf, else refined.
__device__ DevStatus box_status_dev(const TreeK& t, int J, long long x, long long y, long long z, int* err) {
  DevStatus st;
  st.type = kTypeNone;
  st.octant = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) st.slot[c] = -1;
  const int kx = wrap_axis(x, (long long)t.nroot[0] << J);
  const int ky = wrap_axis(y, (long long)t.nroot[1] << J);
  const int kz = wrap_axis(z, (long long)t.nroot[2] << J);
  int4 key[10];
  key[0] = make_int4(J, kx, ky, kz);
  key[1] = make_int4(J - 1, kx >> 1, ky >> 1, kz >> 1);      // only meaningful for J > 0
#pragma unroll
  for (int c = 0; c < 8; ++c) key[2 + c] = make_int4(J + 1, 2 * kx + (c & 1), 2 * ky + ((c >> 1) & 1), 2 * kz + ((c >> 2) & 1));
  size_t pos[10];
  int s[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    pos[q] = (size_t)(leaf_hash(key[q].x, key[q].y, key[q].z, key[q].w) & t.mask);
    s[q] = (q == 1 && J == 0) ? -1 : t.tab[pos[q]];
  }
  int4 kb[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) kb[q] = s[q] >= 0 ? t.box[s[q]] : make_int4(-1, 0, 0, 0);
  int res[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    if (s[q] < 0) {
      res[q] = -1;
    } else if (kb[q].x == key[q].x && kb[q].y == key[q].y && kb[q].z == key[q].z && kb[q].w == key[q].w) {
      res[q] = s[q];
    } else {
      // the first entry holds another box: continue the probe sequence
      res[q] = -1;
      size_t i = (pos[q] + 1) & (size_t)t.mask;
      unsigned long long n = 1;
      for (; n <= t.mask; ++n) {
        const int e = t.tab[i];
        if (e < 0) break;
        const int4 k = t.box[e];
        if (k.x == key[q].x && k.y == key[q].y && k.z == key[q].z && k.w == key[q].w) {
          res[q] = e;
          break;
        }
        i = (i + 1) & (size_t)t.mask;
      }
      if (n > t.mask) atomicOr(err, 4);
    }
  }
  if (res[0] >= 0) {
    st.type = kTypeLeaf;
    st.slot[0] = res[0];
    return st;
  }
  if (J > 0 && res[1] >= 0) {
    st.type = kTypeCoarser;
    st.slot[0] = res[1];
    st.octant = (kx & 1) | ((ky & 1) << 1) | ((kz & 1) << 2);
    return st;
  }
  bool any = false;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    st.slot[c] = res[2 + c];
    any = any || res[2 + c] >= 0;
  }
  if (any) st.type = kTypeRefined;
  return st;
}

// One warp per block (rank), lane d < 27 = neighbour box d.  Writes the block's neighbourhood
// row, whether a neighbour box is refined (finer), the mask of refined boxes (fine-wins tasks)
// and of faces covered by a coarser leaf (halo slabs).  A box that is missing, or refined with
// a touching child missing, breaks the 2:1 grading the kernels rely on: error flag bit 2.
__global__ void __launch_bounds__(256) k_rows(TreeK t, const int4* binfo, int64_t n, int32_t* nbh,
                                              uint8_t* finer, uint32_t* fwmask, uint32_t* slabmask, int* err) {
  const int64_t rank = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (rank >= n) return;
  const int4 b = binfo[rank];
  int32_t* row = nbh + rank * kNbhStride;
  int type = kTypeNone;
  if (lane < 27) {
    const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
    const DevStatus st = box_status_dev(t, b.x, (long long)b.y + dx, (long long)b.z + dy, (long long)b.w + dz, err);
    bool bad = st.type == kTypeNone;
    if (st.type == kTypeRefined) {
      // every child touching the block must be a leaf (kernels index these slots)
      const int dd[3] = {dx, dy, dz};
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        bool touch = true;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int cq = (c >> q) & 1;
          if ((dd[q] == 1 && cq != 0) || (dd[q] == -1 && cq != 1)) touch = false;
        }
        if (touch && st.slot[c] < 0) bad = true;
      }
    }
    if (bad) atomicOr(err, 2);
#pragma unroll
    for (int c = 0; c < 8; ++c) row[8 * lane + c] = st.type == kTypeNone ? -1 : st.slot[c];
    row[kNbhType + lane] = st.type == kTypeNone ? -1 : (st.type | (st.octant << 4));
    type = st.type;
  } else {
    for (int e = kNbhType + 27 + (lane - 27); e < kNbhStride; e += 5) row[e] = -1;
  }
  const unsigned refined = __ballot_sync(0xffffffffu, lane < 27 && lane != 13 && type == kTypeRefined);
  const unsigned coarser = __ballot_sync(0xffffffffu, lane < 27 && type == kTypeCoarser);
  if (lane == 0) {
    unsigned faces = 0;
#pragma unroll
    for (int F = 0; F < 6; ++F)
      if ((coarser >> kFaceBoxT[F]) & 1u) faces |= 1u << F;
    finer[rank] = refined != 0;
    fwmask[rank] = refined;
    slabmask[rank] = faces;
  }
}

// Exclusive prefix sums of the per-block task counts (one CTA; each thread scans a contiguous
// chunk); counts[0] = fine-wins tasks, counts[1] = slabs.
constexpr int kScanNT = 1024;
__global__ void __launch_bounds__(kScanNT) k_scan(const uint32_t* fwmask, const uint32_t* slabmask, int64_t n,
                                                  int32_t* fw_off, int32_t* slab_off, int32_t* counts) {
  __shared__ int32_t sa[kScanNT], sb[kScanNT];
  const int tid = threadIdx.x;
  const int64_t per = (n + kScanNT - 1) / kScanNT;
  const int64_t lo = tid * per, hi = lo + per < n ? lo + per : n;
  int32_t a = 0, b = 0;
  for (int64_t r = lo; r < hi; ++r) {
    a += __popc(fwmask[r]);
    b += __popc(slabmask[r]);
  }
  sa[tid] = a;
  sb[tid] = b;
  __syncthreads();
  // Hillis-Steele inclusive scan of the chunk sums
  for (int o = 1; o < kScanNT; o <<= 1) {
    const int32_t va = tid >= o ? sa[tid - o] : 0, vb = tid >= o ? sb[tid - o] : 0;
    __syncthreads();
    sa[tid] += va;
    sb[tid] += vb;
    __syncthreads();
  }
  int32_t oa = sa[tid] - a, ob = sb[tid] - b;
  for (int64_t r = lo; r < hi; ++r) {
    fw_off[r] = oa;
    slab_off[r] = ob;
    oa += __popc(fwmask[r]);
    ob += __popc(slabmask[r]);
  }
  if (tid == kScanNT - 1) {
    counts[0] = sa[tid];
    counts[1] = sb[tid];
  }
}

// Task lists in block order, then ascending box index / face: fine-wins task (rank, d) per refined
// neighbour box; slab (rank, face, index) per face covered by a coarser leaf, and the block's
// slab index per face (-1: none).
__global__ void __launch_bounds__(256) k_fill(const uint32_t* fwmask, const uint32_t* slabmask, const int32_t* fw_off,
                                              const int32_t* slab_off, int64_t n, int2* fw, int4* slabt,
                                              int32_t* slabidx) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint32_t m = fwmask[r];
  int j = fw_off[r];
  for (int d = 0; d < 27; ++d)
    if ((m >> d) & 1u) fw[j++] = make_int2((int)r, d);
  const uint32_t sm = slabmask[r];
  int k = slab_off[r];
  for (int F = 0; F < 8; ++F) {
    int idx = -1;
    if (F < 6 && ((sm >> F) & 1u)) {
      idx = k++;
      slabt[idx] = make_int4((int)r, F, idx, 0);
    }
    slabidx[r * 8 + F] = idx;
  }
}

}  // namespace

void launch_topology(const TreeK& t, int* tab, int4* box, const int4* binfo, const int32_t* blist, int64_t n,
                     int32_t* nbh, uint8_t* finer, uint32_t* fwmask, uint32_t* slabmask, int32_t* fw_off,
                     int32_t* slab_off, int32_t* counts, int2* fw, int4* slabt, int32_t* slabidx, int* err,
                     cudaStream_t st) {
  cudaMemsetAsync(tab, 0xff, (size_t)(t.mask + 1) * sizeof(int), st);
  if (n <= 0) {
    cudaMemsetAsync(counts, 0, 2 * sizeof(int32_t), st);
    return;
  }
  k_index<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(t, binfo, blist, n, tab, box, err);
  k_rows<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(t, binfo, n, nbh, finer, fwmask, slabmask, err);
  k_scan<<<1, kScanNT, 0, st>>>(fwmask, slabmask, n, fw_off, slab_off, counts);
  k_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(fwmask, slabmask, fw_off, slab_off, n, fw, slabt, slabidx);
}

}  // namespace acm

namespace acm {

int sm_count() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

}  // namespace acm
