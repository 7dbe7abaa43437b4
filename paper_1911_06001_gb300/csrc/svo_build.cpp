// svo_build.cpp -- host construction of the octree node layout from a leaf list.
//
// Layout (a simplified Laine-Karras child-descriptor structure, as the paper
// uses, Sec. II-B and V; the bit layout is this library's own):
//   node  = 8 bytes: uint32 first_child | uint8 child_mask | uint8 leaf_mask | uint16 0
//   order = breadth first (all level-0 nodes, then level 1, ...), root at 0;
//           within a level, nodes ascend in Morton order, so the children of
//           a node are contiguous and in ascending octant order.
//   child k of a node is at first_child + popcount(child_mask & ((1<<k)-1)).
//   octant bits: bit0 = +x half, bit1 = +y half, bit2 = +z half.
//   Level D-1 nodes have leaf children: leaf_mask == child_mask and
//   first_child indexes the leaf payload (0x00RRGGBB, Morton order).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "svo_build.h"

namespace svo {

static inline uint64_t spread3(uint64_t v) {
  // insert two zero bits between consecutive bits of a 16-bit value
  v &= 0xFFFFull;
  v = (v | (v << 16)) & 0x0000FF0000FFull;
  v = (v | (v << 8)) & 0x00F00F00F00Full;
  v = (v | (v << 4)) & 0x0C30C30C30C3ull;
  v = (v | (v << 2)) & 0x249249249249ull;
  return v;
}

static void radix_sort_pairs(std::vector<uint64_t> &key, std::vector<uint32_t> &val, int bits) {
  const size_t n = key.size();
  std::vector<uint64_t> k2(n);
  std::vector<uint32_t> v2(n);
  for (int shift = 0; shift < bits; shift += 8) {
    size_t count[257] = {0};
    for (size_t i = 0; i < n; ++i) ++count[((key[i] >> shift) & 0xFF) + 1];
    for (int b = 0; b < 256; ++b) count[b + 1] += count[b];
    for (size_t i = 0; i < n; ++i) {
      size_t dst = count[(key[i] >> shift) & 0xFF]++;
      k2[dst] = key[i];
      v2[dst] = val[i];
    }
    key.swap(k2);
    val.swap(v2);
  }
}

int build_octree(int depth, uint64_t n_in, const uint64_t *ids, const uint32_t *rgb_in, BuiltOctree *out) {
  if (depth < 1 || depth > SVO_MAX_DEPTH) return SVO_ERR_ARG;
  if (n_in > 0 && ids == nullptr) return SVO_ERR_ARG;
  if (n_in >= (1ull << 32)) return SVO_ERR_LIMIT;
  const uint64_t mask = (1ull << depth) - 1ull;
  std::vector<uint64_t> code(n_in);
  std::vector<uint32_t> src(n_in);
  uint64_t lo[3] = {mask, mask, mask}, hi[3] = {0, 0, 0};
  for (uint64_t i = 0; i < n_in; ++i) {
    uint64_t v = ids[i];
    uint64_t x = v & mask, y = (v >> depth) & mask, z = (v >> (2 * depth)) & mask;
    if ((v >> (3 * depth)) != 0) return SVO_ERR_ARG;  // coordinates out of range
    lo[0] = x < lo[0] ? x : lo[0];
    lo[1] = y < lo[1] ? y : lo[1];
    lo[2] = z < lo[2] ? z : lo[2];
    hi[0] = x > hi[0] ? x : hi[0];
    hi[1] = y > hi[1] ? y : hi[1];
    hi[2] = z > hi[2] ? z : hi[2];
    code[i] = spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
    src[i] = (uint32_t)i;
  }
  radix_sort_pairs(code, src, 3 * depth);
  // unique leaves (the first entry of equal codes supplies the colour)
  std::vector<uint64_t> lev;  // codes of the current level
  lev.reserve(n_in);
  out->rgb.clear();
  out->rgb.reserve(n_in);
  for (uint64_t i = 0; i < n_in; ++i) {
    if (i > 0 && code[i] == code[i - 1]) continue;
    lev.push_back(code[i]);
    out->rgb.push_back(rgb_in ? rgb_in[src[i]] : 0u);
  }
  out->n_leaves = lev.size();
  out->depth = depth;
  for (int k = 0; k < 3; ++k) {
    out->box_lo[k] = n_in ? (uint32_t)lo[k] : 0u;
    out->box_hi[k] = n_in ? (uint32_t)hi[k] + 1u : 0u;
  }
  // bottom-up: level l nodes are the distinct prefixes code >> 3 of level l+1
  std::vector<std::vector<uint32_t>> first(depth), cmask(depth);
  std::vector<size_t> count(depth + 1, 0);
  count[depth] = lev.size();
  for (int l = depth - 1; l >= 0; --l) {
    std::vector<uint64_t> up;
    up.reserve(lev.size() / 2 + 1);
    for (size_t i = 0; i < lev.size(); ++i) {
      uint64_t p = lev[i] >> 3;
      uint32_t bit = 1u << (lev[i] & 7);
      if (up.empty() || up.back() != p) {
        up.push_back(p);
        first[l].push_back((uint32_t)i);
        cmask[l].push_back(bit);
      } else {
        cmask[l].back() |= bit;
      }
    }
    count[l] = up.size();
    lev.swap(up);
  }
  // breadth-first offsets
  std::vector<uint64_t> offset(depth + 1, 0);
  for (int l = 0; l < depth; ++l) offset[l + 1] = offset[l] + count[l];
  const uint64_t n_nodes = offset[depth];
  if (n_nodes >= (1ull << 32)) return SVO_ERR_LIMIT;
  out->nodes.assign(2 * n_nodes, 0u);
  for (int l = 0; l < depth; ++l) {
    for (size_t j = 0; j < count[l]; ++j) {
      uint64_t idx = offset[l] + j;
      uint32_t fc = first[l][j];
      uint32_t cm = cmask[l][j];
      uint32_t fchild = (l + 1 < depth) ? (uint32_t)(offset[l + 1] + fc) : fc;
      uint32_t lm = (l == depth - 1) ? cm : 0u;
      out->nodes[2 * idx] = fchild;
      out->nodes[2 * idx + 1] = cm | (lm << 8);
    }
  }
  out->n_nodes = n_nodes;
  out->level_start = offset;
  return SVO_OK;
}

}  // namespace svo
