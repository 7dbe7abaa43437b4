// svo_build.h -- host octree builder (see svo_build.cpp for the node layout).
#pragma once

#include <cstdint>
#include <vector>

#include "svoanim.h"

namespace svo {

struct BuiltOctree {
  int depth = 0;
  uint64_t n_nodes = 0;
  uint64_t n_leaves = 0;
  std::vector<uint32_t> nodes;  // 2 words per node
  std::vector<uint32_t> rgb;    // per leaf, Morton order
  std::vector<uint64_t> level_start;  // first node of each level, 0..depth (the last = n_nodes)
  uint32_t box_lo[3] = {0, 0, 0};  // occupied cells: min corner (inclusive)
  uint32_t box_hi[3] = {0, 0, 0};  // ... max corner + 1 (0 when empty)
};

// Returns SVO_OK or an svo_status error code.
int build_octree(int depth, uint64_t n, const uint64_t *ids, const uint32_t *rgb, BuiltOctree *out);

}  // namespace svo
