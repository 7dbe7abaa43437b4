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
};

// Returns SVO_OK or an svo_status error code.
int build_octree(int depth, uint64_t n, const uint64_t *ids, const uint32_t *rgb, BuiltOctree *out);

}  // namespace svo
