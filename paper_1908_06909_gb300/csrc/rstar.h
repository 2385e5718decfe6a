// rstar.h -- R*-tree over the boundary faces (the paper's entry structure).
//
// The paper accelerates the entry search with an R*-tree of the boundary
// elements, at least 4 and at most 10 children per node, searched depth-first
// (Sec. II-E).  This build's default entry structure is a binary BVH; the
// R*-tree is built on request for the comparison (TETPROJ_FLAG_RSTAR_ENTRY).
//
// Device layout (RStarNode, tetproj_internal.h): nodes of up to RSTAR_MAX
// entries, boxes stored structure-of-arrays inside the node.
#pragma once

#include <stdint.h>

#include <vector>

#include "tetproj_internal.h"

namespace tp {

struct RStarStats {
    int64_t nodes = 0, leaves = 0, entries = 0;
    int32_t depth = 0;
    int32_t min_fill = 0, max_fill = 0;
    int32_t ok = 0;  // 1: every invariant holds (see rstar_check)
};

// Builds the tree by one-at-a-time R* insertion of the boxes of `faces`
// (FP32 vertex boxes); node 0 is the root.
void rstar_build(const std::vector<BFace32> &faces, std::vector<RStarNode> &nodes);

// Checks: non-root nodes hold RSTAR_MIN..RSTAR_MAX entries (root >= 2 unless it
// is a leaf), all leaves at one depth, every box contains its subtree, every
// face appears in exactly one leaf.
RStarStats rstar_check(const std::vector<BFace32> &faces, const std::vector<RStarNode> &nodes);

}  // namespace tp
