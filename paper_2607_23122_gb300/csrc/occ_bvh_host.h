// occ_bvh_host.h -- host-side result of the BVH builder.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>

#include "occ_layout.h"

namespace occ {

struct HostBVH {
    std::vector<BvhNode> nodes;   // root at index 0
    std::vector<float4> tris;     // 3 per triangle, leaf order, v0.w = input id bits
    int64_t num_leaves = 0;
    int depth = 0;
    int max_leaf_tris = 0;
};

// Builds the kWidth-wide BVH of T triangles (tris: [T][3][3] floats).  Returns false with
// a message for invalid input or a tree too deep for the traversal stack.
bool build_bvh4(const float* tris, int64_t T, HostBVH* out, std::string* err);

}  // namespace occ
