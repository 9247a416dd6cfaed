// occ_layout.h -- device data layouts shared by the host BVH builder and the kernels.
#pragma once

#include <cstdint>
#include <vector_types.h>

namespace occ {

// ---------------------------------------------------------------------------------------
// BVH layout.  One node = 128 bytes: the bounds of its (up to) four children in
// structure-of-arrays form, then four packed child references.
//   internal child : node index (bit 31 clear)
//   leaf child     : bit 31 | (count - 1) << 26 | first triangle (count <= 32)
//   empty slot     : kEmptyRef with an empty box
// Triangles: three float4 per triangle in leaf order; v0.w holds the input id.
// ---------------------------------------------------------------------------------------
struct __align__(16) Node4 {
    float4 lox, hix, loy, hiy, loz, hiz;
    uint4 child;
    uint4 pad;
};
static_assert(sizeof(Node4) == 128, "Node4 must be 128 bytes");

constexpr uint32_t kEmptyRef = 0x7FFFFFFFu;
constexpr uint32_t kLeafBit = 0x80000000u;
constexpr int kLeafCountShift = 26;
constexpr uint32_t kLeafFirstMask = (1u << kLeafCountShift) - 1u;
constexpr int kMaxLeafTris = 32;
constexpr int kStackSize = 64;
constexpr uint32_t kNoHit = 0xFFFFFFFFu;

// Device status word bits (set by kernels, read back and cleared by occ_sync).
constexpr uint32_t kStatusStackOverflowBit = 1u << 0;
constexpr uint32_t kStatusWaitTimeoutBit = 1u << 1;
constexpr uint32_t kStatusBadIndexBit = 1u << 2;

struct DevBVH {
    const Node4* nodes;
    const float4* tris;
};

}  // namespace occ
