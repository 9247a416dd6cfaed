// occ_layout.h -- device data layouts shared by the host BVH builder and the kernels.
#pragma once

#include <cstdint>
#include <vector_types.h>

namespace occ {

// ---------------------------------------------------------------------------------------
// BVH layout.  A node of width W (4 or 8, OCC_BVH_WIDTH) is W/4 cache lines: the bounds
// of its (up to) W children in structure-of-arrays form -- planes lox, hix, loy, hiy,
// loz, hiz, each W/4 float4 -- then W/4 uint4 of packed child references.
//   internal child : node index (bit 31 clear)
//   leaf child     : bit 31 | (count - 1) << 26 | first triangle (count <= 32)
//   empty slot     : kEmptyRef with an empty box
// Plane p (0..5) of children 4h .. 4h + 3 is float4 p * W/4 + h; the far plane of an axis
// is the near one's index xor W/4.
// Triangles: three float4 per triangle in leaf order; v0.w holds the input id.
// ---------------------------------------------------------------------------------------
#ifndef OCC_BVH_WIDTH
#define OCC_BVH_WIDTH 4
#endif
constexpr int kWidth = OCC_BVH_WIDTH;
constexpr int kPlaneVecs = kWidth / 4;
static_assert(kWidth == 4 || kWidth == 8, "BVH width must be 4 or 8");

// ---------------------------------------------------------------------------------------
// Compressed 8-wide layout (OCC_BVH_CW8=1), after the compressed wide BVH of Ylitie, Karras
// and Laine ("Efficient Incoherent Ray Traversal on GPUs Through Compressed Wide BVHs",
// HPG 2017): an 80-byte node holds 8 child boxes quantised to 8 bits per plane on a grid
// anchored at the node (origin p, per-axis power-of-two step 2^(e - 127)), its internal
// children stored contiguously from child_base in slot order, the triangles of its leaf
// children (at most 3 each, 24 per node) contiguously from tri_base.
//   float4 0: p.x, p.y, p.z, bytes (e_x, e_y, e_z, imask: bit s = slot s is internal)
//   float4 1: child_base, tri_base, meta[0..3], meta[4..7]
//             meta of an internal child: 0x20 | (24 + s); of a leaf child:
//             (unary triangle count: 1, 3 or 7) << 5 | offset from tri_base; empty slot: 0
//   float4 2: lo_x[0..7], lo_y[0..7]      (bytes, child s in byte s)
//   float4 3: lo_z[0..7], hi_x[0..7]
//   float4 4: hi_y[0..7], hi_z[0..7]
// Every box is widened by one grid step on each side beyond its conservative rounding, so
// that the traversal may evaluate each plane as one FMA of the biased byte value (see
// occ_device.cuh).  Empty slots hold the inverted box lo = 255, hi = 0.
// ---------------------------------------------------------------------------------------
#ifndef OCC_BVH_CW8
#define OCC_BVH_CW8 0
#endif

struct __align__(16) BvhNodeCW {
    float4 v[5];
};
static_assert(sizeof(BvhNodeCW) == 80, "a compressed node is 80 bytes");
constexpr int kCwMaxLeafTris = 3;

struct __align__(16) BvhNode4 {
    float4 plane[6 * kPlaneVecs];
    uint4 child[kPlaneVecs];
    uint4 pad[kPlaneVecs];
};
static_assert(sizeof(BvhNode4) == 128 * kPlaneVecs, "a node is W/4 cache lines");

#if OCC_BVH_CW8
using BvhNode = BvhNodeCW;
#else
using BvhNode = BvhNode4;
#endif

constexpr uint32_t kEmptyRef = 0x7FFFFFFFu;
constexpr uint32_t kLeafBit = 0x80000000u;
static_assert((kEmptyRef & kLeafBit) == 0 && kEmptyRef == kLeafBit - 1u,
              "internal references lie below kEmptyRef and leaf references above it");
constexpr int kLeafCountShift = 26;
constexpr uint32_t kLeafFirstMask = (1u << kLeafCountShift) - 1u;
constexpr int kMaxLeafTris = 32;
// stack entries: node references (uncompressed layouts), or node groups (compressed: one
// entry per tree level at most)
constexpr int kStackSize = OCC_BVH_CW8 ? 32 : (kWidth == 8 ? 96 : 64);
constexpr uint32_t kNoHit = 0xFFFFFFFFu;

// Device status word bits (set by kernels, read back and cleared by occ_sync).
constexpr uint32_t kStatusStackOverflowBit = 1u << 0;
constexpr uint32_t kStatusWaitTimeoutBit = 1u << 1;
constexpr uint32_t kStatusBadIndexBit = 1u << 2;

// OCC_COUNTERS=1 (the "counters" library variant): every node visit and triangle test of
// the traversal is counted, and the distinct nodes and triangles touched are marked in
// bitmaps, so that the bytes a launch must read from the BVH can be measured.  The product
// library is built without it.
#ifndef OCC_COUNTERS
#define OCC_COUNTERS 0
#endif

struct DevBVH {
    const BvhNode* nodes;
    const float4* tris;
    uint32_t n_nodes = 0, n_tris = 0;   // bounds the OCC_CHECKS build verifies
#if OCC_COUNTERS
    unsigned long long* ctr = nullptr;   // [0] node visits, [1] triangle tests
    uint32_t* node_bits = nullptr;       // one bit per node touched
    uint32_t* tri_bits = nullptr;        // one bit per triangle slot touched
#endif
};

// OCC_CHECKS=1: the traversal checks every node and triangle index it follows against the
// BVH's sizes; a bad one sets kStatusBadIndexBit and ends that ray (no trap).
#ifndef OCC_CHECKS
#define OCC_CHECKS 0
#endif

}  // namespace occ
