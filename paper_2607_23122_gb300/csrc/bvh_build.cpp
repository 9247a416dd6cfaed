// bvh_build.cpp -- host construction of the wide BVH (4 or 8 children per node,
// OCC_BVH_WIDTH) used by the traversal kernels.
//
// A binary BVH is built top-down with binned SAH (128 bins per axis over the
// centroid bounds; the top levels run in parallel threads), then collapsed into
// wide nodes by a dynamic program over the surface-area cost (SahCollapser; the greedy
// collapse that opens the child with the largest surface area remains as Collapser).
// Leaves keep their triangles contiguous, so the triangle array is stored in leaf
// order as three float4 per triangle with the input id in v0.w.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <future>
#include <limits>
#include <thread>
#include <vector>

#include <vector_functions.h>
#include <vector_types.h>

#include "occ_bvh_host.h"
#include "occ_layout.h"

namespace occ {
namespace {

struct AABB {
    float lo[3], hi[3];
    AABB() {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::numeric_limits<float>::infinity();
            hi[a] = -std::numeric_limits<float>::infinity();
        }
    }
    void grow(const AABB& b) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
        }
    }
    void grow(const float* p) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], p[a]);
            hi[a] = std::max(hi[a], p[a]);
        }
    }
    bool empty() const { return lo[0] > hi[0]; }
    float area() const {
        if (empty()) return 0.0f;
        const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0f * (dx * dy + dy * dz + dz * dx);
    }
};

struct BNode {
    AABB box;
    int32_t left = -1, right = -1;   // children (internal)
    uint32_t first = 0, count = 0;   // leaf range in the permutation
};

// Bins per axis and the traversal cost (in triangle tests) of the SAH.  1080p AO trace on
// the 1M-triangle terrain: 16 bins and cost 1.2, 0.371 ms; 32 bins and 0.8, 0.359 ms;
// 128 bins and 0.8, 0.354 ms (256 bins, costs 0.6 / 1.0 / 1.2 and leaves of 4 or 6 were
// no better); the shadow trace stays at 0.265 ms.
#ifndef OCC_SAH_BINS
#define OCC_SAH_BINS 128
#endif
constexpr int kBins = OCC_SAH_BINS;
#ifndef OCC_SAH_TRAVERSE
#define OCC_SAH_TRAVERSE 0.8f
#endif
#ifndef OCC_SAH_LEAFMAX
#define OCC_SAH_LEAFMAX 8
#endif
constexpr float kTraverseCost = OCC_SAH_TRAVERSE;
constexpr float kIntersectCost = 1.0f;
constexpr uint32_t kLeafMax = OCC_SAH_LEAFMAX;   // never keep a leaf bigger than this
constexpr uint32_t kParallelMin = 1u << 15;

struct Builder {
    const std::vector<AABB>& tb;           // triangle bounds
    const std::vector<std::array<float, 3>>& tc;   // centroids
    std::vector<uint32_t>& perm;
    uint32_t leaf_max = kLeafMax;          // never keep a leaf bigger than this

    // Builds the subtree of perm[begin, end) into `out` (root at out[base]) and returns the
    // index of its root.
    int32_t build(std::vector<BNode>& out, uint32_t begin, uint32_t end, int spawn_depth) {
        const int32_t me = (int32_t)out.size();
        out.emplace_back();
        AABB box, cbox;
        for (uint32_t i = begin; i < end; ++i) {
            box.grow(tb[perm[i]]);
            cbox.grow(tc[perm[i]].data());
        }
        out[me].box = box;
        const uint32_t n = end - begin;
        auto make_leaf = [&]() {
            out[me].first = begin;
            out[me].count = n;
            return me;
        };
        if (n <= 1) return make_leaf();

        int best_axis = -1, best_bin = -1;
        float best_cost = std::numeric_limits<float>::infinity();
        for (int a = 0; a < 3; ++a) {
            const float ext = cbox.hi[a] - cbox.lo[a];
            if (!(ext > 0.0f)) continue;
            AABB bb[kBins];
            uint32_t bc[kBins] = {0};
            const float k = kBins * (1.0f - 1e-6f) / ext;
            for (uint32_t i = begin; i < end; ++i) {
                int b = (int)((tc[perm[i]][a] - cbox.lo[a]) * k);
                b = std::min(std::max(b, 0), kBins - 1);
                bb[b].grow(tb[perm[i]]);
                ++bc[b];
            }
            AABB racc;
            float rarea[kBins];
            uint32_t rcnt[kBins];
            uint32_t acc = 0;
            for (int b = kBins - 1; b > 0; --b) {
                racc.grow(bb[b]);
                acc += bc[b];
                rarea[b] = racc.area();
                rcnt[b] = acc;
            }
            AABB lacc;
            uint32_t lcnt = 0;
            for (int b = 0; b < kBins - 1; ++b) {
                lacc.grow(bb[b]);
                lcnt += bc[b];
                if (lcnt == 0 || rcnt[b + 1] == 0) continue;
                const float c = lacc.area() * lcnt + rarea[b + 1] * rcnt[b + 1];
                if (c < best_cost) {
                    best_cost = c;
                    best_axis = a;
                    best_bin = b;
                }
            }
        }
        const float parea = box.area();
        const float split_cost =
            kTraverseCost + kIntersectCost * best_cost / (parea > 0.0f ? parea : 1.0f);
        const float leaf_cost = kIntersectCost * n;
        // small ranges become leaves when SAH does not favour a split; larger ones always split
        if (n <= leaf_max && (best_axis < 0 || split_cost >= leaf_cost)) return make_leaf();
        uint32_t mid;
        if (best_axis < 0) {
            mid = begin + n / 2;   // all centroids coincide: split the range
        } else {
            const float ext = cbox.hi[best_axis] - cbox.lo[best_axis];
            const float k = kBins * (1.0f - 1e-6f) / ext;
            auto it = std::partition(perm.begin() + begin, perm.begin() + end, [&](uint32_t t) {
                int b = (int)((tc[t][best_axis] - cbox.lo[best_axis]) * k);
                b = std::min(std::max(b, 0), kBins - 1);
                return b <= best_bin;
            });
            mid = (uint32_t)(it - perm.begin());
            if (mid == begin || mid == end) mid = begin + n / 2;
        }
        if (spawn_depth > 0 && n >= kParallelMin) {
            std::vector<BNode> lv, rv;
            auto fut = std::async(std::launch::async, [&]() { build(lv, begin, mid, spawn_depth - 1); });
            build(rv, mid, end, spawn_depth - 1);
            fut.get();
            const int32_t lbase = (int32_t)out.size();
            append(out, lv, lbase);
            const int32_t rbase = (int32_t)out.size();
            append(out, rv, rbase);
            out[me].left = lbase;
            out[me].right = rbase;
        } else {
            const int32_t l = build(out, begin, mid, 0);
            const int32_t r = build(out, mid, end, 0);
            out[me].left = l;
            out[me].right = r;
        }
        return me;
    }

    static void append(std::vector<BNode>& out, const std::vector<BNode>& sub, int32_t base) {
        for (const BNode& b : sub) {
            BNode c = b;
            if (c.left >= 0) {
                c.left += base;
                c.right += base;
            }
            out.push_back(c);
        }
    }
};

// Component c (child index) of plane p of a node.
#if !OCC_BVH_CW8
inline float& plane_at(BvhNode& n, int p, int c) {
    float4& v = n.plane[p * kPlaneVecs + c / 4];
    return (&v.x)[c % 4];
}

inline void set_child(BvhNode& n, int c, uint32_t ref) {
    uint4& v = n.child[c / 4];
    (&v.x)[c % 4] = ref;
}

// An empty node: every child slot empty (inverted box, kEmptyRef).
inline BvhNode empty_node() {
    BvhNode n;
    std::memset(&n, 0, sizeof(n));
    const float inf = std::numeric_limits<float>::infinity();
    for (int c = 0; c < kWidth; ++c) {
        for (int a = 0; a < 3; ++a) {
            plane_at(n, 2 * a, c) = inf;
            plane_at(n, 2 * a + 1, c) = -inf;
        }
        set_child(n, c, kEmptyRef);
    }
    return n;
}

struct Collapser {
    const std::vector<BNode>& bn;
    std::vector<BvhNode>& nodes;
    float pad;          // absolute growth of every child box (see build_bvh4)
    int max_depth = 0;
    int64_t leaves = 0;
    uint32_t max_leaf = 0;

    static uint32_t leaf_ref(const BNode& b) {
        return kLeafBit | ((b.count - 1u) << kLeafCountShift) | b.first;
    }

    // Emits the kWidth-wide node standing for binary node `b` (internal) and returns its
    // index: the binary subtree's children are opened largest-area first until kWidth
    // children (or only leaves) remain.
    uint32_t emit(int32_t b, int depth) {
        max_depth = std::max(max_depth, depth);
        std::vector<int32_t> kids = {bn[b].left, bn[b].right};
        while ((int)kids.size() < kWidth) {
            int pick = -1;
            float best = -1.0f;
            for (int i = 0; i < (int)kids.size(); ++i) {
                const BNode& c = bn[kids[i]];
                if (c.left < 0) continue;
                const float a = c.box.area();
                if (a > best) {
                    best = a;
                    pick = i;
                }
            }
            if (pick < 0) break;
            const int32_t open = kids[pick];
            kids[pick] = bn[open].left;
            kids.push_back(bn[open].right);
        }
        const uint32_t me = (uint32_t)nodes.size();
        nodes.push_back(empty_node());
        uint32_t ref[kWidth];
        for (int c = 0; c < (int)kids.size(); ++c) {
            const BNode& k = bn[kids[c]];
            if (k.left < 0) {
                ref[c] = leaf_ref(k);
                ++leaves;
                max_leaf = std::max(max_leaf, k.count);
            } else {
                ref[c] = emit(kids[c], depth + 1);
            }
        }
        BvhNode& n = nodes[me];   // after the recursion: the vector may have moved
        for (int c = 0; c < (int)kids.size(); ++c) {
            const BNode& k = bn[kids[c]];
            for (int a = 0; a < 3; ++a) {
                plane_at(n, 2 * a, c) = k.box.lo[a] - pad;
                plane_at(n, 2 * a + 1, c) = k.box.hi[a] + pad;
            }
            set_child(n, c, ref[c]);
        }
        return me;
    }
};

// SAH-optimal collapse (OCC_COLLAPSE_SAH=1): instead of opening the largest child greedily,
// a dynamic program over the binary tree picks for every wide node the cut of its binary
// subtree into at most kWidth children, and for every subtree whether it becomes a leaf (any
// subtree of at most leaf_cap triangles, whose triangles are contiguous) or a wide node,
// minimising the surface-area cost
//     cost(wide node n) = A(n) c_node + sum over its children of cost(child),
//     cost(leaf m)      = A(m) c_tri count(m).
// With F(n) the best cost of subtree n as one child slot and H(n, k) the best cost of subtree
// n spread over at most k slots:
//     H(n, 1) = F(n),   H(n, k) = min(F(n), min_j H(left, j) + H(right, k - j)),
//     F(n)    = min(leaf cost, A(n) c_node + min_j H(left, j) + H(right, kWidth - j)).
// c_node in triangle tests.  1080p on the 1M-triangle terrain against the greedy collapse:
// c_node 1.5, AO trace 0.352 against 0.356 ms, shadow trace 0.256 against 0.266 ms (205,661
// instead of 278,891 nodes: the wide nodes are fuller); c_node 1: 0.351 / 0.259 ms;
// 2: 0.354 / 0.257 ms; 3: 0.362 / 0.258 ms.
#ifndef OCC_COLLAPSE_SAH
#define OCC_COLLAPSE_SAH 1
#endif
#ifndef OCC_COLLAPSE_CNODE
#define OCC_COLLAPSE_CNODE 1.5f
#endif
struct SahCollapser {
    const std::vector<BNode>& bn;
    std::vector<BvhNode>& nodes;
    float pad;
    uint32_t leaf_cap;
    int max_depth = 0;
    int64_t leaves = 0;
    uint32_t max_leaf = 0;

    std::vector<uint32_t> first, cnt;          // triangle range of each subtree
    std::vector<uint8_t> contiguous;           // subtree triangles form one range
    std::vector<float> F;                      // best cost as one slot
    std::vector<uint8_t> as_leaf;              // F chose a leaf
    std::vector<std::array<float, kWidth + 1>> Hc;     // H(n, k), k = 1 .. kWidth
    std::vector<std::array<uint8_t, kWidth + 1>> Hj;   // 0: one slot (F); j: j slots left

    void solve() {
        const size_t N = bn.size();
        first.assign(N, 0);
        cnt.assign(N, 0);
        contiguous.assign(N, 1);
        F.assign(N, 0.0f);
        as_leaf.assign(N, 0);
        Hc.assign(N, {});
        Hj.assign(N, {});
        // post-order without recursion
        std::vector<int32_t> order, stack = {0};
        order.reserve(N);
        while (!stack.empty()) {
            const int32_t n = stack.back();
            stack.pop_back();
            order.push_back(n);
            if (bn[n].left >= 0) {
                stack.push_back(bn[n].left);
                stack.push_back(bn[n].right);
            }
        }
        const float inf = std::numeric_limits<float>::infinity();
        for (size_t i = order.size(); i-- > 0;) {
            const int32_t n = order[i];
            const BNode& b = bn[n];
            const float A = b.box.area();
            if (b.left < 0) {
                first[n] = b.first;
                cnt[n] = b.count;
                F[n] = A * kIntersectCost * (float)b.count;
                as_leaf[n] = 1;
                for (int k = 1; k <= kWidth; ++k) {
                    Hc[n][k] = F[n];
                    Hj[n][k] = 0;
                }
                continue;
            }
            const int32_t l = b.left, r = b.right;
            cnt[n] = cnt[l] + cnt[r];
            first[n] = std::min(first[l], first[r]);
            contiguous[n] = contiguous[l] && contiguous[r] &&
                            (first[l] + cnt[l] == first[r] || first[r] + cnt[r] == first[l]);
            float split = inf;
            for (int j = 1; j < kWidth; ++j) split = std::min(split, Hc[l][j] + Hc[r][kWidth - j]);
            const float wide = A * OCC_COLLAPSE_CNODE + split;
            const float leaf = (cnt[n] <= leaf_cap && contiguous[n]) ? A * kIntersectCost * (float)cnt[n] : inf;
            as_leaf[n] = leaf <= wide;
            F[n] = std::min(leaf, wide);
            Hc[n][1] = F[n];
            Hj[n][1] = 0;
            for (int k = 2; k <= kWidth; ++k) {
                float best = F[n];
                uint8_t bj = 0;
                for (int j = 1; j < k; ++j) {
                    const float c = Hc[l][j] + Hc[r][k - j];
                    if (c < best) {
                        best = c;
                        bj = (uint8_t)j;
                    }
                }
                Hc[n][k] = best;
                Hj[n][k] = bj;
            }
        }
    }

    // the child slots of subtree m given k slots
    void collect(int32_t m, int k, std::vector<int32_t>& out) const {
        const int j = Hj[m][k];
        if (j == 0 || bn[m].left < 0) {
            out.push_back(m);
            return;
        }
        collect(bn[m].left, j, out);
        collect(bn[m].right, k - j, out);
    }

    uint32_t leaf_ref_of(int32_t m) {
        ++leaves;
        max_leaf = std::max(max_leaf, cnt[m]);
        return kLeafBit | ((cnt[m] - 1u) << kLeafCountShift) | first[m];
    }

    // Emits binary node n (internal) as a wide node and returns its index.
    uint32_t emit(int32_t n, int depth) {
        max_depth = std::max(max_depth, depth);
        const int32_t l = bn[n].left, r = bn[n].right;
        int bj = 1;
        float best = std::numeric_limits<float>::infinity();
        for (int j = 1; j < kWidth; ++j) {
            const float c = Hc[l][j] + Hc[r][kWidth - j];
            if (c < best) {
                best = c;
                bj = j;
            }
        }
        std::vector<int32_t> kids;
        collect(l, bj, kids);
        collect(r, kWidth - bj, kids);
        const uint32_t me = (uint32_t)nodes.size();
        nodes.push_back(empty_node());
        uint32_t ref[kWidth];
        for (size_t c = 0; c < kids.size(); ++c) {
            const int32_t k = kids[c];
            ref[c] = (bn[k].left < 0 || as_leaf[k]) ? leaf_ref_of(k) : emit(k, depth + 1);
        }
        BvhNode& node = nodes[me];   // after the recursion: the vector may have moved
        for (size_t c = 0; c < kids.size(); ++c) {
            const BNode& k = bn[kids[c]];
            for (int a = 0; a < 3; ++a) {
                plane_at(node, 2 * a, (int)c) = k.box.lo[a] - pad;
                plane_at(node, 2 * a + 1, (int)c) = k.box.hi[a] + pad;
            }
            set_child(node, (int)c, ref[c]);
        }
        return me;
    }
};

#endif  // !OCC_BVH_CW8

#if OCC_BVH_CW8
// Collapse of the binary tree (leaves of at most 3 triangles) into compressed 8-wide nodes
// (layout in occ_layout.h).  A node takes up to 8 children by opening its largest-area
// internal children; the children are placed in slots so that slot s holds the child
// nearest the corner of octant s (high on the axes whose bit is set), which the traversal
// visits first for rays whose direction signs are the complement of s; internal children
// go to consecutive node indices in slot order and the leaf children's triangles to
// consecutive triangle slots.
struct CwCollapser {
    const std::vector<BNode>& bn;
    const std::vector<uint32_t>& perm;
    const float* tris;               // input triangles [T][3][3]
    float pad;                       // absolute growth of every child box
    std::vector<BvhNode>& nodes;
    std::vector<float4>& otris;      // triangles in node order, 3 float4 each
    int max_depth = 0;
    int64_t leaves = 0;
    uint32_t max_leaf = 0;

    static void put_byte(float4& v, int word, int byte, uint32_t val) {
        unsigned char* b = reinterpret_cast<unsigned char*>(&v);
        b[4 * word + byte] = (unsigned char)(val & 0xFFu);   // little-endian word layout
    }
    static void put_word(float4& v, int word, uint32_t val) {
        std::memcpy(reinterpret_cast<unsigned char*>(&v) + 4 * word, &val, 4);
    }

    void append_tri(uint32_t id) {
        const float* v = tris + 9 * (int64_t)id;
        float idf;
        std::memcpy(&idf, &id, sizeof(idf));
        otris.push_back(make_float4(v[0], v[1], v[2], idf));
        otris.push_back(make_float4(v[3], v[4], v[5], 0.0f));
        otris.push_back(make_float4(v[6], v[7], v[8], 0.0f));
    }

    // Fills node `me` for binary node b (internal; or a leaf standing alone as the root).
    void fill(uint32_t me, int32_t b, int depth) {
        max_depth = std::max(max_depth, depth);
        std::vector<int32_t> kids;
        if (bn[b].left < 0) {
            kids.push_back(b);
        } else {
            kids = {bn[b].left, bn[b].right};
            while ((int)kids.size() < 8) {
                int pick = -1;
                float best = -1.0f;
                for (int i = 0; i < (int)kids.size(); ++i) {
                    const BNode& c = bn[kids[i]];
                    if (c.left < 0) continue;
                    const float a = c.box.area();
                    if (a > best) {
                        best = a;
                        pick = i;
                    }
                }
                if (pick < 0) break;
                const int32_t open = kids[pick];
                kids[pick] = bn[open].left;
                kids.push_back(bn[open].right);
            }
        }
        // the node's grid covers the padded children, one step of margin on each side
        AABB box;
        for (int32_t k : kids) box.grow(bn[k].box);
        float lo[3], hi[3], step[3];
        uint32_t ebits[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = box.lo[a] - pad;
            hi[a] = box.hi[a] + pad;
            const double ext = (double)hi[a] - (double)lo[a];
            int e = -126;
            while (e < 126 && std::ldexp(1.0, e) * 252.0 < ext) ++e;   // ext + 3 steps <= 255 steps
            step[a] = (float)std::ldexp(1.0, e);
            ebits[a] = (uint32_t)(e + 127);
            lo[a] = (float)((double)lo[a] - (double)step[a]);   // one step below the padded box
        }
        // slot assignment: greedy by distance into each octant's corner
        const int n = (int)kids.size();
        float pc[3];
        for (int a = 0; a < 3; ++a) pc[a] = 0.5f * (box.lo[a] + box.hi[a]);
        int slot_of[8], kid_in[8];
        for (int s = 0; s < 8; ++s) kid_in[s] = -1;
        std::vector<bool> placed(n, false);
        for (int round = 0; round < n; ++round) {
            float best = std::numeric_limits<float>::infinity();
            int bk = -1, bs = -1;
            for (int k = 0; k < n; ++k) {
                if (placed[k]) continue;
                const AABB& cb = bn[kids[k]].box;
                for (int s = 0; s < 8; ++s) {
                    if (kid_in[s] >= 0) continue;
                    float cost = 0.0f;
                    for (int a = 0; a < 3; ++a) {
                        const float d = 0.5f * (cb.lo[a] + cb.hi[a]) - pc[a];
                        cost += ((s >> a) & 1) ? -d : d;
                    }
                    if (cost < best) {
                        best = cost;
                        bk = k;
                        bs = s;
                    }
                }
            }
            placed[bk] = true;
            kid_in[bs] = bk;
            slot_of[bk] = bs;
        }
        (void)slot_of;
        // internal children in slot order, then the node's own fields
        uint32_t imask = 0, n_int = 0;
        for (int s = 0; s < 8; ++s)
            if (kid_in[s] >= 0 && bn[kids[kid_in[s]]].left >= 0) {
                imask |= 1u << s;
                ++n_int;
            }
        const uint32_t child_base = (uint32_t)nodes.size();
        nodes.resize(nodes.size() + n_int);
        const uint32_t tri_base = (uint32_t)(otris.size() / 3);
        BvhNode node;
        std::memset(&node, 0, sizeof(node));
        node.v[0] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        put_word(node.v[0], 3, ebits[0] | (ebits[1] << 8) | (ebits[2] << 16) | (imask << 24));
        put_word(node.v[1], 0, child_base);
        put_word(node.v[1], 1, tri_base);
        uint32_t tri_off = 0;
        for (int s = 0; s < 8; ++s) {
            uint32_t meta = 0, ql[3] = {255, 255, 255}, qh[3] = {0, 0, 0};
            if (kid_in[s] >= 0) {
                const BNode& c = bn[kids[kid_in[s]]];
                if (c.left >= 0) {
                    meta = 0x20u | (24u + (uint32_t)s);
                } else {
                    meta = (((1u << c.count) - 1u) << 5) | tri_off;
                    for (uint32_t i = 0; i < c.count; ++i) append_tri(perm[c.first + i]);
                    tri_off += c.count;
                    ++leaves;
                    max_leaf = std::max(max_leaf, c.count);
                }
                for (int a = 0; a < 3; ++a) {
                    // conservative grid cells of the padded child box, widened by one more step
                    const double l = ((double)c.box.lo[a] - pad - lo[a]) / step[a];
                    const double h = ((double)c.box.hi[a] + pad - lo[a]) / step[a];
                    ql[a] = (uint32_t)std::max(0.0, std::floor(l) - 1.0);
                    qh[a] = (uint32_t)std::min(255.0, std::ceil(h) + 1.0);
                }
            }
            put_byte(node.v[1], 2 + s / 4, s % 4, meta);
            put_byte(node.v[2], s / 4, s % 4, ql[0]);
            put_byte(node.v[2], 2 + s / 4, s % 4, ql[1]);
            put_byte(node.v[3], s / 4, s % 4, ql[2]);
            put_byte(node.v[3], 2 + s / 4, s % 4, qh[0]);
            put_byte(node.v[4], s / 4, s % 4, qh[1]);
            put_byte(node.v[4], 2 + s / 4, s % 4, qh[2]);
        }
        nodes[me] = node;
        uint32_t next = child_base;
        for (int s = 0; s < 8; ++s)
            if ((imask >> s) & 1u) fill(next++, kids[kid_in[s]], depth + 1);
    }
};
#endif  // OCC_BVH_CW8

}  // namespace

bool build_bvh4(const float* tris, int64_t T, HostBVH* out, std::string* err) {
    if (T <= 0 || T > (int64_t)kLeafFirstMask) {
        *err = "triangle count must be in [1, 2^26)";
        return false;
    }
    std::vector<AABB> tb((size_t)T);
    std::vector<std::array<float, 3>> tc((size_t)T);
    for (int64_t t = 0; t < T; ++t) {
        const float* v = tris + 9 * t;
        for (int q = 0; q < 3; ++q) {
            for (int a = 0; a < 3; ++a) {
                if (!std::isfinite(v[3 * q + a])) {
                    *err = "triangle coordinates must be finite";
                    return false;
                }
            }
            tb[t].grow(v + 3 * q);
        }
        for (int a = 0; a < 3; ++a) tc[t][a] = 0.5f * (tb[t].lo[a] + tb[t].hi[a]);
    }
    std::vector<uint32_t> perm((size_t)T);
    for (int64_t t = 0; t < T; ++t) perm[t] = (uint32_t)t;
    std::vector<BNode> bn;
    bn.reserve((size_t)(2 * T));
    Builder b{tb, tc, perm};
    if (OCC_BVH_CW8) b.leaf_max = kCwMaxLeafTris;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    int spawn = 0;
    while ((1u << spawn) < hw && spawn < 6) ++spawn;
    b.build(bn, 0, (uint32_t)T, spawn);

    // Child boxes grow by 2^-17 of the largest coordinate magnitude.  The traversal's
    // slab test takes one FMA per plane (lo * idir - o * idir), whose rounding moves a
    // plane by at most about 2^-23 of the coordinate magnitude; the growth keeps every
    // box conservative for rays whose origins lie within a few scene radii.
    float mag = 1.0f;
    for (int64_t i = 0; i < 9 * T; ++i) mag = std::max(mag, std::fabs(tris[i]));
    out->nodes.clear();
#if OCC_BVH_CW8
    out->tris.clear();
    out->tris.reserve((size_t)(3 * T));
    CwCollapser cw{bn, perm, tris, std::ldexp(mag, -17), out->nodes, out->tris};
    out->nodes.resize(1);
    cw.fill(0, 0, 0);
    // one stack entry (node group) per level
    if (cw.max_depth + 1 > kStackSize) {
        *err = "BVH too deep for the traversal stack";
        return false;
    }
    out->num_leaves = cw.leaves;
    out->depth = cw.max_depth + 1;
    out->max_leaf_tris = (int)cw.max_leaf;
    return true;
#else
    Collapser col{bn, out->nodes, std::ldexp(mag, -17)};
    if (bn[0].left < 0) {
        // the whole scene is one leaf: a root node with that single child
        BvhNode n = empty_node();
        const float p = col.pad;
        for (int a = 0; a < 3; ++a) {
            plane_at(n, 2 * a, 0) = bn[0].box.lo[a] - p;
            plane_at(n, 2 * a + 1, 0) = bn[0].box.hi[a] + p;
        }
        set_child(n, 0, Collapser::leaf_ref(bn[0]));
        out->nodes.push_back(n);
        col.leaves = 1;
        col.max_leaf = bn[0].count;
        col.max_depth = 0;
    } else if (OCC_COLLAPSE_SAH) {
        SahCollapser sc{bn, out->nodes, col.pad, kLeafMax};
        sc.solve();
        sc.emit(0, 0);
        col.leaves = sc.leaves;
        col.max_leaf = sc.max_leaf;
        col.max_depth = sc.max_depth;
    } else {
        col.emit(0, 0);
    }
    if ((kWidth - 1) * (col.max_depth + 1) > kStackSize) {
        *err = "BVH too deep for the traversal stack";
        return false;
    }
    out->tris.resize((size_t)(3 * T));
    for (int64_t i = 0; i < T; ++i) {
        const uint32_t id = perm[i];
        const float* v = tris + 9 * (int64_t)id;
        float idf;
        std::memcpy(&idf, &id, sizeof(idf));
        out->tris[3 * i + 0] = make_float4(v[0], v[1], v[2], idf);
        out->tris[3 * i + 1] = make_float4(v[3], v[4], v[5], 0.0f);
        out->tris[3 * i + 2] = make_float4(v[6], v[7], v[8], 0.0f);
    }
    out->num_leaves = col.leaves;
    out->depth = col.max_depth + 1;
    out->max_leaf_tris = (int)col.max_leaf;
    return true;
#endif
}

}  // namespace occ
