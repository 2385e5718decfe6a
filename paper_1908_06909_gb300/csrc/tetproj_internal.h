// tetproj_internal.h -- data layout shared by the host builder and the kernels.
//
// Device mesh (Sec. II-B: "each element contains nD+1 nodes and nD+1 ordered
// neighbour indexes"), stored as structure-of-arrays records indexed by the
// tet's position h along a 3-D Hilbert curve of tet centroids:
//
//   TetRec32  64 B  the four vertices in FP32 (12 floats, three float4) and the
//                   packed neighbours adj[k] = (h' << 2) | k' across the face
//                   opposite local vertex k (k' = that face's index in h'),
//                   or -1 on the boundary.  One walk step reads exactly these
//                   two 32-byte sectors.
//   TetRec64 128 B  the same vertices in FP64 (exact inputs of the predicate
//                   fallback and of the FP64 path), adj, and the user's tet id.
//
// Each tet's local vertices are positively oriented: orient3d(v0,v1,v2,v3) > 0.
// Face f is opposite v_f; FACE_TRIPLE[f] lists its vertices so that
// orient3d(a, b, c, v_f) > 0 (v_f on the positive side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "predicates.cuh"

namespace tp {

// v[k].xyz: local vertex k in FP32; v[k].w: int bits of the neighbour across
// the face opposite vertex k, (h << 2) | f (f: that face's index in the
// neighbour), or -1 on the boundary.  A walk step loads v[f] and the face
// triple of face f by index, so no per-coordinate selection is needed.
struct __align__(16) TetRec32 {
    float4 v[4];
};
static_assert(sizeof(TetRec32) == 64, "TetRec32 must be 64 bytes");

struct __align__(16) TetRec64 {
    double v[12];  // v0..v3 xyz
    int4 adj;
    int4 extra;    // x: user tet id
};
static_assert(sizeof(TetRec64) == 128, "TetRec64 must be 128 bytes");

// Boundary face, FP32 copy in FACE_TRIPLE order; a.w holds the int bits of
// (h << 2) | f.
struct __align__(16) BFace32 {
    float4 a, b, c;
};

// Binary BVH node holding both children's boxes (one 64-byte load tests two
// boxes).  child >= 0: internal node index; child < 0: leaf ~(first << 3 | count).
struct __align__(16) BvhNode {
    float4 lmin;  // xyz, w = bits of left child code
    float4 lmax;  // xyz, w unused
    float4 rmin;  // xyz, w = bits of right child code
    float4 rmax;
};

// R*-tree node over boundary faces (the paper's entry structure, Sec. II-E):
// at least RSTAR_MIN and at most RSTAR_MAX entries per node (the paper's 4 and
// 10); child boxes structure-of-arrays; leaves list boundary-face indices.
constexpr int RSTAR_MIN = 4;
constexpr int RSTAR_MAX = 10;
constexpr int RSTAR_MAX_DEPTH = 12;  // device DFS stack: 9 * depth + 1 entries

struct __align__(16) RStarNode {
    float lo[3][RSTAR_MAX];
    float hi[3][RSTAR_MAX];
    int32_t child[RSTAR_MAX];  // internal: node index; leaf: boundary-face index
    int32_t count;
    int32_t leaf;  // 1: children are boundary faces
    int32_t pad[2];
};

struct AngleFrame {
    double S[3], C[3], U[3], V[3];
};

struct DevCounters {
    unsigned long long rays, hits, segments, fp64, exact, sos, bvh_nodes, bvh_faces, deferred;
    int error;
    int error_count;
    unsigned long long grazing;  // crossings placed again from the FP64 records
};

struct MeshView {
    const TetRec32 *rec32;
    const TetRec64 *rec64;
    const BvhNode *bvh;
    const BFace32 *bfaces;
    const int32_t *perm;  // h -> user tet id
    const int4 *vid;      // h -> user vertex ids in local order
    const RStarNode *rstar;  // R*-tree of the boundary faces (built on request)
    int64_t nt, nb, nnodes;
    int32_t root;         // root code (0, or a leaf code for tiny meshes)
    float radius;         // max |coordinate| over all vertices
    DevCounters *counters;
};

struct GeoView {
    const AngleFrame *frames;
    int32_t nu, nv, na;
    double du, dv;
};

TP_HD void face_triple(int f, int &a, int &b, int &c) {
    // f0: (1,3,2) f1: (0,2,3) f2: (0,3,1) f3: (0,1,2)
    a = (f == 0) ? 1 : 0;
    b = (f == 0) ? 3 : (f == 1 ? 2 : (f == 2 ? 3 : 1));
    c = (f == 0) ? 2 : (f == 1 ? 3 : (f == 2 ? 1 : 2));
}

// The same table packed 2 bits per index: face f's triple is
// (FACE_TRIPLES >> 6f) & 63 = a | b << 2 | c << 4.
constexpr int kFaceTriple0 = 1 | 3 << 2 | 2 << 4, kFaceTriple1 = 0 | 2 << 2 | 3 << 4,
              kFaceTriple2 = 0 | 3 << 2 | 1 << 4, kFaceTriple3 = 0 | 1 << 2 | 2 << 4;
constexpr int FACE_TRIPLES = kFaceTriple0 | kFaceTriple1 << 6 | kFaceTriple2 << 12 |
                             kFaceTriple3 << 18;

}  // namespace tp
