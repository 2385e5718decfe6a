// mesh_build.cpp -- host preprocessing of a tetrahedral mesh (one-time).
//
// Sec. II-B of the paper turns the mesh into a graph: each element keeps its
// nD+1 nodes and nD+1 ordered neighbour indices; Sec. II-E adds a list of the
// elements on the mesh boundary and a search tree over them so that each ray
// finds its first element without an exhaustive search.  Sec. II-D requires the
// mesh to be convex.  This file builds all of that on the host:
//
//   1. index checks; exact orientation of every tet (zero -> rejected,
//      negative -> local vertices 2 and 3 swapped);
//   2. face adjacency by bucketing faces on their smallest vertex id; a face
//      shared by more than two tets, or by two tets on the same side, is
//      rejected;
//   3. boundary checks: the boundary faces must form a closed, consistently
//      oriented surface that is convex at every edge, and the tets must be
//      connected (then the boundary is a convex polyhedron and a ray enters it
//      at most once);
//   4. tets renumbered along a 3-D Hilbert curve of their centroids (neighbours
//      in space become neighbours in memory, which is what keeps a walk step's
//      two 32-byte sectors in L2);
//   5. packed records (TetRec32 / TetRec64) and a binary BVH over the boundary
//      faces (median split on the longest centroid axis, <= 4 faces per leaf,
//      nodes numbered breadth-first so the top levels are a prefix).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mesh_build.h"

namespace tp {


static inline d3 vtx(const double *V, int32_t i) { return {V[3 * i], V[3 * i + 1], V[3 * i + 2]}; }

// sign of det[b - a, c - a, d - a] (exact, no tie-break)
static int orient_sign(const d3 &a, const d3 &b, const d3 &c, const d3 &d) {
    Filt64Vert v = filt64_vert(a, sub(b, a), c);
    double val;
    int s = filt64_side(v, d, val);
    if (s != 0) return s;
    return side_exact_sign(a, b, c, d);
}

// parity of the permutation taking (x0,x1,x2) to (y0,y1,y2) (same set): 0 even, 1 odd
static int triple_parity(const int32_t x[3], const int32_t y[3]) {
    int p[3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (y[i] == x[j]) p[i] = j;
    int inv = (p[0] > p[1]) + (p[0] > p[2]) + (p[1] > p[2]);
    return inv & 1;
}

struct Topology {
    std::vector<int32_t> tets;  // oriented, [nt][4]
    std::vector<int32_t> adj;   // [nt][4]: neighbour*4 + face, or -1
    std::vector<int64_t> bface; // boundary faces t*4 + f
    int64_t nflipped = 0;
};

// Steps 1-3.
static tetproj_status build_topology(const double *V, int64_t nv, const int32_t *T, int64_t nt,
                                     Topology &topo) {
    if (!V || !T || nv < 4 || nt < 1) return TETPROJ_ERR_ARG;
    if (nt >= (int64_t(1) << 29) || nv >= (int64_t(1) << 31) - 1) return TETPROJ_ERR_TOO_LARGE;
    for (int64_t i = 0; i < 3 * nv; ++i)
        if (!(std::fabs(V[i]) < 1e9)) return TETPROJ_ERR_ARG;
    topo.tets.assign(T, T + 4 * nt);
    int32_t *tt = topo.tets.data();
    topo.nflipped = 0;
    for (int64_t t = 0; t < nt; ++t) {
        int32_t *q = tt + 4 * t;
        for (int k = 0; k < 4; ++k)
            if (q[k] < 0 || q[k] >= nv) return TETPROJ_ERR_INDEX;
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (q[a] == q[b]) return TETPROJ_ERR_INDEX;
        int s = orient_sign(vtx(V, q[0]), vtx(V, q[1]), vtx(V, q[2]), vtx(V, q[3]));
        if (s == 0) return TETPROJ_ERR_DEGENERATE_TET;
        if (s < 0) {
            std::swap(q[2], q[3]);
            ++topo.nflipped;
        }
    }
    // faces bucketed by smallest vertex id
    struct FaceKey { int32_t j, k; int64_t tf; };
    std::vector<int64_t> start(nv + 1, 0);
    auto face_sorted = [&](int64_t t, int f, int32_t &i, int32_t &j, int32_t &k) {
        int32_t w[3];
        int n = 0;
        for (int m = 0; m < 4; ++m)
            if (m != f) w[n++] = tt[4 * t + m];
        std::sort(w, w + 3);
        i = w[0]; j = w[1]; k = w[2];
    };
    for (int64_t t = 0; t < nt; ++t)
        for (int f = 0; f < 4; ++f) {
            int32_t i, j, k;
            face_sorted(t, f, i, j, k);
            start[i + 1]++;
        }
    for (int64_t i = 0; i < nv; ++i) start[i + 1] += start[i];
    std::vector<FaceKey> faces(4 * nt);
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t t = 0; t < nt; ++t)
            for (int f = 0; f < 4; ++f) {
                int32_t i, j, k;
                face_sorted(t, f, i, j, k);
                faces[fill[i]++] = {j, k, 4 * t + f};
            }
    }
    topo.adj.assign(4 * nt, -1);
    topo.bface.clear();
    for (int64_t i = 0; i < nv; ++i) {
        FaceKey *b = faces.data() + start[i], *e = faces.data() + start[i + 1];
        std::sort(b, e, [](const FaceKey &x, const FaceKey &y) {
            return x.j != y.j ? x.j < y.j : (x.k != y.k ? x.k < y.k : x.tf < y.tf);
        });
        for (FaceKey *p = b; p < e;) {
            FaceKey *q = p + 1;
            while (q < e && q->j == p->j && q->k == p->k) ++q;
            int64_t cnt = q - p;
            if (cnt == 1) {
                topo.bface.push_back(p->tf);
            } else if (cnt == 2) {
                int64_t t1 = p[0].tf >> 2, t2 = p[1].tf >> 2;
                int f1 = (int)(p[0].tf & 3), f2 = (int)(p[1].tf & 3);
                if (t1 == t2) return TETPROJ_ERR_NONMANIFOLD;
                int a, bb, c;
                face_triple(f1, a, bb, c);
                int32_t x[3] = {tt[4 * t1 + a], tt[4 * t1 + bb], tt[4 * t1 + c]};
                face_triple(f2, a, bb, c);
                int32_t y[3] = {tt[4 * t2 + a], tt[4 * t2 + bb], tt[4 * t2 + c]};
                if (triple_parity(x, y) != 1) return TETPROJ_ERR_NONMANIFOLD;
                topo.adj[p[0].tf] = (int32_t)(4 * t2 + f2);
                topo.adj[p[1].tf] = (int32_t)(4 * t1 + f1);
            } else {
                return TETPROJ_ERR_NONMANIFOLD;
            }
            p = q;
        }
    }
    // boundary: closed, consistently oriented, convex at every edge
    struct DEdge { uint64_t key; int64_t face; int32_t third; };
    std::vector<DEdge> edges;
    edges.reserve(3 * topo.bface.size());
    for (size_t q = 0; q < topo.bface.size(); ++q) {
        int64_t t = topo.bface[q] >> 2;
        int f = (int)(topo.bface[q] & 3);
        int a, b, c;
        face_triple(f, a, b, c);
        int32_t w[3] = {tt[4 * t + a], tt[4 * t + b], tt[4 * t + c]};
        for (int e = 0; e < 3; ++e) {
            uint64_t u = (uint32_t)w[e], v = (uint32_t)w[(e + 1) % 3];
            edges.push_back({(u << 32) | v, (int64_t)q, w[(e + 2) % 3]});
        }
    }
    std::sort(edges.begin(), edges.end(),
              [](const DEdge &x, const DEdge &y) { return x.key < y.key; });
    for (size_t k = 1; k < edges.size(); ++k)
        if (edges[k].key == edges[k - 1].key) return TETPROJ_ERR_NONMANIFOLD;
    for (const DEdge &e : edges) {
        uint64_t u = e.key >> 32, v = e.key & 0xffffffffu;
        uint64_t rk = (v << 32) | u;
        auto it = std::lower_bound(edges.begin(), edges.end(), rk,
                                   [](const DEdge &x, uint64_t k) { return x.key < k; });
        if (it == edges.end() || it->key != rk) return TETPROJ_ERR_NONMANIFOLD;
        // face of e in table order (inner side positive); it->third must not be outside
        int64_t t = topo.bface[e.face] >> 2;
        int f = (int)(topo.bface[e.face] & 3);
        int a, b, c;
        face_triple(f, a, b, c);
        int s = orient_sign(vtx(V, tt[4 * t + a]), vtx(V, tt[4 * t + b]), vtx(V, tt[4 * t + c]),
                            vtx(V, it->third));
        if (s < 0) return TETPROJ_ERR_NONCONVEX;
    }
    // connected
    std::vector<char> seen(nt, 0);
    std::vector<int64_t> stack{0};
    seen[0] = 1;
    int64_t nseen = 1;
    while (!stack.empty()) {
        int64_t t = stack.back();
        stack.pop_back();
        for (int f = 0; f < 4; ++f) {
            int32_t n = topo.adj[4 * t + f];
            if (n >= 0 && !seen[n >> 2]) {
                seen[n >> 2] = 1;
                ++nseen;
                stack.push_back(n >> 2);
            }
        }
    }
    if (nseen != nt) return TETPROJ_ERR_NONCONVEX;
    return TETPROJ_OK;
}

// 3-D Hilbert index of integer coordinates with `bits` bits each, by the
// transpose method of J. Skilling, "Programming the Hilbert curve" (2004):
// undo excess work top-down, Gray-encode, then interleave the bits.
static uint64_t hilbert3(uint32_t x, uint32_t y, uint32_t z, int bits) {
    uint32_t X[3] = {x, y, z};
    uint32_t M = 1u << (bits - 1);
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

static float round_down(double x) {
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -INFINITY);
    return f;
}
static float round_up(double x) {
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}
static float int_bits_as_float(int32_t v) {
    float f;
    std::memcpy(&f, &v, 4);
    return f;
}

struct BuildFace {
    int32_t h, f;
    double lo[3], hi[3], c[3];
};

struct BvhBuilder {
    std::vector<BuildFace> &F;
    std::vector<BvhNode> nodes;  // DFS order during build
    explicit BvhBuilder(std::vector<BuildFace> &f) : F(f) {}

    void bounds(int64_t b, int64_t e, double lo[3], double hi[3]) {
        for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
        for (int64_t i = b; i < e; ++i)
            for (int k = 0; k < 3; ++k) {
                lo[k] = std::min(lo[k], F[i].lo[k]);
                hi[k] = std::max(hi[k], F[i].hi[k]);
            }
    }
    int32_t build(int64_t b, int64_t e) {
        if (e - b <= 4) return ~(int32_t)((b << 3) | (e - b));
        double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = b; i < e; ++i)
            for (int k = 0; k < 3; ++k) {
                clo[k] = std::min(clo[k], F[i].c[k]);
                chi[k] = std::max(chi[k], F[i].c[k]);
            }
        int axis = 0;
        for (int k = 1; k < 3; ++k)
            if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
        int64_t m = (b + e) / 2;
        std::nth_element(F.begin() + b, F.begin() + m, F.begin() + e,
                         [axis](const BuildFace &x, const BuildFace &y) {
                             return x.c[axis] != y.c[axis] ? x.c[axis] < y.c[axis]
                                                           : (x.h != y.h ? x.h < y.h : x.f < y.f);
                         });
        int32_t idx = (int32_t)nodes.size();
        nodes.push_back(BvhNode{});
        int32_t l = build(b, m);
        int32_t r = build(m, e);
        double llo[3], lhi[3], rlo[3], rhi[3];
        bounds(b, m, llo, lhi);
        bounds(m, e, rlo, rhi);
        BvhNode &n = nodes[idx];
        n.lmin = make_float4(round_down(llo[0]), round_down(llo[1]), round_down(llo[2]),
                             int_bits_as_float(l));
        n.lmax = make_float4(round_up(lhi[0]), round_up(lhi[1]), round_up(lhi[2]), 0.f);
        n.rmin = make_float4(round_down(rlo[0]), round_down(rlo[1]), round_down(rlo[2]),
                             int_bits_as_float(r));
        n.rmax = make_float4(round_up(rhi[0]), round_up(rhi[1]), round_up(rhi[2]), 0.f);
        return idx;
    }
};

static int32_t float_bits(float f) {
    int32_t v;
    std::memcpy(&v, &f, 4);
    return v;
}

tetproj_status build_host_mesh(const double *V, int64_t nv, const int32_t *T, int64_t nt,
                               HostMesh &M) {
    Topology topo;
    tetproj_status st = build_topology(V, nv, T, nt, topo);
    if (st != TETPROJ_OK) return st;
    M.nt = nt;
    M.nv = nv;
    M.nflipped = topo.nflipped;
    M.nb = (int64_t)topo.bface.size();
    const int32_t *tt = topo.tets.data();

    // bounding box / radius
    for (int k = 0; k < 3; ++k) { M.bbox[k] = INFINITY; M.bbox[3 + k] = -INFINITY; }
    double rad = 0.0;
    for (int64_t i = 0; i < nv; ++i)
        for (int k = 0; k < 3; ++k) {
            M.bbox[k] = std::min(M.bbox[k], V[3 * i + k]);
            M.bbox[3 + k] = std::max(M.bbox[3 + k], V[3 * i + k]);
            rad = std::max(rad, std::fabs(V[3 * i + k]));
        }
    M.radius = round_up(rad);

    // Hilbert order of centroids
    const int bits = 21;
    const double span = (double)((1u << bits) - 1);
    double ext[3];
    for (int k = 0; k < 3; ++k) ext[k] = std::max(M.bbox[3 + k] - M.bbox[k], 1e-300);
    std::vector<std::pair<uint64_t, int32_t>> keys(nt);
    for (int64_t t = 0; t < nt; ++t) {
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            double c = 0.25 * (V[3 * tt[4 * t] + k] + V[3 * tt[4 * t + 1] + k] +
                               V[3 * tt[4 * t + 2] + k] + V[3 * tt[4 * t + 3] + k]);
            double u = (c - M.bbox[k]) / ext[k] * span;
            q[k] = (uint32_t)std::min(std::max(u, 0.0), span);
        }
        keys[t] = {hilbert3(q[0], q[1], q[2], bits), (int32_t)t};
    }
    std::sort(keys.begin(), keys.end());
    M.perm.resize(nt);
    std::vector<int32_t> inv(nt);
    for (int64_t h = 0; h < nt; ++h) {
        M.perm[h] = keys[h].second;
        inv[keys[h].second] = (int32_t)h;
    }
    keys.clear();
    keys.shrink_to_fit();

    // records
    M.rec32.resize(nt);
    M.rec64.resize(nt);
    M.vid.resize(nt);
    for (int64_t h = 0; h < nt; ++h) {
        int64_t t = M.perm[h];
        M.vid[h] = make_int4(tt[4 * t], tt[4 * t + 1], tt[4 * t + 2], tt[4 * t + 3]);
        TetRec64 &r = M.rec64[h];
        float c[12];
        for (int k = 0; k < 4; ++k)
            for (int m = 0; m < 3; ++m) {
                r.v[3 * k + m] = V[3 * tt[4 * t + k] + m];
                c[3 * k + m] = (float)r.v[3 * k + m];
            }
        int32_t a[4];
        for (int k = 0; k < 4; ++k) {
            int32_t n = topo.adj[4 * t + k];
            a[k] = n < 0 ? -1 : ((inv[n >> 2] << 2) | (n & 3));
        }
        r.adj = make_int4(a[0], a[1], a[2], a[3]);
        r.extra = make_int4((int32_t)t, 0, 0, 0);
        TetRec32 &s = M.rec32[h];
        for (int k = 0; k < 4; ++k)
            s.v[k] = make_float4(c[3 * k], c[3 * k + 1], c[3 * k + 2], int_bits_as_float(a[k]));
    }

    // boundary faces + BVH
    std::vector<BuildFace> F(M.nb);
    for (int64_t q = 0; q < M.nb; ++q) {
        int64_t t = topo.bface[q] >> 2;
        int f = (int)(topo.bface[q] & 3);
        BuildFace &b = F[q];
        b.h = inv[t];
        b.f = f;
        for (int k = 0; k < 3; ++k) { b.lo[k] = INFINITY; b.hi[k] = -INFINITY; b.c[k] = 0; }
        for (int m = 0; m < 4; ++m) {
            if (m == f) continue;
            for (int k = 0; k < 3; ++k) {
                double x = V[3 * tt[4 * t + m] + k];
                b.lo[k] = std::min(b.lo[k], x);
                b.hi[k] = std::max(b.hi[k], x);
                b.c[k] += x / 3.0;
            }
        }
    }
    std::sort(F.begin(), F.end(), [](const BuildFace &x, const BuildFace &y) {
        return x.h != y.h ? x.h < y.h : x.f < y.f;
    });
    BvhBuilder B(F);
    int32_t root = B.build(0, M.nb);
    if (root < 0) {
        M.root = root;
        M.bvh.clear();
    } else {
        // breadth-first renumbering (top levels become a prefix)
        std::vector<int32_t> order, newidx(B.nodes.size(), -1);
        order.push_back(root);
        newidx[root] = 0;
        for (size_t k = 0; k < order.size(); ++k) {
            const BvhNode &n = B.nodes[order[k]];
            int32_t ch[2] = {float_bits(n.lmin.w), float_bits(n.rmin.w)};
            for (int s = 0; s < 2; ++s)
                if (ch[s] >= 0) {
                    newidx[ch[s]] = (int32_t)order.size();
                    order.push_back(ch[s]);
                }
        }
        M.bvh.resize(order.size());
        for (size_t k = 0; k < order.size(); ++k) {
            BvhNode n = B.nodes[order[k]];
            int32_t l = float_bits(n.lmin.w), r = float_bits(n.rmin.w);
            if (l >= 0) n.lmin.w = int_bits_as_float(newidx[l]);
            if (r >= 0) n.rmin.w = int_bits_as_float(newidx[r]);
            M.bvh[k] = n;
        }
        M.root = 0;
    }
    M.bfaces.resize(M.nb);
    for (int64_t q = 0; q < M.nb; ++q) {
        const TetRec32 &s = M.rec32[F[q].h];
        int a, b, cc;
        face_triple(F[q].f, a, b, cc);
        BFace32 &o = M.bfaces[q];
        o.a = make_float4(s.v[a].x, s.v[a].y, s.v[a].z, int_bits_as_float((F[q].h << 2) | F[q].f));
        o.b = make_float4(s.v[b].x, s.v[b].y, s.v[b].z, 0.f);
        o.c = make_float4(s.v[cc].x, s.v[cc].y, s.v[cc].z, 0.f);
    }
    return TETPROJ_OK;
}

tetproj_status topology_host(const double *V, int64_t nv, const int32_t *T, int64_t nt,
                             int32_t *adj_out, int64_t *nboundary, int64_t *nflipped) {
    Topology topo;
    tetproj_status st = build_topology(V, nv, T, nt, topo);
    if (st != TETPROJ_OK) return st;
    for (int64_t t = 0; t < nt; ++t) {
        bool flipped = topo.tets[4 * t + 2] != T[4 * t + 2];
        for (int k = 0; k < 4; ++k) {
            int kk = k;
            if (flipped && k >= 2) kk = 5 - k;  // input vertex 2 <-> 3
            int32_t n = topo.adj[4 * t + kk];
            if (adj_out) adj_out[4 * t + k] = n < 0 ? -1 : (n >> 2);
        }
    }
    if (nboundary) *nboundary = (int64_t)topo.bface.size();
    if (nflipped) *nflipped = topo.nflipped;
    return TETPROJ_OK;
}

}  // namespace tp
