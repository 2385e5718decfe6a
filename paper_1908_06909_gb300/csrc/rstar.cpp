// rstar.cpp -- R*-tree construction by one-at-a-time insertion, written from
// the published algorithm (Beckmann, Kriegel, Schneider, Seeger, SIGMOD 1990),
// with the paper's node capacities (at least 4, at most 10 entries).
//
//   ChooseSubtree: in nodes whose children are leaves, the entry needing the
//     least overlap enlargement (ties: least volume enlargement, then least
//     volume); higher up, the least volume enlargement (ties: least volume).
//   OverflowTreatment: the first overflow on a level during one insertion
//     forcibly reinserts the 30% of entries whose centres lie farthest from
//     the node's centre (closest first); later overflows split.
//   Split: the axis with the least sum of margins over all distributions of
//     the entries sorted by lower and by upper bound; on it, the distribution
//     with the least overlap (ties: least total volume).
// Boundary faces of a polyhedral mesh often lie in common planes, so their
// boxes can be flat: every "volume" comparison falls back to the boxes'
// surface area when the volumes are equal.
#include "rstar.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

namespace tp {

namespace {

struct Box {
    float lo[3], hi[3];
};

struct Measure {  // compared lexicographically: volume, then surface area
    double vol, surf;
    bool operator<(const Measure &o) const { return vol < o.vol || (vol == o.vol && surf < o.surf); }
    bool operator==(const Measure &o) const { return vol == o.vol && surf == o.surf; }
    Measure operator-(const Measure &o) const { return {vol - o.vol, surf - o.surf}; }
    Measure operator+(const Measure &o) const { return {vol + o.vol, surf + o.surf}; }
};

Box empty_box() {
    Box b;
    for (int k = 0; k < 3; ++k) {
        b.lo[k] = std::numeric_limits<float>::infinity();
        b.hi[k] = -std::numeric_limits<float>::infinity();
    }
    return b;
}

Box merge(const Box &a, const Box &b) {
    Box r;
    for (int k = 0; k < 3; ++k) {
        r.lo[k] = std::min(a.lo[k], b.lo[k]);
        r.hi[k] = std::max(a.hi[k], b.hi[k]);
    }
    return r;
}

Measure measure(const Box &b) {
    double e[3];
    for (int k = 0; k < 3; ++k) e[k] = std::max(0.0, (double)b.hi[k] - (double)b.lo[k]);
    return {e[0] * e[1] * e[2], 2.0 * (e[0] * e[1] + e[1] * e[2] + e[2] * e[0])};
}

double margin(const Box &b) {
    double s = 0;
    for (int k = 0; k < 3; ++k) s += std::max(0.0, (double)b.hi[k] - (double)b.lo[k]);
    return s;
}

Measure overlap(const Box &a, const Box &b) {
    Box r;
    for (int k = 0; k < 3; ++k) {
        r.lo[k] = std::max(a.lo[k], b.lo[k]);
        r.hi[k] = std::min(a.hi[k], b.hi[k]);
        if (r.lo[k] > r.hi[k]) return {0.0, 0.0};
    }
    return measure(r);
}

double centre_dist2(const Box &a, const Box &b) {
    double s = 0;
    for (int k = 0; k < 3; ++k) {
        double d = 0.5 * ((double)a.lo[k] + a.hi[k]) - 0.5 * ((double)b.lo[k] + b.hi[k]);
        s += d * d;
    }
    return s;
}

struct Entry {
    Box b;
    int32_t ref;  // child node, or face index at level 0
};

struct BNode {
    int level = 0;  // 0: leaf (entries are faces)
    int parent = -1;
    std::vector<Entry> e;
};

class Builder {
  public:
    std::vector<BNode> N;
    int root = 0;

    Builder() {
        N.emplace_back();
        root = 0;
    }

    void insert_face(const Box &b, int32_t face) {
        std::memset(reinserted_, 0, sizeof(reinserted_));
        insert_entry({b, face}, 0);
    }

  private:
    bool reinserted_[64];

    Box node_box(int n) const {
        Box b = empty_box();
        for (const Entry &x : N[n].e) b = merge(b, x.b);
        return b;
    }

    void set_child(int n, const Entry &x) {
        if (N[n].level > 0) N[x.ref].parent = n;
    }

    // entry of child c inside its parent p
    Entry &entry_of(int p, int c) {
        for (Entry &x : N[p].e)
            if (x.ref == c) return x;
        return N[p].e[0];  // unreachable for a consistent tree
    }

    int choose_subtree(int n, const Box &b) const {
        const std::vector<Entry> &E = N[n].e;
        int best = 0;
        if (N[n].level == 1) {
            Measure bo{0, 0}, bv{0, 0}, ba{0, 0};
            for (size_t i = 0; i < E.size(); ++i) {
                const Box grown = merge(E[i].b, b);
                Measure o_old{0, 0}, o_new{0, 0};
                for (size_t j = 0; j < E.size(); ++j) {
                    if (j == i) continue;
                    o_old = o_old + overlap(E[i].b, E[j].b);
                    o_new = o_new + overlap(grown, E[j].b);
                }
                const Measure dov = o_new - o_old, dv = measure(grown) - measure(E[i].b),
                              a = measure(E[i].b);
                if (i == 0 || dov < bo || (dov == bo && (dv < bv || (dv == bv && a < ba)))) {
                    best = (int)i;
                    bo = dov;
                    bv = dv;
                    ba = a;
                }
            }
            return best;
        }
        Measure bv{0, 0}, ba{0, 0};
        for (size_t i = 0; i < E.size(); ++i) {
            const Measure dv = measure(merge(E[i].b, b)) - measure(E[i].b), a = measure(E[i].b);
            if (i == 0 || dv < bv || (dv == bv && a < ba)) {
                best = (int)i;
                bv = dv;
                ba = a;
            }
        }
        return best;
    }

    void insert_entry(const Entry &x, int level) {
        int n = root;
        while (N[n].level > level) n = N[n].e[choose_subtree(n, x.b)].ref;
        N[n].e.push_back(x);
        set_child(n, x);
        adjust(n);
    }

    // refresh boxes from n upward, treating overflows on the way
    void adjust(int n) {
        while (true) {
            if ((int)N[n].e.size() > RSTAR_MAX) {
                const int lvl = N[n].level;
                if (n != root && lvl < 64 && !reinserted_[lvl]) {
                    reinserted_[lvl] = true;
                    reinsert(n);
                    return;
                }
                const int nn = split(n);
                if (n == root) {
                    BNode r;
                    r.level = lvl + 1;
                    r.e.push_back({node_box(n), n});
                    r.e.push_back({node_box(nn), nn});
                    N.push_back(r);
                    root = (int)N.size() - 1;
                    N[n].parent = root;
                    N[nn].parent = root;
                    return;
                }
                const int p = N[n].parent;
                entry_of(p, n).b = node_box(n);
                N[p].e.push_back({node_box(nn), nn});
                N[nn].parent = p;
                n = p;
                continue;
            }
            if (n == root) return;
            const int p = N[n].parent;
            entry_of(p, n).b = node_box(n);
            n = p;
        }
    }

    void reinsert(int n) {
        const Box c = node_box(n);
        std::vector<Entry> E = N[n].e;
        std::stable_sort(E.begin(), E.end(), [&](const Entry &a, const Entry &b) {
            return centre_dist2(a.b, c) > centre_dist2(b.b, c);
        });
        const int p = (int)std::lround(0.3 * (RSTAR_MAX + 1));
        std::vector<Entry> out(E.begin(), E.begin() + p);
        N[n].e.assign(E.begin() + p, E.end());
        for (int m = n; m != root;) {  // the node shrank: refresh the path
            const int q = N[m].parent;
            entry_of(q, m).b = node_box(m);
            m = q;
        }
        const int level = N[n].level;
        for (int k = p - 1; k >= 0; --k) insert_entry(out[k], level);  // closest first
    }

    int split(int n) {
        std::vector<Entry> E = N[n].e;
        const int total = (int)E.size();
        auto sorted = [&](int axis, bool by_upper) {
            std::vector<Entry> s = E;
            std::stable_sort(s.begin(), s.end(), [&](const Entry &a, const Entry &b) {
                float ka = by_upper ? a.b.hi[axis] : a.b.lo[axis];
                float kb = by_upper ? b.b.hi[axis] : b.b.lo[axis];
                if (ka != kb) return ka < kb;
                float la = by_upper ? a.b.lo[axis] : a.b.hi[axis];
                float lb = by_upper ? b.b.lo[axis] : b.b.hi[axis];
                return la < lb;
            });
            return s;
        };
        auto group_boxes = [&](const std::vector<Entry> &s, int k, Box &g1, Box &g2) {
            g1 = empty_box();
            g2 = empty_box();
            for (int i = 0; i < total; ++i) (i < k ? g1 : g2) = merge(i < k ? g1 : g2, s[i].b);
        };
        // ChooseSplitAxis
        int axis = 0;
        double best_s = 0;
        for (int a = 0; a < 3; ++a) {
            double S = 0;
            for (int u = 0; u < 2; ++u) {
                const std::vector<Entry> s = sorted(a, u == 1);
                for (int k = RSTAR_MIN; k <= total - RSTAR_MIN; ++k) {
                    Box g1, g2;
                    group_boxes(s, k, g1, g2);
                    S += margin(g1) + margin(g2);
                }
            }
            if (a == 0 || S < best_s) {
                best_s = S;
                axis = a;
            }
        }
        // ChooseSplitIndex
        std::vector<Entry> best;
        int best_k = RSTAR_MIN;
        Measure bo{0, 0}, bv{0, 0};
        bool first = true;
        for (int u = 0; u < 2; ++u) {
            const std::vector<Entry> s = sorted(axis, u == 1);
            for (int k = RSTAR_MIN; k <= total - RSTAR_MIN; ++k) {
                Box g1, g2;
                group_boxes(s, k, g1, g2);
                const Measure o = overlap(g1, g2), v = measure(g1) + measure(g2);
                if (first || o < bo || (o == bo && v < bv)) {
                    first = false;
                    bo = o;
                    bv = v;
                    best = s;
                    best_k = k;
                }
            }
        }
        BNode nn;
        nn.level = N[n].level;
        nn.parent = N[n].parent;
        nn.e.assign(best.begin() + best_k, best.end());
        N[n].e.assign(best.begin(), best.begin() + best_k);
        N.push_back(nn);
        const int id = (int)N.size() - 1;
        if (N[id].level > 0)
            for (const Entry &x : N[id].e) N[x.ref].parent = id;
        return id;
    }
};

Box face_box(const BFace32 &f) {
    Box b;
    const float4 *v[3] = {&f.a, &f.b, &f.c};
    for (int k = 0; k < 3; ++k) {
        const float c0 = k == 0 ? v[0]->x : (k == 1 ? v[0]->y : v[0]->z);
        const float c1 = k == 0 ? v[1]->x : (k == 1 ? v[1]->y : v[1]->z);
        const float c2 = k == 0 ? v[2]->x : (k == 1 ? v[2]->y : v[2]->z);
        b.lo[k] = std::min(c0, std::min(c1, c2));
        b.hi[k] = std::max(c0, std::max(c1, c2));
    }
    return b;
}

}  // namespace

void rstar_build(const std::vector<BFace32> &faces, std::vector<RStarNode> &nodes) {
    Builder B;
    for (size_t q = 0; q < faces.size(); ++q) B.insert_face(face_box(faces[q]), (int32_t)q);
    // breadth-first renumbering, root first
    nodes.clear();
    std::vector<int> order{B.root}, index(B.N.size(), -1);
    index[B.root] = 0;
    for (size_t i = 0; i < order.size(); ++i)
        for (const Entry &x : B.N[order[i]].e)
            if (B.N[order[i]].level > 0) {
                index[x.ref] = (int)order.size();
                order.push_back(x.ref);
            }
    nodes.resize(order.size());
    for (size_t i = 0; i < order.size(); ++i) {
        const BNode &s = B.N[order[i]];
        RStarNode &d = nodes[i];
        std::memset(&d, 0, sizeof(d));
        d.count = (int32_t)s.e.size();
        d.leaf = s.level == 0;
        for (int k = 0; k < d.count; ++k) {
            for (int a = 0; a < 3; ++a) {
                d.lo[a][k] = s.e[k].b.lo[a];
                d.hi[a][k] = s.e[k].b.hi[a];
            }
            d.child[k] = d.leaf ? s.e[k].ref : index[s.e[k].ref];
        }
    }
}

RStarStats rstar_check(const std::vector<BFace32> &faces, const std::vector<RStarNode> &nodes) {
    RStarStats st;
    st.nodes = (int64_t)nodes.size();
    if (nodes.empty()) return st;
    std::vector<int> seen(faces.size(), 0);
    bool ok = true;
    int leaf_depth = -1;
    st.min_fill = RSTAR_MAX;
    struct Item { int node, depth; Box box; bool has_box; };
    std::vector<Item> stack{{0, 0, Box(), false}};
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        const RStarNode &n = nodes[it.node];
        if (it.node != 0) {
            st.min_fill = std::min(st.min_fill, n.count);
            st.max_fill = std::max(st.max_fill, n.count);
            if (n.count < RSTAR_MIN || n.count > RSTAR_MAX) ok = false;
        } else if (n.count > RSTAR_MAX || (!n.leaf && n.count < 2)) {
            ok = false;
        }
        for (int k = 0; k < n.count; ++k) {
            Box b;
            for (int a = 0; a < 3; ++a) {
                b.lo[a] = n.lo[a][k];
                b.hi[a] = n.hi[a][k];
            }
            if (it.has_box)
                for (int a = 0; a < 3; ++a)
                    if (b.lo[a] < it.box.lo[a] || b.hi[a] > it.box.hi[a]) ok = false;
            if (n.leaf) {
                const int q = n.child[k];
                if (q < 0 || q >= (int)faces.size()) { ok = false; continue; }
                ++seen[q];
                const Box fb = face_box(faces[q]);
                for (int a = 0; a < 3; ++a)
                    if (fb.lo[a] < b.lo[a] || fb.hi[a] > b.hi[a]) ok = false;
                ++st.entries;
            } else {
                if (n.child[k] <= it.node || n.child[k] >= (int)nodes.size()) { ok = false; continue; }
                stack.push_back({n.child[k], it.depth + 1, b, true});
            }
        }
        if (n.leaf) {
            ++st.leaves;
            if (leaf_depth < 0) leaf_depth = it.depth;
            else if (leaf_depth != it.depth) ok = false;
        }
    }
    for (int s : seen)
        if (s != 1) ok = false;
    st.depth = leaf_depth + 1;
    st.ok = ok ? 1 : 0;
    return st;
}

}  // namespace tp
