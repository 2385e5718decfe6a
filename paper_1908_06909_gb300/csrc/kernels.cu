// kernels.cu -- the per-ray hot path: ray generation, boundary entry search,
// tet-to-tet walk with exact-sign exit decisions, forward accumulation,
// backprojection scatter and row tracing.
//
// Paper map: Alg. 2 (robust ray propagation: one thread per detector pixel,
// l = |R2 - R1|, sum += l (t2 - t1) mu, step to the neighbour across the face
// where t2 happened, stop at -1), Sec. II-E (initialisation: the first tet is
// found through a search tree over boundary elements, depth first, keeping
// the earliest hit), Sec. II-F (pixels in small square blocks; backprojection
// launched like the projection with atomic adds).
//
// What differs from the paper's kernels (which target Pascal):
// * exit faces come from the signs of three side products per step (the three
//   edges from the new vertex), decided exactly (predicates.cuh), instead of
//   four Moeller-Trumbore tests with a growing epsilon;
// * the entry face is THE boundary face the (perturbed) line crosses inward:
//   for a convex mesh it is unique, so the BVH search stops at the first hit;
// * a step reads one 64-byte record (four FP32 vertices + packed neighbours);
//   the entry point of the next tet is carried in registers as a point, and a
//   segment length is (X_out - X_in).d/|d| with X_out from barycentric weights
//   given by the side products (no absolute t, so lengths keep relative
//   accuracy near the origin of fine regions);
// * every warp runs its 32 rays in lock-step (the loop condition is a warp
//   vote), which makes warp-level aggregation of backprojection atomics legal.
#include <cuda_runtime.h>

#include <atomic>
#include <math.h>

#include "../../include/tetproj.h"
#include "kernels.cuh"

namespace tp {

#define FULL_MASK 0xffffffffu

struct LocalCnt {
    unsigned rays, hits, segs, fp64, exact, sos, nodes, faces, graze;
};

__device__ __forceinline__ void report_error(DevCounters *C, int code) {
    atomicCAS(&C->error, 0, code);
    atomicAdd(&C->error_count, 1);
}

__device__ __forceinline__ void flush_counters(DevCounters *C, const LocalCnt &c) {
    unsigned v[9] = {c.rays, c.hits, c.segs, c.fp64, c.exact, c.sos, c.nodes, c.faces, c.graze};
    unsigned long long *dst[9] = {&C->rays, &C->hits, &C->segments, &C->fp64, &C->exact,
                                  &C->sos, &C->bvh_nodes, &C->bvh_faces, &C->grazing};
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        unsigned s = __reduce_add_sync(FULL_MASK, v[k]);
        if (lane == 0 && s) atomicAdd(dst[k], (unsigned long long)s);
    }
}

// ------------------------------------------------------------------ rays

__device__ __forceinline__ void cone_ray(const GeoView &g, int a, int iv, int iu, d3 &S, d3 &P) {
    const AngleFrame *F = g.frames + a;
    double u = ((double)iu - 0.5 * (double)(g.nu - 1)) * g.du;
    double v = ((double)iv - 0.5 * (double)(g.nv - 1)) * g.dv;
    S = mk(__ldg(&F->S[0]), __ldg(&F->S[1]), __ldg(&F->S[2]));
    P.x = (__ldg(&F->C[0]) + u * __ldg(&F->U[0])) + v * __ldg(&F->V[0]);
    P.y = (__ldg(&F->C[1]) + u * __ldg(&F->U[1])) + v * __ldg(&F->V[1]);
    P.z = (__ldg(&F->C[2]) + u * __ldg(&F->U[2])) + v * __ldg(&F->V[2]);
}

__device__ __forceinline__ void load_ray(const KParams &p, int64_t ray, d3 &S, d3 &P) {
    if (p.src_kind == 0) {
        int iu = (int)(ray % p.g.nu);
        int64_t r2 = ray / p.g.nu;
        int iv = (int)(r2 % p.g.nv);
        int a = (int)(r2 / p.g.nv);
        cone_ray(p.g, a, iv, iu, S, P);
    } else {
        const double *s = p.rsrc + 3 * ray, *d = p.rdst + 3 * ray;
        S = mk(__ldg(s), __ldg(s + 1), __ldg(s + 2));
        P = mk(__ldg(d), __ldg(d + 1), __ldg(d + 2));
    }
}

__device__ __forceinline__ void morton_local(int t, int bx, int by, int &x, int &y) {
    x = 0;
    y = 0;
    int ix = 0, iy = 0, bit = 0;
    while (ix < bx || iy < by) {
        if (ix < bx) { x |= ((t >> bit) & 1) << ix; ++ix; ++bit; }
        if (iy < by) { y |= ((t >> bit) & 1) << iy; ++iy; ++bit; }
    }
}

// Ray of this thread in tile / ray block `b` (cone tiles are enumerated
// tile_u fastest, then tile_v, then angle).
// Ray of in-tile thread t of tile b (cone tiles), or of thread t of block b
// (explicit rays, blocks of blockDim.x rays).
__device__ __forceinline__ bool thread_ray_at(const KParams &p, int64_t b, int t, int64_t &ray) {
    if (p.src_kind == 0) {
        int lu, lv;
        if (p.morton) morton_local(t, p.log_tu, p.log_tv, lu, lv);
        else { lu = t & (p.tu - 1); lv = t >> p.log_tu; }
        int tid_u = (int)(b % p.tiles_u);
        int64_t rest = b / p.tiles_u;
        int tid_v = (int)(rest % p.tiles_v);
        int a = (int)(rest / p.tiles_v);
        int iu = tid_u * p.tu + lu, iv = tid_v * p.tv + lv;
        if (iu >= p.g.nu || iv >= p.g.nv || a >= p.g.na) return false;
        ray = ((int64_t)a * p.g.nv + iv) * p.g.nu + iu;
        return true;
    }
    ray = b * blockDim.x + t;
    return ray < p.nrays;
}

__device__ __forceinline__ bool thread_ray_in(const KParams &p, int64_t b, int64_t &ray) {
    return thread_ray_at(p, b, threadIdx.x, ray);
}

__device__ __forceinline__ bool thread_ray(const KParams &p, int64_t &ray) {
    return thread_ray_in(p, (int64_t)blockIdx.x + p.block_offset, ray);
}

// ---------------------------------------------------------- vector helpers

__device__ __forceinline__ f3 f3add(const f3 &a, const f3 &b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 f3axpy(float s, const f3 &x, const f3 &y) {
    return {fmaf(s, x.x, y.x), fmaf(s, x.y, y.y), fmaf(s, x.z, y.z)};
}
__device__ __forceinline__ d3 d3axpy(double s, const d3 &x, const d3 &y) {
    return {fma(s, x.x, y.x), fma(s, x.y, y.y), fma(s, x.z, y.z)};
}
__device__ __forceinline__ int sel4(const int4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
__device__ __forceinline__ d3 rec64_vertex(const TetRec64 *r, int k) {
    return mk(__ldg(&r->v[3 * k]), __ldg(&r->v[3 * k + 1]), __ldg(&r->v[3 * k + 2]));
}
// Exit face of the walk from the signs of side(n->a), side(n->b), side(n->c)
// (face opposite a, b or c; -1: none)
__host__ __device__ constexpr int exit_rule(int sa, int sb, int sc) {
    return (sb > 0 && sc < 0) ? 0 : (sc > 0 && sa < 0) ? 1 : (sa > 0 && sb < 0) ? 2 : -1;
}
// The same for three non-zero signs, as a table over the three "positive"
// bits: 2 bits per entry, 3 = none.
__host__ __device__ constexpr unsigned exit_rule_table() {
    unsigned t = 0;
    for (int c = 0; c < 8; ++c) {
        const int x = exit_rule(c & 1 ? 1 : -1, c & 2 ? 1 : -1, c & 4 ? 1 : -1);
        t |= (unsigned)(x < 0 ? 3 : x) << (2 * c);
    }
    return t;
}
constexpr unsigned EXIT_RULE_TABLE = exit_rule_table();
__device__ __forceinline__ int exit_rule_pos(bool pa, bool pb, bool pc) {
    const int v = (int)((EXIT_RULE_TABLE >> (2 * ((int)pa | (int)pb << 1 | (int)pc << 2))) & 3u);
    return v == 3 ? -1 : v;
}
__device__ __forceinline__ int filt_sign(float v, float B) { return (v > B) - (v < -B); }

// Accumulator reductions in the .global state space.  The accumulator
// pointers of the batched walk come from shared memory (the per-warp
// parameter slot), so the compiler cannot infer their space on its own.
__device__ __forceinline__ void red_add_global(float *a, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(a)), "f"(v));
}
__device__ __forceinline__ void red_add_global(float4 *a, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(__cvta_generic_to_global(a)),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w));
}
__device__ __forceinline__ void red_add_global(double *a, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(a)), "d"(v));
}

// ------------------------------------------------ robust (FP64+) fallbacks
//
// Used by both walks when a fast sign is uncertain.  They reload the exact
// FP64 inputs, finish the cascade, and compute the crossing point in FP64
// from barycentric weights; weights whose side product is exactly zero are 0,
// and a face whose three side products are exactly zero (the line lies in its
// plane) is crossed, in the limit of the perturbed line, at t = 1, i.e. at P.

// exact-or-symbolic sign of side(S,P,p,q) once the FP64 filter is known to be
// uncertain; *zero = 1 when the exact value is 0, *val = the exact value to a
// few ulps (the FP64 estimate can be all rounding error here, and the crossing
// point of a face nearly containing the ray depends on these tiny weights).
__device__ __noinline__ int side_exact_or_sos(const d3 S, const d3 P, const d3 p, const d3 q,
                                              int *zero, double *val, DevCounters *C) {
    atomicAdd(&C->exact, 1ull);
    int s = side_exact_sign(S, P, p, q, val);
    if (s != 0) { *zero = 0; return s; }
    atomicAdd(&C->sos, 1ull);
    *zero = 1;
    *val = 0.0;
    return side_sos_sign(S, P, p, q);
}

// Exit decision of one step in FP64.  known[j] != 0: sign already certain.
// Returns the exit index x (0..2 in face-triple order) or -1; X receives the
// exit point.
__device__ __noinline__ int step_robust(const KParams *p, int64_t ray, int h, int f,
                                        const int known[3], d3 *X) {
    d3 S, P;
    load_ray(*p, ray, S, P);
    DevCounters *C = p->m.counters;
    const TetRec64 *r = p->m.rec64 + h;
    int ia, ib, ic;
    face_triple(f, ia, ib, ic);
    d3 n = rec64_vertex(r, f);
    d3 k[3] = {rec64_vertex(r, ia), rec64_vertex(r, ib), rec64_vertex(r, ic)};
    d3 d = sub(P, S);
    Filt64Vert Vn = filt64_vert(S, d, n);
    double val[3], bnd[3];
    int sg[3], zero[3];
    for (int j = 0; j < 3; ++j) {
        int s = filt64_side(Vn, k[j], val[j], bnd[j]);
        zero[j] = 0;
        if (known[j] != 0) {
            sg[j] = known[j];
        } else if (s != 0) {
            sg[j] = s;
        } else {
            sg[j] = side_exact_or_sos(S, P, n, k[j], &zero[j], &val[j], C);
            bnd[j] = 0.0;
        }
    }
    int x = exit_rule(sg[0], sg[1], sg[2]);
    if (x < 0) return -1;
    int y = (x + 1) % 3, z = (x + 2) % 3;
    // weights of the exit face (n, k[y], k[z]): exact values where poorly determined
    for (int j = y; ; j = z) {
        if (!zero[j] && fabs(val[j]) < TP_WEIGHT_MARGIN * bnd[j])
            side_exact_or_sos(S, P, n, k[j], &zero[j], &val[j], C);
        if (j == z) break;
    }
    double wy = zero[z] ? 0.0 : fmax(0.0, -val[z]);
    double wz = zero[y] ? 0.0 : fmax(0.0, val[y]);
    Filt64Vert Vy = filt64_vert(S, d, k[y]);
    double vn, bn;
    filt64_side(Vy, k[z], vn, bn);
    double wn = fmax(0.0, vn);
    if (fabs(vn) < TP_WEIGHT_MARGIN * bn) {
        int zz;
        side_exact_or_sos(S, P, k[y], k[z], &zz, &vn, C);
        wn = zz ? 0.0 : fmax(0.0, vn);
    }
    double W = wn + wy + wz;
    if (W == 0.0) {
        *X = P;
    } else {
        double iw = 1.0 / W;
        d3 t = d3axpy(wy * iw, sub(k[y], n), n);
        *X = d3axpy(wz * iw, sub(k[z], n), t);
    }
    return x;
}

// Exit point of a step whose signs are certain but whose exit face the ray
// meets at a grazing angle.  The FP32 vertices carry rounding of ~u |v|, which
// moves the face plane by that much and the crossing by ~u |v| / sin(angle)
// along the ray (measured: 2e-5 at sin = 1e-3 on a unit cube); the FP64
// vertices and weights place it to FP64 accuracy.  Weights as in step_robust:
// exit face (n, k_y, k_z), w_y = -side(n->k_z), w_z = side(n->k_y),
// w_n = side(k_y->k_z).
__device__ __forceinline__ d3 crossing64d(const KParams &p, const d3 &S, const d3 &P, int h, int f,
                                          int x) {
    const TetRec64 *r = p.m.rec64 + h;
    int k3[3];
    face_triple(f, k3[0], k3[1], k3[2]);
    const d3 n = rec64_vertex(r, f);
    const d3 ky = rec64_vertex(r, k3[(x + 1) % 3]), kz = rec64_vertex(r, k3[(x + 2) % 3]);
    const d3 d = sub(P, S);
    const Filt64Vert Vn = filt64_vert(S, d, n), Vy = filt64_vert(S, d, ky);
    double sy, sz, sn;
    filt64_side(Vn, ky, sy);
    filt64_side(Vn, kz, sz);
    filt64_side(Vy, kz, sn);
    const double wy = fmax(0.0, -sz), wz = fmax(0.0, sy), wn = fmax(0.0, sn);
    const double W = wn + wy + wz;
    if (W == 0.0) return P;
    const double iw = 1.0 / W;
    return d3axpy(wz * iw, sub(kz, n), d3axpy(wy * iw, sub(ky, n), n));
}
// The same for the robust walk (which calls out of line anyway), in FP32.
__device__ __noinline__ f3 crossing64(const KParams *p, int64_t ray, int h, int f, int x) {
    d3 S, P;
    load_ray(*p, ray, S, P);
    return tof(crossing64d(*p, S, P, h, f, x));
}

// Entry point through boundary face (h, f) when its signs are certain but the
// ray meets it at a grazing angle (as crossing64): weights w_a = side(b->c),
// w_b = side(c->a), w_c = side(a->b) of the face triple in FP64.
__device__ __noinline__ f3 entry64(const KParams *p, int64_t ray, int h, int f) {
    d3 S, P;
    load_ray(*p, ray, S, P);
    const TetRec64 *r = p->m.rec64 + h;
    int ia, ib, ic;
    face_triple(f, ia, ib, ic);
    const d3 a = rec64_vertex(r, ia), b = rec64_vertex(r, ib), c = rec64_vertex(r, ic);
    const d3 d = sub(P, S);
    const Filt64Vert Va = filt64_vert(S, d, a), Vb = filt64_vert(S, d, b);
    double sab, sbc, sca;
    filt64_side(Va, b, sab);
    filt64_side(Vb, c, sbc);
    filt64_side(filt64_vert(S, d, c), a, sca);
    const double wa = fmax(0.0, sbc), wb = fmax(0.0, sca), wc = fmax(0.0, sab);
    const double W = wa + wb + wc;
    if (W == 0.0) return tof(a);
    const double iw = 1.0 / W;
    return tof(d3axpy(wc * iw, sub(c, a), d3axpy(wb * iw, sub(b, a), a)));
}

// Entry test of boundary face (h, f) in FP64 (+exact, symbolic).  known[j]:
// certain signs of side(a->b), side(b->c), side(c->a) or 0.  Returns 1 if the
// line enters the tet through the face, with the entry point in X.
__device__ __noinline__ int entry_robust(const KParams *p, int64_t ray, int h, int f,
                                         const int known[3], d3 *X, int count_fp64) {
    d3 S, P;
    load_ray(*p, ray, S, P);
    DevCounters *C = p->m.counters;
    const TetRec64 *r = p->m.rec64 + h;
    int ia, ib, ic;
    face_triple(f, ia, ib, ic);
    d3 v[3] = {rec64_vertex(r, ia), rec64_vertex(r, ib), rec64_vertex(r, ic)};
    d3 d = sub(P, S);
    double val[3], bnd[3];
    int zero[3];
    for (int j = 0; j < 3; ++j) {  // side(v_j -> v_{j+1})
        Filt64Vert Vj = filt64_vert(S, d, v[j]);
        int s = filt64_side(Vj, v[(j + 1) % 3], val[j], bnd[j]);
        zero[j] = 0;
        if (known[j] != 0) {
            s = known[j];
        } else {
            if (count_fp64) atomicAdd(&C->fp64, 1ull);
            if (s == 0) {
                s = side_exact_or_sos(S, P, v[j], v[(j + 1) % 3], &zero[j], &val[j], C);
                bnd[j] = 0.0;
            }
        }
        if (s < 0) return 0;
    }
    for (int j = 0; j < 3; ++j)
        if (!zero[j] && fabs(val[j]) < TP_WEIGHT_MARGIN * bnd[j])
            side_exact_or_sos(S, P, v[j], v[(j + 1) % 3], &zero[j], &val[j], C);
    // weights: w_a = side(b->c) = val[1], w_b = side(c->a) = val[2], w_c = side(a->b) = val[0]
    double wa = zero[1] ? 0.0 : fmax(0.0, val[1]);
    double wb = zero[2] ? 0.0 : fmax(0.0, val[2]);
    double wc = zero[0] ? 0.0 : fmax(0.0, val[0]);
    double W = wa + wb + wc;
    if (W == 0.0) {
        *X = P;
    } else {
        double iw = 1.0 / W;
        d3 t = d3axpy(wb * iw, sub(v[1], v[0]), v[0]);
        *X = d3axpy(wc * iw, sub(v[2], v[0]), t);
    }
    return 1;
}

// ------------------------------------------------------------- BVH search
//
// Depth-first, nearer child first, over boxes rounded outward to FP32 and
// widened per ray by 16u(|S| + mesh radius), with a relative slack on the
// interval test, so no box holding a face the exact line crosses is culled.
// The whole LINE is searched (no t >= 0 cut): a source inside the mesh enters
// through a face behind it, and the walk then clips its segments at t = 0.
// The top `smem_nodes` nodes (breadth-first numbering) come from shared memory.

__device__ __forceinline__ bool slab(const float4 &lo, const float4 &hi, const f3 &S, const f3 &inv,
                                     float m, float &tn) {
    float tx0 = (lo.x - m - S.x) * inv.x, tx1 = (hi.x + m - S.x) * inv.x;
    float ty0 = (lo.y - m - S.y) * inv.y, ty1 = (hi.y + m - S.y) * inv.y;
    float tz0 = (lo.z - m - S.z) * inv.z, tz1 = (hi.z + m - S.z) * inv.z;
    float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fminf(tz0, tz1));
    float tmax = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
    tn = tmin;
    return tmin <= tmax + 1e-5f * fabsf(tmax) + 1e-7f;
}

__device__ __forceinline__ f3 safe_inv(const f3 &d) {
    auto s = [](float x) { return fabsf(x) < 1e-30f ? (x < 0.f ? -1e30f : 1e30f) : 1.f / x; };
    return {s(d.x), s(d.y), s(d.z)};
}

// Generic DFS; FaceTest(q, found) tests boundary face q and returns true to stop.
template <class FaceTest>
__device__ __forceinline__ void bvh_search(const MeshView &m, const BvhNode *snodes, int nsm,
                                           const f3 &S, const f3 &inv, float margin,
                                           LocalCnt &cnt, FaceTest &&test) {
    int stack[48];
    int sp = 0;
    int code = m.root;
    while (true) {
        if (code >= 0) {
            BvhNode n;
            if (code < nsm) {
                n = snodes[code];
            } else {
                const float4 *g = reinterpret_cast<const float4 *>(m.bvh + code);
                n.lmin = __ldg(g);
                n.lmax = __ldg(g + 1);
                n.rmin = __ldg(g + 2);
                n.rmax = __ldg(g + 3);
            }
            cnt.nodes += 2;
            float tl, tr;
            bool hl = slab(n.lmin, n.lmax, S, inv, margin, tl);
            bool hr = slab(n.rmin, n.rmax, S, inv, margin, tr);
            int cl = __float_as_int(n.lmin.w), cr = __float_as_int(n.rmin.w);
            if (hl && hr) {
                if (tl <= tr) { code = cl; if (sp < 48) stack[sp++] = cr; }
                else { code = cr; if (sp < 48) stack[sp++] = cl; }
                continue;
            }
            if (hl) { code = cl; continue; }
            if (hr) { code = cr; continue; }
        } else {
            int first = (~code) >> 3, count = (~code) & 7;
            for (int q = first; q < first + count; ++q) {
                ++cnt.faces;
                if (test(q)) return;
            }
        }
        if (sp == 0) return;
        code = stack[--sp];
    }
}

// R*-tree depth-first search (the paper's entry search, Sec. II-E): children
// whose boxes the ray meets are pushed; FaceTest(q) tests boundary face q and
// returns true to stop.  The stack holds 9 * depth + 1 <= 109 entries.
template <class FaceTest>
__device__ __forceinline__ void rstar_search(const MeshView &m, const f3 &S, const f3 &inv,
                                             float margin, LocalCnt &cnt, FaceTest &&test) {
    int stack[9 * RSTAR_MAX_DEPTH + 1];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const RStarNode *n = m.rstar + stack[--sp];
        const int count = __ldg(&n->count), leaf = __ldg(&n->leaf);
        for (int k = 0; k < count; ++k) {
            const float4 lo = make_float4(__ldg(&n->lo[0][k]), __ldg(&n->lo[1][k]),
                                          __ldg(&n->lo[2][k]), 0.f);
            const float4 hi = make_float4(__ldg(&n->hi[0][k]), __ldg(&n->hi[1][k]),
                                          __ldg(&n->hi[2][k]), 0.f);
            ++cnt.nodes;
            float tn;
            if (!slab(lo, hi, S, inv, margin, tn)) continue;
            const int c = __ldg(&n->child[k]);
            if (leaf) {
                ++cnt.faces;
                if (test(c)) return;
            } else if (sp < 9 * RSTAR_MAX_DEPTH + 1) {
                stack[sp++] = c;
            }
        }
    }
}

// ======================================================= filtered FP32 walk
//
// Two kernels share one body.  The FAST kernel (ROBUST = false) takes only
// decisions the FP32 filter certifies; a ray that meets an undecided side
// product (or an undecided entry face) stops, and when the warp's walk loop
// ends it is appended to the deferral queue with its walk state.  The fast
// kernel therefore contains no call to the FP64 / exact / symbolic stages;
// it is capped at 56 registers (no spills), so 36 warps fit on an SM.  The
// RESUME kernel (ROBUST = true) continues each queued walk from that state
// with the full cascade.  Every decision the fast kernel took was exact, so
// the two parts together visit the same tets, in the same order, as one
// robust walk.  (Running the FP64 steps in place, inside the fast warps, was
// measured 1.7x slower on the full-size workload: GB300's FP64 rate is low and
// the other 31 lanes wait.)

// Warp-aggregated append to the deferral queue.  All 32 lanes must call it
// (converged); lanes with want = true write their entry.
template <int C>
__device__ __forceinline__ void defer_append(const KParams &p, bool want, int64_t ray, int h,
                                             int fs, const f3 &X, int nvis, const float *acc,
                                             const float *comp) {
    unsigned m = __ballot_sync(FULL_MASK, want);
    if (!m) return;
    ray |= p.qtag;  // read only when some lane defers
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(p.q_count, (unsigned long long)__popc(m));
    base = __shfl_sync(FULL_MASK, base, leader);
    if (want) {
        unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
        if (slot < (unsigned long long)p.q_cap) {
            QEntry *e = p.q + slot;
            e->ray = ray;
            e->h = h;
            e->fs = fs;
            e->x = make_float4(X.x, X.y, X.z, __int_as_float(nvis));
            e->acc = make_float4(acc[0], acc[1 % C], acc[2 % C], acc[3 % C]);
            e->comp = make_float4(comp[0], comp[1 % C], comp[2 % C], comp[3 % C]);
        } else {
            report_error(p.m.counters, TETPROJ_ERR_TOO_LARGE);  // host sizes chunks <= capacity
        }
    }
}

// Queues the FP64 correction of a grazing crossing (see XFix); false when the
// chunk's fix list is full.  Called in divergent code: the lanes that arrive
// together share one atomic on the list's counter.
__device__ __forceinline__ bool xfix_append(const KParams &p, int64_t ray, int h, int hn,
                                            const f3 &X, int fx) {
    const unsigned long long cap = (unsigned long long)(p.q_cap / 2);
    const unsigned m = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(p.q_count + 1, (unsigned long long)__popc(m));
    base = __shfl_sync(m, base, leader);
    const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
    if (slot >= cap) return false;
    XFix *e = queue_fixes(p.q, p.q_cap) + slot;
    e->ray = ray | p.qtag;
    e->h = h;
    e->hn = hn;
    e->x = X.x;
    e->y = X.y;
    e->z = X.z;
    e->fx = fx;
    return true;
}

// First segment-buffer slot of cone ray `ray` (MODE_SEG): its tile block's
// offset, minus the chunk's base, plus the ray's offset inside the block.
__device__ __forceinline__ int64_t seg_slot(const KParams &p, int64_t ray) {
    const int64_t t = ray / p.g.nu;
    const int iu = (int)(ray - t * p.g.nu);
    const int64_t a = t / p.g.nv;
    const int iv = (int)(t - a * p.g.nv);
    const int64_t b = (a * p.tiles_v + (iv >> p.log_tv)) * p.tiles_u + (iu >> p.log_tu);
    return __ldg(p.block_off + b) - p.seg_base + __ldg(p.ray_off + ray);
}

// One filtered walk.  Fast kernel (ROBUST = false): `valid` rays start from
// scratch.  Resume kernel (ROBUST = true): `qe` is the ray's queue entry; the
// walk continues from the saved state (or from the entry search when the ray
// was deferred there).
template <int C, int MODE, bool ROBUST, int ENTRY = ENTRY_BVH>
__device__ __forceinline__ void walk32_ray(const KParams &p, const BvhNode *snodes, int nsm,
                                           int64_t ray, const bool valid, const QEntry *qe) {
    LocalCnt cnt = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    Filt32Ray fr;
    f3 Xin = {0.f, 0.f, 0.f};
    float il = 0.f;  // 1 / |d|
    int h = 0, f = 0, err = 0, steps = 0, nvis = 0;
    bool alive = false, deferred = false, clip0 = false;
    float acc[C], comp[C], yv[C];
#pragma unroll
    for (int c = 0; c < C; ++c) { acc[c] = 0.f; comp[c] = 0.f; yv[c] = 0.f; }

    if (valid) {
        d3 S, P;
        load_ray(p, ray, S, P);
        fr = filt32_ray(S, P, p.m.radius);
        il = rsqrtf(dotf(fr.d, fr.d));
        const bool from_entry = !ROBUST || qe->fs < 0;
        if (!ROBUST) cnt.rays = 1;
        if (from_entry) {
            f3 inv = safe_inv(fr.d);
            f3 S32 = tof(S);
            float smax = fmaxf(fmaxf(fabsf(S32.x), fabsf(S32.y)), fabsf(S32.z));
            float margin = 16.f * 5.9604645e-8f * (smax + p.m.radius);
            auto entry_test = [&](int q) -> bool {
                const float4 *g = reinterpret_cast<const float4 *>(p.m.bfaces + q);
                float4 A = __ldg(g), B = __ldg(g + 1), Cc = __ldg(g + 2);
                f3 a = {A.x, A.y, A.z}, b = {B.x, B.y, B.z}, c = {Cc.x, Cc.y, Cc.z};
                float sab, sbc, sca, bab, bbc, bca;
                int gab = filt32_side(filt32_vert(fr, a), b, sab, bab);
                if (gab < 0) return false;
                int gbc = filt32_side(filt32_vert(fr, b), c, sbc, bbc);
                if (gbc < 0) return false;
                int gca = filt32_side(filt32_vert(fr, c), a, sca, bca);
                if (gca < 0) return false;
                int hf = __float_as_int(A.w);
                if (gab > 0 && gbc > 0 && gca > 0 &&
                    sab + sbc + sca >= (float)TP_WEIGHT_MARGIN * (bab + bbc + bca)) {
                    const f3 N = crossf(sub(b, a), sub(c, a));
                    if ((sab + sbc + sca) * il * (1.0f / TP_GRAZE_SIN) <
                        fabsf(N.x) + fabsf(N.y) + fabsf(N.z)) {
                        // grazing entry face: the entry point comes from the FP64
                        // records, in the robust walk
                        if (!ROBUST) {
                            deferred = true;
                            h = -1;
                            return true;
                        }
                        Xin = entry64(&p, ray, hf >> 2, hf & 3);
                    } else {
                        float iw = __frcp_rn(sab + sbc + sca);
                        Xin = f3axpy(sca * iw, sub(b, a), f3axpy(sab * iw, sub(c, a), a));
                    }
                } else if (!ROBUST) {
                    deferred = true;  // undecided entry face: finish the ray robustly
                    h = -1;           // (queued with fs = -1: resume from the entry search)
                    return true;
                } else {
                    int known[3] = {gab, gbc, gca};
                    d3 X;
                    if (!entry_robust(&p, ray, hf >> 2, hf & 3, known, &X, 1)) return false;
                    Xin = tof(X);
                }
                h = hf >> 2;
                f = hf & 3;
                alive = true;
                return true;
            };
            if (ENTRY == ENTRY_RSTAR) {
                rstar_search(p.m, S32, inv, margin, cnt, entry_test);
            } else {
                // the face the entry map drew at this ray's pixel, if it is the one
                bool found = false;
                if (!ROBUST && p.emap) {
                    const int64_t r = ray - p.emap_base;
                    const int q = (r >= 0 && r < p.emap_len) ? __ldg(p.emap + r) : -1;
                    if (q >= 0 && q < p.m.nb) {
                        ++cnt.faces;
                        found = entry_test(q);
                    }
                }
                if (!found) bvh_search(p.m, snodes, nsm, S32, inv, margin, cnt, entry_test);
            }
            if (alive) {
                cnt.hits = 1;
                // entry behind the source (source inside the mesh, or the mesh behind
                // it): t_in = 1/2 + (X_in - O).d / |d|^2 < 0, clip segments at t = 0
                clip0 = dotf(sub(Xin, fr.O), fr.d) < -0.5f * dotf(fr.d, fr.d);
            }
        } else {
            // continue where the fast kernel stopped
            h = qe->h;
            f = qe->fs & 3;
            clip0 = (qe->fs >> 2) & 1;
            steps = qe->fs >> 3;
            float4 x = qe->x;
            Xin = {x.x, x.y, x.z};
            nvis = __float_as_int(x.w);
            float4 a4 = qe->acc, c4 = qe->comp;
            acc[0] = a4.x; comp[0] = c4.x;
            if (C == 4) {
                acc[1 % C] = a4.y; acc[2 % C] = a4.z; acc[3 % C] = a4.w;
                comp[1 % C] = c4.y; comp[2 % C] = c4.z; comp[3 % C] = c4.w;
            }
            alive = true;
        }
        if ((MODE == MODE_BWD || MODE == MODE_SEG || MODE == MODE_BWD64) && alive) {
            const float *y = reinterpret_cast<const float *>(p.in) + ray * C;
#pragma unroll
            for (int c = 0; c < C; ++c) yv[c] = __ldg(y + c);
        }
    }
    if (MODE == MODE_ENTRY) {  // entry search only
        if (valid && !deferred) p.tr_count[ray] = alive ? __ldg(p.m.perm + h) : -1;
        alive = false;
    }
    // MODE_SEG: this ray's next slot in the segment buffer
    int64_t spos = 0;
    if (MODE == MODE_SEG && valid) spos = seg_slot(p, ray) + steps;
    flush_counters(p.m.counters, cnt);
    cnt = {0, 0, 0, 0, 0, 0, 0, 0, 0};

    const TetRec32 *rec = p.m.rec32;
    const float *mu = reinterpret_cast<const float *>(p.in);
    float *accbuf = reinterpret_cast<float *>(p.out);
    const int lane = threadIdx.x & 31;

    while (__any_sync(FULL_MASK, alive)) {
        bool did = alive;
        const int hcur = h;
        bool defer_now = false;
        float len = 0.f;
        if (alive) {
            // n = v_f and face f's canonical triple (a, b, c), loaded by index;
            // the .w of a, b, c are the neighbours across the faces opposite them
            const float4 *R4 = rec->v;
            const unsigned h4 = (unsigned)h << 2, tri = (FACE_TRIPLES >> (6 * f)) & 63;
            const float4 vn = __ldg(R4 + (h4 | f)), va = __ldg(R4 + (h4 | (tri & 3))),
                         vb = __ldg(R4 + (h4 | ((tri >> 2) & 3))), vc = __ldg(R4 + (h4 | (tri >> 4)));
            float muv[C];
            if (MODE == MODE_FWD) {
                if (C == 4) {
                    float4 m4 = __ldg(reinterpret_cast<const float4 *>(mu) + h);
                    muv[0] = m4.x; muv[1 % C] = m4.y; muv[2 % C] = m4.z; muv[3 % C] = m4.w;
                } else {
                    muv[0] = __ldg(mu + h);
                }
            }
            const f3 n = {vn.x, vn.y, vn.z}, a = {va.x, va.y, va.z}, b = {vb.x, vb.y, vb.z},
                     c = {vc.x, vc.y, vc.z};
            Filt32Vert Vn = filt32_vert(fr, n);
            f3 ea = sub(a, n), eb = sub(b, n), ec = sub(c, n);
            float sa, sb, sc, ba, bb, bc;
            filt32_side_e(Vn, ea, sa, ba);
            filt32_side_e(Vn, eb, sb, bb);
            filt32_side_e(Vn, ec, sc, bc);
            int x = -1;
            f3 Xout = Xin;
            // all three signs certain: each side exceeds its error bound
            bool fast = (fabsf(sa) > ba) & (fabsf(sb) > bb) & (fabsf(sc) > bc);
            if (fast) {
                x = exit_rule_pos(sa > 0.f, sb > 0.f, sc > 0.f);
                // exit face (n, y, z): barycentric weights w_y = -side(n->z),
                // w_z = side(n->y), and their sum = d . ((y - n) x (z - n))
                const bool x0 = x == 0, x1 = x == 1;
                f3 ey = x0 ? eb : (x1 ? ec : ea), ez = x0 ? ec : (x1 ? ea : eb);
                float wy = x0 ? -sc : (x1 ? -sa : -sb), wz = x0 ? sb : (x1 ? sc : sa);
                float bw = x0 ? bc + bb : (x1 ? ba + bc : bb + ba);
                const f3 N = crossf(ey, ez);
                float W = dotf(fr.d, N);
                // the crossing nearly coincides with a vertex or edge of the
                // exit face (weights within the margin of their bounds):
                // finish the ray robustly
                fast = x < 0 || wy + wz >= (float)TP_WEIGHT_MARGIN * bw;
                if (fast) {
                    // approximate reciprocal (2 ulp): W only scales the crossing
                    // offset, whose weights carry far larger certified errors
                    float iw = __fdividef(1.0f, W);
                    Xout = f3axpy(wz * iw, ez, f3axpy(wy * iw, ey, n));
                    // grazing exit face: |W| / |d| = |N| sin(angle); with the 1-norm
                    // of N this flags every sine below TP_GRAZE_SIN (and some up to
                    // sqrt(3) times it)
                    if (x >= 0 && fabsf(W) * il * (1.0f / TP_GRAZE_SIN) <
                                      fabsf(N.x) + fabsf(N.y) + fabsf(N.z)) {
                        ++cnt.graze;
                        if (ROBUST || (MODE != MODE_FWD && MODE != MODE_BWD && MODE != MODE_BWD64)) {
                            Xout = crossing64(&p, ray, h, f, x);
                        } else {
                            // keep the FP32 crossing and queue its FP64 correction; a ray
                            // whose segment is clipped at t = 0 here, or that finds the
                            // fix list full, is finished by the robust walk instead
                            const int nx = __float_as_int(x == 0 ? va.w : (x == 1 ? vb.w : vc.w));
                            defer_now = clip0 || !xfix_append(p, ray, h, nx < 0 ? -1 : nx >> 2, Xout,
                                                              f | (x << 2));
                        }
                    }
                }
            }
            if (!fast) {
                if (!ROBUST) {
                    defer_now = true;
                } else {
                    const int ga = filt_sign(sa, ba), gb = filt_sign(sb, bb), gc = filt_sign(sc, bc);
                    cnt.fp64 += (ga == 0) + (gb == 0) + (gc == 0);
                    int known[3] = {ga, gb, gc};
                    d3 X;
                    x = step_robust(&p, ray, h, f, known, &X);
                    Xout = tof(X);
                }
            }
            if (defer_now) {
                alive = false;
                did = false;
                deferred = true;
            } else if (x < 0) {
                err = TETPROJ_ERR_RAY_LIMIT;
                alive = false;
                did = false;
            } else {
                ++cnt.segs;
                // the exit face is opposite a (x = 0), b (1) or c (2)
                const int nxt = __float_as_int(x == 0 ? va.w : (x == 1 ? vb.w : vc.w));
                len = dotf(sub(Xout, Xin), fr.d) * il;
                if (clip0) {  // only the part with t >= 0 counts
                    float dd = dotf(fr.d, fr.d);
                    float ti = 0.5f + dotf(sub(Xin, fr.O), fr.d) / dd;
                    float to = 0.5f + dotf(sub(Xout, fr.O), fr.d) / dd;
                    len = fmaxf(0.f, to - fmaxf(ti, 0.f)) * sqrtf(dd);
                    clip0 = to < 0.f;
                }
                if (MODE == MODE_FWD) {
#pragma unroll
                    for (int cc = 0; cc < C; ++cc) {  // Kahan
                        float yk = muv[cc] * len - comp[cc];
                        float t = acc[cc] + yk;
                        comp[cc] = (t - acc[cc]) - yk;
                        acc[cc] = t;
                    }
                }
                if (MODE == MODE_TRACE) {
                    if (nvis < p.max_visits) {
                        p.tr_tet[ray * p.max_visits + nvis] = __ldg(p.m.perm + h);
                        p.tr_len[ray * p.max_visits + nvis] = (double)len;
                    }
                    ++nvis;
                }
                ++steps;
                Xin = Xout;
                if (nxt < 0) {
                    alive = false;
                } else {
                    h = nxt >> 2;
                    f = nxt & 3;
                    if (steps >= p.max_steps) {
                        err = TETPROJ_ERR_RAY_LIMIT;
                        alive = false;
                    }
                }
            }
        }
        if (MODE == MODE_SEG && did) {
            if (spos >= 0 && spos < p.seg_cap) {
                if (C == 4) {
                    p.seg_key[spos] = (uint32_t)hcur;
                    reinterpret_cast<float4 *>(p.seg_val)[spos] =
                        make_float4(len * yv[0], len * yv[1 % C], len * yv[2 % C], len * yv[3 % C]);
                } else {
                    reinterpret_cast<uint2 *>(p.seg_key)[spos] =
                        make_uint2((uint32_t)hcur, __float_as_uint(len * yv[0]));
                }
            } else {
                err = TETPROJ_ERR_TOO_LARGE;  // the plan's counts disagree with this walk
                alive = false;
            }
            ++spos;
        }
        if (MODE == MODE_BWD64) {  // FP64 accumulation: no drift with many segments
            if (!ROBUST && p.scatter == TETPROJ_SCATTER_WARP) {
                // lanes at the same tet add their contributions in FP64 first
                // (in lane order), then one reduction per tet and channel
                unsigned peers = __match_any_sync(FULL_MASK, did ? hcur : -1 - lane);
                if (did) {
                    double v[C];
#pragma unroll
                    for (int cc = 0; cc < C; ++cc) v[cc] = (double)(len * yv[cc]);
                    if (__popc(peers) > 1) {
                        double t[C];
#pragma unroll
                        for (int cc = 0; cc < C; ++cc) t[cc] = 0.0;
                        unsigned mm = peers;
                        while (mm) {
                            const int src = __ffs(mm) - 1;
                            mm &= mm - 1;
#pragma unroll
                            for (int cc = 0; cc < C; ++cc) t[cc] += __shfl_sync(peers, v[cc], src);
                        }
#pragma unroll
                        for (int cc = 0; cc < C; ++cc) v[cc] = t[cc];
                    }
                    if (lane == __ffs(peers) - 1) {
                        double *acc64 = reinterpret_cast<double *>(p.out) + (int64_t)hcur * C;
#pragma unroll
                        for (int cc = 0; cc < C; ++cc) red_add_global(acc64 + cc, v[cc]);
                    }
                }
            } else if (did) {
                double *acc64 = reinterpret_cast<double *>(p.out) + (int64_t)hcur * C;
#pragma unroll
                for (int cc = 0; cc < C; ++cc) red_add_global(acc64 + cc, (double)(len * yv[cc]));
            }
        }
        if (MODE == MODE_BWD) {
            if (!ROBUST && p.scatter == TETPROJ_SCATTER_WARP) {
                unsigned peers = __match_any_sync(FULL_MASK, did ? hcur : -1 - lane);
                if (did) {
                    float v[C];
#pragma unroll
                    for (int cc = 0; cc < C; ++cc) v[cc] = len * yv[cc];
                    if (__popc(peers) > 1) {
                        float s[C];
#pragma unroll
                        for (int cc = 0; cc < C; ++cc) s[cc] = 0.f;
                        unsigned mm = peers;
                        while (mm) {
                            int src = __ffs(mm) - 1;
                            mm &= mm - 1;
#pragma unroll
                            for (int cc = 0; cc < C; ++cc) s[cc] += __shfl_sync(peers, v[cc], src);
                        }
#pragma unroll
                        for (int cc = 0; cc < C; ++cc) v[cc] = s[cc];
                    }
                    if (lane == __ffs(peers) - 1) {
                        if (C == 4)
                            red_add_global(reinterpret_cast<float4 *>(accbuf) + hcur,
                                           make_float4(v[0], v[1 % C], v[2 % C], v[3 % C]));
                        else
                            red_add_global(accbuf + hcur, v[0]);
                    }
                }
            } else if (did) {
                if (C == 4)
                    red_add_global(reinterpret_cast<float4 *>(accbuf) + hcur,
                                   make_float4(len * yv[0], len * yv[1 % C], len * yv[2 % C],
                                               len * yv[3 % C]));
                else
                    red_add_global(accbuf + hcur, len * yv[0]);
            }
        }
    }
    // rays that stopped at an uncertain decision go to the resume kernel with
    // their walk state (h, f, clip flag, step count, entry point, partial sums;
    // none of these changes once a lane defers), or with fs = -1 when the
    // entry face itself was uncertain
    if (!ROBUST)
        defer_append<C>(p, deferred, ray, h < 0 ? 0 : h,
                        h < 0 ? -1 : f | ((int)clip0 << 2) | (steps << 3), Xin, nvis, acc, comp);

    if (valid && !deferred) {
        if (MODE == MODE_FWD) {
            float *o = reinterpret_cast<float *>(p.out) + ray * C;
            if (C == 4) {
                float4 r4 = err ? make_float4(NAN, NAN, NAN, NAN)
                                : make_float4(acc[0], acc[1 % C], acc[2 % C], acc[3 % C]);
                *reinterpret_cast<float4 *>(o) = r4;
            } else {
                o[0] = err ? NAN : acc[0];
            }
        }
        if (MODE == MODE_TRACE) p.tr_count[ray] = err ? -1 : nvis;
        if (err) report_error(p.m.counters, err);
    }
    if (!ROBUST) {
        // rays handed to the resume kernel
        unsigned dm = __ballot_sync(FULL_MASK, valid && deferred);
        if ((threadIdx.x & 31) == 0 && dm) atomicAdd(&p.m.counters->deferred, (unsigned long long)__popc(dm));
    }
    flush_counters(p.m.counters, cnt);
}

__device__ __forceinline__ const BvhNode *stage_bvh_top(const KParams &p, float4 *smem) {
    for (int i = threadIdx.x; i < p.smem_nodes * 4; i += blockDim.x)
        smem[i] = __ldg(reinterpret_cast<const float4 *>(p.m.bvh) + i);
    __syncthreads();
    return reinterpret_cast<const BvhNode *>(smem);
}

template <int C, int MODE, int ENTRY = ENTRY_BVH>
__global__ void __maxnreg__(56) k_walk32(const __grid_constant__ KParams p) {
    extern __shared__ float4 smem[];
    const BvhNode *snodes = stage_bvh_top(p, smem);
    int64_t ray = 0;
    const bool valid = thread_ray(p, ray);
    walk32_ray<C, MODE, false, ENTRY>(p, snodes, p.smem_nodes, ray, valid, nullptr);
}

// Resume kernel: grid-stride over the queued rays (count set by k_walk32).
template <int C, int MODE>
__global__ void __launch_bounds__(128, 4) k_resume32(const __grid_constant__ KParams p) {
    extern __shared__ float4 smem[];
    const BvhNode *snodes = stage_bvh_top(p, smem);
    // entries past the capacity were never written (the append reported an error)
    const unsigned long long n = min(*p.q_count, (unsigned long long)p.q_cap);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n;
         base += stride) {
        const unsigned long long k = base + threadIdx.x;
        const bool valid = k < n;
        const QEntry *qe = p.q + (valid ? k : 0);
        int64_t ray = valid ? qe->ray : 0;
        walk32_ray<C, MODE, true>(p, snodes, p.smem_nodes, ray, valid, qe);
    }
}

// Correction of one queued grazing crossing (see XFix): the crossing placed
// again from the FP64 records moves by delta along the ray, so the segment
// that ends there (tet h) grows by delta and the one that starts there (tet
// hn) shrinks by it.  Forward: proj += delta (mu_h - mu_hn); backward:
// acc_h += delta y, acc_hn -= delta y.
template <int C, int MODE>
__device__ __forceinline__ void fix_apply(const KParams &p, const XFix &r) {
    const int64_t ray = r.ray & ((int64_t(1) << 40) - 1);  // drop a batched launch's problem tag
    d3 S, P;
    load_ray(p, ray, S, P);
    const d3 X = crossing64d(p, S, P, r.h, r.fx & 3, r.fx >> 2);
    const d3 d = sub(P, S);
    const double delta = ((X.x - (double)r.x) * d.x + (X.y - (double)r.y) * d.y +
                          (X.z - (double)r.z) * d.z) / sqrt(dotd(d, d));
    if (MODE == MODE_FWD) {
        const float *mu = reinterpret_cast<const float *>(p.in);
        float *o = reinterpret_cast<float *>(p.out) + ray * C;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const double dm = (double)__ldg(mu + (int64_t)r.h * C + c) -
                              (r.hn >= 0 ? (double)__ldg(mu + (int64_t)r.hn * C + c) : 0.0);
            atomicAdd(o + c, (float)(delta * dm));
        }
    } else if (MODE == MODE_BWD) {
        const float *y = reinterpret_cast<const float *>(p.in) + ray * C;
        float *acc = reinterpret_cast<float *>(p.out);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float v = (float)(delta * (double)__ldg(y + c));
            red_add_global(acc + (int64_t)r.h * C + c, v);
            if (r.hn >= 0) red_add_global(acc + (int64_t)r.hn * C + c, -v);
        }
    } else if (MODE == MODE_BWD64) {
        const float *y = reinterpret_cast<const float *>(p.in) + ray * C;
        double *acc = reinterpret_cast<double *>(p.out);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const double v = delta * (double)__ldg(y + c);
            red_add_global(acc + (int64_t)r.h * C + c, v);
            if (r.hn >= 0) red_add_global(acc + (int64_t)r.hn * C + c, -v);
        }
    }
}

// The fixes a chunk's fast walk queued (after its resume kernel, which may
// still write the forward results of deferred rays).
template <int C, int MODE>
__global__ void __launch_bounds__(128) k_fix32(const __grid_constant__ KParams p) {
    const XFix *xf = queue_fixes(p.q, p.q_cap);
    const unsigned long long n = min(p.q_count[1], (unsigned long long)(p.q_cap / 2));
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += stride)
        fix_apply<C, MODE>(p, xf[k]);
}

// Modes whose fast walk queues crossing fixes (the others place grazing
// crossings in FP64 in place).
template <int MODE>
constexpr bool queues_fixes() {
    return MODE == MODE_FWD || MODE == MODE_BWD || MODE == MODE_BWD64;
}

template <int C, int MODE>
static cudaError_t launch_fix(const KParams &p, unsigned grid, cudaStream_t stream) {
    if constexpr (queues_fixes<MODE>()) {
        k_fix32<C, MODE><<<grid, 128, 0, stream>>>(p);
        note_launch();
        return cudaGetLastError();
    }
    return cudaSuccess;
}

// ========================================================= plain FP64 walk

// FP64 sign of side(n->k) for the plain path: FP64 filter, then exact/SoS.
__device__ __forceinline__ int side64_plain(const Filt64Vert &Vn, const d3 &k, double &val,
                                            int &zero) {
    zero = 0;
    return filt64_side(Vn, k, val);
}

template <int C, int MODE>
__global__ void __launch_bounds__(256) k_walk64(const __grid_constant__ KParams p) {
    extern __shared__ float4 smem[];
    const int nsm = p.smem_nodes;
    for (int i = threadIdx.x; i < nsm * 4; i += blockDim.x)
        smem[i] = __ldg(reinterpret_cast<const float4 *>(p.m.bvh) + i);
    __syncthreads();
    const BvhNode *snodes = reinterpret_cast<const BvhNode *>(smem);

    LocalCnt cnt = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int64_t ray = 0;
    const bool valid = thread_ray(p, ray);
    d3 S = {0, 0, 0}, d = {0, 0, 0}, dhat = {0, 0, 0}, Xin = {0, 0, 0};
    int h = 0, f = 0, err = 0, steps = 0, nvis = 0;
    bool alive = false, clip0 = false;
    double acc[C], yv[C];
#pragma unroll
    for (int c = 0; c < C; ++c) { acc[c] = 0.0; yv[c] = 0.0; }

    if (valid) {
        cnt.rays = 1;
        d3 P;
        load_ray(p, ray, S, P);
        d = sub(P, S);
        double il = 1.0 / sqrt(dotd(d, d));
        dhat = {d.x * il, d.y * il, d.z * il};
        f3 S32 = tof(S), d32 = tof(d);
        f3 inv = safe_inv(d32);
        float smax = fmaxf(fmaxf(fabsf(S32.x), fabsf(S32.y)), fabsf(S32.z));
        float margin = 16.f * 5.9604645e-8f * (smax + p.m.radius);
        bvh_search(p.m, snodes, nsm, S32, inv, margin, cnt, [&](int q) -> bool {
            int hf = __float_as_int(__ldg(reinterpret_cast<const float *>(p.m.bfaces + q) + 3));
            int hh = hf >> 2, ff = hf & 3;
            const TetRec64 *r = p.m.rec64 + hh;
            int ia, ib, ic;
            face_triple(ff, ia, ib, ic);
            d3 v[3] = {rec64_vertex(r, ia), rec64_vertex(r, ib), rec64_vertex(r, ic)};
            double val[3], bnd[3];
            int known[3];
            bool unsure = false;
            for (int j = 0; j < 3; ++j) {
                int s = filt64_side(filt64_vert(S, d, v[j]), v[(j + 1) % 3], val[j], bnd[j]);
                if (s < 0) return false;
                known[j] = s;
                unsure |= (s == 0) || fabs(val[j]) < TP_WEIGHT_MARGIN * bnd[j];
            }
            if (!unsure) {
                double W = val[0] + val[1] + val[2], iw = 1.0 / W;
                Xin = d3axpy(val[0] * iw, sub(v[2], v[0]), d3axpy(val[2] * iw, sub(v[1], v[0]), v[0]));
            } else {
                d3 X;
                if (!entry_robust(&p, ray, hh, ff, known, &X, 0)) return false;
                Xin = X;
            }
            h = hh;
            f = ff;
            alive = true;
            return true;
        });
        if (alive) {
            cnt.hits = 1;
            clip0 = dotd(sub(Xin, S), d) < 0.0;  // entry behind the source: clip at t = 0
        }
        if (MODE == MODE_BWD && alive) {
            const double *y = reinterpret_cast<const double *>(p.in) + ray * C;
#pragma unroll
            for (int c = 0; c < C; ++c) yv[c] = __ldg(y + c);
        }
    }

    flush_counters(p.m.counters, cnt);
    cnt = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double *mu = reinterpret_cast<const double *>(p.in);
    double *accbuf = reinterpret_cast<double *>(p.out);
    const int lane = threadIdx.x & 31;

    while (__any_sync(FULL_MASK, alive)) {
        const bool did = alive;
        const int hcur = h;
        double len = 0.0;
        if (alive) {
            const TetRec64 *r = p.m.rec64 + h;
            const double2 *g = reinterpret_cast<const double2 *>(r);
            double2 e0 = __ldg(g), e1 = __ldg(g + 1), e2 = __ldg(g + 2);
            double2 e3 = __ldg(g + 3), e4 = __ldg(g + 4), e5 = __ldg(g + 5);
            int4 adj = __ldg(reinterpret_cast<const int4 *>(g + 6));
            d3 v0 = {e0.x, e0.y, e1.x}, v1 = {e1.y, e2.x, e2.y};
            d3 v2 = {e3.x, e3.y, e4.x}, v3 = {e4.y, e5.x, e5.y};
            double muv[C];
            if (MODE == MODE_FWD) {
#pragma unroll
                for (int cc = 0; cc < C; ++cc) muv[cc] = __ldg(mu + (int64_t)h * C + cc);
            }
            d3 n, a, b, c;
            if (f == 0) { n = v0; a = v1; b = v3; c = v2; }
            else if (f == 1) { n = v1; a = v0; b = v2; c = v3; }
            else if (f == 2) { n = v2; a = v0; b = v3; c = v1; }
            else { n = v3; a = v0; b = v1; c = v2; }
            Filt64Vert Vn = filt64_vert(S, d, n);
            double sa, sb, sc, ba, bb, bc;
            int ga = filt64_side(Vn, a, sa, ba);
            int gb = filt64_side(Vn, b, sb, bb);
            int gc = filt64_side(Vn, c, sc, bc);
            int x = -1;
            d3 Xout;
            bool fast = (ga != 0) & (gb != 0) & (gc != 0);
            d3 y, z;
            double wy, wz, bw, wn = 0.0;
            if (fast) {
                x = exit_rule(ga, gb, gc);
                if (x == 0) { y = b; z = c; wy = -sc; wz = sb; bw = bc + bb; }
                else if (x == 1) { y = c; z = a; wy = -sa; wz = sc; bw = ba + bc; }
                else { y = a; z = b; wy = -sb; wz = sa; bw = bb + ba; }
                double vn, bn;
                filt64_side(filt64_vert(S, d, y), z, vn, bn);
                wn = fmax(vn, 0.0);
                // weights near their error bounds: the ray nearly lies in the exit face
                fast = x < 0 || (wy + wz >= TP_WEIGHT_MARGIN * bw && fabs(vn) >= TP_WEIGHT_MARGIN * bn);
            }
            if (fast) {
                double iw = 1.0 / (wn + wy + wz);
                Xout = d3axpy(wz * iw, sub(z, n), d3axpy(wy * iw, sub(y, n), n));
            } else {
                int known[3] = {ga, gb, gc};
                x = step_robust(&p, ray, h, f, known, &Xout);
            }
            ++cnt.segs;
            if (x < 0) {
                err = TETPROJ_ERR_RAY_LIMIT;
                alive = false;
            } else {
                int ia, ib, ic;
                face_triple(f, ia, ib, ic);
                int loc = x == 0 ? ia : (x == 1 ? ib : ic);
                int nxt = sel4(adj, loc);
                len = dotd(sub(Xout, Xin), dhat);
                if (clip0) {  // only the part with t >= 0 counts
                    double dd = dotd(d, d);
                    double ti = dotd(sub(Xin, S), d) / dd, to = dotd(sub(Xout, S), d) / dd;
                    len = fmax(0.0, to - fmax(ti, 0.0)) * sqrt(dd);
                    clip0 = to < 0.0;
                }
                if (MODE == MODE_FWD) {
#pragma unroll
                    for (int cc = 0; cc < C; ++cc) acc[cc] = fma(muv[cc], len, acc[cc]);
                }
                if (MODE == MODE_TRACE) {
                    if (nvis < p.max_visits) {
                        p.tr_tet[ray * p.max_visits + nvis] = __ldg(&r->extra.x);
                        p.tr_len[ray * p.max_visits + nvis] = len;
                    }
                    ++nvis;
                }
                Xin = Xout;
                if (nxt < 0) {
                    alive = false;
                } else {
                    h = nxt >> 2;
                    f = nxt & 3;
                    if (++steps >= p.max_steps) {
                        err = TETPROJ_ERR_RAY_LIMIT;
                        alive = false;
                    }
                }
            }
        }
        if (MODE == MODE_BWD) {
            if (p.scatter == TETPROJ_SCATTER_WARP) {
                unsigned peers = __match_any_sync(FULL_MASK, did ? hcur : -1 - lane);
                if (did) {
                    double v[C];
#pragma unroll
                    for (int cc = 0; cc < C; ++cc) v[cc] = len * yv[cc];
                    if (__popc(peers) > 1) {
                        double s[C];
#pragma unroll
                        for (int cc = 0; cc < C; ++cc) s[cc] = 0.0;
                        unsigned mm = peers;
                        while (mm) {
                            int src = __ffs(mm) - 1;
                            mm &= mm - 1;
#pragma unroll
                            for (int cc = 0; cc < C; ++cc) s[cc] += __shfl_sync(peers, v[cc], src);
                        }
#pragma unroll
                        for (int cc = 0; cc < C; ++cc) v[cc] = s[cc];
                    }
                    if (lane == __ffs(peers) - 1) {
#pragma unroll
                        for (int cc = 0; cc < C; ++cc) atomicAdd(accbuf + (int64_t)hcur * C + cc, v[cc]);
                    }
                }
            } else if (did) {
#pragma unroll
                for (int cc = 0; cc < C; ++cc)
                    atomicAdd(accbuf + (int64_t)hcur * C + cc, len * yv[cc]);
            }
        }
    }

    if (valid) {
        if (MODE == MODE_FWD) {
            double *o = reinterpret_cast<double *>(p.out) + ray * C;
#pragma unroll
            for (int cc = 0; cc < C; ++cc) o[cc] = err ? NAN : acc[cc];
        }
        if (MODE == MODE_TRACE) p.tr_count[ray] = err ? -1 : nvis;
        if (err) report_error(p.m.counters, err);
    }
    flush_counters(p.m.counters, cnt);
}


static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// ============================================================ entry map

// Candidate entry faces for the cone rays of angles a0 .. a0 + gridDim.y - 1
// (KParams::emap).  A convex mesh seen from a source outside it projects onto
// the detector as the union of the projections of the boundary faces that
// face the source, and a ray entering through a face passes through the
// face's projection; so each such face writes its index to the pixels whose
// centres its projection covers.  The projection is computed in FP32 (FP64 is
// 1/64 of the FP32 rate on GB300 and made this kernel cost more than the
// searches it saves) and grown by 2e-3 pixel; faces within 1e-5 of edge-on
// are drawn too.  Pixels on shared edges get one of the faces.  Nothing here
// is trusted: the walk tests the face with its exact entry test and searches
// the BVH when it fails, so rounding here only costs searches.
__global__ void __launch_bounds__(128) k_entry_raster(const MeshView m, const GeoView g, int a0,
                                                      int32_t *emap) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int ai = blockIdx.y;
    if (q >= m.nb) return;
    const AngleFrame *F = g.frames + a0 + ai;
    auto ld3 = [](const double *v) {
        return mkf((float)__ldg(v), (float)__ldg(v + 1), (float)__ldg(v + 2));
    };
    const f3 S = ld3(F->S), Cd = ld3(F->C), U = ld3(F->U), V = ld3(F->V);
    const float4 *bf = reinterpret_cast<const float4 *>(m.bfaces + q);
    const float4 A = __ldg(bf), B = __ldg(bf + 1), Cf = __ldg(bf + 2);
    const f3 v[3] = {mkf(A.x, A.y, A.z), mkf(B.x, B.y, B.z), mkf(Cf.x, Cf.y, Cf.z)};
    // the mesh lies on the positive side of (b - a) x (c - a)
    const f3 N = crossf(sub(v[1], v[0]), sub(v[2], v[0]));
    const f3 sa = sub(S, v[0]);
    if (dotf(N, sa) > 1e-5f * sqrtf(dotf(N, N) * dotf(sa, sa))) return;
    const f3 W = sub(Cd, S);
    const float ww = dotf(W, W);
    const float idu = 1.0f / (float)g.du, idv = 1.0f / (float)g.dv;
    const float hu = 0.5f * (float)(g.nu - 1), hv = 0.5f * (float)(g.nv - 1);
    float px[3], py[3];
    for (int k = 0; k < 3; ++k) {
        const f3 D = sub(v[k], S);
        const float dw = dotf(D, W);
        if (!(dw > 0.f)) return;  // not in front of the source
        const float t = ww / dw;
        const f3 rel = mkf(S.x + t * D.x - Cd.x, S.y + t * D.y - Cd.y, S.z + t * D.z - Cd.z);
        px[k] = dotf(rel, U) * idu + hu;
        py[k] = dotf(rel, V) * idv + hv;
    }
    const float eps = 2e-3f;
    const float ulo = fminf(fminf(px[0], px[1]), px[2]) - eps, uhi = fmaxf(fmaxf(px[0], px[1]), px[2]) + eps;
    const float vlo = fminf(fminf(py[0], py[1]), py[2]) - eps, vhi = fmaxf(fmaxf(py[0], py[1]), py[2]) + eps;
    if (!(uhi >= 0.f && vhi >= 0.f && ulo <= (float)(g.nu - 1) && vlo <= (float)(g.nv - 1))) return;
    // clamped to the detector before the conversion (a vertex near the
    // source's plane projects arbitrarily far)
    const int iu0 = (int)ceilf(fmaxf(ulo, 0.f)), iu1 = (int)floorf(fminf(uhi, (float)(g.nu - 1)));
    const int iv0 = (int)ceilf(fmaxf(vlo, 0.f)), iv1 = (int)floorf(fminf(vhi, (float)(g.nv - 1)));
    const float area = (px[1] - px[0]) * (py[2] - py[0]) - (py[1] - py[0]) * (px[2] - px[0]);
    const float sg = area >= 0.f ? 1.f : -1.f;
    float ex[3], ey[3], el[3];
    for (int k = 0; k < 3; ++k) {
        const int j = k == 2 ? 0 : k + 1;
        ex[k] = px[j] - px[k];
        ey[k] = py[j] - py[k];
        el[k] = -eps * sqrtf(ex[k] * ex[k] + ey[k] * ey[k]);
    }
    int32_t *row0 = emap + (int64_t)ai * g.nv * g.nu;
    for (int iv = iv0; iv <= iv1; ++iv)
        for (int iu = iu0; iu <= iu1; ++iu) {
            const float x = (float)iu, y = (float)iv;
            bool in = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) in &= sg * (ex[k] * (y - py[k]) - ey[k] * (x - px[k])) >= el[k];
            if (in) row0[(int64_t)iv * g.nu + iu] = (int32_t)q;
        }
}

// Draws the entry map of the tile blocks [b0, b0 + nb) (cone rays) into
// p.emap_buf and points p's map view at it.  Leaves p without a map when the
// buffer is too small for the chunk's angles.
static cudaError_t launch_entry_map(KParams &p, int64_t b0, int64_t nb, cudaStream_t stream) {
    p.emap = nullptr;
    if (!p.emap_buf || p.src_kind != 0 || nb <= 0) return cudaSuccess;
    const int64_t per = (int64_t)p.tiles_u * p.tiles_v, pix = (int64_t)p.g.nu * p.g.nv;
    const int64_t a_lo = b0 / per, a_hi = (b0 + nb - 1) / per;
    const int64_t len = (a_hi - a_lo + 1) * pix;
    if (len > p.emap_cap || a_hi - a_lo + 1 > 65535) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(p.emap_buf, 0xff, (size_t)len * sizeof(int32_t), stream);
    if (e != cudaSuccess) return e;
    if (p.m.nb > 0) {
        dim3 grid((unsigned)((p.m.nb + 127) / 128), (unsigned)(a_hi - a_lo + 1));
        k_entry_raster<<<grid, 128, 0, stream>>>(p.m, p.g, (int)a_lo, p.emap_buf);
        note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    p.emap = p.emap_buf;
    p.emap_base = a_lo * pix;
    p.emap_len = len;
    return cudaSuccess;
}

// ============================================================ batched walk
//
// Many meshes and geometries in one persistent launch.  The unit of work is a
// WARP item: 32 consecutive in-tile threads of one detector tile of one angle
// of one problem (the rays a warp of the single-problem kernel walks).  Work
// is handed out in two levels:
//   * a CTA claims CHUNKS of kBatchChunk consecutive warp items (whole tiles,
//     as every problem's item range starts at a multiple of the chunk) from a
//     global counter, so the warps walking neighbouring rays of one tile share
//     the SM's L1 (spreading the warps of a tile over SMs cut the L1 hit rate
//     from 67% to 49%);
//   * the CTA's warps take items from a shared-memory ticket counter on their
//     own and never wait at a CTA barrier for the slowest warp.
// A ticket t belongs to CTA-local chunk t / kBatchChunk; the warp drawing the
// chunk's first ticket claims it and publishes its base in a ring slot, which
// it may reuse only after every ticket of the slot's previous chunk has read
// it.  Both waits are between warps of one CTA and bounded (TETPROJ_ERR_TIMEOUT,
// and the warp stops).  Per warp, the problem's parameters sit in a private
// shared-memory slot, refreshed only when the warp moves to another problem.
// Deferred rays carry the problem index in bits 40+ of their queue entry and
// are finished by k_batch_resume32.

#define TP_BATCH_TAG_SHIFT 40
#define TP_BATCH_THREADS 128
#define TP_BATCH_RING 4

// 7 resident CTAs per SM: at most 72 registers, no spills (8 CTAs cap it at 64 with
// spills in the backprojection; 24 jittered Kuhn meshes of 16^3-118^3 cells,
// 1.6G rays, C = 4: 2,746 vs 2,835 ms per forward + backprojection)
#ifndef TP_BATCH_MIN_BLOCKS
#define TP_BATCH_MIN_BLOCKS 7
#endif

constexpr int kBatchParamVec = (int)((sizeof(KParams) + 15) / 16);

// bounded wait for *a == v on a shared-memory word written by another warp:
// at most `limit` polls.  A test of the timeout path passes a non-zero
// `offset`, so that the awaited value is one no warp ever writes.
__device__ __forceinline__ bool batch_wait_eq(volatile int *a, int v, BatchWait w) {
    for (int i = 0; i < w.limit; ++i) {
        if (*a == v + w.offset) return true;
        __nanosleep(32);
    }
    return false;
}

template <int C, int MODE>
__global__ void __launch_bounds__(TP_BATCH_THREADS, TP_BATCH_MIN_BLOCKS)
    k_batch32(const BatchProblem *__restrict__ probs, const int64_t *__restrict__ item_begin,
              int nprob, int64_t round_begin, int64_t round_end, unsigned *chunk_counter,
              int nsm_max, QEntry *q, unsigned long long *q_count, BatchWait wait,
              const EmapView *__restrict__ views) {
    extern __shared__ float4 smem[];
    __shared__ unsigned s_ticket;
    __shared__ long long s_base[TP_BATCH_RING];
    __shared__ int s_gen[TP_BATCH_RING];
    __shared__ int s_used[TP_BATCH_RING];
    if (threadIdx.x == 0) s_ticket = 0;
    if (threadIdx.x < TP_BATCH_RING) {
        s_gen[threadIdx.x] = -1;
        s_used[threadIdx.x] = kBatchChunk;  // slot free
    }
    __syncthreads();  // the only CTA barrier

    // per-warp slot: the current problem's parameters (its smem_nodes field
    // clamped to the nodes staged here), then the staged BVH nodes.  The
    // walk reads everything it needs from the slot, so little state stays in
    // registers across it.
    const int lane = threadIdx.x & 31;
    KParams *sp = reinterpret_cast<KParams *>(smem + (threadIdx.x >> 5) *
                                                         (kBatchParamVec + 4 * nsm_max));
    int cur = -1;
    while (true) {
        long long it = 0;
        if (lane == 0) {
            const unsigned t = atomicAdd(&s_ticket, 1u);
            const int c = (int)(t / kBatchChunk), o = (int)(t % kBatchChunk);
            const int r = c % TP_BATCH_RING;
            bool ok = true;
            if (o == 0) {
                // claim chunk c: wait until slot r's previous chunk is fully read
                ok = batch_wait_eq(&s_used[r], kBatchChunk, wait);
                if (ok) {
                    s_used[r] = 0;
                    const unsigned g = atomicAdd(chunk_counter, 1u);
                    s_base[r] = round_begin + (long long)g * kBatchChunk;
                    __threadfence_block();
                    *(volatile int *)&s_gen[r] = c;
                }
            }
            if (ok) ok = batch_wait_eq(&s_gen[r], c, wait);
            if (ok) {
                __threadfence_block();
                it = *(volatile long long *)&s_base[r] + o;
                __threadfence_block();
                atomicAdd(&s_used[r], 1);
            } else {
                report_error(probs[cur < 0 ? 0 : cur].p.m.counters, TETPROJ_ERR_TIMEOUT);
                it = round_end;
            }
        }
        it = __shfl_sync(FULL_MASK, it, 0);
        if (it >= round_end) break;
        // problem k with item_begin[k] <= it < item_begin[k + 1] (warp-uniform)
        int k = 0, hi = nprob - 1;
        while (k < hi) {
            const int mid = (k + hi + 1) >> 1;
            if (__ldg(item_begin + mid) <= it) k = mid;
            else hi = mid - 1;
        }
        if (k != cur) {
            __syncwarp();
            float4 *dst = reinterpret_cast<float4 *>(sp);
            const float4 *src = reinterpret_cast<const float4 *>(&probs[k].p);
            for (int i = lane; i < kBatchParamVec; i += 32) dst[i] = __ldg(src + i);
            const int want = __ldg(&probs[k].p.smem_nodes);
            const int nsm = want < nsm_max ? want : nsm_max;
            const float4 *bv = reinterpret_cast<const float4 *>(__ldg(
                reinterpret_cast<const unsigned long long *>(&probs[k].p.m.bvh)));
            for (int i = lane; i < nsm * 4; i += 32) dst[kBatchParamVec + i] = __ldg(bv + i);
            __syncwarp();
            if (lane == 0) {
                sp->smem_nodes = nsm;
                sp->q = q;  // this round's deferral queue (rounds may alternate queues)
                sp->q_count = q_count;
                // this round's entry map of the problem, if it has one
                const EmapView ev = views ? views[k] : EmapView{nullptr, 0, 0};
                sp->emap = ev.emap;
                sp->emap_base = ev.base;
                sp->emap_len = ev.len;
            }
            __syncwarp();
            cur = k;
        }
        // items of one problem number < 2^31; items past the problem's last
        // tile (padding to a whole chunk) map to no ray.  Warps per tile:
        // tu * tv / 32, a power of two.
        const int wpt_log = sp->log_tu + sp->log_tv - 5;
        const int local = (int)(it - __ldg(item_begin + k));
        const int t = ((local & ((1 << wpt_log) - 1)) << 5) + lane;
        int64_t ray = 0;
        const bool valid = thread_ray_at(*sp, (int64_t)(local >> wpt_log), t, ray);
        walk32_ray<C, MODE, false>(*sp,
                                   reinterpret_cast<const BvhNode *>(
                                       reinterpret_cast<const float4 *>(sp) + kBatchParamVec),
                                   sp->smem_nodes, ray, valid, nullptr);
    }
}

template <int C, int MODE>
__global__ void __launch_bounds__(128, 4)
    k_batch_resume32(const BatchProblem *__restrict__ probs, const QEntry *q,
                     const unsigned long long *q_count, int64_t q_cap) {
    const unsigned long long n = min(*q_count, (unsigned long long)q_cap);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < n;
         base += stride) {
        const unsigned long long kq = base + threadIdx.x;
        const bool valid = kq < n;
        const QEntry *qe = q + (valid ? kq : 0);
        const int64_t tagged = valid ? qe->ray : 0;
        const int prob = (int)(tagged >> TP_BATCH_TAG_SHIFT);
        const int64_t ray = tagged & ((int64_t(1) << TP_BATCH_TAG_SHIFT) - 1);
        walk32_ray<C, MODE, true>(probs[prob].p, nullptr, 0, ray, valid, qe);
    }
}

// The fixes one round of the batched walk queued; each names its problem in
// the ray's tag bits.
template <int C, int MODE>
__global__ void __launch_bounds__(128) k_batch_fix32(const BatchProblem *__restrict__ probs,
                                                     QEntry *q, const unsigned long long *q_count,
                                                     int64_t q_cap) {
    const XFix *xf = queue_fixes(q, q_cap);
    const unsigned long long n = min(q_count[1], (unsigned long long)(q_cap / 2));
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += stride) {
        const XFix r = xf[k];
        fix_apply<C, MODE>(probs[(int)(r.ray >> TP_BATCH_TAG_SHIFT)].p, r);
    }
}

template <int C, int MODE>
static cudaError_t launch_batch_fix(const BatchProblem *probs, QEntry *q,
                                    const unsigned long long *q_count, int64_t q_cap,
                                    unsigned grid, cudaStream_t stream) {
    if constexpr (queues_fixes<MODE>()) {
        k_batch_fix32<C, MODE><<<grid, 128, 0, stream>>>(probs, q, q_count, q_cap);
        note_launch();
        return cudaGetLastError();
    }
    return cudaSuccess;
}

static size_t batch_smem(int smem_nodes) {
    return (size_t)(TP_BATCH_THREADS / 32) * (kBatchParamVec * 16 + (size_t)smem_nodes * sizeof(BvhNode));
}

template <int C, int MODE>
static cudaError_t batch_grid_mode(int smem_nodes, unsigned &grid) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch32<C, MODE>,
                                                                  TP_BATCH_THREADS,
                                                                  batch_smem(smem_nodes));
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    grid = (unsigned)(per_sm * sm_count());
    return cudaSuccess;
}

cudaError_t batch_grid(int channels, int mode, int smem_nodes, unsigned &grid) {
    if (mode == MODE_FWD)
        return channels == 4 ? batch_grid_mode<4, MODE_FWD>(smem_nodes, grid)
                             : batch_grid_mode<1, MODE_FWD>(smem_nodes, grid);
    if (mode == MODE_BWD64)
        return channels == 4 ? batch_grid_mode<4, MODE_BWD64>(smem_nodes, grid)
                             : batch_grid_mode<1, MODE_BWD64>(smem_nodes, grid);
    return channels == 4 ? batch_grid_mode<4, MODE_BWD>(smem_nodes, grid)
                         : batch_grid_mode<1, MODE_BWD>(smem_nodes, grid);
}

template <int C, int MODE>
static cudaError_t launch_batch_mode(const BatchProblem *probs, const int64_t *item_begin,
                                     int nprob, int64_t nitems, unsigned grid,
                                     unsigned rgrid, QEntry *q, unsigned long long *q_count,
                                     int64_t q_cap, unsigned *item_counter,
                                     int smem_nodes, cudaStream_t stream,
                                     const ResumeOverlap *ov, const int64_t *cuts,
                                     int ncuts, const AccMerge *merges, int nmerge,
                                     BatchWait wait, const BatchEmap *em) {
    // rounds of warp items (32 rays each), at most q_cap rays: uniform, or
    // [cuts[i], cuts[i + 1]) when cuts are given
    if (nmerge > 0 && MODE != MODE_BWD) return cudaErrorInvalidValue;
    const int64_t round_items = batch_round_items(q_cap);
    // round i's entry maps (before its walk; the previous round's walk, the
    // map's only reader, precedes it on the same stream)
    auto draw_maps = [&](int64_t i, cudaStream_t st) -> cudaError_t {
        if (!em) return cudaSuccess;
        const BatchEmapRound &R = em->rounds[i];
        if (R.len <= 0) return cudaSuccess;
        cudaError_t e = cudaMemsetAsync(em->buf, 0xff, (size_t)R.len * sizeof(int32_t), st);
        for (int j = R.first; j < R.first + R.count && e == cudaSuccess; ++j) {
            const BatchEmapJob &J = em->jobs[j];
            const KParams &P = em->probs[J.prob];
            if (P.m.nb <= 0) continue;
            dim3 g((unsigned)((P.m.nb + 127) / 128), (unsigned)J.na);
            k_entry_raster<<<g, 128, 0, st>>>(P.m, P.g, J.a_lo, em->buf + J.off);
            note_launch();
            e = cudaGetLastError();
        }
        return e;
    };
    auto views_of = [&](int64_t i) -> const EmapView * {
        return em ? em->views + i * em->nprob : nullptr;
    };
    if (round_items < 1) return cudaErrorInvalidValue;
    const int64_t nrounds = cuts ? (int64_t)ncuts - 1 : (nitems + round_items - 1) / round_items;
    if (cuts) {
        if (ncuts < 2 || cuts[0] != 0 || cuts[ncuts - 1] != nitems) return cudaErrorInvalidValue;
        for (int i = 0; i + 1 < ncuts; ++i)
            if (cuts[i + 1] <= cuts[i] || cuts[i + 1] - cuts[i] > round_items)
                return cudaErrorInvalidValue;
    }
    auto round_of = [&](int64_t i, int64_t &r0, int64_t &r1) {
        if (cuts) {
            r0 = cuts[i];
            r1 = cuts[i + 1];
        } else {
            r0 = i * round_items;
            r1 = nitems - r0 < round_items ? nitems : r0 + round_items;
        }
    };
    auto merge_all = [&](cudaStream_t st) {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < nmerge && e == cudaSuccess; ++i)
            e = launch_acc_merge(merges[i].acc32, merges[i].acc64, merges[i].n, st);
        return e;
    };
    if (ov && nrounds > 1) {
        // resume of round r on ov->aux while round r + 1 runs (queues alternate)
        cudaError_t e = cudaEventRecord(ov->ev_start, stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ov->aux, ov->ev_start, 0);
        int used = 0;
        for (int64_t i = 0; i < nrounds && e == cudaSuccess; ++i) {
            const int j = (int)(i & 1);
            QEntry *qj = j ? ov->q2 : q;
            unsigned long long *cj = j ? ov->q2_count : q_count;
            int64_t r0, r1;
            round_of(i, r0, r1);
            if (i >= 2) e = cudaStreamWaitEvent(stream, ov->ev_res[j], 0);
            if (e == cudaSuccess) e = cudaMemsetAsync(item_counter, 0, sizeof(unsigned), stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(cj, 0, kQueueCountBytes, stream);
            if (e == cudaSuccess) e = draw_maps(i, stream);
            if (e != cudaSuccess) break;
            k_batch32<C, MODE><<<grid, TP_BATCH_THREADS, batch_smem(smem_nodes), stream>>>(
                probs, item_begin, nprob, r0, r1, item_counter, smem_nodes, qj, cj, wait, views_of(i));
            note_launch();
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(ov->ev_fast[j], stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ov->aux, ov->ev_fast[j], 0);
            if (e != cudaSuccess) break;
            k_batch_resume32<C, MODE><<<rgrid, 128, 0, ov->aux>>>(probs, qj, cj, q_cap);
            note_launch();
            e = cudaGetLastError();
            if (e == cudaSuccess) e = launch_batch_fix<C, MODE>(probs, qj, cj, q_cap, rgrid, ov->aux);
            if (e == cudaSuccess) e = merge_all(ov->aux);
            if (e == cudaSuccess) e = cudaEventRecord(ov->ev_res[j], ov->aux);
            used |= 1 << j;
        }
        for (int j = 0; j < 2 && e == cudaSuccess; ++j)
            if (used & (1 << j)) e = cudaStreamWaitEvent(stream, ov->ev_res[j], 0);
        return e;
    }
    for (int64_t i = 0; i < nrounds; ++i) {
        int64_t r0, r1;
        round_of(i, r0, r1);
        cudaError_t e = cudaMemsetAsync(item_counter, 0, sizeof(unsigned), stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(q_count, 0, kQueueCountBytes, stream);
        if (e == cudaSuccess) e = draw_maps(i, stream);
        if (e != cudaSuccess) return e;
        k_batch32<C, MODE><<<grid, TP_BATCH_THREADS, batch_smem(smem_nodes), stream>>>(
            probs, item_begin, nprob, r0, r1, item_counter, smem_nodes, q, q_count, wait, views_of(i));
        note_launch();
        k_batch_resume32<C, MODE><<<rgrid, 128, 0, stream>>>(probs, q, q_count, q_cap);
        note_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_batch_fix<C, MODE>(probs, q, q_count, q_cap, rgrid, stream);
        if (e == cudaSuccess) e = merge_all(stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_batch(const BatchProblem *probs, const int64_t *item_begin, int nprob,
                         int64_t nitems, int channels, int mode, unsigned grid,
                         unsigned rgrid, QEntry *q, unsigned long long *q_count, int64_t q_cap,
                         unsigned *item_counter, int smem_nodes, cudaStream_t stream,
                         const ResumeOverlap *ov, const int64_t *cuts, int ncuts,
                         const AccMerge *merges, int nmerge, BatchWait wait,
                         const BatchEmap *em) {
    if (nitems <= 0) return cudaSuccess;
    if (wait.limit < 1) return cudaErrorInvalidValue;
    if (grid < 1 || rgrid < 1) return cudaErrorInvalidValue;
#define TP_BATCH_ARGS probs, item_begin, nprob, nitems, grid, rgrid, q, q_count, q_cap, \
                      item_counter, smem_nodes, stream, ov, cuts, ncuts, merges, nmerge, wait, em
    if (mode == MODE_FWD)
        return channels == 4 ? launch_batch_mode<4, MODE_FWD>(TP_BATCH_ARGS)
                             : launch_batch_mode<1, MODE_FWD>(TP_BATCH_ARGS);
    if (mode == MODE_BWD64)
        return channels == 4 ? launch_batch_mode<4, MODE_BWD64>(TP_BATCH_ARGS)
                             : launch_batch_mode<1, MODE_BWD64>(TP_BATCH_ARGS);
    return channels == 4 ? launch_batch_mode<4, MODE_BWD>(TP_BATCH_ARGS)
                         : launch_batch_mode<1, MODE_BWD>(TP_BATCH_ARGS);
#undef TP_BATCH_ARGS
}

int device_sm_count() { return sm_count(); }

// ========================================== the paper's walk (comparison)
//
// Alg. 1 and 2 as the paper prints them, kept as a comparison mode for the
// floating-point experiment of Sec. III-C (not the product path, which decides
// exit faces with exact signs).  Per ray: l = |R2 - R1|; the entry tet is the
// boundary face with the smallest Moller-Trumbore parameter t >= 0 (the
// paper's R*-tree search keeps the minimum t; the same boundary-face BVH is
// traversed here without early exit; ties go to the smaller user tet id, then
// the face opposite the smaller vertex id);
// then per tet all four faces are tested with the safety margin eps = 1e-9,
// multiplied by 10 until two faces are hit; t1 / t2 are the smallest /
// largest hit parameters, sum += l (t2 - t1) mu, and the walk moves through
// the face of t2.  Readings of what the paper leaves open: the eps loop stops
// at 1e-2 (status 1, "halt": a missed intersection); the walk stops after
// max_steps tets (status 2, "loop"); "if t2 = t1 check if they need to be
// swapped" is read as: when the two parameters are equal and the face of t2
// is the face the ray entered through, leave through the face of t1 instead;
// Alg. 1's v = f (d x r) is read as the dot product f (d . r).  The face's
// vertices enter Alg. 1 in increasing user vertex id, and a tet's faces are
// tested in increasing id of their opposite vertex (t1 = the first minimum,
// t2 = the last maximum in that order), so every description of the same mesh
// gives the same arithmetic and the same decisions.

template <typename T>
struct MtV {
    T x, y, z;
};
template <typename T>
__device__ __forceinline__ MtV<T> mt_sub(const MtV<T> &a, const MtV<T> &b) {
    return {a.x - b.x, a.y - b.y, a.z - b.z};
}
template <typename T>
__device__ __forceinline__ MtV<T> mt_cross(const MtV<T> &a, const MtV<T> &b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T>
__device__ __forceinline__ T mt_dot(const MtV<T> &a, const MtV<T> &b) {
    return (a.x * b.x + a.y * b.y) + a.z * b.z;
}

// Alg. 1: does the line R1 + t d cross triangle (P1, P2, P3), with the
// barycentric bounds widened by eps?  t on success.
template <typename T>
__device__ __forceinline__ bool mt_hit(const MtV<T> &R1, const MtV<T> &d, const MtV<T> &P1,
                                       const MtV<T> &P2, const MtV<T> &P3, T eps, T &t) {
    const MtV<T> E1 = mt_sub(P2, P1), E2 = mt_sub(P3, P1);
    const MtV<T> q = mt_cross(d, E2);
    const T a = mt_dot(E1, q);
    if (a > T(-1e-8) && a < T(1e-8)) return false;
    const T f = T(1) / a;
    const MtV<T> s = mt_sub(R1, P1);
    const T u = f * mt_dot(s, q);
    if (u < T(0) - eps) return false;
    const MtV<T> r = mt_cross(s, E1);
    const T v = f * mt_dot(d, r);
    if (v < T(0) - eps || u + v > T(1) + eps) return false;
    t = f * mt_dot(E2, r);
    return true;
}

template <typename T>
__device__ __forceinline__ MtV<T> mt_vertex(const MeshView &m, int h, int k);
template <>
__device__ __forceinline__ MtV<float> mt_vertex<float>(const MeshView &m, int h, int k) {
    const float4 v = __ldg(m.rec32[h].v + k);  // xyz of local vertex k
    return {v.x, v.y, v.z};
}
template <>
__device__ __forceinline__ MtV<double> mt_vertex<double>(const MeshView &m, int h, int k) {
    const double *r = m.rec64[h].v;
    return {__ldg(r + 3 * k), __ldg(r + 3 * k + 1), __ldg(r + 3 * k + 2)};
}

// Alg. 1 on face f of tet h (the face opposite local vertex f)
template <typename T>
__device__ __forceinline__ bool mt_face(const MeshView &m, int h, int f, const int4 &vid,
                                        const MtV<T> &R1, const MtV<T> &d, T eps, T &t) {
    int a, b, c;
    face_triple(f, a, b, c);
    int ia = sel4(vid, a), ib = sel4(vid, b), ic = sel4(vid, c);
    // increasing user vertex id
    if (ia > ib) { int x = a; a = b; b = x; x = ia; ia = ib; ib = x; }
    if (ib > ic) { int x = b; b = c; c = x; x = ib; ib = ic; ic = x; }
    if (ia > ib) { int x = a; a = b; b = x; x = ia; ia = ib; ib = x; }
    return mt_hit<T>(R1, d, mt_vertex<T>(m, h, a), mt_vertex<T>(m, h, b), mt_vertex<T>(m, h, c),
                     eps, t);
}

template <typename T>
__global__ void __launch_bounds__(128) k_walk_mt(const __grid_constant__ KParams p,
                                                 int8_t *__restrict__ status) {
    int64_t ray = 0;
    if (!thread_ray(p, ray)) return;  // no warp-collective operations below
    d3 S, P;
    load_ray(p, ray, S, P);
    const MtV<T> R1 = {(T)S.x, (T)S.y, (T)S.z}, R2 = {(T)P.x, (T)P.y, (T)P.z};
    const MtV<T> d = mt_sub(R2, R1);
    const T l = sqrt(mt_dot(d, d));
    // entry: the boundary face with the smallest t >= 0
    const f3 S32 = tof(S);
    const f3 d32 = {(float)(P.x - S.x), (float)(P.y - S.y), (float)(P.z - S.z)};
    const float smax = fmaxf(fmaxf(fabsf(S32.x), fabsf(S32.y)), fabsf(S32.z));
    const float margin = 16.f * 5.9604645e-8f * (smax + p.m.radius);
    LocalCnt cnt = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    T tbest = T(0);
    int hbest = -1, fbest = -1, ubest = 0, obest = 0;
    bvh_search(p.m, nullptr, 0, S32, safe_inv(d32), margin, cnt, [&](int q) -> bool {
        const int code = __float_as_int(__ldg(&p.m.bfaces[q].a.w));
        const int hq = code >> 2, fq = code & 3;
        T t;
        const int4 vq = __ldg(p.m.vid + hq);
        if (mt_face<T>(p.m, hq, fq, vq, R1, d, T(1e-9), t) && t >= T(0)) {
            const int uq = __ldg(p.m.perm + hq), oq = sel4(vq, fq);
            if (hbest < 0 || t < tbest || (t == tbest && (uq < ubest ||
                                                          (uq == ubest && oq < obest)))) {
                tbest = t; hbest = hq; fbest = fq; ubest = uq; obest = oq;
            }
        }
        return false;  // visit every candidate: the minimum is wanted
    });
    T sum = T(0);
    int st = 0;
    const T *mu = reinterpret_cast<const T *>(p.in);
    int h = hbest, fin = fbest, steps = 0;
    while (h >= 0) {
        const int4 vid = __ldg(p.m.vid + h);
        // faces in increasing id of the opposite vertex
        int ord[4] = {0, 1, 2, 3};
#pragma unroll
        for (int i = 1; i < 4; ++i)
#pragma unroll
            for (int j = i; j > 0; --j)
                if (sel4(vid, ord[j - 1]) > sel4(vid, ord[j])) {
                    const int x = ord[j]; ord[j] = ord[j - 1]; ord[j - 1] = x;
                }
        T th[4];
        int fh[4];
        int nh = 0;
        T eps = T(1e-9);
        while (true) {
            nh = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int f = ord[j];
                T t;
                if (mt_face<T>(p.m, h, f, vid, R1, d, eps, t)) { th[nh] = t; fh[nh] = f; ++nh; }
            }
            if (nh >= 2) break;
            eps = eps * T(10);
            if (eps > T(1e-2)) break;
        }
        if (nh < 2) { st = 1; break; }
        int i1 = 0, i2 = 0;
        for (int k = 1; k < nh; ++k) {
            if (th[k] < th[i1]) i1 = k;
            if (th[k] >= th[i2]) i2 = k;
        }
        const T t1 = th[i1], t2 = th[i2];
        int fout = fh[i2];
        if (t2 == t1 && fout == fin) fout = fh[i1];
        sum = sum + (l * (t2 - t1)) * __ldg(mu + h);
        const int nx = __float_as_int(__ldg(&p.m.rec32[h].v[fout].w));
        if (nx < 0) break;
        h = nx >> 2;
        fin = nx & 3;
        if (++steps >= p.max_steps) { st = 2; break; }
    }
    reinterpret_cast<T *>(p.out)[ray] = sum;
    if (status) status[ray] = (int8_t)st;
}

cudaError_t launch_walk_mt(const KParams &p, int f64, int8_t *status, cudaStream_t stream) {
    int64_t nblocks;
    int threads;
    if (p.src_kind == 0) {
        threads = p.tu * p.tv;
        nblocks = (int64_t)p.g.na * p.tiles_u * p.tiles_v;
    } else {
        threads = 128;
        nblocks = (p.nrays + threads - 1) / threads;
    }
    if (nblocks <= 0) return cudaSuccess;
    if (nblocks > 0x7fffffff || threads > 128) return cudaErrorInvalidConfiguration;
    if (f64)
        k_walk_mt<double><<<(unsigned)nblocks, threads, 0, stream>>>(p, status);
    else
        k_walk_mt<float><<<(unsigned)nblocks, threads, 0, stream>>>(p, status);
    note_launch();
    return cudaGetLastError();
}

// ============================================================ small kernels

template <typename T>
__global__ void k_gather_perm(const int32_t *__restrict__ perm, int64_t nt, int C,
                              const T *__restrict__ src, T *__restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt * C) return;
    int64_t h = i / C;
    int c = (int)(i - h * C);
    dst[i] = src[(int64_t)__ldg(perm + h) * C + c];
}
template <typename T>
__global__ void k_scatter_perm(const int32_t *__restrict__ perm, int64_t nt, int C,
                               const T *__restrict__ src, T *__restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt * C) return;
    int64_t h = i / C;
    int c = (int)(i - h * C);
    dst[(int64_t)__ldg(perm + h) * C + c] = src[i];
}

__global__ void k_scatter_perm_d2f(const int32_t *__restrict__ perm, int64_t nt, int C,
                                   const double *__restrict__ src, float *__restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt * C) return;
    int64_t h = i / C;
    int c = (int)(i - h * C);
    dst[(int64_t)__ldg(perm + h) * C + c] = (float)src[i];
}

cudaError_t launch_scatter_perm_d2f(const int32_t *perm, int64_t nt, int channels,
                                    const double *src_h, float *dst_user, cudaStream_t stream) {
    int64_t blocks = (nt * channels + 255) / 256;
    if (blocks <= 0) return cudaSuccess;
    k_scatter_perm_d2f<<<(unsigned)blocks, 256, 0, stream>>>(perm, nt, channels, src_h, dst_user);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_geometry_rays(GeoView g, const int64_t *idx, int64_t n, double *src,
                                double *dst) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int64_t j = idx ? idx[k] : k;
    int iu = (int)(j % g.nu);
    int64_t r2 = j / g.nu;
    int iv = (int)(r2 % g.nv);
    int a = (int)(r2 / g.nv);
    if (a < 0 || a >= g.na) return;
    d3 S, P;
    cone_ray(g, a, iv, iu, S, P);
    src[3 * k] = S.x; src[3 * k + 1] = S.y; src[3 * k + 2] = S.z;
    dst[3 * k] = P.x; dst[3 * k + 1] = P.y; dst[3 * k + 2] = P.z;
}

__global__ void k_side(const double *S, const double *P, const double *p, const double *q,
                       int64_t n, int8_t *sign, int8_t *stage) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    auto ld = [](const double *a, int64_t k) { return mk(a[3 * k], a[3 * k + 1], a[3 * k + 2]); };
    int st = 0;
    int s = side_sign_cascade(ld(S, k), ld(P, k), ld(p, k), ld(q, k), &st);
    sign[k] = (int8_t)s;
    stage[k] = (int8_t)st;
}

// ================================================================ launchers

template <int C, int MODE, int ENTRY = ENTRY_BVH>
static cudaError_t launch_mode(const KParams &p0, int precision, int64_t nblocks, int threads,
                               size_t smem, cudaStream_t stream, const ResumeOverlap *ov,
                               const AccMerge *mg) {
    KParams p = p0;
    if constexpr (ENTRY == ENTRY_BVH && MODE != MODE_BWD64 && MODE != MODE_ENTRY) {
        if (precision != TETPROJ_FILTERED) {
            p.block_offset = 0;
            k_walk64<C, MODE><<<(unsigned)nblocks, threads, smem, stream>>>(p);
            note_launch();
            return cudaGetLastError();
        }
    } else {
        if (precision != TETPROJ_FILTERED) return cudaErrorInvalidValue;
    }
    // chunks of at most q_cap rays (and mg->chunk_rays), each followed by
    // the resume kernel (and the accumulator merge)
    if (mg && MODE != MODE_BWD) return cudaErrorInvalidValue;
    int64_t chunk = p.q_cap / threads;
    if (mg && mg->chunk_rays / threads < chunk) chunk = mg->chunk_rays / threads;
    if (chunk < 1) return cudaErrorInvalidValue;
    const unsigned rgrid = (unsigned)(4 * sm_count());
    if (ov && nblocks > chunk) {
        // resume of chunk i on ov->aux, overlapping the fast walk of chunk i + 1;
        // queue i % 2; chunk i + 2 reuses a queue after its resume has read it
        cudaError_t e = cudaEventRecord(ov->ev_start, stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ov->aux, ov->ev_start, 0);
        int used = 0;
        for (int64_t b0 = 0, i = 0; b0 < nblocks && e == cudaSuccess; b0 += chunk, ++i) {
            const int j = (int)(i & 1);
            KParams pc = p;
            pc.block_offset = b0;
            pc.q = j ? ov->q2 : p.q;
            pc.q_count = j ? ov->q2_count : p.q_count;
            const int64_t nb = nblocks - b0 < chunk ? nblocks - b0 : chunk;
            if (i >= 2) e = cudaStreamWaitEvent(stream, ov->ev_res[j], 0);
            if (e == cudaSuccess) e = cudaMemsetAsync(pc.q_count, 0, kQueueCountBytes, stream);
            if (e == cudaSuccess && ENTRY == ENTRY_BVH) e = launch_entry_map(pc, b0, nb, stream);
            if (e != cudaSuccess) break;
            k_walk32<C, MODE, ENTRY><<<(unsigned)nb, threads, smem, stream>>>(pc);
            note_launch();
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(ov->ev_fast[j], stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ov->aux, ov->ev_fast[j], 0);
            if (e != cudaSuccess) break;
            k_resume32<C, MODE><<<rgrid, 128, smem, ov->aux>>>(pc);
            note_launch();
            e = cudaGetLastError();
            if (e == cudaSuccess) e = launch_fix<C, MODE>(pc, rgrid, ov->aux);
            if (e == cudaSuccess && mg) e = launch_acc_merge(mg->acc32, mg->acc64, mg->n, ov->aux);
            if (e == cudaSuccess) e = cudaEventRecord(ov->ev_res[j], ov->aux);
            used |= 1 << j;
        }
        for (int j = 0; j < 2 && e == cudaSuccess; ++j)  // join the auxiliary stream
            if (used & (1 << j)) e = cudaStreamWaitEvent(stream, ov->ev_res[j], 0);
        return e;
    }
    for (int64_t b0 = 0; b0 < nblocks; b0 += chunk) {
        int64_t nb = nblocks - b0 < chunk ? nblocks - b0 : chunk;
        p.block_offset = b0;
        cudaError_t e = cudaMemsetAsync(p.q_count, 0, kQueueCountBytes, stream);
        if (e == cudaSuccess && ENTRY == ENTRY_BVH) e = launch_entry_map(p, b0, nb, stream);
        if (e != cudaSuccess) return e;
        k_walk32<C, MODE, ENTRY><<<(unsigned)nb, threads, smem, stream>>>(p);
        note_launch();
        k_resume32<C, MODE><<<rgrid, 128, smem, stream>>>(p);
        note_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_fix<C, MODE>(p, rgrid, stream);
        if (e == cudaSuccess && mg) e = launch_acc_merge(mg->acc32, mg->acc64, mg->n, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

__global__ void k_acc_merge(float *acc32, double *acc64, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float v = atomicExch(acc32 + i, 0.f);
        if (v != 0.f) acc64[i] += (double)v;
    }
}

cudaError_t launch_acc_merge(float *acc32, double *acc64, int64_t n, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)8 * sm_count();
    if (blocks > cap) blocks = cap;
    k_acc_merge<<<(unsigned)blocks, 256, 0, stream>>>(acc32, acc64, n);
    note_launch();
    return cudaGetLastError();
}

template <int C, int MODE>
static cudaError_t launch_blocks_mode(const KParams &p0, int64_t b0, int64_t b1,
                                      cudaStream_t stream) {
    KParams p = p0;
    const int threads = p.tu * p.tv;
    const size_t smem = (size_t)p.smem_nodes * sizeof(BvhNode);
    if (b1 <= b0) return cudaSuccess;
    if ((b1 - b0) * threads > p.q_cap || b1 - b0 > 0x7fffffff) return cudaErrorInvalidValue;
    p.block_offset = b0;
    cudaError_t e = cudaMemsetAsync(p.q_count, 0, kQueueCountBytes, stream);
    if (e != cudaSuccess) return e;
    k_walk32<C, MODE><<<(unsigned)(b1 - b0), threads, smem, stream>>>(p);
    note_launch();
    k_resume32<C, MODE><<<(unsigned)(4 * sm_count()), 128, smem, stream>>>(p);
    note_launch();
    cudaError_t e2 = cudaGetLastError();
    if (e2 == cudaSuccess) e2 = launch_fix<C, MODE>(p, (unsigned)(4 * sm_count()), stream);
    return e2;
}

cudaError_t launch_walk_blocks(const KParams &p, int channels, int mode, int64_t b0, int64_t b1,
                               cudaStream_t stream) {
    if (p.src_kind != 0) return cudaErrorInvalidValue;
    switch (mode) {
    case MODE_FWD:
        return channels == 4 ? launch_blocks_mode<4, MODE_FWD>(p, b0, b1, stream)
                             : launch_blocks_mode<1, MODE_FWD>(p, b0, b1, stream);
    case MODE_BWD:
        return channels == 4 ? launch_blocks_mode<4, MODE_BWD>(p, b0, b1, stream)
                             : launch_blocks_mode<1, MODE_BWD>(p, b0, b1, stream);
    case MODE_SEG:
        return channels == 4 ? launch_blocks_mode<4, MODE_SEG>(p, b0, b1, stream)
                             : launch_blocks_mode<1, MODE_SEG>(p, b0, b1, stream);
    default:
        return launch_blocks_mode<1, MODE_TRACE>(p, b0, b1, stream);
    }
}

// one CTA per tile block, threads = tile size (<= 256)
__global__ void k_block_offsets(const __grid_constant__ KParams p, const int32_t *__restrict__ count,
                                int32_t *__restrict__ ray_off, int64_t *__restrict__ block_cnt) {
    __shared__ int64_t wsum[8];
    int64_t ray = 0;
    const bool valid = thread_ray_in(p, (int64_t)blockIdx.x, ray);
    const int c = valid ? max(__ldg(count + ray), 0) : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = c;  // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int64_t before = 0, total = 0;
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) {
        if (i < w) before += wsum[i];
        total += wsum[i];
    }
    if (valid) ray_off[ray] = (int32_t)(before + x - c);
    if (threadIdx.x == 0) block_cnt[blockIdx.x] = total;
}

cudaError_t launch_block_offsets(const KParams &p, const int32_t *count, int32_t *ray_off,
                                 int64_t *block_cnt, int64_t nblocks, cudaStream_t stream) {
    if (nblocks <= 0) return cudaSuccess;
    if (nblocks > 0x7fffffff || p.src_kind != 0) return cudaErrorInvalidValue;
    k_block_offsets<<<(unsigned)nblocks, p.tu * p.tv, 0, stream>>>(p, count, ray_off, block_cnt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_walk(const KParams &p, int precision, int channels, int mode,
                        cudaStream_t stream, const ResumeOverlap *ov, const AccMerge *mg) {
    if (mg && mode != MODE_BWD) return cudaErrorInvalidValue;
    int64_t nblocks;
    int threads;
    if (p.src_kind == 0) {
        threads = p.tu * p.tv;
        nblocks = (int64_t)p.g.na * p.tiles_u * p.tiles_v;
    } else {
        threads = 128;
        nblocks = (p.nrays + threads - 1) / threads;
    }
    if (nblocks <= 0) return cudaSuccess;
    if (nblocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
    size_t smem = (size_t)p.smem_nodes * sizeof(BvhNode);
    if (mode == MODE_FWD) {
        if (p.entry == ENTRY_RSTAR) {  // the paper's entry structure: FP32, C = 1
            if (precision != TETPROJ_FILTERED || channels != 1) return cudaErrorInvalidValue;
            return launch_mode<1, MODE_FWD, ENTRY_RSTAR>(p, precision, nblocks, threads, smem, stream, ov, mg);
        }
        return channels == 4 ? launch_mode<4, MODE_FWD>(p, precision, nblocks, threads, smem, stream, ov, mg)
                             : launch_mode<1, MODE_FWD>(p, precision, nblocks, threads, smem, stream, ov, mg);
    }
    if (mode == MODE_BWD) {
        return channels == 4 ? launch_mode<4, MODE_BWD>(p, precision, nblocks, threads, smem, stream, ov, mg)
                             : launch_mode<1, MODE_BWD>(p, precision, nblocks, threads, smem, stream, ov, mg);
    }
    if (mode == MODE_BWD64) {
        if (precision != TETPROJ_FILTERED) return cudaErrorInvalidValue;
        return channels == 4 ? launch_mode<4, MODE_BWD64>(p, precision, nblocks, threads, smem, stream, ov, mg)
                             : launch_mode<1, MODE_BWD64>(p, precision, nblocks, threads, smem, stream, ov, mg);
    }
    if (mode == MODE_ENTRY) {
        if (precision != TETPROJ_FILTERED) return cudaErrorInvalidValue;
        return p.entry == ENTRY_RSTAR
                   ? launch_mode<1, MODE_ENTRY, ENTRY_RSTAR>(p, precision, nblocks, threads, smem, stream, ov, mg)
                   : launch_mode<1, MODE_ENTRY>(p, precision, nblocks, threads, smem, stream, ov, mg);
    }
    return launch_mode<1, MODE_TRACE>(p, precision, nblocks, threads, smem, stream, ov, mg);
}

cudaError_t launch_gather_perm(const int32_t *perm, int64_t nt, int channels, int f64,
                               const void *src_user, void *dst_h, cudaStream_t stream) {
    int64_t n = nt * channels;
    int64_t blocks = (n + 255) / 256;
    if (f64)
        k_gather_perm<double><<<(unsigned)blocks, 256, 0, stream>>>(
            perm, nt, channels, (const double *)src_user, (double *)dst_h);
    else
        k_gather_perm<float><<<(unsigned)blocks, 256, 0, stream>>>(
            perm, nt, channels, (const float *)src_user, (float *)dst_h);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_scatter_perm(const int32_t *perm, int64_t nt, int channels, int f64,
                                const void *src_h, void *dst_user, cudaStream_t stream) {
    int64_t n = nt * channels;
    int64_t blocks = (n + 255) / 256;
    if (f64)
        k_scatter_perm<double><<<(unsigned)blocks, 256, 0, stream>>>(
            perm, nt, channels, (const double *)src_h, (double *)dst_user);
    else
        k_scatter_perm<float><<<(unsigned)blocks, 256, 0, stream>>>(
            perm, nt, channels, (const float *)src_h, (float *)dst_user);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_geometry_rays(const GeoView &g, const int64_t *idx, int64_t n, double *src,
                                 double *dst, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    k_geometry_rays<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(g, idx, n, src, dst);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_side_device(const double *S, const double *P, const double *p,
                               const double *q, int64_t n, int8_t *sign, int8_t *stage,
                               cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    k_side<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(S, P, p, q, n, sign, stage);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tp
