/*
 * mt.c -- CPU reference of the paper's own ray walk (Alg. 1 and 2).
 *
 * TEST INFRASTRUCTURE ONLY (same rules as oracle.c: only tests/, smoke() and
 * bench.py's reference legs use it; it shares no code with the CUDA library).
 *
 * Unlike oracle.c, which evaluates the plain definition a_ij = |ray cap tet|,
 * this file follows the paper's heuristic walk step by step, because the
 * quantity of interest is what that algorithm does in a given precision
 * (Sec. II-C.1, Sec. III-C "Floating point errors"):
 *
 *   Alg. 1 (Moller-Trumbore with safety parameter eps), for ray R1 + t d and
 *   triangle P1 P2 P3:  E1 = P2 - P1, E2 = P3 - P1, q = d x E2, a = E1 . q;
 *   |a| < 1e-8 -> no hit; f = 1/a; s = R1 - P1; u = f (s . q); u < -eps -> no;
 *   r = s x E1; v = f (d . r); v < -eps or u + v > 1 + eps -> no;
 *   t = f (E2 . r).
 *
 *   Alg. 2, per ray: l = |R2 - R1|; eps = 1e-9; the entry tet is the boundary
 *   face with the smallest t >= 0 (Sec. II-E keeps the minimum parameter);
 *   in each tet all four faces are tested, eps *= 10 until two are hit;
 *   t1, t2 = smallest and largest hit parameter; sum += l (t2 - t1) mu;
 *   move to the neighbour across the face of t2.
 *
 * Readings where the paper is silent (identical in the CUDA comparison mode):
 *   - Alg. 1 prints v = f (d x r): read as the dot product;
 *   - the eps loop has no bound in the paper: it stops once eps > 1e-2
 *     (status 1, a missed intersection that ends the walk);
 *   - no loop guard in the paper: more than max_steps tets gives status 2;
 *   - "if t2 = t1 check if they need to be swapped": when t1 == t2 and the
 *     face of t2 is the face the ray came in through, leave through the face
 *     of t1;
 *   - a tet's faces are tested in increasing index of their opposite vertex;
 *     t1 is the first minimum in that order, t2 the last maximum; equal entry
 *     parameters go to the smaller tet index, then to the face opposite the
 *     smaller vertex index;
 *   - the three vertices of a face enter Alg. 1 in increasing vertex index,
 *     so the arithmetic does not depend on how a tet lists its vertices.
 *
 * Precision: every step runs in T = float or double (the mesh coordinates,
 * the ray endpoints and mu are rounded to T first).  Expressions are written
 * as (x*x' + y*y') + z*z' and (a*b - c*d) with separately rounded operations;
 * compile with -ffp-contract=off.
 *
 * Adjacency is built here from the tets (faces matched by sorting their
 * vertex triples), independently of the library's mesh builder.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t v[3]; /* sorted vertex ids */
    int64_t owner; /* tet * 4 + local face (the face opposite local vertex) */
} mt_face_rec;

static int mt_face_cmp(const void *a, const void *b) {
    const mt_face_rec *x = (const mt_face_rec *)a, *y = (const mt_face_rec *)b;
    for (int k = 0; k < 3; ++k)
        if (x->v[k] != y->v[k]) return x->v[k] < y->v[k] ? -1 : 1;
    return x->owner < y->owner ? -1 : (x->owner > y->owner);
}

static void sort3(int32_t *a) {
    int32_t t;
    if (a[0] > a[1]) { t = a[0]; a[0] = a[1]; a[1] = t; }
    if (a[1] > a[2]) { t = a[1]; a[1] = a[2]; a[2] = t; }
    if (a[0] > a[1]) { t = a[0]; a[0] = a[1]; a[1] = t; }
}

/* nbr[4 t + k] = 4 t' + k' across the face opposite local vertex k, or -1 */
static int mt_adjacency(const int32_t *T, int64_t nt, int64_t *nbr) {
    mt_face_rec *F = (mt_face_rec *)malloc(sizeof(mt_face_rec) * (size_t)(4 * nt));
    if (!F) return -1;
    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 4; ++k) {
            mt_face_rec *f = &F[4 * t + k];
            int m = 0;
            for (int j = 0; j < 4; ++j)
                if (j != k) f->v[m++] = T[4 * t + j];
            sort3(f->v);
            f->owner = 4 * t + k;
        }
    qsort(F, (size_t)(4 * nt), sizeof(mt_face_rec), mt_face_cmp);
    for (int64_t i = 0; i < 4 * nt; ++i) nbr[i] = -1;
    for (int64_t i = 0; i + 1 < 4 * nt; ++i) {
        if (memcmp(F[i].v, F[i + 1].v, sizeof(F[i].v)) == 0) {
            nbr[F[i].owner] = F[i + 1].owner;
            nbr[F[i + 1].owner] = F[i].owner;
            ++i;
        }
    }
    free(F);
    return 0;
}

#define MT_DEFINE(T, SUF, SQRT)                                                              \
    typedef struct { T x, y, z; } mtv_##SUF;                                                 \
    static mtv_##SUF sub_##SUF(mtv_##SUF a, mtv_##SUF b) {                                   \
        mtv_##SUF r = {a.x - b.x, a.y - b.y, a.z - b.z};                                     \
        return r;                                                                            \
    }                                                                                        \
    static mtv_##SUF cross_##SUF(mtv_##SUF a, mtv_##SUF b) {                                 \
        mtv_##SUF r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; \
        return r;                                                                            \
    }                                                                                        \
    static T dot_##SUF(mtv_##SUF a, mtv_##SUF b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; } \
    /* Alg. 1 */                                                                             \
    static int mt_##SUF(mtv_##SUF R1, mtv_##SUF d, mtv_##SUF P1, mtv_##SUF P2, mtv_##SUF P3,  \
                        T eps, T *t) {                                                       \
        mtv_##SUF E1 = sub_##SUF(P2, P1), E2 = sub_##SUF(P3, P1);                            \
        mtv_##SUF q = cross_##SUF(d, E2);                                                    \
        T a = dot_##SUF(E1, q);                                                              \
        if (a > (T)(-1e-8) && a < (T)(1e-8)) return 0;                                       \
        T f = (T)1 / a;                                                                      \
        mtv_##SUF s = sub_##SUF(R1, P1);                                                     \
        T u = f * dot_##SUF(s, q);                                                           \
        if (u < (T)0 - eps) return 0;                                                        \
        mtv_##SUF r = cross_##SUF(s, E1);                                                    \
        T v = f * dot_##SUF(d, r);                                                           \
        if (v < (T)0 - eps || u + v > (T)1 + eps) return 0;                                  \
        *t = f * dot_##SUF(E2, r);                                                           \
        return 1;                                                                            \
    }                                                                                        \
    static mtv_##SUF vtx_##SUF(const double *V, int32_t i) {                                 \
        mtv_##SUF r = {(T)V[3 * i], (T)V[3 * i + 1], (T)V[3 * i + 2]};                       \
        return r;                                                                            \
    }                                                                                        \
    /* face k of tet t (opposite local vertex k), vertices in increasing id */               \
    static int face_##SUF(const double *V, const int32_t *Tt, int64_t t, int k,             \
                          mtv_##SUF R1, mtv_##SUF d, T eps, T *tt) {                         \
        int32_t id[3];                                                                       \
        int m = 0;                                                                           \
        for (int j = 0; j < 4; ++j)                                                          \
            if (j != k) id[m++] = Tt[4 * t + j];                                             \
        sort3(id);                                                                           \
        return mt_##SUF(R1, d, vtx_##SUF(V, id[0]), vtx_##SUF(V, id[1]), vtx_##SUF(V, id[2]), \
                        eps, tt);                                                            \
    }                                                                                        \
    /* Alg. 2 for one ray; returns the status, *out the (partial) sum */                     \
    static int walk_##SUF(const double *V, const int32_t *Tt, int64_t nt, const int64_t *nbr, \
                          const int64_t *bnd, int64_t nb, const double *mu, const double *S, \
                          const double *P, int64_t max_steps, double *out) {                 \
        mtv_##SUF R1 = {(T)S[0], (T)S[1], (T)S[2]}, R2 = {(T)P[0], (T)P[1], (T)P[2]};        \
        mtv_##SUF d = sub_##SUF(R2, R1);                                                     \
        T l = SQRT(dot_##SUF(d, d));                                                         \
        int64_t h = -1;                                                                      \
        int fin = -1;                                                                        \
        T tbest = 0;                                                                         \
        for (int64_t b = 0; b < nb; ++b) {                                                   \
            int64_t t0 = bnd[b] >> 2;                                                        \
            int k0 = (int)(bnd[b] & 3);                                                      \
            T t;                                                                             \
            if (face_##SUF(V, Tt, t0, k0, R1, d, (T)1e-9, &t) && t >= (T)0) {                \
                if (h < 0 || t < tbest ||                                                    \
                    (t == tbest && (t0 < h || (t0 == h && Tt[4 * t0 + k0] < Tt[4 * h + fin])))) { \
                    tbest = t;                                                               \
                    h = t0;                                                                  \
                    fin = k0;                                                                \
                }                                                                            \
            }                                                                                \
        }                                                                                    \
        T sum = 0;                                                                           \
        int st = 0;                                                                          \
        int64_t steps = 0;                                                                   \
        (void)nt;                                                                            \
        while (h >= 0) {                                                                     \
            T th[4];                                                                         \
            int fh[4], nh = 0;                                                               \
            T eps = (T)1e-9;                                                                 \
            int ord[4] = {0, 1, 2, 3};                                                       \
            for (int i = 1; i < 4; ++i)                                                      \
                for (int j = i; j > 0; --j)                                                  \
                    if (Tt[4 * h + ord[j - 1]] > Tt[4 * h + ord[j]]) {                       \
                        int x = ord[j];                                                      \
                        ord[j] = ord[j - 1];                                                 \
                        ord[j - 1] = x;                                                      \
                    }                                                                        \
            for (;;) {                                                                       \
                nh = 0;                                                                      \
                for (int jj = 0; jj < 4; ++jj) {                                             \
                    const int k = ord[jj];                                                   \
                    T t;                                                                     \
                    if (face_##SUF(V, Tt, h, k, R1, d, eps, &t)) {                           \
                        th[nh] = t;                                                          \
                        fh[nh] = k;                                                          \
                        ++nh;                                                                \
                    }                                                                        \
                }                                                                            \
                if (nh >= 2) break;                                                          \
                eps = eps * (T)10;                                                           \
                if (eps > (T)1e-2) break;                                                    \
            }                                                                                \
            if (nh < 2) { st = 1; break; }                                                   \
            int i1 = 0, i2 = 0;                                                              \
            for (int k = 1; k < nh; ++k) {                                                   \
                if (th[k] < th[i1]) i1 = k;                                                  \
                if (th[k] >= th[i2]) i2 = k;                                                 \
            }                                                                                \
            T t1 = th[i1], t2 = th[i2];                                                      \
            int fout = fh[i2];                                                               \
            if (t2 == t1 && fout == fin) fout = fh[i1];                                      \
            sum = sum + (l * (t2 - t1)) * (T)mu[h];                                          \
            int64_t nx = nbr[4 * h + fout];                                                  \
            if (nx < 0) break;                                                               \
            h = nx >> 2;                                                                     \
            fin = (int)(nx & 3);                                                             \
            if (++steps >= max_steps) { st = 2; break; }                                     \
        }                                                                                    \
        *out = (double)sum;                                                                  \
        return st;                                                                           \
    }

MT_DEFINE(float, f32, sqrtf)
MT_DEFINE(double, f64, sqrt)

/* The paper's walk for n explicit rays (S, P: [n][3]) in single (prec = 4)
 * or double (prec = 8) precision.  Writes out[n] and status[n]
 * (0 done, 1 halted, 2 step limit).  Returns 0, or -1 on bad input. */
int oracle_mt_forward_rays(const double *V, int64_t nv, const int32_t *T, int64_t nt,
                           const double *mu, const double *S, const double *P, int64_t n,
                           int prec, int64_t max_steps, double *out, int8_t *status) {
    if (nv <= 0 || nt <= 0 || n < 0 || (prec != 4 && prec != 8)) return -1;
    int64_t *nbr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(4 * nt));
    if (!nbr) return -1;
    if (mt_adjacency(T, nt, nbr) != 0) { free(nbr); return -1; }
    int64_t nb = 0;
    for (int64_t i = 0; i < 4 * nt; ++i) nb += nbr[i] < 0;
    int64_t *bnd = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
    if (!bnd) { free(nbr); return -1; }
    nb = 0;
    for (int64_t i = 0; i < 4 * nt; ++i)
        if (nbr[i] < 0) bnd[nb++] = i;
    for (int64_t j = 0; j < n; ++j) {
        status[j] = (int8_t)(prec == 4
                                 ? walk_f32(V, T, nt, nbr, bnd, nb, mu, S + 3 * j, P + 3 * j,
                                            max_steps, out + j)
                                 : walk_f64(V, T, nt, nbr, bnd, nb, mu, S + 3 * j, P + 3 * j,
                                            max_steps, out + j));
    }
    free(bnd);
    free(nbr);
    return 0;
}
