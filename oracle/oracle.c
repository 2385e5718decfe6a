/*
 * oracle.c -- plain FP64 CPU reference for the tetrahedral-mesh projectors.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg use it.  It shares no code with the CUDA library.
 *
 * What it computes is the paper's plain definition, not its algorithm:
 *
 *   Eq. 1   A x = b + e,  a_ij = length of (ray j  intersected with element i)
 *   Eq. 2   b_j = sum_i a_ij x_i                        (forward projection)
 *   Eq. 3   x_i = sum_j a_ij b_j                        (backprojection; the
 *           paper prints b_i under a sum over j, read as b_j)
 *
 * a_ij is evaluated by brute force for every (ray, tet) pair: the half-line
 * X(t) = S + t (P - S), t >= 0, is clipped against the four face half-spaces of
 * the closed tet (Cyrus-Beck), giving the parameter interval [lo, hi]; then
 * a_ij = max(0, hi - lo) * |P - S|.  There is no traversal, no adjacency, no
 * acceleration structure: every tet is tested against every ray.
 *
 * Ray convention (the paper leaves it implicit; Alg. 2 launches one ray per
 * detector pixel and uses l = |R2 - R1|): R1 = source S, R2 = pixel centre P.
 * Circular cone beam about the z axis, for angle theta:
 *   S = (dso cos, dso sin, 0), C = S - dsd (cos, sin, 0), U = (-sin, cos, 0),
 *   V = (0, 0, 1), P = C + u U + v V with
 *   u = (iu - (nu-1)/2) du, v = (iv - (nv-1)/2) dv.
 * Ray index j = (a * nv + iv) * nu + iu.  Every product and sum is rounded
 * separately (this file must be compiled with -ffp-contract=off) so that the
 * rays are bit-identical to any other implementation of the same convention.
 *
 * Sums over tets (forward) and over rays (backward) use Neumaier compensated
 * summation in FP64.  Backward sums are accumulated per thread over disjoint
 * ray ranges and added in thread order, so results do not depend on timing.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_VERSION 1

int64_t oracle_version(void) { return ORACLE_VERSION; }

/* ---------------------------------------------------------------- geometry */

typedef struct {
    double dso, dsd, du, dv;
    int64_t nu, nv, na;
    const double *angles;
} cone_geom;

static void cone_ray(const cone_geom *g, int64_t j, double S[3], double P[3]) {
    int64_t iu = j % g->nu;
    int64_t iv = (j / g->nu) % g->nv;
    int64_t a = j / (g->nu * g->nv);
    double th = g->angles[a];
    double c = cos(th), s = sin(th);
    double Sx = g->dso * c, Sy = g->dso * s, Sz = 0.0;
    double Cx = Sx - g->dsd * c, Cy = Sy - g->dsd * s, Cz = 0.0;
    double Ux = -s, Uy = c, Uz = 0.0;
    double Vx = 0.0, Vy = 0.0, Vz = 1.0;
    double u = ((double)iu - 0.5 * (double)(g->nu - 1)) * g->du;
    double v = ((double)iv - 0.5 * (double)(g->nv - 1)) * g->dv;
    S[0] = Sx; S[1] = Sy; S[2] = Sz;
    P[0] = (Cx + u * Ux) + v * Vx;
    P[1] = (Cy + u * Uy) + v * Vy;
    P[2] = (Cz + u * Uz) + v * Vz;
}

/* Ray endpoints for a list of ray indices (or all rays when idx == NULL). */
void oracle_cone_rays(double dso, double dsd, int64_t nu, int64_t nv, double du, double dv,
                      const double *angles, int64_t na, const int64_t *idx, int64_t n,
                      double *S_out, double *P_out) {
    cone_geom g = {dso, dsd, du, dv, nu, nv, na, angles};
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = idx ? idx[k] : k;
        cone_ray(&g, j, S_out + 3 * k, P_out + 3 * k);
    }
}

/* ------------------------------------------------------------ one tet clip */

static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void sub3(const double a[3], const double b[3], double r[3]) {
    r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2];
}
static void cross3(const double a[3], const double b[3], double r[3]) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

/*
 * Clip the half-line S + t d (t >= 0) against the closed tet with vertices
 * v[0..3].  Face k is the triangle of the three vertices other than v[k]; its
 * normal is turned to point away from v[k] (outward).  A point X is inside the
 * face's half-space iff n.(X - q) <= 0 for a face vertex q, i.e.
 *   t (n.d) <= n.(q - S).
 * Returns 0 if the tet is degenerate (a face plane contains the opposite
 * vertex), 1 otherwise; *lo, *hi receive the clipped parameter interval
 * (empty when *hi <= *lo).
 *
 * A ray lying in a face plane (|n.d| and |n.(q-S)| both below PLANE_TOL
 * relative) is on the boundary of both tets sharing that face, so the closed
 * measure counts it twice and FP64 cannot tell the sides apart.  *planar is
 * set for such rays.  When a side direction w is given, the face constraint is
 * replaced by its limit for the ray moved by +0*w: satisfied if n.w < 0, empty
 * otherwise.  That gives the one-sided limits of the integral.
 */
#define PLANE_TOL 1e-12
static int tet_clip_range(const double v[4][3], const double S[3], const double d[3],
                          const double *w, double t0, double t1, double *lo, double *hi,
                          int *planar) {
    double l = t0, h = t1;
    int empty = 0;
    *planar = 0;
    double dd = sqrt(dot3(d, d));
    for (int k = 0; k < 4; ++k) {
        const double *q0 = v[(k + 1) & 3], *q1 = v[(k + 2) & 3], *q2 = v[(k + 3) & 3];
        double e1[3], e2[3], n[3], x[3];
        sub3(q1, q0, e1);
        sub3(q2, q0, e2);
        cross3(e1, e2, n);
        sub3(v[k], q0, x);
        double side = dot3(n, x);
        if (side == 0.0) return 0;
        if (side > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
        double qs[3];
        sub3(q0, S, qs);
        double num = dot3(n, qs);
        double den = dot3(n, d);
        double nn = sqrt(dot3(n, n));
        int inplane = fabs(den) <= PLANE_TOL * nn * dd &&
                      fabs(num) <= PLANE_TOL * nn * sqrt(dot3(qs, qs));
        if (inplane) {
            *planar = 1;
            if (w) {
                if (dot3(n, w) >= 0.0) empty = 1;
                continue;
            }
        }
        if (den > 0.0) {
            double t = num / den;
            if (t < h) h = t;
        } else if (den < 0.0) {
            double t = num / den;
            if (t > l) l = t;
        } else if (num < 0.0) {
            empty = 1;
        }
    }
    if (empty) { *lo = 1.0; *hi = 0.0; return 1; }
    *lo = l;
    *hi = h;
    return 1;
}

/* the half-line t >= 0 */
static int tet_clip(const double v[4][3], const double S[3], const double d[3],
                    const double *w, double *lo, double *hi, int *planar) {
    return tet_clip_range(v, S, d, w, 0.0, INFINITY, lo, hi, planar);
}

static void load_tet(const double *verts, const int32_t *tets, int64_t i, double v[4][3]) {
    for (int k = 0; k < 4; ++k) {
        const double *p = verts + 3 * (int64_t)tets[4 * i + k];
        v[k][0] = p[0]; v[k][1] = p[1]; v[k][2] = p[2];
    }
}

/* a_ij for one (ray, tet) pair; also returns the parameter interval. */
double oracle_tet_chord(const double v_flat[12], const double S[3], const double P[3],
                        double *t_lo, double *t_hi) {
    double v[4][3], d[3], lo, hi;
    int planar;
    memcpy(v, v_flat, sizeof(v));
    sub3(P, S, d);
    if (!tet_clip(v, S, d, NULL, &lo, &hi, &planar)) { *t_lo = 0; *t_hi = 0; return 0.0; }
    *t_lo = lo;
    *t_hi = hi;
    return hi > lo ? (hi - lo) * sqrt(dot3(d, d)) : 0.0;
}

/* Neumaier compensated accumulator */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

/* ---------------------------------------------------------------- threading */

typedef struct {
    const double *verts;
    const int32_t *tets;
    int64_t nt;
    int C;
    /* rays: explicit (S, P arrays) or cone-beam (geom + optional index list) */
    const double *S, *P;
    const double *W;      /* per-ray side vectors for one-sided limits, or NULL */
    const double *T0, *T1; /* per-ray parameter range [T0, T1] (NULL: [0, inf)) */
    const cone_geom *geom;
    const int64_t *ray_idx;
    int64_t ray_begin, ray_end;
    /* forward */
    const double *mu;
    double *out;
    /* backward */
    const double *y;
    double *acc;          /* per-thread [nt * C] (nsum pairs when compensated) */
    nsum *nacc;
    /* backward over a tet subset, all rays */
    const int64_t *tet_idx;
    int64_t tet_begin, tet_end, nrays_all;
    /* trace */
    int64_t max_visits;
    int32_t *tr_tet;
    double *tr_lo, *tr_hi;
    int64_t *tr_count;
    double *tr_margin;
    int32_t *tr_planar;
} job;

static void get_ray(const job *jb, int64_t k, double S[3], double P[3]) {
    if (jb->geom) {
        int64_t j = jb->ray_idx ? jb->ray_idx[k] : k;
        cone_ray(jb->geom, j, S, P);
    } else {
        memcpy(S, jb->S + 3 * k, 3 * sizeof(double));
        memcpy(P, jb->P + 3 * k, 3 * sizeof(double));
    }
}

static int run_threads(void *(*fn)(void *), job *jobs, int nthreads) {
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return -1;
    for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, fn, &jobs[i]);
    for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    free(th);
    return 0;
}

static void split(int64_t n, int nthreads, int i, int64_t *b, int64_t *e) {
    *b = n * i / nthreads;
    *e = n * (i + 1) / nthreads;
}

/* ------------------------------------------------------------ Eq. 2 forward */

static void *fwd_worker(void *arg) {
    job *jb = (job *)arg;
    nsum acc[16];
    for (int64_t k = jb->ray_begin; k < jb->ray_end; ++k) {
        double S[3], P[3], d[3];
        get_ray(jb, k, S, P);
        sub3(P, S, d);
        const double *w = jb->W ? jb->W + 3 * k : NULL;
        double t0 = jb->T0 ? jb->T0[k] : 0.0, t1 = jb->T1 ? jb->T1[k] : INFINITY;
        double len = sqrt(dot3(d, d));
        for (int c = 0; c < jb->C; ++c) acc[c].s = acc[c].c = 0.0;
        for (int64_t i = 0; i < jb->nt; ++i) {
            double v[4][3], lo, hi;
            int planar;
            load_tet(jb->verts, jb->tets, i, v);
            if (!tet_clip_range(v, S, d, w, t0, t1, &lo, &hi, &planar) || !(hi > lo)) continue;
            double a = (hi - lo) * len;
            for (int c = 0; c < jb->C; ++c) nadd(&acc[c], a * jb->mu[i * jb->C + c]);
        }
        for (int c = 0; c < jb->C; ++c) jb->out[k * jb->C + c] = nval(&acc[c]);
    }
    return NULL;
}

static int forward_common(job *proto, int64_t nrays, int nthreads) {
    if (proto->C < 1 || proto->C > 16) return -2;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nrays && nrays > 0) nthreads = (int)nrays;
    job *jobs = (job *)calloc((size_t)nthreads, sizeof(job));
    if (!jobs) return -1;
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = *proto;
        split(nrays, nthreads, i, &jobs[i].ray_begin, &jobs[i].ray_end);
    }
    int rc = run_threads(fwd_worker, jobs, nthreads);
    free(jobs);
    return rc;
}

/* b = A mu for explicit rays (S, P: [nrays][3]); mu: [nt][C]; out: [nrays][C].
 * W: NULL, or per-ray side directions [nrays][3] selecting one-sided limits for
 * rays that lie in a face plane (see tet_clip). */
int oracle_forward_rays(const double *verts, int64_t nv, const int32_t *tets, int64_t nt,
                        const double *mu, int C, const double *S, const double *P,
                        const double *W, int64_t nrays, double *out, int nthreads) {
    (void)nv;
    job p;
    memset(&p, 0, sizeof(p));
    p.verts = verts; p.tets = tets; p.nt = nt; p.C = C; p.S = S; p.P = P; p.W = W;
    p.mu = mu; p.out = out;
    return forward_common(&p, nrays, nthreads);
}

/* b = A mu restricted to the parameter range [T0[j], T1[j]] of each explicit
 * ray, with optional side vectors W (see tet_clip_range). */
int oracle_forward_rays_range(const double *verts, int64_t nv, const int32_t *tets, int64_t nt,
                              const double *mu, int C, const double *S, const double *P,
                              const double *W, const double *T0, const double *T1,
                              int64_t nrays, double *out, int nthreads) {
    (void)nv;
    job p;
    memset(&p, 0, sizeof(p));
    p.verts = verts; p.tets = tets; p.nt = nt; p.C = C; p.S = S; p.P = P; p.W = W;
    p.T0 = T0; p.T1 = T1; p.mu = mu; p.out = out;
    return forward_common(&p, nrays, nthreads);
}

/* b = A mu for cone-beam rays; ray_idx selects rays (NULL: all na*nv*nu, in order). */
int oracle_forward_cone(const double *verts, int64_t nv_, const int32_t *tets, int64_t nt,
                        const double *mu, int C, double dso, double dsd, int64_t nu, int64_t nv,
                        double du, double dv, const double *angles, int64_t na,
                        const int64_t *ray_idx, int64_t nsel, double *out, int nthreads) {
    (void)nv_;
    cone_geom g = {dso, dsd, du, dv, nu, nv, na, angles};
    job p;
    memset(&p, 0, sizeof(p));
    p.verts = verts; p.tets = tets; p.nt = nt; p.C = C; p.geom = &g; p.ray_idx = ray_idx;
    p.mu = mu; p.out = out;
    int64_t n = ray_idx ? nsel : na * nv * nu;
    return forward_common(&p, n, nthreads);
}

/* ----------------------------------------------------------- Eq. 3 backward */

static void *bwd_rays_worker(void *arg) {
    job *jb = (job *)arg;
    for (int64_t k = jb->ray_begin; k < jb->ray_end; ++k) {
        double S[3], P[3], d[3];
        get_ray(jb, k, S, P);
        sub3(P, S, d);
        const double *w = jb->W ? jb->W + 3 * k : NULL;
        double len = sqrt(dot3(d, d));
        for (int64_t i = 0; i < jb->nt; ++i) {
            double v[4][3], lo, hi;
            int planar;
            load_tet(jb->verts, jb->tets, i, v);
            if (!tet_clip(v, S, d, w, &lo, &hi, &planar) || !(hi > lo)) continue;
            double a = (hi - lo) * len;
            for (int c = 0; c < jb->C; ++c) nadd(&jb->nacc[i * jb->C + c], a * jb->y[k * jb->C + c]);
        }
    }
    return NULL;
}

static int backward_rays_common(job *proto, int64_t nrays, double *out, int nthreads) {
    if (proto->C < 1 || proto->C > 16) return -2;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nrays && nrays > 0) nthreads = (int)nrays;
    int64_t m = proto->nt * proto->C;
    job *jobs = (job *)calloc((size_t)nthreads, sizeof(job));
    nsum *bufs = (nsum *)calloc((size_t)(m * nthreads), sizeof(nsum));
    if (!jobs || !bufs) { free(jobs); free(bufs); return -1; }
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = *proto;
        jobs[i].nacc = bufs + (int64_t)i * m;
        split(nrays, nthreads, i, &jobs[i].ray_begin, &jobs[i].ray_end);
    }
    int rc = run_threads(bwd_rays_worker, jobs, nthreads);
    for (int64_t q = 0; q < m; ++q) {
        nsum s = {0.0, 0.0};
        for (int i = 0; i < nthreads; ++i) {
            nadd(&s, bufs[(int64_t)i * m + q].s);
            nadd(&s, bufs[(int64_t)i * m + q].c);
        }
        out[q] = nval(&s);
    }
    free(jobs);
    free(bufs);
    return rc;
}

/* x = A^T y for explicit rays; y: [nrays][C]; out: [nt][C] (overwritten); W as above. */
int oracle_backward_rays(const double *verts, int64_t nv, const int32_t *tets, int64_t nt,
                         const double *y, int C, const double *S, const double *P,
                         const double *W, int64_t nrays, double *out, int nthreads) {
    (void)nv;
    job p;
    memset(&p, 0, sizeof(p));
    p.verts = verts; p.tets = tets; p.nt = nt; p.C = C; p.S = S; p.P = P; p.W = W; p.y = y;
    return backward_rays_common(&p, nrays, out, nthreads);
}

/* x = A^T y for all cone-beam rays; y: [na][nv][nu][C]; out: [nt][C]. */
int oracle_backward_cone(const double *verts, int64_t nv_, const int32_t *tets, int64_t nt,
                         const double *y, int C, double dso, double dsd, int64_t nu, int64_t nv,
                         double du, double dv, const double *angles, int64_t na, double *out,
                         int nthreads) {
    (void)nv_;
    cone_geom g = {dso, dsd, du, dv, nu, nv, na, angles};
    job p;
    memset(&p, 0, sizeof(p));
    p.verts = verts; p.tets = tets; p.nt = nt; p.C = C; p.geom = &g; p.y = y;
    return backward_rays_common(&p, na * nv * nu, out, nthreads);
}

/* x_i = sum_j a_ij y_j for a subset of tets, over all cone-beam rays. */
static void *bwd_subset_worker(void *arg) {
    job *jb = (job *)arg;
    for (int64_t q = jb->tet_begin; q < jb->tet_end; ++q) {
        int64_t i = jb->tet_idx[q];
        double v[4][3];
        load_tet(jb->verts, jb->tets, i, v);
        nsum acc[16];
        for (int c = 0; c < jb->C; ++c) acc[c].s = acc[c].c = 0.0;
        for (int64_t j = 0; j < jb->nrays_all; ++j) {
            double S[3], P[3], d[3], lo, hi;
            int planar;
            cone_ray(jb->geom, j, S, P);
            sub3(P, S, d);
            if (!tet_clip(v, S, d, NULL, &lo, &hi, &planar) || !(hi > lo)) continue;
            double a = (hi - lo) * sqrt(dot3(d, d));
            for (int c = 0; c < jb->C; ++c) nadd(&acc[c], a * jb->y[j * jb->C + c]);
        }
        for (int c = 0; c < jb->C; ++c) jb->out[q * jb->C + c] = nval(&acc[c]);
    }
    return NULL;
}

int oracle_backward_cone_subset(const double *verts, int64_t nv_, const int32_t *tets, int64_t nt,
                                const double *y, int C, double dso, double dsd, int64_t nu,
                                int64_t nv, double du, double dv, const double *angles, int64_t na,
                                const int64_t *tet_idx, int64_t nsel, double *out, int nthreads) {
    (void)nv_;
    (void)nt;
    if (C < 1 || C > 16) return -2;
    cone_geom g = {dso, dsd, du, dv, nu, nv, na, angles};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nsel && nsel > 0) nthreads = (int)nsel;
    job *jobs = (job *)calloc((size_t)nthreads, sizeof(job));
    if (!jobs) return -1;
    for (int i = 0; i < nthreads; ++i) {
        memset(&jobs[i], 0, sizeof(job));
        jobs[i].verts = verts; jobs[i].tets = tets; jobs[i].C = C; jobs[i].geom = &g;
        jobs[i].y = y; jobs[i].out = out; jobs[i].tet_idx = tet_idx;
        jobs[i].nrays_all = na * nv * nu;
        split(nsel, nthreads, i, &jobs[i].tet_begin, &jobs[i].tet_end);
    }
    int rc = run_threads(bwd_subset_worker, jobs, nthreads);
    free(jobs);
    return rc;
}

/* ---------------------------------------------------------------- traces */

typedef struct { double lo, hi; int32_t tet; } visit;

static int visit_cmp(const void *a, const void *b) {
    const visit *x = (const visit *)a, *y = (const visit *)b;
    if (x->lo < y->lo) return -1;
    if (x->lo > y->lo) return 1;
    if (x->hi < y->hi) return -1;
    if (x->hi > y->hi) return 1;
    return (x->tet > y->tet) - (x->tet < y->tet);
}

static void *trace_worker(void *arg) {
    job *jb = (job *)arg;
    int64_t cap = 64;
    visit *vs = (visit *)malloc(sizeof(visit) * (size_t)cap);
    for (int64_t k = jb->ray_begin; k < jb->ray_end; ++k) {
        double S[3], P[3], d[3];
        get_ray(jb, k, S, P);
        sub3(P, S, d);
        const double *w = jb->W ? jb->W + 3 * k : NULL;
        double len = sqrt(dot3(d, d));
        int64_t n = 0;
        double margin = INFINITY;
        int planar_any = 0;
        for (int64_t i = 0; i < jb->nt; ++i) {
            double v[4][3], lo, hi;
            int planar;
            load_tet(jb->verts, jb->tets, i, v);
            if (!tet_clip(v, S, d, w, &lo, &hi, &planar)) continue;
            if (planar) planar_any = 1;
            double m = fabs(hi - lo) * len;
            if (m < margin) margin = m;
            if (!(hi > lo)) continue;
            if (n == cap) {
                cap *= 2;
                vs = (visit *)realloc(vs, sizeof(visit) * (size_t)cap);
            }
            vs[n].lo = lo; vs[n].hi = hi; vs[n].tet = (int32_t)i;
            ++n;
        }
        qsort(vs, (size_t)n, sizeof(visit), visit_cmp);
        int64_t m = n < jb->max_visits ? n : jb->max_visits;
        for (int64_t q = 0; q < m; ++q) {
            jb->tr_tet[k * jb->max_visits + q] = vs[q].tet;
            jb->tr_lo[k * jb->max_visits + q] = vs[q].lo;
            jb->tr_hi[k * jb->max_visits + q] = vs[q].hi;
        }
        jb->tr_count[k] = n;
        jb->tr_margin[k] = margin;
        jb->tr_planar[k] = planar_any;
    }
    free(vs);
    return NULL;
}

/*
 * Row j of A for explicit rays: the tets with a_ij > 0 sorted by entry
 * parameter, with their parameter intervals.  out_count[j] is the full count
 * (entries beyond max_visits are dropped).  out_margin[j] is the smallest
 * |hi - lo| * |P - S| over all tets whose clipped interval is near-empty or
 * non-empty: a small margin flags a ray that grazes an edge or vertex.
 * out_planar[j] is 1 when the ray runs exactly inside some face plane.
 */
int oracle_trace_rays(const double *verts, int64_t nv, const int32_t *tets, int64_t nt,
                      const double *S, const double *P, int64_t nrays, int64_t max_visits,
                      int32_t *out_tet, double *out_lo, double *out_hi, int64_t *out_count,
                      double *out_margin, int32_t *out_planar, int nthreads) {
    (void)nv;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nrays && nrays > 0) nthreads = (int)nrays;
    job *jobs = (job *)calloc((size_t)nthreads, sizeof(job));
    if (!jobs) return -1;
    for (int i = 0; i < nthreads; ++i) {
        memset(&jobs[i], 0, sizeof(job));
        jobs[i].verts = verts; jobs[i].tets = tets; jobs[i].nt = nt; jobs[i].S = S; jobs[i].P = P;
        jobs[i].max_visits = max_visits; jobs[i].tr_tet = out_tet; jobs[i].tr_lo = out_lo;
        jobs[i].tr_hi = out_hi; jobs[i].tr_count = out_count; jobs[i].tr_margin = out_margin;
        jobs[i].tr_planar = out_planar;
        split(nrays, nthreads, i, &jobs[i].ray_begin, &jobs[i].ray_end);
    }
    int rc = run_threads(trace_worker, jobs, nthreads);
    free(jobs);
    return rc;
}

/* ---------------------------------------------------------------- walker */
/*
 * The oracle walker: the same a_ij (each from tet_clip, the brute-force
 * clipper's own arithmetic), but only the tets a ray passes through are
 * clipped, found by walking face adjacency.  The adjacency is built here from
 * the tets' vertex ids (faces matched by their sorted vertex triples), not
 * taken from the CUDA path.
 *
 *   entry  among the tets with a boundary face whose bounding box the
 *          half-line meets, the one with the smallest clipped lo (hi > lo);
 *          the face that sets lo must be a boundary face (a ray that meets
 *          the mesh's box but crosses no such tet is not walked);
 *   step   the exit face is the face (n.d > 0) whose plane sets hi; the next
 *          tet is its neighbour; the walk ends at a boundary face.
 *
 * A ray whose walk meets a near-tie -- two entry candidates, or two exit
 * planes, within WALK_TOL in t, a visit shorter than WALK_TOL, a tet whose lo
 * is not the previous hi, a face plane containing the ray, or more steps than
 * tets -- is not walked: its row of A is computed by the brute-force clipper
 * over all tets instead (status 1; status 2 if the ray lies in a face plane,
 * where the closed-tet measure counts both sides of the plane).  Both give
 * the plain definition; the walk is only the faster way to the same tets.
 */
#define WALK_TOL 1e-9

typedef struct {
    const double *verts;
    const int32_t *tets;
    int64_t nt, nb;
    int32_t *adj;   /* [nt][4]: tet across the face opposite vertex k, or -1 */
    int32_t *btet;  /* tets with at least one boundary face */
    double *bbox;   /* [nb][6]: their boxes, min xyz then max xyz */
    double box[6];  /* the mesh's box */
    double radius;  /* the largest |coordinate| */
    double *tbox;   /* [nt][6]: every tet's box, for the brute-force rows */
} walker;

typedef struct { int32_t b, c, code; } face_rec; /* code = tet * 4 + k */

void oracle_walker_destroy(void *h) {
    walker *w = (walker *)h;
    if (!w) return;
    free(w->adj);
    free(w->btet);
    free(w->bbox);
    free(w->tbox);
    free(w);
}

static void sort3(int32_t *a, int32_t *b, int32_t *c) {
    int32_t t;
    if (*a > *b) { t = *a; *a = *b; *b = t; }
    if (*b > *c) { t = *b; *b = *c; *c = t; }
    if (*a > *b) { t = *a; *a = *b; *b = t; }
}

/* status: 0 ok, -1 out of memory, -3 a face shared by more than two tets,
 * -4 a vertex id out of range. */
void *oracle_walker_create(const double *verts, int64_t nv, const int32_t *tets, int64_t nt,
                           int *status) {
    *status = -1;
    walker *w = (walker *)calloc(1, sizeof(walker));
    int64_t nf = 4 * nt;
    int64_t *start = (int64_t *)calloc((size_t)nv + 1, sizeof(int64_t));
    face_rec *rec = (face_rec *)malloc(sizeof(face_rec) * (size_t)(nf > 0 ? nf : 1));
    if (!w || !start || !rec) { free(start); free(rec); oracle_walker_destroy(w); return NULL; }
    w->verts = verts; w->tets = tets; w->nt = nt;
    w->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nf > 0 ? nf : 1));
    if (!w->adj) { free(start); free(rec); oracle_walker_destroy(w); return NULL; }
    for (int64_t q = 0; q < nf; ++q) {
        int32_t v = tets[q];
        if (v < 0 || v >= nv) { *status = -4; free(start); free(rec); oracle_walker_destroy(w); return NULL; }
        w->adj[q] = -1;
    }
    /* bucket the faces by their smallest vertex id (counting sort), then sort
     * each bucket by the other two ids */
    for (int64_t i = 0; i < nt; ++i)
        for (int k = 0; k < 4; ++k) {
            int32_t a = tets[4 * i + ((k + 1) & 3)], b = tets[4 * i + ((k + 2) & 3)],
                    c = tets[4 * i + ((k + 3) & 3)];
            sort3(&a, &b, &c);
            start[a + 1]++;
        }
    for (int64_t v = 0; v < nv; ++v) start[v + 1] += start[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nv > 0 ? nv : 1));
    if (!fill) { free(start); free(rec); oracle_walker_destroy(w); return NULL; }
    memcpy(fill, start, sizeof(int64_t) * (size_t)nv);
    for (int64_t i = 0; i < nt; ++i)
        for (int k = 0; k < 4; ++k) {
            int32_t a = tets[4 * i + ((k + 1) & 3)], b = tets[4 * i + ((k + 2) & 3)],
                    c = tets[4 * i + ((k + 3) & 3)];
            sort3(&a, &b, &c);
            face_rec r = {b, c, (int32_t)(4 * i + k)};
            rec[fill[a]++] = r;
        }
    free(fill);
    *status = 0;
    for (int64_t v = 0; v < nv && *status == 0; ++v) {
        face_rec *f = rec + start[v];
        int64_t n = start[v + 1] - start[v];
        for (int64_t x = 1; x < n; ++x) {  /* insertion sort: buckets are small */
            face_rec r = f[x];
            int64_t y = x - 1;
            while (y >= 0 && (f[y].b > r.b || (f[y].b == r.b && f[y].c > r.c))) { f[y + 1] = f[y]; --y; }
            f[y + 1] = r;
        }
        for (int64_t x = 0; x < n;) {
            int64_t e = x + 1;
            while (e < n && f[e].b == f[x].b && f[e].c == f[x].c) ++e;
            if (e - x > 2) { *status = -3; break; }
            if (e - x == 2) {
                w->adj[f[x].code] = f[x + 1].code >> 2;
                w->adj[f[x + 1].code] = f[x].code >> 2;
            }
            x = e;
        }
    }
    free(start);
    free(rec);
    if (*status) { oracle_walker_destroy(w); return NULL; }
    int64_t nb = 0;
    for (int64_t i = 0; i < nt; ++i)
        if (w->adj[4 * i] < 0 || w->adj[4 * i + 1] < 0 || w->adj[4 * i + 2] < 0 || w->adj[4 * i + 3] < 0) ++nb;
    w->nb = nb;
    w->tbox = (double *)malloc(sizeof(double) * 6 * (size_t)(nt > 0 ? nt : 1));
    if (!w->tbox) { *status = -1; oracle_walker_destroy(w); return NULL; }
    for (int64_t i = 0; i < nt; ++i) {
        double *bx = w->tbox + 6 * i;
        for (int q = 0; q < 3; ++q) { bx[q] = INFINITY; bx[3 + q] = -INFINITY; }
        for (int k = 0; k < 4; ++k) {
            const double *p = verts + 3 * (int64_t)tets[4 * i + k];
            for (int q = 0; q < 3; ++q) {
                if (p[q] < bx[q]) bx[q] = p[q];
                if (p[q] > bx[3 + q]) bx[3 + q] = p[q];
            }
        }
    }
    w->btet = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nb > 0 ? nb : 1));
    w->bbox = (double *)malloc(sizeof(double) * 6 * (size_t)(nb > 0 ? nb : 1));
    if (!w->btet || !w->bbox) { *status = -1; oracle_walker_destroy(w); return NULL; }
    for (int q = 0; q < 3; ++q) { w->box[q] = INFINITY; w->box[3 + q] = -INFINITY; }
    for (int64_t v = 0; v < nv; ++v)
        for (int q = 0; q < 3; ++q) {
            if (verts[3 * v + q] < w->box[q]) w->box[q] = verts[3 * v + q];
            if (verts[3 * v + q] > w->box[3 + q]) w->box[3 + q] = verts[3 * v + q];
            if (fabs(verts[3 * v + q]) > w->radius) w->radius = fabs(verts[3 * v + q]);
        }
    nb = 0;
    for (int64_t i = 0; i < nt; ++i) {
        if (!(w->adj[4 * i] < 0 || w->adj[4 * i + 1] < 0 || w->adj[4 * i + 2] < 0 || w->adj[4 * i + 3] < 0))
            continue;
        double *bx = w->bbox + 6 * nb;
        for (int q = 0; q < 3; ++q) { bx[q] = INFINITY; bx[3 + q] = -INFINITY; }
        for (int k = 0; k < 4; ++k) {
            const double *p = verts + 3 * (int64_t)tets[4 * i + k];
            for (int q = 0; q < 3; ++q) {
                if (p[q] < bx[q]) bx[q] = p[q];
                if (p[q] > bx[3 + q]) bx[3 + q] = p[q];
            }
        }
        w->btet[nb++] = (int32_t)i;
    }
    return w;
}

/* Outward face planes of tet v along the ray (the orientation rule of
 * tet_clip_range): den[k] = n_k.d, for den[k] != 0 tf[k] = the t at which the
 * ray meets face k's plane, sn[k] = |n_k.d| / (|n_k| |d|), the sine of the
 * angle between the ray and that plane, and, if kap != NULL, kap[k] = the sum
 * of the face's squared edge lengths over 2 |n_k| (sqrt 3 for an equilateral
 * face, ~1 / sin of the smallest angle for a sliver: the factor by which the
 * rounding of the cross product n_k turns its direction). */
static void tet_face_params(const double v[4][3], const double S[3], const double d[3],
                            double tf[4], double den[4], double sn[4], double *kap) {
    for (int k = 0; k < 4; ++k) {
        const double *q0 = v[(k + 1) & 3], *q1 = v[(k + 2) & 3], *q2 = v[(k + 3) & 3];
        double e1[3], e2[3], n[3], x[3], qs[3];
        sub3(q1, q0, e1);
        sub3(q2, q0, e2);
        cross3(e1, e2, n);
        sub3(v[k], q0, x);
        if (dot3(n, x) > 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
        sub3(q0, S, qs);
        den[k] = dot3(n, d);
        tf[k] = den[k] != 0.0 ? dot3(n, qs) / den[k] : 0.0;
        sn[k] = fabs(den[k]) / (sqrt(dot3(n, n)) * sqrt(dot3(d, d)));
        if (kap) {
            double e3[3];
            sub3(q2, q1, e3);
            kap[k] = (dot3(e1, e1) + dot3(e2, e2) + dot3(e3, e3)) / (2.0 * sqrt(dot3(n, n)));
        }
    }
}

/* One entry of a row: tet, a_ij, its clipped interval, and for the crossings
 * where the ray enters (i) and leaves (o) it: the inverse sine of the angle
 * with the face plane (g), the face's shape factor (c, see tet_face_params)
 * and the distance from the source plus the mesh radius (w); gi = 0 when the
 * interval starts at the source (t = 0). */
typedef struct { int32_t tet; double a, lo, hi, gi, go, ci, co, wi, wo; } wseg;
typedef struct { wseg *s; int64_t n, cap; } wbuf;

static int wgrow(wbuf *b) {
    if (b->n < b->cap) return 0;
    int64_t cap = b->cap ? 2 * b->cap : 256;
    wseg *s = (wseg *)realloc(b->s, sizeof(wseg) * (size_t)cap);
    if (!s) return -1;
    b->s = s;
    b->cap = cap;
    return 0;
}

static int wappend(wbuf *b, const wseg *e) {
    if (wgrow(b)) return -1;
    b->s[b->n++] = *e;
    return 0;
}

static int wpush(wbuf *b, int32_t tet, double a, double lo, double hi) {
    if (wgrow(b)) return -1;
    wseg *e = b->s + b->n++;
    memset(e, 0, sizeof(*e));
    e->tet = tet;
    e->a = a;
    e->lo = lo;
    e->hi = hi;
    return 0;
}

static int ray_meets_box(const double *bx, const double S[3], const double d[3], double pad);

/* Row j of A by brute force over the tets whose boxes (grown by pad) the
 * half-line meets -- a tet it crosses, or touches, lies in its box, so this
 * is every tet with a_ij > 0; 2 if a face plane of one of them contains the
 * ray (the closed-tet measure then counts both sides of that plane). */
static int walk_brute(const walker *w, const double S[3], const double d[3], double len, wbuf *out) {
    int planar_any = 0;
    const double pad = 1e-9 * (1.0 + fabs(S[0]) + fabs(S[1]) + fabs(S[2]) + len);
    out->n = 0;
    for (int64_t i = 0; i < w->nt; ++i) {
        if (!ray_meets_box(w->tbox + 6 * i, S, d, pad)) continue;
        double v[4][3], lo, hi;
        int planar;
        load_tet(w->verts, w->tets, i, v);
        if (!tet_clip(v, S, d, NULL, &lo, &hi, &planar)) continue;
        if (planar) planar_any = 1;
        /* tets the ray only touches (an edge or vertex: hi within WALK_TOL of
         * lo) are listed with a_ij = 0: they add nothing to the sums, but a
         * computed walk may visit them with a chord of the size of its
         * rounding, and their crossings' conditioning bounds that */
        if (hi > lo - WALK_TOL &&
            wpush(out, (int32_t)i, hi > lo ? (hi - lo) * len : 0.0, lo, hi > lo ? hi : lo))
            return -1;
    }
    return planar_any ? 2 : 1;
}

/* Does the half-line S + t d, t >= 0, meet the box (grown by pad)? */
static int ray_meets_box(const double *bx, const double S[3], const double d[3], double pad) {
    double t0 = 0.0, t1 = INFINITY;
    for (int q = 0; q < 3; ++q) {
        double lo = bx[q] - pad, hi = bx[3 + q] + pad;
        if (d[q] == 0.0) {
            if (S[q] < lo || S[q] > hi) return 0;
            continue;
        }
        double a = (lo - S[q]) / d[q], b = (hi - S[q]) / d[q];
        if (a > b) { double t = a; a = b; b = t; }
        if (a > t0) t0 = a;
        if (b < t1) t1 = b;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* Row j of A (the tets with a_ij > 0 and their a_ij) by the walk: 0; or, for a
 * ray the walk does not take (see above), by brute force: 1 or 2. -1: no memory. */
static int walk_row(const walker *w, const double S[3], const double P[3], wbuf *out) {
    double d[3];
    sub3(P, S, d);
    const double len = sqrt(dot3(d, d));
    const double pad = 1e-9 * (1.0 + fabs(S[0]) + fabs(S[1]) + fabs(S[2]) + len);
    out->n = 0;
    int32_t cur = -1;
    double lo = INFINITY, hi = 0.0, second = INFINITY;
    for (int64_t q = 0; q < w->nb; ++q) {
        if (!ray_meets_box(w->bbox + 6 * q, S, d, pad)) continue;
        double v[4][3], l, h;
        int planar;
        load_tet(w->verts, w->tets, w->btet[q], v);
        if (!tet_clip(v, S, d, NULL, &l, &h, &planar)) return walk_brute(w, S, d, len, out);
        if (planar) return walk_brute(w, S, d, len, out);
        if (!(h > l)) continue;
        if (l < lo) { second = lo; lo = l; hi = h; cur = w->btet[q]; }
        else if (l < second) second = l;
    }
    if (cur < 0) {
        /* no tet with a boundary face is crossed: the half-line misses the
         * mesh, or enters it through a boundary edge or vertex into a tet
         * that touches the boundary only there */
        if (!ray_meets_box(w->box, S, d, pad)) return 0;
        return walk_brute(w, S, d, len, out);
    }
    if (second - lo <= WALK_TOL) return walk_brute(w, S, d, len, out);
    {
        /* the entry must be through a boundary face: the face plane that sets lo */
        double v[4][3], tf[4], den[4], sn[4];
        load_tet(w->verts, w->tets, cur, v);
        tet_face_params(v, S, d, tf, den, sn, NULL);
        int nset = 0, bnd = 0;
        for (int k = 0; k < 4; ++k)
            if (den[k] < 0.0 && fabs(tf[k] - lo) <= WALK_TOL) { ++nset; bnd = w->adj[4 * (int64_t)cur + k] < 0; }
        if (nset != 1 || !bnd) return walk_brute(w, S, d, len, out);
    }
    for (int64_t steps = 0; steps < w->nt; ++steps) {
        if (hi - lo <= WALK_TOL) return walk_brute(w, S, d, len, out);
        if (wpush(out, cur, (hi - lo) * len, lo, hi)) return -1;
        double v[4][3], tf[4], den[4], sn[4];
        load_tet(w->verts, w->tets, cur, v);
        tet_face_params(v, S, d, tf, den, sn, NULL);
        int g = -1;
        for (int k = 0; k < 4; ++k)
            if (den[k] > 0.0 && (g < 0 || tf[k] < tf[g])) g = k;
        if (g < 0 || fabs(tf[g] - hi) > WALK_TOL) return walk_brute(w, S, d, len, out);
        for (int k = 0; k < 4; ++k)
            if (k != g && den[k] > 0.0 && tf[k] - tf[g] <= WALK_TOL) return walk_brute(w, S, d, len, out);
        const int32_t nxt = w->adj[4 * (int64_t)cur + g];
        if (nxt < 0) return 0;
        int planar;
        load_tet(w->verts, w->tets, nxt, v);
        if (!tet_clip(v, S, d, NULL, &lo, &hi, &planar) || planar || fabs(lo - tf[g]) > WALK_TOL)
            return walk_brute(w, S, d, len, out);
        cur = nxt;
    }
    return walk_brute(w, S, d, len, out);
}

/* Crossing data of a row (see wseg), in order along the ray. */
static int seg_lo_cmp(const void *x, const void *y) {
    const wseg *a = (const wseg *)x, *b = (const wseg *)y;
    return (a->lo > b->lo) - (a->lo < b->lo);
}

static void row_cond(const walker *w, const double S[3], const double d[3], double len, wbuf *row,
                     int sorted) {
    if (!sorted) qsort(row->s, (size_t)row->n, sizeof(wseg), seg_lo_cmp);
    for (int64_t q = 0; q < row->n; ++q) {
        wseg *e = row->s + q;
        double v[4][3], tf[4], den[4], sn[4], kap[4];
        load_tet(w->verts, w->tets, e->tet, v);
        tet_face_params(v, S, d, tf, den, sn, kap);
        /* the faces whose planes pass through the entry and the exit point:
         * one each for a crossing through a face's interior; two or three
         * when the ray crosses an edge or a vertex (a tet it only touches has
         * entry = exit), where a computed walk may cross any of them -- take
         * the largest inverse sine and the largest shape factor among them */
        double gi = 0.0, go = 0.0, ci = 0.0, co = 0.0;
        for (int k = 0; k < 4; ++k) {
            const double g = 1.0 / fmax(sn[k], 1e-300);
            if (den[k] == 0.0) continue;  /* parallel to the ray: not crossed */
            if (fabs(tf[k] - e->lo) <= WALK_TOL) { gi = fmax(gi, g); ci = fmax(ci, kap[k]); }
            if (fabs(tf[k] - e->hi) <= WALK_TOL) { go = fmax(go, g); co = fmax(co, kap[k]); }
        }
        e->gi = e->lo > 0.0 ? gi : 0.0;  /* no entry crossing when the interval starts at the source */
        e->ci = e->lo > 0.0 ? ci : 0.0;
        e->go = go;
        e->co = co;
        e->wi = e->lo * len + w->radius;
        e->wo = e->hi * len + w->radius;
    }
}

typedef struct {
    const walker *w;
    const cone_geom *geom;
    const int64_t *ray_idx;
    const double *S, *P;
    const double *mu, *y;
    int C;
    double cap;
    int want_cond;  /* fill the rows' crossing data (for out_kf / out_kb) */
    int64_t begin, end;
    double *out;    /* forward: [n][C] */
    double *kf;     /* forward conditioning: [n][C][2] */
    int8_t *status; /* [n] */
    wbuf rows;      /* backward: this thread's rows, concatenated */
    int64_t *row_end; /* [end - begin]: end of each ray's row in rows */
    int rc;
} wjob;

static void *walk_worker(void *arg) {
    wjob *jb = (wjob *)arg;
    wbuf row = {NULL, 0, 0};
    for (int64_t k = jb->begin; k < jb->end; ++k) {
        double S[3], P[3], d[3];
        if (jb->geom) {
            cone_ray(jb->geom, jb->ray_idx ? jb->ray_idx[k] : k, S, P);
        } else {
            memcpy(S, jb->S + 3 * k, sizeof(S));
            memcpy(P, jb->P + 3 * k, sizeof(P));
        }
        int st = walk_row(jb->w, S, P, &row);
        if (st < 0) { jb->rc = -1; break; }
        jb->status[k] = (int8_t)st;
        sub3(P, S, d);
        if (jb->want_cond) row_cond(jb->w, S, d, sqrt(dot3(d, d)), &row, st == 0);
        const int C = jb->C;
        if (jb->mu) {
            nsum acc[16];
            for (int c = 0; c < C; ++c) acc[c].s = acc[c].c = 0.0;
            for (int64_t q = 0; q < row.n; ++q)
                for (int c = 0; c < C; ++c)
                    nadd(&acc[c], row.s[q].a * jb->mu[(int64_t)row.s[q].tet * C + c]);
            for (int c = 0; c < C; ++c) jb->out[k * C + c] = nval(&acc[c]);
        }
        if (jb->mu && jb->kf) {
            /* sum over the crossings of |mu before - mu after| (w / sin), with
             * 1 / sin capped at cap ([0]) and not ([1]); mu = 0 outside */
            for (int c = 0; c < C; ++c) {
                double s0 = 0.0, s1 = 0.0, prev = 0.0, g = 0.0, wd = 0.0;
                for (int64_t q = 0; q <= row.n; ++q) {
                    double cur = q < row.n ? jb->mu[(int64_t)row.s[q].tet * C + c] : 0.0;
                    double kp;
                    if (q == 0) {
                        g = row.n ? row.s[0].gi : 0.0;
                        wd = row.n ? row.s[0].wi : 0.0;
                        kp = row.n ? row.s[0].ci : 0.0;
                    } else if (q == row.n) {
                        g = row.s[q - 1].go;
                        wd = row.s[q - 1].wo;
                        kp = row.s[q - 1].co;
                    } else {
                        g = fmax(row.s[q - 1].go, row.s[q].gi);
                        wd = fmax(row.s[q - 1].wo, row.s[q].wi);
                        kp = fmax(row.s[q - 1].co, row.s[q].ci);
                    }
                    double jump = fabs(prev - cur) * wd * kp;
                    s0 += jump * fmin(g, jb->cap);
                    s1 += jump * g;
                    prev = cur;
                }
                jb->kf[(k * C + c) * 2] = s0;
                jb->kf[(k * C + c) * 2 + 1] = s1;
            }
        }
        if (jb->y) {
            for (int64_t q = 0; q < row.n && !jb->rc; ++q)
                if (wappend(&jb->rows, &row.s[q])) jb->rc = -1;
            jb->row_end[k - jb->begin] = jb->rows.n;
        }
        if (jb->rc) break;
    }
    free(row.s);
    return NULL;
}

/*
 * Rows of A for n rays by the walker: cone rays ray_idx[0..n) of the geometry
 * (geom_* given, S = P = NULL), or explicit rays S, P [n][3].
 *   mu != NULL: out_fwd[k][c] = sum_i a_ik mu[i][c]        (Eq. 2)
 *   y  != NULL: out_bwd[i][c] = sum_k a_ik y[k][c]          (Eq. 3 over these
 *               rays only; y is indexed by k, not by the cone ray index), and,
 *               if out_count != NULL, out_count[i] = #{k : a_ik > 0}
 * (rows of rays not walked also list the tets the ray only touches, with
 * a_ik = 0: they count in the conditioning sums below, not in out_count)
 * Conditioning of the crossings (for error bounds: under rounding a crossing
 * moves along the ray by ~u w kappa / sin, w = its distance from the source +
 * the mesh radius, sin = of the angle between ray and face plane, kappa = the
 * face's shape factor, see tet_face_params), with 1 / sin capped at `cap` in
 * [..][0] and uncapped in [..][1]:
 *   out_kf [n][C][2] (with mu): sum over a ray's crossings of
 *       |mu before - mu after| w kappa / sin, mu = 0 outside the mesh;
 *   out_kb [nt][C][2] (with y): sum over the rays crossing tet i of
 *       |y[k][c]| (w_in kappa_in / sin_in + w_out kappa_out / sin_out).
 * status[k]: 0 walked, 1 brute force, 2 brute force and a face plane contains
 * the ray (closed-tet measure: the integral counts both sides).  Backward sums
 * are added in ray order after the threads finish (deterministic).
 * Returns 0, -1 (no memory) or -2 (C outside 1..16).
 */
int oracle_walk(void *h, const double *mu, const double *y, int C, double dso, double dsd,
                int64_t nu, int64_t nv, double du, double dv, const double *angles, int64_t na,
                const int64_t *ray_idx, const double *S, const double *P, int64_t n,
                double *out_fwd, double *out_bwd, int64_t *out_count, double cap,
                double *out_kf, double *out_kb, int8_t *status, int nthreads) {
    const walker *w = (const walker *)h;
    if (C < 1 || C > 16) return -2;
    cone_geom g = {dso, dsd, du, dv, nu, nv, na, angles};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n && n > 0) nthreads = (int)n;
    wjob *jobs = (wjob *)calloc((size_t)nthreads, sizeof(wjob));
    if (!jobs) return -1;
    int rc = 0;
    for (int i = 0; i < nthreads; ++i) {
        wjob *j = &jobs[i];
        j->w = w; j->geom = S ? NULL : &g; j->ray_idx = ray_idx; j->S = S; j->P = P;
        j->mu = mu; j->y = y; j->C = C; j->cap = cap; j->out = out_fwd; j->kf = out_kf;
        j->want_cond = out_kf != NULL || out_kb != NULL;
        j->status = status;
        split(n, nthreads, i, &j->begin, &j->end);
        if (y) {
            j->row_end = (int64_t *)malloc(sizeof(int64_t) * (size_t)(j->end - j->begin + 1));
            if (!j->row_end) rc = -1;
        }
    }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) rc = -1;
    if (!rc) {
        for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, walk_worker, &jobs[i]);
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
        for (int i = 0; i < nthreads; ++i) if (jobs[i].rc) rc = jobs[i].rc;
    }
    if (!rc && y) {
        int64_t m = w->nt * C;
        nsum *acc = (nsum *)calloc((size_t)(m > 0 ? m : 1), sizeof(nsum));
        if (!acc) rc = -1;
        for (int i = 0; i < nthreads && !rc; ++i) {
            wjob *j = &jobs[i];
            int64_t q = 0;
            for (int64_t k = j->begin; k < j->end; ++k)
                for (; q < j->row_end[k - j->begin]; ++q)
                    for (int c = 0; c < C; ++c)
                        nadd(&acc[(int64_t)j->rows.s[q].tet * C + c], j->rows.s[q].a * y[k * C + c]);
        }
        if (!rc) for (int64_t q = 0; q < m; ++q) out_bwd[q] = nval(&acc[q]);
        free(acc);
        if (!rc && out_count) {
            memset(out_count, 0, sizeof(int64_t) * (size_t)w->nt);
            for (int i = 0; i < nthreads; ++i)
                for (int64_t q = 0; q < jobs[i].rows.n; ++q)
                    if (jobs[i].rows.s[q].a > 0.0) out_count[jobs[i].rows.s[q].tet]++;
        }
        if (!rc && out_kb) {
            memset(out_kb, 0, sizeof(double) * (size_t)(2 * m));
            for (int i = 0; i < nthreads; ++i) {
                wjob *j = &jobs[i];
                int64_t q = 0;
                for (int64_t k = j->begin; k < j->end; ++k)
                    for (; q < j->row_end[k - j->begin]; ++q) {
                        const wseg *e = j->rows.s + q;
                        double c0 = e->wi * e->ci * fmin(e->gi, cap) + e->wo * e->co * fmin(e->go, cap);
                        double c1 = e->wi * e->ci * e->gi + e->wo * e->co * e->go;
                        for (int c = 0; c < C; ++c) {
                            double ay = fabs(y[k * C + c]);
                            out_kb[((int64_t)e->tet * C + c) * 2] += ay * c0;
                            out_kb[((int64_t)e->tet * C + c) * 2 + 1] += ay * c1;
                        }
                    }
            }
        }
    }
    for (int i = 0; i < nthreads; ++i) { free(jobs[i].rows.s); free(jobs[i].row_end); }
    free(th);
    free(jobs);
    return rc;
}

typedef struct {
    const walker *w;
    const double *S, *P;
    int64_t begin, end, max_visits;
    int32_t *tet;   /* [n][max_visits] */
    double *len;    /* [n][max_visits] */
    double *cond;   /* [n][max_visits][2] or NULL */
    int64_t *count; /* [n] */
    int8_t *status; /* [n] */
    int rc;
} tjob;

static void *trace_walk_worker(void *arg) {
    tjob *jb = (tjob *)arg;
    wbuf row = {NULL, 0, 0};
    for (int64_t k = jb->begin; k < jb->end; ++k) {
        double S[3], P[3];
        memcpy(S, jb->S + 3 * k, sizeof(S));
        memcpy(P, jb->P + 3 * k, sizeof(P));
        int st = walk_row(jb->w, S, P, &row);
        if (st < 0) { jb->rc = -1; break; }
        jb->status[k] = (int8_t)st;
        double d[3];
        sub3(P, S, d);
        row_cond(jb->w, S, d, sqrt(dot3(d, d)), &row, st == 0);
        jb->count[k] = row.n;
        for (int64_t q = 0; q < row.n && q < jb->max_visits; ++q) {
            const wseg *e = row.s + q;
            jb->tet[k * jb->max_visits + q] = e->tet;
            jb->len[k * jb->max_visits + q] = e->a;
            if (jb->cond) {
                jb->cond[(k * jb->max_visits + q) * 2] =
                    e->wi * e->ci * fmin(e->gi, 64.0) + e->wo * e->co * fmin(e->go, 64.0);
                jb->cond[(k * jb->max_visits + q) * 2 + 1] = e->wi * e->ci * e->gi + e->wo * e->co * e->go;
            }
        }
    }
    free(row.s);
    return NULL;
}

/* Row j of A as the sequence of tets the ray visits (walk order; for rays not
 * walked, status 1 or 2, the brute-force row sorted by entry parameter, which
 * also lists the tets the ray only touches, with a_ij = 0) with each a_ij, for
 * explicit rays S, P [n][3].  out_count[k] is the full count
 * (visits past max_visits are dropped).  out_cond (or NULL) [n][max_visits][2]:
 * each visit's w_in kappa_in / sin_in + w_out kappa_out / sin_out (see
 * oracle_walk), with 1 / sin
 * capped at 64 and uncapped.  Returns 0 or -1 (no memory). */
int oracle_walk_trace(void *h, const double *S, const double *P, int64_t n, int64_t max_visits,
                      int32_t *out_tet, double *out_len, double *out_cond, int64_t *out_count,
                      int8_t *status, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n && n > 0) nthreads = (int)n;
    tjob *jobs = (tjob *)calloc((size_t)nthreads, sizeof(tjob));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int rc = (!jobs || !th) ? -1 : 0;
    if (!rc) {
        for (int i = 0; i < nthreads; ++i) {
            tjob *j = &jobs[i];
            j->w = (const walker *)h; j->S = S; j->P = P; j->max_visits = max_visits;
            j->tet = out_tet; j->len = out_len; j->cond = out_cond; j->count = out_count;
            j->status = status;
            split(n, nthreads, i, &j->begin, &j->end);
            pthread_create(&th[i], NULL, trace_walk_worker, j);
        }
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
        for (int i = 0; i < nthreads; ++i) if (jobs[i].rc) rc = jobs[i].rc;
    }
    free(th);
    free(jobs);
    return rc;
}
