// predicates.cuh -- exact-sign side predicates for ray / tet-edge tests.
//
// The paper's tet-ray intersection (Sec. II-C) is four ray-triangle tests, and
// its robustness discussion (Sec. II-C, II-C.1, II-D) is about those tests
// misfiring near edges and vertices: leaks (halted rays) and loops (the
// Fig. 3 configuration).  Its answer is an epsilon that grows by 10x until two
// faces are hit (Alg. 1, Alg. 2) plus FP64 arithmetic.  This file replaces
// that with a decision procedure that cannot misfire:
//
//   side(S, P, p, q) = det[P - S, p - S, q - S]
//
// is the Pluecker side of the ray line S->P against the directed edge p->q.
// A line crosses a triangle iff the three edge sides agree in sign, and the
// exit face of a tet entered through face (a, b, c) follows from the signs of
// side(n->a), side(n->b), side(n->c) alone (n = the fourth vertex).  Every tet
// that shares an edge evaluates the same function of the same FP64 inputs, so
// as long as each evaluation returns the EXACT sign the walk is consistent.
//
// Cascade (cheapest first; each stage is only trusted when provably right):
//   1. FP32 with a forward error bound (inputs rounded from FP64 included).
//   2. FP64 with a forward error bound.
//   3. Exact: expansion arithmetic (error-free two-sum / FMA two-product and
//      expansion sums after Shewchuk 1997, written here from the published
//      algorithms).
//   4. The exact value is 0: the ray line meets the edge line.  The sign is
//      then that of the symbolically perturbed line through
//      S + (e, e^2, e^4) and P + (e^8, e^16, e^32), e -> 0+ (Simulation of
//      Simplicity, Edelsbrunner & Muecke 1990, applied to the ray instead of
//      the vertices).  side is affine in S and in P, so its expansion in e
//      has the constant term, the gradients
//         d side/dS = -(p - P) x (q - P),   d side/dP = (p - S) x (q - S)
//      at exponents (1, 2, 4) and (8, 16, 32), and the bilinear term
//      (q - p).(s x r) at exponents 2^i + 2^(3+j).  The first non-zero
//      coefficient in exponent order decides.  All tets see the same perturbed
//      line, so the walk follows it: no backtracking and no loops.
//
// All code here is __host__ __device__ so the host build can be tested on the
// CPU against exact rationals.  Non-inlined functions take points by value.  Compile with FMA contraction OFF (nvcc
// -fmad=false, gcc -ffp-contract=off): every fused multiply-add below is an
// explicit fma()/fmaf() call, which the error bounds account for.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define TP_HD __host__ __device__ __forceinline__
#define TP_HDN static __host__ __device__ __noinline__
#else
#define TP_HD inline
#define TP_HDN static
#endif
// Expansion primitives are kept out of line on the device: with nvcc 13.0 the
// fully inlined exact 2-D orientation of (a, a, c) returned a non-zero sign
// (the optimiser mis-evaluated the chain of inlined expansion sums; storing
// the intermediates, or calling the same primitives out of line, gave 0).
// The device/host cascade comparison test guards this.
#define TP_EXP TP_HDN

namespace tp {

struct d3 { double x, y, z; };
struct f3 { float x, y, z; };

TP_HD d3 mk(double x, double y, double z) { return {x, y, z}; }
TP_HD f3 mkf(float x, float y, float z) { return {x, y, z}; }
TP_HD f3 tof(const d3 &a) { return {(float)a.x, (float)a.y, (float)a.z}; }
TP_HD d3 sub(const d3 &a, const d3 &b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
TP_HD f3 sub(const f3 &a, const f3 &b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
TP_HD d3 dabs(const d3 &a) { return {fabs(a.x), fabs(a.y), fabs(a.z)}; }
TP_HD f3 fabs3(const f3 &a) { return {fabsf(a.x), fabsf(a.y), fabsf(a.z)}; }

// cross product with one FMA per component: c_x = a_y b_z - a_z b_y
TP_HD f3 crossf(const f3 &a, const f3 &b) {
    return {fmaf(a.y, b.z, -(a.z * b.y)), fmaf(a.z, b.x, -(a.x * b.z)),
            fmaf(a.x, b.y, -(a.y * b.x))};
}
TP_HD d3 crossd(const d3 &a, const d3 &b) {
    return {fma(a.y, b.z, -(a.z * b.y)), fma(a.z, b.x, -(a.x * b.z)),
            fma(a.x, b.y, -(a.y * b.x))};
}
// |a| x |b| with absolute values: the magnitude that bounds the cross product
TP_HD f3 abscrossf(const f3 &a, const f3 &b) {
    return {fmaf(a.y, b.z, a.z * b.y), fmaf(a.z, b.x, a.x * b.z), fmaf(a.x, b.y, a.y * b.x)};
}
TP_HD d3 abscrossd(const d3 &a, const d3 &b) {
    return {fma(a.y, b.z, a.z * b.y), fma(a.z, b.x, a.x * b.z), fma(a.x, b.y, a.y * b.x)};
}
TP_HD float dotf(const f3 &a, const f3 &b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
TP_HD double dotd(const d3 &a, const d3 &b) { return fma(a.x, b.x, fma(a.y, b.y, a.z * b.z)); }

// ------------------------------------------------------------------ FP32 stage
//
// side(S, P, p, q) = det[D, p - O, q - p] for ANY point O of the ray line
// (D = P - S); the FP32 stage uses the midpoint O = (S + P)/2, which keeps
// |p - O| ~ the object size instead of the source distance.  For one vertex n
// shared by three edges n->k the walk computes  w = d32 x (n32 - O32)  once and
// side(n->k) ~ w . (k32 - n32).  Error analysis (u = 2^-24, round to nearest;
// d32 = fl32(fl64(P - S)), O32 = fl32(fl64(S + P)/2), x32 = fl32(x)):
//   |side32 - side| <= u [ Z1 . |e| + Z2 . (|k| + |n|) ] + O(u^2)
//   Z1 = 3.02 X + Y + 4.01 |w|,   Z2 = 1.01 |w| + 1e-6 (X + Y)
// with a = n - O, e = k - n, X = |d| x |a| and Y = |d| x Ma, where x is the
// cross product of absolute values and Ma = |a| + 1.01 (|n| + |O|) +
// 1e-8 max_i(|S_i| + |P_i|) bounds |a32 - (n - O)| / u.  Terms: 3.01u|w|.|e| for the
// FMA dot, 2.01u X.|e| for the FMA cross, and the input errors |dd| <=
// 1.01u|d|, |da| <= u Ma, |de| <= u(|e| + 1.01|k| + 1.01|n|) pushed through the
// trilinear form; the de term multiplies |D x A| <= |w| + u(3.02 X + Y), whence
// |w| (small when n is near the ray) and the 1e-6 (X + Y) guard in Z2.  The
// constant is 2^-24 * 1.0234: it covers the O(u^2) terms and the rounding of
// the bound itself (non-negative terms, ~10 operations).
//   Per edge the walk evaluates a bound that is never below the one above,
// in a folded form with per-vertex Z, c and a per-ray guard G:
//     u [ Z . |e32| + c ],   Z = 3.03 X + 5.04 |w| + Y',   c = 2.05 |w| . |n| + G,
// with Y' = |d| x Ma' and Ma' = 1.0101 (|n| + |O|) + 1.00002 |a| +
// 1.00002e-8 max_i(|S_i| + |P_i|) >= 1.00002 Ma.  As x is linear in its second
// argument, 3.03 X + Y' = |d| x M2 with M2 = 4.031 |a| + 1.0101 (|n| + |O|) +
// 1.00002e-8 max_i(|S_i| + |P_i|), one product instead of two.  Why it dominates: |k| <=
// |n| + |k - n| and |k - n| <= (1 + 1.01u)|e32| (e32 = fl(k - n)), so
// Z2 . (|k| + |n|) <= 1.01 Z2 . |e32| + 2.02 Z2 . |n|; expanding Z1 + 1.01 Z2
// gives 3.02 X + 5.0301 |w| + Y plus 1.01e-6 (X + Y), which 3.03 X and Y'
// cover; 2.02 Z2 . |n| = 2.0402 |w| . |n| + 2.02e-6 (X + Y) . |n|, and the
// second term is at most G = 2.03e-6 R sum_i (Xm + Ym)_i, where R >= every
// |n32_i| of the mesh, Xm = |d| x A and Ym = |d| x (A + 1.01 (R + |O|) +
// Oext) with A = 1.001 (R + |O|) >= |a32| (so X <= Xm, Y <= Ym).  The factors'
// slack (>= 0.2%) covers the roundings of Z, c and G.  Per vertex this costs
// about 50 operations, per edge one dot product and one FMA.
struct Filt32Ray {
    f3 O, d;     // midpoint and direction, rounded to FP32
    float Oext;  // 1.00002e-8 max_i(|S_i| + |P_i|): covers fl64 rounding of (S + P)/2
    float G;     // guard of the folded bound (see above)
};
struct Filt32Vert {
    f3 n, w, Z;
    float c;
};
#define TP_FILT32_U 6.1e-8f
#define TP_FILT32_TINY 1e-30f

// R: an upper bound of |coordinate| over every FP32 vertex the ray is tested
// against (the mesh radius, rounded up)
TP_HD Filt32Ray filt32_ray(const d3 &S, const d3 &P, float R) {
    Filt32Ray r;
    d3 O = {(S.x + P.x) * 0.5, (S.y + P.y) * 0.5, (S.z + P.z) * 0.5};
    r.O = tof(O);
    r.d = tof(sub(P, S));
    double e = fmax(fmax(fabs(S.x) + fabs(P.x), fabs(S.y) + fabs(P.y)), fabs(S.z) + fabs(P.z));
    r.Oext = 1.00002e-8f * (float)e;
    const f3 Oabs = fabs3(r.O), dabs = fabs3(r.d);
    const f3 A = {1.001f * (R + Oabs.x), 1.001f * (R + Oabs.y), 1.001f * (R + Oabs.z)};
    const f3 M = {fmaf(2.011f, R + Oabs.x, r.Oext), fmaf(2.011f, R + Oabs.y, r.Oext),
                  fmaf(2.011f, R + Oabs.z, r.Oext)};
    const f3 Xm = abscrossf(dabs, A), Ym = abscrossf(dabs, M);
    r.G = 2.03e-6f * R * ((Xm.x + Ym.x) + (Xm.y + Ym.y) + (Xm.z + Ym.z));
    return r;
}
TP_HD Filt32Vert filt32_vert(const Filt32Ray &r, const f3 &n) {
    Filt32Vert v;
    v.n = n;
    const f3 a = sub(n, r.O);
    v.w = crossf(r.d, a);
    const f3 nabs = fabs3(n), aabs = fabs3(a), dabs = fabs3(r.d), Oabs = fabs3(r.O);
    const f3 M2 = {fmaf(4.031f, aabs.x, fmaf(1.0101f, nabs.x + Oabs.x, r.Oext)),
                   fmaf(4.031f, aabs.y, fmaf(1.0101f, nabs.y + Oabs.y, r.Oext)),
                   fmaf(4.031f, aabs.z, fmaf(1.0101f, nabs.z + Oabs.z, r.Oext))};
    const f3 wa = fabs3(v.w);
    // Z = |d| x M2 + 5.04 |w|
    v.Z = {fmaf(dabs.y, M2.z, fmaf(dabs.z, M2.y, 5.04f * wa.x)),
           fmaf(dabs.z, M2.x, fmaf(dabs.x, M2.z, 5.04f * wa.y)),
           fmaf(dabs.x, M2.y, fmaf(dabs.y, M2.x, 5.04f * wa.z))};
    v.c = fmaf(2.05f, dotf(wa, nabs), r.G);
    return v;
}
// side(n->k) with e = k - n already computed: value, its error bound, and the
// certain sign (+1/-1) or 0 when |value| does not exceed the bound
TP_HD int filt32_side_e(const Filt32Vert &v, const f3 &e, float &val, float &B) {
    val = dotf(v.w, e);
    const float m = fmaf(v.Z.x, fabsf(e.x), fmaf(v.Z.y, fabsf(e.y), fmaf(v.Z.z, fabsf(e.z), v.c)));
    B = fmaf(TP_FILT32_U, m, TP_FILT32_TINY);
    return (val > B) - (val < -B);
}
TP_HD int filt32_side(const Filt32Vert &v, const f3 &k, float &val, float &B) {
    return filt32_side_e(v, sub(k, v.n), val, B);
}
TP_HD int filt32_side(const Filt32Vert &v, const f3 &k, float &val) {
    float B;
    return filt32_side(v, k, val, B);
}

// ------------------------------------------------------------------ FP64 stage
//
// Same formula in FP64 on exact inputs: |side64 - side| <= 8.04 u64 X.|e|
// (3.01 dot + 2.01 cross + 3 x input differences), u64 = 2^-53; constant
// 8.2 * 2^-53 with margin, plus a tiny absolute term against underflow.
#define TP_FILT64_U 9.1e-16
#define TP_FILT64_TINY 1e-290
struct Filt64Vert {
    d3 n, w, X;
};
TP_HD Filt64Vert filt64_vert(const d3 &S, const d3 &d, const d3 &n) {
    Filt64Vert v;
    v.n = n;
    d3 a = sub(n, S);
    v.w = crossd(d, a);
    v.X = abscrossd(dabs(d), dabs(a));
    return v;
}
TP_HD int filt64_side(const Filt64Vert &v, const d3 &k, double &val, double &B) {
    d3 e = sub(k, v.n);
    val = dotd(v.w, e);
    B = fma(TP_FILT64_U, dotd(v.X, dabs(e)), TP_FILT64_TINY);
    return (val > B) - (val < -B);
}
TP_HD int filt64_side(const Filt64Vert &v, const d3 &k, double &val) {
    double B;
    return filt64_side(v, k, val, B);
}

// A barycentric weight is used as computed only when it exceeds its error
// bound by this factor; otherwise the crossing point it helps place is
// ill-conditioned (the ray nearly lies in the face) and the exact value is
// taken instead.
#define TP_WEIGHT_MARGIN 128.0

// A face the ray meets at an angle whose sine is below 1/64 is crossed at a
// point that FP32 vertices (rounded by up to u |v|) place up to ~u |v| / sin
// off along the ray; such crossings are placed again from the FP64 vertices.
// Above 1/64 the FP32 placement error stays below ~64 u |v| (measured at most
// ~4e-8 / sin on the unit cube, i.e. 7e-7); on jittered meshes about 3e-3 of
// crossings fall below it (the test's 1-norm also flags some up to sqrt(3)/64).
#define TP_GRAZE_SIN (1.0f / 64.0f)

// ------------------------------------------------------- exact arithmetic
// An expansion is an array of doubles, non-overlapping, increasing magnitude;
// its value is the exact sum, and its sign is that of the last component.

TP_HD void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    double bv = s - a;
    double av = s - bv;
    e = (a - av) + (b - bv);
}
TP_HD void two_prod(double a, double b, double &p, double &e) {
    p = a * b;
    e = fma(a, b, -p);
}

// h = e + f, zero-eliminating; returns |h|.  Merges by magnitude, then a chain
// of two-sums (Fast-Expansion-Sum of the 1997 paper).  h may not alias e or f.
TP_EXP int exp_sum(int elen, const double *e, int flen, const double *f, double *h) {
    int i = 0, j = 0, n = 0;
    double Q;
    if (elen == 0 && flen == 0) { h[0] = 0.0; return 1; }
    if (j >= flen || (i < elen && fabs(e[i]) <= fabs(f[j]))) Q = e[i++];
    else Q = f[j++];
    while (i < elen || j < flen) {
        double g;
        if (j >= flen || (i < elen && fabs(e[i]) <= fabs(f[j]))) g = e[i++];
        else g = f[j++];
        double s, err;
        two_sum(Q, g, s, err);
        if (err != 0.0) h[n++] = err;
        Q = s;
    }
    if (Q != 0.0 || n == 0) h[n++] = Q;
    return n;
}
// h = b * e, zero-eliminating (Scale-Expansion); h may not alias e.
TP_EXP int exp_scale(int elen, const double *e, double b, double *h) {
    int n = 0;
    double Q, hh;
    two_prod(e[0], b, Q, hh);
    if (hh != 0.0) h[n++] = hh;
    for (int i = 1; i < elen; ++i) {
        double T, t, s;
        two_prod(e[i], b, T, t);
        two_sum(Q, t, s, hh);
        if (hh != 0.0) h[n++] = hh;
        two_sum(T, s, Q, hh);
        if (hh != 0.0) h[n++] = hh;
    }
    if (Q != 0.0 || n == 0) h[n++] = Q;
    return n;
}
TP_HD int exp_sign(int n, const double *e) {
    double v = e[n - 1];
    return (v > 0.0) - (v < 0.0);
}
// The expansion's value rounded to double: summing its non-overlapping
// components from the smallest up gives it to a few ulps.
TP_HD double exp_approx(int n, const double *e) {
    double v = 0.0;
    for (int k = 0; k < n; ++k) v += e[k];
    return v;
}
// x1*y1 - x2*y2 exactly (<= 4 components); the subtraction negates an input of
// the error-free product, which is exact.
TP_EXP int exp_minor(double x1, double y1, double x2, double y2, double *h) {
    double ah, al, bh, bl;
    two_prod(x1, y1, ah, al);
    two_prod(-x2, y2, bh, bl);
    const double aa[2] = {al, ah};
    const double bb[2] = {bl, bh};
    const int na = (al != 0.0) ? 2 : 1, nb = (bl != 0.0) ? 2 : 1;
    return exp_sum(na, al != 0.0 ? aa : aa + 1, nb, bl != 0.0 ? bb : bb + 1, h);
}

// Exact sign of side(S, P, p, q) = det[P-S, p-S, q-S]; *approx (if given)
// receives its value to a few ulps (used as a barycentric weight when the
// FP64 estimate is below its own error bound).
// With rows a=S, b=P, c=p, d=q and the 4x4 determinant D4 of rows (x, 1):
//   side = -D4 = det3(b,c,d) - det3(a,c,d) + det3(a,b,d) - det3(a,b,c),
//   det3(x,y,z) = x.z m(y,z) - y.z m(x,z) + z.z m(x,y),  m(x,y) = x.x y.y - y.x x.y,
// so side is a signed sum of 12 products z * m(.,.) of exact 4-term minors.
TP_HDN int side_exact_sign(const d3 a, const d3 b, const d3 c, const d3 d, double *approx = nullptr) {
    double m_ab[4], m_ac[4], m_ad[4], m_bc[4], m_bd[4], m_cd[4];
    int n_ab = exp_minor(a.x, b.y, b.x, a.y, m_ab);
    int n_ac = exp_minor(a.x, c.y, c.x, a.y, m_ac);
    int n_ad = exp_minor(a.x, d.y, d.x, a.y, m_ad);
    int n_bc = exp_minor(b.x, c.y, c.x, b.y, m_bc);
    int n_bd = exp_minor(b.x, d.y, d.x, b.y, m_bd);
    int n_cd = exp_minor(c.x, d.y, d.x, c.y, m_cd);
    // 12 terms (minor, coefficient): from the expansion above
    const double *mins[12] = {m_cd, m_bd, m_bc, m_cd, m_ad, m_ac, m_bd, m_ad, m_ab, m_bc, m_ac, m_ab};
    const int lens[12] = {n_cd, n_bd, n_bc, n_cd, n_ad, n_ac, n_bd, n_ad, n_ab, n_bc, n_ac, n_ab};
    const double coef[12] = {b.z, -c.z, d.z, -a.z, c.z, -d.z, a.z, -b.z, d.z, -a.z, b.z, -c.z};
    // accumulate in two buffers alternating at compile time (no dynamic index)
    double A[104], B[104], prod[8];
    int nA = 1, nB = 0, np;
    A[0] = 0.0;
#pragma unroll
    for (int k = 0; k < 12; k += 2) {
        np = exp_scale(lens[k], mins[k], coef[k], prod);
        nB = exp_sum(nA, A, np, prod, B);
        np = exp_scale(lens[k + 1], mins[k + 1], coef[k + 1], prod);
        nA = exp_sum(nB, B, np, prod, A);
    }
    if (approx) *approx = exp_approx(nA, A);
    return exp_sign(nA, A);
}

// Exact sign of the 2-D orientation over axes (i, j):
//   O(a, b, c) = (b_i - a_i)(c_j - a_j) - (b_j - a_j)(c_i - a_i)
//              = m(b, c) - m(a, c) + m(a, b),  m(x, y) = x_i y_j - y_i x_j.
TP_HD double comp(const d3 &v, int axis) { return axis == 0 ? v.x : (axis == 1 ? v.y : v.z); }
TP_HDN int orient2d_sign(const d3 a, const d3 b, const d3 c, int i, int j) {
    double ai = comp(a, i), aj = comp(a, j), bi = comp(b, i), bj = comp(b, j);
    double ci = comp(c, i), cj = comp(c, j);
    // FP64 filter: differences (u each), products, subtraction
    double x1 = bi - ai, y1 = cj - aj, x2 = bj - aj, y2 = ci - ai;
    double v = x1 * y1 - x2 * y2;
    double B = 5.0 * 1.1102230246251565e-16 * (fabs(x1 * y1) + fabs(x2 * y2)) + 1e-300;
    if (v > B) return 1;
    if (v < -B) return -1;
    double m1[4], m2[4], m3[4], t[8], r[12];
    int n1 = exp_minor(bi, cj, ci, bj, m1);   //  m(b, c)
    int n2 = exp_minor(ci, aj, ai, cj, m2);   // -m(a, c)
    int n3 = exp_minor(ai, bj, bi, aj, m3);   //  m(a, b)
    int nt = exp_sum(n1, m1, n2, m2, t);
    int nr = exp_sum(nt, t, n3, m3, r);
    return exp_sign(nr, r);
}

// Symbolic tie-break for side(S, P, p, q) == 0 exactly (see the header).
//   O_yz = axes (1,2), O_zx = (2,0), O_xy = (0,1); (p-S)x(q-S) = (O_yz, O_zx, O_xy)(S, p, q).
TP_HDN int side_sos_sign(const d3 S, const d3 P, const d3 p, const d3 q) {
    int s;
    // exponents 1, 2, 4: -(p - P) x (q - P)
    if ((s = orient2d_sign(P, p, q, 1, 2)) != 0) return -s;
    if ((s = orient2d_sign(P, p, q, 2, 0)) != 0) return -s;
    if ((s = orient2d_sign(P, p, q, 0, 1)) != 0) return -s;
    // exponent 8: ((p - S) x (q - S)).x
    if ((s = orient2d_sign(S, p, q, 1, 2)) != 0) return s;
    // bilinear (q - p).(s x r): exponent 10 -> -(q-p).z, 12 -> (q-p).y
    if (q.z != p.z) return q.z > p.z ? -1 : 1;
    if (q.y != p.y) return q.y > p.y ? 1 : -1;
    // exponent 16: ((p - S) x (q - S)).y
    if ((s = orient2d_sign(S, p, q, 2, 0)) != 0) return s;
    // 17 -> (q-p).z (already zero), 20 -> -(q-p).x
    if (q.x != p.x) return q.x > p.x ? -1 : 1;
    // exponent 32: ((p - S) x (q - S)).z; 33, 34 -> components already zero
    if ((s = orient2d_sign(S, p, q, 0, 1)) != 0) return s;
    return 0;  // p == q
}

// FP64 filter -> exact -> symbolic.  stage: 1 FP64, 2 exact, 3 symbolic.
TP_HDN int side_sign_robust64(const d3 S, const d3 P, const d3 p, const d3 q, int *stage) {
    d3 d = sub(P, S);
    Filt64Vert v = filt64_vert(S, d, p);
    double val;
    int s = filt64_side(v, q, val);
    if (s != 0) { *stage = 1; return s; }
    s = side_exact_sign(S, P, p, q);
    if (s != 0) { *stage = 2; return s; }
    *stage = 3;
    return side_sos_sign(S, P, p, q);
}

// Full cascade from FP64 inputs (used by the validation entry points).
TP_HDN int side_sign_cascade(const d3 S, const d3 P, const d3 p, const d3 q, int *stage) {
    const f3 p32 = tof(p), q32 = tof(q);
    const float R = fmaxf(fmaxf(fmaxf(fabsf(p32.x), fabsf(p32.y)), fabsf(p32.z)),
                          fmaxf(fmaxf(fabsf(q32.x), fabsf(q32.y)), fabsf(q32.z)));
    Filt32Ray r = filt32_ray(S, P, R);
    Filt32Vert v = filt32_vert(r, p32);
    float val;
    int s = filt32_side(v, q32, val);
    if (s != 0) { *stage = 0; return s; }
    return side_sign_robust64(S, P, p, q, stage);
}

}  // namespace tp
