// faceclip.cuh -- the paper's face samples of Sec. 4.1 ("Face samples") for
// one (slave triangle, master triangle) pair, shared by the standalone
// sampler (ipc_face_clip_samples) and the contact pass in its clipped-
// overlap mode.
//
// Both triangles are projected onto the tangent plane of the slave triangle
// T_s, the projected master triangle is clipped by T_s (Sutherland-Hodgman,
// one directed edge of T_s at a time), the clipped polygon is triangulated
// as a fan from its first vertex, and every sub-triangle gets the 3-point,
// degree-2 Gauss rule (points at barycentric coordinates (2/3, 1/6, 1/6) and
// permutations, weight one third of its area).  Each sample point lies on
// T_s; cast along the slave normal it meets the master plane, which gives
// the gap (Eq. gap) and the master barycentrics (Eq. gram).  Translation
// units that include this must be compiled without FMA contraction (each
// product and sum rounded once), so that the clipping decisions are those of
// a plain IEEE evaluation in this operation order.
#pragma once
#include <cmath>

namespace gmcp {
namespace fclip {

constexpr int kMaxPoly = 9;   // a triangle clipped by three half-planes keeps at most 6 vertices
constexpr int kMaxSamples = 12;

struct P3 {
    double x, y, z;
};
__device__ __forceinline__ P3 at(const double* X, int64_t v) { return {X[3 * v], X[3 * v + 1], X[3 * v + 2]}; }
__device__ __forceinline__ P3 minus(P3 a, P3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dotp(P3 a, P3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ P3 crossp(P3 a, P3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// signed area test of p against the directed edge a -> b (left = positive)
__device__ __forceinline__ double side(const double* a, const double* b, const double* p) {
    return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0]);
}

// The samples of slave triangle (s0, s1, s2) against master triangle (m0, m1,
// m2): emit(bs, bm, g, w) is called for each, with the slave and master
// barycentrics bs[3], bm[3], the gap g along the slave normal and the weight
// w; returns their number (0 to 12; 0 when the overlap has no area or the
// master plane contains the slave normal).
template <class Emit>
__device__ __forceinline__ int clip_samples(P3 s0, P3 s1, P3 s2, P3 m0, P3 m1, P3 m2, Emit&& emit) {
    // plane basis: n = e1 x e2 normalised, t1 along e1, t2 = n x t1
    const P3 e1 = minus(s1, s0), e2 = minus(s2, s0);
    P3 nn = crossp(e1, e2);
    const double nl = sqrt(dotp(nn, nn));
    nn = {nn.x / nl, nn.y / nl, nn.z / nl};
    const double l1 = sqrt(dotp(e1, e1));
    const P3 t1 = {e1.x / l1, e1.y / l1, e1.z / l1};
    const P3 t2 = crossp(nn, t1);
    double A[3][2], poly[kMaxPoly][2], tmp[kMaxPoly][2];
    const P3 sv[3] = {s0, s1, s2}, mv[3] = {m0, m1, m2};
    for (int c = 0; c < 3; ++c) {
        const P3 d = minus(sv[c], s0);
        A[c][0] = dotp(d, t1); A[c][1] = dotp(d, t2);
        const P3 q = minus(mv[c], s0);
        poly[c][0] = dotp(q, t1); poly[c][1] = dotp(q, t2);
    }
    int m = 3;
    for (int e = 0; e < 3 && m > 0; ++e) {
        const double* a = A[e];
        const double* b = A[(e + 1) % 3];
        int mo = 0;
        for (int q = 0; q < m; ++q) {
            const double* pp = poly[(q + m - 1) % m];
            const double* qq = poly[q];
            const double sp = side(a, b, pp), sq = side(a, b, qq);
            if (sq >= 0.0) {
                if (sp < 0.0) {
                    const double t = sp / (sp - sq);
                    tmp[mo][0] = pp[0] + t * (qq[0] - pp[0]); tmp[mo][1] = pp[1] + t * (qq[1] - pp[1]); ++mo;
                }
                tmp[mo][0] = qq[0]; tmp[mo][1] = qq[1]; ++mo;
            } else if (sp >= 0.0) {
                const double t = sp / (sp - sq);
                tmp[mo][0] = pp[0] + t * (qq[0] - pp[0]); tmp[mo][1] = pp[1] + t * (qq[1] - pp[1]); ++mo;
            }
        }
        m = mo;
        for (int q = 0; q < m; ++q) { poly[q][0] = tmp[q][0]; poly[q][1] = tmp[q][1]; }
    }
    if (m < 3) return 0;
    const P3 f1 = minus(m1, m0), f2 = minus(m2, m0);
    const P3 N = crossp(f1, f2);
    const double den = dotp(N, nn);
    if (den == 0.0) return 0;
    const double a11 = A[1][0] - A[0][0], a12 = A[2][0] - A[0][0];
    const double a21 = A[1][1] - A[0][1], a22 = A[2][1] - A[0][1];
    const double det = a11 * a22 - a12 * a21;
    // master Gram system (Eq. gram)
    const double g11 = dotp(f1, f1), g12 = dotp(f1, f2), g22 = dotp(f2, f2);
    const double gdet = g11 * g22 - g12 * g12;
    const double w1 = 2.0 / 3.0, w2 = 1.0 / 6.0;
    int ns = 0;
    for (int f = 1; f + 1 < m; ++f) {
        const double *q0 = poly[0], *q1 = poly[f], *q2 = poly[f + 1];
        const double area = 0.5 * fabs((q1[0] - q0[0]) * (q2[1] - q0[1]) - (q1[1] - q0[1]) * (q2[0] - q0[0]));
        if (!(area > 0.0)) continue;
        for (int gp = 0; gp < 3; ++gp) {
            const double c0 = gp == 0 ? w1 : w2, c1 = gp == 1 ? w1 : w2, c2 = gp == 2 ? w1 : w2;
            const double u = c0 * q0[0] + c1 * q1[0] + c2 * q2[0];
            const double v = c0 * q0[1] + c1 * q1[1] + c2 * q2[1];
            const double ru = u - A[0][0], rv = v - A[0][1];
            const double b1 = (a22 * ru - a12 * rv) / det;
            const double b2 = (a11 * rv - a21 * ru) / det;
            const double b0 = 1.0 - b1 - b2;
            const P3 x = {b0 * s0.x + b1 * s1.x + b2 * s2.x, b0 * s0.y + b1 * s1.y + b2 * s2.y,
                          b0 * s0.z + b1 * s1.z + b2 * s2.z};
            const double g = dotp(N, minus(m0, x)) / den;
            const P3 hit = {x.x + g * nn.x, x.y + g * nn.y, x.z + g * nn.z};
            const P3 d = minus(hit, m0);
            const double r1 = dotp(d, f1), r2 = dotp(d, f2);
            const double bm1 = (g22 * r1 - g12 * r2) / gdet;
            const double bm2 = (g11 * r2 - g12 * r1) / gdet;
            const double bs[3] = {b0, b1, b2}, bm[3] = {1.0 - bm1 - bm2, bm1, bm2};
            emit(bs, bm, g, area / 3.0);
            ++ns;
        }
    }
    return ns;
}

}  // namespace fclip
}  // namespace gmcp
