// FP32 tests of the anisotropic shapes with certified margins.
//
// Each test returns 1 (overlap, certain), 0 (no overlap, certain) or -1
// (within the margin: the caller re-takes the decision with the exact FP64
// statement in hpmc_shapes.cuh).  "Certain" means: true for the exact poses
// the FP32 values approximate, given the host-derived bounds
//   * E_pos: error of a cell-relative FP32 coordinate difference,
//   * 64 u |v|: error of rotating v with an FP32 frame built from an FP32
//     quaternion (rounded from the FP64 state, or the FP32 image of a
//     rotation proposal),
// folded into one distance margin Rep::m_d (depletant tests) and one margin
// Rep::m_pair (colloid pairs).  The point-to-body distance is 1-Lipschitz in
// the point, and a body's support function is R_circ-Lipschitz in the
// direction, which is what turns coordinate errors into distance errors.
// Since the FP64 statement decides exactly except within ~1e-12 of contact, a
// certain FP32 decision equals the FP64 decision.
#pragma once

#include "hpmc_common.cuh"
#include "hpmc_shapes.cuh"

namespace hpmc {

struct Frame32 {
    float m[9];   // body -> lab rotation, row major
};

// Rotation matrix of the (unit) quaternion q = (s, x, y, z) = (q.x .. q.w).
__device__ __forceinline__ Frame32 frame32(float4 q)
{
    const float s = q.x, x = q.y, y = q.z, z = q.w;
    Frame32 F;
    F.m[0] = 1.0f - 2.0f * (y * y + z * z);
    F.m[1] = 2.0f * (x * y - s * z);
    F.m[2] = 2.0f * (x * z + s * y);
    F.m[3] = 2.0f * (x * y + s * z);
    F.m[4] = 1.0f - 2.0f * (x * x + z * z);
    F.m[5] = 2.0f * (y * z - s * x);
    F.m[6] = 2.0f * (x * z - s * y);
    F.m[7] = 2.0f * (y * z + s * x);
    F.m[8] = 1.0f - 2.0f * (x * x + y * y);
    return F;
}

__device__ __forceinline__ float3 to_body32(const Frame32 &F, float3 v)
{
    return make_float3(F.m[0] * v.x + F.m[3] * v.y + F.m[6] * v.z,
                       F.m[1] * v.x + F.m[4] * v.y + F.m[7] * v.z,
                       F.m[2] * v.x + F.m[5] * v.y + F.m[8] * v.z);
}

__device__ __forceinline__ float3 to_lab32(const Frame32 &F, float3 b)
{
    return make_float3(F.m[0] * b.x + F.m[1] * b.y + F.m[2] * b.z,
                       F.m[3] * b.x + F.m[4] * b.y + F.m[5] * b.z,
                       F.m[6] * b.x + F.m[7] * b.y + F.m[8] * b.z);
}

__device__ __forceinline__ float dot3f(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3f(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 sub3f(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 add3f(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 scale3f(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }

__device__ __forceinline__ int tri_less(float d, float thr, float m)
{
    return d < thr - m ? 1 : (d > thr + m ? 0 : -1);
}

// Spheroid (a, a, c), body point p, outside the quick tests below: certified
// "dist(p, E) < r" by Newton's method for the meridian foot point, which
// gives an ellipse point X (an upper bound |P - X| on the distance) and its
// normal n (a lower bound n.P - h(n), h the ellipse's support function).
__device__ __noinline__ int spheroid_newton32(float a, float c, float r, float m, float rho2, float z)
{
    const float A2 = a * a, C2 = c * c;
    const float rho = sqrtf(rho2);
    float t = 0.0f;
    // the certificate holds for any t (X is a point of the ellipse, n its
    // normal there), so it is tried after a few steps and the iteration stops
    // as soon as it decides
#pragma unroll 1
    for (int it = 1; it <= 24; ++it) {
        const float d1 = t + A2, d2 = t + C2;
        const float g1 = a * rho / d1, g2 = c * z / d2;
        const float F = g1 * g1 + g2 * g2 - 1.0f;
        const float D = g1 * g1 / d1 + g2 * g2 / d2;
        const float tn = t + F / (2.0f * D);
        const bool done = !(tn > t) || it == 24;
        if (!done) t = tn;
        if (done || it == 3 || it == 6 || it == 12) {
            // foot point, projected radially onto the ellipse
            float x0 = A2 * rho / (t + A2), x1 = C2 * z / (t + C2);
            const float sc = rsqrtf(x0 * x0 / A2 + x1 * x1 / C2);
            x0 *= sc;
            x1 *= sc;
            const float e0 = rho - x0, e1 = z - x1;
            const float hi = sqrtf(e0 * e0 + e1 * e1);
            // outward normal of the ellipse at X
            float n0 = x0 / A2, n1 = x1 / C2;
            const float nl = rsqrtf(n0 * n0 + n1 * n1);
            n0 *= nl;
            n1 *= nl;
            const float lo = n0 * rho + n1 * z - sqrtf(A2 * n0 * n0 + C2 * n1 * n1);
            if (hi < r - m) return 1;
            if (lo > r + m) return 0;
            if (done) return -1;
        }
    }
    return -1;
}

// Spheroid quick tests, with s_X^2 = rho^2 / A^2 + z^2 / C^2 for a spheroid X
// of semi-axes (A, A, C): inside E (s_E <= 1): overlap.  Inside the inner
// spheroid (a + r, c + r), which lies inside E + ball(r), by more than m
// (s_in < 1 - m / min semi-axis): overlap.  Outside the outer spheroid
// (host: the smallest coaxial one containing E + ball(r) with one axis equal
// to its extent) by more than m (s_out > 1 + m / min semi-axis): none.  A
// point on the boundary of sX is at least (s - 1) min(A, C) from X, which
// turns the s thresholds into distances.  The band between inner and outer
// spheroid (~2% of the sampling ball for the discoid) goes to Newton.
__device__ __forceinline__ int spheroid_tri32(const Rep &R, float m, float3 p)
{
    const float rho2 = p.x * p.x + p.y * p.y;
    const float z2 = p.z * p.z;
    if (rho2 * R.sp_iA2 + z2 * R.sp_iC2 <= 1.0f) return 1;
    if (rho2 * R.sp_inA + z2 * R.sp_inC < R.sp_kin2) return 1;
    if (rho2 * R.sp_outA + z2 * R.sp_outC > R.sp_kout2) return 0;
    return spheroid_newton32(R.sh_a32, R.sh_c32, R.r_dep32, m, rho2, fabsf(p.z));
}

// Depletant at v (lab frame, relative to the colloid's reference point)
// against an anisotropic colloid with frame F.
__device__ __forceinline__ int dep_tri32(const Rep &R, float3 v, const Frame32 &F)
{
    const float m = R.m_d;
    const float Rr = R.R_circ32 + R.r_dep32;
    const float v2 = dot3f(v, v);
    if (v2 > (Rr + m) * (Rr + m)) return 0;
    const float3 p = to_body32(F, v);
    const float r = R.r_dep32;
    if (R.shape == kHemisphere) {
        const float Rh = R.sh_R32;
        float d;
        if (p.z >= 0.0f) {
            d = sqrtf(dot3f(p, p)) - Rh;
            if (d < 0.0f) d = 0.0f;
        } else {
            const float rho2 = p.x * p.x + p.y * p.y;
            if (rho2 <= Rh * Rh) {
                d = -p.z;
            } else {
                const float dr = sqrtf(rho2) - Rh;
                d = sqrtf(dr * dr + p.z * p.z);
            }
        }
        return tri_less(d, r, m);
    }
    return spheroid_tri32(R, m, p);
}

// Support point (body frame) in direction n, FP32.
__device__ __forceinline__ float3 support_body32(const Rep &R, float3 n)
{
    if (R.shape == kHemisphere) {
        const float Rh = R.sh_R32;
        if (n.z >= 0.0f) {
            const float l2 = dot3f(n, n);
            if (l2 > 0.0f) return scale3f(n, Rh * rsqrtf(l2));
        } else {
            const float rho2 = n.x * n.x + n.y * n.y;
            if (rho2 > 0.0f) {
                const float k = Rh * rsqrtf(rho2);
                return make_float3(n.x * k, n.y * k, 0.0f);
            }
        }
        return make_float3(0.0f, 0.0f, 0.0f);
    }
    const float A2 = R.sh_a32 * R.sh_a32, C2 = R.sh_c32 * R.sh_c32;
    const float h2 = A2 * (n.x * n.x + n.y * n.y) + C2 * n.z * n.z;
    if (!(h2 > 0.0f)) return make_float3(0.0f, 0.0f, 0.0f);
    const float k = rsqrtf(h2);
    return make_float3(A2 * n.x * k, A2 * n.y * k, C2 * n.z * k);
}

// Depth of a body point inside the body (a lower bound on the distance to its
// boundary; negative outside): hemisphere min(R - |p|, p_z); spheroid
// (1 - s) c with s the spheroid "radius" of p (the ball of radius (1 - s) c
// around p lies in the body).
__device__ __forceinline__ float depth32(const Rep &R, float3 p)
{
    if (R.shape == kHemisphere) return fminf(R.sh_R32 - sqrtf(dot3f(p, p)), p.z);
    const float s2 = (p.x * p.x + p.y * p.y) / (R.sh_a32 * R.sh_a32) + p.z * p.z / (R.sh_c32 * R.sh_c32);
    return (1.0f - sqrtf(s2)) * fminf(R.sh_a32, R.sh_c32);
}

struct Body32 {
    Frame32 F;
    float3 x;        // reference point (lab, relative to the moved colloid's new position)
};

__device__ __forceinline__ float3 sup_lab32(const Rep &R, const Body32 &B, float3 n)
{
    return add3f(to_lab32(B.F, support_body32(R, to_body32(B.F, n))), B.x);
}

__device__ __forceinline__ float3 interior32(const Rep &R, const Body32 &B)
{
    const float3 b = make_float3(0.0f, 0.0f, R.shape == kHemisphere ? 0.5f * R.sh_R32 : 0.0f);
    return add3f(to_lab32(B.F, b), B.x);
}

struct PairTri {
    int res;       // 1 overlap, 0 separated, -1 undecided
    float3 n;      // last portal normal (a separating / contact direction estimate)
};

// Colloid-colloid test in FP32: the portal refinement of hpmc_shapes.cuh run
// in FP32, with certificates instead of tolerances.  Separated: a direction n
// whose computed support value of M = B - A is below -m_pair.  Overlap: the
// midpoint of A's and B's support points along the converged portal normal
// lies inside both bodies by more than m_pair.  Anything else is undecided.
__device__ __noinline__ PairTri pair_tri32(const Rep &R, const Body32 &A, const Body32 &B)
{
    PairTri out;
    out.res = -1;
    const float m = R.m_pair;
    const float3 v0 = sub3f(interior32(R, B), interior32(R, A));
    float3 n = scale3f(v0, -1.0f);
    out.n = n;
    if (dot3f(v0, v0) < 1e-12f) return out;
    auto supd = [&](float3 d, float3 &a, float3 &b) {
        b = sup_lab32(R, B, d);
        a = sup_lab32(R, A, scale3f(d, -1.0f));
        return sub3f(b, a);
    };
    auto sep_cert = [&](float3 v, float3 d) {
        const float l2 = dot3f(d, d);
        return l2 > 0.0f && dot3f(v, d) * rsqrtf(l2) < -m;
    };
    float3 a, b;
    float3 v1 = supd(n, a, b);
    if (dot3f(v1, n) <= 0.0f) {
        out.res = sep_cert(v1, n) ? 0 : -1;
        return out;
    }
    n = cross3f(v1, v0);
    if (dot3f(n, n) < 1e-20f) return out;
    float3 v2 = supd(n, a, b);
    if (dot3f(v2, n) <= 0.0f) {
        out.res = sep_cert(v2, n) ? 0 : -1;
        out.n = n;
        return out;
    }
    n = cross3f(sub3f(v1, v0), sub3f(v2, v0));
    if (dot3f(n, v0) > 0.0f) {
        const float3 t = v1;
        v1 = v2;
        v2 = t;
        n = scale3f(n, -1.0f);
    }
    float3 v3 = v1;
    bool found = false;
#pragma unroll 1
    for (int it = 0; it < 32 && !found; ++it) {
        v3 = supd(n, a, b);
        if (dot3f(v3, n) <= 0.0f) {
            out.res = sep_cert(v3, n) ? 0 : -1;
            out.n = n;
            return out;
        }
        if (dot3f(cross3f(v1, v3), v0) < 0.0f) {
            v2 = v3;
            n = cross3f(sub3f(v1, v0), sub3f(v3, v0));
            continue;
        }
        if (dot3f(cross3f(v3, v2), v0) < 0.0f) {
            v1 = v3;
            n = cross3f(sub3f(v3, v0), sub3f(v2, v0));
            continue;
        }
        found = true;
    }
    if (!found) return out;
    bool hit = false;
#pragma unroll 1
    for (int it = 0; it < 32; ++it) {
        n = cross3f(sub3f(v2, v1), sub3f(v3, v1));
        const float l2 = dot3f(n, n);
        if (!(l2 > 1e-30f)) break;
        n = scale3f(n, rsqrtf(l2));
        out.n = n;
        if (dot3f(n, v1) >= 0.0f) hit = true;
        const float3 v4 = supd(n, a, b);
        const float h = dot3f(v4, n);
        if (h < -m) {
            out.res = 0;
            return out;
        }
        if (h <= 0.0f) break;
        if (dot3f(sub3f(v4, v3), n) <= 2e-6f) {
            // converged: try the overlap witness along n
            if (hit || h > m) {
                const float3 x = scale3f(add3f(a, b), 0.5f);
                const float gA = depth32(R, to_body32(A.F, sub3f(x, A.x)));
                const float gB = depth32(R, to_body32(B.F, sub3f(x, B.x)));
                if (gA > m && gB > m) out.res = 1;
            }
            return out;
        }
        if (dot3f(cross3f(v4, v1), v0) < 0.0f) {
            if (dot3f(cross3f(v4, v2), v0) < 0.0f) v1 = v4;
            else v3 = v4;
        } else {
            if (dot3f(cross3f(v4, v3), v0) < 0.0f) v2 = v4;
            else v1 = v4;
        }
    }
    // not converged: a last witness try along the final normal
    if (hit) {
        const float3 v4 = supd(out.n, a, b);
        (void)v4;
        const float3 x = scale3f(add3f(a, b), 0.5f);
        const float gA = depth32(R, to_body32(A.F, sub3f(x, A.x)));
        const float gB = depth32(R, to_body32(B.F, sub3f(x, B.x)));
        if (gA > m && gB > m) out.res = 1;
    }
    return out;
}

// FP64 certificates seeded by an FP32 direction n (A at the origin, B at xb):
// separated if the support value of M along n is below -1e-11, overlapping
// if the midpoint of the two support points lies inside both bodies with
// depths summing to more than 1e-11 (M then contains a ball of that radius
// around the origin).  Both are beyond the FP64 statement's 1e-12 tolerance,
// so they agree with it.  -1 if neither holds.
__device__ __forceinline__ double depth64(const Rep &R, Vec3 p)
{
    if (R.shape == kHemisphere) return fmin(R.sh_R - sqrt(dot3(p, p)), p.z);
    const double s2 = (p.x * p.x + p.y * p.y) / (R.sh_a * R.sh_a) + p.z * p.z / (R.sh_c * R.sh_c);
    return (1.0 - sqrt(s2)) * fmin(R.sh_a, R.sh_c);
}

__device__ __noinline__ int pair_cert64(const Rep &R, double4 qa, double4 qb, Vec3 xb, float3 nf)
{
    const double l = sqrt((double)nf.x * nf.x + (double)nf.y * nf.y + (double)nf.z * nf.z);
    if (!(l > 0.0)) return -1;
    const Vec3 n = v3(nf.x / l, nf.y / l, nf.z / l);
    const Vec3 zero = v3(0.0, 0.0, 0.0);
    const Vec3 b = support_lab(R, qb, xb, n);
    const Vec3 a = support_lab(R, qa, zero, v3(-n.x, -n.y, -n.z));
    const double h = dot3(sub3(b, a), n);
    if (h < -1e-11) return 0;
    const Vec3 x = v3(0.5 * (a.x + b.x), 0.5 * (a.y + b.y), 0.5 * (a.z + b.z));
    const double gA = depth64(R, rot_to_body(qa, x));
    const double gB = depth64(R, rot_to_body(qb, sub3(x, xb)));
    if (gA > 0.0 && gB > 0.0 && gA + gB > 1e-11) return 1;
    return -1;
}

}  // namespace hpmc
