// Anisotropic colloids (Sec. V): hemispheres (Sec. V.A) and discoids, the
// oblate spheroid x^2/a^2 + y^2/a^2 + z^2/c^2 <= 1 (Sec. V.B), with quaternion
// orientations and rotation moves.  Every function is the plain FP64 statement
// of the library's specification, in its operation order (compiled with
// -fmad=false): decisions are bit-identical to any faithful implementation.
//
// Conventions.  Orientation q = (s, u) = (q.x, q.y, q.z, q.w) of a double4, a
// unit quaternion mapping body-frame vectors to the lab frame.  Reference
// point: the centre of a sphere or spheroid; the centre of the flat face of a
// hemisphere, whose face lies in the body plane z = 0 and whose dome is on
// z >= 0.  A depletant (diameter q) overlaps a colloid iff its centre is
// closer than r = q/2 to the body; touching is not an overlap.
#pragma once

#include "hpmc_common.cuh"

namespace hpmc {

enum ShapeKind { kSphere = 0, kHemisphere = 1, kSpheroid = 2 };

struct Vec3 {
    double x, y, z;
};

__device__ __forceinline__ Vec3 v3(double x, double y, double z)
{
    Vec3 v;
    v.x = x;
    v.y = y;
    v.z = z;
    return v;
}
__device__ __forceinline__ double dot3(Vec3 a, Vec3 b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
__device__ __forceinline__ Vec3 cross3(Vec3 a, Vec3 b)
{
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ Vec3 sub3(Vec3 a, Vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ bool is_zero3(Vec3 a) { return a.x == 0.0 && a.y == 0.0 && a.z == 0.0; }

// body -> lab: b + s t + u x t with t = 2 u x b
__device__ __forceinline__ Vec3 rot_to_lab(double4 q, Vec3 b)
{
    const double s = q.x, ux = q.y, uy = q.z, uz = q.w;
    const double tx = 2.0 * (uy * b.z - uz * b.y);
    const double ty = 2.0 * (uz * b.x - ux * b.z);
    const double tz = 2.0 * (ux * b.y - uy * b.x);
    return v3((b.x + s * tx) + (uy * tz - uz * ty), (b.y + s * ty) + (uz * tx - ux * tz),
              (b.z + s * tz) + (ux * ty - uy * tx));
}

// lab -> body (the conjugate rotation): v - s t + u x t with t = 2 u x v
__device__ __forceinline__ Vec3 rot_to_body(double4 q, Vec3 v)
{
    const double s = q.x, ux = q.y, uy = q.z, uz = q.w;
    const double tx = 2.0 * (uy * v.z - uz * v.y);
    const double ty = 2.0 * (uz * v.x - ux * v.z);
    const double tz = 2.0 * (ux * v.y - uy * v.x);
    return v3((v.x - s * tx) + (uy * tz - uz * ty), (v.y - s * ty) + (uz * tx - ux * tz),
              (v.z - s * tz) + (ux * ty - uy * tx));
}

// Is dist(p, E) < r for the spheroid E with semi-axes (a, a, c) (body frame)?
// Inside E => yes; inside the spheroid (a + r, a + r, c + r), which lies inside
// E + ball(r), => yes; outside the slab |z| < c + r or the cylinder
// rho < a + r, which contain E + ball(r), => no.  Otherwise the meridian-plane
// foot point (a^2 rho/(t + a^2), c^2 z/(t + c^2)), t the root of the convex
// decreasing F(t) = (a rho/(t + a^2))^2 + (c z/(t + c^2))^2 - 1, reached by
// Newton's method from t = 0, which climbs monotonically and stops when a step
// no longer increases t.
__device__ __noinline__ bool spheroid_point_within(double a, double c, double r, Vec3 p)
{
    const double A2 = a * a, C2 = c * c;
    const double rho2 = p.x * p.x + p.y * p.y;
    const double z = fabs(p.z);
    const double z2 = z * z;
    if (rho2 / A2 + z2 / C2 <= 1.0) return true;
    const double ar = a + r, cr = c + r;
    if (rho2 / (ar * ar) + z2 / (cr * cr) < 1.0) return true;
    if (z >= cr) return false;
    if (rho2 >= ar * ar) return false;
    const double rho = sqrt(rho2);
    double t = 0.0;
    for (int it = 0; it < 64; ++it) {
        const double d1 = t + A2, d2 = t + C2;
        const double g1 = (a * rho) / d1, g2 = (c * z) / d2;
        const double g11 = g1 * g1, g22 = g2 * g2;
        const double F = (g11 + g22) - 1.0;
        const double D = g11 / d1 + g22 / d2;
        const double tn = t + F / (2.0 * D);
        if (!(tn > t)) break;
        t = tn;
    }
    const double x0 = (A2 * rho) / (t + A2), x1 = (C2 * z) / (t + C2);
    const double e0 = rho - x0, e1 = z - x1;
    return e0 * e0 + e1 * e1 < r * r;
}

// Depletant at v (lab frame, relative to the reference point) against an
// anisotropic colloid of orientation q.
__device__ __forceinline__ bool dep_aniso(const Rep &R, Vec3 v, double4 q)
{
    const double r2v = (v.x * v.x + v.y * v.y) + v.z * v.z;
    const double Rr = R.R_circ + R.r_dep;
    if (!(r2v < Rr * Rr)) return false;          // the body lies within R_circ
    const Vec3 p = rot_to_body(q, v);
    if (R.shape == kHemisphere) {
        const double Rh = R.sh_R;
        if (p.z >= 0.0) return true;             // dome side: |p| < R + r already
        const double rho2 = p.x * p.x + p.y * p.y;
        if (rho2 <= Rh * Rh) return -p.z < R.r_dep;  // under the flat face
        const double dr = sqrt(rho2) - Rh;           // under and outside the rim
        return dr * dr + p.z * p.z < R.r_dep * R.r_dep;
    }
    return spheroid_point_within(R.sh_a, R.sh_c, R.r_dep, p);
}

// Support point of the body (body frame) in direction n.  Hemisphere: dome
// point R n/|n| for n_z >= 0, else the rim point R (n_x, n_y, 0)/rho_n (the
// face centre if rho_n = 0).  Spheroid: (a^2 n_x, a^2 n_y, c^2 n_z)/h with
// h = sqrt(a^2 (n_x^2 + n_y^2) + c^2 n_z^2).  Zero direction: reference point.
__device__ __forceinline__ Vec3 support_body(const Rep &R, Vec3 n)
{
    Vec3 s = v3(0.0, 0.0, 0.0);
    if (R.shape == kHemisphere) {
        const double Rh = R.sh_R;
        if (n.z >= 0.0) {
            const double l = sqrt((n.x * n.x + n.y * n.y) + n.z * n.z);
            if (l > 0.0) s = v3((Rh * n.x) / l, (Rh * n.y) / l, (Rh * n.z) / l);
        } else {
            const double rho = sqrt(n.x * n.x + n.y * n.y);
            if (rho > 0.0) s = v3((Rh * n.x) / rho, (Rh * n.y) / rho, 0.0);
        }
    } else {
        const double A2 = R.sh_a * R.sh_a, C2 = R.sh_c * R.sh_c;
        const double h = sqrt(A2 * (n.x * n.x + n.y * n.y) + C2 * (n.z * n.z));
        if (h > 0.0) s = v3((A2 * n.x) / h, (A2 * n.y) / h, (C2 * n.z) / h);
    }
    return s;
}

__device__ __forceinline__ Vec3 support_lab(const Rep &R, double4 q, Vec3 x, Vec3 n)
{
    const Vec3 sl = rot_to_lab(q, support_body(R, rot_to_body(q, n)));
    return v3(sl.x + x.x, sl.y + x.y, sl.z + x.z);
}

// Interior point: the hemisphere's inscribed-ball centre (0, 0, R/2), the
// spheroid's centre.
__device__ __forceinline__ Vec3 interior_lab(const Rep &R, double4 q, Vec3 x)
{
    Vec3 b = v3(0.0, 0.0, 0.0);
    if (R.shape == kHemisphere) b.z = 0.5 * R.sh_R;
    const Vec3 l = rot_to_lab(q, b);
    return v3(l.x + x.x, l.y + x.y, l.z + x.z);
}

// Support of M = B - A: S_B(n) - S_A(-n).  A sits at the origin.
__device__ __forceinline__ Vec3 support_diff(const Rep &R, double4 qa, double4 qb, Vec3 xb, Vec3 n)
{
    const Vec3 zero = v3(0.0, 0.0, 0.0);
    const Vec3 sb = support_lab(R, qb, xb, n);
    const Vec3 sa = support_lab(R, qa, zero, v3(-n.x, -n.y, -n.z));
    return sub3(sb, sa);
}

// Overlap of colloid A (reference point at the origin, orientation qa) and
// colloid B (at xb, orientation qb): Minkowski portal refinement (Snethen,
// "XenoCollide", Game Programming Gems 7, 2008) on M = B - A from the
// interior point v0 = c_B - c_A.  At most 64 portal-discovery and 64
// refinement steps; "no overlap" when a support plane separates the origin
// from M or the portal lies within 1e-12 of the boundary of M.
__device__ __noinline__ bool mpr_overlap(const Rep &R, double4 qa, double4 qb, Vec3 xb)
{
    const Vec3 cA = interior_lab(R, qa, v3(0.0, 0.0, 0.0));
    const Vec3 cB = interior_lab(R, qb, xb);
    const Vec3 v0 = sub3(cB, cA);
    if (is_zero3(v0)) return true;
    Vec3 n = v3(-v0.x, -v0.y, -v0.z);
    Vec3 v1 = support_diff(R, qa, qb, xb, n);
    if (dot3(v1, n) <= 0.0) return false;
    n = cross3(v1, v0);
    if (is_zero3(n)) return true;
    Vec3 v2 = support_diff(R, qa, qb, xb, n);
    if (dot3(v2, n) <= 0.0) return false;
    n = cross3(sub3(v1, v0), sub3(v2, v0));
    if (dot3(n, v0) > 0.0) {
        const Vec3 t = v1;
        v1 = v2;
        v2 = t;
        n = v3(-n.x, -n.y, -n.z);
    }
    Vec3 v3p;
    bool found = false;
    for (int it = 0; it < 64 && !found; ++it) {
        v3p = support_diff(R, qa, qb, xb, n);
        if (dot3(v3p, n) <= 0.0) return false;
        if (dot3(cross3(v1, v3p), v0) < 0.0) {
            v2 = v3p;
            n = cross3(sub3(v1, v0), sub3(v3p, v0));
            continue;
        }
        if (dot3(cross3(v3p, v2), v0) < 0.0) {
            v1 = v3p;
            n = cross3(sub3(v3p, v0), sub3(v2, v0));
            continue;
        }
        found = true;
    }
    if (!found) return false;
    for (int it = 0; it < 64; ++it) {
        n = cross3(sub3(v2, v1), sub3(v3p, v1));
        if (is_zero3(n)) return true;
        const double nn = sqrt(dot3(n, n));
        n = v3(n.x / nn, n.y / nn, n.z / nn);
        if (dot3(n, v1) >= 0.0) return true;
        const Vec3 v4 = support_diff(R, qa, qb, xb, n);
        if (dot3(v4, n) <= 0.0) return false;
        if (dot3(sub3(v4, v3p), n) <= 1e-12) return false;
        if (dot3(cross3(v4, v1), v0) < 0.0) {
            if (dot3(cross3(v4, v2), v0) < 0.0) v1 = v4;
            else v3p = v4;
        } else {
            if (dot3(cross3(v4, v3p), v0) < 0.0) v2 = v4;
            else v1 = v4;
        }
    }
    return false;
}

// Colloid-colloid overlap for reference points separated by d (A to B).
// Beyond twice the circumsphere radius two colloids cannot overlap.
__device__ __forceinline__ bool pair_aniso(const Rep &R, Vec3 d, double4 qa, double4 qb)
{
    const double r2 = (d.x * d.x + d.y * d.y) + d.z * d.z;
    const double D = 2.0 * R.R_circ;
    if (!(r2 < D * D)) return false;
    return mpr_overlap(R, qa, qb, d);
}

// Rotation proposal: v uniform in the unit ball from the purpose-2 attempt
// stream (at most 64 attempts), q' = (q_r q)/|q_r q| with q_r = (1, alpha v).
// Returns false if the attempt stream hit its cap.
__device__ __noinline__ bool propose_rotation(const Rep &R, uint32_t sweep, uint32_t tag,
                                              double4 qo, double4 *qn)
{
    double vx = 0.0, vy = 0.0, vz = 0.0;
    bool ok = false;
    for (uint32_t t = 0; t < 64u && !ok; ++t) {
        const uint4 w = draw(R.key0, R.key1, sweep, tag, kPRot, 0, t);
        vx = s11(w.x);
        vy = s11(w.y);
        vz = s11(w.z);
        ok = (vx * vx + vy * vy) + vz * vz < 1.0;
    }
    if (!ok) return false;
    const double s1 = 1.0, x1 = R.alpha * vx, y1 = R.alpha * vy, z1 = R.alpha * vz;
    const double s2 = qo.x, x2 = qo.y, y2 = qo.z, z2 = qo.w;
    const double ms = s1 * s2 - ((x1 * x2 + y1 * y2) + z1 * z2);
    const double mx = (s1 * x2 + s2 * x1) + (y1 * z2 - z1 * y2);
    const double my = (s1 * y2 + s2 * y1) + (z1 * x2 - x1 * z2);
    const double mz = (s1 * z2 + s2 * z1) + (x1 * y2 - y1 * x2);
    const double nrm = sqrt(((ms * ms + mx * mx) + my * my) + mz * mz);
    *qn = make_double4(ms / nrm, mx / nrm, my / nrm, mz / nrm);
    return true;
}

}  // namespace hpmc
