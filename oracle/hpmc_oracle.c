/*
 * Oracle for implicit-depletant hard-particle Monte Carlo
 * (Glaser, Karas & Glotzer, "A parallel algorithm for implicit depletant
 * simulations", arXiv:1508.07077).
 *
 * TEST INFRASTRUCTURE.  This file is the plain, serial, FP64 statement of what
 * the GPU library computes.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load it.  It shares no code,
 * header, table or constant generator with the CUDA library: the two sides
 * implement the same written specification independently.
 *
 * What it computes, step by step, in the paper's order:
 *   - Sec. III.E: checkerboard sweep.  Cells of width >= d_colloid + d_depletant,
 *     2x2x2 colouring, random colour order and random grid shift per sweep,
 *     particles may not leave their cell.
 *   - Sec. III.B, Eqs. (3)-(4): propose a colloid move; reject on colloid overlap
 *     (U_ij = infinity); draw N_p ~ Poisson(z_p V_0) depletants uniformly in V_0.
 *   - Sec. III.C (choice of V_0): V_0 is the circumsphere of diameter
 *     d_colloid + d_depletant around the moved colloid in its NEW pose.
 *     Depletants overlapping the old configuration (old pose of the moved
 *     colloid or any other colloid) are ignored; a depletant overlapping only
 *     the new pose blocks the move.
 *   - Sec. III.D, Eq. (12): with n_trial > 0 each blocking depletant is
 *     reinserted (configurational bias) and the move is accepted with the
 *     product of per-depletant weights.
 *
 * Threads (oracle_run_threads, n_threads > 1; OpenMP, -fopenmp): Sec. III.E
 * makes the active cells of one colour independent (a colloid moves only
 * inside its cell and interacts only with its 26 neighbour cells, none of
 * which is active at the same time), so their trial moves may run in any
 * order.  The cells of a colour phase are then handed out to threads; each
 * thread keeps its own counters, summed at the end of the phase.  Positions
 * and counters are identical to the serial run for every thread count.
 *
 * Readings where the paper is silent (RNG, op order, sampling details) are the
 * ones listed in the design notes; every floating-point expression below is
 * written in the exact operation order that specification fixes, and must be
 * compiled with -ffp-contract=off (no fused multiply-add).
 *
 *   - Sec. III.C, closing remark (option v0_mode 1): for sphere translations
 *     V_0 may be restricted to the shell of the moved colloid's excluded
 *     volume that can hold points overlapping only the new pose; the shell
 *     thickness is quantised into 32 levels chosen from the move's words.
 *     Option v0_mode 2: V_0 is the axis-aligned cube around the circumsphere
 *     (every attempt is a depletant; no rejection).
 *   - Sec. IV.B (coexistence): Gibbs-ensemble colloid exchange between two
 *     boxes with depletants inserted at the new position and reinserted in
 *     the old box (configurational bias), spheres.
 *   - Sec. VI (the remark that the scheme generalises to soft interactions,
 *     option soft_eps > 0): a Hertz colloid-depletant potential; a depletant
 *     blocks with probability e^(-U_others) max(0, e^(-u_old) - e^(-u_new)).
 *   - Sec. V: anisotropic colloids (hemispheres, discoids = oblate spheroids)
 *     with quaternion rotation moves; overlap of two convex colloids by
 *     Minkowski portal refinement on their support functions.
 *
 * Parity pins (tests/test_oracle_*.py): Poisson moments and pmf (chi^2),
 * Philox uniformity, brute-force neighbour enumeration, the two-colloid
 * Asakura-Oosawa distribution (detailed balance, Eqs. 5-11 and 12), the
 * hard-sphere Carnahan-Starling contact value at z_p = 0, and the exact
 * free-volume fraction of a single colloid; for the anisotropic shapes,
 * point and pair tests against a general constrained minimiser and against
 * touching distances on symmetry axes, the Steiner excluded volume, the
 * rotation-proposal distribution and detailed balance of rotation moves; for
 * the shell V_0, lens containment by brute force, the uniformity of the shell
 * points, the Poisson mean of the shell volume, equality of the acceptance
 * probability with the circumsphere's, detailed balance and the
 * Asakura-Oosawa distribution; for the Gibbs exchange, detailed balance of
 * one exchange against the closed form (Gibbs prior times exp(z_p dV_f)),
 * the binomial box occupancy of an ideal gas, conservation and validity;
 * for the soft interaction, the shared exponential against the library's,
 * detailed balance against a quadrature of the semigrand weight ratio and
 * the two-colloid distribution against a quadrature of the effective
 * attraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Counter-based RNG: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).    */
/* The paper does not name its RNG; this is the chosen reading.              */
/* ------------------------------------------------------------------------ */

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Purposes, placed in the top byte of counter word 2. */
enum { P_SCHED = 0, P_MOVE = 1, P_ROT = 2, P_POISSON = 3, P_DEP = 4,
       P_CB_FWD = 5, P_CB_REV = 6, P_ACCEPT = 7, P_PROBE = 8 };

typedef struct { uint32_t k[2]; } okey;

static void draw(okey key, uint32_t sweep, uint32_t stream, uint32_t purpose,
                 uint32_t sub, uint32_t t, uint32_t w[4])
{
    uint32_t ctr[4] = {sweep, stream, (purpose << 24) | (sub & 0xFFFFFFu), t};
    oracle_philox4x32_10(ctr, key.k, w);
}

/* uniform in (0,1): (w + 1/2) 2^-32 */
static double u01(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }
/* uniform in (-1,1): 2 u01(w) - 1, exact in double */
static double s11(uint32_t w) { return ((double)w + 0.5) * (1.0 / 2147483648.0) - 1.0; }
/* uniform in [0,1) with 53 bits */
static double u53(uint32_t w0, uint32_t w1)
{
    return ((double)(w0 >> 5) * 67108864.0 + (double)(w1 >> 6)) *
           (1.0 / 9007199254740992.0);
}

/* uniform in (-1,1) from a 21-bit integer: (a + 1/2) 2^-20 - 1 (exact) */
static double s21(uint32_t a) { return ((double)a + 0.5) * (1.0 / 1048576.0) - 1.0; }

/* Paired points of a depletant stream (hard interactions, circumsphere or
 * cube V_0): one Philox call gives the coordinates of two attempts.  The
 * attempts come in blocks of 64: attempt t is half h = floor(t / 32) mod 2 of
 * call 32 floor(t / 64) + (t mod 32), so attempts 64b .. 64b + 31 are the
 * first halves of calls 32b .. 32b + 31 and the next 32 attempts their second
 * halves.  Half 0 is the top 21 bits of words 0, 1, 2; half 1 is, for
 * coordinate d, the low 11 bits of word d below bits 10d .. 10d + 9 of word 3
 * (126 bits, each used once).  Coordinate d of the point is R_s s21(a_d). */
static void paired_fields(const uint32_t w[4], uint32_t h, uint32_t a[3])
{
    for (int d = 0; d < 3; ++d) {
        if (h == 0) a[d] = w[d] >> 11;
        else a[d] = (w[d] & 0x7FFu) | (((w[3] >> (10 * d)) & 0x3FFu) << 11);
    }
}

static void paired_point(okey key, double R_s, uint32_t sweep, uint32_t tag, uint32_t t,
                         double e[3])
{
    uint32_t w[4], a[3];
    draw(key, sweep, tag, P_DEP, 0, 32u * (t >> 6) + (t & 31u), w);
    paired_fields(w, (t >> 5) & 1u, a);
    e[0] = R_s * s21(a[0]);
    e[1] = R_s * s21(a[1]);
    e[2] = R_s * s21(a[2]);
}

double oracle_u01(uint32_t w) { return u01(w); }
double oracle_s11(uint32_t w) { return s11(w); }
double oracle_s21(uint32_t a) { return s21(a); }

/* The paired points of attempts t = 0 .. n_att - 1 of stream (sweep, tag)
 * under key (seed), radius R_s: all of them into e (3 per attempt), for the
 * tests of the stream. */
void oracle_paired_points(double R_s, uint64_t seed, uint32_t sweep, uint32_t tag,
                          uint32_t n_att, double *e)
{
    okey key;
    key.k[0] = (uint32_t)seed;
    key.k[1] = (uint32_t)(seed >> 32);
    for (uint32_t t = 0; t < n_att; ++t) paired_point(key, R_s, sweep, tag, t, e + 3 * (size_t)t);
}
double oracle_u53(uint32_t w0, uint32_t w1) { return u53(w0, w1); }

/* ------------------------------------------------------------------------ */
/* Poisson(lambda) by inversion, Sec. III.B step 2 ("N_p ~ Poisson(z_p V)")  */
/* ------------------------------------------------------------------------ */

#define ORACLE_PI 3.141592653589793

/* lambda = z_p |V_0|, V_0 the sphere of radius R_s (Sec. III.C). */
double oracle_lambda(double R_s, double n_r)
{
    double v0 = ((4.0 / 3.0) * ORACLE_PI) * ((R_s * R_s) * R_s);
    return n_r * v0;
}

/* Cumulative table F[k] = sum_{m<=k} e^-lambda lambda^m / m!, built by the
 * recurrence p_0 = exp(-lambda), p_k = p_{k-1} * lambda / k.  Stops after the
 * first k > lambda with p_k < 2^-64.  Returns the length or -1 if cap is hit. */
int oracle_poisson_table(double lambda, double *F, int cap)
{
    if (!(lambda >= 0.0) || lambda > 700.0) return -1;
    double p = exp(-lambda);
    double cdf = p;
    int n = 0;
    if (cap < 1) return -1;
    F[n++] = cdf;
    for (int k = 1;; ++k) {
        p = (p * lambda) / (double)k;
        cdf = cdf + p;
        if (n >= cap) return -1;
        F[n++] = cdf;
        if ((double)k > lambda && p < 5.421010862427522e-20 /* 2^-64 */) break;
    }
    return n;
}

/* N_p = number of table entries F[k] <= u (inversion: min{k : u < F[k]}). */
static int poisson_invert(const double *F, int n, double u)
{
    int k = 0;
    while (k < n && F[k] <= u) ++k;
    return k;
}

int oracle_poisson_sample(const double *F, int n, double u)
{
    return poisson_invert(F, n, u);
}

/* ------------------------------------------------------------------------ */
/* Shapes (Secs. IV-V): the colloid is a sphere of diameter d, a hemisphere  */
/* of diameter d (Sec. V.A) or an oblate spheroid with semi-axes a = b, c    */
/* (the discoid of Sec. V.B).  Depletants are penetrable spheres of diameter */
/* q that interact with colloids only (Sec. II).                             */
/* ------------------------------------------------------------------------ */

enum { SHAPE_SPHERE = 0, SHAPE_HEMISPHERE = 1, SHAPE_SPHEROID = 2 };

typedef struct {
    int kind;
    double d;       /* sphere / hemisphere diameter */
    double a, c;    /* spheroid semi-axes (body x = y, body z) */
    double R_circ;  /* circumsphere radius about the reference point */
} oshape;

/* Reference point and body frame.  Sphere and spheroid: the centre.  Hemisphere:
 * the centre of the flat face, the face in the body plane z = 0 and the dome
 * on the side z >= 0.  An orientation is a unit quaternion (s, x, y, z); it
 * maps body-frame vectors to the lab frame. */

/* body -> lab: b + s t + u x t with t = 2 u x b, u = (x, y, z). */
static void rot_to_lab(const double q[4], const double b[3], double v[3])
{
    double s = q[0], ux = q[1], uy = q[2], uz = q[3];
    double tx = 2.0 * (uy * b[2] - uz * b[1]);
    double ty = 2.0 * (uz * b[0] - ux * b[2]);
    double tz = 2.0 * (ux * b[1] - uy * b[0]);
    v[0] = (b[0] + s * tx) + (uy * tz - uz * ty);
    v[1] = (b[1] + s * ty) + (uz * tx - ux * tz);
    v[2] = (b[2] + s * tz) + (ux * ty - uy * tx);
}

/* lab -> body (rotation by the conjugate): v - s t + u x t, t = 2 u x v. */
static void rot_to_body(const double q[4], const double v[3], double b[3])
{
    double s = q[0], ux = q[1], uy = q[2], uz = q[3];
    double tx = 2.0 * (uy * v[2] - uz * v[1]);
    double ty = 2.0 * (uz * v[0] - ux * v[2]);
    double tz = 2.0 * (ux * v[1] - uy * v[0]);
    b[0] = (v[0] - s * tx) + (uy * tz - uz * ty);
    b[1] = (v[1] - s * ty) + (uz * tx - ux * tz);
    b[2] = (v[2] - s * tz) + (ux * ty - uy * tx);
}

static const double QUAT_ID[4] = {1.0, 0.0, 0.0, 0.0};

/* Distance test of a point against the spheroid x^2/a^2 + y^2/a^2 + z^2/c^2
 * <= 1 (body frame): is dist(p, E) < r?  The closest boundary point of E to
 * an outside point P = (rho, z) of the meridian plane is
 * (a^2 rho / (t + a^2), c^2 z / (t + c^2)) where t > 0 is the root of
 * F(t) = (a rho / (t + a^2))^2 + (c z / (t + c^2))^2 - 1, a convex decreasing
 * function for t > -min(a^2, c^2); Newton's method from t = 0 (F(0) > 0)
 * climbs monotonically to the root and stops when a step no longer increases
 * t.  Before that: inside E => overlap; inside the spheroid with semi-axes
 * (a + r, c + r), which lies inside E + ball(r), => overlap; outside the
 * slab |z| < c + r or the cylinder rho < a + r, which contain E + ball(r),
 * => no overlap. */
static int spheroid_point_within(double a, double c, double r, const double p[3])
{
    double A2 = a * a, C2 = c * c;
    double rho2 = p[0] * p[0] + p[1] * p[1];
    double z = fabs(p[2]);
    double z2 = z * z;
    if (rho2 / A2 + z2 / C2 <= 1.0) return 1;
    double ar = a + r, cr = c + r;
    if (rho2 / (ar * ar) + z2 / (cr * cr) < 1.0) return 1;
    if (z >= cr) return 0;
    if (rho2 >= ar * ar) return 0;
    double rho = sqrt(rho2);
    double t = 0.0;
    for (int it = 0; it < 64; ++it) {
        double d1 = t + A2, d2 = t + C2;
        double g1 = (a * rho) / d1, g2 = (c * z) / d2;
        double g11 = g1 * g1, g22 = g2 * g2;
        double F = (g11 + g22) - 1.0;
        double D = g11 / d1 + g22 / d2;
        double tn = t + F / (2.0 * D);
        if (!(tn > t)) break;
        t = tn;
    }
    double x0 = (A2 * rho) / (t + A2), x1 = (C2 * z) / (t + C2);
    double e0 = rho - x0, e1 = z - x1;
    return e0 * e0 + e1 * e1 < r * r;
}

/* Does a depletant (penetrable sphere of diameter q) at v, given relative to
 * the colloid's reference point in the lab frame, overlap the colloid of
 * orientation quat (NULL = identity)?  Strict: touching is not an overlap.
 * The depletant overlaps iff its centre is closer than r = q/2 to the body. */
static int dep_overlap(const oshape *sh, double q, const double v[3],
                       const double *quat)
{
    double r2v = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
    if (sh->kind == SHAPE_SPHERE) {
        double R = 0.5 * sh->d + 0.5 * q;
        return r2v < R * R;
    }
    double r = 0.5 * q;
    double Rr = sh->R_circ + r;
    if (!(r2v < Rr * Rr)) return 0;        /* the body lies within R_circ */
    double p[3];
    rot_to_body(quat ? quat : QUAT_ID, v, p);
    if (sh->kind == SHAPE_HEMISPHERE) {
        double R = 0.5 * sh->d;
        /* z >= 0: distance max(0, |p| - R), and |p| < R + r holds */
        if (p[2] >= 0.0) return 1;
        double rho2 = p[0] * p[0] + p[1] * p[1];
        /* below the flat face: distance -z */
        if (rho2 <= R * R) return -p[2] < r;
        /* below and outside the rim: distance to the rim circle */
        double dr = sqrt(rho2) - R;
        return dr * dr + p[2] * p[2] < r * r;
    }
    return spheroid_point_within(sh->a, sh->c, r, p);
}

/* Support point of the body (body frame) in direction n: the point of the
 * body maximising n . x.  Hemisphere: on the dome R n/|n| when n_z >= 0,
 * else on the rim R (n_x, n_y, 0)/rho_n (the face centre when rho_n = 0).
 * Spheroid: (a^2 n_x, a^2 n_y, c^2 n_z) / sqrt(a^2 (n_x^2 + n_y^2) + c^2 n_z^2).
 * A zero direction gives the reference point. */
static void support_body(const oshape *sh, const double n[3], double s[3])
{
    s[0] = 0.0; s[1] = 0.0; s[2] = 0.0;
    if (sh->kind == SHAPE_HEMISPHERE) {
        double R = 0.5 * sh->d;
        if (n[2] >= 0.0) {
            double l = sqrt((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
            if (l > 0.0) {
                s[0] = (R * n[0]) / l;
                s[1] = (R * n[1]) / l;
                s[2] = (R * n[2]) / l;
            }
        } else {
            double rho = sqrt(n[0] * n[0] + n[1] * n[1]);
            if (rho > 0.0) {
                s[0] = (R * n[0]) / rho;
                s[1] = (R * n[1]) / rho;
            }
        }
    } else {
        double A2 = sh->a * sh->a, C2 = sh->c * sh->c;
        double h = sqrt(A2 * (n[0] * n[0] + n[1] * n[1]) + C2 * (n[2] * n[2]));
        if (h > 0.0) {
            s[0] = (A2 * n[0]) / h;
            s[1] = (A2 * n[1]) / h;
            s[2] = (C2 * n[2]) / h;
        }
    }
}

/* One colloid placed in the lab frame: reference point at x, orientation q. */
typedef struct {
    const oshape *sh;
    const double *q;
    double x[3];
} obody;

static void support_lab(const obody *B, const double n[3], double out[3])
{
    double nb[3], sb[3], sl[3];
    rot_to_body(B->q, n, nb);
    support_body(B->sh, nb, sb);
    rot_to_lab(B->q, sb, sl);
    out[0] = sl[0] + B->x[0];
    out[1] = sl[1] + B->x[1];
    out[2] = sl[2] + B->x[2];
}

/* A point strictly inside the body: the centre of the hemisphere's inscribed
 * ball (0, 0, R/2) in body coordinates; the spheroid's centre. */
static void interior_lab(const obody *B, double out[3])
{
    double b[3] = {0.0, 0.0, 0.0}, l[3];
    if (B->sh->kind == SHAPE_HEMISPHERE) b[2] = 0.25 * B->sh->d;
    rot_to_lab(B->q, b, l);
    out[0] = l[0] + B->x[0];
    out[1] = l[1] + B->x[1];
    out[2] = l[2] + B->x[2];
}

static double dot3(const double a[3], const double b[3])
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void sub3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}

static void copy3(double o[3], const double a[3]) { o[0] = a[0]; o[1] = a[1]; o[2] = a[2]; }

/* Support point of the Minkowski difference M = B - A = {b - a}. */
static void support_diff(const obody *A, const obody *B, const double n[3], double out[3])
{
    double m[3] = {-n[0], -n[1], -n[2]}, sa[3], sb[3];
    support_lab(B, n, sb);
    support_lab(A, m, sa);
    sub3(sb, sa, out);
}

/* Do two convex colloids overlap?  A and B overlap iff the origin lies in
 * M = B - A.  Minkowski portal refinement (Snethen, "XenoCollide", Game
 * Programming Gems 7, 2008): from an interior point v0 of M, find a triangle
 * of support points (the portal) that the ray from v0 through the origin
 * crosses, then push the portal out along its normal until the origin is
 * inside the tetrahedron (v0, portal) (overlap), a support plane separates
 * the origin from M (no overlap), or the portal lies within 1e-12 of the
 * boundary of M (no overlap: touching or closer than the tolerance). */
static int mpr_overlap(const obody *A, const obody *B)
{
    double cA[3], cB[3], v0[3], v1[3], v2[3], v3[3], v4[3], n[3], e1[3], e2[3], t[3];
    interior_lab(A, cA);
    interior_lab(B, cB);
    sub3(cB, cA, v0);
    if (v0[0] == 0.0 && v0[1] == 0.0 && v0[2] == 0.0) return 1;
    n[0] = -v0[0]; n[1] = -v0[1]; n[2] = -v0[2];
    support_diff(A, B, n, v1);
    if (dot3(v1, n) <= 0.0) return 0;
    cross3(v1, v0, n);
    if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0) return 1;
    support_diff(A, B, n, v2);
    if (dot3(v2, n) <= 0.0) return 0;
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, n);
    if (dot3(n, v0) > 0.0) {
        copy3(t, v1); copy3(v1, v2); copy3(v2, t);
        n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2];
    }
    /* portal discovery */
    int found = 0;
    for (int it = 0; it < 64 && !found; ++it) {
        support_diff(A, B, n, v3);
        if (dot3(v3, n) <= 0.0) return 0;
        cross3(v1, v3, t);
        if (dot3(t, v0) < 0.0) {
            copy3(v2, v3);
            sub3(v1, v0, e1);
            sub3(v3, v0, e2);
            cross3(e1, e2, n);
            continue;
        }
        cross3(v3, v2, t);
        if (dot3(t, v0) < 0.0) {
            copy3(v1, v3);
            sub3(v3, v0, e1);
            sub3(v2, v0, e2);
            cross3(e1, e2, n);
            continue;
        }
        found = 1;
    }
    if (!found) return 0;
    /* portal refinement */
    for (int it = 0; it < 64; ++it) {
        sub3(v2, v1, e1);
        sub3(v3, v1, e2);
        cross3(e1, e2, n);
        if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0) return 1;
        double nn = sqrt(dot3(n, n));
        n[0] = n[0] / nn; n[1] = n[1] / nn; n[2] = n[2] / nn;
        if (dot3(n, v1) >= 0.0) return 1;
        support_diff(A, B, n, v4);
        if (dot3(v4, n) <= 0.0) return 0;
        sub3(v4, v3, t);
        if (dot3(t, n) <= 1e-12) return 0;
        cross3(v4, v1, t);
        if (dot3(t, v0) < 0.0) {
            cross3(v4, v2, t);
            if (dot3(t, v0) < 0.0) copy3(v1, v4);
            else copy3(v3, v4);
        } else {
            cross3(v4, v3, t);
            if (dot3(t, v0) < 0.0) copy3(v2, v4);
            else copy3(v1, v4);
        }
    }
    return 0;
}

/* Do two colloids whose reference points are separated by r (from the first
 * to the second) overlap?  U_ij = infinity for overlapping hard colloids.
 * Beyond twice the circumsphere radius they cannot (the strict convention
 * makes touching circumspheres non-overlapping). */
static int pair_overlap(const oshape *sh, const double r[3], const double *qa,
                        const double *qb)
{
    double r2 = (r[0] * r[0] + r[1] * r[1]) + r[2] * r[2];
    if (sh->kind == SHAPE_SPHERE) return r2 < sh->d * sh->d;
    double D = 2.0 * sh->R_circ;
    if (!(r2 < D * D)) return 0;
    obody A = {sh, qa ? qa : QUAT_ID, {0.0, 0.0, 0.0}};
    obody B = {sh, qb ? qb : QUAT_ID, {r[0], r[1], r[2]}};
    return mpr_overlap(&A, &B);
}

/* Shape parameters: sphere {d}, hemisphere {d}, spheroid {a, c}. */
static int shape_init(oshape *sh, int kind, const double *params, int nparams)
{
    memset(sh, 0, sizeof *sh);
    sh->kind = kind;
    if (!params) return -1;
    if (kind == SHAPE_SPHERE || kind == SHAPE_HEMISPHERE) {
        if (nparams < 1 || !(params[0] > 0.0)) return -1;
        sh->d = params[0];
        sh->R_circ = 0.5 * params[0];
        return 0;
    }
    if (kind == SHAPE_SPHEROID) {
        if (nparams < 2 || !(params[0] > 0.0) || !(params[1] > 0.0)) return -1;
        sh->a = params[0];
        sh->c = params[1];
        sh->R_circ = params[0] > params[1] ? params[0] : params[1];
        return 0;
    }
    return -1;
}

/* Exported single tests (used by the pins of the shape primitives). */
int oracle_dep_overlap(int kind, const double *params, int nparams, double q,
                       const double *v, const double *quat)
{
    oshape sh;
    if (shape_init(&sh, kind, params, nparams) != 0 || !v) return -1;
    return dep_overlap(&sh, q, v, quat);
}

int oracle_pair_overlap(int kind, const double *params, int nparams,
                        const double *r, const double *qa, const double *qb)
{
    oshape sh;
    if (shape_init(&sh, kind, params, nparams) != 0 || !r) return -1;
    return pair_overlap(&sh, r, qa, qb);
}

/* ------------------------------------------------------------------------ */
/* Checkerboard geometry, Sec. III.E                                         */
/* ------------------------------------------------------------------------ */

static int cell_coord(double x, double sigma, double L, double w, int nc)
{
    double s = x - sigma;
    if (s < 0.0) s = s + L;
    int c = (int)(s / w);
    if (c >= nc) c = nc - 1;
    if (c < 0) c = 0;
    return c;
}

static double min_image(double d, double L)
{
    double h = 0.5 * L;
    if (d > h) d = d - L;
    else if (d < -h) d = d + L;
    return d;
}

/* Grid shift sigma in [0,w)^3 and colour order perm[8] for one sweep. */
void oracle_schedule(uint64_t seed, uint32_t replica, uint32_t sweep, double w,
                     double sigma[3], int perm[8])
{
    okey key = {{(uint32_t)seed, (uint32_t)(seed >> 32) ^ replica}};
    uint32_t a[4], b[4], c[4];
    draw(key, sweep, 0xFFFFFFFFu, P_SCHED, 0, 0, a);
    sigma[0] = w * u01(a[0]);
    sigma[1] = w * u01(a[1]);
    sigma[2] = w * u01(a[2]);
    draw(key, sweep, 0xFFFFFFFFu, P_SCHED, 1, 0, b);
    draw(key, sweep, 0xFFFFFFFFu, P_SCHED, 2, 0, c);
    uint32_t words[8] = {b[0], b[1], b[2], b[3], c[0], c[1], c[2], c[3]};
    for (int i = 0; i < 8; ++i) perm[i] = i;
    for (int i = 7; i >= 1; --i) {
        int j = (int)(((uint64_t)words[7 - i] * (uint64_t)(i + 1)) >> 32);
        int t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* Cell list for one sweep: cell_start[nc^3 + 1], cell_idx[n], particles of a
 * cell in ascending tag order. */
int oracle_cell_list(int n, double L, int nc, const double *pos, uint64_t seed,
                     uint32_t replica, uint32_t sweep, int *cell_start,
                     int *cell_idx)
{
    if (n < 0 || nc < 2 || (nc & 1)) return -1;
    double w = L / (double)nc;
    double sigma[3];
    int perm[8];
    oracle_schedule(seed, replica, sweep, w, sigma, perm);
    int ncell = nc * nc * nc;
    int *cnt = (int *)calloc((size_t)ncell, sizeof(int));
    int *cell_of = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!cnt || !cell_of) { free(cnt); free(cell_of); return -1; }
    for (int i = 0; i < n; ++i) {
        int cx = cell_coord(pos[3 * i + 0], sigma[0], L, w, nc);
        int cy = cell_coord(pos[3 * i + 1], sigma[1], L, w, nc);
        int cz = cell_coord(pos[3 * i + 2], sigma[2], L, w, nc);
        cell_of[i] = cx + nc * (cy + nc * cz);
        cnt[cell_of[i]]++;
    }
    cell_start[0] = 0;
    for (int c = 0; c < ncell; ++c) cell_start[c + 1] = cell_start[c] + cnt[c];
    memset(cnt, 0, sizeof(int) * (size_t)ncell);
    for (int i = 0; i < n; ++i) {
        int c = cell_of[i];
        cell_idx[cell_start[c] + cnt[c]++] = i;
    }
    free(cnt);
    free(cell_of);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The sampler                                                               */
/* ------------------------------------------------------------------------ */

enum {
    C_MOVES = 0, C_ACCEPT, C_REJ_CELL, C_REJ_OVERLAP, C_REJ_DEP, C_REJ_CB,
    C_DEP_DRAWN, C_DEP_BLOCKING, C_CB_FWD_OK, C_CB_REV_OK, C_CAP, C_TRANSLATE,
    C_DEP_EVAL, C_N = 16
};

typedef struct {
    int n;
    double L;
    oshape sh;
    double q, n_r, R_s, R_s2, lambda;
    int n_trial, cb_mode;
    double d_max, a_max, p_translate, alpha;
    okey key;
    int nc;
    double w;
    int brute_force;
    double *F;
    int nF;
    /* shell-restricted V_0 (v0_mode 1, sphere translations): per level k =
     * 1..SHELL_LEVELS the inner radius, the thickness and the Poisson table */
    int v0_mode;
    double soft_eps;   /* > 0: Hertz colloid-depletant interaction of strength soft_eps kT */
    double R_s4, dd;
    double s_rin[32], s_h[32];
    double *sF[32];
    int snF[32];
} osim;

typedef struct {
    int j;
    double d[3];     /* r_j - r_i' (minimum image) */
    const double *qj;
} onb;

/* All colloids j != i that can interact with colloid i at reference point xn:
 * every particle of the (deduplicated) 27 neighbouring cells, or every other
 * particle in brute-force mode.  Extra far-away entries are harmless: every
 * test against them is false. */
static int gather_neighbours(const osim *S, int i, const double xn[3],
                             const int ci[3], const double *pos,
                             const double *quat, const int *cell_start,
                             const int *cell_idx, onb *out)
{
    int m = 0;
    if (S->brute_force) {
        for (int j = 0; j < S->n; ++j) {
            if (j == i) continue;
            out[m].j = j;
            for (int d = 0; d < 3; ++d)
                out[m].d[d] = min_image(pos[3 * j + d] - xn[d], S->L);
            out[m].qj = quat ? quat + 4 * j : NULL;
            ++m;
        }
        return m;
    }
    int nc = S->nc;
    int off_n = nc == 2 ? 2 : 3;
    for (int oz = 0; oz < off_n; ++oz)
        for (int oy = 0; oy < off_n; ++oy)
            for (int ox = 0; ox < off_n; ++ox) {
                int cx, cy, cz;
                if (nc == 2) { cx = ox; cy = oy; cz = oz; }
                else {
                    cx = (ci[0] + ox - 1 + nc) % nc;
                    cy = (ci[1] + oy - 1 + nc) % nc;
                    cz = (ci[2] + oz - 1 + nc) % nc;
                }
                int c = cx + nc * (cy + nc * cz);
                for (int s = cell_start[c]; s < cell_start[c + 1]; ++s) {
                    int j = cell_idx[s];
                    if (j == i) continue;
                    out[m].j = j;
                    for (int d = 0; d < 3; ++d)
                        out[m].d[d] = min_image(pos[3 * j + d] - xn[d], S->L);
                    out[m].qj = quat ? quat + 4 * j : NULL;
                    ++m;
                }
            }
    return m;
}

/* Next point of an attempt stream, uniform in the ball |e| < R_s (rejection
 * from the cube [-R_s, R_s]^3).  *t is the running attempt index; returns 0
 * once *t reaches t_max. */
/* ------------------------------------------------------------------------ */
/* Soft colloid-depletant interaction (Sec. VI: the scheme generalises to    */
/* soft potentials such as the Hertz potential).  u(r) = eps (1 - r/s)^(5/2) */
/* for r < s = (d + q)/2, else 0; colloids stay hard among themselves.       */
/* Reading: a depletant at x blocks the move with probability                */
/*   b(x) = e^(-U_others(x)) max(0, e^(-u(|x - r_old|)) - e^(-u(|x - r_new|))) */
/* (U_others: the other colloids' energy, summed in ascending index), which  */
/* gives P(M->M')/P(M'->M) = exp(z_p Int[e^(-U') - e^(-U)] dx), the         */
/* semigrand weight ratio; for hard interactions b is the indicator of       */
/* "overlaps only the new configuration".                                    */
/* ------------------------------------------------------------------------ */

/* e^(-y), y >= 0: Cody-Waite reduction y = k ln2 + r (ln2 split into a
 * 29-bit head and a tail), |r| <= ln2/2, then the degree-14 Taylor
 * polynomial of e^(-r) by Horner (truncation error < 2^-60), times 2^-k. */
static double exp_neg(double y)
{
    if (!(y < 700.0)) return 0.0;
    const double ln2_hi = 0x1.62e42ff000000p-1, ln2_lo = -0x1.718432a1b0e26p-35;
    double kd = floor(y * 0x1.71547652b82fep+0 + 0.5);
    double r = (y - kd * ln2_hi) - kd * ln2_lo;
    double x = -r;
    double p = 1.0 / 87178291200.0;
    p = p * x + 1.0 / 6227020800.0;
    p = p * x + 1.0 / 479001600.0;
    p = p * x + 1.0 / 39916800.0;
    p = p * x + 1.0 / 3628800.0;
    p = p * x + 1.0 / 362880.0;
    p = p * x + 1.0 / 40320.0;
    p = p * x + 1.0 / 5040.0;
    p = p * x + 1.0 / 720.0;
    p = p * x + 1.0 / 120.0;
    p = p * x + 1.0 / 24.0;
    p = p * x + 1.0 / 6.0;
    p = p * x + 0.5;
    p = p * x + 1.0;
    p = p * x + 1.0;
    return ldexp(p, -(int)kd);
}

double oracle_exp_neg(double y) { return exp_neg(y); }

/* Hertz energy (kT) of a depletant at squared distance r2 from a colloid. */
static double hertz(const osim *S, double r2)
{
    if (!(r2 < S->R_s2)) return 0.0;
    double t = 1.0 - sqrt(r2) / S->R_s;
    return S->soft_eps * ((t * t) * sqrt(t));
}

double oracle_hertz(double eps, double sigma, double r2)
{
    osim S;
    memset(&S, 0, sizeof S);
    S.soft_eps = eps;
    S.R_s = sigma;
    S.R_s2 = sigma * sigma;
    return hertz(&S, r2);
}

static int next_in_ball_w(const osim *S, uint32_t sweep, uint32_t tag,
                          uint32_t purpose, uint32_t sub, uint32_t *t,
                          uint32_t t_max, double e[3], uint32_t *w3)
{
    while (*t < t_max) {
        uint32_t w[4];
        draw(S->key, sweep, tag, purpose, sub, *t, w);
        *t += 1;
        e[0] = S->R_s * s11(w[0]);
        e[1] = S->R_s * s11(w[1]);
        e[2] = S->R_s * s11(w[2]);
        double r2 = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
        if (r2 < S->R_s2) {
            if (w3) *w3 = w[3];
            return 1;
        }
    }
    return 0;
}

static int next_in_ball(const osim *S, uint32_t sweep, uint32_t tag,
                        uint32_t purpose, uint32_t sub, uint32_t *t,
                        uint32_t t_max, double e[3])
{
    return next_in_ball_w(S, sweep, tag, purpose, sub, t, t_max, e, NULL);
}

/* The same for the paired depletant stream of a trial move. */
static int next_in_ball_paired(const osim *S, uint32_t sweep, uint32_t tag, uint32_t *t,
                               uint32_t t_max, double e[3])
{
    while (*t < t_max) {
        paired_point(S->key, S->R_s, sweep, tag, *t, e);
        *t += 1;
        double r2 = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
        if (r2 < S->R_s2) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Shell-restricted V_0 (Sec. III.C, the closing remark): for a sphere      */
/* translated by D, a depletant overlapping the new pose but not the old     */
/* one lies at distance >= R_s - |D| from the new centre, so the spherical   */
/* shell R_in <= |e| < R_s with R_in <= R_s - |D| is a valid V_0.  The shell */
/* is taken from SHELL_LEVELS quantised thicknesses so that each has a       */
/* precomputed Poisson table.                                                */
/* ------------------------------------------------------------------------ */
#define SHELL_LEVELS 32

/* Level of a translation from its move words w[0..2].  D_d = d_max n_d 2^-32
 * with n_d = 2 w_d + 1 - 2^32 (odd, |n_d| < 2^32); a_d = floor(|n_d| 2^-16)
 * + 1 exceeds |n_d| 2^-16, so with S = sum a_d^2 the displacement obeys
 * |D| < d_max sqrt(S) 2^-16.  The level is the smallest k >= 1 with
 * S <= 3 k^2 2^22, hence |D| < k sqrt(3) d_max / 32 = k dd.  Integer-only. */
static int shell_level_words(const uint32_t w[3])
{
    uint64_t S = 0;
    for (int d = 0; d < 3; ++d) {
        int64_t n = 2 * (int64_t)w[d] + 1 - ((int64_t)1 << 32);
        uint64_t a = ((uint64_t)(n < 0 ? -n : n) >> 16) + 1;
        S += a * a;
    }
    int k = 1;
    while (k < SHELL_LEVELS && S > (((uint64_t)3 * (uint64_t)k * (uint64_t)k) << 22)) ++k;
    return k;
}

int oracle_shell_level(const uint32_t w[3]) { return shell_level_words(w); }

/* Geometry of level k: thickness k dd plus 1e-9 R_s (so that rounding never
 * leaves a lens point outside), inner radius clamped at 0. */
static void shell_geometry(double R_s, double dd, int k, double *R_in, double *h)
{
    double t = (double)k * dd + 1e-9 * R_s;
    double r = R_s - t;
    if (r < 0.0) r = 0.0;
    *R_in = r;
    *h = R_s - r;
}

/* Mean depletant number of a shell: z_p (4 pi / 3) (R_s^3 - R_in^3). */
double oracle_shell_lambda(double R_s, double R_in, double n_r)
{
    double v = ((4.0 / 3.0) * ORACLE_PI) * (((R_s * R_s) * R_s) - ((R_in * R_in) * R_in));
    return n_r * v;
}

/* Next point of the depletant attempt stream uniform in the shell of level
 * lvl.  Attempt t: v_d = s11(w_d) uniform in the cube; r = R_in + h u01(w_3)
 * uniform in [R_in, R_s); accepted iff |v|^6 R_s^4 < r^4, i.e.
 * |v|^3 < (r / R_s)^2.  For v in the unit ball |v|^3 is uniform on [0, 1]
 * and independent of the direction v / |v|, so the accepted r has density
 * proportional to r^2 on [R_in, R_s) and the direction is uniform: e =
 * v (r / |v|) is uniform in the shell.  (r < R_s forces |v| < 1.) */
static int next_in_shell(const osim *S, int lvl, uint32_t sweep, uint32_t tag,
                         uint32_t *t, uint32_t t_max, double e[3])
{
    const double R_in = S->s_rin[lvl - 1], h = S->s_h[lvl - 1];
    while (*t < t_max) {
        uint32_t w[4];
        draw(S->key, sweep, tag, P_DEP, 0, *t, w);
        *t += 1;
        double v0 = s11(w[0]), v1 = s11(w[1]), v2 = s11(w[2]);
        double p2 = (v0 * v0 + v1 * v1) + v2 * v2;
        double r = R_in + h * u01(w[3]);
        double r2 = r * r;
        if (!(((p2 * p2) * p2) * S->R_s4 < r2 * r2)) continue;
        double sc = r / sqrt(p2);
        e[0] = v0 * sc;
        e[1] = v1 * sc;
        e[2] = v2 * sc;
        return 1;
    }
    return 0;
}

/* Cube V_0 (v0_mode 2; "any convenient V_0", Sec. III.C): the axis-aligned
 * cube [-R_s, R_s)^3 around the new reference point contains the new pose's
 * circumsphere, so every attempt is a depletant: e = R_s (s11(w_0), s11(w_1),
 * s11(w_2)) at attempt t = its index, and N_p ~ Poisson(z_p (2 R_s)^3). */
static void cube_point(const osim *S, uint32_t sweep, uint32_t tag, uint32_t t, double e[3],
                       uint32_t *w3)
{
    uint32_t w[4];
    draw(S->key, sweep, tag, P_DEP, 0, t, w);
    e[0] = S->R_s * s11(w[0]);
    e[1] = S->R_s * s11(w[1]);
    e[2] = S->R_s * s11(w[2]);
    *w3 = w[3];
}

double oracle_cube_lambda(double R_s, double n_r)
{
    double a = 2.0 * R_s;
    return n_r * ((a * a) * a);
}

/* Points of the shell generator for tests: attempts t = 0 .. n_att - 1 of
 * stream (sweep, tag) at level lvl of a sphere system; writes the accepted
 * points to e (3 per point) and returns their count. */
long oracle_shell_points(double R_s, double d_max, int lvl, uint64_t seed,
                         uint32_t sweep, uint32_t tag, uint32_t n_att, double *e)
{
    osim S;
    memset(&S, 0, sizeof S);
    if (lvl < 1 || lvl > SHELL_LEVELS || !(R_s > 0.0) || !(d_max >= 0.0)) return -1;
    S.R_s = R_s;
    S.R_s2 = R_s * R_s;
    S.R_s4 = S.R_s2 * S.R_s2;
    S.dd = (sqrt(3.0) * d_max) / 32.0;
    S.key.k[0] = (uint32_t)seed;
    S.key.k[1] = (uint32_t)(seed >> 32);
    shell_geometry(R_s, S.dd, lvl, &S.s_rin[lvl - 1], &S.s_h[lvl - 1]);
    uint32_t t = 0;
    long m = 0;
    while (next_in_shell(&S, lvl, sweep, tag, &t, n_att, e + 3 * m)) ++m;
    return m;
}

/* Is v (relative to the new reference point) free of every other colloid? */
static int free_of_neighbours(const osim *S, const double v[3], const onb *nb,
                              int m)
{
    for (int a = 0; a < m; ++a) {
        double u[3] = {v[0] - nb[a].d[0], v[1] - nb[a].d[1], v[2] - nb[a].d[2]};
        if (dep_overlap(&S->sh, S->q, u, nb[a].qj)) return 0;
    }
    return 1;
}

/* Configurational-bias weight of blocking depletant k, Sec. III.D, Eq. (12).
 * Forward: n_trial reinsertion trials uniform in the old circumsphere; a
 * success overlaps the old pose, not the new pose and no other colloid
 * (N'_insert).  Reverse: the original depletant plus n_trial - 1 trials
 * uniform in the new circumsphere; a success overlaps the new pose, not the
 * old pose and no other colloid (N_insert + 1).  cb_mode 1 is the literal
 * printed form with the lens counts N_k. */
static double cb_factor(const osim *S, uint32_t sweep, uint32_t tag, uint32_t k,
                        const double o[3], const double *q_old,
                        const double *q_new, const onb *nb, int m,
                        uint64_t *cnt)
{
    int n_fwd_trials = S->n_trial;
    int n_rev_trials = S->cb_mode == 0 ? S->n_trial - 1 : S->n_trial;
    uint32_t t = 0, t_max = 64u * (uint32_t)(n_fwd_trials + 1);
    int n_ins_fwd = 0, n_lens_fwd = 0, found = 0;
    double e[3];
    while (found < n_fwd_trials &&
           next_in_ball(S, sweep, tag, P_CB_FWD, k, &t, t_max, e)) {
        ++found;
        double y[3] = {o[0] + e[0], o[1] + e[1], o[2] + e[2]};
        if (!dep_overlap(&S->sh, S->q, e, q_old)) continue;
        if (dep_overlap(&S->sh, S->q, y, q_new)) continue;
        ++n_lens_fwd;
        if (!free_of_neighbours(S, y, nb, m)) continue;
        ++n_ins_fwd;
    }
    if (found < n_fwd_trials) cnt[C_CAP]++;
    t = 0;
    t_max = 64u * (uint32_t)(n_rev_trials + 1);
    found = 0;
    int n_ins_rev = 0;
    while (found < n_rev_trials &&
           next_in_ball(S, sweep, tag, P_CB_REV, k, &t, t_max, e)) {
        ++found;
        double u[3] = {e[0] - o[0], e[1] - o[1], e[2] - o[2]};
        if (!dep_overlap(&S->sh, S->q, e, q_new)) continue;
        if (dep_overlap(&S->sh, S->q, u, q_old)) continue;
        if (!free_of_neighbours(S, e, nb, m)) continue;
        ++n_ins_rev;
    }
    if (found < n_rev_trials) cnt[C_CAP]++;
    cnt[C_CB_FWD_OK] += (uint64_t)n_ins_fwd;
    cnt[C_CB_REV_OK] += (uint64_t)n_ins_rev;
    if (S->cb_mode == 0)
        return (double)n_ins_fwd / (double)(n_ins_rev + 1);
    if (n_lens_fwd == 0) return 0.0;
    return ((double)n_ins_fwd * (double)(n_lens_fwd + 1)) /
           ((double)(n_ins_rev + 1) * (double)n_lens_fwd);
}

/* Acceptance of one proposed move of colloid i to the pose (xn, qn); o is the
 * old reference point relative to the new one (zero for a rotation).
 * Sec. III.B-III.D.  Returns 1 to accept, 0 to reject. */
static int accept_move(const osim *S, uint32_t sweep, int i, const double xn[3],
                       const double qn[4], const double o[3], const double *qo,
                       int lvl, const int ci[3], const double *pos, const double *quat,
                       const int *cell_start, const int *cell_idx, onb *nb,
                       uint64_t *cnt)
{
    uint32_t tag = (uint32_t)i;

    /* Colloid-colloid overlap at the new pose: Delta H_cc = infinity. */
    int m = gather_neighbours(S, i, xn, ci, pos, quat, cell_start, cell_idx, nb);
    if (S->soft_eps > 0.0) {
        /* soft interactions sum the neighbours' energies in ascending index */
        for (int a = 1; a < m; ++a) {
            onb v = nb[a];
            int b = a - 1;
            while (b >= 0 && nb[b].j > v.j) { nb[b + 1] = nb[b]; --b; }
            nb[b + 1] = v;
        }
    }
    for (int a = 0; a < m; ++a) {
        if (pair_overlap(&S->sh, nb[a].d, qn, nb[a].qj)) {
            cnt[C_REJ_OVERLAP]++;
            return 0;
        }
    }
    if (!(S->lambda > 0.0)) return 1;

    /* N_p ~ Poisson(z_p |V_0|) depletants uniform in V_0 (Sec. III.B step 2);
     * V_0 is the circumsphere, or the shell of level lvl > 0 (Sec. III.C). */
    uint32_t wp[4];
    draw(S->key, sweep, tag, P_POISSON, 0, 0, wp);
    int n_p = lvl > 0 ? poisson_invert(S->sF[lvl - 1], S->snF[lvl - 1], u53(wp[0], wp[1]))
                      : poisson_invert(S->F, S->nF, u53(wp[0], wp[1]));
    cnt[C_DEP_DRAWN] += (uint64_t)n_p;
    uint32_t t = 0, t_max = 64u * (uint32_t)(n_p + 1);
    int n_block = 0;
    double W = 1.0;
    for (int k = 0; k < n_p; ++k) {
        double e[3];
        int got;
        uint32_t w3 = 0;
        if (S->v0_mode == 2 && S->soft_eps > 0.0) {
            cube_point(S, sweep, tag, t, e, &w3);
            t += 1;
            got = 1;
        } else if (S->v0_mode == 2) {
            /* hard, cube: the paired stream, every attempt a depletant */
            paired_point(S->key, S->R_s, sweep, tag, t, e);
            t += 1;
            got = 1;
        } else if (lvl > 0) {
            got = next_in_shell(S, lvl, sweep, tag, &t, t_max, e);
        } else if (S->soft_eps > 0.0) {
            /* soft: one point per call, its fourth word decides blocking */
            got = next_in_ball_w(S, sweep, tag, P_DEP, 0, &t, t_max, e, &w3);
        } else {
            got = next_in_ball_paired(S, sweep, tag, &t, t_max, e);
        }
        if (!got) {
            cnt[C_CAP]++;
            break;
        }
        cnt[C_DEP_EVAL]++;
        if (S->soft_eps > 0.0) {
            /* soft: blocks with probability b(e), decided by the attempt's
             * fourth word */
            double u[3] = {e[0] - o[0], e[1] - o[1], e[2] - o[2]};
            double e_new = exp_neg(hertz(S, (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]));
            double e_old = exp_neg(hertz(S, (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]));
            if (!(e_old > e_new)) continue;
            double U = 0.0;
            for (int a = 0; a < m; ++a) {
                double v[3] = {e[0] - nb[a].d[0], e[1] - nb[a].d[1], e[2] - nb[a].d[2]};
                U = U + hertz(S, (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
            }
            double b = exp_neg(U) * (e_old - e_new);
            if (!(u01(w3) < b)) continue;
        } else {
            /* irrelevant unless it overlaps the new pose */
            if (!dep_overlap(&S->sh, S->q, e, qn)) continue;
            /* ignored if it overlaps the old configuration */
            double u[3] = {e[0] - o[0], e[1] - o[1], e[2] - o[2]};
            if (dep_overlap(&S->sh, S->q, u, qo)) continue;
            if (!free_of_neighbours(S, e, nb, m)) continue;
        }
        /* overlaps only the new configuration: blocks the move */
        cnt[C_DEP_BLOCKING]++;
        ++n_block;
        if (S->n_trial == 0) {
            cnt[C_REJ_DEP]++;
            return 0;
        }
        double f = cb_factor(S, sweep, tag, (uint32_t)k, o, qo, qn, nb, m, cnt);
        if (f == 0.0) {
            cnt[C_REJ_CB]++;
            return 0;
        }
        W = W * f;
    }
    if (n_block > 0) {
        uint32_t wa[4];
        draw(S->key, sweep, tag, P_ACCEPT, 0, 0, wa);
        if (!(u53(wa[0], wa[1]) < W)) {
            cnt[C_REJ_CB]++;
            return 0;
        }
    }
    return 1;
}

/* Rotation proposal (Sec. V: orientational moves of anisotropic colloids).
 * v uniform in the unit ball from the purpose-2 attempt stream (rejection
 * from the cube, at most 64 attempts); q' = (q_r q)/|q_r q| with
 * q_r = (1, alpha v): a rotation about v/|v| by 2 atan(alpha |v|) <= a_max
 * when alpha = tan(a_max / 2).  The proposal density of q_r equals that of its
 * inverse (v -> -v), so the move is symmetric.  Returns 0 if the cap is hit. */
static int propose_rotation(okey key, uint32_t sweep, uint32_t tag, double alpha,
                            const double qo[4], double qn[4])
{
    double v[3];
    int ok = 0;
    for (uint32_t t = 0; t < 64u && !ok; ++t) {
        uint32_t w[4];
        draw(key, sweep, tag, P_ROT, 0, t, w);
        v[0] = s11(w[0]);
        v[1] = s11(w[1]);
        v[2] = s11(w[2]);
        ok = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2] < 1.0;
    }
    if (!ok) return 0;
    double s1 = 1.0, x1 = alpha * v[0], y1 = alpha * v[1], z1 = alpha * v[2];
    double s2 = qo[0], x2 = qo[1], y2 = qo[2], z2 = qo[3];
    double ms = s1 * s2 - ((x1 * x2 + y1 * y2) + z1 * z2);
    double mx = (s1 * x2 + s2 * x1) + (y1 * z2 - z1 * y2);
    double my = (s1 * y2 + s2 * y1) + (z1 * x2 - x1 * z2);
    double mz = (s1 * z2 + s2 * z1) + (x1 * y2 - y1 * x2);
    double nrm = sqrt(((ms * ms + mx * mx) + my * my) + mz * mz);
    qn[0] = ms / nrm;
    qn[1] = mx / nrm;
    qn[2] = my / nrm;
    qn[3] = mz / nrm;
    return 1;
}

int oracle_rotation_proposal(uint64_t seed, uint32_t replica, uint32_t sweep,
                             uint32_t tag, double a_max, const double *q_in,
                             double *q_out)
{
    okey key = {{(uint32_t)seed, (uint32_t)(seed >> 32) ^ replica}};
    if (!q_in || !q_out || !(a_max > 0.0) || a_max >= 3.0) return -1;
    return propose_rotation(key, sweep, tag, tan(0.5 * a_max), q_in, q_out);
}

/* One trial move of colloid i in the active cell ci: proposal, cell check,
 * acceptance, commit. */
static void trial_move(const osim *S, uint32_t sweep, int i, const int ci[3],
                       const double sigma[3], double *pos, double *quat,
                       const int *cell_start, const int *cell_idx, onb *nb,
                       uint64_t *cnt)
{
    uint32_t tag = (uint32_t)i;
    uint32_t w[4];
    cnt[C_MOVES]++;
    draw(S->key, sweep, tag, P_MOVE, 0, 0, w);
    const double *qo = quat ? quat + 4 * i : NULL;

    int translate = 1;
    if (S->sh.kind != SHAPE_SPHERE && S->a_max > 0.0 && qo) {
        if (S->p_translate <= 0.0) translate = 0;
        else if (S->p_translate < 1.0) translate = u01(w[3]) < S->p_translate;
    }

    double xn[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    double qn[4] = {1.0, 0.0, 0.0, 0.0};
    if (qo) { qn[0] = qo[0]; qn[1] = qo[1]; qn[2] = qo[2]; qn[3] = qo[3]; }
    double o[3] = {0.0, 0.0, 0.0};
    int lvl = 0;

    if (translate) {
        cnt[C_TRANSLATE]++;
        for (int d = 0; d < 3; ++d) {
            double x = pos[3 * i + d] + S->d_max * s11(w[d]);
            if (x < 0.0) x = x + S->L;
            if (x >= S->L) x = x - S->L;
            xn[d] = x;
        }
        /* Sec. III.E: particles are not allowed to move outside their cells. */
        for (int d = 0; d < 3; ++d) {
            if (cell_coord(xn[d], sigma[d], S->L, S->w, S->nc) != ci[d]) {
                cnt[C_REJ_CELL]++;
                return;
            }
        }
        for (int d = 0; d < 3; ++d) o[d] = min_image(pos[3 * i + d] - xn[d], S->L);
        if (S->v0_mode == 1) lvl = shell_level_words(w);
    } else if (!propose_rotation(S->key, sweep, tag, S->alpha, qo, qn)) {
        cnt[C_CAP]++;
        return;
    }

    if (!accept_move(S, sweep, i, xn, qn, o, qo, lvl, ci, pos, quat, cell_start,
                     cell_idx, nb, cnt))
        return;

    pos[3 * i] = xn[0];
    pos[3 * i + 1] = xn[1];
    pos[3 * i + 2] = xn[2];
    if (quat) {
        quat[4 * i] = qn[0]; quat[4 * i + 1] = qn[1];
        quat[4 * i + 2] = qn[2]; quat[4 * i + 3] = qn[3];
    }
    cnt[C_ACCEPT]++;
}

/* Largest even cell count with cell width >= 2 R_circ + q (Sec. III.E). */
int oracle_auto_cells(double L, double R_circ, double q)
{
    double w_min = 2.0 * R_circ + q;
    int nc = (int)(L / w_min);
    if (nc & 1) nc -= 1;
    return nc;
}

static void sim_free(osim *S)
{
    free(S->F);
    S->F = NULL;
    for (int k = 0; k < SHELL_LEVELS; ++k) { free(S->sF[k]); S->sF[k] = NULL; }
}

static int sim_init(osim *S, int n, double L, int shape,
                    const double *shape_params, int n_shape_params, double q,
                    double n_r, int n_trial, int cb_mode, int v0_mode, double soft_eps,
                    double d_max, double a_max, double p_translate, uint64_t seed,
                    uint32_t replica, int n_cell, int brute_force)
{
    memset(S, 0, sizeof *S);
    if (n < 1 || !(L > 0.0) || !shape_params) return -1;
    if (shape_init(&S->sh, shape, shape_params, n_shape_params) != 0) return -1;
    S->n = n;
    S->L = L;
    S->q = q;
    S->n_r = n_r;
    S->R_s = S->sh.R_circ + 0.5 * q;
    S->R_s2 = S->R_s * S->R_s;
    S->lambda = n_r > 0.0 ? (v0_mode == 2 ? oracle_cube_lambda(S->R_s, n_r)
                                          : oracle_lambda(S->R_s, n_r)) : 0.0;
    S->n_trial = n_trial;
    S->cb_mode = cb_mode;
    S->d_max = d_max;
    S->a_max = a_max;
    S->p_translate = p_translate;
    /* rotation by angle 2 atan(alpha |v|) <= a_max about v/|v|, |v| < 1 */
    S->alpha = a_max > 0.0 ? tan(0.5 * a_max) : 0.0;
    if (!(a_max >= 0.0) || a_max >= 3.0) return -1;
    S->key.k[0] = (uint32_t)seed;
    S->key.k[1] = (uint32_t)(seed >> 32) ^ replica;
    S->nc = n_cell > 0 ? n_cell : oracle_auto_cells(L, S->sh.R_circ, q);
    S->brute_force = brute_force;
    if (S->nc < 2 || (S->nc & 1) || n_trial < 0 || q < 0.0 || n_r < 0.0) return -1;
    S->w = L / (double)S->nc;
    if (S->w < 2.0 * S->sh.R_circ + q) return -1;
    if (!(d_max >= 0.0) || d_max >= S->w) return -1;
    if (S->lambda > 0.0) {
        int cap = 8192;
        S->F = (double *)malloc(sizeof(double) * (size_t)cap);
        if (!S->F) return -1;
        S->nF = oracle_poisson_table(S->lambda, S->F, cap);
        if (S->nF < 0) { sim_free(S); return -1; }
    }
    /* shell V_0: spheres only (anisotropic colloids keep the circumsphere) */
    if (v0_mode < 0 || v0_mode > 2 || (v0_mode == 1 && shape != SHAPE_SPHERE)) {
        sim_free(S);
        return -1;
    }
    /* soft colloid-depletant interaction: spheres, no CB, a V_0 that holds
     * the new circumsphere (not the shell) */
    if (!(soft_eps >= 0.0) ||
        (soft_eps > 0.0 && (shape != SHAPE_SPHERE || n_trial != 0 || v0_mode == 1))) {
        sim_free(S);
        return -1;
    }
    S->soft_eps = soft_eps;
    S->v0_mode = v0_mode;
    S->R_s4 = S->R_s2 * S->R_s2;
    S->dd = (sqrt(3.0) * d_max) / 32.0;
    if (v0_mode == 1) {
        for (int k = 1; k <= SHELL_LEVELS; ++k) {
            shell_geometry(S->R_s, S->dd, k, &S->s_rin[k - 1], &S->s_h[k - 1]);
            if (!(S->lambda > 0.0)) continue;
            int cap = 8192;
            S->sF[k - 1] = (double *)malloc(sizeof(double) * (size_t)cap);
            if (!S->sF[k - 1]) { sim_free(S); return -1; }
            double lam = oracle_shell_lambda(S->R_s, S->s_rin[k - 1], n_r);
            S->snF[k - 1] = oracle_poisson_table(lam, S->sF[k - 1], cap);
            if (S->snF[k - 1] < 0) { sim_free(S); return -1; }
        }
    }
    return 0;
}

/*
 * Run n_sweeps sweeps starting at sweep index sweep0, in place on pos (n x 3)
 * and quat (n x 4 or NULL).  counters: C_N uint64 accumulated.  If hist is
 * non-NULL, after every sweep all pair distances r < hist_rmax are binned into
 * hist[hist_bins] (minimum image).  n_threads > 1 moves the active cells of a
 * colour on that many threads (identical results).  Returns 0 or a negative
 * error.  oracle_run is the serial form.
 */
int oracle_run_threads(int n, double L, int shape, const double *shape_params,
                       int n_shape_params, double q, double n_r, int n_trial,
                       int cb_mode, int v0_mode, double soft_eps, double d_max, double a_max,
                       double p_translate, uint64_t seed, uint32_t replica, int n_cell,
                       int brute_force, double *pos, double *quat, uint64_t sweep0,
                       int n_sweeps, uint64_t *counters, int hist_bins, double hist_rmax,
                       uint64_t *hist, int n_threads)
{
    osim S;
    if (!pos || !counters || n_sweeps < 0 || n_threads < 1) return -1;
    /* brute-force neighbours read every colloid: only the serial order */
    if (brute_force) n_threads = 1;
    if (sim_init(&S, n, L, shape, shape_params, n_shape_params, q, n_r, n_trial,
                 cb_mode, v0_mode, soft_eps, d_max, a_max, p_translate, seed, replica, n_cell,
                 brute_force) != 0)
        return -1;
    int ncell = S.nc * S.nc * S.nc;
    int *cell_start = (int *)malloc(sizeof(int) * (size_t)(ncell + 1));
    int *cell_idx = (int *)malloc(sizeof(int) * (size_t)n);
    /* one neighbour buffer per thread */
    onb *nb = (onb *)malloc(sizeof(onb) * (size_t)n * (size_t)n_threads);
    int rc = 0;
    if (!cell_start || !cell_idx || !nb) { rc = -1; goto out; }

    for (int sw = 0; sw < n_sweeps; ++sw) {
        uint32_t sweep = (uint32_t)(sweep0 + (uint64_t)sw);
        double sigma[3];
        int perm[8];
        oracle_schedule(seed, replica, sweep, S.w, sigma, perm);
        if (oracle_cell_list(n, L, S.nc, pos, seed, replica, sweep, cell_start,
                             cell_idx) != 0) { rc = -1; goto out; }
        for (int p = 0; p < 8; ++p) {
            int colour = perm[p];
            if (n_threads == 1) {
                for (int c = 0; c < ncell; ++c) {
                    int cx = c % S.nc, cy = (c / S.nc) % S.nc, cz = c / (S.nc * S.nc);
                    int col = (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
                    if (col != colour) continue;
                    int ci[3] = {cx, cy, cz};
                    for (int s = cell_start[c]; s < cell_start[c + 1]; ++s)
                        trial_move(&S, sweep, cell_idx[s], ci, sigma, pos, quat,
                                   cell_start, cell_idx, nb, counters);
                }
                continue;
            }
            /* the active cells of this colour over the threads (Sec. III.E) */
#pragma omp parallel num_threads(n_threads)
            {
                int th = 0;
#ifdef _OPENMP
                th = omp_get_thread_num();
#endif
                onb *nbt = nb + (size_t)th * (size_t)n;
                uint64_t ct[C_N];
                memset(ct, 0, sizeof ct);
#pragma omp for schedule(dynamic, 8)
                for (int c = 0; c < ncell; ++c) {
                    int cx = c % S.nc, cy = (c / S.nc) % S.nc, cz = c / (S.nc * S.nc);
                    int col = (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
                    if (col != colour) continue;
                    int ci[3] = {cx, cy, cz};
                    for (int s = cell_start[c]; s < cell_start[c + 1]; ++s)
                        trial_move(&S, sweep, cell_idx[s], ci, sigma, pos, quat,
                                   cell_start, cell_idx, nbt, ct);
                }
#pragma omp critical
                for (int k = 0; k < C_N; ++k) counters[k] += ct[k];
            }
        }
        if (hist && hist_bins > 0) {
            double binw = hist_rmax / (double)hist_bins;
            for (int a = 0; a < n; ++a)
                for (int b = a + 1; b < n; ++b) {
                    double r2 = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        double dd = min_image(pos[3 * b + d] - pos[3 * a + d], L);
                        r2 += dd * dd;
                    }
                    double r = sqrt(r2);
                    if (r < hist_rmax) {
                        int bin = (int)(r / binw);
                        if (bin < hist_bins) hist[bin]++;
                    }
                }
        }
    }
out:
    sim_free(&S);
    free(cell_start);
    free(cell_idx);
    free(nb);
    return rc;
}

int oracle_run(int n, double L, int shape, const double *shape_params,
               int n_shape_params, double q, double n_r, int n_trial,
               int cb_mode, int v0_mode, double soft_eps, double d_max, double a_max,
               double p_translate, uint64_t seed, uint32_t replica, int n_cell, int brute_force,
               double *pos, double *quat, uint64_t sweep0, int n_sweeps,
               uint64_t *counters, int hist_bins, double hist_rmax,
               uint64_t *hist)
{
    return oracle_run_threads(n, L, shape, shape_params, n_shape_params, q, n_r, n_trial,
                              cb_mode, v0_mode, soft_eps, d_max, a_max, p_translate, seed,
                              replica, n_cell, brute_force, pos, quat, sweep0, n_sweeps,
                              counters, hist_bins, hist_rmax, hist, 1);
}

/*
 * Acceptance count of one fixed proposed move: colloid i from its pose in
 * (pos, quat) to (xn, qn), evaluated n_rep times with the independent random
 * streams of sweep indices sweep0 .. sweep0 + n_rep - 1.  Neighbours by brute
 * force.  Used to check detailed balance of the acceptance rule directly.
 */
long oracle_acceptance(int n, double L, int shape, const double *shape_params,
                       int n_shape_params, double q, double n_r, int n_trial,
                       int cb_mode, int v0_mode, double soft_eps, double d_max, uint64_t seed,
                       const double *pos,
                       const double *quat, int i, const double *xn_in,
                       const double *qn_in, uint64_t sweep0, long n_rep,
                       uint64_t *counters)
{
    osim S;
    if (!pos || !xn_in || i < 0 || i >= n || n_rep < 0 || !counters) return -1;
    if (sim_init(&S, n, L, shape, shape_params, n_shape_params, q, n_r, n_trial,
                 cb_mode, v0_mode, soft_eps, d_max, 0.0, 1.0, seed, 0, 0, 1) != 0)
        return -1;
    onb *nb = (onb *)malloc(sizeof(onb) * (size_t)n);
    if (!nb) { sim_free(&S); return -1; }
    double xn[3] = {xn_in[0], xn_in[1], xn_in[2]};
    double qn[4] = {1.0, 0.0, 0.0, 0.0};
    const double *qo = quat ? quat + 4 * i : NULL;
    if (qn_in) { qn[0] = qn_in[0]; qn[1] = qn_in[1]; qn[2] = qn_in[2]; qn[3] = qn_in[3]; }
    else if (qo) { qn[0] = qo[0]; qn[1] = qo[1]; qn[2] = qo[2]; qn[3] = qo[3]; }
    double o[3];
    for (int d = 0; d < 3; ++d) o[d] = min_image(pos[3 * i + d] - xn[d], L);
    int ci[3] = {0, 0, 0};
    /* shell V_0 for a given displacement: the thinnest level whose shell
     * holds every point that overlaps the new pose but not the old one */
    int lvl = 0;
    if (S.v0_mode == 1) {
        double dl = sqrt((o[0] * o[0] + o[1] * o[1]) + o[2] * o[2]);
        lvl = 1;
        while (lvl < SHELL_LEVELS && S.s_h[lvl - 1] < dl) ++lvl;
        if (S.s_h[lvl - 1] < dl && S.s_rin[lvl - 1] > 0.0) {
            free(nb);
            sim_free(&S);
            return -1;
        }
    }
    long acc = 0;
    for (long r = 0; r < n_rep; ++r)
        acc += accept_move(&S, (uint32_t)(sweep0 + (uint64_t)r), i, xn, qn, o, qo,
                           lvl, ci, pos, quat, NULL, NULL, nb, counters);
    free(nb);
    sim_free(&S);
    return acc;
}

/*
 * Depletant free-volume probe (Sec. IV.A observable): count how many of
 * n_probe uniform points in the box overlap no colloid.  Brute force over
 * all colloids.  Probe points use purpose P_PROBE with stream = probe index.
 */
long oracle_free_volume(int n, double L, int shape, const double *shape_params,
                        double q, const double *pos, const double *quat,
                        uint64_t seed, uint32_t sample, long n_probe)
{
    oshape sh;
    if (shape_init(&sh, shape, shape_params, shape == SHAPE_SPHEROID ? 2 : 1) != 0) return -1;
    okey key = {{(uint32_t)seed, (uint32_t)(seed >> 32)}};
    long free_count = 0;
    for (long m = 0; m < n_probe; ++m) {
        uint32_t w[4];
        draw(key, sample, (uint32_t)m, P_PROBE, (uint32_t)(m >> 32), 0, w);
        double p[3] = {L * u01(w[0]), L * u01(w[1]), L * u01(w[2])};
        int hit = 0;
        for (int j = 0; j < n && !hit; ++j) {
            double v[3];
            for (int d = 0; d < 3; ++d) v[d] = min_image(p[d] - pos[3 * j + d], L);
            hit = dep_overlap(&sh, q, v, quat ? quat + 4 * j : NULL);
        }
        if (!hit) ++free_count;
    }
    return free_count;
}

/* ------------------------------------------------------------------------ */
/* Gibbs-ensemble colloid exchange with configurational bias (Sec. IV.B,    */
/* coexistence of the penetrable-hard-sphere model): two boxes share one    */
/* depletant reservoir (fugacity z_p); a colloid leaves one box for a       */
/* uniform random position in the other.  Depletants are inserted at the    */
/* new position; those that overlap the inserted colloid and no other       */
/* colloid of that box block the move, or, with n_trial > 0, are reinserted */
/* in the old box around the removed colloid (the weight of Eq. 12).  The   */
/* Gibbs factor N_s V_d / ((N_d + 1) V_s) enters by a Metropolis test.      */
/* Spheres.  Boxes keep their colloids in slots 0..n-1: a removed colloid's */
/* slot takes the box's last colloid; an inserted one takes slot n.         */
/* ------------------------------------------------------------------------ */

enum { G_ATTEMPT = 0, G_ACCEPT, G_REJ_EMPTY, G_REJ_RATIO, G_REJ_OVERLAP, G_REJ_DEP,
       G_REJ_CB, G_DEP_DRAWN, G_N = 8 };

#define GIBBS_STREAM 0xFFFFFFFEu   /* RNG stream word of the exchange moves */

typedef struct {
    int n;
    double L;
    double *pos;
} obox;

static void gibbs_draw(const osim *S, uint32_t step, uint32_t purpose, uint32_t sub,
                       uint32_t t, uint32_t w[4])
{
    draw(S->key, step, GIBBS_STREAM, purpose, sub, t, w);
}

/* Is the point x + v of box b free of every colloid of b except slot skip? */
static int gibbs_free(const osim *S, const obox *b, const double x[3], const double v[3],
                      int skip)
{
    for (int j = 0; j < b->n; ++j) {
        if (j == skip) continue;
        double u[3];
        for (int d = 0; d < 3; ++d) u[d] = v[d] - min_image(b->pos[3 * j + d] - x[d], b->L);
        if (dep_overlap(&S->sh, S->q, u, NULL)) return 0;
    }
    return 1;
}

/* CB weight of blocking depletant k: forward trials in the old colloid's
 * circumsphere in the source box (overlapping it, free of the source's
 * other colloids), reverse trials in the new one in the destination box
 * (overlapping the inserted colloid, free of the others):
 * f = N'_insert / (N_insert + 1), with n_trial - 1 reverse trials. */
static double gibbs_cb(const osim *S, uint32_t step, uint32_t k, const obox *src, int i,
                       const double xo[3], const obox *dst, const double xn[3], uint64_t *cnt)
{
    int n_fwd = S->n_trial, n_rev = S->n_trial - 1, found = 0, nf = 0, nr = 0;
    uint32_t t = 0, t_max = 64u * (uint32_t)(n_fwd + 1);
    double e[3];
    while (found < n_fwd && next_in_ball(S, step, GIBBS_STREAM, P_CB_FWD, k, &t, t_max, e)) {
        ++found;
        if (!dep_overlap(&S->sh, S->q, e, NULL)) continue;
        if (!gibbs_free(S, src, xo, e, i)) continue;
        ++nf;
    }
    if (found < n_fwd) cnt[C_CAP]++;
    t = 0;
    t_max = 64u * (uint32_t)(n_rev + 1);
    found = 0;
    while (found < n_rev && next_in_ball(S, step, GIBBS_STREAM, P_CB_REV, k, &t, t_max, e)) {
        ++found;
        if (!dep_overlap(&S->sh, S->q, e, NULL)) continue;
        if (!gibbs_free(S, dst, xn, e, -1)) continue;
        ++nr;
    }
    if (found < n_rev) cnt[C_CAP]++;
    cnt[C_CB_FWD_OK] += (uint64_t)nf;
    cnt[C_CB_REV_OK] += (uint64_t)nr;
    return (double)nf / (double)(nr + 1);
}

/* Acceptance of the exchange of slot i of box src to position xn of box dst
 * (the Gibbs test, then Sec. III.B-D at the new position). */
static int gibbs_accept(const osim *S, uint32_t step, obox *src, int i, obox *dst,
                        const double xn[3], uint64_t *g, uint64_t *cnt)
{
    double Vs = (src->L * src->L) * src->L, Vd = (dst->L * dst->L) * dst->L;
    double G = ((double)src->n * Vd) / ((double)(dst->n + 1) * Vs);
    uint32_t wa[4];
    gibbs_draw(S, step, P_ACCEPT, 1, 0, wa);
    if (!(u53(wa[0], wa[1]) < G)) { g[G_REJ_RATIO]++; return 0; }
    for (int j = 0; j < dst->n; ++j) {
        double v[3];
        for (int d = 0; d < 3; ++d) v[d] = min_image(dst->pos[3 * j + d] - xn[d], dst->L);
        if ((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2] < S->sh.d * S->sh.d) {
            g[G_REJ_OVERLAP]++;
            return 0;
        }
    }
    if (!(S->lambda > 0.0)) return 1;
    const double *xo = src->pos + 3 * i;
    uint32_t wp[4];
    gibbs_draw(S, step, P_POISSON, 0, 0, wp);
    int n_p = poisson_invert(S->F, S->nF, u53(wp[0], wp[1]));
    g[G_DEP_DRAWN] += (uint64_t)n_p;
    cnt[C_DEP_DRAWN] += (uint64_t)n_p;
    uint32_t t = 0, t_max = 64u * (uint32_t)(n_p + 1);
    int n_block = 0;
    double W = 1.0;
    for (int k = 0; k < n_p; ++k) {
        double e[3];
        if (!next_in_ball(S, step, GIBBS_STREAM, P_DEP, 0, &t, t_max, e)) {
            cnt[C_CAP]++;
            break;
        }
        cnt[C_DEP_EVAL]++;
        if (!dep_overlap(&S->sh, S->q, e, NULL)) continue;
        if (!gibbs_free(S, dst, xn, e, -1)) continue;
        cnt[C_DEP_BLOCKING]++;
        ++n_block;
        if (S->n_trial == 0) { g[G_REJ_DEP]++; return 0; }
        double f = gibbs_cb(S, step, (uint32_t)k, src, i, xo, dst, xn, cnt);
        if (f == 0.0) { g[G_REJ_CB]++; return 0; }
        W = W * f;
    }
    if (n_block > 0) {
        uint32_t w2[4];
        gibbs_draw(S, step, P_ACCEPT, 0, 0, w2);
        if (!(u53(w2[0], w2[1]) < W)) { g[G_REJ_CB]++; return 0; }
    }
    return 1;
}

/* One exchange attempt at step index `step`: source box from the top bit of
 * the first word, slot i = floor(w_1 n_src / 2^32), new position
 * L_dst u01(w) from the second draw. */
static void gibbs_exchange(const osim *S, uint32_t step, obox box[2], uint64_t *g, uint64_t *cnt)
{
    uint32_t w[4], wx[4];
    g[G_ATTEMPT]++;
    gibbs_draw(S, step, P_MOVE, 0, 0, w);
    int s = (int)(w[0] >> 31), dd = 1 - s;
    obox *src = &box[s], *dst = &box[dd];
    if (src->n == 0) { g[G_REJ_EMPTY]++; return; }
    int i = (int)(((uint64_t)w[1] * (uint64_t)src->n) >> 32);
    gibbs_draw(S, step, P_MOVE, 1, 0, wx);
    double xn[3] = {dst->L * u01(wx[0]), dst->L * u01(wx[1]), dst->L * u01(wx[2])};
    if (!gibbs_accept(S, step, src, i, dst, xn, g, cnt)) return;
    for (int d = 0; d < 3; ++d) dst->pos[3 * dst->n + d] = xn[d];
    dst->n++;
    src->n--;
    for (int d = 0; d < 3; ++d) src->pos[3 * i + d] = src->pos[3 * src->n + d];
    g[G_ACCEPT]++;
}

/*
 * A Gibbs pair of sphere boxes (replicas rep0, rep1 of seed; the exchange
 * streams use rep0's key): n_cycles of { sweeps_per_cycle checkerboard
 * sweeps of each box (sweep indices sweep0, sweep0 + 1, ...), then
 * ex_per_cycle exchange attempts (steps step0, step0 + 1, ...) }.  pos0,
 * pos1: capacity n[0] + n[1] slots each (3 doubles); n updated.  counters:
 * 2 x C_N (sweeps and exchange depletant work of each box; the exchange's
 * depletant counts go to the source box), g: G_N exchange counters.
 */
int oracle_gibbs_run(double diameter, double q, double n_r, int n_trial, double d_max0,
                     double d_max1, uint64_t seed, uint32_t rep0, uint32_t rep1, double L0,
                     double L1, int *n, double *pos0, double *pos1, uint64_t sweep0,
                     uint64_t step0, int n_cycles, int sweeps_per_cycle, int ex_per_cycle,
                     uint64_t *counters, uint64_t *g)
{
    if (!n || !pos0 || !pos1 || !counters || !g || n[0] < 0 || n[1] < 0 || n_cycles < 0)
        return -1;
    osim S;
    double sp[1] = {diameter};
    /* the pair's parameters (table, key) as box 0's; its box length is not used */
    if (sim_init(&S, 1, L0, SHAPE_SPHERE, sp, 1, q, n_r, n_trial, 0, 0, 0.0, 0.0, 0.0, 1.0,
                 seed, rep0, 0, 1) != 0)
        return -1;
    obox box[2] = {{n[0], L0, pos0}, {n[1], L1, pos1}};
    uint64_t sweep = sweep0, step = step0;
    int rc = 0;
    for (int cy = 0; cy < n_cycles && rc == 0; ++cy) {
        for (int b = 0; b < 2 && rc == 0; ++b) {
            if (box[b].n == 0 || sweeps_per_cycle == 0) continue;
            rc = oracle_run(box[b].n, box[b].L, SHAPE_SPHERE, sp, 1, q, n_r, n_trial, 0, 0, 0.0,
                            b == 0 ? d_max0 : d_max1, 0.0, 1.0, seed, b == 0 ? rep0 : rep1, 0, 0,
                            box[b].pos, NULL, sweep, sweeps_per_cycle, counters + b * C_N, 0,
                            0.0, NULL);
        }
        sweep += (uint64_t)sweeps_per_cycle;
        for (int e = 0; e < ex_per_cycle && rc == 0; ++e) {
            uint32_t w[4];
            gibbs_draw(&S, (uint32_t)step, P_MOVE, 0, 0, w);
            int src = (int)(w[0] >> 31);
            gibbs_exchange(&S, (uint32_t)step, box, g, counters + src * C_N);
            ++step;
        }
    }
    n[0] = box[0].n;
    n[1] = box[1].n;
    sim_free(&S);
    return rc;
}

/* Acceptance count of one fixed exchange: slot i of box src (0 or 1) to the
 * position xn of the other box, over n_rep independent steps step0 ...
 * (Gibbs test included).  Used to check detailed balance directly. */
long oracle_gibbs_acceptance(double diameter, double q, double n_r, int n_trial, uint64_t seed,
                             uint32_t rep0, double L0, double L1, int n0, int n1,
                             const double *pos0, const double *pos1, int src, int i,
                             const double *xn, uint64_t step0, long n_rep, uint64_t *g)
{
    if (!pos0 || !pos1 || !xn || !g || src < 0 || src > 1 || n_rep < 0) return -1;
    int ns = src == 0 ? n0 : n1;
    if (i < 0 || i >= ns) return -1;
    osim S;
    double sp[1] = {diameter};
    if (sim_init(&S, 1, L0, SHAPE_SPHERE, sp, 1, q, n_r, n_trial, 0, 0, 0.0, 0.0, 0.0, 1.0,
                 seed, rep0, 0, 1) != 0)
        return -1;
    obox box[2] = {{n0, L0, (double *)pos0}, {n1, L1, (double *)pos1}};
    uint64_t cnt[C_N] = {0};
    long acc = 0;
    for (long r = 0; r < n_rep; ++r)
        acc += gibbs_accept(&S, (uint32_t)(step0 + (uint64_t)r), &box[src], i, &box[1 - src], xn,
                            g, cnt);
    sim_free(&S);
    return acc;
}
