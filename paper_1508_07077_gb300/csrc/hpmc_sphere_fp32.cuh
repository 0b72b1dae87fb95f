// FP32 form of a colour phase for hard spheres, with a certified margin.
//
// Every distance test of the FP64 specification, `r2 < T`, is first taken in
// FP32 on cell-relative coordinates.  m_r2 bounds |r2_fp32 - r2_fp64| plus the
// rounding of T (derived on the host from the cell width, R_s and d_max); a
// test with |r2_fp32 - T| <= m_r2 is re-taken exactly as the FP64
// specification states.  Hence every decision equals the FP64 decision, and
// positions are still accumulated in FP64.  The exact re-takes are rare; they
// recompute the FP64 quantities from global memory rather than keep them live.
#pragma once

#include "hpmc_common.cuh"
#include "hpmc_sphere_fp64.cuh"

namespace hpmc {

// --- exact FP64 re-takes, as the specification states them -----------------
//
// They run rarely and out of line (behind warp votes), and recompute what
// they need: the move words are re-drawn and FP64 positions re-read.  Moves
// accepted by this CTA are committed to FP64 only when the CTA finishes, so a
// colloid of the list acc[0..nacc) is at its moved position.

// Exact FP64 position of colloid j after its move of this sweep: computed
// once per sweep, one thread per colloid, by the cell-list kernel (GB300's
// FP64 issue is slow, and a single-lane FP64 sequence costs a whole warp's
// time, so it is kept off the colour phases).
__device__ __forceinline__ double4 moved64(const SimParams &P, const Rep &R, uint32_t sweep, int j)
{
    (void)R;
    (void)sweep;
    return P.prop_pos[j];
}

__device__ __forceinline__ double4 pos_now(const SimParams &P, const Rep &R, uint32_t sweep, int j,
                                           const int *acc, int nacc)
{
    for (int a = 0; a < nacc; ++a)
        if (acc[a] == j) return moved64(P, R, sweep, j);
    return P.pos[j];
}

struct Move64 {
    double x0, x1, x2;  // new position, wrapped into [0, L)
    double o0, o1, o2;  // old position relative to the new one (minimum image)
};

__device__ __forceinline__ Move64 move64(const SimParams &P, const Rep &R, uint32_t sweep, int i)
{
    const double4 pi = P.pos[i];
    const double4 x = moved64(P, R, sweep, i);
    Move64 m;
    m.x0 = x.x;
    m.x1 = x.y;
    m.x2 = x.z;
    m.o0 = min_image(pi.x - m.x0, R.L, R.half_L);
    m.o1 = min_image(pi.y - m.x1, R.L, R.half_L);
    m.o2 = min_image(pi.z - m.x2, R.L, R.half_L);
    return m;
}

__device__ __forceinline__ void center64(const SimParams &P, const Rep &R, const Move64 &m, double4 pj,
                                         double &c0, double &c1, double &c2)
{
    c0 = min_image(pj.x - m.x0, R.L, R.half_L);
    c1 = min_image(pj.y - m.x1, R.L, R.half_L);
    c2 = min_image(pj.z - m.x2, R.L, R.half_L);
}

__device__ __noinline__ bool exact_cell_exit(const SimParams &P, const Rep &R, const Sched *S,
                                             uint32_t sweep, int i, int cx, int cy, int cz)
{
    const double4 x = moved64(P, R, sweep, i);
    return cell_coord(x.x, S->sigma[0], R.L, R.w, R.nc) != cx ||
           cell_coord(x.y, S->sigma[1], R.L, R.w, R.nc) != cy ||
           cell_coord(x.z, S->sigma[2], R.L, R.w, R.nc) != cz;
}

// colloid i at its new position overlaps colloid j
__device__ __noinline__ bool exact_pair(const SimParams &P, const Rep &R, uint32_t sweep, int i, int j,
                                        const int *acc, int nacc)
{
    const Move64 m = move64(P, R, sweep, i);
    double c0, c1, c2;
    center64(P, R, m, pos_now(P, R, sweep, j, acc, nacc), c0, c1, c2);
    return norm2(c0, c1, c2) < R.contact2;
}

// FP64 coordinates of a point from its Philox words: half < 0, one point per
// call (R_s s11 of words 0..2: CB trials, the soft interaction's depletants);
// half 0 or 1, that half of a paired call (the hard depletant streams).
__device__ __forceinline__ void point64(const Rep &R, uint4 w, int half, double &e0, double &e1,
                                        double &e2)
{
    if (half < 0) {
        e0 = R.R_s * s11(w.x);
        e1 = R.R_s * s11(w.y);
        e2 = R.R_s * s11(w.z);
    } else {
        const uint3 a = paired_fields(w, (uint32_t)half);
        e0 = R.R_s * s21(a.x);
        e1 = R.R_s * s21(a.y);
        e2 = R.R_s * s21(a.z);
    }
}

__device__ __noinline__ bool exact_ball(const SimParams &P, const Rep &R, uint4 w, int half = -1)
{
    double e0, e1, e2;
    point64(R, w, half, e0, e1, e2);
    return norm2(e0, e1, e2) < R.R_s2;
}

// Exact test of a depletant point against one colloid.
//   what 0: point e (around the new reference point) vs the old pose
//   what 1: forward CB trial y = o + e (around the old reference point) vs the new pose
//   what 2: point e vs neighbour j
//   what 3: forward CB trial y = o + e vs neighbour j
// e: the point of words w (half as in point64): a circumsphere point (a
// depletant with the circumsphere V_0, or a CB trial).
__device__ __noinline__ bool exact_dep(const SimParams &P, const Rep &R, uint32_t sweep, int i, uint4 w, int what,
                                       int j, const int *acc, int nacc, int half = -1)
{
    const Move64 m = move64(P, R, sweep, i);
    double e0, e1, e2;
    point64(R, w, half, e0, e1, e2);
    double v0 = e0, v1 = e1, v2 = e2;
    if (what == 1 || what == 3) {
        v0 = m.o0 + e0;
        v1 = m.o1 + e1;
        v2 = m.o2 + e2;
    }
    if (what == 0) return SphereFP64::dep(R, v0 - m.o0, v1 - m.o1, v2 - m.o2);
    if (what == 1) return SphereFP64::dep(R, v0, v1, v2);
    double c0, c1, c2;
    center64(P, R, m, pos_now(P, R, sweep, j, acc, nacc), c0, c1, c2);
    return SphereFP64::dep(R, v0 - c0, v1 - c1, v2 - c2);
}

// Exact FP64 coordinates of attempt w of colloid i's depletant stream with
// the shell V_0 (a point of the level of i's move).
__device__ __noinline__ double3 shell_dep_point64(const Rep &R, uint32_t sweep, int i, uint4 w)
{
    const uint4 wm = draw(R.key0, R.key1, sweep, (uint32_t)(i - R.off), kPMove, 0, 0);
    double3 e;
    (void)shell_point64(R, shell_level(wm.x, wm.y, wm.z), w, e.x, e.y, e.z);
    return e;
}

// The same tests for a depletant of the shell V_0 (attempt w of colloid i's
// stream): what 0: vs the old pose;  what 4: vs the new pose
__device__ __noinline__ bool exact_dep_shell(const SimParams &P, const Rep &R, uint32_t sweep, int i, uint4 w,
                                             int what)
{
    const double3 e = shell_dep_point64(R, sweep, i, w);
    if (what == 4) return SphereFP64::dep(R, e.x, e.y, e.z);
    const Move64 m = move64(P, R, sweep, i);
    return SphereFP64::dep(R, e.x - m.o0, e.y - m.o1, e.z - m.o2);
}

// A lens point (attempt t of the depletant stream) free of every neighbour?
// (hard interactions: the shell's own points, else the paired stream)
__device__ __noinline__ bool exact_free_nb(const SimParams &P, const Rep &R, uint32_t sweep, int i, uint32_t t,
                                           const float4 *nb, int nnb, const int *acc, int nacc)
{
    double e0, e1, e2;
    if (R.v0_shell) {
        const uint4 w = draw(R.key0, R.key1, sweep, (uint32_t)(i - R.off), kPDep, 0, t);
        const double3 e = shell_dep_point64(R, sweep, i, w);
        e0 = e.x;
        e1 = e.y;
        e2 = e.z;
    } else {
        paired_point64(R.key0, R.key1, R.R_s, sweep, (uint32_t)(i - R.off), t, e0, e1, e2);
    }
    const Move64 m = move64(P, R, sweep, i);
    for (int a = 0; a < nnb; ++a) {
        double c0, c1, c2;
        center64(P, R, m, pos_now(P, R, sweep, __float_as_int(nb[a].w), acc, nacc), c0, c1, c2);
        if (SphereFP64::dep(R, e0 - c0, e1 - c1, e2 - c2)) return false;
    }
    return true;
}

// Soft interaction, FP32 form.  hertz32: u(r) = eps (1 - r/s)^(5/2) from r^2
// in FP32.  soft_may_block32: false when the point (FP32 image e,
// displacement image o = old - new, attempt word w) certainly does not
// block, by either of the FP64 statement's early exits (r_new >= r_old;
// u01(w_3) >= e^-u_old - e^-u_new) taken outside the bands derived with the
// Rep; true when it may (the lens keeps it).
__device__ __forceinline__ float hertz32(const Rep &R, float r2)
{
    const float t = 1.0f - __fsqrt_rn(r2) * R.soft_inv_s32;
    return t > 0.0f ? R.soft_eps32 * ((t * t) * __fsqrt_rn(t)) : 0.0f;
}

__device__ __forceinline__ bool soft_may_block32(const Rep &R, uint32_t w3, float e0, float e1, float e2,
                                                 float o0, float o1, float o2)
{
    const float r2n = norm2f(e0, e1, e2);
    const float r2o = norm2f(e0 - o0, e1 - o1, e2 - o2);
    if (r2n - r2o > R.soft_r2band) return false;
    const float d = expf(-hertz32(R, r2o)) - expf(-hertz32(R, r2n));
    const float v = __uint2float_rn(w3) * 0x1p-32f;
    return !(v - d > R.soft_vband);
}

// Soft interaction: the FP64 statement for lens point t of colloid i's
// move (the FP32 test was inside its band): the early exits, then the other
// colloids' energies at the point summed in ascending index (nb: the
// neighbours within reach, any order; those out of range add 0), then
// u01(w_3) < e^-U (e^-u_old - e^-u_new).
__device__ __noinline__ bool exact_soft_nb(const SimParams &P, const Rep &R, uint32_t sweep, int i, uint32_t t,
                                           const float4 *nb, int nnb, const int *acc, int nacc)
{
    const uint4 w = draw(R.key0, R.key1, sweep, (uint32_t)(i - R.off), kPDep, 0, t);
    const double e0 = R.R_s * s11(w.x), e1 = R.R_s * s11(w.y), e2 = R.R_s * s11(w.z);
    const Move64 m = move64(P, R, sweep, i);
    const double u0 = e0 - m.o0, u1 = e1 - m.o1, u2 = e2 - m.o2;
    const double r2n = norm2(e0, e1, e2), r2o = norm2(u0, u1, u2);
    if (!(r2n < r2o)) return false;
    const double e_new = exp_neg_spec(hertz_spec(R, r2n));
    const double e_old = exp_neg_spec(hertz_spec(R, r2o));
    if (!(e_old > e_new)) return false;
    const double v = u01(w.w);
    if (!(v < e_old - e_new)) return false;
    double U = 0.0;
    int last = -1;
    for (int a = 0; a < nnb; ++a) {
        int j = 0x7FFFFFFF;   // the next index in ascending order
        for (int b = 0; b < nnb; ++b) {
            const int jb = __float_as_int(nb[b].w);
            if (jb > last && jb < j) j = jb;
        }
        last = j;
        double c0, c1, c2;
        center64(P, R, m, pos_now(P, R, sweep, j, acc, nacc), c0, c1, c2);
        U = U + hertz_spec(R, norm2(e0 - c0, e1 - c1, e2 - c2));
    }
    return v < exp_neg_spec(U) * (e_old - e_new);
}

// Soft interaction in FP32: does lens point t (FP32 point e relative to the
// new position, displacement image o = old - new) block?  1 certainly, 0
// certainly not, -1 inside the band (the FP64 statement decides).  nb: the
// neighbours' FP32 offsets from the new position.
__device__ __forceinline__ int soft_cls32(const Rep &R, uint32_t sweep, uint32_t tag, uint32_t t, float e0,
                                          float e1, float e2, float o0, float o1, float o2,
                                          const float4 *nb, int nnb)
{
    float U = 0.0f;
    int n_in = 0;
    const float reach = R.T_s32 * 1.001f;
    for (int b = 0; b < nnb; ++b) {
        const float4 d = nb[b];
        const float r2 = norm2f(e0 - d.x, e1 - d.y, e2 - d.z);
        if (r2 < reach) {
            ++n_in;
            U += hertz32(R, r2);
        }
    }
    const float dd = expf(-hertz32(R, norm2f(e0 - o0, e1 - o1, e2 - o2))) -
                     expf(-hertz32(R, norm2f(e0, e1, e2)));
    const uint4 w = draw(R.key0, R.key1, sweep, tag, kPDep, 0, t);
    const float v = __uint2float_rn(w.w) * 0x1p-32f;
    const float b = expf(-U) * dd;
    const float band = R.soft_bband + 2.0f * (float)n_in * (R.soft_du_nb + 0x1p-24f * U);
    return v < b - band ? 1 : (v > b + band ? 0 : -1);
}

// Shell attempt decided in FP64 (the FP32 test was inside its margin):
// returns acceptance and the point rounded to float.
__device__ __noinline__ bool exact_shell_pt(const Rep &R, int lvl, uint4 w, float &e0, float &e1, float &e2)
{
    double d0, d1, d2;
    const bool in = shell_point64(R, lvl, w, d0, d1, d2);
    e0 = (float)d0;
    e1 = (float)d1;
    e2 = (float)d2;
    return in;
}

// Shell attempt in FP32 (the acceptance |v|^6 R_s^4 < r^4 and the point
// e = v r / |v|): 1 accepted and e set, 0 rejected, -1 undecided in FP32.
// Error bounds, u = 2^-24, against the FP64 values the specification
// defines: v_d = float(w_d - 2^31) 2^-31 errs by <= u |v_d| + 2^-31, so for
// |v| >= 2^-7 the FP32 |v|^2 errs by <= 12 u |v|^2 (relative); r =
// fma(h, float(w_3) 2^-32, R_in) errs by <= 5 u R_s.  Then |A32 - A| <=
// 3 * 12 u A + 5 u A (A = |v|^6 R_s^4, five roundings) and |B32 - B| <=
// 4 r^3 (5 u R_s) + 3 u B (B = r^4), and the decision is certain when B - A
// exceeds twice their sum.  The point then errs by <= 16 u R_s per component
// (direction 2 u r, radius 5 u R_s, |v|^2 in the scale 6 u r, sqrt, division
// and product 3 u r).  |v| < 2^-7 (probability 2^-21) is left to FP64.
__device__ __forceinline__ int shell_point32(const Rep &R, float rin, float h, uint4 w, float &e0, float &e1,
                                             float &e2, float &r_out)
{
    constexpr float u = 0x1p-24f;
    const float v0 = __int2float_rn((int)(w.x ^ 0x80000000u)) * 0x1p-31f;
    const float v1 = __int2float_rn((int)(w.y ^ 0x80000000u)) * 0x1p-31f;
    const float v2 = __int2float_rn((int)(w.z ^ 0x80000000u)) * 0x1p-31f;
    const float p2 = norm2f(v0, v1, v2);
    const float r = __fmaf_rn(h, __uint2float_rn(w.w) * 0x1p-32f, rin);
    r_out = r;
    const float r2 = r * r;
    const float A = ((p2 * p2) * p2) * R.R_s4_32;
    const float B = r2 * r2;
    const float err = 2.0f * ((41.0f * u) * A + (20.0f * u) * R.R_s32 * (r * r2) + (3.0f * u) * B) +
                      R.shell_band * B;
    if (p2 < 0x1p-14f) return -1;
    const float diff = B - A;
    if (diff < -err) return 0;
    if (!(diff > err)) return -1;
    const float sc = __fdiv_rn(r, __fsqrt_rn(p2));
    e0 = v0 * sc;
    e1 = v1 * sc;
    e2 = v2 * sc;
    return 1;
}

// --- FP32 tests with exact fallback -----------------------------------------

// Is v (FP32, relative to the new reference point) free of every neighbour?
// kind 2: v is a point e; kind 3: v is a forward trial o + e.
__device__ __forceinline__ bool free_nb32(const SimParams &P, const Rep &R, float v0, float v1, float v2,
                                          const float4 *nb, int nnb, uint32_t sweep, int i,
                                          uint4 w, int kind, const int *acc, int nacc,
                                          uint32_t &rck)
{
    for (int a = 0; a < nnb; ++a) {
        const float4 d = nb[a];
        const int t = tri(norm2f(v0 - d.x, v1 - d.y, v2 - d.z), R.T_dep32, R.m_r2);
        if constexpr (kChecked) {
            // a decision taken as certain, against the FP64 statement
            if (t != -1)
                (void)HPMC_CHECK_FAILS(
                    P, exact_dep(P, R, sweep, i, w, kind, __float_as_int(d.w), acc, nacc) == (t == 1), 16);
        }
        if (t == 1) return false;
        if (t == -1) {
            ++rck;
            if (exact_dep(P, R, sweep, i, w, kind, __float_as_int(d.w), acc, nacc)) return false;
        }
    }
    return true;
}

struct CbResult32 {
    double f;
    uint32_t fwd_ok, rev_ok, caps, rck;
};

// CB factor of one blocking depletant k (Sec. III.D, Eq. 12), FP32 form,
// computed by a whole warp (all 32 lanes call it with the same k).  The
// trials of a direction are the first n_fwd (n_rev) attempts of the stream
// (purpose, k) that fall inside the sampling ball: lanes take consecutive
// attempts, a ballot ranks the in-ball ones, and the lanes holding trials
// test them.  For spheres "overlaps the pose the ball is centred on" is the
// ball test itself.  Returns the same values in every lane except rck (the
// lane's own FP64 re-takes).
__device__ __noinline__ CbResult32 cb_factor_warp32(const SimParams &P, const Rep &R, uint32_t sweep, int i,
                                                    uint32_t k, float o0, float o1, float o2,
                                                    const float4 *nb, int nnb, const int *acc,
                                                    int nacc)
{
    CbResult32 r = {0.0, 0u, 0u, 0u, 0u};
    const uint32_t tag = (uint32_t)(i - R.off);
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    for (int dir = 0; dir < 2; ++dir) {
        const bool fwd = dir == 0;
        const int n_want = fwd ? R.n_trial : R.n_trial - 1;
        const uint32_t purpose = fwd ? kPCbFwd : kPCbRev;
        const uint32_t t_max = 64u * (uint32_t)(n_want + 1);
        int found = 0, ok = 0;
        for (uint32_t t0 = 0; found < n_want && t0 < t_max; t0 += 32u) {
            const uint32_t t = t0 + (threadIdx.x & 31);
            uint4 w = make_uint4(0u, 0u, 0u, 0u);
            float e0 = 0.f, e1 = 0.f, e2 = 0.f;
            int in = 0;
            if (t < t_max) {
                w = draw(R.key0, R.key1, sweep, tag, purpose, k, t);
                e0 = coord32(w.x, R.R_s32);
                e1 = coord32(w.y, R.R_s32);
                e2 = coord32(w.z, R.R_s32);
                in = tri(norm2f(e0, e1, e2), R.T_s32, R.m_r2);
                if constexpr (kChecked) {
                    if (in != -1) (void)HPMC_CHECK_FAILS(P, exact_ball(P, R, w) == (in == 1), 11);
                }
                if (in == -1) {
                    ++r.rck;
                    in = exact_ball(P, R, w) ? 1 : 0;
                }
            }
            const unsigned bal = __ballot_sync(kFull, in != 0);
            bool good = false;
            if (in && found + __popc(bal & lt) < n_want) {
                if (fwd) {
                    // forward trial around the old pose: must miss the new pose
                    const float y0 = o0 + e0, y1 = o1 + e1, y2 = o2 + e2;
                    int tn = tri(norm2f(y0, y1, y2), R.T_dep32, R.m_r2);
                    if constexpr (kChecked) {
                        if (tn != -1)
                            (void)HPMC_CHECK_FAILS(P, exact_dep(P, R, sweep, i, w, 1, 0, acc, nacc) == (tn == 1), 12);
                    }
                    if (tn == -1) {
                        ++r.rck;
                        tn = exact_dep(P, R, sweep, i, w, 1, 0, acc, nacc) ? 1 : 0;
                    }
                    good = !tn && free_nb32(P, R, y0, y1, y2, nb, nnb, sweep, i, w, 3, acc, nacc, r.rck);
                } else {
                    // reverse trial around the new pose: must miss the old pose
                    int to = tri(norm2f(e0 - o0, e1 - o1, e2 - o2), R.T_dep32, R.m_r2);
                    if constexpr (kChecked) {
                        if (to != -1)
                            (void)HPMC_CHECK_FAILS(P, exact_dep(P, R, sweep, i, w, 0, 0, acc, nacc) == (to == 1), 12);
                    }
                    if (to == -1) {
                        ++r.rck;
                        to = exact_dep(P, R, sweep, i, w, 0, 0, acc, nacc) ? 1 : 0;
                    }
                    good = !to && free_nb32(P, R, e0, e1, e2, nb, nnb, sweep, i, w, 2, acc, nacc, r.rck);
                }
            }
            ok += __popc(__ballot_sync(kFull, good));
            found += min(__popc(bal), n_want - found);
        }
        if (found < n_want) ++r.caps;
        if (fwd) r.fwd_ok = (uint32_t)ok;
        else r.rev_ok = (uint32_t)ok;
    }
    r.f = (double)r.fwd_ok / (double)(r.rev_ok + 1);
    return r;
}

// Shared scratch of the per-move depletant evaluation; f and k point into the
// dynamic shared memory (blockDim doubles, then blockDim ints).
struct DepShared {
    double *f;
    int *k;
    int warp[kMaxThreads / 32];
    unsigned mask[kMaxThreads / 32];
    int kmin, flag;
};

// Outcome of one move's depletants (values valid in thread 0 for W and the
// counters marked "thread 0"; rejected is block-uniform).
struct DepOutcome {
    double W;
    int rejected, nblock;
    uint32_t eval, block, cap, rck, fwd, rev;  // eval, block: thread 0
};

// CB bookkeeping of one pass: slots in ascending depletant index, product in
// order, stop at a zero factor.  Called by every thread; has: the thread's
// slot holds a factor f (zero: f is 0) of depletant k.
__device__ __forceinline__ bool cb_pass(DepShared &sh, int tid, int nslots, bool has, double f,
                                        bool zero, int k, DepOutcome &o, int eval_if_full)
{
    const unsigned bal = __ballot_sync(kFull, has);
    if ((tid & 31) == 0) sh.mask[tid >> 5] = bal;
    if (has) {
        sh.f[tid] = f;
        sh.k[tid] = zero ? -1 - k : k;
    }
    __syncthreads();
    if (tid == 0) {
        int n_fact = 0;
        const int kz = cb_walk(sh.mask, (nslots + 31) >> 5, sh.k, sh.f, o.W, n_fact);
        o.nblock += n_fact;
        o.block += (uint32_t)n_fact;
        if (kz >= 0) o.eval += (uint32_t)(kz + 1);
        else if (eval_if_full >= 0) o.eval += (uint32_t)eval_if_full;
        sh.flag = kz >= 0 ? 1 : 0;
    }
    __syncthreads();
    return sh.flag != 0;
}

// ---------------------------------------------------------------------------
// Depletant lens lists (Sec. III.B-C).  Everything about a move's depletants
// that does not involve other colloids is fixed by the move's own random
// streams: the proposal, N_p, the points of the attempt stream, "inside the
// new pose's circumsphere" (= overlaps the new pose, for spheres) and
// "overlaps the old pose".  Only the points left after those tests, the lens
// of the move, can block it, and only they need the neighbours, which the
// colour phases test in order.  A list holds at most N_p <= (Poisson table
// length) points, the capacity it is allocated with, so it cannot overflow.
// ---------------------------------------------------------------------------
// One move's lens list, warp-cooperative (all 32 lanes call it).  V0: the
// depletant region; 0 the circumsphere, 2 the cube around it (every attempt
// a depletant).  (The shell, 1, has its own kernel below.)  Writes the FP32
// displacement to *mv (lane 0), and the lens points, in depletant order, to
// sdst[slot] for slot < room and to gdst[slot] beyond (gdst is the move's
// list of capacity lens_cap).  Returns (N_p, depletants obtained from the
// stream, lens points, FP64 re-takes), the same in every lane.  SOFT: the
// soft interaction keeps the points neither of whose early exits is certain
// in FP32 (instead of those outside the old pose).
// lens_of_move for hard interactions with the circumsphere (V0 = 0) or cube
// (V0 = 2) V_0: the paired depletant stream.  A pass covers a block of 64
// attempts: each lane draws one Philox call and the warp takes the first
// halves (attempts t0 + lane), then the second halves (t0 + 32 + lane), each
// sub-pass ranked by ballot as the one-point form ranks its passes.  Same
// output as lens_of_move.
template <int V0>
__device__ __forceinline__ int4 lens_of_move_paired(const SimParams &P, const Rep &R, int g,
                                                    uint32_t sweep, float4 *mv, float4 *sdst,
                                                    int room, float4 *gdst)
{
    constexpr bool CUBE = V0 == 2;
    const int lane = threadIdx.x & 31;
    const int i = g;
    const uint32_t tag = (uint32_t)(g - R.off);
    const RoundKeys K = round_keys(R.key0, R.key1);
    // the move's words (lane 0) and its Poisson words (lane 1) in one
    // evaluation of the generator, then shared
    const uint4 wl = philox_rk(make_uint4(sweep, tag, (lane == 1 ? kPPoisson : kPMove) << 24, 0u), K);
    const uint32_t wm0 = __shfl_sync(kFull, wl.x, 0), wm1 = __shfl_sync(kFull, wl.y, 0),
                   wm2 = __shfl_sync(kFull, wl.z, 0);
    const uint32_t wp0 = __shfl_sync(kFull, wl.x, 1), wp1 = __shfl_sync(kFull, wl.y, 1);
    const float D0 = coord32(wm0, R.d_max32);
    const float D1 = coord32(wm1, R.d_max32);
    const float D2 = coord32(wm2, R.d_max32);
    if (lane == 0) *mv = make_float4(D0, D1, D2, 0.0f);
    if (!R.has_dep) return make_int4(0, 0, 0, 0);
    uint32_t rck = 0;
    const float o0 = -D0, o1 = -D1, o2 = -D2;
    const int n_p = poisson_count(P.T + R.t_off, R.nF, u53_int(wp0, wp1), lane);
    const uint32_t t_max = 64u * (uint32_t)(n_p + 1);   // a multiple of 64: whole blocks
    const unsigned lt = (1u << lane) - 1u;
    uint32_t t0 = 0;
    int k0 = 0, m = 0;
    while (k0 < n_p && t0 < t_max) {
        const uint4 w = philox_rk(make_uint4(sweep, tag, kPDep << 24, (t0 >> 1) + (uint32_t)lane), K);
#pragma unroll 1
        for (int h = 0; h < 2 && k0 < n_p; ++h) {
            const uint32_t t = t0 + 32u * (uint32_t)h + (uint32_t)lane;
            const uint3 f = paired_fields(w, (uint32_t)h);
            const float e0 = s21f_bits(f.x) * R.R_s32, e1 = s21f_bits(f.y) * R.R_s32,
                        e2 = s21f_bits(f.z) * R.R_s32;
            if constexpr (!CUBE) {
                // the common case first: every decision certain and no lens
                // candidate (each point in the ball certainly overlaps the
                // old pose), where a sub-pass only counts its ball points
                const float r2 = norm2f(e0, e1, e2);
                const float r2o = norm2f(e0 - o0, e1 - o1, e2 - o2);
                const bool in_c = r2 < R.T_s32 - R.m_r2, out_c = r2 > R.T_s32 + R.m_r2;
                const bool ov_c = r2o < R.T_dep32 - R.m_r2;
                if (!__any_sync(kFull, !(in_c || out_c) || (in_c && !ov_c))) {
                    if constexpr (kChecked) {
                        // the decisions taken as certain, against the FP64
                        // statement: in the ball, and (in it) over the old pose
                        (void)HPMC_CHECK_FAILS(P, exact_ball(P, R, w, h) == in_c, 11);
                        if (in_c)
                            (void)HPMC_CHECK_FAILS(P, exact_dep(P, R, sweep, i, w, 0, 0, nullptr, 0, h), 12);
                    }
                    k0 += __popc(__ballot_sync(kFull, in_c));
                    continue;
                }
            }
            // in the sampling region (the ball; the cube takes every point)
            int in = CUBE ? 1 : tri(norm2f(e0, e1, e2), R.T_s32, R.m_r2);
            // overlaps the new pose (the cube's points only inside the ball;
            // for the ball it is the same test) and the old pose: 1 yes, 0
            // no, -1 within the margin; one vote for every uncertain decision
            int tn = CUBE ? tri(norm2f(e0, e1, e2), R.T_dep32, R.m_r2) : 1;
            int to = in != 0 && tn != 0 ? tri(norm2f(e0 - o0, e1 - o1, e2 - o2), R.T_dep32, R.m_r2)
                                        : 1;
            if constexpr (kChecked) {
                // every decision taken as certain, against the FP64 statement
                if (!CUBE && in != -1) (void)HPMC_CHECK_FAILS(P, exact_ball(P, R, w, h) == (in == 1), 11);
                if (CUBE && tn != -1) (void)HPMC_CHECK_FAILS(P, exact_ball(P, R, w, h) == (tn == 1), 11);
                if (in == 1 && tn == 1 && to != -1)
                    (void)HPMC_CHECK_FAILS(
                        P, exact_dep(P, R, sweep, i, w, 0, 0, nullptr, 0, h) == (to == 1), 12);
            }
            if (__any_sync(kFull, in == -1 || tn == -1 || to == -1)) {
                if (in == -1) {
                    ++rck;
                    in = exact_ball(P, R, w, h) ? 1 : 0;
                }
                if (CUBE && tn == -1) {
                    ++rck;
                    tn = exact_ball(P, R, w, h) ? 1 : 0;
                }
                if (to == -1 && in == 1 && tn == 1) {
                    ++rck;
                    to = exact_dep(P, R, sweep, i, w, 0, 0, nullptr, 0, h) ? 1 : 0;
                }
            }
            const unsigned bal = __ballot_sync(kFull, in == 1);
            // lens candidates are rare (a few per move against ~9 sub-passes):
            // their depletant index and list slot are ranked only in a
            // sub-pass that has one
            const bool cand = in == 1 && tn == 1 && to == 0;
            if (__any_sync(kFull, cand)) {
                const int k = k0 + __popc(bal & lt);
                const bool lens = cand && k < n_p;
                const unsigned lb = __ballot_sync(kFull, lens);
                const int slot = m + __popc(lb & lt);
                if (lens) {
                    const float4 v = make_float4(e0, e1, e2, __int_as_float((int)((t << 16) | (uint32_t)k)));
                    if (slot < room) sdst[slot] = v;
                    else if (slot < P.lens_cap) gdst[slot] = v;
                }
                m += __popc(lb);
            }
            k0 += __popc(bal);
        }
        t0 += 64u;
    }
    if (lane == 0 && m > P.lens_cap) atomicCAS(P.err, kErrNone, kErrCandCap);
    rck = __reduce_add_sync(kFull, rck);
    return make_int4(n_p, min(k0, n_p), min(m, P.lens_cap), (int)rck);
}

template <int V0, bool SOFT>
__device__ __forceinline__ int4 lens_of_move(const SimParams &P, const Rep &R, int g, uint32_t sweep, float4 *mv,
                                          float4 *sdst, int room, float4 *gdst)
{
    if constexpr (!SOFT) {
        return lens_of_move_paired<V0>(P, R, g, sweep, mv, sdst, room, gdst);
    } else {
        static_assert(V0 == 0 || V0 == 2, "circumsphere or cube");
        constexpr bool CUBE = V0 == 2;
        const int lane = threadIdx.x & 31;
        const uint32_t tag = (uint32_t)(g - R.off);
        const uint4 wm = draw(R.key0, R.key1, sweep, tag, kPMove, 0, 0);
        const float D0 = coord32(wm.x, R.d_max32);
        const float D1 = coord32(wm.y, R.d_max32);
        const float D2 = coord32(wm.z, R.d_max32);
        if (lane == 0) *mv = make_float4(D0, D1, D2, 0.0f);
        if (!R.has_dep) return make_int4(0, 0, 0, 0);
        uint32_t rck = 0;
        const float o0 = -D0, o1 = -D1, o2 = -D2;
        const uint4 wp = draw(R.key0, R.key1, sweep, tag, kPPoisson, 0, 0);
        const int n_p = poisson_count(P.T + R.t_off, R.nF, u53_int(wp.x, wp.y), lane);
        const uint32_t t_max = 64u * (uint32_t)(n_p + 1);
        const RoundKeys K = round_keys(R.key0, R.key1);
        const unsigned lt = (1u << lane) - 1u;
        uint32_t t0 = 0;
        int k0 = 0, m = 0, qn = 0;
        // The soft tests (the early exits' exponentials) dominate: a pass queues
        // its depletants (ball points of index k < N_p) in shared memory and the
        // tests run on full batches of 32 queued points, so every lane tests a
        // depletant; the queue is in depletant order, as the list needs.
        __shared__ float4 s_q[4][64];      // (e, (t << 16) | k)
        __shared__ uint32_t s_w3[4][64];   // the attempt's fourth word
        const int wq = (threadIdx.x >> 5) & 3;
        auto test_batch = [&](int nb) {
            const bool act = lane < nb;
            const float4 v = act ? s_q[wq][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            const uint32_t w3 = act ? s_w3[wq][lane] : 0u;
            // the points that may block (neither early exit of the FP64
            // statement certain in FP32); the phases decide them
            const bool lens = act && soft_may_block32(R, w3, v.x, v.y, v.z, o0, o1, o2);
            // (list slots are ranked only in a batch that has a lens point)
            if (__any_sync(kFull, lens)) {
                const unsigned lb = __ballot_sync(kFull, lens);
                const int slot = m + __popc(lb & lt);
                if (lens) {
                    if (slot < room) sdst[slot] = v;
                    else if (slot < P.lens_cap) gdst[slot] = v;
                }
                m += __popc(lb);
            }
        };
        while (k0 < n_p && t0 < t_max) {
            const uint32_t t = t0 + (uint32_t)lane;
            uint4 w = make_uint4(0, 0, 0, 0);
            float e0 = 0.f, e1 = 0.f, e2 = 0.f;
            int in = 0;
            if (t < t_max) {
                w = philox_rk(make_uint4(sweep, tag, kPDep << 24, t), K);
                e0 = coord32(w.x, R.R_s32);
                e1 = coord32(w.y, R.R_s32);
                e2 = coord32(w.z, R.R_s32);
                in = CUBE ? 1 : tri(norm2f(e0, e1, e2), R.T_s32, R.m_r2);
            }
            {
                const bool unsure = in == -1;
                if (__any_sync(kFull, unsure)) {
                    if (unsure) {
                        ++rck;
                        in = exact_ball(P, R, w) ? 1 : 0;
                    }
                }
            }
            const unsigned bal = __ballot_sync(kFull, in == 1);
            const int k = k0 + __popc(bal & lt);
            bool dep = in == 1 && k < n_p;
            if (CUBE) {
                // a cube point overlaps the new pose only inside the circumsphere
                int tn = dep ? tri(norm2f(e0, e1, e2), R.T_dep32, R.m_r2) : 1;
                const bool unsure = tn == -1;
                if (__any_sync(kFull, unsure)) {
                    if (unsure) {
                        ++rck;
                        tn = exact_ball(P, R, w) ? 1 : 0;
                    }
                }
                dep = dep && tn == 1;
            }
            const unsigned db = __ballot_sync(kFull, dep);
            if (dep) {
                const int qi = qn + __popc(db & lt);
                s_q[wq][qi] = make_float4(e0, e1, e2, __int_as_float((int)((t << 16) | (uint32_t)k)));
                s_w3[wq][qi] = w.w;
            }
            qn += __popc(db);
            k0 += __popc(bal);
            t0 += 32u;
            __syncwarp();
            if (qn >= 32) {
                test_batch(32);
                // the rest (fewer than 32) to the front of the queue
                const int rest = qn - 32;
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                uint32_t xw = 0u;
                __syncwarp();
                if (lane < rest) {
                    x = s_q[wq][32 + lane];
                    xw = s_w3[wq][32 + lane];
                }
                __syncwarp();
                if (lane < rest) {
                    s_q[wq][lane] = x;
                    s_w3[wq][lane] = xw;
                }
                __syncwarp();
                qn = rest;
            }
        }
        if (qn > 0) test_batch(qn);
        if (lane == 0 && m > P.lens_cap) atomicCAS(P.err, kErrNone, kErrCandCap);
        rck = __reduce_add_sync(kFull, rck);
        return make_int4(n_p, min(k0, n_p), min(m, P.lens_cap), (int)rck);
    }
}

// The lens lists of all moves of the sweep, one warp per colloid, filed under
// the colloids' bin slots (used when the colour phases do not build them
// themselves).
template <int V0, bool SOFT = false>
__global__ void __launch_bounds__(128, 8) k_lens_sphere_fp32(const __grid_constant__ SimParams P)
{
    __shared__ float4 s_mv[4];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int g = blockIdx.x * (blockDim.x >> 5) + wl;
    if (g >= P.n_total) return;
    // Launched with programmatic dependent launch behind the cell-list kernel:
    // the depletant work below needs nothing that kernel writes (the sweep
    // index is the counter the previous sweep advanced); only the bin slot
    // the results are filed under does, and it is read after pdl_wait().
    // (This kernel does not release its own successor early: the colour
    // phases read its results before they wait.)
    const int r = P.rep_of[g];
    const Rep &R = P.reps[r];
    if (g - R.off >= P.n_live[r]) return;   // a slot not in use (Gibbs pair)
    const uint32_t sweep = (uint32_t)(*P.sweep);
    float4 *out = P.lens + (size_t)g * P.lens_cap;
    const int4 h = lens_of_move<V0, SOFT>(P, R, g, sweep, &s_mv[wl], nullptr, 0, out);
    // file the header, the displacement and the first lens points under the
    // colloid's bin slot, where the colour phase reads them with the cell list
    __syncwarp();
    pdl_wait();
    int bp = P.binpos[g];
    if (HPMC_CHECK_FAILS(P, bp < P.n_cells * P.cap, 9)) bp = -1;
    if (bp >= 0) {
        if (lane == 0) {
            P.mv_bin[bp] = s_mv[wl];
            if (R.has_dep) P.hdr_bin[bp] = make_int4(h.x, h.y, h.z, 0);
        }
        if (lane < min(h.z, kLensInline)) P.lens_bin[(size_t)bp * kLensInline + lane] = out[lane];
    }
    if (lane == 0 && h.w) count_one(P, r, kRechecks, (unsigned long long)h.w);
}

// Shell V_0, one thread per colloid.  A shell holds few depletants (the
// level's thickness is of the order of the step size), so a warp per move
// would leave most lanes of its one pass idle and repeat the move's draws on
// every lane; here each thread walks its own attempt stream.  Same output
// contract as k_lens_sphere_fp32.
__device__ __forceinline__ int poisson_count1(const unsigned long long *T, int nF, unsigned long long m)
{
    int lo = 0, hi = nF;   // the table is non-decreasing: count = first index with T > m
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(T + mid) <= m) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(128, 4) k_lens_shell_fp32(const __grid_constant__ SimParams P)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.n_total) {
        pdl_wait();
        return;
    }
    const int r = P.rep_of[g];
    const Rep &R = P.reps[r];
    if (g - R.off >= P.n_live[r]) {   // a slot not in use (Gibbs pair)
        pdl_wait();
        return;
    }
    const int i = g;
    const uint32_t sweep = (uint32_t)(*P.sweep);
    const uint32_t tag = (uint32_t)(g - R.off);
    const uint4 wm = draw(R.key0, R.key1, sweep, tag, kPMove, 0, 0);
    const float D0 = coord32(wm.x, R.d_max32);
    const float D1 = coord32(wm.y, R.d_max32);
    const float D2 = coord32(wm.z, R.d_max32);
    if (!R.has_dep) {
        pdl_wait();
        const int bp = P.binpos[g];
        if (bp >= 0) P.mv_bin[bp] = make_float4(D0, D1, D2, 0.0f);
        return;
    }
    uint32_t rck = 0;
    const int lvl = shell_level(wm.x, wm.y, wm.z);
    const float rin32 = R.sh_rin32[lvl - 1], h32 = R.sh_h32[lvl - 1];
    const uint4 wp = draw(R.key0, R.key1, sweep, tag, kPPoisson, 0, 0);
    const int n_p = poisson_count1(P.T + R.t_off + (size_t)(lvl - 1) * (size_t)R.nF, R.nF,
                                   u53_int(wp.x, wp.y));
    const uint32_t t_max = 64u * (uint32_t)(n_p + 1);
    const RoundKeys K = round_keys(R.key0, R.key1);
    float4 *out = P.lens + (size_t)g * P.lens_cap;
    int k = 0, m = 0;
    for (uint32_t t = 0; k < n_p && t < t_max; ++t) {
        const uint4 w = philox_rk(make_uint4(sweep, tag, kPDep << 24, t), K);
        float e0 = 0.f, e1 = 0.f, e2 = 0.f, r32 = 0.f;
        int in = shell_point32(R, rin32, h32, w, e0, e1, e2, r32);
        if (in == -1) {
            ++rck;
            in = exact_shell_pt(R, lvl, w, e0, e1, e2) ? 1 : 0;
            r32 = R.R_s32;   // (no radius bound from the FP64 path)
        }
        if (!in) continue;
        const int kk = k++;
        // overlaps the new pose: certain when the radius is clear of R_s (r32
        // errs by <= 5u R_s, and |e|^2 in FP64 by a few 2^-53 relative, so
        // r < R_s (1 - 2^-18) - 5u R_s puts |e|^2 below R_s^2); else tested
        int tn = r32 < R.R_s32 * (1.0f - 0x1p-18f) ? 1 : tri(norm2f(e0, e1, e2), R.T_dep32, R.m_r2);
        if (tn == -1) {
            ++rck;
            tn = exact_dep_shell(P, R, sweep, i, w, 4) ? 1 : 0;
        }
        if (tn != 1) continue;
        int to = tri(norm2f(e0 + D0, e1 + D1, e2 + D2), R.T_dep32, R.m_r2);   // the old pose
        if (to == -1) {
            ++rck;
            to = exact_dep_shell(P, R, sweep, i, w, 0) ? 1 : 0;
        }
        if (to != 0) continue;
        if (m < P.lens_cap) out[m] = make_float4(e0, e1, e2, __int_as_float((int)((t << 16) | (uint32_t)kk)));
        ++m;
    }
    pdl_wait();
    const int bp = P.binpos[g];
    if (bp >= 0) {
        P.mv_bin[bp] = make_float4(D0, D1, D2, 0.0f);
        P.hdr_bin[bp] = make_int4(n_p, min(k, n_p), min(m, P.lens_cap), 0);
        const int ni = min(m, kLensInline);
        for (int a = 0; a < ni; ++a) P.lens_bin[(size_t)bp * kLensInline + a] = out[a];
    }
    if (m > P.lens_cap) atomicCAS(P.err, kErrNone, kErrCandCap);
    // recheck count, summed over the lanes of the same replica
    const unsigned peers = __match_any_sync(__activemask(), r);
    rck = __reduce_add_sync(peers, rck);
    if ((threadIdx.x & 31) == __ffs(peers) - 1 && rck) count_one(P, r, kRechecks, (unsigned long long)rck);
}

constexpr int kMaxLensCTA = 64;    // lens points of one cell staged in shared memory (more: read
                                   // from global memory)
// neighbours within reach of a depletant, per cell-bin capacity: the widest
// cells (large depletants) get the larger list
__host__ __device__ constexpr int max_nb(int cap) { return cap >= kMaxCellCap ? 128 : 64; }

// CTA-wide barrier / OR, reduced to warp operations when the CTA is one warp.
template <bool WARP>
__device__ __forceinline__ void cta_sync()
{
    if (WARP) __syncwarp();
    else __syncthreads();
}

template <bool WARP>
__device__ __forceinline__ bool cta_any(bool p)
{
    if (WARP) return __any_sync(kFull, p);
    return __syncthreads_or(p) != 0;
}

// ---------------------------------------------------------------------------
// Per-cell work of a colour phase (FP32 form), shared by the per-phase kernel
// and the persistent sweep kernel.  The CTA stages its 27-cell neighbourhood,
// the cell's colloids (ascending index), their displacements and their lens
// points in shared memory, then moves the colloids one after another.
// tk: the task-table entry of the cell (global cell, replica, coordinates,
// n_c and count parity); the cell is not empty.  CB: configurational bias on
// (n_trial > 0) or off.  WARP: the CTA is a single warp (barriers become warp
// operations).  CAP: capacity of a cell bin (the cell list's stride).
// PERSIST: instead of waiting for the whole previous phase (programmatic
// dependent launch), wait only for the non-empty stencil cells of earlier
// phases of this sweep, through their readiness counters (epoch: the value a
// counter holds once its cell is done in this sweep); if a wait runs out,
// record HPMC's timeout error and return without moving (the caller still
// publishes the cell as done, so no other wait depends on it).
// ---------------------------------------------------------------------------
template <bool CB, bool WARP, int CAP, bool SOFT, bool PERSIST>
__device__ __forceinline__ void phase_cell(const SimParams &P, int phase, int4 tk, uint32_t epoch)
{
    __shared__ float4 s_cpos[cand_cap(CAP)];  // candidates relative to this cell's origin; index in .w
    __shared__ float4 s_nb[max_nb(CAP)];      // neighbours relative to the new position; index in .w
    __shared__ float4 s_lens[kMaxLensCTA];
    __shared__ int4 s_hdr[CAP];                  // own cell, bin order
    __shared__ float4 s_mv[CAP];
    __shared__ float4 s_lin[2][kLensInline];     // inline lens points of bin slots 0, 1
    __shared__ int s_tmp_i[CAP], s_tmp_slot[CAP];
    __shared__ int s_own[CAP], s_own_slot[CAP], s_own_bin[CAP];
    __shared__ int s_loff[CAP], s_accl[CAP];
    __shared__ DepShared sh;
    __shared__ int s_ncand, s_nnb, s_acc, s_nacc;
    extern __shared__ double s_dyn[];

    const int tid = threadIdx.x, nthr = WARP ? 32 : (int)blockDim.x;
    const int lane = tid & 31;
    const unsigned lt = (1u << lane) - 1u;
    if (tid == 0) {
        sh.f = s_dyn;
        sh.k = (int *)(s_dyn + nthr);
    }
    const int cell = tk.x, r = tk.y;
    const int cx = tk.z & 1023, cy = (tk.z >> 10) & 1023, cz = tk.z >> 20;
    const int nc = tk.w & 0xFFFF, par = tk.w >> 16;
    const int ns = nc == 2 ? 2 : 3, n_st = ns * ns * ns;
    const int t_own = ns == 3 ? 13 : cx + 2 * cy + 4 * cz;
    const int cell_off = cell - (cx + nc * (cy + nc * cz));
    const int *count = P.count[par];
    // the replica's FP32 parameters, loaded now so that their latency overlaps
    // the stencil loads below
    const Rep &R = P.reps[r];
    const float w32 = R.w32, L32 = R.L32, half_L32 = R.half_L32, m_r2 = R.m_r2,
                m_cell = R.m_cell, nb_cut2 = R.nb_cut2_32, T_dep = R.T_dep32,
                T_contact = R.T_contact32;
    const int has_dep = R.has_dep;

    // Loads, most of them before the wait for the neighbours (everything
    // about the own cell is fixed for the sweep or written only by this CTA):
    // first load, every stencil cell's population (lanes 0..26) and, on spare
    // lanes, the own cell's first two bin entries, displacements, headers and
    // inline lens points (speculatively: most cells hold at most two
    // colloids); a second load (only for more colloids) the rest of the own cell's
    // slots, one lane each; after the wait one round for the neighbour cells'
    // entries (up to four per cell at once).
    int c_nb = 0, m_nb = 0, dx = 0, dy = 0, dz = 0;
    const size_t own0 = bin_at(P, cell, 0), own1 = bin_at(P, cell, 1);
    float4 p_a = make_float4(0.f, 0.f, 0.f, 0.f), p_b = p_a;
    int4 h_a = make_int4(0, 0, 0, 0), h_b = h_a;
    if (tid < n_st) {
        c_nb = stencil_cell_nc(nc, cell_off, tid, cx, cy, cz, dx, dy, dz);
        if (HPMC_CHECK_FAILS(P, c_nb >= cell_off && c_nb < cell_off + nc * nc * nc &&
                                    c_nb < P.n_cells, 1))
            c_nb = cell;
        m_nb = min(count[c_nb], P.cap);
    } else if (tid == 27) {
        p_a = P.bins[own0];
        p_b = P.bins[own1];
    } else if (tid == 28) {
        p_a = P.mv_bin[own0];
        p_b = P.mv_bin[own1];
        h_a = P.hdr_bin[own0];
        h_b = P.hdr_bin[own1];
    } else if (tid == 29 || tid == 30) {
        const float4 *src = P.lens_bin + (tid == 29 ? own0 : own1) * kLensInline;
#pragma unroll
        for (int j = 0; j < kLensInline; ++j) s_lin[tid - 29][j] = src[j];
    }
    const Sched *S = P.sched + r;
    int n_own = 0, M = 0, base = 0, base_own = 0;
    if (tid < 32) {
        n_own = __shfl_sync(kFull, m_nb, t_own);
        int incl = m_nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        base = incl - m_nb;
        M = __shfl_sync(kFull, incl, 31);
        base_own = __shfl_sync(kFull, base, t_own);
        if (!WARP && tid == 0) {
            s_ncand = M;
            s_nacc = n_own;
            s_acc = base_own;
        }
    }
    if (!WARP) {
        __syncthreads();
        M = s_ncand;
        n_own = s_nacc;
        base_own = s_acc;
        __syncthreads();
    }
    if (n_own == 0) return;
    if (M > cand_cap(CAP)) {
        if (tid == 0) atomicCAS(P.err, kErrNone, kErrCandCap);
        return;
    }
    // the own cell's slots (its candidates, in bin order) and their move data
    if (tid == 27) {
        s_cpos[base_own] = p_a;
        s_tmp_i[0] = __float_as_int(p_a.w);
        s_tmp_slot[0] = base_own;
        if (n_own > 1) {
            s_cpos[base_own + 1] = p_b;
            s_tmp_i[1] = __float_as_int(p_b.w);
            s_tmp_slot[1] = base_own + 1;
        }
    } else if (tid == 28) {
        s_mv[0] = p_a;
        s_hdr[0] = h_a;
        s_mv[1] = p_b;
        s_hdr[1] = h_b;
    }
    for (int q = 2 + tid; q < n_own; q += nthr) {
        const size_t oq = bin_at(P, cell, q);
        const float4 e = P.bins[oq];
        s_mv[q] = P.mv_bin[oq];
        s_hdr[q] = P.hdr_bin[oq];
        s_cpos[base_own + q] = e;
        s_tmp_i[q] = __float_as_int(e.w);
        s_tmp_slot[q] = base_own + q;
    }
    if (tid == 0) s_nacc = 0;
    cta_sync<WARP>();
    // the cell's colloids in ascending index (the order they move in), and
    // where each one's lens points go in shared memory (bin order)
    for (int q = tid; q < n_own; q += nthr) {
        const int v = s_tmp_i[q];
        int rk = 0;
        for (int u = 0; u < n_own; ++u) rk += s_tmp_i[u] < v ? 1 : 0;
        if (HPMC_CHECK_FAILS(P, rk < n_own && n_own <= CAP, 6)) continue;
        s_own[rk] = v;
        s_own_slot[rk] = s_tmp_slot[q];
        s_own_bin[rk] = q;
    }
    if (has_dep && tid == 0) {
        int off = 0;
        for (int q = 0; q < n_own; ++q) {
            const int n = s_hdr[q].z;
            if (n > 0 && off + n <= kMaxLensCTA) {
                s_loff[q] = off;
                off += n;
            } else {
                s_loff[q] = -1;
            }
        }
    }
    cta_sync<WARP>();
    // lens points: the first kLensInline of slots 0 and 1 came with the first load;
    // other short lists are beside their bin slots, long ones in the lens
    // array
    if (has_dep) {
        for (int q = 0; q < n_own; ++q) {
            const int n = s_hdr[q].z, o = s_loff[q];
            if (o < 0) continue;
            if (n <= kLensInline && q < 2) {
                if (tid < n) s_lens[o + tid] = s_lin[q][tid];
            } else if (n <= kLensInline) {
                if (tid < n) s_lens[o + tid] = P.lens_bin[bin_at(P, cell, q) * kLensInline + tid];
            } else {
                const float4 *src = P.lens + (size_t)s_tmp_i[q] * P.lens_cap;
                for (int m = tid; m < n; m += nthr) s_lens[o + m] = src[m];
            }
        }
    }
    const uint32_t sweep = S->sweep;
    if (PERSIST) {
        // the non-empty stencil cells of earlier phases of this sweep must be
        // done (their moves committed) before this cell reads them; those of
        // later phases wait for this one in turn, so no cell reads what
        // another writes while it writes (Sec. III.E)
        bool need = false;
        if (tid < n_st && m_nb > 0 && tid != t_own) {
            const int col = ((cx + dx) & 1) | (((cy + dy) & 1) << 1) | (((cz + dz) & 1) << 2);
            need = (int)((S->phase_of >> (4 * col)) & 15u) < phase;
        }
        // (each waiting lane's acquire load, then the warp barrier, order this
        // warp's later loads after the neighbours' released writes; the bins
        // are read through L2)
        const bool ok = !need || wait_ready(P.done + c_nb, epoch, P.wait_ns);
        if (!__all_sync(kFull, ok)) {
            if (tid == 0) atomicCAS(P.err, kErrNone, kErrTimeout);
            return;
        }
    } else {
        // the previous phase's moves are visible from here on
        pdl_wait();
    }
    // the neighbour cells' entries, relative to this cell's origin: up to four
    // per cell in one round, any further ones after it
    if (tid < n_st && tid != t_own) {
        const float fx = (float)dx * w32, fy = (float)dy * w32, fz = (float)dz * w32;
        // slot s of the cell at b[s * ncs]
        const float4 *b = P.bins + c_nb;
        const size_t ncs = (size_t)P.n_cells;
        auto stage = [&](const float4 v, int s) {
            const int slot = base + s;
            if (kChecked) {
                const int j = __float_as_int(v.w);
                // a candidate of this replica, binned in this very cell this sweep
                if (HPMC_CHECK_FAILS(P, slot < cand_cap(CAP), 2)) return;
                (void)HPMC_CHECK_FAILS(P, j >= R.off && j < R.off + R.n, 3);
                (void)HPMC_CHECK_FAILS(P, P.binpos == nullptr || (j >= 0 && j < P.n_total &&
                                                            bin_cell(P, P.binpos[j]) == c_nb), 4);
                // Sec. III.E: no other cell of the neighbourhood is active in
                // this phase (the own cell is staged above)
                const int col = ((cx + dx) & 1) | (((cy + dy) & 1) << 1) | (((cz + dz) & 1) << 2);
                const int own_col = (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
                (void)HPMC_CHECK_FAILS(P, col != own_col, 5);
            }
            s_cpos[slot] = make_float4(fx + v.x, fy + v.y, fz + v.z, v.w);
        };
        float4 e0 = make_float4(0.f, 0.f, 0.f, 0.f), e1 = e0, e2 = e0, e3 = e0;
        if (m_nb > 0) e0 = __ldcg(b);
        if (m_nb > 1) e1 = __ldcg(b + ncs);
        if (m_nb > 2) e2 = __ldcg(b + 2 * ncs);
        if (m_nb > 3) e3 = __ldcg(b + 3 * ncs);
        if (m_nb > 0) stage(e0, 0);
        if (m_nb > 1) stage(e1, 1);
        if (m_nb > 2) stage(e2, 2);
        if (m_nb > 3) stage(e3, 3);
        for (int s = 4; s < m_nb; ++s) stage(__ldcg(b + s * ncs), s);
    }
    cta_sync<WARP>();

    uint32_t c_acc = 0, c_cell = 0, c_ov = 0, c_dep = 0, c_cb = 0, c_eval = 0, c_block = 0,
             c_fwd = 0, c_rev = 0, c_cap = 0, c_rck = 0;
    unsigned long long c_drawn = 0;

    for (int q = 0; q < n_own; ++q) {
        const int i = s_own[q];
        const int nacc = s_nacc;
        const float4 ri = s_cpos[s_own_slot[q]];
        const int qb = s_own_bin[q];
        const float4 mv = s_mv[qb];
        const float rn0 = ri.x + mv.x, rn1 = ri.y + mv.y, rn2 = ri.z + mv.z;
        // a3: cell-exit check with margin (exact when within it)
        const float mc = m_cell, wc = w32;
        const bool out = rn0 < -mc || rn0 > wc + mc || rn1 < -mc || rn1 > wc + mc ||
                         rn2 < -mc || rn2 > wc + mc;
        const bool edge = rn0 <= mc || rn0 >= wc - mc || rn1 <= mc || rn1 >= wc - mc ||
                          rn2 <= mc || rn2 >= wc - mc;
        bool exits = out;
        if (!out && edge) {
            exits = exact_cell_exit(P, R, S, sweep, i, cx, cy, cz);
            if (tid == 0) ++c_rck;
        } else if (kChecked && tid == 0) {
            // the decision taken as certain, against the FP64 statement
            (void)HPMC_CHECK_FAILS(P, exact_cell_exit(P, R, S, sweep, i, cx, cy, cz) == out, 13);
        }
        if (exits) {
            ++c_cell;
            continue;
        }
        const float o0 = ri.x - rn0, o1 = ri.y - rn1, o2 = ri.z - rn2;

        // a4: colloid overlap at the new pose; neighbours in range
        if (!WARP) {
            if (tid == 0) s_nnb = 0;
            __syncthreads();
        }
        int ov = 0, nnb = 0;
        // the neighbour list is needed only if the move has lens points (or CB)
        const bool need_nb = has_dep && (CB || s_hdr[qb].z > 0);
        for (int j0 = 0; j0 < M; j0 += nthr) {
            const int j = j0 + tid;
            int t = 0, pj = -1;
            float d0 = 0.f, d1 = 0.f, d2 = 0.f, r2 = 1e30f;
            if (j < M) {
                const float4 cp = s_cpos[j];
                pj = __float_as_int(cp.w);
                if (pj == i) {
                    pj = -1;
                } else {
                    // candidates are relative to this cell's origin: with 4 or
                    // more cells per side |d| < 2w <= L/2 and the minimum image
                    // is d itself; only n_c = 2 folds
                    d0 = cp.x - rn0;
                    d1 = cp.y - rn1;
                    d2 = cp.z - rn2;
                    if (nc == 2) {
                        if (d0 > half_L32) d0 -= L32; else if (d0 < -half_L32) d0 += L32;
                        if (d1 > half_L32) d1 -= L32; else if (d1 < -half_L32) d1 += L32;
                        if (d2 > half_L32) d2 -= L32; else if (d2 < -half_L32) d2 += L32;
                    }
                    r2 = norm2f(d0, d1, d2);
                    t = tri(r2, T_contact, m_r2);
                }
            }
            if constexpr (kChecked) {
                if (pj >= 0 && t != -1)
                    (void)HPMC_CHECK_FAILS(P, exact_pair(P, R, sweep, i, pj, s_accl, nacc) == (t == 1), 14);
            }
            const bool unsure = t == -1;
            if (__any_sync(kFull, unsure)) {
                if (unsure) {
                    ++c_rck;
                    t = exact_pair(P, R, sweep, i, pj, s_accl, nacc) ? 1 : 0;
                }
            }
            if (t == 1) ov = 1;
            if (!need_nb) continue;
            const bool take = pj >= 0 && r2 < nb_cut2;
            if (WARP) {
                const unsigned b = __ballot_sync(kFull, take);
                const int slot = nnb + __popc(b & lt);
                if (take && slot < max_nb(CAP)) s_nb[slot] = make_float4(d0, d1, d2, __int_as_float(pj));
                nnb += __popc(b);
            } else if (take) {
                const int slot = atomicAdd(&s_nnb, 1);
                if (slot < max_nb(CAP)) s_nb[slot] = make_float4(d0, d1, d2, __int_as_float(pj));
            }
        }
        if (cta_any<WARP>(ov)) {
            ++c_ov;
            continue;
        }
        if (!WARP) nnb = s_nnb;
        if (nnb > max_nb(CAP)) {
            if (tid == 0) atomicCAS(P.err, kErrNone, kErrCandCap);
            return;
        }

        bool accept = true;
        if (has_dep) {
            // a5: N_p and the lens points come from the lens kernel
            const int4 hd = s_hdr[qb];
            const int n_p = hd.x;
            c_drawn += (unsigned long long)n_p;
            DepOutcome o = {1.0, 0, 0, 0u, 0u, 0u, 0u, 0u, 0u};
            // a6: the lens points in depletant order; one free of every
            // neighbour blocks the move (or enters the CB weight)
            int n_lens = hd.z;
            if (HPMC_CHECK_FAILS(P, n_lens >= 0 && n_lens <= P.lens_cap &&
                                        (s_loff[qb] < 0 || s_loff[qb] + n_lens <= kMaxLensCTA), 7))
                n_lens = 0;
            const float4 *lens = s_loff[qb] >= 0 ? s_lens + s_loff[qb]
                                                : P.lens + (size_t)i * P.lens_cap;
            if (!CB && !WARP) {
                if (tid == 0) sh.kmin = 0x7FFFFFFF;
                __syncthreads();
            }
            for (int m0 = 0; m0 < n_lens; m0 += nthr) {
                const int m = m0 + tid;
                int cls = 0, kk = 0x7FFFFFFF;
                uint32_t tt = 0;
                if (SOFT && m < n_lens) {
                    const float4 Lm = lens[m];
                    const uint32_t tk = (uint32_t)__float_as_int(Lm.w);
                    kk = (int)(tk & 0xFFFFu);
                    tt = tk >> 16;
                    cls = soft_cls32(R, sweep, (uint32_t)(i - R.off), tt, Lm.x, Lm.y, Lm.z, -mv.x, -mv.y,
                                     -mv.z, s_nb, nnb);
                } else if (!SOFT && m < n_lens) {
                    const float4 Lm = lens[m];
                    const uint32_t tk = (uint32_t)__float_as_int(Lm.w);
                    kk = (int)(tk & 0xFFFFu);
                    tt = tk >> 16;
                    bool unsure = false, hit = false;
                    for (int b = 0; b < nnb; ++b) {
                        const float4 d = s_nb[b];
                        const int tn = tri(norm2f(Lm.x - d.x, Lm.y - d.y, Lm.z - d.z),
                                           T_dep, m_r2);
                        if (tn == 1) {
                            hit = true;
                            break;
                        }
                        unsure = unsure || tn == -1;
                    }
                    cls = hit ? 0 : (unsure ? -1 : 1);
                    if constexpr (kChecked) {
                        // a class taken as certain, against the FP64 statement
                        if (cls != -1)
                            (void)HPMC_CHECK_FAILS(
                                P, exact_free_nb(P, R, sweep, i, tt, s_nb, nnb, s_accl, nacc) == (cls == 1), 15);
                    }
                }
                {
                    const bool unsure = cls == -1;
                    if (__any_sync(kFull, unsure)) {
                        if (unsure) {
                            ++o.rck;
                            cls = (SOFT ? exact_soft_nb(P, R, sweep, i, tt, s_nb, nnb, s_accl, nacc)
                                        : exact_free_nb(P, R, sweep, i, tt, s_nb, nnb, s_accl, nacc))
                                      ? 1 : 0;
                        }
                    }
                }
                const bool blocking = cls == 1;
                if (!CB) {
                    int kmin;
                    bool any;
                    if (WARP) {
                        kmin = __reduce_min_sync(kFull, blocking ? kk : 0x7FFFFFFF);
                        any = kmin != 0x7FFFFFFF;
                    } else {
                        if (blocking) atomicMin(&sh.kmin, kk);
                        any = __syncthreads_or(blocking) != 0;
                        kmin = sh.kmin;
                    }
                    if (any) {
                        o.block += 1;
                        o.eval += (uint32_t)(kmin + 1);
                        o.rejected = 1;
                        break;
                    }
                } else {
                    // the factors of the warp's blocking depletants in
                    // ascending k, each by the whole warp; a zero factor
                    // rejects the move, so the ones after it are not needed
                    double f = 0.0;
                    bool has = false, zero = false;
                    unsigned bm = __ballot_sync(kFull, blocking);
                    while (bm) {
                        const int b = __ffs(bm) - 1;
                        bm &= bm - 1u;
                        const uint32_t kb = (uint32_t)__shfl_sync(kFull, kk, b);
                        const CbResult32 r = cb_factor_warp32(P, R, sweep, i, kb, o0, o1, o2, s_nb, nnb,
                                                              s_accl, nacc);
                        o.rck += r.rck;
                        if (lane == b) {
                            f = r.f;
                            has = true;
                            zero = r.fwd_ok == 0;
                            o.fwd += r.fwd_ok;
                            o.rev += r.rev_ok;
                            o.cap += r.caps;
                        }
                        if (r.fwd_ok == 0) break;
                    }
                    if (cb_pass(sh, tid, nthr, has, f, zero, kk, o, -1)) {
                        o.rejected = 1;
                        break;
                    }
                }
            }
            if (!o.rejected) {
                o.eval += (uint32_t)hd.y;
                if (hd.y < n_p && tid == 0) ++o.cap;
            }
            c_eval += o.eval;
            c_block += o.block;
            c_cap += o.cap;
            c_rck += o.rck;
            c_fwd += o.fwd;
            c_rev += o.rev;
            if (o.rejected) {
                accept = false;
                // (a replica without CB in a batch that has some: its first
                // blocking depletant rejects the move as a depletant rejection)
                if (!CB || R.n_trial == 0) ++c_dep;
                else ++c_cb;
            } else if (CB && tid == 0 && o.nblock > 0) {
                const uint4 wa = draw(R.key0, R.key1, sweep, (uint32_t)(i - R.off), kPAccept, 0, 0);
                if (!(u53(wa.x, wa.y) < o.W)) {
                    accept = false;
                    ++c_cb;
                }
            }
            if (CB) {
                if (WARP) {
                    accept = __shfl_sync(kFull, accept ? 1 : 0, 0) != 0;
                } else {
                    if (tid == 0) s_acc = accept ? 1 : 0;
                    __syncthreads();
                    accept = s_acc != 0;
                }
            }
        }
        // a8: accepted: the FP32 working copies move now (shared neighbourhood
        // and the cell bin later phases stage from), the FP64 position when
        // this CTA finishes
        if (accept) {
            ++c_acc;
            if (tid == 0) {
                const float4 rnew = make_float4(rn0, rn1, rn2, __int_as_float(i));
                s_cpos[s_own_slot[q]] = rnew;
                P.bins[bin_at(P, cell, s_own_bin[q])] = rnew;
                s_accl[nacc] = i;
                s_nacc = nacc + 1;
            }
        }
        cta_sync<WARP>();
    }

    // deferred FP64 commit of the accepted moves, one colloid per lane
    const int nacc = s_nacc;
    for (int a = tid; a < nacc; a += nthr) {
        const int j = s_accl[a];
        if (HPMC_CHECK_FAILS(P, a < CAP && j >= R.off && j < R.off + R.n, 8)) continue;
        P.pos[j] = P.prop_pos[j];
    }

    unsigned long long cnt[kNumCounters] = {0};
    if (tid == 0) {
        cnt[kMoves] = (unsigned long long)n_own;
        cnt[kTranslate] = (unsigned long long)n_own;
        cnt[kAccept] = c_acc;
        cnt[kRejCell] = c_cell;
        cnt[kRejOverlap] = c_ov;
        cnt[kRejDep] = c_dep;
        cnt[kRejCb] = c_cb;
        cnt[kDepDrawn] = c_drawn;
        cnt[kDepEval] = c_eval;
        cnt[kDepBlocking] = c_block;
    }
    cnt[kCbFwdOk] = c_fwd;
    cnt[kCbRevOk] = c_rev;
    cnt[kCapHits] = c_cap;
    cnt[kRechecks] = c_rck;
    flush_counters(P, r, cnt);
}

// Sizes of a phase's four population classes (the task ordering kernel's
// counts), by a load the compiler keeps where it stands.
__device__ __forceinline__ int4 ld_cls_count(const SimParams &P, int phase)
{
    int4 v;
    asm volatile("ld.global.nc.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(P.cls_count + 4 * phase));
    return v;
}

__device__ __forceinline__ int cls_busy(const SimParams &P, int phase)
{
    const int4 v = ld_cls_count(P, phase);
    return v.x + v.y + v.z;
}

// One colour phase (FP32 form): the non-empty cells of every replica in the
// task table's order (fullest cells first); empty cells have no work (the
// task ordering kernel cleared their next-sweep populations).  LOOP false: a
// CTA per cell of the phase (grid n_cta; CTAs past the non-empty cells return
// at once).  LOOP true: a few waves of resident one-warp CTAs, CTA b taking
// cells b, b + gridDim, ... (the cells of a phase are independent), which
// saves a CTA launch per cell where a phase has many cells per SM; the loop
// needs more registers per thread (24 resident CTAs per SM instead of 32).
template <bool CB, bool WARP, int CAP, bool SOFT = false, bool LOOP = false>
__global__ void __launch_bounds__(WARP ? 32 : kMaxThreads,
                                  WARP ? ((CB || SOFT) ? 16 : (LOOP ? 24 : 32)) : 1)
    k_phase_sphere_fp32(const __grid_constant__ SimParams P, int phase)
{
    // The phases are launched with programmatic dependent launch: the next
    // phase's CTAs may start while this one drains.  Everything read before
    // pdl_wait() is fixed for the whole sweep (task table, populations, replica
    // record, lens headers, displacements and lens points); positions (bins,
    // FP64 state) are read and written only after it.
    pdl_trigger();
    if (phase == 7 && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(P.sweep, 1ull);
    // this grid must not complete before its predecessor, even with no cell
    // to move (a later phase's wait covers only this grid)
    if (blockIdx.x == 0 && cls_busy(P, phase) == 0) pdl_wait();
#pragma unroll 1
    for (int b = blockIdx.x;; b += gridDim.x) {
        // the class sizes are re-read for every cell (an L1 hit) rather than
        // kept across the cell's work, which needs every register
        const int4 cc = ld_cls_count(P, phase);
        if (b >= cc.x + cc.y + cc.z) break;
        int idx = b, cls = 0;
        if (idx >= cc.x) {
            idx -= cc.x;
            cls = 1;
            if (idx >= cc.y) {
                idx -= cc.y;
                cls = 2;
            }
        }
        const int4 tk = P.task_ord[(size_t)(phase * 4 + cls) * P.n_cta + idx];
        phase_cell<CB, WARP, CAP, SOFT, false>(P, phase, tk, 0u);
        if (!LOOP) break;
        // the shared-memory stage is the next cell's
        cta_sync<WARP>();
    }
}

// All eight colour phases of a sweep in one persistent launch of one-warp
// CTAs.  The work items are the non-empty active cells, in phase order and,
// within a phase, fullest cells first; a CTA takes the next item from a
// ticket counter and waits only for the non-empty stencil cells of earlier
// phases (readiness counters, bounded waits), so a cell of phase p + 1 starts
// as soon as its own neighbourhood has finished phase p instead of after the
// whole grid has.  Deadlock-free for any grid size and residency: an item
// waits only for items with smaller tickets, all taken earlier by CTAs that
// are running (a CTA works through its chunk in order), and the smallest
// unfinished item never waits.
template <bool CB, int CAP, bool SOFT = false>
__global__ void __launch_bounds__(32, (CB || SOFT) ? 16 : 32)
    k_sweep_sphere_fp32(const __grid_constant__ SimParams P)
{
    const int lane = threadIdx.x;
    pdl_wait();
    const uint32_t epoch0 = ld_acquire_u32(P.epoch);
    if (blockIdx.x == 0 && lane == 0) atomicAdd(P.sweep, 1ull);
    // non-empty tasks per phase (population classes 0..2): their exclusive
    // prefix over the phases and the first two class sizes, kept in shared
    // memory (registers are the phase work's)
    __shared__ int s_start[9], s_n0[8], s_n1[8];
    __shared__ uint32_t s_epoch;
    __shared__ int s_cell;
    {
        int ne = 0;
        int4 cc = make_int4(0, 0, 0, 0);
        if (lane < 8) {
            cc = reinterpret_cast<const int4 *>(P.cls_count)[lane];
            ne = cc.x + cc.y + cc.z;
        }
        int incl = ne;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < 8) {
            s_start[lane + 1] = incl;
            s_n0[lane] = cc.x;
            s_n1[lane] = cc.y;
        }
        if (lane == 0) {
            s_start[0] = 0;
            s_epoch = epoch0;
        }
        __syncwarp();
    }
    // tickets are taken in chunks of P.ticket_chunk consecutive items (one
    // atomic per chunk: the counter is a single hot address), processed in
    // order, which keeps the schedule deadlock-free; the next chunk is
    // claimed while the current item runs (its atomic's latency hidden)
    const int chunk = P.ticket_chunk;
    int t = 0, t_end = 0, t_ahead = 0;
    if (lane == 0) t_ahead = atomicAdd(P.ticket, chunk);
    while (true) {
        if (t == t_end) {
            t = __shfl_sync(kFull, t_ahead, 0);
            t_end = t + chunk;
            if (lane == 0 && t < s_start[8]) t_ahead = atomicAdd(P.ticket, chunk);
        }
        if (t >= s_start[8]) break;
        // the ticket's phase: the number of phases that end at or before t
        const int phase = __popc(__ballot_sync(kFull, lane < 8 && s_start[lane + 1] <= t));
        int idx = t - s_start[phase], cls = 0;
        const int n0 = s_n0[phase], n1 = s_n1[phase];
        if (idx >= n0) {
            idx -= n0;
            cls = 1;
            if (idx >= n1) {
                idx -= n1;
                cls = 2;
            }
        }
        const int4 tk = P.task_ord[(size_t)(phase * 4 + cls) * P.n_cta + idx];
        if (lane == 0) s_cell = tk.x;
        phase_cell<CB, true, CAP, SOFT, true>(P, phase, tk, s_epoch);
        // publish the cell: every lane's writes first, then its readiness
        // (a cell withheld for a test of the bounded waits is never published)
        __syncwarp();
        if (lane == 0 && s_cell != P.withhold) st_release_u32(P.done + s_cell, s_epoch);
        ++t;
    }
}

// Configuration check (positions in the box, no overlapping pair), FP32
// sphere form: distances from the FP32 cell-relative copies the cell-list
// kernel filed in the bins (its bin slot from binpos), decided with the
// certified margin and re-taken in FP64 (the positions, minimum image) only
// inside it.  One thread per (colloid, stencil cell): every thread's loads
// are two dependent rounds (the cell's population, then its entries).  Each
// pair is tested once: from the colloid's own cell (partners of higher
// index) and the 13 stencil cells that follow it in stencil order (every
// partner; the other 13 are the preceding cells, whose colloids test this
// one); with two cells per side, where the stencil is the whole box, every
// cell with partners of higher index.
constexpr int kCheckStencil = 14;

__global__ void k_check_spheres32(const __grid_constant__ SimParams P, int *flag)
{
    const size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int g = (int)(gt / kCheckStencil), t = (int)(gt % kCheckStencil);
    if (g >= P.n_total) return;
    const int r = P.rep_of[g];
    const Rep &R = P.reps[r];
    if (g - R.off >= P.n_live[r]) return;
    const double4 pi = P.pos[g];
    if (!(pi.x >= 0.0 && pi.x < R.L && pi.y >= 0.0 && pi.y < R.L && pi.z >= 0.0 && pi.z < R.L)) {
        if (t == 0) atomicOr(flag, 2);
        return;
    }
    const int nc = R.nc;
    const int ns = nc == 2 ? 2 : 3;
    if (ns == 2 && t >= 8) return;
    const int ts = ns == 3 ? 13 + t : t;      // the stencil cell
    const bool higher = ns == 2 || ts == 13;  // partners of higher index only
    const int bp = P.binpos[g];
    if (bp < 0) return;   // a full cell: the cell-list kernel has flagged it
    const int cl = bin_cell(P, bp) - R.cell_off;
    const int cx = cl % nc, cy = (cl / nc) % nc, cz = cl / (nc * nc);
    const float4 ri = P.bins[bp];
    const Sched &S = P.sched[r];
    const int *count = P.count[S.sweep & 1u];
    const float w32 = R.w32, L32 = R.L32, half_L32 = R.half_L32;
    int dx, dy, dz;
    const int c = stencil_cell_nc(nc, R.cell_off, ts, cx, cy, cz, dx, dy, dz);
    const int m = min(count[c], P.cap);
    const float fx = (float)dx * w32 - ri.x, fy = (float)dy * w32 - ri.y, fz = (float)dz * w32 - ri.z;
    for (int s = 0; s < m; ++s) {
        const float4 e = P.bins[bin_at(P, c, s)];
        const int j = __float_as_int(e.w);
        if (j == g || (higher && j < g)) continue;
        float d0 = fx + e.x, d1 = fy + e.y, d2 = fz + e.z;
        if (nc == 2) {
            if (d0 > half_L32) d0 -= L32; else if (d0 < -half_L32) d0 += L32;
            if (d1 > half_L32) d1 -= L32; else if (d1 < -half_L32) d1 += L32;
            if (d2 > half_L32) d2 -= L32; else if (d2 < -half_L32) d2 += L32;
        }
        int o = tri(norm2f(d0, d1, d2), R.T_contact32, R.m_r2);
        if (o == -1) {
            const double4 pj = P.pos[j];
            const double r2 = norm2(min_image(pj.x - pi.x, R.L, R.half_L),
                                    min_image(pj.y - pi.y, R.L, R.half_L),
                                    min_image(pj.z - pi.z, R.L, R.half_L));
            o = r2 < R.contact2 ? 1 : 0;
        }
        if (o == 1) atomicOr(flag, 1);
    }
}

}  // namespace hpmc
