// FP32 form for anisotropic colloids (hemispheres, discoids; Sec. V) with
// translation and rotation moves.
//
// Per sweep: k_propose_aniso computes every colloid's proposed pose exactly
// (FP64, one thread per colloid, so the FP64 work is spread over all lanes);
// k_lens_aniso_fp32 builds the depletant lens lists (one warp per colloid);
// the eight colour phases (k_phase_aniso_fp32) test colloid pairs and lens
// points against neighbours.  Every test is taken in FP32 with a certified
// margin (hpmc_shapes32.cuh); a test inside its margin is re-taken with the
// exact FP64 statement (hpmc_shapes.cuh), so all decisions equal the FP64
// form's.  Accepted poses are committed from the exact proposals.
#pragma once

#include "hpmc_common.cuh"
#include "hpmc_shapes.cuh"
#include "hpmc_shapes32.cuh"
#include "hpmc_sphere_fp32.cuh"

namespace hpmc {

// ---------------------------------------------------------------------------
// Exact proposals: prop_pos[g] = (new position, kind) with kind 1 translation,
// 0 rotation, -1 rotation attempt stream capped (the move is rejected);
// prop_quat[g] = new orientation (the old one for a translation).
// ---------------------------------------------------------------------------
__global__ void k_propose_aniso(const __grid_constant__ SimParams P)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.n_total) return;
    const int r = P.rep_of[g];
    const Rep &R = P.reps[r];
    const uint32_t sweep = P.sched[r].sweep;
    const uint32_t tag = (uint32_t)(g - R.off);
    const uint4 wm = draw(R.key0, R.key1, sweep, tag, kPMove, 0, 0);
    bool translate = true;
    if (R.rot_on) {
        if (R.p_translate <= 0.0) translate = false;
        else if (R.p_translate < 1.0) translate = u01(wm.w) < R.p_translate;
    }
    const double4 p = P.pos[g];
    const double4 qo = P.quat[g];
    if (translate) {
        P.prop_pos[g] = make_double4(wrap_box(p.x + R.d_max * s11(wm.x), R.L),
                                     wrap_box(p.y + R.d_max * s11(wm.y), R.L),
                                     wrap_box(p.z + R.d_max * s11(wm.z), R.L), 1.0);
        P.prop_quat[g] = qo;
        return;
    }
    double4 qn = qo;
    const bool ok = propose_rotation(R, sweep, tag, qo, &qn);
    P.prop_pos[g] = make_double4(p.x, p.y, p.z, ok ? 0.0 : -1.0);
    P.prop_quat[g] = qn;
}

__device__ __forceinline__ float4 quat32(double4 q)
{
    return make_float4((float)q.x, (float)q.y, (float)q.z, (float)q.w);
}

// Exact current pose of colloid j: its proposal if this CTA accepted its
// move (commits are deferred to the end of the CTA), else the state.
__device__ __forceinline__ void pose_now(const SimParams &P, int j, const int *acc, int nacc,
                                         double4 &x, double4 &q)
{
    for (int a = 0; a < nacc; ++a)
        if (acc[a] == j) {
            x = P.prop_pos[j];
            q = P.prop_quat[j];
            return;
        }
    x = P.pos[j];
    q = P.quat[j];
}

// Exact depletant test.  The point is R_s s11(w) around the new reference
// point of colloid i (base 0) or around its old one (base 1); it is tested
// against i's new pose (target 0), i's old pose (target 1) or neighbour j
// (target 2).
__device__ __noinline__ bool exact_dep_aniso(const SimParams &P, const Rep &R, int i, uint4 w,
                                             int base, int target, int j, const int *acc, int nacc,
                                             int half = -1)
{
    const double4 xn = P.prop_pos[i];
    const double4 xo = P.pos[i];
    const Vec3 o = v3(min_image(xo.x - xn.x, R.L, R.half_L), min_image(xo.y - xn.y, R.L, R.half_L),
                      min_image(xo.z - xn.z, R.L, R.half_L));
    double p0, p1, p2;
    point64(R, w, half, p0, p1, p2);
    Vec3 v = v3(p0, p1, p2);
    if (base == 1) v = v3(o.x + v.x, o.y + v.y, o.z + v.z);
    if (target == 0) return dep_aniso(R, v, P.prop_quat[i]);
    if (target == 1) return dep_aniso(R, v3(v.x - o.x, v.y - o.y, v.z - o.z), P.quat[i]);
    double4 xj, qj;
    pose_now(P, j, acc, nacc, xj, qj);
    const Vec3 c = v3(min_image(xj.x - xn.x, R.L, R.half_L), min_image(xj.y - xn.y, R.L, R.half_L),
                      min_image(xj.z - xn.z, R.L, R.half_L));
    return dep_aniso(R, v3(v.x - c.x, v.y - c.y, v.z - c.z), qj);
}

// Exact colloid pair test of i at its proposed pose against j now: FP64
// certificates along the FP32 direction first, the full FP64 statement if
// they do not decide.
__device__ __noinline__ bool exact_pair_aniso(const SimParams &P, const Rep &R, int i, int j,
                                              const int *acc, int nacc, float3 nf, uint32_t &stage3)
{
    const double4 xn = P.prop_pos[i];
    const double4 qn = P.prop_quat[i];
    double4 xj, qj;
    pose_now(P, j, acc, nacc, xj, qj);
    const Vec3 d = v3(min_image(xj.x - xn.x, R.L, R.half_L), min_image(xj.y - xn.y, R.L, R.half_L),
                      min_image(xj.z - xn.z, R.L, R.half_L));
    const int c = pair_cert64(R, qn, qj, d, nf);
    if (c >= 0) return c == 1;
    ++stage3;
    return pair_aniso(R, d, qn, qj);
}

// ---------------------------------------------------------------------------
// Depletant lens lists, one warp per colloid (as for spheres, but "overlaps
// the new pose" is a shape test, not the sampling-ball test).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_lens_aniso_fp32(const __grid_constant__ SimParams P)
{
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= P.n_total) return;
    const int r = P.rep_of[g];
    const Rep &R = P.reps[r];
    const uint32_t sweep = P.sched[r].sweep;
    const uint32_t tag = (uint32_t)(g - R.off);
    const double kind = P.prop_pos[g].w;
    float D0 = 0.0f, D1 = 0.0f, D2 = 0.0f;
    if (kind > 0.5) {
        const uint4 wm = draw(R.key0, R.key1, sweep, tag, kPMove, 0, 0);
        D0 = coord32(wm.x, R.d_max32);
        D1 = coord32(wm.y, R.d_max32);
        D2 = coord32(wm.z, R.d_max32);
    }
    // displacement, move kind, header and the first lens points go to the
    // colloid's bin slot, where the colour phase reads them
    const int bp = P.binpos[g];
    if (lane == 0 && bp >= 0) P.mv_bin[bp] = make_float4(D0, D1, D2, (float)kind);
    if (!R.has_dep) return;
    if (kind < -0.5) {
        if (lane == 0 && bp >= 0) P.hdr_bin[bp] = make_int4(0, 0, 0, 0);
        return;
    }
    if (kind > 0.5) {
        const float4 ri = P.rel[g];
        const float rn0 = ri.x + D0, rn1 = ri.y + D1, rn2 = ri.z + D2;
        const float mc = R.m_cell, wc = R.w32;
        if (rn0 < -mc || rn0 > wc + mc || rn1 < -mc || rn1 > wc + mc || rn2 < -mc ||
            rn2 > wc + mc) {
            if (lane == 0 && bp >= 0) P.hdr_bin[bp] = make_int4(0, 0, 0, 0);
            return;
        }
    }
    // the two frames live in shared memory (fewer registers, more resident warps)
    __shared__ Frame32 s_F[4][2];
    const int wib = threadIdx.x >> 5;
    if (lane == 0) {
        s_F[wib][0] = frame32(quat32(P.prop_quat[g]));
        s_F[wib][1] = frame32(quat32(P.quat[g]));
    }
    __syncwarp();
    const Frame32 &Fn = s_F[wib][0];
    const Frame32 &Fo = s_F[wib][1];
    uint32_t rck = 0;
    const float o0 = -D0, o1 = -D1, o2 = -D2;
    const uint4 wp = draw(R.key0, R.key1, sweep, tag, kPPoisson, 0, 0);
    const int n_p = poisson_count(P.T + R.t_off, R.nF, u53_int(wp.x, wp.y), lane);
    const uint32_t t_max = 64u * (uint32_t)(n_p + 1);
    float4 *out = P.lens + (size_t)g * P.lens_cap;
    const unsigned lt = (1u << lane) - 1u;
    // The shape tests dominate: a pass queues its depletants (ball points of
    // index k < N_p, in depletant order) in shared memory, and the tests run
    // on full batches of 32 queued points (the last batch partial), so every
    // lane tests a depletant instead of half of them testing nothing.  Lens
    // points leave the queue in depletant order, as the list needs them.
    __shared__ float4 s_q[4][64];   // (e, (t << 16) | k) per queued depletant
    int m = 0;
    auto test_batch = [&](int nb) {
        const bool act = lane < nb;
        const float4 v = act ? s_q[wib][lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t tk = (uint32_t)__float_as_int(v.w);
        const uint32_t t = tk >> 16;
        // overlaps the new pose?
        int tn = act ? dep_tri32(R, make_float3(v.x, v.y, v.z), Fn) : 0;
        if constexpr (kChecked) {
            // a decision taken as certain, against the FP64 statement
            if (act && tn != -1) {
                const uint4 w = draw(R.key0, R.key1, sweep, tag, kPDep, 0, paired_call(t));
                (void)HPMC_CHECK_FAILS(
                    P, exact_dep_aniso(P, R, g, w, 0, 0, 0, nullptr, 0, (int)paired_half(t)) == (tn == 1), 17);
            }
        }
        {
            const bool unsure = tn == -1;
            if (__any_sync(kFull, unsure)) {
                if (unsure) {
                    ++rck;
                    const uint4 w = draw(R.key0, R.key1, sweep, tag, kPDep, 0, paired_call(t));
                    tn = exact_dep_aniso(P, R, g, w, 0, 0, 0, nullptr, 0, (int)paired_half(t)) ? 1 : 0;
                }
            }
        }
        // and not the old pose?
        int to = 1;
        if (tn == 1) to = dep_tri32(R, make_float3(v.x - o0, v.y - o1, v.z - o2), Fo);
        if constexpr (kChecked) {
            if (act && tn == 1 && to != -1) {
                const uint4 w = draw(R.key0, R.key1, sweep, tag, kPDep, 0, paired_call(t));
                (void)HPMC_CHECK_FAILS(
                    P, exact_dep_aniso(P, R, g, w, 0, 1, 0, nullptr, 0, (int)paired_half(t)) == (to == 1), 17);
            }
        }
        {
            const bool unsure = to == -1;
            if (__any_sync(kFull, unsure)) {
                if (unsure) {
                    ++rck;
                    const uint4 w = draw(R.key0, R.key1, sweep, tag, kPDep, 0, paired_call(t));
                    to = exact_dep_aniso(P, R, g, w, 0, 1, 0, nullptr, 0, (int)paired_half(t)) ? 1 : 0;
                }
            }
        }
        // lens points are rare: their list slots are ranked only in a batch
        // that has one
        const bool lens = tn == 1 && to == 0;
        if (__any_sync(kFull, lens)) {
            const unsigned lb = __ballot_sync(kFull, lens);
            const int slot = m + __popc(lb & lt);
            if (lens && slot < P.lens_cap) out[slot] = v;
            m += __popc(lb);
        }
    };
    uint32_t t0 = 0;
    int k0 = 0, qn = 0;
    uint4 wc = make_uint4(0, 0, 0, 0);
    while (k0 < n_p && t0 < t_max) {
        const uint32_t t = t0 + (uint32_t)lane;
        float e0 = 0.f, e1 = 0.f, e2 = 0.f;
        int in = 0;
        // the paired stream: attempt t is half paired_half(t) of call
        // paired_call(t); a pass of 32 attempts takes one half of the lanes'
        // 32 calls, so the words are drawn on the first half's pass and kept
        // for the second (t_max is a multiple of 64: whole blocks)
        const int half = (int)paired_half(t);
        if ((t0 & 32u) == 0u) wc = draw(R.key0, R.key1, sweep, tag, kPDep, 0, paired_call(t));
        const uint4 w = wc;
        if (t < t_max) {
            const uint3 f = paired_fields(w, (uint32_t)half);
            e0 = s21f_bits(f.x) * R.R_s32;
            e1 = s21f_bits(f.y) * R.R_s32;
            e2 = s21f_bits(f.z) * R.R_s32;
            in = R.v0_cube ? 1 : tri(norm2f(e0, e1, e2), R.T_s32, R.m_r2);
            if constexpr (kChecked) {
                if (!R.v0_cube && in != -1) (void)HPMC_CHECK_FAILS(P, exact_ball(P, R, w, half) == (in == 1), 11);
            }
        }
        {
            const bool unsure = in == -1;
            if (__any_sync(kFull, unsure)) {
                if (unsure) {
                    ++rck;
                    in = exact_ball(P, R, w, half) ? 1 : 0;
                }
            }
        }
        const unsigned bal = __ballot_sync(kFull, in == 1);
        const int k = k0 + __popc(bal & lt);
        const bool dep = in == 1 && k < n_p;
        const unsigned db = __ballot_sync(kFull, dep);
        if (dep) s_q[wib][qn + __popc(db & lt)] = make_float4(e0, e1, e2, __int_as_float((int)((t << 16) | (uint32_t)k)));
        qn += __popc(db);
        k0 += __popc(bal);
        t0 += 32u;
        __syncwarp();
        if (qn >= 32) {
            test_batch(32);
            // the rest (fewer than 32) to the front of the queue
            const int rest = qn - 32;
            float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncwarp();
            if (lane < rest) x = s_q[wib][32 + lane];
            __syncwarp();
            if (lane < rest) s_q[wib][lane] = x;
            __syncwarp();
            qn = rest;
        }
    }
    if (qn > 0) test_batch(qn);
    __syncwarp();
    if (bp >= 0) {
        if (lane == 0) P.hdr_bin[bp] = make_int4(n_p, min(k0, n_p), min(m, P.lens_cap), 0);
        if (lane < min(m, kLensInline)) P.lens_bin[(size_t)bp * kLensInline + lane] = out[lane];
    }
    if (lane == 0 && m > P.lens_cap) atomicCAS(P.err, kErrNone, kErrCandCap);
    rck = __reduce_add_sync(kFull, rck);
    if (lane == 0 && rck) count_one(P, r, kRechecks, (unsigned long long)rck);
}

// ---------------------------------------------------------------------------
// Neighbour tests of one point and the CB factor, FP32 with exact re-takes.
// ---------------------------------------------------------------------------
struct Nb32 {
    float4 d;       // offset from the moved colloid's new reference point; index in .w
    Frame32 F;
};

// Is the point y (relative to the new reference point; drawn around base with
// word w) free of every neighbour?
__device__ __forceinline__ bool free_nb_aniso32(const SimParams &P, const Rep &R, float3 y,
                                                const Nb32 *nb, int nnb, int i, uint4 w, int base,
                                                const int *acc, int nacc, uint32_t &rck)
{
    for (int a = 0; a < nnb; ++a) {
        const float4 d = nb[a].d;
        const int t = dep_tri32(R, make_float3(y.x - d.x, y.y - d.y, y.z - d.z), nb[a].F);
        if constexpr (kChecked) {
            if (t != -1)
                (void)HPMC_CHECK_FAILS(
                    P, exact_dep_aniso(P, R, i, w, base, 2, __float_as_int(d.w), acc, nacc) == (t == 1), 20);
        }
        if (t == 1) return false;
        if (t == -1) {
            ++rck;
            if (exact_dep_aniso(P, R, i, w, base, 2, __float_as_int(d.w), acc, nacc)) return false;
        }
    }
    return true;
}

__device__ __forceinline__ int dep_self32(const SimParams &P, const Rep &R, float3 v, const Frame32 &F,
                                          int i, uint4 w, int base, int target, uint32_t &rck)
{
    int t = dep_tri32(R, v, F);
    if constexpr (kChecked) {
        if (t != -1)
            (void)HPMC_CHECK_FAILS(P, exact_dep_aniso(P, R, i, w, base, target, 0, nullptr, 0) == (t == 1), 20);
    }
    if (t == -1) {
        ++rck;
        t = exact_dep_aniso(P, R, i, w, base, target, 0, nullptr, 0) ? 1 : 0;
    }
    return t;
}

// CB factor of one blocking depletant k (Sec. III.D, Eq. 12), FP32 form,
// computed by a whole warp (all 32 lanes call it with the same k): the trials
// of a direction are the first n_fwd (n_rev) attempts of the stream
// (purpose, k) inside the sampling ball; lanes take consecutive attempts and
// a ballot ranks the in-ball ones.  Returns the same values in every lane
// except rck (the lane's own FP64 re-takes).
__device__ __noinline__ CbResult32 cb_factor_aniso32(const SimParams &P, const Rep &R, uint32_t sweep,
                                                     int i, uint32_t k, float3 o, const Frame32 &Fn,
                                                     const Frame32 &Fo, const Nb32 *nb, int nnb,
                                                     const int *acc, int nacc)
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
                const float3 e = make_float3(e0, e1, e2);
                if (fwd) {
                    // must overlap the old pose and miss the new one
                    const float3 y = make_float3(o.x + e0, o.y + e1, o.z + e2);
                    good = dep_self32(P, R, e, Fo, i, w, 1, 1, r.rck) != 0 &&
                           dep_self32(P, R, y, Fn, i, w, 1, 0, r.rck) != 1 &&
                           free_nb_aniso32(P, R, y, nb, nnb, i, w, 1, acc, nacc, r.rck);
                } else {
                    // must overlap the new pose and miss the old one
                    good = dep_self32(P, R, e, Fn, i, w, 0, 0, r.rck) != 0 &&
                           dep_self32(P, R, make_float3(e0 - o.x, e1 - o.y, e2 - o.z), Fo, i, w, 0, 1,
                                      r.rck) != 1 &&
                           free_nb_aniso32(P, R, e, nb, nnb, i, w, 0, acc, nacc, r.rck);
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

// A lens point free of every neighbour, exactly.
__device__ __noinline__ bool exact_free_nb_aniso(const SimParams &P, const Rep &R, uint32_t sweep, int i,
                                                 uint32_t t, const Nb32 *nb, int nnb, const int *acc,
                                                 int nacc)
{
    // (the paired stream)
    const uint4 w = draw(R.key0, R.key1, sweep, (uint32_t)(i - R.off), kPDep, 0, paired_call(t));
    for (int a = 0; a < nnb; ++a)
        if (exact_dep_aniso(P, R, i, w, 0, 2, __float_as_int(nb[a].d.w), acc, nacc,
                            (int)paired_half(t)))
            return false;
    return true;
}

constexpr int kMaxNbAniso = 128;   // neighbours within reach of a depletant (checked on the host)

// ---------------------------------------------------------------------------
// One colour phase, FP32 form, anisotropic colloids: as k_phase_sphere_fp32,
// plus orientations (FP32 copies of the candidates' quaternions in shared
// memory, frames of the neighbours in range) and rotation moves.
// ---------------------------------------------------------------------------
template <bool CB, bool WARP, int CAP>
__global__ void __launch_bounds__(WARP ? 32 : kMaxThreads, WARP ? 8 : 1)
    k_phase_aniso_fp32(const __grid_constant__ SimParams P, int phase)
{
    __shared__ float4 s_cpos[kMaxCand];
    __shared__ float4 s_cq[kMaxCand];
    __shared__ Nb32 s_nb[kMaxNbAniso];
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
    // Launched with programmatic dependent launch, as the sphere phases: the
    // task, populations, replica record and the lens kernel's per-slot data
    // are fixed for the sweep and read before pdl_wait(); positions and
    // orientations (bins, FP64 state) only after it.
    pdl_trigger();
    if (phase == 7 && blockIdx.x == 0 && tid == 0) atomicAdd(P.sweep, 1ull);
    // the phase's non-empty cells come first in the task order; an empty cell
    // has no work (its next-sweep population was cleared by the task ordering
    // kernel), so CTAs past them return at once; this grid must still not
    // complete before its predecessor when no cell has work (a later phase's
    // wait covers only this grid)
    int cls = 0, idx = blockIdx.x;
    {
        const int4 cc = reinterpret_cast<const int4 *>(P.cls_count)[phase];
        if (blockIdx.x == 0 && cc.x + cc.y + cc.z == 0) pdl_wait();
        if (idx >= cc.x + cc.y + cc.z) return;
        if (idx >= cc.x) {
            idx -= cc.x;
            cls = 1;
            if (idx >= cc.y) {
                idx -= cc.y;
                cls = 2;
            }
        }
    }
    const int4 tk = P.task_ord[(size_t)(phase * 4 + cls) * P.n_cta + idx];
    const int cell = tk.x, r = tk.y;
    const int cx = tk.z & 1023, cy = (tk.z >> 10) & 1023, cz = tk.z >> 20;
    const int nc = tk.w & 0xFFFF, par = tk.w >> 16;
    const int ns = nc == 2 ? 2 : 3, n_st = ns * ns * ns;
    const int t_own = ns == 3 ? 13 : cx + 2 * cy + 4 * cz;
    const int cell_off = cell - (cx + nc * (cy + nc * cz));
    const int *count = P.count[par];
    const Rep &R = P.reps[r];
    const float w32 = R.w32;
    const int has_dep = R.has_dep;
    const Sched *S = P.sched + r;

    // populations of the stencil; the own cell's lens data (slots 0 and 1)
    int c_nb = 0, m_nb = 0, dx = 0, dy = 0, dz = 0;
    if (tid < n_st) {
        c_nb = stencil_cell_nc(nc, cell_off, tid, cx, cy, cz, dx, dy, dz);
        m_nb = count[c_nb];
        if (tid == t_own) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const size_t bs = bin_at(P, c_nb, s);
                s_mv[s] = P.mv_bin[bs];
                s_hdr[s] = P.hdr_bin[bs];
#pragma unroll
                for (int j = 0; j < kLensInline; ++j)
                    s_lin[s][j] = P.lens_bin[bs * kLensInline + j];
            }
        }
        m_nb = min(m_nb, P.cap);
    }
    int n_own = 0, M = 0, base = 0;
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
        if (!WARP && tid == 0) {
            s_ncand = M;
            s_nacc = n_own;
        }
    }
    if (!WARP) {
        __syncthreads();
        M = s_ncand;
        n_own = s_nacc;
        __syncthreads();
    }
    if (n_own == 0) return;
    if (M > kMaxCand) {
        if (tid == 0) atomicCAS(P.err, kErrNone, kErrCandCap);
        return;
    }
    const uint32_t sweep = S->sweep;
    if (tid == 0) s_nacc = 0;
    // the previous phase's moves are visible from here on
    pdl_wait();
    // candidates (positions and FP32 orientations) relative to this cell's
    // origin; the own cell's entries beyond slot 1 with their lens data
    if (tid < n_st) {
        const float fx = (float)dx * w32, fy = (float)dy * w32, fz = (float)dz * w32;
        const bool own = tid == t_own;
        for (int s = 0; s < m_nb; ++s) {
            const size_t bs = bin_at(P, c_nb, s);
            const float4 e = P.bins[bs];
            const int slot = base + s;
            s_cpos[slot] = make_float4(fx + e.x, fy + e.y, fz + e.z, e.w);
            s_cq[slot] = P.bin_q[bs];
            if (own) {
                s_tmp_i[s] = __float_as_int(e.w);
                s_tmp_slot[s] = slot;
                if (s >= 2) {
                    s_mv[s] = P.mv_bin[bs];
                    s_hdr[s] = P.hdr_bin[bs];
                }
            }
        }
    }
    cta_sync<WARP>();
    // the cell's colloids in ascending index (the order they move in), and
    // where each one's lens points go (bin order)
    for (int q = tid; q < n_own; q += nthr) {
        const int v = s_tmp_i[q];
        int rk = 0;
        for (int u = 0; u < n_own; ++u) rk += s_tmp_i[u] < v ? 1 : 0;
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
        cta_sync<WARP>();
    }

    uint32_t c_acc = 0, c_cell = 0, c_ov = 0, c_dep = 0, c_cb = 0, c_eval = 0, c_block = 0,
             c_fwd = 0, c_rev = 0, c_cap = 0, c_rck = 0, c_tr = 0;
    unsigned long long c_drawn = 0;
    const float D2c = 2.0f * R.R_circ32;

    for (int q = 0; q < n_own; ++q) {
        const int i = s_own[q];
        const int nacc = s_nacc;
        const int qb = s_own_bin[q];
        const float4 ri = s_cpos[s_own_slot[q]];
        const float4 mv = s_mv[qb];
        const float kind = mv.w;
        if (kind < -0.5f) {          // rotation attempt stream capped: rejected
            if (tid == 0) ++c_cap;
            continue;
        }
        const bool translate = kind > 0.5f;
        if (translate) ++c_tr;
        const float rn0 = ri.x + mv.x, rn1 = ri.y + mv.y, rn2 = ri.z + mv.z;
        if (translate) {
            const float mc = R.m_cell, wc = R.w32;
            const bool out = rn0 < -mc || rn0 > wc + mc || rn1 < -mc || rn1 > wc + mc ||
                             rn2 < -mc || rn2 > wc + mc;
            const bool edge = rn0 <= mc || rn0 >= wc - mc || rn1 <= mc || rn1 >= wc - mc ||
                              rn2 <= mc || rn2 >= wc - mc;
            bool exits = out;
            if (!out && edge) {
                const double4 x = P.prop_pos[i];
                exits = cell_coord(x.x, S->sigma[0], R.L, R.w, R.nc) != cx ||
                        cell_coord(x.y, S->sigma[1], R.L, R.w, R.nc) != cy ||
                        cell_coord(x.z, S->sigma[2], R.L, R.w, R.nc) != cz;
                if (tid == 0) ++c_rck;
            }
            if (exits) {
                ++c_cell;
                continue;
            }
        }
        const float4 qo32 = s_cq[s_own_slot[q]];
        const float4 qn32 = translate ? qo32 : quat32(P.prop_quat[i]);
        const Frame32 Fo = frame32(qo32);
        const Frame32 Fn = translate ? Fo : frame32(qn32);
        const float3 o = make_float3(ri.x - rn0, ri.y - rn1, ri.z - rn2);

        // a4: colloid overlap at the new pose; neighbours in range
        if (!WARP) {
            if (tid == 0) s_nnb = 0;
            __syncthreads();
        }
        int ov = 0, nnb = 0;
        uint32_t st3 = 0;
        for (int j0 = 0; j0 < M; j0 += nthr) {
            const int j = j0 + tid;
            int t = 0, pj = -1;
            float d0 = 0.f, d1 = 0.f, d2 = 0.f, r2 = 1e30f;
            float4 qj = make_float4(1.f, 0.f, 0.f, 0.f);
            if (j < M) {
                const float4 cp = s_cpos[j];
                pj = __float_as_int(cp.w);
                if (pj == i) {
                    pj = -1;
                } else {
                    d0 = cp.x - rn0;
                    d1 = cp.y - rn1;
                    d2 = cp.z - rn2;
                    if (d0 > R.half_L32) d0 -= R.L32; else if (d0 < -R.half_L32) d0 += R.L32;
                    if (d1 > R.half_L32) d1 -= R.L32; else if (d1 < -R.half_L32) d1 += R.L32;
                    if (d2 > R.half_L32) d2 -= R.L32; else if (d2 < -R.half_L32) d2 += R.L32;
                    r2 = norm2f(d0, d1, d2);
                    qj = s_cq[j];
                    const float lim = D2c + R.m_pair;
                    if (r2 < lim * lim) {
                        Body32 A, B;
                        A.F = Fn;
                        A.x = make_float3(0.f, 0.f, 0.f);
                        B.F = frame32(qj);
                        B.x = make_float3(d0, d1, d2);
                        const PairTri pt = pair_tri32(R, A, B);
                        t = pt.res;
                        if constexpr (kChecked) {
                            // a decision taken as certain, against the FP64 statement
                            uint32_t st = 0;
                            if (t != -1)
                                (void)HPMC_CHECK_FAILS(
                                    P, exact_pair_aniso(P, R, i, pj, s_accl, nacc, pt.n, st) == (t == 1), 18);
                        }
                        if (t == -1) {
                            ++c_rck;
                            t = exact_pair_aniso(P, R, i, pj, s_accl, nacc, pt.n, st3) ? 1 : 0;
                        }
                    } else if (kChecked) {
                        // apart by more than the circumspheres and the margin
                        uint32_t st = 0;
                        (void)HPMC_CHECK_FAILS(P, !exact_pair_aniso(P, R, i, pj, s_accl, nacc,
                                                                    make_float3(-d0, -d1, -d2), st), 18);
                    }
                }
            }
            if (t == 1) ov = 1;
            const bool take = pj >= 0 && r2 < R.nb_cut2_32;
            if (WARP) {
                const unsigned b = __ballot_sync(kFull, take);
                const int slot = nnb + __popc(b & lt);
                if (take && slot < kMaxNbAniso) {
                    s_nb[slot].d = make_float4(d0, d1, d2, __int_as_float(pj));
                    s_nb[slot].F = frame32(qj);
                }
                nnb += __popc(b);
            } else if (take) {
                const int slot = atomicAdd(&s_nnb, 1);
                if (slot < kMaxNbAniso) {
                    s_nb[slot].d = make_float4(d0, d1, d2, __int_as_float(pj));
                    s_nb[slot].F = frame32(qj);
                }
            }
        }
        c_rck += st3;
        if (cta_any<WARP>(ov)) {
            ++c_ov;
            continue;
        }
        if (!WARP) nnb = s_nnb;
        if (nnb > kMaxNbAniso) {
            if (tid == 0) atomicCAS(P.err, kErrNone, kErrCandCap);
            return;
        }
        cta_sync<WARP>();

        bool accept = true;
        if (R.has_dep) {
            const int4 hd = s_hdr[qb];
            const int n_p = hd.x;
            c_drawn += (unsigned long long)n_p;
            DepOutcome od = {1.0, 0, 0, 0u, 0u, 0u, 0u, 0u, 0u};
            const int n_lens = hd.z;
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
                if (m < n_lens) {
                    const float4 Lm = lens[m];
                    const uint32_t tk = (uint32_t)__float_as_int(Lm.w);
                    kk = (int)(tk & 0xFFFFu);
                    tt = tk >> 16;
                    bool unsure = false, hit = false;
                    for (int b = 0; b < nnb; ++b) {
                        const float4 d = s_nb[b].d;
                        const int tn = dep_tri32(R, make_float3(Lm.x - d.x, Lm.y - d.y, Lm.z - d.z),
                                                 s_nb[b].F);
                        if (tn == 1) {
                            hit = true;
                            break;
                        }
                        unsure = unsure || tn == -1;
                    }
                    cls = hit ? 0 : (unsure ? -1 : 1);
                    if constexpr (kChecked) {
                        if (cls != -1)
                            (void)HPMC_CHECK_FAILS(
                                P, exact_free_nb_aniso(P, R, sweep, i, tt, s_nb, nnb, s_accl, nacc) == (cls == 1), 19);
                    }
                }
                {
                    const bool unsure = cls == -1;
                    if (__any_sync(kFull, unsure)) {
                        if (unsure) {
                            ++od.rck;
                            cls = exact_free_nb_aniso(P, R, sweep, i, tt, s_nb, nnb, s_accl, nacc) ? 1 : 0;
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
                        od.block += 1;
                        od.eval += (uint32_t)(kmin + 1);
                        od.rejected = 1;
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
                        const CbResult32 cr = cb_factor_aniso32(P, R, sweep, i, kb, o, Fn, Fo, s_nb, nnb,
                                                                s_accl, nacc);
                        od.rck += cr.rck;
                        if (lane == b) {
                            f = cr.f;
                            has = true;
                            zero = cr.fwd_ok == 0;
                            od.fwd += cr.fwd_ok;
                            od.rev += cr.rev_ok;
                            od.cap += cr.caps;
                        }
                        if (cr.fwd_ok == 0) break;
                    }
                    if (cb_pass(sh, tid, nthr, has, f, zero, kk, od, -1)) {
                        od.rejected = 1;
                        break;
                    }
                }
            }
            if (!od.rejected) {
                od.eval += (uint32_t)hd.y;
                if (hd.y < n_p && tid == 0) ++od.cap;
            }
            c_eval += od.eval;
            c_block += od.block;
            c_cap += od.cap;
            c_rck += od.rck;
            c_fwd += od.fwd;
            c_rev += od.rev;
            if (od.rejected) {
                accept = false;
                // (a replica without CB in a batch that has some: its first
                // blocking depletant rejects the move as a depletant rejection)
                if (!CB || R.n_trial == 0) ++c_dep;
                else ++c_cb;
            } else if (CB && tid == 0 && od.nblock > 0) {
                const uint4 wa = draw(R.key0, R.key1, sweep, (uint32_t)(i - R.off), kPAccept, 0, 0);
                if (!(u53(wa.x, wa.y) < od.W)) {
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
        // a8: the FP32 working copies move now, the exact pose at the CTA's end
        if (accept) {
            ++c_acc;
            if (tid == 0) {
                const float4 rnew = make_float4(rn0, rn1, rn2, __int_as_float(i));
                s_cpos[s_own_slot[q]] = rnew;
                s_cq[s_own_slot[q]] = qn32;
                if (translate) P.bins[bin_at(P, cell, qb)] = rnew;
                else P.bin_q[bin_at(P, cell, qb)] = qn32;
                s_accl[nacc] = i;
                s_nacc = nacc + 1;
            }
        }
        cta_sync<WARP>();
    }

    const int nacc = s_nacc;
    for (int a = tid; a < nacc; a += nthr) {
        const int j = s_accl[a];
        const double4 x = P.prop_pos[j];
        P.pos[j] = make_double4(x.x, x.y, x.z, 0.0);
        P.quat[j] = P.prop_quat[j];
    }

    unsigned long long cnt[kNumCounters] = {0};
    if (tid == 0) {
        cnt[kMoves] = (unsigned long long)n_own;
        cnt[kTranslate] = c_tr;
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

}  // namespace hpmc
