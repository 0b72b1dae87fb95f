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

// R * s11(w) in FP32: s11(w) = v 2^-31 + 2^-32 with v = (int)(w ^ 2^31); one
// rounding of v, one of the fma (r_hi = R 2^-31, r_lo = R 2^-32).
__device__ __forceinline__ float scaled_s11f(uint32_t w, float r_hi, float r_lo)
{
    return __fmaf_rn((float)(int)(w ^ 0x80000000u), r_hi, r_lo);
}

__device__ __forceinline__ float norm2f(float a, float b, float c)
{
    return __fmaf_rn(a, a, __fmaf_rn(b, b, c * c));
}

// 1: r2 < T certainly, 0: r2 >= T certainly, -1: inside the margin
__device__ __forceinline__ int tri(float r2, float T, float m)
{
    return r2 < T - m ? 1 : (r2 > T + m ? 0 : -1);
}

// --- exact FP64 re-takes, as the specification states them -----------------
//
// They run rarely and out of line (behind warp votes), and recompute what
// they need: the move words are re-drawn and FP64 positions re-read.  Moves
// accepted by this CTA are committed to FP64 only when the CTA finishes, so a
// colloid of the list acc[0..nacc) is at its moved position.

// Exact FP64 position of colloid j after its move of this sweep.
__device__ __forceinline__ double4 moved64(const SimParams &P, uint32_t sweep, int j)
{
    const uint4 wm = draw(P.key0, P.key1, sweep, (uint32_t)j, kPMove, 0, 0);
    const double4 p = P.pos[j];
    return make_double4(wrap_box(p.x + P.d_max * s11(wm.x), P.L),
                        wrap_box(p.y + P.d_max * s11(wm.y), P.L),
                        wrap_box(p.z + P.d_max * s11(wm.z), P.L), 0.0);
}

__device__ __forceinline__ double4 pos_now(const SimParams &P, uint32_t sweep, int j,
                                           const int *acc, int nacc)
{
    for (int a = 0; a < nacc; ++a)
        if (acc[a] == j) return moved64(P, sweep, j);
    return P.pos[j];
}

struct Move64 {
    double x0, x1, x2;  // new position, wrapped into [0, L)
    double o0, o1, o2;  // old position relative to the new one (minimum image)
};

__device__ __forceinline__ Move64 move64(const SimParams &P, uint32_t sweep, int i)
{
    const double4 pi = P.pos[i];
    const double4 x = moved64(P, sweep, i);
    Move64 m;
    m.x0 = x.x;
    m.x1 = x.y;
    m.x2 = x.z;
    m.o0 = min_image(pi.x - m.x0, P.L, P.half_L);
    m.o1 = min_image(pi.y - m.x1, P.L, P.half_L);
    m.o2 = min_image(pi.z - m.x2, P.L, P.half_L);
    return m;
}

__device__ __forceinline__ void center64(const SimParams &P, const Move64 &m, double4 pj,
                                         double &c0, double &c1, double &c2)
{
    c0 = min_image(pj.x - m.x0, P.L, P.half_L);
    c1 = min_image(pj.y - m.x1, P.L, P.half_L);
    c2 = min_image(pj.z - m.x2, P.L, P.half_L);
}

__device__ __noinline__ bool exact_cell_exit(const SimParams &P, uint32_t sweep, int i, int cx,
                                             int cy, int cz)
{
    const double4 x = moved64(P, sweep, i);
    const Sched *S = P.sched;
    return cell_coord(x.x, S->sigma[0], P.L, P.w, P.nc) != cx ||
           cell_coord(x.y, S->sigma[1], P.L, P.w, P.nc) != cy ||
           cell_coord(x.z, S->sigma[2], P.L, P.w, P.nc) != cz;
}

// colloid i at its new position overlaps colloid j
__device__ __noinline__ bool exact_pair(const SimParams &P, uint32_t sweep, int i, int j,
                                        const int *acc, int nacc)
{
    const Move64 m = move64(P, sweep, i);
    double c0, c1, c2;
    center64(P, m, pos_now(P, sweep, j, acc, nacc), c0, c1, c2);
    return norm2(c0, c1, c2) < P.contact2;
}

__device__ __noinline__ bool exact_ball(const SimParams &P, uint4 w)
{
    const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
    return norm2(e0, e1, e2) < P.R_s2;
}

// Exact test of a depletant point against one colloid.
//   what 0: point e (around the new reference point) vs the old pose
//   what 1: forward CB trial y = o + e (around the old reference point) vs the new pose
//   what 2: point e vs neighbour j
//   what 3: forward CB trial y = o + e vs neighbour j
__device__ __noinline__ bool exact_dep(const SimParams &P, uint32_t sweep, int i, uint4 w, int what,
                                       int j, const int *acc, int nacc)
{
    const Move64 m = move64(P, sweep, i);
    const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
    double v0 = e0, v1 = e1, v2 = e2;
    if (what == 1 || what == 3) {
        v0 = m.o0 + e0;
        v1 = m.o1 + e1;
        v2 = m.o2 + e2;
    }
    if (what == 0) return SphereFP64::dep(P, v0 - m.o0, v1 - m.o1, v2 - m.o2);
    if (what == 1) return SphereFP64::dep(P, v0, v1, v2);
    double c0, c1, c2;
    center64(P, m, pos_now(P, sweep, j, acc, nacc), c0, c1, c2);
    return SphereFP64::dep(P, v0 - c0, v1 - c1, v2 - c2);
}

// A lens point (attempt t of the depletant stream) free of every neighbour?
__device__ __noinline__ bool exact_free_nb(const SimParams &P, uint32_t sweep, int i, uint32_t t,
                                           const float4 *nb, int nnb, const int *acc, int nacc)
{
    const uint4 w = draw(P.key0, P.key1, sweep, (uint32_t)i, kPDep, 0, t);
    for (int a = 0; a < nnb; ++a)
        if (exact_dep(P, sweep, i, w, 2, __float_as_int(nb[a].w), acc, nacc)) return false;
    return true;
}

// --- FP32 tests with exact fallback -----------------------------------------

// Is v (FP32, relative to the new reference point) free of every neighbour?
// kind 2: v is a point e; kind 3: v is a forward trial o + e.
__device__ __forceinline__ bool free_nb32(const SimParams &P, float v0, float v1, float v2,
                                          const float4 *nb, int nnb, uint32_t sweep, int i,
                                          uint4 w, int kind, const int *acc, int nacc,
                                          uint32_t &rck)
{
    for (int a = 0; a < nnb; ++a) {
        const float4 d = nb[a];
        const int t = tri(norm2f(v0 - d.x, v1 - d.y, v2 - d.z), P.T_dep32, P.m_r2);
        if (t == 1) return false;
        if (t == -1) {
            ++rck;
            if (exact_dep(P, sweep, i, w, kind, __float_as_int(d.w), acc, nacc)) return false;
        }
    }
    return true;
}

// Next point of an attempt stream inside the sampling ball.
__device__ __forceinline__ bool next_in_ball32(const SimParams &P, uint32_t sweep, uint32_t tag,
                                               uint32_t purpose, uint32_t sub, uint32_t &t,
                                               uint32_t t_max, float r_hi, float r_lo, uint4 &w,
                                               float &e0, float &e1, float &e2, uint32_t &rck)
{
    while (t < t_max) {
        w = draw(P.key0, P.key1, sweep, tag, purpose, sub, t);
        ++t;
        e0 = scaled_s11f(w.x, r_hi, r_lo);
        e1 = scaled_s11f(w.y, r_hi, r_lo);
        e2 = scaled_s11f(w.z, r_hi, r_lo);
        int in = tri(norm2f(e0, e1, e2), P.T_s32, P.m_r2);
        if (in == -1) {
            ++rck;
            in = exact_ball(P, w) ? 1 : 0;
        }
        if (in) return true;
    }
    return false;
}

struct CbResult32 {
    double f;
    uint32_t fwd_ok, rev_ok, caps, rck;
};

// CB factor of one blocking depletant (Sec. III.D, Eq. 12), FP32 form.  For
// spheres "overlaps the pose the ball is centred on" is the ball test itself.
__device__ __noinline__ CbResult32 cb_factor_fp32(const SimParams &P, uint32_t sweep, int i,
                                                  uint32_t k, float o0, float o1, float o2,
                                                  const float4 *nb, int nnb, const int *acc,
                                                  int nacc, float r_hi, float r_lo)
{
    CbResult32 r = {0.0, 0u, 0u, 0u, 0u};
    const uint32_t tag = (uint32_t)i;
    const int n_fwd = P.n_trial, n_rev = P.n_trial - 1;
    int nf = 0, nr = 0, found = 0;
    uint32_t t = 0;
    uint4 w;
    float e0, e1, e2;
    while (found < n_fwd && next_in_ball32(P, sweep, tag, kPCbFwd, k, t, 64u * (uint32_t)(n_fwd + 1),
                                           r_hi, r_lo, w, e0, e1, e2, r.rck)) {
        ++found;
        const float y0 = o0 + e0, y1 = o1 + e1, y2 = o2 + e2;
        int tn = tri(norm2f(y0, y1, y2), P.T_dep32, P.m_r2);  // overlaps the new pose?
        if (tn == -1) {
            ++r.rck;
            tn = exact_dep(P, sweep, i, w, 1, 0, acc, nacc) ? 1 : 0;
        }
        if (tn) continue;
        if (!free_nb32(P, y0, y1, y2, nb, nnb, sweep, i, w, 3, acc, nacc, r.rck)) continue;
        ++nf;
    }
    if (found < n_fwd) ++r.caps;
    t = 0;
    found = 0;
    while (found < n_rev && next_in_ball32(P, sweep, tag, kPCbRev, k, t, 64u * (uint32_t)(n_rev + 1),
                                           r_hi, r_lo, w, e0, e1, e2, r.rck)) {
        ++found;
        int to = tri(norm2f(e0 - o0, e1 - o1, e2 - o2), P.T_dep32, P.m_r2);  // old pose?
        if (to == -1) {
            ++r.rck;
            to = exact_dep(P, sweep, i, w, 0, 0, acc, nacc) ? 1 : 0;
        }
        if (to) continue;
        if (!free_nb32(P, e0, e1, e2, nb, nnb, sweep, i, w, 2, acc, nacc, r.rck)) continue;
        ++nr;
    }
    if (found < n_rev) ++r.caps;
    r.fwd_ok = (uint32_t)nf;
    r.rev_ok = (uint32_t)nr;
    r.f = (double)nf / (double)(nr + 1);
    return r;
}

// Classify one depletant point e (FP32 first, exact where needed): blocking
// iff it is not in the old pose's excluded volume nor any neighbour's (it is in
// the new pose's, being inside the ball).  Returns 1 blocking, 0 not.
__device__ __noinline__ int exact_classify(const SimParams &P, uint32_t sweep, int i, uint4 w,
                                           const float4 *nb, int nnb, const int *acc, int nacc)
{
    if (exact_dep(P, sweep, i, w, 0, 0, acc, nacc)) return 0;
    for (int a = 0; a < nnb; ++a)
        if (exact_dep(P, sweep, i, w, 2, __float_as_int(nb[a].w), acc, nacc)) return 0;
    return 1;
}

// ---------------------------------------------------------------------------
// Depletant lens lists (Sec. III.B-C), one warp per colloid, all colloids of
// the sweep at once.  Everything about a move's depletants that does not
// involve other colloids is fixed by the move's own random streams: the
// proposal, N_p, the points of the attempt stream, "inside the new pose's
// circumsphere" (= overlaps the new pose, for spheres) and "overlaps the old
// pose".  Only the points left after those tests, the lens of the move, can
// block it, and only they need the neighbours, which the colour phases test
// in order.  Moves that certainly leave their cell draw nothing.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_lens_sphere_fp32(const __grid_constant__ SimParams P)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= P.n) return;
    const uint32_t sweep = P.sched->sweep;
    const uint32_t tag = (uint32_t)i;
    const float dm_hi = P.d_max32 * 0x1p-31f, dm_lo = P.d_max32 * 0x1p-32f;
    const float r_hi = P.R_s32 * 0x1p-31f, r_lo = P.R_s32 * 0x1p-32f;
    const uint4 wm = draw(P.key0, P.key1, sweep, tag, kPMove, 0, 0);
    const float D0 = scaled_s11f(wm.x, dm_hi, dm_lo);
    const float D1 = scaled_s11f(wm.y, dm_hi, dm_lo);
    const float D2 = scaled_s11f(wm.z, dm_hi, dm_lo);
    {
        // the same FP32 expression the colour phase uses for the cell-exit test
        const float4 ri = P.rel[i];
        const float rn0 = ri.x + D0, rn1 = ri.y + D1, rn2 = ri.z + D2;
        const float mc = P.m_cell, wc = P.w32;
        if (rn0 < -mc || rn0 > wc + mc || rn1 < -mc || rn1 > wc + mc || rn2 < -mc ||
            rn2 > wc + mc) {
            if (lane == 0) P.lens_hdr[i] = make_int4(0, 0, 0, 0);
            return;
        }
    }
    uint32_t rck = 0;
    const float o0 = -D0, o1 = -D1, o2 = -D2;
    const uint4 wp = draw(P.key0, P.key1, sweep, tag, kPPoisson, 0, 0);
    const int n_p = poisson_count(P.T, P.nF, u53_int(wp.x, wp.y), lane);
    const uint32_t t_max = 64u * (uint32_t)(n_p + 1);
    float4 *out = P.lens + (size_t)i * P.lens_cap;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t t0 = 0;
    int k0 = 0, m = 0;
    while (k0 < n_p && t0 < t_max) {
        const uint32_t t = t0 + (uint32_t)lane;
        uint4 w = make_uint4(0, 0, 0, 0);
        float e0 = 0.f, e1 = 0.f, e2 = 0.f;
        int in = 0;
        if (t < t_max) {
            w = draw(P.key0, P.key1, sweep, tag, kPDep, 0, t);
            e0 = scaled_s11f(w.x, r_hi, r_lo);
            e1 = scaled_s11f(w.y, r_hi, r_lo);
            e2 = scaled_s11f(w.z, r_hi, r_lo);
            in = tri(norm2f(e0, e1, e2), P.T_s32, P.m_r2);
        }
        {
            const bool unsure = in == -1;
            if (__any_sync(kFull, unsure)) {
                if (unsure) {
                    ++rck;
                    in = exact_ball(P, w) ? 1 : 0;
                }
            }
        }
        const unsigned bal = __ballot_sync(kFull, in == 1);
        const int k = k0 + __popc(bal & lt);
        const bool dep = in == 1 && k < n_p;
        int to = 1;  // overlaps the old pose: 1 yes, 0 no, -1 within the margin
        if (dep) to = tri(norm2f(e0 - o0, e1 - o1, e2 - o2), P.T_dep32, P.m_r2);
        {
            const bool unsure = to == -1;
            if (__any_sync(kFull, unsure)) {
                if (unsure) {
                    ++rck;
                    to = exact_dep(P, sweep, i, w, 0, 0, nullptr, 0) ? 1 : 0;
                }
            }
        }
        const bool lens = dep && to == 0;
        const unsigned lb = __ballot_sync(kFull, lens);
        const int slot = m + __popc(lb & lt);
        if (lens && slot < P.lens_cap)
            out[slot] = make_float4(e0, e1, e2, __int_as_float((int)((t << 16) | (uint32_t)k)));
        m += __popc(lb);
        k0 += __popc(bal);
        t0 += 32u;
    }
    if (lane == 0) P.lens_hdr[i] = make_int4(n_p, min(k0, n_p), m <= P.lens_cap ? m : -1, 0);
    rck = __reduce_add_sync(kFull, rck);
    if (lane == 0 && rck)
        atomicAdd(P.counters + (size_t)(i % kCounterSlots) * kNumCounters + kRechecks,
                  (unsigned long long)rck);
}

// ILP: attempts each thread carries per pass (independent Philox chains);
// the pass covers ILP * blockDim attempts of the stream, in order.
template <int ILP>
__global__ void __launch_bounds__(kMaxThreads, 2)
    k_phase_sphere_fp32(const __grid_constant__ SimParams P, int phase)
{
    __shared__ int s_own[kMaxCellCap], s_tmp[kMaxCellCap], s_accl[kMaxCellCap];
    __shared__ float4 s_cpos[kMaxCand];  // candidates relative to this cell's origin; index in .w
    __shared__ float4 s_nb[kMaxCand];    // neighbours relative to the new position; index in .w
    __shared__ double s_f[ILP * kMaxThreads];
    __shared__ int s_k[ILP * kMaxThreads];
    __shared__ int s_warp[ILP][kMaxThreads / 32];
    __shared__ int s_ncand, s_nnb, s_flag, s_acc, s_kmin, s_self, s_nacc;

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const Sched S = *P.sched;
    if (phase == 7 && blockIdx.x == 0 && tid == 0) atomicAdd(P.sweep, 1ull);
    const uint32_t sweep = S.sweep;
    const CellTask T = cell_task(P, S, phase);
    clear_next(P, S, T.cell);
    const int n_own = min(T.n_own, P.cap);
    if (n_own == 0) return;
    own_members_sorted(P, T.cell, n_own, s_tmp, s_own);
    const int cx = T.cx, cy = T.cy, cz = T.cz;

    // candidates of the 27-cell stencil, relative to this cell's origin
    if (tid == 0) {
        s_ncand = 0;
        s_nacc = 0;
    }
    __syncthreads();
    if (tid < P.n_stencil * P.n_stencil * P.n_stencil) {
        int dx, dy, dz;
        const int c = stencil_cell(P, tid, cx, cy, cz, dx, dy, dz);
        const float fx = (float)dx * P.w32, fy = (float)dy * P.w32, fz = (float)dz * P.w32;
        const int m = min(T.count[c], P.cap);
        for (int s = 0; s < m; ++s) {
            const int j = P.bins[(size_t)c * P.cap + s];
            const float4 r = P.rel[j];
            const int slot = atomicAdd(&s_ncand, 1);
            if (slot < kMaxCand)
                s_cpos[slot] = make_float4(fx + r.x, fy + r.y, fz + r.z, __int_as_float(j));
        }
    }
    __syncthreads();
    const int M = s_ncand;
    if (M > kMaxCand) {
        if (tid == 0) atomicCAS(P.err, kErrNone, kErrCandCap);
        return;
    }
    const float r_hi = P.R_s32 * 0x1p-31f, r_lo = P.R_s32 * 0x1p-32f;
    const float dm_hi = P.d_max32 * 0x1p-31f, dm_lo = P.d_max32 * 0x1p-32f;

    // uniform counters (taken by thread 0) and per-thread ones
    uint32_t c_moves = 0, c_acc = 0, c_cell = 0, c_ov = 0, c_dep = 0, c_cb = 0, c_eval = 0,
             c_block = 0, c_fwd = 0, c_rev = 0, c_cap = 0, c_rck = 0;
    unsigned long long c_drawn = 0;

    for (int q = 0; q < n_own; ++q) {
        const int i = s_own[q];
        const uint32_t tag = (uint32_t)i;
        const int nacc = s_nacc;
        ++c_moves;
        float rn0, rn1, rn2;
        const float4 ri = P.rel[i];
        {
            const uint4 wm = draw(P.key0, P.key1, sweep, tag, kPMove, 0, 0);
            rn0 = ri.x + scaled_s11f(wm.x, dm_hi, dm_lo);
            rn1 = ri.y + scaled_s11f(wm.y, dm_hi, dm_lo);
            rn2 = ri.z + scaled_s11f(wm.z, dm_hi, dm_lo);
        }
        // a3: cell-exit check with margin (exact when within it)
        const float mc = P.m_cell, wc = P.w32;
        const bool out = rn0 < -mc || rn0 > wc + mc || rn1 < -mc || rn1 > wc + mc ||
                         rn2 < -mc || rn2 > wc + mc;
        const bool edge = rn0 <= mc || rn0 >= wc - mc || rn1 <= mc || rn1 >= wc - mc ||
                          rn2 <= mc || rn2 >= wc - mc;
        bool exits = out;
        if (!out && edge) {
            exits = exact_cell_exit(P, sweep, i, cx, cy, cz);
            if (tid == 0) ++c_rck;
        }
        if (exits) {
            ++c_cell;
            continue;
        }
        const float o0 = ri.x - rn0, o1 = ri.y - rn1, o2 = ri.z - rn2;

        // a4: colloid overlap at the new pose; neighbours in range
        if (tid == 0) {
            s_nnb = 0;
            s_kmin = 0x7FFFFFFF;
        }
        __syncthreads();
        int ov = 0;
        for (int j0 = 0; j0 < M; j0 += nthr) {
            const int j = j0 + tid;
            int t = 0, pj = -1;
            float d0 = 0.f, d1 = 0.f, d2 = 0.f, r2 = 1e30f;
            if (j < M) {
                const float4 cp = s_cpos[j];
                pj = __float_as_int(cp.w);
                if (pj == i) {
                    s_self = j;
                    pj = -1;
                } else {
                    d0 = cp.x - rn0;
                    d1 = cp.y - rn1;
                    d2 = cp.z - rn2;
                    if (d0 > P.half_L32) d0 -= P.L32; else if (d0 < -P.half_L32) d0 += P.L32;
                    if (d1 > P.half_L32) d1 -= P.L32; else if (d1 < -P.half_L32) d1 += P.L32;
                    if (d2 > P.half_L32) d2 -= P.L32; else if (d2 < -P.half_L32) d2 += P.L32;
                    r2 = norm2f(d0, d1, d2);
                    t = tri(r2, P.T_contact32, P.m_r2);
                }
            }
            const bool unsure = t == -1;
            if (__any_sync(kFull, unsure)) {
                if (unsure) {
                    ++c_rck;
                    t = exact_pair(P, sweep, i, pj, s_accl, nacc) ? 1 : 0;
                }
            }
            if (t == 1) ov = 1;
            if (pj >= 0 && r2 < P.nb_cut2_32) {
                const int slot = atomicAdd(&s_nnb, 1);
                s_nb[slot] = make_float4(d0, d1, d2, __int_as_float(pj));
            }
        }
        if (__syncthreads_or(ov)) {
            ++c_ov;
            continue;
        }
        const int nnb = s_nnb;

        bool accept = true;
        if (P.has_dep) {
            // a5: N_p and the lens points come from the lens kernel
            const int4 hd = P.lens_hdr[i];
            const int n_p = hd.x;
            c_drawn += (unsigned long long)n_p;
            int nblock = 0;
            double W = 1.0;
            bool rejected = false;
            if (hd.z >= 0) {
                // a6: the lens points in depletant order; one free of every neighbour
                // blocks the move
                const int n_lens = hd.z;
                const float4 *lens = P.lens + (size_t)i * P.lens_cap;
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
                            const float4 d = s_nb[b];
                            const int tn = tri(norm2f(Lm.x - d.x, Lm.y - d.y, Lm.z - d.z),
                                               P.T_dep32, P.m_r2);
                            if (tn == 1) {
                                hit = true;
                                break;
                            }
                            unsure = unsure || tn == -1;
                        }
                        cls = hit ? 0 : (unsure ? -1 : 1);
                    }
                    {
                        const bool unsure = cls == -1;
                        if (__any_sync(kFull, unsure)) {
                            if (unsure) {
                                ++c_rck;
                                cls = exact_free_nb(P, sweep, i, tt, s_nb, nnb, s_accl, nacc) ? 1
                                                                                              : 0;
                            }
                        }
                    }
                    const bool blocking = cls == 1;
                    if (P.n_trial == 0) {
                        if (blocking) atomicMin(&s_kmin, kk);
                        if (__syncthreads_or(blocking)) {
                            ++c_block;
                            c_eval += (uint32_t)(s_kmin + 1);
                            rejected = true;
                            break;
                        }
                    } else {
                        double f = -1.0;
                        if (blocking) {
                            const CbResult32 r = cb_factor_fp32(P, sweep, i, (uint32_t)kk, o0, o1,
                                                                o2, s_nb, nnb, s_accl, nacc, r_hi,
                                                                r_lo);
                            f = r.f;
                            c_fwd += r.fwd_ok;
                            c_rev += r.rev_ok;
                            c_cap += r.caps;
                            c_rck += r.rck;
                        }
                        s_f[tid] = f;
                        s_k[tid] = kk;
                        __syncthreads();
                        if (tid == 0) {
                            int zero = 0;
                            for (int u = 0; u < nthr; ++u) {
                                const double fu = s_f[u];
                                if (fu < 0.0) continue;
                                ++nblock;
                                ++c_block;
                                if (fu == 0.0) {
                                    zero = 1;
                                    c_eval += (uint32_t)(s_k[u] + 1);
                                    break;
                                }
                                W = W * fu;
                            }
                            s_flag = zero;
                        }
                        __syncthreads();
                        if (s_flag) {
                            rejected = true;
                            break;
                        }
                    }
                }
                if (!rejected) {
                    c_eval += (uint32_t)hd.y;
                    if (hd.y < n_p && tid == 0) ++c_cap;
                }
            } else {
            // a6 (lens list overflowed): the whole attempt stream, ILP * nthr
            // attempts per pass
            const uint32_t t_max = 64u * (uint32_t)(n_p + 1);
            const uint32_t per_pass = (uint32_t)(ILP * nthr);
            uint32_t t0 = 0;
            int k0 = 0;
            while (k0 < n_p && t0 < t_max) {
                uint4 w[ILP];
                float e0[ILP], e1[ILP], e2[ILP];
                int in[ILP];
#pragma unroll
                for (int a = 0; a < ILP; ++a) {
                    const uint32_t t = t0 + (uint32_t)(a * nthr + tid);
                    w[a] = make_uint4(0, 0, 0, 0);
                    e0[a] = e1[a] = e2[a] = 0.f;
                    in[a] = 0;
                    if (t < t_max) {
                        w[a] = draw(P.key0, P.key1, sweep, tag, kPDep, 0, t);
                        e0[a] = scaled_s11f(w[a].x, r_hi, r_lo);
                        e1[a] = scaled_s11f(w[a].y, r_hi, r_lo);
                        e2[a] = scaled_s11f(w[a].z, r_hi, r_lo);
                        in[a] = tri(norm2f(e0[a], e1[a], e2[a]), P.T_s32, P.m_r2);
                    }
                }
#pragma unroll
                for (int a = 0; a < ILP; ++a) {
                    const bool unsure = in[a] == -1;
                    if (__any_sync(kFull, unsure)) {
                        if (unsure) {
                            ++c_rck;
                            in[a] = exact_ball(P, w[a]) ? 1 : 0;
                        }
                    }
                }
                // depletant index of each inside attempt: prefix over the pass
                int k[ILP], total = 0;
                unsigned bal[ILP];
#pragma unroll
                for (int a = 0; a < ILP; ++a) bal[a] = __ballot_sync(kFull, in[a] == 1);
                if (nwarps > 1) {
                    if (lane == 0) {
#pragma unroll
                        for (int a = 0; a < ILP; ++a) s_warp[a][warp] = __popc(bal[a]);
                    }
                    __syncthreads();
#pragma unroll
                    for (int a = 0; a < ILP; ++a) {
                        int base = 0, tot = 0;
                        for (int u = 0; u < nwarps; ++u) {
                            const int c = s_warp[a][u];
                            base += u < warp ? c : 0;
                            tot += c;
                        }
                        k[a] = k0 + total + base + __popc(bal[a] & ((1u << lane) - 1u));
                        total += tot;
                    }
                } else {
#pragma unroll
                    for (int a = 0; a < ILP; ++a) {
                        k[a] = k0 + total + __popc(bal[a] & ((1u << lane) - 1u));
                        total += __popc(bal[a]);
                    }
                }
                // inside the ball = overlaps the new pose (spheres).  Blocking iff it
                // overlaps neither the old pose nor a neighbour: 1 yes, 0 no, -1 unsure
                int cls[ILP];
#pragma unroll
                for (int a = 0; a < ILP; ++a) {
                    cls[a] = 0;
                    if (in[a] == 1 && k[a] < n_p) {
                        const int to = tri(norm2f(e0[a] - o0, e1[a] - o1, e2[a] - o2), P.T_dep32,
                                           P.m_r2);
                        if (to != 1) {
                            bool unsure = to == -1, hit = false;
                            for (int b = 0; b < nnb; ++b) {
                                const float4 d = s_nb[b];
                                const int tn = tri(norm2f(e0[a] - d.x, e1[a] - d.y, e2[a] - d.z),
                                                   P.T_dep32, P.m_r2);
                                if (tn == 1) {
                                    hit = true;
                                    break;
                                }
                                unsure = unsure || tn == -1;
                            }
                            cls[a] = hit ? 0 : (unsure ? -1 : 1);
                        }
                    }
                }
#pragma unroll
                for (int a = 0; a < ILP; ++a) {
                    const bool unsure = cls[a] == -1;
                    if (__any_sync(kFull, unsure)) {
                        if (unsure) {
                            ++c_rck;
                            cls[a] = exact_classify(P, sweep, i, w[a], s_nb, nnb, s_accl, nacc);
                        }
                    }
                }
                if (P.n_trial == 0) {
                    bool any = false;
#pragma unroll
                    for (int a = 0; a < ILP; ++a) {
                        if (cls[a] == 1) {
                            atomicMin(&s_kmin, k[a]);
                            any = true;
                        }
                    }
                    if (__syncthreads_or(any)) {
                        ++c_block;
                        c_eval += (uint32_t)(s_kmin - k0 + 1);
                        rejected = true;
                        break;
                    }
                    c_eval += (uint32_t)min(total, n_p - k0);
                } else {
#pragma unroll
                    for (int a = 0; a < ILP; ++a) {
                        double f = -1.0;
                        if (cls[a] == 1) {
                            const CbResult32 r = cb_factor_fp32(P, sweep, i, (uint32_t)k[a], o0, o1,
                                                                o2, s_nb, nnb, s_accl, nacc, r_hi,
                                                                r_lo);
                            f = r.f;
                            c_fwd += r.fwd_ok;
                            c_rev += r.rev_ok;
                            c_cap += r.caps;
                            c_rck += r.rck;
                        }
                        s_f[a * nthr + tid] = f;
                        s_k[a * nthr + tid] = k[a];
                    }
                    __syncthreads();
                    if (tid == 0) {
                        // slots in attempt order = ascending depletant index
                        int zero = 0;
                        for (int u = 0; u < ILP * nthr; ++u) {
                            const double fu = s_f[u];
                            if (fu < 0.0) continue;
                            ++nblock;
                            ++c_block;
                            if (fu == 0.0) {
                                zero = 1;
                                c_eval += (uint32_t)(s_k[u] - k0 + 1);
                                break;
                            }
                            W = W * fu;
                        }
                        if (!zero) c_eval += (uint32_t)min(total, n_p - k0);
                        s_flag = zero;
                    }
                    __syncthreads();
                    if (s_flag) {
                        rejected = true;
                        break;
                    }
                }
                k0 += total;
                t0 += per_pass;
            }
            if (!rejected && k0 < n_p && tid == 0) ++c_cap;
            }
            if (rejected) {
                accept = false;
                if (P.n_trial == 0) ++c_dep;
                else ++c_cb;
            } else if (P.n_trial > 0 && tid == 0 && nblock > 0) {
                const uint4 wa = draw(P.key0, P.key1, sweep, tag, kPAccept, 0, 0);
                if (!(u53(wa.x, wa.y) < W)) {
                    accept = false;
                    ++c_cb;
                }
            }
            if (P.n_trial > 0) {
                if (tid == 0) s_acc = accept ? 1 : 0;
                __syncthreads();
                accept = s_acc != 0;
            }
        }
        // a8: accepted: the FP32 working copies move now, the FP64 position
        // when this CTA finishes
        if (accept) {
            ++c_acc;
            if (tid == 0) {
                const float4 rnew = make_float4(rn0, rn1, rn2, __int_as_float(i));
                s_cpos[s_self] = rnew;
                P.rel[i] = make_float4(rn0, rn1, rn2, 0.0f);
                s_accl[s_nacc] = i;
                s_nacc = nacc + 1;
            }
        }
        __syncthreads();
    }

    // deferred FP64 commit of the accepted moves, one colloid per lane
    const int nacc = s_nacc;
    for (int a = tid; a < nacc; a += nthr) {
        const int j = s_accl[a];
        P.pos[j] = moved64(P, sweep, j);
    }

    unsigned long long cnt[kNumCounters] = {0};
    if (tid == 0) {
        cnt[kMoves] = c_moves;
        cnt[kTranslate] = c_moves;
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
    flush_counters(P, cnt);
}

}  // namespace hpmc
