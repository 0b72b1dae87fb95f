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

struct Move64 {
    double x0, x1, x2;  // new position, wrapped into [0, L)
    double o0, o1, o2;  // old position relative to the new one (minimum image)
};

__device__ __forceinline__ Move64 move64(const SimParams &P, int i, uint4 wm)
{
    const double4 pi = P.pos[i];
    Move64 m;
    m.x0 = wrap_box(pi.x + P.d_max * s11(wm.x), P.L);
    m.x1 = wrap_box(pi.y + P.d_max * s11(wm.y), P.L);
    m.x2 = wrap_box(pi.z + P.d_max * s11(wm.z), P.L);
    m.o0 = min_image(pi.x - m.x0, P.L, P.half_L);
    m.o1 = min_image(pi.y - m.x1, P.L, P.half_L);
    m.o2 = min_image(pi.z - m.x2, P.L, P.half_L);
    return m;
}

__device__ __forceinline__ bool exact_cell_exit(const SimParams &P, int i, uint4 wm, int cx, int cy,
                                             int cz)
{
    const Move64 m = move64(P, i, wm);
    const Sched *S = P.sched;
    return cell_coord(m.x0, S->sigma[0], P.L, P.w, P.nc) != cx ||
           cell_coord(m.x1, S->sigma[1], P.L, P.w, P.nc) != cy ||
           cell_coord(m.x2, S->sigma[2], P.L, P.w, P.nc) != cz;
}

// colloid i at its new position overlaps colloid j
__device__ __forceinline__ bool exact_pair(const SimParams &P, int i, uint4 wm, int j)
{
    const Move64 m = move64(P, i, wm);
    const double4 pj = P.pos[j];
    return norm2(min_image(pj.x - m.x0, P.L, P.half_L), min_image(pj.y - m.x1, P.L, P.half_L),
                 min_image(pj.z - m.x2, P.L, P.half_L)) < P.contact2;
}

__device__ __forceinline__ bool exact_ball(const SimParams &P, uint4 w)
{
    const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
    return norm2(e0, e1, e2) < P.R_s2;
}

// point e (sampled around the new reference point) vs the old pose
__device__ __forceinline__ bool exact_dep_old(const SimParams &P, uint4 w, int i, uint4 wm)
{
    const Move64 m = move64(P, i, wm);
    const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
    return SphereFP64::dep(P, e0 - m.o0, e1 - m.o1, e2 - m.o2);
}

// forward CB trial y = o + e (sampled around the old reference point) vs the new pose
__device__ __forceinline__ bool exact_fwd_new(const SimParams &P, uint4 w, int i, uint4 wm)
{
    const Move64 m = move64(P, i, wm);
    const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
    const double y0 = m.o0 + e0, y1 = m.o1 + e1, y2 = m.o2 + e2;
    return SphereFP64::dep(P, y0, y1, y2);
}

// kind 0: point e vs neighbour j; kind 1: forward trial y = o + e vs neighbour j
__device__ __forceinline__ bool exact_dep_nb(const SimParams &P, uint4 w, int kind, int i, uint4 wm,
                                          int j)
{
    const Move64 m = move64(P, i, wm);
    const double4 pj = P.pos[j];
    const double d0 = min_image(pj.x - m.x0, P.L, P.half_L);
    const double d1 = min_image(pj.y - m.x1, P.L, P.half_L);
    const double d2 = min_image(pj.z - m.x2, P.L, P.half_L);
    const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
    if (kind == 0) return SphereFP64::dep(P, e0 - d0, e1 - d1, e2 - d2);
    const double y0 = m.o0 + e0, y1 = m.o1 + e1, y2 = m.o2 + e2;
    return SphereFP64::dep(P, y0 - d0, y1 - d1, y2 - d2);
}

// a8: commit the accepted move in FP64; returns the new FP32 cell offset (index in .w)
__device__ __forceinline__ float4 commit_move(const SimParams &P, int i, uint4 wm, int cx, int cy,
                                           int cz)
{
    const Move64 m = move64(P, i, wm);
    const Sched *S = P.sched;
    P.pos[i] = make_double4(m.x0, m.x1, m.x2, 0.0);
    const float4 r = make_float4(cell_rel(m.x0, S->sigma[0], P.L, P.w, cx),
                                 cell_rel(m.x1, S->sigma[1], P.L, P.w, cy),
                                 cell_rel(m.x2, S->sigma[2], P.L, P.w, cz), __int_as_float(i));
    P.rel[i] = make_float4(r.x, r.y, r.z, 0.0f);
    return r;
}

// --- FP32 tests with exact fallback -----------------------------------------

// Is v (FP32, relative to the new reference point) free of every neighbour?
__device__ __forceinline__ bool free_nb32(const SimParams &P, float v0, float v1, float v2,
                                          const float4 *nb, int nnb, uint4 w, int kind, int i,
                                          uint4 wm, uint32_t &rck)
{
    for (int a = 0; a < nnb; ++a) {
        const float4 d = nb[a];
        const int t = tri(norm2f(v0 - d.x, v1 - d.y, v2 - d.z), P.T_dep32, P.m_r2);
        if (t == 1) return false;
        if (t == -1) {
            ++rck;
            if (exact_dep_nb(P, w, kind, i, wm, __float_as_int(d.w))) return false;
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
__device__ __forceinline__ CbResult32 cb_factor_fp32(const SimParams &P, uint32_t sweep, uint32_t tag,
                                                  uint32_t k, float o0, float o1, float o2, int i,
                                                  uint4 wm, const float4 *nb, int nnb, float r_hi,
                                                  float r_lo)
{
    CbResult32 r = {0.0, 0u, 0u, 0u, 0u};
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
            tn = exact_fwd_new(P, w, i, wm) ? 1 : 0;
        }
        if (tn) continue;
        if (!free_nb32(P, y0, y1, y2, nb, nnb, w, 1, i, wm, r.rck)) continue;
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
            to = exact_dep_old(P, w, i, wm) ? 1 : 0;
        }
        if (to) continue;
        if (!free_nb32(P, e0, e1, e2, nb, nnb, w, 0, i, wm, r.rck)) continue;
        ++nr;
    }
    if (found < n_rev) ++r.caps;
    r.fwd_ok = (uint32_t)nf;
    r.rev_ok = (uint32_t)nr;
    r.f = (double)nf / (double)(nr + 1);
    return r;
}

__global__ void __launch_bounds__(kMaxThreads, 3)
    k_phase_sphere_fp32(const __grid_constant__ SimParams P, int phase)
{
    __shared__ int s_own[kMaxCellCap], s_tmp[kMaxCellCap];
    __shared__ float4 s_cpos[kMaxCand];  // candidates relative to this cell's origin; index in .w
    __shared__ float4 s_nb[kMaxCand];    // neighbours relative to the new position; index in .w
    __shared__ double s_f[kMaxThreads];
    __shared__ int s_k[kMaxThreads];
    __shared__ int s_warp[kMaxThreads / 32];
    __shared__ int s_ncand, s_nnb, s_flag, s_acc, s_kmin, s_self;

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
    if (tid == 0) s_ncand = 0;
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
        ++c_moves;
        const uint4 wm = draw(P.key0, P.key1, sweep, tag, kPMove, 0, 0);
        const float4 ri = P.rel[i];

        // a3: proposal in cell-relative FP32; cell-exit check with margin
        const float rn0 = ri.x + scaled_s11f(wm.x, dm_hi, dm_lo);
        const float rn1 = ri.y + scaled_s11f(wm.y, dm_hi, dm_lo);
        const float rn2 = ri.z + scaled_s11f(wm.z, dm_hi, dm_lo);
        const float mc = P.m_cell, wc = P.w32;
        const bool out = rn0 < -mc || rn0 > wc + mc || rn1 < -mc || rn1 > wc + mc ||
                         rn2 < -mc || rn2 > wc + mc;
        const bool edge = rn0 <= mc || rn0 >= wc - mc || rn1 <= mc || rn1 >= wc - mc ||
                          rn2 <= mc || rn2 >= wc - mc;
        bool exits = out;
        if (!out && edge) {
            exits = exact_cell_exit(P, i, wm, cx, cy, cz);
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
        for (int j = tid; j < M; j += nthr) {
            const float4 cp = s_cpos[j];
            const int pj = __float_as_int(cp.w);
            if (pj == i) {
                s_self = j;
                continue;
            }
            float d0 = cp.x - rn0, d1 = cp.y - rn1, d2 = cp.z - rn2;
            if (d0 > P.half_L32) d0 -= P.L32; else if (d0 < -P.half_L32) d0 += P.L32;
            if (d1 > P.half_L32) d1 -= P.L32; else if (d1 < -P.half_L32) d1 += P.L32;
            if (d2 > P.half_L32) d2 -= P.L32; else if (d2 < -P.half_L32) d2 += P.L32;
            const float r2 = norm2f(d0, d1, d2);
            int t = tri(r2, P.T_contact32, P.m_r2);
            if (t == -1) {
                ++c_rck;
                t = exact_pair(P, i, wm, pj) ? 1 : 0;
            }
            if (t == 1) ov = 1;
            if (r2 < P.nb_cut2_32) {
                const int slot = atomicAdd(&s_nnb, 1);
                s_nb[slot] = make_float4(d0, d1, d2, cp.w);
            }
        }
        if (__syncthreads_or(ov)) {
            ++c_ov;
            continue;
        }
        const int nnb = s_nnb;

        bool accept = true;
        if (P.has_dep) {
            // a5: Poisson count (integer table, exact)
            const uint4 wp = draw(P.key0, P.key1, sweep, tag, kPPoisson, 0, 0);
            const int n_p = poisson_count(P.T, P.nF, u53_int(wp.x, wp.y), lane);
            c_drawn += (unsigned long long)n_p;

            // a6: attempt stream, nthr attempts per pass
            const uint32_t t_max = 64u * (uint32_t)(n_p + 1);
            uint32_t t0 = 0;
            int k0 = 0, nblock = 0;
            double W = 1.0;
            bool rejected = false;
            while (k0 < n_p && t0 < t_max) {
                const uint32_t t = t0 + (uint32_t)tid;
                uint4 w = make_uint4(0, 0, 0, 0);
                float e0 = 0.f, e1 = 0.f, e2 = 0.f;
                bool inside = false;
                if (t < t_max) {
                    w = draw(P.key0, P.key1, sweep, tag, kPDep, 0, t);
                    e0 = scaled_s11f(w.x, r_hi, r_lo);
                    e1 = scaled_s11f(w.y, r_hi, r_lo);
                    e2 = scaled_s11f(w.z, r_hi, r_lo);
                    int in = tri(norm2f(e0, e1, e2), P.T_s32, P.m_r2);
                    if (in == -1) {
                        ++c_rck;
                        in = exact_ball(P, w) ? 1 : 0;
                    }
                    inside = in != 0;
                }
                const unsigned bal = __ballot_sync(kFull, inside);
                int base = 0, total = __popc(bal);
                if (nwarps > 1) {
                    if (lane == 0) s_warp[warp] = total;
                    __syncthreads();
                    total = 0;
                    for (int u = 0; u < nwarps; ++u) {
                        const int c = s_warp[u];
                        base += u < warp ? c : 0;
                        total += c;
                    }
                }
                const int k = k0 + base + __popc(bal & ((1u << lane) - 1u));
                bool blocking = false;
                if (inside && k < n_p) {
                    // inside the ball = overlaps the new pose (spheres); ignored if it
                    // overlaps the old configuration
                    int to = tri(norm2f(e0 - o0, e1 - o1, e2 - o2), P.T_dep32, P.m_r2);
                    if (to == -1) {
                        ++c_rck;
                        to = exact_dep_old(P, w, i, wm) ? 1 : 0;
                    }
                    if (!to) blocking = free_nb32(P, e0, e1, e2, s_nb, nnb, w, 0, i, wm, c_rck);
                }
                if (P.n_trial == 0) {
                    if (blocking) atomicMin(&s_kmin, k);
                    if (__syncthreads_or(blocking)) {
                        ++c_block;
                        c_eval += (uint32_t)(s_kmin - k0 + 1);
                        rejected = true;
                        break;
                    }
                    c_eval += (uint32_t)min(total, n_p - k0);
                } else {
                    double f = -1.0;
                    if (blocking) {
                        const CbResult32 r = cb_factor_fp32(P, sweep, tag, (uint32_t)k, o0, o1, o2,
                                                            i, wm, s_nb, nnb, r_hi, r_lo);
                        f = r.f;
                        c_fwd += r.fwd_ok;
                        c_rev += r.rev_ok;
                        c_cap += r.caps;
                        c_rck += r.rck;
                    }
                    s_f[tid] = f;
                    s_k[tid] = k;
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
                t0 += (uint32_t)nthr;
            }
            if (!rejected && k0 < n_p && tid == 0) ++c_cap;
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
        // a8: commit in FP64; refresh the FP32 working copies
        if (accept) {
            ++c_acc;
            if (tid == 0) s_cpos[s_self] = commit_move(P, i, wm, cx, cy, cz);
        }
        __syncthreads();
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
