// Gibbs-ensemble colloid exchange with configurational bias (Sec. IV.B):
// replicas 2p and 2p + 1 form the two boxes of pair p (spheres, one
// depletant reservoir).  An exchange moves a colloid to a uniform random
// position in the other box: a Metropolis test on the Gibbs factor
// N_s V_d / ((N_d + 1) V_s), the hard-core test in the new box, then the
// implicit depletants inserted at the new position (Sec. III.B), those that
// overlap the inserted colloid and no other colloid of the new box
// blocking it, or, with n_trial > 0, reinserted around the old position in
// the old box (the weight of Eq. 12).  FP64 in the specification's order.
// A box keeps its colloids in slots 0..n_live-1: the removed colloid's slot
// takes the box's last colloid, the inserted one takes slot n_live.
#pragma once

#include "hpmc_common.cuh"
#include "hpmc_sphere_fp64.cuh"
#include "hpmc_sphere_fp32.cuh"

namespace hpmc {

constexpr uint32_t kGibbsStream = 0xFFFFFFFEu;   // RNG stream word of the exchanges
constexpr int kGibbsCounters = 8;   // attempts, accept, empty, ratio, overlap, depletant, cb, drawn
constexpr int kMaxGibbsNb = 192;    // colloids within reach of the new (old) circumsphere

__device__ __forceinline__ float fmin_image32(float d, float L, float half_L)
{
    if (d > half_L) d = d - L;
    else if (d < -half_L) d = d + L;
    return d;
}

// Block-wide count and rank of a predicate over the CTA's threads (in thread
// order).  s_warp: one int per warp; every thread must call it.  Calls must
// alternate between two s_warp buffers (the barrier of one call orders the
// reads of the previous call's buffer before the next write to it).
__device__ __forceinline__ int block_rank(bool p, int *s_warp, int &rank)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const unsigned bal = __ballot_sync(kFull, p);
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    int base = 0, total = 0;
    for (int u = 0; u < nwarps; ++u) {
        const int c = s_warp[u];
        base += u < warp ? c : 0;
        total += c;
    }
    rank = base + __popc(bal & ((1u << lane) - 1u));
    return total;
}

// Point e (attempt word w of a depletant or CB stream, FP32 copy e32) free of
// every colloid of the list (offsets d from the point's centre, FP64 and FP32
// copies)?  F32: certified FP32 test, FP64 inside the margin.
template <bool F32>
__device__ __forceinline__ bool gibbs_free(const Rep &R, uint4 w, float3 e32, const double4 *nb,
                                           const float4 *nb32, int nnb, uint32_t &rck)
{
    for (int a = 0; a < nnb; ++a) {
        int t;
        if (F32) {
            const float4 d = nb32[a];
            t = tri(norm2f(e32.x - d.x, e32.y - d.y, e32.z - d.z), R.T_dep32, R.m_r2);
        } else {
            t = -1;
        }
        if (t == -1) {
            if (F32) ++rck;
            const double e0 = R.R_s * s11(w.x), e1 = R.R_s * s11(w.y), e2 = R.R_s * s11(w.z);
            const double4 d = nb[a];
            t = SphereFP64::dep(R, e0 - d.x, e1 - d.y, e2 - d.z) ? 1 : 0;
        }
        if (t == 1) return false;
    }
    return true;
}

// Attempt w inside the circumsphere (the sampling ball)?  Returns the FP32
// copy of the point in e32.
template <bool F32>
__device__ __forceinline__ bool gibbs_ball(const Rep &R, uint4 w, float3 &e32, uint32_t &rck)
{
    if (F32) {
        e32 = make_float3(coord32(w.x, R.R_s32), coord32(w.y, R.R_s32), coord32(w.z, R.R_s32));
        const int t = tri(norm2f(e32.x, e32.y, e32.z), R.T_s32, R.m_r2);
        if (t != -1) return t == 1;
        ++rck;
    }
    const double e0 = R.R_s * s11(w.x), e1 = R.R_s * s11(w.y), e2 = R.R_s * s11(w.z);
    return norm2(e0, e1, e2) < R.R_s2;
}

// One direction of the CB trials of blocking depletant k, by one warp (all
// 32 lanes call it): the first n_want attempts of stream (purpose, k) inside
// the ball, each counted when free of the list.  Lanes take consecutive
// attempts; a ballot ranks the in-ball ones.  Returns the count; *found the
// trials obtained (fewer than n_want when the attempt cap is hit).
template <bool F32>
__device__ int gibbs_trials(const Rep &R, uint32_t step, uint32_t purpose, uint32_t k, int n_want,
                            const double4 *nb, const float4 *nb32, int nnb, int &found, uint32_t &rck)
{
    const uint32_t lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint32_t t_max = 64u * (uint32_t)(n_want + 1);
    int ok_total = 0;
    found = 0;
    for (uint32_t t0 = 0; found < n_want && t0 < t_max; t0 += 32u) {
        const uint32_t t = t0 + lane;
        uint4 w = make_uint4(0, 0, 0, 0);
        float3 e32 = make_float3(0.f, 0.f, 0.f);
        bool in = false;
        if (t < t_max) {
            w = draw(R.key0, R.key1, step, kGibbsStream, purpose, k, t);
            in = gibbs_ball<F32>(R, w, e32, rck);
        }
        const unsigned bal = __ballot_sync(kFull, in);
        // (for spheres, inside the ball = overlapping the colloid it is centred on)
        const bool ok = in && found + __popc(bal & lt) < n_want &&
                        gibbs_free<F32>(R, w, e32, nb, nb32, nnb, rck);
        ok_total += __popc(__ballot_sync(kFull, ok));
        found += min(__popc(bal), n_want - found);
    }
    return ok_total;
}

constexpr int kGibbsAhead = 32;    // attempts whose random words are drawn ahead, one per lane
constexpr int kGibbsTab = 1024;    // Poisson table entries staged in shared memory (longer: global)

// One attempt's draws, made ahead (they depend on the counter only): source
// box, slot word, new position (FP64 and its FP32 image), the Metropolis and
// CB-acceptance uniforms, N_p.
struct GibbsDraw {
    double x[3];
    double u_ratio, u_acc;
    float x32[3];
    float u_ratio32;
    uint32_t wy;
    int src, n_p;
};

// N_p = #{k : T[k] <= m} by binary search (T non-decreasing), one lane.
__device__ __forceinline__ int poisson_count_lane(const unsigned long long *T, int nF,
                                                  unsigned long long m)
{
    int lo = 0, hi = nF;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (T[mid] <= m) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// n_attempts exchanges of every pair, one after another; one CTA per pair.
// F32: FP32 tests with certified margins, FP64 inside them; the FP32 images
// of the pair's positions are kept in pos32 (filled at the start, updated on
// every accepted exchange).
template <bool F32>
__global__ void __launch_bounds__(kMaxThreads, 1) k_gibbs_exchange(const __grid_constant__ SimParams P,
                                                                   int n_attempts)
{
    __shared__ double4 s_nb[kMaxGibbsNb], s_nbo[kMaxGibbsNb];
    __shared__ float4 s_nb32[kMaxGibbsNb], s_nbo32[kMaxGibbsNb];
    __shared__ int s_nbj[kMaxGibbsNb], s_nboj[kMaxGibbsNb];
    __shared__ unsigned long long s_tab[kGibbsTab];
    __shared__ GibbsDraw s_draw[kGibbsAhead];
    __shared__ int s_blk[kMaxThreads];
    __shared__ int s_warp[2][kMaxThreads / 32];
    __shared__ int4 s_cb[kMaxThreads / 32];     // (nf, nr, forward cap, reverse cap) of a round
    __shared__ double s_cbf[kMaxThreads / 32];  // and its factor nf / (nr + 1)
    __shared__ int s_n[2], s_nnb[2], s_nnbo[2], s_stop;
    __shared__ unsigned long long s_cnt[2][kNumCounters], s_g[kGibbsCounters];

    const int pr = blockIdx.x, tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int r0 = 2 * pr;
    // the pair's depletant parameters, table and key: box 0's (the host
    // requires equal parameters in both boxes)
    const Rep &R = P.reps[r0];
    const Rep &R1 = P.reps[r0 + 1];
    const double V[2] = {(R.L * R.L) * R.L, (R1.L * R1.L) * R1.L};
    const float V32[2] = {(float)V[0], (float)V[1]};
    const bool tab_smem = R.nF <= kGibbsTab;
    const unsigned long long *Tab = tab_smem ? s_tab : P.T + R.t_off;
    if (tab_smem)
        for (int k = tid; k < R.nF; k += nthr) s_tab[k] = P.T[R.t_off + k];
    if (tid < 2) {
        s_n[tid] = P.n_live[r0 + tid];
        s_nnb[tid] = 0;
        s_nnbo[tid] = 0;
    }
    for (int k = tid; k < 2 * kNumCounters; k += nthr) s_cnt[k / kNumCounters][k % kNumCounters] = 0ull;
    if (tid < kGibbsCounters) s_g[tid] = 0ull;
    if (F32) {
        // FP32 images of the pair's colloids
        for (int b = 0; b < 2; ++b) {
            const Rep &Rb = b ? R1 : R;
            const int nb = P.n_live[r0 + b];
            for (int j = tid; j < nb; j += nthr) {
                const double4 p = P.pos[Rb.off + j];
                P.pos32[Rb.off + j] = make_float4((float)p.x, (float)p.y, (float)p.z, 0.0f);
            }
        }
    }
    const unsigned long long step0 = P.gibbs_step[pr];
    uint32_t rck = 0;
    int par = 0;   // block_rank buffer
    __syncthreads();

    for (int a = 0; a < n_attempts; ++a) {
        const uint32_t step = (uint32_t)(step0 + (unsigned long long)a);
        __syncthreads();   // the previous attempt is committed and its draws are read
        if ((a & (kGibbsAhead - 1)) == 0) {
            // the next kGibbsAhead attempts' draws, one lane each
            if (warp == 0 && a + lane < n_attempts) {
                const uint32_t st = step + (uint32_t)lane;
                const uint4 w = draw(R.key0, R.key1, st, kGibbsStream, kPMove, 0, 0);
                const uint4 wx = draw(R.key0, R.key1, st, kGibbsStream, kPMove, 1, 0);
                const uint4 wr = draw(R.key0, R.key1, st, kGibbsStream, kPAccept, 1, 0);
                const uint4 wc = draw(R.key0, R.key1, st, kGibbsStream, kPAccept, 0, 0);
                const uint4 wp = draw(R.key0, R.key1, st, kGibbsStream, kPPoisson, 0, 0);
                GibbsDraw d;
                d.src = (int)(w.x >> 31);
                d.wy = w.y;
                const double Ld = (d.src ? R : R1).L;
                d.x[0] = Ld * u01(wx.x);
                d.x[1] = Ld * u01(wx.y);
                d.x[2] = Ld * u01(wx.z);
                for (int c = 0; c < 3; ++c) d.x32[c] = (float)d.x[c];
                d.u_ratio = u53(wr.x, wr.y);
                d.u_ratio32 = (float)d.u_ratio;
                d.u_acc = u53(wc.x, wc.y);
                d.n_p = R.has_dep ? poisson_count_lane(Tab, R.nF, u53_int(wp.x, wp.y)) : 0;
                s_draw[lane] = d;
            }
            __syncthreads();
        }
        // candidate counts alternate by attempt: the next attempt's are
        // cleared now (the previous attempt, which used them, is over)
        if (tid == 0) {
            s_nnb[(a + 1) & 1] = 0;
            s_nnbo[(a + 1) & 1] = 0;
        }
        const GibbsDraw &D = s_draw[a & (kGibbsAhead - 1)];
        const int src = D.src, dst = 1 - src;
        const int ns = s_n[src], nd = s_n[dst];
        if (tid == 0) s_g[0]++;
        if (ns == 0) {
            if (tid == 0) s_g[2]++;
            continue;
        }
        const int i = (int)(((unsigned long long)D.wy * (unsigned long long)ns) >> 32);
        // the Metropolis test u < G = N_s V_d / ((N_d + 1) V_s), by every
        // thread: in FP32 when u is clear of G by more than the rounding of
        // both (ns, nd + 1 < 2^24 exact; G32 errs by <= 6 u G), else in FP64
        bool pass;
        {
            const float g32 = ((float)ns * V32[dst]) / ((float)(nd + 1) * V32[src]);
            const float band = g32 * 0x1p-20f;
            if (ns < (1 << 24) && nd + 1 < (1 << 24) && D.u_ratio32 < g32 - band) pass = true;
            else if (ns < (1 << 24) && nd + 1 < (1 << 24) && D.u_ratio32 > g32 + band) pass = false;
            else pass = D.u_ratio < ((double)ns * V[dst]) / ((double)(nd + 1) * V[src]);
        }
        if (!pass) {
            if (tid == 0) s_g[3]++;
            continue;
        }
        const Rep &Rd = dst ? R1 : R, &Rs = src ? R1 : R;
        const bool cb = R.has_dep && R.n_trial > 0;
        // hard core in the new box, and the colloids within reach of the new
        // circumsphere (with CB also the old box's within reach of the old
        // one): candidates by FP32 distances with the box margin (every one
        // for the FP64 form), then their exact FP64 offsets
        int *const nnb_ctr = &s_nnb[a & 1], *const nnbo_ctr = &s_nnbo[a & 1];
        int ov = 0;
        if (F32) {
            const float x0 = D.x32[0], x1 = D.x32[1], x2 = D.x32[2];
            for (int j = tid; j < nd; j += nthr) {
                const float4 pj = P.pos32[Rd.off + j];
                const float f0 = fmin_image32(pj.x - x0, Rd.L32, Rd.half_L32);
                const float f1 = fmin_image32(pj.y - x1, Rd.L32, Rd.half_L32);
                const float f2 = fmin_image32(pj.z - x2, Rd.L32, Rd.half_L32);
                const float r2f = norm2f(f0, f1, f2);
                const int t = tri(r2f, R.T_contact32, Rd.m_box32);
                if (t == 1) ov = 1;
                if (t == -1 || r2f < R.nb_cut2_32 + Rd.m_box32) {
                    const int slot = atomicAdd(nnb_ctr, 1);
                    if (slot < kMaxGibbsNb) s_nbj[slot] = j;
                }
            }
            if (cb) {
                const float4 po = P.pos32[Rs.off + i];
                for (int j = tid; j < ns; j += nthr) {
                    if (j == i) continue;
                    const float4 pj = P.pos32[Rs.off + j];
                    const float f0 = fmin_image32(pj.x - po.x, Rs.L32, Rs.half_L32);
                    const float f1 = fmin_image32(pj.y - po.y, Rs.L32, Rs.half_L32);
                    const float f2 = fmin_image32(pj.z - po.z, Rs.L32, Rs.half_L32);
                    if (norm2f(f0, f1, f2) < R.nb_cut2_32 + Rs.m_box32) {
                        const int slot = atomicAdd(nnbo_ctr, 1);
                        if (slot < kMaxGibbsNb) s_nboj[slot] = j;
                    }
                }
            }
            // a certain overlap rejects before any FP64 work
            if (__syncthreads_or(ov)) {
                if (tid == 0) s_g[4]++;
                continue;
            }
        } else {
            const double x0 = D.x[0], x1 = D.x[1], x2 = D.x[2];
            for (int j = tid; j < nd; j += nthr) {
                const double4 pj = P.pos[Rd.off + j];
                const double r2 = norm2(min_image(pj.x - x0, Rd.L, Rd.half_L),
                                        min_image(pj.y - x1, Rd.L, Rd.half_L),
                                        min_image(pj.z - x2, Rd.L, Rd.half_L));
                if (r2 < R.contact2) ov = 1;
                if (r2 < R.nb_cut2) {
                    const int slot = atomicAdd(nnb_ctr, 1);
                    if (slot < kMaxGibbsNb) s_nbj[slot] = j;
                }
            }
            if (cb) {
                const double4 po = P.pos[Rs.off + i];
                for (int j = tid; j < ns; j += nthr) {
                    if (j == i) continue;
                    const double4 pj = P.pos[Rs.off + j];
                    const double r2 = norm2(min_image(pj.x - po.x, Rs.L, Rs.half_L),
                                            min_image(pj.y - po.y, Rs.L, Rs.half_L),
                                            min_image(pj.z - po.z, Rs.L, Rs.half_L));
                    if (r2 < R.nb_cut2) {
                        const int slot = atomicAdd(nnbo_ctr, 1);
                        if (slot < kMaxGibbsNb) s_nboj[slot] = j;
                    }
                }
            }
            if (__syncthreads_or(ov)) {
                if (tid == 0) s_g[4]++;
                continue;
            }
        }
        const int nnb = *nnb_ctr, nnbo = *nnbo_ctr;
        if (nnb > kMaxGibbsNb || nnbo > kMaxGibbsNb) {
            if (tid == 0) atomicCAS(P.err, kErrNone, kErrCandCap);
            break;
        }
        // exact offsets of the candidates, one thread each (the FP32 form
        // also settles the hard core of the pairs its FP32 test left open)
        for (int c = tid; c < nnb + nnbo; c += nthr) {
            const bool nw = c < nnb;
            const int slot = nw ? c : c - nnb;
            const Rep &Rb = nw ? Rd : Rs;
            const int j = nw ? s_nbj[slot] : s_nboj[slot];
            double y0, y1, y2;
            if (nw) {
                y0 = D.x[0];
                y1 = D.x[1];
                y2 = D.x[2];
            } else {
                const double4 po = P.pos[Rs.off + i];
                y0 = po.x;
                y1 = po.y;
                y2 = po.z;
            }
            const double4 pj = P.pos[Rb.off + j];
            const double d0 = min_image(pj.x - y0, Rb.L, Rb.half_L);
            const double d1 = min_image(pj.y - y1, Rb.L, Rb.half_L);
            const double d2 = min_image(pj.z - y2, Rb.L, Rb.half_L);
            if (nw && F32 && norm2(d0, d1, d2) < R.contact2) ov = 1;
            (nw ? s_nb : s_nbo)[slot] = make_double4(d0, d1, d2, 0.0);
            (nw ? s_nb32 : s_nbo32)[slot] = make_float4((float)d0, (float)d1, (float)d2, 0.0f);
        }
        if (__syncthreads_or(ov)) {
            if (tid == 0) s_g[4]++;
            continue;
        }
        bool accept = true;
        if (R.has_dep) {
            const int n_p = D.n_p;
            if (tid == 0) {
                s_g[7] += (unsigned long long)n_p;
                s_cnt[src][kDepDrawn] += (unsigned long long)n_p;
            }
            const uint32_t t_max = 64u * (uint32_t)(n_p + 1);
            uint32_t t0 = 0;
            int k0 = 0;
            double W = 1.0;     // (thread 0)
            int nblock = 0;
            bool rejected = false;
            while (k0 < n_p && t0 < t_max) {
                const uint32_t t = t0 + (uint32_t)tid;
                uint4 w = make_uint4(0, 0, 0, 0);
                float3 e32 = make_float3(0.f, 0.f, 0.f);
                bool inside = false;
                if (t < t_max) {
                    w = draw(R.key0, R.key1, step, kGibbsStream, kPDep, 0, t);
                    inside = gibbs_ball<F32>(R, w, e32, rck);
                }
                int rank;
                const int total = block_rank(inside, s_warp[par], rank);
                par ^= 1;
                const int k = k0 + rank;
                // blocking: overlaps the inserted colloid (inside, for spheres)
                // and no other colloid of its box
                const bool blocking = inside && k < n_p &&
                                      gibbs_free<F32>(R, w, e32, s_nb, s_nb32, nnb, rck);
                int brank;
                const int nblk = block_rank(blocking, s_warp[par], brank);
                par ^= 1;
                if (blocking) s_blk[brank] = k;    // ascending k
                if (tid == 0) s_stop = -1;
                __syncthreads();
                int stop = -1;   // index of the depletant that rejects the move
                if (R.n_trial == 0) {
                    if (nblk > 0) stop = s_blk[0];
                } else {
                    // the CB factors in rounds of one blocking depletant per
                    // warp (each warp's lane 0 forms f = nf / (nr + 1) in
                    // FP64), then taken in ascending k by thread 0; f is zero
                    // iff nf is, and a zero factor ends the pass
                    for (int b0 = 0; b0 < nblk && stop < 0; b0 += nwarps) {
                        const int b = b0 + warp;
                        if (b < nblk) {
                            const uint32_t kb = (uint32_t)s_blk[b];
                            int found_f, found_r;
                            const int nf = gibbs_trials<F32>(R, step, kPCbFwd, kb, R.n_trial, s_nbo,
                                                             s_nbo32, nnbo, found_f, rck);
                            const int nr = gibbs_trials<F32>(R, step, kPCbRev, kb, R.n_trial - 1, s_nb,
                                                             s_nb32, nnb, found_r, rck);
                            if (lane == 0) {
                                s_cb[warp] = make_int4(nf, nr, found_f < R.n_trial ? 1 : 0,
                                                       found_r < R.n_trial - 1 ? 1 : 0);
                                s_cbf[warp] = (double)nf / (double)(nr + 1);
                            }
                        }
                        __syncthreads();
                        if (tid == 0) {
                            for (int u = 0; u < nwarps && b0 + u < nblk; ++u) {
                                const int4 c4 = s_cb[u];
                                s_cnt[src][kCbFwdOk] += (unsigned long long)c4.x;
                                s_cnt[src][kCbRevOk] += (unsigned long long)c4.y;
                                s_cnt[src][kCapHits] += (unsigned long long)(c4.z + c4.w);
                                s_cnt[src][kDepBlocking]++;
                                ++nblock;
                                if (c4.x == 0) {
                                    s_stop = s_blk[b0 + u];
                                    break;
                                }
                                W = W * s_cbf[u];
                            }
                        }
                        __syncthreads();
                        stop = s_stop;
                    }
                }
                if (stop >= 0) {
                    if (tid == 0) {
                        if (R.n_trial == 0) s_cnt[src][kDepBlocking]++;
                        s_cnt[src][kDepEval] += (unsigned long long)(stop - k0 + 1);
                    }
                    rejected = true;
                    break;
                }
                if (tid == 0) s_cnt[src][kDepEval] += (unsigned long long)min(total, n_p - k0);
                k0 += total;
                t0 += (uint32_t)nthr;
            }
            if (tid == 0) {
                if (!rejected && k0 < n_p) s_cnt[src][kCapHits]++;
                if (rejected) {
                    accept = false;
                    s_g[R.n_trial == 0 ? 5 : 6]++;
                } else if (R.n_trial > 0 && nblock > 0) {
                    if (!(D.u_acc < W)) {
                        accept = false;
                        s_g[6]++;
                    }
                }
            }
        }
        // commit: the new box gains slot nd, the old one's last colloid fills slot i
        if (tid == 0 && accept) {
            P.pos[Rd.off + nd] = make_double4(D.x[0], D.x[1], D.x[2], 0.0);
            P.pos[Rs.off + i] = P.pos[Rs.off + ns - 1];
            if (F32) {
                P.pos32[Rd.off + nd] = make_float4(D.x32[0], D.x32[1], D.x32[2], 0.0f);
                P.pos32[Rs.off + i] = P.pos32[Rs.off + ns - 1];
            }
            s_n[dst] = nd + 1;
            s_n[src] = ns - 1;
            s_g[1]++;
        }
    }
    __syncthreads();
    if (tid < 2) P.n_live[r0 + tid] = s_n[tid];
    if (tid == 0) P.gibbs_step[pr] = step0 + (unsigned long long)n_attempts;
    if (tid < kGibbsCounters) P.gibbs_cnt[(size_t)pr * kGibbsCounters + tid] += s_g[tid];
    for (int k = tid; k < 2 * kNumCounters; k += nthr) {
        const unsigned long long v = s_cnt[k / kNumCounters][k % kNumCounters];
        if (v) atomicAdd(P.counters + (size_t)(r0 + k / kNumCounters) * kRepSlots * kNumCounters +
                             (k % kNumCounters), v);
    }
    // FP64 re-takes, to box 0's counters
    rck = __reduce_add_sync(kFull, rck);
    if (lane == 0 && rck) atomicAdd(P.counters + (size_t)r0 * kRepSlots * kNumCounters + kRechecks,
                                    (unsigned long long)rck);
}

}  // namespace hpmc
