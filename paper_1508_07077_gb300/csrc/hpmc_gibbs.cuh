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
// order).  s_warp: one int per warp; every thread must call it.
__device__ __forceinline__ int block_rank(bool p, int *s_warp, int &rank)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const unsigned bal = __ballot_sync(kFull, p);
    __syncthreads();                     // the previous call's counts are consumed
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

// One direction of the CB trials of blocking depletant k, by the whole CTA:
// the first n_want attempts of stream (purpose, k) inside the ball, each
// counted when free of the list.  Returns the count; *found the trials
// obtained (fewer than n_want when the attempt cap is hit).
template <bool F32>
__device__ int gibbs_trials(const Rep &R, uint32_t step, uint32_t purpose, uint32_t k, int n_want,
                            const double4 *nb, const float4 *nb32, int nnb, int *s_warp, int &found,
                            uint32_t &rck)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    const uint32_t t_max = 64u * (uint32_t)(n_want + 1);
    int ok_total = 0;
    found = 0;
    for (uint32_t t0 = 0; found < n_want && t0 < t_max; t0 += (uint32_t)nthr) {
        const uint32_t t = t0 + (uint32_t)tid;
        uint4 w = make_uint4(0, 0, 0, 0);
        float3 e32 = make_float3(0.f, 0.f, 0.f);
        bool in = false;
        if (t < t_max) {
            w = draw(R.key0, R.key1, step, kGibbsStream, purpose, k, t);
            in = gibbs_ball<F32>(R, w, e32, rck);
        }
        int rank;
        const int n_in = block_rank(in, s_warp, rank);
        // (for spheres, inside the ball = overlapping the colloid it is centred on)
        const bool take = in && found + rank < n_want;
        const bool ok = take && gibbs_free<F32>(R, w, e32, nb, nb32, nnb, rck);
        int dummy;
        ok_total += block_rank(ok, s_warp, dummy);
        found += min(n_in, n_want - found);
    }
    return ok_total;
}

// n_attempts exchanges of every pair, one after another; one CTA per pair.
// F32: FP32 depletant tests with the certified margin (FP64 inside it).
template <bool F32>
__global__ void __launch_bounds__(kMaxThreads) k_gibbs_exchange(const __grid_constant__ SimParams P,
                                                                int n_attempts)
{
    __shared__ double4 s_nb[kMaxGibbsNb], s_nbo[kMaxGibbsNb];
    __shared__ float4 s_nb32[kMaxGibbsNb], s_nbo32[kMaxGibbsNb];
    __shared__ int s_blk[kMaxThreads];
    __shared__ int s_warp[kMaxThreads / 32];
    __shared__ int s_n[2], s_src, s_i, s_go, s_nnb, s_nnbo;
    __shared__ double s_x[3], s_xo[3];
    __shared__ unsigned long long s_cnt[2][kNumCounters], s_g[kGibbsCounters];

    const int pr = blockIdx.x, tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31;
    const int r0 = 2 * pr;
    // the pair's depletant parameters, table and key: box 0's (the host
    // requires equal parameters in both boxes)
    const Rep &R = P.reps[r0];
    const Rep *RB[2] = {&P.reps[r0], &P.reps[r0 + 1]};
    const unsigned long long *Tab = P.T + R.t_off;
    if (tid < 2) s_n[tid] = P.n_live[r0 + tid];
    for (int k = tid; k < 2 * kNumCounters; k += nthr) s_cnt[k / kNumCounters][k % kNumCounters] = 0ull;
    if (tid < kGibbsCounters) s_g[tid] = 0ull;
    const unsigned long long step0 = P.gibbs_step[pr];
    uint32_t rck = 0;
    __syncthreads();

    for (int a = 0; a < n_attempts; ++a) {
        const uint32_t step = (uint32_t)(step0 + (unsigned long long)a);
        __syncthreads();   // every thread is done with the previous attempt's shared state
        if (tid == 0) {
            s_g[0]++;
            int go = 1;
            const uint4 w = draw(R.key0, R.key1, step, kGibbsStream, kPMove, 0, 0);
            const int src = (int)(w.x >> 31), dst = 1 - src;
            const int ns = s_n[src], nd = s_n[dst];
            s_src = src;
            if (ns == 0) {
                s_g[2]++;
                go = 0;
            } else {
                const int i = (int)(((unsigned long long)w.y * (unsigned long long)ns) >> 32);
                s_i = i;
                const double Ld = RB[dst]->L, Ls = RB[src]->L;
                const uint4 wx = draw(R.key0, R.key1, step, kGibbsStream, kPMove, 1, 0);
                s_x[0] = Ld * u01(wx.x);
                s_x[1] = Ld * u01(wx.y);
                s_x[2] = Ld * u01(wx.z);
                const double4 po = P.pos[RB[src]->off + i];
                s_xo[0] = po.x;
                s_xo[1] = po.y;
                s_xo[2] = po.z;
                const double Vs = (Ls * Ls) * Ls, Vd = (Ld * Ld) * Ld;
                const double G = ((double)ns * Vd) / ((double)(nd + 1) * Vs);
                const uint4 wa = draw(R.key0, R.key1, step, kGibbsStream, kPAccept, 1, 0);
                if (!(u53(wa.x, wa.y) < G)) {
                    s_g[3]++;
                    go = 0;
                }
            }
            s_go = go;
            s_nnb = 0;
            s_nnbo = 0;
        }
        __syncthreads();
        if (!s_go) continue;
        const int src = s_src, dst = 1 - src, i = s_i;
        const int ns = s_n[src], nd = s_n[dst];
        const Rep &Rd = *RB[dst], &Rs = *RB[src];
        const double x0 = s_x[0], x1 = s_x[1], x2 = s_x[2];
        // hard core in the new box; its colloids within reach of the new
        // circumsphere (F32: distances from FP32 images of the positions with
        // the box margin, FP64 near the contact distance; the list takes a
        // superset and keeps exact FP64 offsets)
        int ov = 0;
        for (int j = tid; j < nd; j += nthr) {
            const double4 pj = P.pos[Rd.off + j];
            bool near = true;
            if (F32) {
                const float f0 = fmin_image32((float)pj.x - (float)x0, Rd.L32, Rd.half_L32);
                const float f1 = fmin_image32((float)pj.y - (float)x1, Rd.L32, Rd.half_L32);
                const float f2 = fmin_image32((float)pj.z - (float)x2, Rd.L32, Rd.half_L32);
                const float r2f = norm2f(f0, f1, f2);
                const int t = tri(r2f, R.T_contact32, Rd.m_box32);
                if (t == 1) ov = 1;
                near = t == -1 || r2f < R.nb_cut2_32 + Rd.m_box32;
                if (!near) continue;
            }
            const double d0 = min_image(pj.x - x0, Rd.L, Rd.half_L);
            const double d1 = min_image(pj.y - x1, Rd.L, Rd.half_L);
            const double d2 = min_image(pj.z - x2, Rd.L, Rd.half_L);
            const double r2 = norm2(d0, d1, d2);
            if (r2 < R.contact2) ov = 1;
            if (r2 < R.nb_cut2) {
                const int slot = atomicAdd(&s_nnb, 1);
                if (slot < kMaxGibbsNb) {
                    s_nb[slot] = make_double4(d0, d1, d2, 0.0);
                    s_nb32[slot] = make_float4((float)d0, (float)d1, (float)d2, 0.0f);
                }
            }
        }
        // (CB) the old box's colloids within reach of the old circumsphere
        if (R.has_dep && R.n_trial > 0) {
            const double o0 = s_xo[0], o1 = s_xo[1], o2 = s_xo[2];
            for (int j = tid; j < ns; j += nthr) {
                if (j == i) continue;
                const double4 pj = P.pos[Rs.off + j];
                if (F32) {
                    const float f0 = fmin_image32((float)pj.x - (float)o0, Rs.L32, Rs.half_L32);
                    const float f1 = fmin_image32((float)pj.y - (float)o1, Rs.L32, Rs.half_L32);
                    const float f2 = fmin_image32((float)pj.z - (float)o2, Rs.L32, Rs.half_L32);
                    if (!(norm2f(f0, f1, f2) < R.nb_cut2_32 + Rs.m_box32)) continue;
                }
                const double d0 = min_image(pj.x - o0, Rs.L, Rs.half_L);
                const double d1 = min_image(pj.y - o1, Rs.L, Rs.half_L);
                const double d2 = min_image(pj.z - o2, Rs.L, Rs.half_L);
                if (norm2(d0, d1, d2) < R.nb_cut2) {
                    const int slot = atomicAdd(&s_nnbo, 1);
                    if (slot < kMaxGibbsNb) {
                        s_nbo[slot] = make_double4(d0, d1, d2, 0.0);
                        s_nbo32[slot] = make_float4((float)d0, (float)d1, (float)d2, 0.0f);
                    }
                }
            }
        }
        if (__syncthreads_or(ov)) {
            if (tid == 0) s_g[4]++;
            continue;
        }
        const int nnb = s_nnb, nnbo = s_nnbo;
        if (nnb > kMaxGibbsNb || nnbo > kMaxGibbsNb) {
            if (tid == 0) atomicCAS(P.err, kErrNone, kErrCandCap);
            break;
        }
        bool accept = true;
        if (R.has_dep) {
            const uint4 wp = draw(R.key0, R.key1, step, kGibbsStream, kPPoisson, 0, 0);
            const int n_p = poisson_count(Tab, R.nF, u53_int(wp.x, wp.y), lane);
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
                const int total = block_rank(inside, s_warp, rank);
                const int k = k0 + rank;
                // blocking: overlaps the inserted colloid (inside, for spheres)
                // and no other colloid of its box
                const bool blocking = inside && k < n_p &&
                                      gibbs_free<F32>(R, w, e32, s_nb, s_nb32, nnb, rck);
                int brank;
                const int nblk = block_rank(blocking, s_warp, brank);
                if (blocking) s_blk[brank] = k;    // ascending k
                __syncthreads();
                int stop = -1;   // index of the depletant that rejects the move
                if (R.n_trial == 0) {
                    if (nblk > 0) stop = s_blk[0];
                } else {
                    for (int b = 0; b < nblk; ++b) {
                        const int kb = s_blk[b];
                        int found_f, found_r;
                        const int nf = gibbs_trials<F32>(R, step, kPCbFwd, (uint32_t)kb, R.n_trial,
                                                         s_nbo, s_nbo32, nnbo, s_warp, found_f, rck);
                        const int nr = gibbs_trials<F32>(R, step, kPCbRev, (uint32_t)kb,
                                                         R.n_trial - 1, s_nb, s_nb32, nnb, s_warp,
                                                         found_r, rck);
                        if (tid == 0) {
                            s_cnt[src][kCbFwdOk] += (unsigned long long)nf;
                            s_cnt[src][kCbRevOk] += (unsigned long long)nr;
                            if (found_f < R.n_trial) s_cnt[src][kCapHits]++;
                            if (found_r < R.n_trial - 1) s_cnt[src][kCapHits]++;
                            s_cnt[src][kDepBlocking]++;
                            ++nblock;
                        }
                        // f = nf / (nr + 1) is zero iff nf is (the FP64 quotient
                        // and product only in thread 0)
                        if (nf == 0) {
                            stop = kb;
                            break;
                        }
                        if (tid == 0) W = W * ((double)nf / (double)(nr + 1));
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
                    const uint4 wa = draw(R.key0, R.key1, step, kGibbsStream, kPAccept, 0, 0);
                    if (!(u53(wa.x, wa.y) < W)) {
                        accept = false;
                        s_g[6]++;
                    }
                }
            }
        }
        // commit: the new box gains slot nd, the old one's last colloid fills slot i
        if (tid == 0 && accept) {
            P.pos[Rd.off + nd] = make_double4(x0, x1, x2, 0.0);
            P.pos[Rs.off + i] = P.pos[Rs.off + ns - 1];
            s_n[dst] = nd + 1;
            s_n[src] = ns - 1;
            s_g[1]++;
        }
        __syncthreads();
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
