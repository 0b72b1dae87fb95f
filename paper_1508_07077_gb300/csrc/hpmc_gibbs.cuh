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

namespace hpmc {

constexpr uint32_t kGibbsStream = 0xFFFFFFFEu;   // RNG stream word of the exchanges
constexpr int kGibbsCounters = 8;   // attempts, accept, empty, ratio, overlap, depletant, cb, drawn
constexpr int kMaxGibbsNb = 192;    // colloids within reach of the new (old) circumsphere

// Configurational-bias weight of blocking depletant k of the exchange: n_trial
// forward trials in the old circumsphere (overlapping the removed colloid,
// free of the old box's other colloids nbo), n_trial - 1 reverse trials in the
// new one (overlapping the inserted colloid, free of the new box's colloids nb).
__device__ __noinline__ CbResult gibbs_cb(const Rep &R, uint32_t step, uint32_t k, const double4 *nb,
                                          int nnb, const double4 *nbo, int nnbo)
{
    CbResult r = {0.0, 0u, 0u, 0u};
    const int n_fwd = R.n_trial, n_rev = R.n_trial - 1;
    int nf = 0, nr = 0, found = 0;
    uint32_t t = 0, t_max = 64u * (uint32_t)(n_fwd + 1);
    while (found < n_fwd && t < t_max) {
        const uint4 w = draw(R.key0, R.key1, step, kGibbsStream, kPCbFwd, k, t);
        ++t;
        const double e0 = R.R_s * s11(w.x), e1 = R.R_s * s11(w.y), e2 = R.R_s * s11(w.z);
        if (!(norm2(e0, e1, e2) < R.R_s2)) continue;
        ++found;
        if (!SphereFP64::dep(R, e0, e1, e2)) continue;
        if (!free_of_nb_fp64(R, e0, e1, e2, nbo, nnbo)) continue;
        ++nf;
    }
    if (found < n_fwd) ++r.caps;
    t = 0;
    t_max = 64u * (uint32_t)(n_rev + 1);
    found = 0;
    while (found < n_rev && t < t_max) {
        const uint4 w = draw(R.key0, R.key1, step, kGibbsStream, kPCbRev, k, t);
        ++t;
        const double e0 = R.R_s * s11(w.x), e1 = R.R_s * s11(w.y), e2 = R.R_s * s11(w.z);
        if (!(norm2(e0, e1, e2) < R.R_s2)) continue;
        ++found;
        if (!SphereFP64::dep(R, e0, e1, e2)) continue;
        if (!free_of_nb_fp64(R, e0, e1, e2, nb, nnb)) continue;
        ++nr;
    }
    if (found < n_rev) ++r.caps;
    r.fwd_ok = (uint32_t)nf;
    r.rev_ok = (uint32_t)nr;
    r.f = (double)nf / (double)(nr + 1);
    return r;
}

// n_attempts exchanges of every pair, one after another; one CTA per pair.
__global__ void __launch_bounds__(kMaxThreads) k_gibbs_exchange(const __grid_constant__ SimParams P,
                                                                int n_attempts)
{
    __shared__ double4 s_nb[kMaxGibbsNb], s_nbo[kMaxGibbsNb];
    __shared__ double s_f[kMaxThreads];
    __shared__ int s_k[kMaxThreads];
    __shared__ int s_warp[kMaxThreads / 32];
    __shared__ int s_n[2], s_src, s_i, s_go, s_nnb, s_nnbo, s_kmin, s_flag;
    __shared__ double s_x[3], s_xo[3];
    __shared__ unsigned long long s_cnt[2][kNumCounters], s_g[kGibbsCounters];

    const int pr = blockIdx.x, tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
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
            s_kmin = 0x7FFFFFFF;
        }
        __syncthreads();
        if (!s_go) continue;
        const int src = s_src, dst = 1 - src, i = s_i;
        const int ns = s_n[src], nd = s_n[dst];
        const Rep &Rd = *RB[dst], &Rs = *RB[src];
        const double x0 = s_x[0], x1 = s_x[1], x2 = s_x[2];
        // hard core in the new box; its colloids within reach of the new circumsphere
        int ov = 0;
        for (int j = tid; j < nd; j += nthr) {
            const double4 pj = P.pos[Rd.off + j];
            const double d0 = min_image(pj.x - x0, Rd.L, Rd.half_L);
            const double d1 = min_image(pj.y - x1, Rd.L, Rd.half_L);
            const double d2 = min_image(pj.z - x2, Rd.L, Rd.half_L);
            const double r2 = norm2(d0, d1, d2);
            if (r2 < R.contact2) ov = 1;
            if (r2 < R.nb_cut2) {
                const int slot = atomicAdd(&s_nnb, 1);
                if (slot < kMaxGibbsNb) s_nb[slot] = make_double4(d0, d1, d2, 0.0);
            }
        }
        // (CB) the old box's colloids within reach of the old circumsphere
        if (R.has_dep && R.n_trial > 0) {
            const double o0 = s_xo[0], o1 = s_xo[1], o2 = s_xo[2];
            for (int j = tid; j < ns; j += nthr) {
                if (j == i) continue;
                const double4 pj = P.pos[Rs.off + j];
                const double d0 = min_image(pj.x - o0, Rs.L, Rs.half_L);
                const double d1 = min_image(pj.y - o1, Rs.L, Rs.half_L);
                const double d2 = min_image(pj.z - o2, Rs.L, Rs.half_L);
                if (norm2(d0, d1, d2) < R.nb_cut2) {
                    const int slot = atomicAdd(&s_nnbo, 1);
                    if (slot < kMaxGibbsNb) s_nbo[slot] = make_double4(d0, d1, d2, 0.0);
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
            double W = 1.0;
            int nblock = 0;
            bool rejected = false;
            while (k0 < n_p && t0 < t_max) {
                const uint32_t t = t0 + (uint32_t)tid;
                double e0 = 0.0, e1 = 0.0, e2 = 0.0;
                bool inside = false;
                if (t < t_max) {
                    const uint4 w = draw(R.key0, R.key1, step, kGibbsStream, kPDep, 0, t);
                    e0 = R.R_s * s11(w.x);
                    e1 = R.R_s * s11(w.y);
                    e2 = R.R_s * s11(w.z);
                    inside = norm2(e0, e1, e2) < R.R_s2;
                }
                const unsigned bal = __ballot_sync(kFull, inside);
                if (lane == 0) s_warp[warp] = __popc(bal);
                __syncthreads();
                int base = 0, total = 0;
                for (int u = 0; u < nwarps; ++u) {
                    const int c = s_warp[u];
                    base += u < warp ? c : 0;
                    total += c;
                }
                const int k = k0 + base + __popc(bal & ((1u << lane) - 1u));
                // blocking: overlaps the inserted colloid and no other colloid of its box
                const bool blocking = inside && k < n_p && SphereFP64::dep(R, e0, e1, e2) &&
                                      free_of_nb_fp64(R, e0, e1, e2, s_nb, nnb);
                if (R.n_trial == 0) {
                    if (blocking) atomicMin(&s_kmin, k);
                    if (__syncthreads_or(blocking)) {
                        if (tid == 0) {
                            s_cnt[src][kDepBlocking] += 1ull;
                            s_cnt[src][kDepEval] += (unsigned long long)(s_kmin - k0 + 1);
                        }
                        rejected = true;
                        break;
                    }
                    if (tid == 0) s_cnt[src][kDepEval] += (unsigned long long)min(total, n_p - k0);
                } else {
                    double f = -1.0;
                    if (blocking) {
                        const CbResult cr = gibbs_cb(R, step, (uint32_t)k, s_nb, nnb, s_nbo, nnbo);
                        f = cr.f;
                        atomicAdd(&s_cnt[src][kCbFwdOk], (unsigned long long)cr.fwd_ok);
                        atomicAdd(&s_cnt[src][kCbRevOk], (unsigned long long)cr.rev_ok);
                        if (cr.caps) atomicAdd(&s_cnt[src][kCapHits], (unsigned long long)cr.caps);
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
                            s_cnt[src][kDepBlocking]++;
                            if (fu == 0.0) {
                                zero = 1;
                                s_cnt[src][kDepEval] += (unsigned long long)(s_k[u] - k0 + 1);
                                break;
                            }
                            W = W * fu;
                        }
                        if (!zero) s_cnt[src][kDepEval] += (unsigned long long)min(total, n_p - k0);
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
}

}  // namespace hpmc
