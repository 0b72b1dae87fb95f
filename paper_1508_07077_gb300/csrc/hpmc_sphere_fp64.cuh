// Plain FP64 form of a colour phase for hard spheres (every test in FP64, in
// the specification's operation order).
#pragma once

#include "hpmc_common.cuh"

namespace hpmc {

struct SphereFP64 {
    // depletant at v (relative to the colloid centre) overlaps the colloid
    static __device__ __forceinline__ bool dep(const Rep &R, double v0, double v1, double v2)
    {
        return norm2(v0, v1, v2) < R.R_dep2;
    }
};

// Is the point y (relative to the new reference point) free of every
// neighbour in the shared list?
__device__ __forceinline__ bool free_of_nb_fp64(const Rep &R, double y0, double y1, double y2,
                                                const double4 *nb, int nnb)
{
    for (int a = 0; a < nnb; ++a) {
        const double4 d = nb[a];
        if (SphereFP64::dep(R, y0 - d.x, y1 - d.y, y2 - d.z)) return false;
    }
    return true;
}

// --- soft (Hertz) colloid-depletant interaction -----------------------------
// u(r) = eps (1 - r / s)^(5/2) for r < s = (d + q) / 2.  A depletant blocks a
// move with probability e^(-U_others) max(0, e^(-u_old) - e^(-u_new)), the
// neighbours' energies summed in ascending index.

// e^(-y), y >= 0, written out so that every form gives the same bits:
// y = k ln2 + r with ln2 in a 29-bit head and a tail (Cody and Waite's
// reduction), |r| <= ln2 / 2, e^(-r) by its Taylor polynomial of degree 14
// (Horner), then the exact scaling by 2^-k.
__device__ __forceinline__ double exp_neg_spec(double y)
{
    if (!(y < 700.0)) return 0.0;
    const double kd = floor(y * 0x1.71547652b82fep+0 + 0.5);
    const double r = (y - kd * 0x1.62e42ff000000p-1) - kd * -0x1.718432a1b0e26p-35;
    const double x = -r;
    const double c[15] = {1.0 / 87178291200.0, 1.0 / 6227020800.0, 1.0 / 479001600.0,
                          1.0 / 39916800.0, 1.0 / 3628800.0, 1.0 / 362880.0, 1.0 / 40320.0,
                          1.0 / 5040.0, 1.0 / 720.0, 1.0 / 120.0, 1.0 / 24.0, 1.0 / 6.0, 0.5,
                          1.0, 1.0};
    double p = c[0];
#pragma unroll
    for (int n = 1; n < 15; ++n) p = p * x + c[n];
    return ldexp(p, -(int)kd);
}

__device__ __forceinline__ double hertz_spec(const Rep &R, double r2)
{
    if (!(r2 < R.R_s2)) return 0.0;
    const double t = 1.0 - sqrt(r2) / R.R_s;
    return R.soft_eps * ((t * t) * sqrt(t));
}

// Two exits that give the specification's decision without its full cost:
// a point no nearer the new centre than the old one has u_new <= u_old (the
// energy is evaluated monotonically in r2), so e_old - e_new is at most a few
// ulp of rounding and b < 2^-33 <= u01(w); and since e^(-U) <= 1 (U >= 0),
// b <= e_old - e_new, so u01(w) >= e_old - e_new decides "not blocking"
// before the neighbours' energies are summed.
__device__ __noinline__ bool soft_blocks(const Rep &R, uint4 w, double e0, double e1, double e2,
                                         double o0, double o1, double o2, const double4 *nb, int nnb)
{
    const double u0 = e0 - o0, u1 = e1 - o1, u2 = e2 - o2;
    const double r2n = norm2(e0, e1, e2), r2o = norm2(u0, u1, u2);
    if (!(r2n < r2o)) return false;
    const double e_new = exp_neg_spec(hertz_spec(R, r2n));
    const double e_old = exp_neg_spec(hertz_spec(R, r2o));
    if (!(e_old > e_new)) return false;
    const double v = u01(w.w);
    if (!(v < e_old - e_new)) return false;
    double U = 0.0;
    for (int a = 0; a < nnb; ++a) {
        const double4 d = nb[a];
        U = U + hertz_spec(R, norm2(e0 - d.x, e1 - d.y, e2 - d.z));
    }
    const double b = exp_neg_spec(U) * (e_old - e_new);
    return v < b;
}

struct CbResult {
    double f;
    uint32_t fwd_ok, rev_ok, caps;
};

// Configurational-bias factor of blocking depletant k (Sec. III.D, Eq. 12):
// f = N'_insert / (N_insert + 1); n_trial forward trials in the old
// circumsphere, n_trial - 1 reverse trials in the new one.  The trials of a
// direction are the first n_fwd (n_rev) attempts of the stream (purpose, k)
// inside the ball.  Computed by a whole warp (all 32 lanes call it with the
// same k): lanes take consecutive attempts and a ballot ranks the in-ball
// ones.  Returns the same values in every lane.
__device__ __noinline__ CbResult cb_factor_fp64(const Rep &R, uint32_t sweep, uint32_t tag,
                                                uint32_t k, double o0, double o1, double o2,
                                                const double4 *nb, int nnb)
{
    CbResult r = {0.0, 0u, 0u, 0u};
    const uint32_t lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int dir = 0; dir < 2; ++dir) {
        const bool fwd = dir == 0;
        const int n_want = fwd ? R.n_trial : R.n_trial - 1;
        const uint32_t purpose = fwd ? kPCbFwd : kPCbRev;
        const uint32_t t_max = 64u * (uint32_t)(n_want + 1);
        int found = 0, ok = 0;
        for (uint32_t t0 = 0; found < n_want && t0 < t_max; t0 += 32u) {
            const uint32_t t = t0 + lane;
            double e0 = 0.0, e1 = 0.0, e2 = 0.0;
            bool in = false;
            if (t < t_max) {
                const uint4 w = draw(R.key0, R.key1, sweep, tag, purpose, k, t);
                e0 = R.R_s * s11(w.x);
                e1 = R.R_s * s11(w.y);
                e2 = R.R_s * s11(w.z);
                in = norm2(e0, e1, e2) < R.R_s2;
            }
            const unsigned bal = __ballot_sync(kFull, in);
            bool good = false;
            if (in && found + __popc(bal & lt) < n_want) {
                if (fwd) {
                    // must overlap the old pose and miss the new one
                    const double y0 = o0 + e0, y1 = o1 + e1, y2 = o2 + e2;
                    good = SphereFP64::dep(R, e0, e1, e2) && !SphereFP64::dep(R, y0, y1, y2) &&
                           free_of_nb_fp64(R, y0, y1, y2, nb, nnb);
                } else {
                    // must overlap the new pose and miss the old one
                    good = SphereFP64::dep(R, e0, e1, e2) &&
                           !SphereFP64::dep(R, e0 - o0, e1 - o1, e2 - o2) &&
                           free_of_nb_fp64(R, e0, e1, e2, nb, nnb);
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

// One colour phase: a CTA per active cell, blockDim = 32 * warps_per_colloid.
// The cell's colloids move one after another in ascending index; the
// depletants of each move are spread over the CTA's threads (App. A).
template <int CAP>
__global__ void __launch_bounds__(kMaxThreads)
    k_phase_sphere_fp64(const __grid_constant__ SimParams P, int phase)
{
    __shared__ int s_own[CAP], s_tmp[CAP];
    __shared__ int s_cand[kMaxCand];
    __shared__ double4 s_nb[kMaxCand];
    __shared__ double s_f[kMaxThreads];
    __shared__ int s_k[kMaxThreads];
    __shared__ int s_warp[kMaxThreads / 32];
    __shared__ unsigned s_mask[kMaxThreads / 32];
    __shared__ int s_ncand, s_nnb, s_flag, s_acc, s_kmin;

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const int r = P.cta_rep[blockIdx.x];
    const Rep &R = P.reps[r];
    const Sched &S = P.sched[r];
    if (phase == 7 && blockIdx.x == 0 && tid == 0) atomicAdd(P.sweep, 1ull);
    const uint32_t sweep = S.sweep;
    const CellTask T = cell_task(P, R, r, phase);
    clear_next(P, sweep, T.cell);
    const int n_own = min(T.n_own, P.cap);
    if (n_own == 0) return;
    own_members_sorted(P, T.cell, n_own, s_tmp, s_own);
    const int cx = T.cx, cy = T.cy, cz = T.cz, nc = R.nc;
    const unsigned long long *Tab = P.T + R.t_off;

    // candidate neighbours: every colloid of the (deduplicated) 27-cell stencil
    if (tid == 0) s_ncand = 0;
    __syncthreads();
    if (tid < R.n_stencil * R.n_stencil * R.n_stencil) {
        int dx, dy, dz;
        const int c = stencil_cell(R, tid, cx, cy, cz, dx, dy, dz);
        const int m = min(T.count[c], P.cap);
        for (int s = 0; s < m; ++s) {
            const int slot = atomicAdd(&s_ncand, 1);
            if (slot < kMaxCand) s_cand[slot] = __float_as_int(P.bins[bin_at(P, c, s)].w);
        }
    }
    __syncthreads();
    const int M = s_ncand;
    if (M > kMaxCand) {
        if (tid == 0) atomicCAS(P.err, kErrNone, kErrCandCap);
        return;
    }

    unsigned long long cnt[kNumCounters] = {0};

    for (int q = 0; q < n_own; ++q) {
        const int i = s_own[q];
        const uint32_t tag = (uint32_t)(i - R.off);
        const double4 pi = P.pos[i];
        cnt[kMoves]++;
        cnt[kTranslate]++;

        // a3: translation proposal, wrap, cell-exit check
        const uint4 wm = draw(R.key0, R.key1, sweep, tag, kPMove, 0, 0);
        const double xn0 = wrap_box(pi.x + R.d_max * s11(wm.x), R.L);
        const double xn1 = wrap_box(pi.y + R.d_max * s11(wm.y), R.L);
        const double xn2 = wrap_box(pi.z + R.d_max * s11(wm.z), R.L);
        if (cell_coord(xn0, S.sigma[0], R.L, R.w, nc) != cx ||
            cell_coord(xn1, S.sigma[1], R.L, R.w, nc) != cy ||
            cell_coord(xn2, S.sigma[2], R.L, R.w, nc) != cz) {
            cnt[kRejCell]++;
            continue;
        }
        const double o0 = min_image(pi.x - xn0, R.L, R.half_L);
        const double o1 = min_image(pi.y - xn1, R.L, R.half_L);
        const double o2 = min_image(pi.z - xn2, R.L, R.half_L);

        // a4: colloid overlap at the new pose; collect neighbours in range
        if (tid == 0) {
            s_nnb = 0;
            s_kmin = 0x7FFFFFFF;
        }
        __syncthreads();
        int ov = 0;
        for (int j = tid; j < M; j += nthr) {
            const int pj = s_cand[j];
            if (pj == i) continue;
            const double4 xj = P.pos[pj];
            const double d0 = min_image(xj.x - xn0, R.L, R.half_L);
            const double d1 = min_image(xj.y - xn1, R.L, R.half_L);
            const double d2 = min_image(xj.z - xn2, R.L, R.half_L);
            const double r2 = norm2(d0, d1, d2);
            if (r2 < R.contact2) ov = 1;
            if (r2 < R.nb_cut2) {
                const int slot = atomicAdd(&s_nnb, 1);
                s_nb[slot] = make_double4(d0, d1, d2, (double)pj);
            }
        }
        if (__syncthreads_or(ov)) {
            cnt[kRejOverlap]++;
            continue;
        }
        const int nnb = s_nnb;
        if (R.soft_eps > 0.0) {
            // soft interactions sum the neighbours' energies in ascending index
            if (tid == 0)
                for (int a = 1; a < nnb; ++a) {
                    const double4 v = s_nb[a];
                    int b = a - 1;
                    while (b >= 0 && s_nb[b].w > v.w) {
                        s_nb[b + 1] = s_nb[b];
                        --b;
                    }
                    s_nb[b + 1] = v;
                }
            __syncthreads();
        }

        bool accept = true;
        if (R.has_dep) {
            // a5: Poisson count
            // V_0: the circumsphere, or the shell of the move's level
            const int lvl = R.v0_shell ? shell_level(wm.x, wm.y, wm.z) : 0;
            const unsigned long long *TabV = lvl > 0 ? Tab + (size_t)(lvl - 1) * R.nF : Tab;
            const uint4 wp = draw(R.key0, R.key1, sweep, tag, kPPoisson, 0, 0);
            const int n_p = poisson_count(TabV, R.nF, u53_int(wp.x, wp.y), lane);
            cnt[kDepDrawn] += (unsigned long long)n_p;

            // a6: depletants along the attempt stream, nthr attempts per pass
            const uint32_t t_max = 64u * (uint32_t)(n_p + 1);
            uint32_t t0 = 0;
            int k0 = 0, nblock = 0;
            double W = 1.0;
            bool rejected = false;
            while (k0 < n_p && t0 < t_max) {
                const uint32_t t = t0 + (uint32_t)tid;
                double e0 = 0.0, e1 = 0.0, e2 = 0.0;
                bool inside = false;
                uint4 w = make_uint4(0, 0, 0, 0);
                if (t < t_max) {
                    if (lvl > 0) {
                        w = draw(R.key0, R.key1, sweep, tag, kPDep, 0, t);
                        inside = shell_point64(R, lvl, w, e0, e1, e2);
                    } else if (R.soft_eps > 0.0) {
                        // soft: one point per call, its fourth word decides blocking
                        w = draw(R.key0, R.key1, sweep, tag, kPDep, 0, t);
                        e0 = R.R_s * s11(w.x);
                        e1 = R.R_s * s11(w.y);
                        e2 = R.R_s * s11(w.z);
                        inside = R.v0_cube || norm2(e0, e1, e2) < R.R_s2;
                    } else {
                        // hard: the paired stream
                        paired_point64(R.key0, R.key1, R.R_s, sweep, tag, t, e0, e1, e2);
                        inside = R.v0_cube || norm2(e0, e1, e2) < R.R_s2;
                    }
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
                bool blocking = false;
                if (inside && k < n_p) {
                    if (R.soft_eps > 0.0) {
                        // soft: blocks with probability e^-U_others (e^-u_old - e^-u_new)
                        blocking = soft_blocks(R, w, e0, e1, e2, o0, o1, o2, s_nb, nnb);
                    } else if (SphereFP64::dep(R, e0, e1, e2) &&
                               !SphereFP64::dep(R, e0 - o0, e1 - o1, e2 - o2) &&
                               free_of_nb_fp64(R, e0, e1, e2, s_nb, nnb)) {
                        // irrelevant unless it overlaps the new pose; ignored if
                        // it overlaps the old configuration
                        blocking = true;
                    }
                }
                // depletants classified up to an early exit (same count as a serial loop)
                if (R.n_trial == 0) {
                    if (blocking) atomicMin(&s_kmin, k);
                    if (__syncthreads_or(blocking)) {
                        cnt[kDepBlocking] += 1;
                        cnt[kDepEval] += (unsigned long long)(s_kmin - k0 + 1);
                        rejected = true;
                        break;
                    }
                    cnt[kDepEval] += (unsigned long long)min(total, n_p - k0);
                } else {
                    // a7: CB factors of this pass (each warp's blocking
                    // depletants in ascending k, each by the whole warp; a
                    // zero factor rejects, so the ones after it are not
                    // needed), multiplied in ascending k
                    double f = 0.0;
                    bool has = false, zero = false;
                    unsigned bm = __ballot_sync(kFull, blocking);
                    while (bm) {
                        const int b = __ffs(bm) - 1;
                        bm &= bm - 1u;
                        const uint32_t kb = (uint32_t)__shfl_sync(kFull, k, b);
                        const CbResult cr = cb_factor_fp64(R, sweep, tag, kb, o0, o1, o2, s_nb, nnb);
                        if (lane == b) {
                            f = cr.f;
                            has = true;
                            zero = cr.fwd_ok == 0;
                            cnt[kCbFwdOk] += cr.fwd_ok;
                            cnt[kCbRevOk] += cr.rev_ok;
                            cnt[kCapHits] += cr.caps;
                        }
                        if (cr.fwd_ok == 0) break;
                    }
                    // slots holding a factor, by warp ballots; zero factors
                    // as -1 - k (integer tests only in the walk)
                    const unsigned hb = __ballot_sync(kFull, has);
                    if (lane == 0) s_mask[warp] = hb;
                    if (has) {
                        s_f[tid] = f;
                        s_k[tid] = zero ? -1 - k : k;
                    }
                    __syncthreads();
                    if (tid == 0) {
                        int n_fact = 0;
                        const int kz = cb_walk(s_mask, nwarps, s_k, s_f, W, n_fact);
                        nblock += n_fact;
                        cnt[kDepBlocking] += (unsigned long long)n_fact;
                        if (kz >= 0) cnt[kDepEval] += (unsigned long long)(kz - k0 + 1);
                        else cnt[kDepEval] += (unsigned long long)min(total, n_p - k0);
                        s_flag = kz >= 0 ? 1 : 0;
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
            if (!rejected && k0 < n_p && tid == 0) cnt[kCapHits]++;
            if (rejected) {
                accept = false;
                if (R.n_trial == 0) cnt[kRejDep]++;
                else cnt[kRejCb]++;
            } else if (R.n_trial > 0 && tid == 0 && nblock > 0) {
                const uint4 wa = draw(R.key0, R.key1, sweep, tag, kPAccept, 0, 0);
                if (!(u53(wa.x, wa.y) < W)) {
                    accept = false;
                    cnt[kRejCb]++;
                }
            }
            if (R.n_trial > 0) {
                if (tid == 0) s_acc = accept ? 1 : 0;
                __syncthreads();
                accept = s_acc != 0;
            }
        }
        // a8: commit
        if (accept) {
            cnt[kAccept]++;
            if (tid == 0) P.pos[i] = make_double4(xn0, xn1, xn2, 0.0);
        }
        __syncthreads();
    }

    // thread 0 holds the CTA's move counters; every thread its own CB/cap counts
    if (tid != 0) {
#pragma unroll
        for (int k = 0; k < kNumCounters; ++k)
            if (k != kCbFwdOk && k != kCbRevOk && k != kCapHits) cnt[k] = 0;
    }
    flush_counters(P, r, cnt);
}

}  // namespace hpmc
