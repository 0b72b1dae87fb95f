// Plain FP64 form of a colour phase for anisotropic colloids (hemispheres,
// discoids; Sec. V) with translation and rotation moves.  Every test is the
// FP64 statement of the specification (hpmc_shapes.cuh).
#pragma once

#include "hpmc_common.cuh"
#include "hpmc_shapes.cuh"
#include "hpmc_sphere_fp64.cuh"

namespace hpmc {

// Is the point y (relative to the new reference point) free of every
// neighbour in the shared list (offsets d_j and orientations q_j)?
__device__ __forceinline__ bool free_of_nb_aniso(const Rep &R, Vec3 y, const double4 *nb,
                                                 const double4 *nbq, int nnb)
{
    for (int a = 0; a < nnb; ++a) {
        const double4 d = nb[a];
        if (dep_aniso(R, v3(y.x - d.x, y.y - d.y, y.z - d.z), nbq[a])) return false;
    }
    return true;
}

// Configurational-bias factor of blocking depletant k (Sec. III.D, Eq. 12):
// f = N'_insert / (N_insert + 1); n_trial forward trials in the old
// circumsphere (old pose at o, orientation qo), n_trial - 1 reverse trials in
// the new one (origin, orientation qn).  The trials of a direction are the
// first n_fwd (n_rev) attempts of the stream (purpose, k) inside the ball.
// Computed by a whole warp (all 32 lanes call it with the same k): lanes take
// consecutive attempts and a ballot ranks the in-ball ones.  Returns the same
// values in every lane.
__device__ __noinline__ CbResult cb_factor_aniso(const Rep &R, uint32_t sweep, uint32_t tag,
                                                 uint32_t k, Vec3 o, double4 qo, double4 qn,
                                                 const double4 *nb, const double4 *nbq, int nnb)
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
                    const Vec3 y = v3(o.x + e0, o.y + e1, o.z + e2);
                    good = dep_aniso(R, v3(e0, e1, e2), qo) && !dep_aniso(R, y, qn) &&
                           free_of_nb_aniso(R, y, nb, nbq, nnb);
                } else {
                    // must overlap the new pose and miss the old one
                    good = dep_aniso(R, v3(e0, e1, e2), qn) &&
                           !dep_aniso(R, v3(e0 - o.x, e1 - o.y, e2 - o.z), qo) &&
                           free_of_nb_aniso(R, v3(e0, e1, e2), nb, nbq, nnb);
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
// The cell's colloids move one after another in ascending index; each move is
// a translation or a rotation (Sec. V), its colloid tests are spread over the
// CTA's threads, and so are its depletants (App. A).
template <int CAP>
__global__ void __launch_bounds__(kMaxThreads, 1)
    k_phase_aniso_fp64(const __grid_constant__ SimParams P, int phase)
{
    __shared__ int s_own[CAP], s_tmp[CAP];
    __shared__ int s_cand[kMaxCand];
    __shared__ double4 s_nb[kMaxCand];
    __shared__ double4 s_nbq[kMaxCand];
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
    const double D2 = (2.0 * R.R_circ) * (2.0 * R.R_circ);

    for (int qi = 0; qi < n_own; ++qi) {
        const int i = s_own[qi];
        const uint32_t tag = (uint32_t)(i - R.off);
        const double4 pi = P.pos[i];
        const double4 qo = P.quat[i];
        cnt[kMoves]++;

        // a3: move type, translation (with cell-exit check) or rotation
        const uint4 wm = draw(R.key0, R.key1, sweep, tag, kPMove, 0, 0);
        bool translate = true;
        if (R.rot_on) {
            if (R.p_translate <= 0.0) translate = false;
            else if (R.p_translate < 1.0) translate = u01(wm.w) < R.p_translate;
        }
        double xn0 = pi.x, xn1 = pi.y, xn2 = pi.z;
        double4 qn = qo;
        Vec3 o = v3(0.0, 0.0, 0.0);
        if (translate) {
            cnt[kTranslate]++;
            xn0 = wrap_box(pi.x + R.d_max * s11(wm.x), R.L);
            xn1 = wrap_box(pi.y + R.d_max * s11(wm.y), R.L);
            xn2 = wrap_box(pi.z + R.d_max * s11(wm.z), R.L);
            if (cell_coord(xn0, S.sigma[0], R.L, R.w, nc) != cx ||
                cell_coord(xn1, S.sigma[1], R.L, R.w, nc) != cy ||
                cell_coord(xn2, S.sigma[2], R.L, R.w, nc) != cz) {
                cnt[kRejCell]++;
                continue;
            }
            o = v3(min_image(pi.x - xn0, R.L, R.half_L), min_image(pi.y - xn1, R.L, R.half_L),
                   min_image(pi.z - xn2, R.L, R.half_L));
        } else if (!propose_rotation(R, sweep, tag, qo, &qn)) {
            if (tid == 0) cnt[kCapHits]++;
            continue;
        }

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
            if (r2 < D2 || r2 < R.nb_cut2) {
                const double4 qj = P.quat[pj];
                if (r2 < D2 && pair_aniso(R, v3(d0, d1, d2), qn, qj)) ov = 1;
                if (r2 < R.nb_cut2) {
                    const int slot = atomicAdd(&s_nnb, 1);
                    s_nb[slot] = make_double4(d0, d1, d2, 0.0);
                    s_nbq[slot] = qj;
                }
            }
        }
        if (__syncthreads_or(ov)) {
            cnt[kRejOverlap]++;
            continue;
        }
        const int nnb = s_nnb;

        bool accept = true;
        if (R.has_dep) {
            // a5: Poisson count
            const uint4 wp = draw(R.key0, R.key1, sweep, tag, kPPoisson, 0, 0);
            const int n_p = poisson_count(Tab, R.nF, u53_int(wp.x, wp.y), lane);
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
                if (t < t_max) {
                    // the paired stream (hard interactions)
                    paired_point64(R.key0, R.key1, R.R_s, sweep, tag, t, e0, e1, e2);
                    inside = R.v0_cube || norm2(e0, e1, e2) < R.R_s2;
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
                    if (dep_aniso(R, v3(e0, e1, e2), qn) &&
                        !dep_aniso(R, v3(e0 - o.x, e1 - o.y, e2 - o.z), qo) &&
                        free_of_nb_aniso(R, v3(e0, e1, e2), s_nb, s_nbq, nnb))
                        blocking = true;
                }
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
                        const CbResult cr = cb_factor_aniso(R, sweep, tag, kb, o, qo, qn, s_nb, s_nbq,
                                                            nnb);
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
            if (tid == 0) {
                P.pos[i] = make_double4(xn0, xn1, xn2, 0.0);
                P.quat[i] = qn;
            }
        }
        __syncthreads();
    }

    if (tid != 0) {
#pragma unroll
        for (int k = 0; k < kNumCounters; ++k)
            if (k != kCbFwdOk && k != kCbRevOk && k != kCapHits) cnt[k] = 0;
    }
    flush_counters(P, r, cnt);
}

// Configuration check for anisotropic colloids (same contract as
// k_check_spheres): bit 1 of *flag for a coordinate outside [0, L), bit 0 for
// an overlapping pair.
__global__ void k_check_aniso(const __grid_constant__ SimParams P, int *flag)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.n_total) return;
    const int r = P.rep_of[g];
    const Rep &R = P.reps[r];
    if (g - R.off >= P.n_live[r]) return;
    const double4 pi = P.pos[g];
    if (!(pi.x >= 0.0 && pi.x < R.L && pi.y >= 0.0 && pi.y < R.L && pi.z >= 0.0 && pi.z < R.L)) {
        atomicOr(flag, 2);
        return;
    }
    const double4 qi = P.quat[g];
    const Sched &S = P.sched[r];
    const int *count = P.count[S.sweep & 1u];
    const int cx = cell_coord(pi.x, S.sigma[0], R.L, R.w, R.nc);
    const int cy = cell_coord(pi.y, S.sigma[1], R.L, R.w, R.nc);
    const int cz = cell_coord(pi.z, S.sigma[2], R.L, R.w, R.nc);
    const int ns = R.n_stencil;
    for (int t = 0; t < ns * ns * ns; ++t) {
        int dx, dy, dz;
        const int c = stencil_cell(R, t, cx, cy, cz, dx, dy, dz);
        const int m = min(count[c], P.cap);
        for (int s = 0; s < m; ++s) {
            const int j = __float_as_int(P.bins[bin_at(P, c, s)].w);
            if (j == g) continue;
            const double4 pj = P.pos[j];
            const Vec3 d = v3(min_image(pj.x - pi.x, R.L, R.half_L),
                              min_image(pj.y - pi.y, R.L, R.half_L),
                              min_image(pj.z - pi.z, R.L, R.half_L));
            if (pair_aniso(R, d, qi, P.quat[j])) atomicOr(flag, 1);
        }
    }
}

}  // namespace hpmc
