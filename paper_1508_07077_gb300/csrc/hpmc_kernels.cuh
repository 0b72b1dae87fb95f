// Device code of the implicit-depletant HPMC library (sm_103a).
//
// Method: Glaser, Karas & Glotzer, arXiv:1508.07077.
//   Sec. III.E  checkerboard of active cells, random grid shift and colour order
//   Sec. III.B  trial move, Poisson number of depletants, reject on overlap
//   Sec. III.C  depletants sampled in the circumsphere of the NEW pose; those
//               overlapping the old configuration are ignored
//   Sec. III.D  configurational-bias reinsertion, Eq. (12)
//   App. A      depletants of one move are processed by cooperating threads
//
// Every FP64 expression on a decision path is written in the operation order
// of the library's specification and compiled with -fmad=false, so decisions
// and positions are bit-identical to any other faithful implementation.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hpmc {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kMaxCand = 256;        // colloids in a 27-cell neighbourhood (capacity)
constexpr int kMaxThreads = 256;     // 8 warps per colloid at most
constexpr int kCounterSlots = 128;   // counters are spread over slots to avoid hot atomics
constexpr int kNumCounters = 16;

enum Counter {
    kMoves = 0, kAccept, kRejCell, kRejOverlap, kRejDep, kRejCb, kDepDrawn,
    kTranslate, kDepEval, kDepBlocking, kCbFwdOk, kCbRevOk, kCapHits, kRechecks
};

enum DevError { kErrNone = 0, kErrCandCap = 1, kErrTableCap = 2 };

enum Purpose : uint32_t {
    kPSched = 0, kPMove = 1, kPRot = 2, kPPoisson = 3, kPDep = 4,
    kPCbFwd = 5, kPCbRev = 6, kPAccept = 7
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 draw(uint32_t k0, uint32_t k1, uint32_t sweep,
                                      uint32_t stream, uint32_t purpose,
                                      uint32_t sub, uint32_t t)
{
    return philox4x32_10(make_uint4(sweep, stream, (purpose << 24) | (sub & 0xFFFFFFu), t),
                         k0, k1);
}

// word -> real maps (exact in FP64)
__device__ __forceinline__ double u01(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }
__device__ __forceinline__ double s11(uint32_t w) { return ((double)w + 0.5) * 0x1p-31 - 1.0; }
__device__ __forceinline__ double u53(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * 0x1p-53;
}

// ---------------------------------------------------------------------------
// Parameters shared by the kernels of one sweep.
// ---------------------------------------------------------------------------
struct Sched {
    double sigma[3];
    int perm[8];
    int pad;
};

struct SimParams {
    int n, nc, half_nc, n_stencil;
    double L, half_L, w;
    int shape, n_trial, has_dep, nF;
    double R_s, R_s2;      // sampling sphere radius (R_circ + q/2) and its square
    double R_dep2;         // sphere-depletant contact distance squared
    double contact2;       // sphere-sphere contact distance squared
    double nb_cut2;        // neighbours farther than this cannot meet a depletant
    double d_max, alpha, p_translate;
    int move_mode;         // 0 translate only, 1 rotate only, 2 both
    uint32_t key0, key1;
    double4 *pos;
    double4 *quat;
    const int *cell_start;
    const int *cell_idx;
    const double *F;
    const Sched *sched;
    const unsigned long long *sweep;
    unsigned long long *counters;
    int *err;
};

// Sec. III.E: cell coordinate of x under grid shift sigma.
__device__ __forceinline__ int cell_coord(double x, double sigma, double L, double w, int nc)
{
    double s = x - sigma;
    if (s < 0.0) s = s + L;
    int c = (int)(s / w);
    if (c >= nc) c = nc - 1;
    if (c < 0) c = 0;
    return c;
}

__device__ __forceinline__ double min_image(double d, double L, double half_L)
{
    if (d > half_L) d = d - L;
    else if (d < -half_L) d = d + L;
    return d;
}

__device__ __forceinline__ double norm2(double a, double b, double c)
{
    return (a * a + b * b) + c * c;
}

// ---------------------------------------------------------------------------
// Sweep schedule + cell counting (Sec. III.E).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void schedule_shift(uint32_t k0, uint32_t k1, uint32_t sweep,
                                               double w, double sigma[3])
{
    const uint4 a = draw(k0, k1, sweep, 0xFFFFFFFFu, kPSched, 0, 0);
    sigma[0] = w * u01(a.x);
    sigma[1] = w * u01(a.y);
    sigma[2] = w * u01(a.z);
}

__device__ __forceinline__ void schedule_perm(uint32_t k0, uint32_t k1, uint32_t sweep,
                                              int perm[8])
{
    const uint4 b = draw(k0, k1, sweep, 0xFFFFFFFFu, kPSched, 1, 0);
    const uint4 c = draw(k0, k1, sweep, 0xFFFFFFFFu, kPSched, 2, 0);
    const uint32_t words[8] = {b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
    for (int i = 0; i < 8; ++i) perm[i] = i;
    for (int i = 7; i >= 1; --i) {
        const int j = (int)(((unsigned long long)words[7 - i] * (unsigned long long)(i + 1)) >> 32);
        const int t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
}

// One thread per colloid: its cell and the cell's population.  Block 0 also
// writes the sweep's schedule.  pos is read with element stride `stride`
// doubles (4 for the library's double4 storage, 3 for caller arrays).
__global__ void k_cells_count(int n, double L, double w, int nc, const double *pos, int stride,
                              uint32_t k0, uint32_t k1, const unsigned long long *sweep_ptr,
                              unsigned long long sweep_val, int *cell_of, int *count,
                              Sched *sched_out)
{
    const uint32_t sweep = (uint32_t)(sweep_ptr ? *sweep_ptr : sweep_val);
    double sigma[3];
    schedule_shift(k0, k1, sweep, w, sigma);
    if (sched_out && blockIdx.x == 0 && threadIdx.x == 0) {
        Sched s;
        s.sigma[0] = sigma[0];
        s.sigma[1] = sigma[1];
        s.sigma[2] = sigma[2];
        schedule_perm(k0, k1, sweep, s.perm);
        s.pad = 0;
        *sched_out = s;
    }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *p = pos + (size_t)i * stride;
    const int cx = cell_coord(p[0], sigma[0], L, w, nc);
    const int cy = cell_coord(p[1], sigma[1], L, w, nc);
    const int cz = cell_coord(p[2], sigma[2], L, w, nc);
    const int c = cx + nc * (cy + nc * cz);
    cell_of[i] = c;
    atomicAdd(count + c, 1);
}

// Single-block exclusive scan of the cell populations into cell_start; the
// count array is overwritten with the scatter cursors (= cell_start).
__global__ void __launch_bounds__(1024) k_cells_scan(int ncell, int *count, int *cell_start)
{
    __shared__ int s_part[1024];
    const int tid = threadIdx.x;
    const int per = (ncell + blockDim.x - 1) / blockDim.x;
    const int lo = min(tid * per, ncell);
    const int hi = min(lo + per, ncell);
    int sum = 0;
    for (int c = lo; c < hi; ++c) sum += count[c];
    s_part[tid] = sum;
    __syncthreads();
    // Hillis-Steele inclusive scan of the per-thread sums
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int v = tid >= off ? s_part[tid - off] : 0;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    int run = s_part[tid] - sum;
    for (int c = lo; c < hi; ++c) {
        const int k = count[c];
        cell_start[c] = run;
        count[c] = run;
        run += k;
    }
    if (tid == (int)blockDim.x - 1) cell_start[ncell] = s_part[tid];
}

__global__ void k_cells_scatter(int n, const int *cell_of, int *cursor, int *cell_idx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int slot = atomicAdd(cursor + cell_of[i], 1);
    cell_idx[slot] = i;
}

// Within each cell, ascending colloid index (makes the list deterministic).
__global__ void k_cells_sort(int ncell, const int *cell_start, int *cell_idx)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int lo = cell_start[c], hi = cell_start[c + 1];
    for (int a = lo + 1; a < hi; ++a) {
        const int v = cell_idx[a];
        int b = a - 1;
        while (b >= lo && cell_idx[b] > v) {
            cell_idx[b + 1] = cell_idx[b];
            --b;
        }
        cell_idx[b + 1] = v;
    }
}

__global__ void k_sweep_end(unsigned long long *sweep) { *sweep += 1ull; }

// ---------------------------------------------------------------------------
// Poisson depletant count (Sec. III.B step 2): N_p = #{k : F[k] <= u}, F the
// cumulative table; one warp cooperates (3 levels of 32-way ballots, nF <= 32768).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int poisson_count(const double *F, int nF, double u, int lane)
{
    const int i1 = (lane + 1) * 1024 - 1;
    const bool l1 = i1 < nF && F[i1] <= u;
    const int b1 = __popc(__ballot_sync(kFull, l1));
    const int i2 = b1 * 1024 + (lane + 1) * 32 - 1;
    const bool l2 = i2 < nF && F[i2] <= u;
    const int b2 = __popc(__ballot_sync(kFull, l2));
    const int i3 = b1 * 1024 + b2 * 32 + lane;
    const bool l3 = i3 < nF && F[i3] <= u;
    const int b3 = __popc(__ballot_sync(kFull, l3));
    return b1 * 1024 + b2 * 32 + b3;
}

// ---------------------------------------------------------------------------
// Sphere overlap primitives (FP64, specification order).
// ---------------------------------------------------------------------------
struct SphereFP64 {
    // depletant at v (relative to the colloid centre) overlaps the colloid
    static __device__ __forceinline__ bool dep(const SimParams &P, double v0, double v1, double v2)
    {
        return norm2(v0, v1, v2) < P.R_dep2;
    }
};

// Is the point y (relative to the new reference point) free of every
// neighbour in the shared list?
__device__ __forceinline__ bool free_of_nb_fp64(const SimParams &P, double y0, double y1,
                                                double y2, const double4 *nb, int nnb)
{
    for (int a = 0; a < nnb; ++a) {
        const double4 d = nb[a];
        if (SphereFP64::dep(P, y0 - d.x, y1 - d.y, y2 - d.z)) return false;
    }
    return true;
}

// Configurational-bias factor of blocking depletant k (Sec. III.D, Eq. 12):
// f = N'_insert / (N_insert + 1); forward trials in the old circumsphere,
// n_trial - 1 reverse trials in the new one.  One thread evaluates it.
__device__ double cb_factor_fp64(const SimParams &P, uint32_t sweep, uint32_t tag, uint32_t k,
                                 double o0, double o1, double o2, const double4 *nb, int nnb,
                                 unsigned long long &fwd_ok, unsigned long long &rev_ok,
                                 unsigned long long &caps)
{
    const int n_fwd = P.n_trial, n_rev = P.n_trial - 1;
    int nf = 0, nr = 0, found = 0;
    uint32_t t = 0, t_max = 64u * (uint32_t)(n_fwd + 1);
    while (found < n_fwd && t < t_max) {
        const uint4 w = draw(P.key0, P.key1, sweep, tag, kPCbFwd, k, t);
        ++t;
        const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
        if (!(norm2(e0, e1, e2) < P.R_s2)) continue;
        ++found;
        const double y0 = o0 + e0, y1 = o1 + e1, y2 = o2 + e2;
        if (!SphereFP64::dep(P, e0, e1, e2)) continue;      // must overlap the old pose
        if (SphereFP64::dep(P, y0, y1, y2)) continue;       // must not overlap the new pose
        if (!free_of_nb_fp64(P, y0, y1, y2, nb, nnb)) continue;
        ++nf;
    }
    if (found < n_fwd) ++caps;
    t = 0;
    t_max = 64u * (uint32_t)(n_rev + 1);
    found = 0;
    while (found < n_rev && t < t_max) {
        const uint4 w = draw(P.key0, P.key1, sweep, tag, kPCbRev, k, t);
        ++t;
        const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
        if (!(norm2(e0, e1, e2) < P.R_s2)) continue;
        ++found;
        if (!SphereFP64::dep(P, e0, e1, e2)) continue;                  // overlaps the new pose
        if (SphereFP64::dep(P, e0 - o0, e1 - o1, e2 - o2)) continue;   // not the old pose
        if (!free_of_nb_fp64(P, e0, e1, e2, nb, nnb)) continue;
        ++nr;
    }
    if (found < n_rev) ++caps;
    fwd_ok += (unsigned long long)nf;
    rev_ok += (unsigned long long)nr;
    return (double)nf / (double)(nr + 1);
}

// ---------------------------------------------------------------------------
// One colour phase: a CTA per active cell, blockDim = 32 * warps_per_colloid.
// The colloids of the cell move one after another in ascending index; the
// depletants of each move are spread over the CTA's threads (App. A).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMaxThreads) k_phase_sphere_fp64(SimParams P, int phase)
{
    __shared__ int s_cand[kMaxCand];
    __shared__ double4 s_nb[kMaxCand];
    __shared__ double s_f[kMaxThreads];
    __shared__ int s_warp[kMaxThreads / 32];
    __shared__ int s_ncand, s_nnb, s_flag, s_acc;

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
    const uint32_t sweep = (uint32_t)(*P.sweep);
    const Sched S = *P.sched;
    const int colour = S.perm[phase];
    const int h = P.half_nc, nc = P.nc;
    const int a = blockIdx.x;
    const int cx = 2 * (a % h) + (colour & 1);
    const int cy = 2 * ((a / h) % h) + ((colour >> 1) & 1);
    const int cz = 2 * (a / (h * h)) + ((colour >> 2) & 1);
    const int cell = cx + nc * (cy + nc * cz);
    const int begin = P.cell_start[cell], end = P.cell_start[cell + 1];
    if (begin == end) return;

    // Candidate neighbours: every colloid of the (deduplicated) 27-cell stencil.
    if (tid == 0) s_ncand = 0;
    __syncthreads();
    const int ns = P.n_stencil;
    if (tid < ns * ns * ns) {
        const int ox = tid % ns, oy = (tid / ns) % ns, oz = tid / (ns * ns);
        int nx, ny, nz;
        if (nc == 2) { nx = ox; ny = oy; nz = oz; }
        else {
            nx = (cx + ox - 1 + nc) % nc;
            ny = (cy + oy - 1 + nc) % nc;
            nz = (cz + oz - 1 + nc) % nc;
        }
        const int c = nx + nc * (ny + nc * nz);
        const int lo = P.cell_start[c], hi = P.cell_start[c + 1];
        for (int s = lo; s < hi; ++s) {
            const int slot = atomicAdd(&s_ncand, 1);
            if (slot < kMaxCand) s_cand[slot] = P.cell_idx[s];
        }
    }
    __syncthreads();
    const int M = s_ncand;
    if (M > kMaxCand) {
        if (tid == 0) atomicCAS(P.err, kErrNone, kErrCandCap);
        return;
    }

    unsigned long long c_moves = 0, c_acc = 0, c_cell = 0, c_ov = 0, c_dep = 0, c_cb = 0,
                       c_drawn = 0, c_eval = 0, c_block = 0, c_fwd = 0, c_rev = 0, c_cap = 0;

    for (int s = begin; s < end; ++s) {
        const int i = P.cell_idx[s];
        const uint32_t tag = (uint32_t)i;
        const double4 pi = P.pos[i];
        ++c_moves;

        // a3: translation proposal, wrap, cell-exit check
        const uint4 wm = draw(P.key0, P.key1, sweep, tag, kPMove, 0, 0);
        double xn0 = pi.x + P.d_max * s11(wm.x);
        double xn1 = pi.y + P.d_max * s11(wm.y);
        double xn2 = pi.z + P.d_max * s11(wm.z);
        if (xn0 < 0.0) xn0 = xn0 + P.L;
        if (xn0 >= P.L) xn0 = xn0 - P.L;
        if (xn1 < 0.0) xn1 = xn1 + P.L;
        if (xn1 >= P.L) xn1 = xn1 - P.L;
        if (xn2 < 0.0) xn2 = xn2 + P.L;
        if (xn2 >= P.L) xn2 = xn2 - P.L;
        if (cell_coord(xn0, S.sigma[0], P.L, P.w, nc) != cx ||
            cell_coord(xn1, S.sigma[1], P.L, P.w, nc) != cy ||
            cell_coord(xn2, S.sigma[2], P.L, P.w, nc) != cz) {
            ++c_cell;
            continue;
        }
        const double o0 = min_image(pi.x - xn0, P.L, P.half_L);
        const double o1 = min_image(pi.y - xn1, P.L, P.half_L);
        const double o2 = min_image(pi.z - xn2, P.L, P.half_L);

        // a4: colloid overlap at the new pose; collect neighbours in range
        if (tid == 0) s_nnb = 0;
        __syncthreads();
        int ov = 0;
        for (int j = tid; j < M; j += nthr) {
            const int pj = s_cand[j];
            if (pj == i) continue;
            const double4 xj = P.pos[pj];
            const double d0 = min_image(xj.x - xn0, P.L, P.half_L);
            const double d1 = min_image(xj.y - xn1, P.L, P.half_L);
            const double d2 = min_image(xj.z - xn2, P.L, P.half_L);
            const double r2 = norm2(d0, d1, d2);
            if (r2 < P.contact2) ov = 1;
            if (r2 < P.nb_cut2) {
                const int slot = atomicAdd(&s_nnb, 1);
                s_nb[slot] = make_double4(d0, d1, d2, 0.0);
            }
        }
        if (__syncthreads_or(ov)) {
            ++c_ov;
            continue;
        }
        const int nnb = s_nnb;

        bool accept = true;
        if (P.has_dep) {
            // a5: Poisson count
            const uint4 wp = draw(P.key0, P.key1, sweep, tag, kPPoisson, 0, 0);
            const int n_p = poisson_count(P.F, P.nF, u53(wp.x, wp.y), lane);
            c_drawn += (unsigned long long)n_p;

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
                    const uint4 w = draw(P.key0, P.key1, sweep, tag, kPDep, 0, t);
                    e0 = P.R_s * s11(w.x);
                    e1 = P.R_s * s11(w.y);
                    e2 = P.R_s * s11(w.z);
                    inside = norm2(e0, e1, e2) < P.R_s2;
                }
                const unsigned bal = __ballot_sync(kFull, inside);
                if (lane == 0) s_warp[warp] = __popc(bal);
                __syncthreads();
                int base = 0, total = 0;
                for (int q = 0; q < nwarps; ++q) {
                    const int cnt = s_warp[q];
                    base += q < warp ? cnt : 0;
                    total += cnt;
                }
                const int k = k0 + base + __popc(bal & ((1u << lane) - 1u));
                const bool valid = inside && k < n_p;
                bool blocking = false;
                if (valid) {
                    // irrelevant unless it overlaps the new pose; ignored if it
                    // overlaps the old configuration
                    if (SphereFP64::dep(P, e0, e1, e2) &&
                        !SphereFP64::dep(P, e0 - o0, e1 - o1, e2 - o2) &&
                        free_of_nb_fp64(P, e0, e1, e2, s_nb, nnb))
                        blocking = true;
                }
                if (tid == 0) c_eval += (unsigned long long)min(total, n_p - k0);
                if (P.n_trial == 0) {
                    const int any = __syncthreads_or(blocking);
                    if (any) {
                        if (tid == 0) c_block += 1;
                        rejected = true;
                        break;
                    }
                } else {
                    // a7: CB factors of this pass, multiplied in ascending k
                    s_f[tid] = blocking ? cb_factor_fp64(P, sweep, tag, (uint32_t)k, o0, o1, o2,
                                                         s_nb, nnb, c_fwd, c_rev, c_cap)
                                        : -1.0;
                    __syncthreads();
                    if (tid == 0) {
                        int zero = 0;
                        for (int q = 0; q < nthr; ++q) {
                            const double f = s_f[q];
                            if (f < 0.0) continue;
                            ++nblock;
                            ++c_block;
                            if (f == 0.0) { zero = 1; break; }
                            W = W * f;
                        }
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
                // thread 0 alone drew the acceptance uniform
                if (tid == 0) s_acc = accept ? 1 : 0;
                __syncthreads();
                accept = s_acc != 0;
            }
        }
        // a8: commit
        if (accept) {
            ++c_acc;
            if (tid == 0) P.pos[i] = make_double4(xn0, xn1, xn2, 0.0);
        }
        __syncthreads();
    }

    if (tid == 0) {
        unsigned long long *cnt = P.counters + (size_t)(blockIdx.x % kCounterSlots) * kNumCounters;
        atomicAdd(cnt + kMoves, c_moves);
        atomicAdd(cnt + kAccept, c_acc);
        if (c_cell) atomicAdd(cnt + kRejCell, c_cell);
        if (c_ov) atomicAdd(cnt + kRejOverlap, c_ov);
        if (c_dep) atomicAdd(cnt + kRejDep, c_dep);
        if (c_cb) atomicAdd(cnt + kRejCb, c_cb);
        if (c_drawn) atomicAdd(cnt + kDepDrawn, c_drawn);
        atomicAdd(cnt + kTranslate, c_moves);
        if (c_eval) atomicAdd(cnt + kDepEval, c_eval);
        if (c_block) atomicAdd(cnt + kDepBlocking, c_block);
        if (c_fwd) atomicAdd(cnt + kCbFwdOk, c_fwd);
        if (c_rev) atomicAdd(cnt + kCbRevOk, c_rev);
        if (c_cap) atomicAdd(cnt + kCapHits, c_cap);
    } else if (c_fwd || c_rev || c_cap) {
        // CB counts accumulated by other threads
        unsigned long long *cnt = P.counters + (size_t)(blockIdx.x % kCounterSlots) * kNumCounters;
        if (c_fwd) atomicAdd(cnt + kCbFwdOk, c_fwd);
        if (c_rev) atomicAdd(cnt + kCbRevOk, c_rev);
        if (c_cap) atomicAdd(cnt + kCapHits, c_cap);
    }
}

// Overlap check of a whole configuration (one thread per colloid, brute force
// over the 27 cells): sets *flag if any pair of spheres overlaps or a
// coordinate is outside [0, L).
__global__ void k_check_spheres(SimParams P, int *flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const double4 pi = P.pos[i];
    if (!(pi.x >= 0.0 && pi.x < P.L && pi.y >= 0.0 && pi.y < P.L && pi.z >= 0.0 && pi.z < P.L)) {
        atomicOr(flag, 2);
        return;
    }
    const Sched S = *P.sched;
    const int nc = P.nc, ns = P.n_stencil;
    const int cx = cell_coord(pi.x, S.sigma[0], P.L, P.w, nc);
    const int cy = cell_coord(pi.y, S.sigma[1], P.L, P.w, nc);
    const int cz = cell_coord(pi.z, S.sigma[2], P.L, P.w, nc);
    for (int t = 0; t < ns * ns * ns; ++t) {
        const int ox = t % ns, oy = (t / ns) % ns, oz = t / (ns * ns);
        int nx, ny, nz;
        if (nc == 2) { nx = ox; ny = oy; nz = oz; }
        else {
            nx = (cx + ox - 1 + nc) % nc;
            ny = (cy + oy - 1 + nc) % nc;
            nz = (cz + oz - 1 + nc) % nc;
        }
        const int c = nx + nc * (ny + nc * nz);
        for (int s = P.cell_start[c]; s < P.cell_start[c + 1]; ++s) {
            const int j = P.cell_idx[s];
            if (j == i) continue;
            const double4 pj = P.pos[j];
            const double r2 = norm2(min_image(pj.x - pi.x, P.L, P.half_L),
                                    min_image(pj.y - pi.y, P.L, P.half_L),
                                    min_image(pj.z - pi.z, P.L, P.half_L));
            if (r2 < P.contact2) atomicOr(flag, 1);
        }
    }
}

// Layout conversion between caller arrays (n x 3, n x 4) and device storage.
__global__ void k_unpack(int n, const double *pos3, const double *quat4, double4 *pos,
                         double4 *quat)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (pos3) pos[i] = make_double4(pos3[3 * i], pos3[3 * i + 1], pos3[3 * i + 2], 0.0);
    if (quat4 && quat)
        quat[i] = make_double4(quat4[4 * i], quat4[4 * i + 1], quat4[4 * i + 2], quat4[4 * i + 3]);
}

__global__ void k_pack(int n, const double4 *pos, const double4 *quat, double *pos3, double *quat4)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (pos3) {
        const double4 p = pos[i];
        pos3[3 * i] = p.x;
        pos3[3 * i + 1] = p.y;
        pos3[3 * i + 2] = p.z;
    }
    if (quat4 && quat) {
        const double4 q = quat[i];
        quat4[4 * i] = q.x;
        quat4[4 * i + 1] = q.y;
        quat4[4 * i + 2] = q.z;
        quat4[4 * i + 3] = q.w;
    }
}

}  // namespace hpmc
