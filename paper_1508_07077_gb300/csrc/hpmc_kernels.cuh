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
    // FP32 form: thresholds rounded to float, and the certified margins
    float w32, L32, half_L32, R_s32, T_s32, T_dep32, T_contact32, nb_cut2_32, d_max32;
    float m_r2;            // |r2_fp32 - r2_fp64| bound for every squared distance tested
    float m_cell;          // bound on the error of a cell-relative coordinate
    double4 *pos;
    double4 *quat;
    float4 *rel;           // FP32 position relative to the origin of its cell (this sweep)
    const int *cell_start;
    const int *cell_idx;
    const unsigned long long *T;   // Poisson CDF table as integers ceil(F[k] 2^53)
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

// Offset of x from the origin of its cell c (FP32 working copy only).
__device__ __forceinline__ float cell_rel(double x, double sigma, double L, double w, int c)
{
    double s = x - sigma;
    if (s < 0.0) s = s + L;
    return (float)(s - (double)c * w);
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
                              Sched *sched_out, float4 *rel)
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
    if (rel) rel[i] = make_float4(cell_rel(p[0], sigma[0], L, w, cx), cell_rel(p[1], sigma[1], L, w, cy),
                                  cell_rel(p[2], sigma[2], L, w, cz), 0.0f);
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
// Poisson depletant count (Sec. III.B step 2): N_p = #{k : F[k] <= u} with
// u = m 2^-53 the 53-bit uniform.  F[k] <= m 2^-53  <=>  m >= ceil(F[k] 2^53),
// so the table is held as those integers and compared exactly in integer
// arithmetic.  One warp cooperates (3 levels of 32-way ballots, nF <= 32768).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long u53_int(uint32_t a, uint32_t b)
{
    return ((unsigned long long)(a >> 5) << 26) | (unsigned long long)(b >> 6);
}

__device__ __forceinline__ int poisson_count(const unsigned long long *T, int nF,
                                             unsigned long long m, int lane)
{
    const int i1 = (lane + 1) * 1024 - 1;
    const bool l1 = i1 < nF && T[i1] <= m;
    const int b1 = __popc(__ballot_sync(kFull, l1));
    const int i2 = b1 * 1024 + (lane + 1) * 32 - 1;
    const bool l2 = i2 < nF && T[i2] <= m;
    const int b2 = __popc(__ballot_sync(kFull, l2));
    const int i3 = b1 * 1024 + b2 * 32 + lane;
    const bool l3 = i3 < nF && T[i3] <= m;
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
    __shared__ int s_ncand, s_nnb, s_flag, s_acc, s_kmin;
    __shared__ int s_k[kMaxThreads];

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
            const int n_p = poisson_count(P.T, P.nF, u53_int(wp.x, wp.y), lane);
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
                // depletants classified up to an early exit (same count as a serial loop)
                if (P.n_trial == 0) {
                    if (blocking) atomicMin(&s_kmin, k);
                    const int any = __syncthreads_or(blocking);
                    if (any) {
                        if (tid == 0) {
                            c_block += 1;
                            c_eval += (unsigned long long)(s_kmin - k0 + 1);
                        }
                        rejected = true;
                        break;
                    }
                    if (tid == 0) c_eval += (unsigned long long)min(total, n_p - k0);
                } else {
                    // a7: CB factors of this pass, multiplied in ascending k
                    s_f[tid] = blocking ? cb_factor_fp64(P, sweep, tag, (uint32_t)k, o0, o1, o2,
                                                         s_nb, nnb, c_fwd, c_rev, c_cap)
                                        : -1.0;
                    s_k[tid] = k;
                    __syncthreads();
                    if (tid == 0) {
                        int zero = 0;
                        for (int q = 0; q < nthr; ++q) {
                            const double f = s_f[q];
                            if (f < 0.0) continue;
                            ++nblock;
                            ++c_block;
                            if (f == 0.0) {
                                zero = 1;
                                c_eval += (unsigned long long)(s_k[q] - k0 + 1);
                                break;
                            }
                            W = W * f;
                        }
                        if (!zero) c_eval += (unsigned long long)min(total, n_p - k0);
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

// ---------------------------------------------------------------------------
// FP32 form with a certified margin (sphere colloids).
//
// Every distance test of the FP64 specification, `r2 < T`, is first taken in
// FP32 on cell-relative coordinates.  m_r2 bounds |r2_fp32 - r2_fp64| plus the
// rounding of T (derived on the host from the cell width, R_s and d_max); a
// test with |r2_fp32 - T| <= m_r2 is re-taken exactly as the FP64
// specification states.  Hence every decision equals the FP64 decision, and
// positions are still accumulated in FP64.
// ---------------------------------------------------------------------------

// s11 in FP32: (w + 1/2) 2^-31 - 1 = v 2^-31 + 2^-32 with v = (int)(w ^ 2^31)
__device__ __forceinline__ float s11f(uint32_t w)
{
    return __fmaf_rn((float)(int)(w ^ 0x80000000u), 0x1p-31f, 0x1p-32f);
}

// R * s11(w) in FP32 (one rounding of the integer, one of the fma)
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

// Exact FP64 quantities of the current move, computed only when needed.
struct Move64 {
    double x0, x1, x2;  // new position, wrapped into [0, L)
    double o0, o1, o2;  // old position relative to the new one (minimum image)
};

__device__ __forceinline__ double wrap_box(double x, double L)
{
    if (x < 0.0) x = x + L;
    if (x >= L) x = x - L;
    return x;
}

__device__ __noinline__ Move64 move64(const SimParams &P, double4 pi, uint4 wm)
{
    Move64 m;
    m.x0 = wrap_box(pi.x + P.d_max * s11(wm.x), P.L);
    m.x1 = wrap_box(pi.y + P.d_max * s11(wm.y), P.L);
    m.x2 = wrap_box(pi.z + P.d_max * s11(wm.z), P.L);
    m.o0 = min_image(pi.x - m.x0, P.L, P.half_L);
    m.o1 = min_image(pi.y - m.x1, P.L, P.half_L);
    m.o2 = min_image(pi.z - m.x2, P.L, P.half_L);
    return m;
}

// Exact sphere-depletant test of depletant words w (relative to the new
// reference point: e = R_s s11(w)) against a colloid at c relative to the new
// reference point.
__device__ __noinline__ bool dep_exact(const SimParams &P, uint4 w, double c0, double c1, double c2)
{
    const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
    return SphereFP64::dep(P, e0 - c0, e1 - c1, e2 - c2);
}

__device__ __noinline__ bool ball_exact(const SimParams &P, uint4 w)
{
    const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
    return norm2(e0, e1, e2) < P.R_s2;
}

// Forward CB trial (relative to the OLD reference point, y = o + e): exact
// test of y against a colloid at c relative to the new reference point.
__device__ __noinline__ bool fwd_exact(const SimParams &P, uint4 w, const Move64 &M, double c0,
                                      double c1, double c2)
{
    const double e0 = P.R_s * s11(w.x), e1 = P.R_s * s11(w.y), e2 = P.R_s * s11(w.z);
    const double y0 = M.o0 + e0, y1 = M.o1 + e1, y2 = M.o2 + e2;
    return SphereFP64::dep(P, y0 - c0, y1 - c1, y2 - c2);
}

__device__ __forceinline__ void nb_exact_center(const SimParams &P, int j, const Move64 &M,
                                                double &c0, double &c1, double &c2)
{
    const double4 pj = P.pos[j];
    c0 = min_image(pj.x - M.x0, P.L, P.half_L);
    c1 = min_image(pj.y - M.x1, P.L, P.half_L);
    c2 = min_image(pj.z - M.x2, P.L, P.half_L);
}

struct MoveCtx32 {
    double4 pi;        // FP64 old position
    uint4 wm;          // move words
    float o0, o1, o2;  // old position relative to the new one (FP32)
    bool have64;
    Move64 m64;
};

__device__ __forceinline__ const Move64 &need64(const SimParams &P, MoveCtx32 &C)
{
    if (!C.have64) {
        C.m64 = move64(P, C.pi, C.wm);
        C.have64 = true;
    }
    return C.m64;
}

// Is point (v0,v1,v2) (FP32, relative to the new reference point) free of every
// neighbour?  kind 0: main depletant / reverse trial (exact base e),
// kind 1: forward trial (exact base o + e).
__device__ bool free_of_nb_fp32(const SimParams &P, float v0, float v1, float v2, const float4 *nb,
                                int nnb, uint4 w, int kind, MoveCtx32 &C,
                                unsigned long long &rechecks)
{
    for (int a = 0; a < nnb; ++a) {
        const float4 d = nb[a];
        const int t = tri(norm2f(v0 - d.x, v1 - d.y, v2 - d.z), P.T_dep32, P.m_r2);
        if (t == 1) return false;
        if (t == -1) {
            ++rechecks;
            const Move64 &M = need64(P, C);
            double c0, c1, c2;
            nb_exact_center(P, __float_as_int(d.w), M, c0, c1, c2);
            const bool ov = kind == 0 ? dep_exact(P, w, c0, c1, c2) : fwd_exact(P, w, M, c0, c1, c2);
            if (ov) return false;
        }
    }
    return true;
}

// Next point of an attempt stream inside the sampling ball (FP32 + exact
// recheck): returns false when the stream cap is reached.
__device__ __forceinline__ bool next_in_ball_fp32(const SimParams &P, uint32_t sweep, uint32_t tag,
                                                  uint32_t purpose, uint32_t sub, uint32_t &t,
                                                  uint32_t t_max, float r_hi, float r_lo,
                                                  uint4 &w, float &e0, float &e1, float &e2,
                                                  unsigned long long &rechecks)
{
    while (t < t_max) {
        w = draw(P.key0, P.key1, sweep, tag, purpose, sub, t);
        ++t;
        e0 = scaled_s11f(w.x, r_hi, r_lo);
        e1 = scaled_s11f(w.y, r_hi, r_lo);
        e2 = scaled_s11f(w.z, r_hi, r_lo);
        int in = tri(norm2f(e0, e1, e2), P.T_s32, P.m_r2);
        if (in == -1) {
            ++rechecks;
            in = ball_exact(P, w) ? 1 : 0;
        }
        if (in) return true;
    }
    return false;
}

// CB factor of one blocking depletant, FP32 form (same decisions as the FP64
// specification: Sec. III.D, Eq. 12).  For spheres the "overlaps the pose the
// ball is centred on" test is the ball test itself, so it is not repeated.
__device__ double cb_factor_fp32(const SimParams &P, uint32_t sweep, uint32_t tag, uint32_t k,
                                 MoveCtx32 &C, const float4 *nb, int nnb, float r_hi, float r_lo,
                                 unsigned long long &fwd_ok, unsigned long long &rev_ok,
                                 unsigned long long &caps, unsigned long long &rechecks)
{
    const int n_fwd = P.n_trial, n_rev = P.n_trial - 1;
    int nf = 0, nr = 0, found = 0;
    uint32_t t = 0;
    uint4 w;
    float e0, e1, e2;
    while (found < n_fwd &&
           next_in_ball_fp32(P, sweep, tag, kPCbFwd, k, t, 64u * (uint32_t)(n_fwd + 1), r_hi, r_lo,
                             w, e0, e1, e2, rechecks)) {
        ++found;
        const float y0 = C.o0 + e0, y1 = C.o1 + e1, y2 = C.o2 + e2;
        int tn = tri(norm2f(y0, y1, y2), P.T_dep32, P.m_r2);  // overlaps the new pose?
        if (tn == -1) {
            ++rechecks;
            tn = fwd_exact(P, w, need64(P, C), 0.0, 0.0, 0.0) ? 1 : 0;
        }
        if (tn) continue;
        if (!free_of_nb_fp32(P, y0, y1, y2, nb, nnb, w, 1, C, rechecks)) continue;
        ++nf;
    }
    if (found < n_fwd) ++caps;
    t = 0;
    found = 0;
    while (found < n_rev &&
           next_in_ball_fp32(P, sweep, tag, kPCbRev, k, t, 64u * (uint32_t)(n_rev + 1), r_hi, r_lo,
                             w, e0, e1, e2, rechecks)) {
        ++found;
        int to = tri(norm2f(e0 - C.o0, e1 - C.o1, e2 - C.o2), P.T_dep32, P.m_r2);  // old pose?
        if (to == -1) {
            ++rechecks;
            const Move64 &M = need64(P, C);
            to = dep_exact(P, w, M.o0, M.o1, M.o2) ? 1 : 0;
        }
        if (to) continue;
        if (!free_of_nb_fp32(P, e0, e1, e2, nb, nnb, w, 0, C, rechecks)) continue;
        ++nr;
    }
    if (found < n_rev) ++caps;
    fwd_ok += (unsigned long long)nf;
    rev_ok += (unsigned long long)nr;
    return (double)nf / (double)(nr + 1);
}

__global__ void __launch_bounds__(kMaxThreads) k_phase_sphere_fp32(SimParams P, int phase)
{
    __shared__ float4 s_cpos[kMaxCand];  // candidates relative to this cell's origin; index in .w
    __shared__ float4 s_nb[kMaxCand];    // neighbours relative to the new position; index in .w
    __shared__ double s_f[kMaxThreads];
    __shared__ int s_warp[kMaxThreads / 32];
    __shared__ int s_ncand, s_nnb, s_flag, s_acc, s_self, s_kmin;
    __shared__ int s_k[kMaxThreads];

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

    // candidates of the 27-cell stencil, relative to this cell's origin
    if (tid == 0) s_ncand = 0;
    __syncthreads();
    const int ns = P.n_stencil;
    if (tid < ns * ns * ns) {
        const int ox = tid % ns, oy = (tid / ns) % ns, oz = tid / (ns * ns);
        int nx, ny, nz, dx, dy, dz;
        if (nc == 2) {
            nx = ox; ny = oy; nz = oz;
            dx = ox - cx; dy = oy - cy; dz = oz - cz;
        } else {
            nx = (cx + ox - 1 + nc) % nc;
            ny = (cy + oy - 1 + nc) % nc;
            nz = (cz + oz - 1 + nc) % nc;
            dx = ox - 1; dy = oy - 1; dz = oz - 1;
        }
        const float fx = (float)dx * P.w32, fy = (float)dy * P.w32, fz = (float)dz * P.w32;
        const int c = nx + nc * (ny + nc * nz);
        const int lo = P.cell_start[c], hi = P.cell_start[c + 1];
        for (int s = lo; s < hi; ++s) {
            const int j = P.cell_idx[s];
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

    unsigned long long c_moves = 0, c_acc = 0, c_cell = 0, c_ov = 0, c_dep = 0, c_cb = 0,
                       c_drawn = 0, c_eval = 0, c_block = 0, c_fwd = 0, c_rev = 0, c_cap = 0,
                       c_rck = 0;

    for (int s = begin; s < end; ++s) {
        const int i = P.cell_idx[s];
        const uint32_t tag = (uint32_t)i;
        ++c_moves;
        MoveCtx32 C;
        C.have64 = false;
        C.pi = P.pos[i];
        C.wm = draw(P.key0, P.key1, sweep, tag, kPMove, 0, 0);
        const float4 ri = P.rel[i];

        // a3: proposal in cell-relative FP32; cell-exit check with margin
        const float rn0 = ri.x + scaled_s11f(C.wm.x, dm_hi, dm_lo);
        const float rn1 = ri.y + scaled_s11f(C.wm.y, dm_hi, dm_lo);
        const float rn2 = ri.z + scaled_s11f(C.wm.z, dm_hi, dm_lo);
        const float mc = P.m_cell, wc = P.w32;
        const bool out = rn0 < -mc || rn0 > wc + mc || rn1 < -mc || rn1 > wc + mc ||
                         rn2 < -mc || rn2 > wc + mc;
        const bool edge = rn0 <= mc || rn0 >= wc - mc || rn1 <= mc || rn1 >= wc - mc ||
                          rn2 <= mc || rn2 >= wc - mc;
        bool exits = out;
        if (!out && edge) {
            const Move64 &Mx = need64(P, C);
            exits = cell_coord(Mx.x0, S.sigma[0], P.L, P.w, nc) != cx ||
                    cell_coord(Mx.x1, S.sigma[1], P.L, P.w, nc) != cy ||
                    cell_coord(Mx.x2, S.sigma[2], P.L, P.w, nc) != cz;
            if (tid == 0) ++c_rck;
        }
        if (exits) {
            ++c_cell;
            continue;
        }
        C.o0 = ri.x - rn0;
        C.o1 = ri.y - rn1;
        C.o2 = ri.z - rn2;

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
                const Move64 &Mx = need64(P, C);
                double e0, e1, e2;
                nb_exact_center(P, pj, Mx, e0, e1, e2);
                t = norm2(e0, e1, e2) < P.contact2 ? 1 : 0;
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
                        in = ball_exact(P, w) ? 1 : 0;
                    }
                    inside = in != 0;
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
                bool blocking = false;
                if (inside && k < n_p) {
                    // inside the ball = overlaps the new pose (spheres); ignored if it
                    // overlaps the old configuration
                    int to = tri(norm2f(e0 - C.o0, e1 - C.o1, e2 - C.o2), P.T_dep32, P.m_r2);
                    if (to == -1) {
                        ++c_rck;
                        const Move64 &Mx = need64(P, C);
                        to = dep_exact(P, w, Mx.o0, Mx.o1, Mx.o2) ? 1 : 0;
                    }
                    if (!to) blocking = free_of_nb_fp32(P, e0, e1, e2, s_nb, nnb, w, 0, C, c_rck);
                }
                // depletants classified up to an early exit (same count as a serial loop)
                if (P.n_trial == 0) {
                    if (blocking) atomicMin(&s_kmin, k);
                    if (__syncthreads_or(blocking)) {
                        if (tid == 0) {
                            c_block += 1;
                            c_eval += (unsigned long long)(s_kmin - k0 + 1);
                        }
                        rejected = true;
                        break;
                    }
                    if (tid == 0) c_eval += (unsigned long long)min(total, n_p - k0);
                } else {
                    s_f[tid] = blocking ? cb_factor_fp32(P, sweep, tag, (uint32_t)k, C, s_nb, nnb,
                                                         r_hi, r_lo, c_fwd, c_rev, c_cap, c_rck)
                                        : -1.0;
                    s_k[tid] = k;
                    __syncthreads();
                    if (tid == 0) {
                        int zero = 0;
                        for (int q = 0; q < nthr; ++q) {
                            const double f = s_f[q];
                            if (f < 0.0) continue;
                            ++nblock;
                            ++c_block;
                            if (f == 0.0) {
                                zero = 1;
                                c_eval += (unsigned long long)(s_k[q] - k0 + 1);
                                break;
                            }
                            W = W * f;
                        }
                        if (!zero) c_eval += (unsigned long long)min(total, n_p - k0);
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
            if (tid == 0) {
                const Move64 &Mx = need64(P, C);
                P.pos[i] = make_double4(Mx.x0, Mx.x1, Mx.x2, 0.0);
                const float4 rnew = make_float4(cell_rel(Mx.x0, S.sigma[0], P.L, P.w, cx),
                                                cell_rel(Mx.x1, S.sigma[1], P.L, P.w, cy),
                                                cell_rel(Mx.x2, S.sigma[2], P.L, P.w, cz),
                                                __int_as_float(i));
                P.rel[i] = make_float4(rnew.x, rnew.y, rnew.z, 0.0f);
                s_cpos[s_self] = rnew;
            }
        }
        __syncthreads();
    }

    unsigned long long *cnt = P.counters + (size_t)(blockIdx.x % kCounterSlots) * kNumCounters;
    if (tid == 0) {
        atomicAdd(cnt + kMoves, c_moves);
        atomicAdd(cnt + kAccept, c_acc);
        atomicAdd(cnt + kTranslate, c_moves);
        if (c_cell) atomicAdd(cnt + kRejCell, c_cell);
        if (c_ov) atomicAdd(cnt + kRejOverlap, c_ov);
        if (c_dep) atomicAdd(cnt + kRejDep, c_dep);
        if (c_cb) atomicAdd(cnt + kRejCb, c_cb);
        if (c_drawn) atomicAdd(cnt + kDepDrawn, c_drawn);
        if (c_eval) atomicAdd(cnt + kDepEval, c_eval);
        if (c_block) atomicAdd(cnt + kDepBlocking, c_block);
    }
    if (c_fwd) atomicAdd(cnt + kCbFwdOk, c_fwd);
    if (c_rev) atomicAdd(cnt + kCbRevOk, c_rev);
    if (c_cap) atomicAdd(cnt + kCapHits, c_cap);
    if (c_rck) atomicAdd(cnt + kRechecks, c_rck);
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
