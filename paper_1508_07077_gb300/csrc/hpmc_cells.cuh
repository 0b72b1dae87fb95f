// Checkerboard cell lists (Sec. III.E), two layouts.
//
// * Binned (the sweep's own): one kernel per sweep computes the grid shift
//   and colour order and bins every colloid into fixed-capacity cell slots
//   with one atomic each; a slot holds the colloid's FP32 offset from its cell
//   origin and its index.  The order inside a bin is arbitrary; the CTA that
//   moves a cell's colloids restores ascending index order itself.
// * CSR (the standalone hpmc_cell_list): count -> exclusive scan -> scatter ->
//   per-cell sort, giving cell_start[ncell + 1] and cell_idx[n] in ascending
//   index order within each cell.
#pragma once

#include "hpmc_common.cuh"

namespace hpmc {

// Cell of colour-phase CTA `a` of replica r in phase `phase`.
// Entry: (global cell, replica, cx | cy << 10 | cz << 20, nc | (sweep & 1) << 16),
// everything a phase CTA needs to start loading its stencil.
__device__ __forceinline__ int4 phase_task(const Rep &R, int r, const int perm[8], int phase, int a,
                                           uint32_t sweep)
{
    const int colour = perm[phase];
    const int h = R.half_nc, nc = R.nc;
    const int cx = 2 * (a % h) + (colour & 1);
    const int cy = 2 * ((a / h) % h) + ((colour >> 1) & 1);
    const int cz = 2 * (a / (h * h)) + ((colour >> 2) & 1);
    return make_int4(R.cell_off + cx + nc * (cy + nc * cz), r, cx | (cy << 10) | (cz << 20),
                     nc | (int)((sweep & 1u) << 16));
}

// cell_coord without the FP64 division in all but rare cases: the FP32
// quotient (s and 1/w rounded to float, one product: relative error < 4u)
// decides floor(s / w) when it is more than 8u q + 2^-40 away from an
// integer, since then the exact quotient and its FP64 rounding lie in the
// same unit interval; otherwise the FP64 quotient decides.  (GB300 issues
// FP64 at 1/64 of FP32: the division was most of this kernel's time.)
// ... and the colloid's FP32 offset from that cell's origin, rounded from
// the FP64 difference, both from one wrapped difference s = x - sigma (FP64
// is most of this kernel's cost).
__device__ __forceinline__ int cell_coord_rel(double x, double sigma, double L, double w, float iw32,
                                              int nc, float &rel)
{
    double s = x - sigma;
    if (s < 0.0) s = s + L;
    const float q = (float)s * iw32;
    const float fl = floorf(q);
    const float m = 8.0f * 0x1p-24f * fmaxf(q, 1.0f) + 0x1p-40f;
    int c;
    if (q - fl > m && (fl + 1.0f) - q > m) c = (int)fl;
    else c = (int)(s / w);
    if (c >= nc) c = nc - 1;
    if (c < 0) c = 0;
    rel = (float)(s - (double)c * w);
    return c;
}

// One thread per colloid of the batch.  The first colloid of each replica
// also writes that replica's schedule.  When the task table is allocated,
// threads also fill it (one entry per phase and CTA), so that the colour
// phases start from their cell without recomputing the schedule.
// full = 0: the bins, populations and schedules only (a configuration
// check), without the phase task table and the exact proposals.
__global__ void k_cells_bin(const __grid_constant__ SimParams P, int full)
{
    // the lens kernel behind this one may start at once (it waits for this
    // kernel's results only where it files them)
    pdl_trigger();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (P.cls_count && g < 32) P.cls_count[g] = 0;
    // persistent colour phases: a new epoch for the cells' readiness counters
    // and a fresh ticket counter for the sweep that follows
    if (g == 0 && P.epoch) {
        atomicAdd(P.epoch, 1u);
        *P.ticket = 0;
    }
    if (full && P.task && g < 8 * P.n_cta) {
        const int phase = g / P.n_cta, a = g - phase * P.n_cta;
        const int r = P.cta_rep[a];
        const Rep &R = P.reps[r];
        int perm[8];
        const uint32_t sw = (uint32_t)(*P.sweep);
        schedule_perm(R.key0, R.key1, sw, perm);
        P.task[g] = phase_task(R, r, perm, phase, a - R.cta_off, sw);
    }
    if (g >= P.n_total) return;
    const int r = P.rep_of[g];
    const Rep &R = P.reps[r];
    const uint32_t sweep = (uint32_t)(*P.sweep);
    double sigma[3];
    schedule_shift(R.key0, R.key1, sweep, R.w, sigma);
    if (g == R.off) {
        Sched s;
        s.sigma[0] = sigma[0];
        s.sigma[1] = sigma[1];
        s.sigma[2] = sigma[2];
        schedule_perm(R.key0, R.key1, sweep, s.perm);
        s.sweep = sweep;
        s.phase_of = 0u;
        for (int ph = 0; ph < 8; ++ph) s.phase_of |= (uint32_t)ph << (4 * s.perm[ph]);
        P.sched[r] = s;
    }
    if (g - R.off >= P.n_live[r]) {   // a slot not in use (Gibbs pair)
        if (P.binpos) P.binpos[g] = -1;
        return;
    }
    const double4 p = P.pos[g];
    const int nc = R.nc;
    const float iw32 = 1.0f / R.w32;
    float4 rl;
    const int cx = cell_coord_rel(p.x, sigma[0], R.L, R.w, iw32, nc, rl.x);
    const int cy = cell_coord_rel(p.y, sigma[1], R.L, R.w, iw32, nc, rl.y);
    const int cz = cell_coord_rel(p.z, sigma[2], R.L, R.w, iw32, nc, rl.z);
    rl.w = __int_as_float(g);
    const int c = R.cell_off + cx + nc * (cy + nc * cz);
    if (HPMC_CHECK_FAILS(P, c >= R.cell_off && c < R.cell_off + nc * nc * nc, 10)) return;
    const int slot = atomicAdd(P.count[sweep & 1u] + c, 1);
    if (slot < P.cap) P.bins[bin_at(P, c, slot)] = rl;
    else atomicCAS(P.err, kErrNone, kErrCellCap);
    if (P.binpos) P.binpos[g] = slot < P.cap ? (int)bin_at(P, c, slot) : -1;
    if (P.bin_q && slot < P.cap) {
        const double4 q = P.quat[g];
        P.bin_q[bin_at(P, c, slot)] = make_float4((float)q.x, (float)q.y, (float)q.z, (float)q.w);
    }
    // (the cell-relative copy is read only by the anisotropic lens kernel)
    if (P.bin_q) P.rel[g] = rl;
    // FP32 sphere form: the exact proposal of this sweep (translation), for
    // the colour phases' commit and exact re-takes
    if (full && P.task && R.shape == 0) {
        const uint4 wm = draw(R.key0, R.key1, sweep, (uint32_t)(g - R.off), kPMove, 0, 0);
        P.prop_pos[g] = make_double4(wrap_box(p.x + R.d_max * s11(wm.x), R.L),
                                     wrap_box(p.y + R.d_max * s11(wm.y), R.L),
                                     wrap_box(p.z + R.d_max * s11(wm.z), R.L), 0.0);
    }
}

// Order every phase's tasks by the population of their cell, fullest first:
// a phase launch lasts as long as its longest sequential chain of moves, so
// the long chains should start first.  One thread per (phase, CTA) entry; positions
// inside a class come from warp-aggregated atomics (any order is valid: the
// cells of one colour are independent).
__global__ void k_task_order(const __grid_constant__ SimParams P)
{
    pdl_trigger();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < 8 * P.n_cta;
    int key = -1;
    int4 tk = make_int4(0, 0, 0, 0);
    if (valid) {
        const int phase = t / P.n_cta;
        tk = P.task[t];
        const int n = P.count[tk.w >> 16][tk.x];
        // every cell is one task: its population of the next sweep starts
        // from zero (nothing reads that buffer before the next binning)
        P.count[(tk.w >> 16) ^ 1][tk.x] = 0;
        // persistent colour phases: one class of non-empty cells, kept close
        // to the table's spatial order (blocks run in roughly increasing
        // order), so that a cell's neighbours of the previous phase sit about
        // one phase's worth of tickets earlier and are done by the time it is
        // taken
        const int cls = P.persistent ? (n > 0 ? 0 : 3)
                                     : (n >= 3 ? 0 : (n == 2 ? 1 : (n == 1 ? 2 : 3)));
        key = phase * 4 + cls;
    }
    const unsigned peers = __match_any_sync(kFull, key);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(P.cls_count + key, __popc(peers));
    base = __shfl_sync(kFull, base, leader);
    if (valid) {
        const int idx = base + __popc(peers & ((1u << lane) - 1u));
        P.task_ord[(size_t)key * P.n_cta + idx] = tk;
    }
}

// --- CSR layout ------------------------------------------------------------

// pos is read with element stride `stride` doubles.
__global__ void k_csr_count(int n, double L, double w, int nc, const double *pos, int stride,
                            uint32_t k0, uint32_t k1, uint32_t sweep, int *cell_of, int *count)
{
    double sigma[3];
    schedule_shift(k0, k1, sweep, w, sigma);
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
__global__ void __launch_bounds__(1024) k_csr_scan(int ncell, int *count, int *cell_start)
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

__global__ void k_csr_scatter(int n, const int *cell_of, int *cursor, int *cell_idx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int slot = atomicAdd(cursor + cell_of[i], 1);
    cell_idx[slot] = i;
}

// Within each cell, ascending colloid index.
__global__ void k_csr_sort(int ncell, const int *cell_start, int *cell_idx)
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

}  // namespace hpmc
