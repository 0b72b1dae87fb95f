// Depletant free-volume measurement (Sec. IV.A): the fraction alpha of the box
// that a depletant can occupy, estimated as the fraction of uniform probe
// points that overlap no colloid.  phi_p = alpha phi_p^r is the paper's
// depletant packing fraction observable.  Probe m draws Philox4x32-10 under
// the caller's key (seed_lo, seed_hi) with counter (sample, m_lo, purpose 8
// << 24 | m_hi, 0) and sits at L u01(w_d); every overlap test is the FP64
// statement of the shape (exactly the tests the sampler uses), against the
// colloids of the 27 cells around the probe.
#pragma once

#include "hpmc_common.cuh"
#include "hpmc_shapes.cuh"

namespace hpmc {

constexpr uint32_t kPProbe = 8;

// One thread per probe (grid-stride).  cell_start/cell_idx: a CSR cell list
// of the replica with n_c cells per side under the grid shift of
// (ck0, ck1, csweep).
__global__ void k_free_volume(Rep R, int nc, uint32_t ck0, uint32_t ck1, uint32_t csweep,
                              const double4 *pos, const double4 *quat, const int *cell_start,
                              const int *cell_idx, uint32_t k0, uint32_t k1, uint32_t sample,
                              unsigned long long n_probe, unsigned long long *n_free)
{
    const double L = R.L, w = L / (double)nc, half_L = 0.5 * L;
    double sig[3];
    schedule_shift(ck0, ck1, csweep, w, sig);
    const int ns = nc == 2 ? 2 : 3;
    unsigned long long free_count = 0;
    for (unsigned long long m = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; m < n_probe;
         m += (unsigned long long)gridDim.x * blockDim.x) {
        const uint4 wd = draw(k0, k1, sample, (uint32_t)m, kPProbe, (uint32_t)(m >> 32), 0);
        const double p[3] = {L * u01(wd.x), L * u01(wd.y), L * u01(wd.z)};
        int ci[3];
        for (int d = 0; d < 3; ++d) ci[d] = cell_coord(p[d], sig[d], L, w, nc);
        bool hit = false;
        for (int t = 0; t < ns * ns * ns && !hit; ++t) {
            const int ox = t % ns, oy = (t / ns) % ns, oz = t / (ns * ns);
            int c3[3];
            const int o[3] = {ox, oy, oz};
            for (int d = 0; d < 3; ++d) c3[d] = nc == 2 ? o[d] : (ci[d] + o[d] - 1 + nc) % nc;
            const int c = c3[0] + nc * (c3[1] + nc * c3[2]);
            for (int s = cell_start[c]; s < cell_start[c + 1] && !hit; ++s) {
                const int j = cell_idx[s];
                const double4 x = pos[j];
                const Vec3 v = v3(min_image(p[0] - x.x, L, half_L), min_image(p[1] - x.y, L, half_L),
                                  min_image(p[2] - x.z, L, half_L));
                if (R.shape == kSphere) hit = norm2(v.x, v.y, v.z) < R.R_dep2;
                else hit = dep_aniso(R, v, quat[j]);
            }
        }
        if (!hit) ++free_count;
    }
    free_count = __reduce_add_sync(kFull, (unsigned)free_count);
    if ((threadIdx.x & 31) == 0 && free_count) atomicAdd(n_free, free_count);
}

}  // namespace hpmc
