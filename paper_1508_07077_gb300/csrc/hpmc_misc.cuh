// Configuration check and layout conversion kernels.
#pragma once

#include "hpmc_common.cuh"

namespace hpmc {

// One thread per colloid of the batch, over the 27 cells of the binned list
// of the current sweep index: sets bit 1 of *flag if a coordinate is outside
// [0, L), bit 0 if two spheres overlap.
__global__ void k_check_spheres(const __grid_constant__ SimParams P, int *flag)
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
            const double r2 = norm2(min_image(pj.x - pi.x, R.L, R.half_L),
                                    min_image(pj.y - pi.y, R.L, R.half_L),
                                    min_image(pj.z - pi.z, R.L, R.half_L));
            if (r2 < R.contact2) atomicOr(flag, 1);
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

// The device generator on n (counter, key) pairs, for known-answer tests:
// variant 0 is philox4x32_10 (key bumped every round), 1 is philox_rk with the
// ten round keys precomputed (the form the depletant loops use).
__global__ void k_philox(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, int variant)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint32_t k0 = key[2 * i], k1 = key[2 * i + 1];
    const uint4 w = variant == 0 ? philox4x32_10(c, k0, k1) : philox_rk(c, round_keys(k0, k1));
    out[4 * i] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
}

}  // namespace hpmc
