// C ABI of the GB300 implicit-depletant HPMC library (see include/hpmc_dep.h).
//
// Host side: parameter validation, the Poisson tables (Sec. III.B step 2), the
// checkerboard geometry of every replica (Sec. III.E), device buffers, and one
// CUDA graph per sweep of the whole batch (cell lists, depletant lens lists,
// 8 colour phases).  All per-step arithmetic runs in the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/hpmc_dep.h"
#include "hpmc_cells.cuh"
#include "hpmc_common.cuh"
#include "hpmc_misc.cuh"
#include "hpmc_sphere_fp32.cuh"
#include "hpmc_sphere_fp64.cuh"
#include "hpmc_aniso_fp64.cuh"
#include "hpmc_aniso_fp32.cuh"
#include "hpmc_probe.cuh"
#include "hpmc_gibbs.cuh"

using namespace hpmc;

namespace {

constexpr double kPi = 3.141592653589793;
constexpr int kTableCap = 32768;

// parameters shared by every replica of a context
struct Params {
    int shape = HPMC_SPHERE;
    double sp[4] = {1.0, 0.0, 0.0, 0.0};
    int nsp = 1;
    int warps = 1;
    int schedule = HPMC_PHASES_LAUNCHES;  // colour phases: 8 launches or one persistent kernel
    double margin = 0.0;
    int v0_mode = HPMC_V0_CIRCUMSPHERE;
    double soft_eps = 0.0;
};

// one replica as the caller described it
struct RepHost {
    int n = 0;
    double L = 0.0;
    double q = 0.0, n_r = 0.0;
    int n_trial = 0;
    double d_max = 0.1, a_max = 0.0, p_translate = 1.0;
    uint32_t replica = 0;
    int nc_req = 0;
};

}  // namespace

struct hpmc_ctx {
    int device = 0;
    uint64_t seed = 0;
    int precision = HPMC_FP64;
    Params prm;
    std::vector<RepHost> reps;
    std::vector<Rep> rdev;        // derived per-replica records (host copy)
    int n_total = 0, n_cells = 0, n_cta = 0, nF_max = 0;
    int cap = kSmallCellCap;      // cell bin capacity of this context

    // device buffers
    double4 *d_pos = nullptr, *d_quat = nullptr;
    float4 *d_rel = nullptr;
    double *d_stage = nullptr;    // n_total x 4 doubles: layout conversion
    int *d_count = nullptr;       // 2 x n_cells populations (double-buffered by sweep parity)
    float4 *d_bins = nullptr;     // n_cells x cap (cell offset, global index)
    int cells_alloc = -1;
    float4 *d_lens = nullptr;     // n_total x lens_cap depletant lens points (FP32 form)
    double4 *d_prop_pos = nullptr, *d_prop_quat = nullptr;
    int lens_cap = 0;
    int4 *d_task = nullptr;       // FP32 sphere form: per-phase cell of every CTA
    int4 *d_task_ord = nullptr;   // and ordered by population class
    int *d_cls_count = nullptr;
    int task_alloc = -1;
    int *d_binpos = nullptr;      // bin slot of every colloid
    int4 *d_hdr_bin = nullptr;    // lens header and displacement per bin slot
    float4 *d_mv_bin = nullptr;
    float4 *d_lens_bin = nullptr; // first lens points per bin slot
    long long aux_alloc = -1;
    float4 *d_bin_q = nullptr;    // FP32 orientation per bin slot (anisotropic FP32 form)
    long long binq_alloc = -1;
    Rep *d_reps = nullptr;
    int *d_rep_of = nullptr;
    int *d_cta_rep = nullptr;
    int cta_alloc = -1;
    Sched *d_sched = nullptr;
    unsigned long long *d_T = nullptr;
    unsigned long long *d_sweep = nullptr, *d_counters = nullptr;
    int *d_err = nullptr, *d_flag = nullptr;
    // persistent colour phases: per-cell readiness counters, epoch, ticket
    uint32_t *d_done = nullptr, *d_epoch = nullptr;
    int *d_ticket = nullptr;
    int done_alloc = -1;
    double wait_s = 1.0;      // bound of every device-side wait
    int withhold = -1;        // test only: a cell whose readiness is never published
    int ticket_chunk = 1;     // persistent colour phases: work items per ticket atomic
    int phase_waves = -1;     // FP32 sphere phases: CTA waves per launch (0: a CTA per cell; -1 automatic)

    bool timing = false;
    std::vector<cudaEvent_t> tev;   // pairs (start, stop)
    std::vector<int> tkind;         // kind of each pair
    std::vector<cudaEvent_t> tpool; // reusable events

    cudaStream_t cap_stream = nullptr;
    // pinned host staging of the small device-to-host reads (sweep index,
    // error word, check flag, counters), so that a call issues all its copies
    // and synchronises once
    unsigned long long *h_pin = nullptr;   // [kPinHead + counters]
    // colloids in use per replica; Gibbs pairs' exchange steps and counters
    int *d_n_live = nullptr;
    unsigned long long *d_gibbs_step = nullptr, *d_gibbs_cnt = nullptr;
    float4 *d_gibbs_pos32 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t check_exec = nullptr;   // the configuration check of an upload
    bool dirty = true;        // parameters changed: re-derive and re-record the graph
    bool state_dirty = true;  // configuration replaced: re-check overlaps only
};

namespace {

// Pinned staging slots (h_pin): sweep index, error word, check flag, sweep
// index to upload, then the counters.
constexpr int kPinSweep = 0, kPinErr = 1, kPinFlag = 2, kPinUp = 3, kPinHead = 4;

size_t counter_words(const hpmc_ctx *c)
{
    return (size_t)c->reps.size() * kRepSlots * kNumCounters;
}

int cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return HPMC_OK;
    if (getenv("HPMC_VERBOSE")) fprintf(stderr, "hpmc: %s: %s\n", what, cudaGetErrorString(e));
    return HPMC_ERR_CUDA;
}

#define CK(call)                                                \
    do {                                                        \
        int _rc = cuda_fail((call), #call);                     \
        if (_rc != HPMC_OK) return _rc;                         \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Circumsphere radius of the shape about its reference point.
double circum_radius(const Params &p)
{
    switch (p.shape) {
    case HPMC_SPHERE: return 0.5 * p.sp[0];
    case HPMC_HEMISPHERE: return 0.5 * p.sp[0];
    case HPMC_SPHEROID: return p.sp[0] > p.sp[1] ? p.sp[0] : p.sp[1];
    default: return -1.0;
    }
}

// Poisson CDF table: p_0 = exp(-lambda), p_k = p_{k-1} lambda / k, cumulative
// sum; stop after the first k > lambda with p_k < 2^-64.
int build_table(double lambda, std::vector<double> &F)
{
    F.clear();
    if (!(lambda >= 0.0) || lambda > 700.0) return HPMC_ERR_ARG;
    double p = std::exp(-lambda);
    double cdf = p;
    F.push_back(cdf);
    for (int k = 1;; ++k) {
        p = (p * lambda) / (double)k;
        cdf = cdf + p;
        if ((int)F.size() >= kTableCap) return HPMC_ERR_CAP;
        F.push_back(cdf);
        if ((double)k > lambda && p < 5.421010862427522e-20) break;
    }
    return HPMC_OK;
}

// Derive one replica's device record.  Returns HPMC_OK or an error.
int derive_rep(const hpmc_ctx *c, const RepHost &h, Rep &R, std::vector<double> &F)
{
    const Params &p = c->prm;
    std::memset(&R, 0, sizeof R);
    const double R_circ = circum_radius(p);
    if (!(R_circ > 0.0)) return HPMC_ERR_ARG;
    if (!(h.q >= 0.0) || !(h.n_r >= 0.0) || h.n_trial < 0 || h.n_trial > 100000) return HPMC_ERR_ARG;
    const double R_s = R_circ + 0.5 * h.q;
    // |V_0|: the circumsphere, or the cube of side 2 R_s around it
    const double a_cube = 2.0 * R_s;
    const double v0 = p.v0_mode == HPMC_V0_CUBE ? (a_cube * a_cube) * a_cube
                                                : ((4.0 / 3.0) * kPi) * ((R_s * R_s) * R_s);
    const double lambda = h.n_r > 0.0 ? h.n_r * v0 : 0.0;
    const double w_min = 2.0 * R_circ + h.q;
    int nc = h.nc_req;
    if (nc == 0) {
        nc = (int)(h.L / w_min);
        if (nc & 1) nc -= 1;
    }
    if (nc < 2 || (nc & 1)) return HPMC_ERR_ARG;
    if (nc > 1024) return HPMC_ERR_CAP;
    const double w = h.L / (double)nc;
    if (w < w_min) return HPMC_ERR_ARG;
    if (!(h.d_max >= 0.0) || h.d_max >= w) return HPMC_ERR_ARG;
    // a cell bin holds at most (w + 2 R_circ)^3 * pack / v colloids of volume v:
    // pack = 0.7405 (densest sphere packing) for spheres, 0.78 for the
    // anisotropic shapes (above the densest known ellipsoid packing, 0.7707,
    // and hemispheres, which pair into spheres)
    double v_shape = (kPi / 6.0) * p.sp[0] * p.sp[0] * p.sp[0];
    if (p.shape == HPMC_HEMISPHERE) v_shape = 0.5 * v_shape;
    if (p.shape == HPMC_SPHEROID) v_shape = (4.0 / 3.0 * kPi) * p.sp[0] * p.sp[0] * p.sp[1];
    const double pack = p.shape == HPMC_SPHERE ? 0.7405 : 0.78;
    const double ext = w + 2.0 * R_circ;
    const double cell_bound = ext * ext * ext * pack / v_shape;
    if (cell_bound >= (double)kMaxCellCap) return HPMC_ERR_CAP;
    R.pad_cell_bound = cell_bound;
    // Neighbours that can meet a depletant: a depletant of the new circumsphere
    // lies within R_s of the new reference point and meets colloid j only if
    // |x_j - y| < R_circ + q/2 = R_s, so |d_j| < 2 R_s; the forward CB trials
    // lie in the OLD circumsphere, centred |o| <= sqrt(3) d_max away, which
    // widens the range by that much.  0.01 covers the FP32 rounding of |d_j|.
    const double cut = 2.0 * R_s + (h.n_trial > 0 ? std::sqrt(3.0) * h.d_max : 0.0) + 0.01;
    // in the FP32 form that neighbourhood must fit the phase kernel's list:
    // 128 for the anisotropic shapes (kMaxNbAniso); for spheres 64, or 128 in
    // the widest cells (max_nb), checked in prepare() once the cell capacity
    // is known (the FP64 forms keep every candidate of the 27 cells)
    const double nb_ext = cut + R_circ;
    R.pad_nb_bound = nb_ext * nb_ext * nb_ext * (4.0 / 3.0 * kPi) * pack / v_shape;
    if (c->precision == HPMC_FP32_RECHECK && p.shape != HPMC_SPHERE && R.pad_nb_bound >= 128.0)
        return HPMC_ERR_CAP;
    F.clear();
    if (lambda > 0.0) {
        int rc = build_table(lambda, F);
        if (rc != HPMC_OK) return rc;
        // lens points pack the attempt index t < 64 (N_p + 1) into 16 bits
        if (c->precision == HPMC_FP32_RECHECK && F.size() > 1023) return HPMC_ERR_CAP;
    }
    // shell-restricted V_0 (Sec. III.C, closing remark; spheres only): level k
    // samples R_in <= |e| < R_s with thickness k dd + 1e-9 R_s, dd =
    // sqrt(3) d_max / 32, which exceeds the length of every move of that
    // level.  One Poisson table per level, each padded to the longest with
    // entries no 53-bit uniform reaches (2.0), so that level k's table is the
    // block of nF entries at (k - 1) nF.
    int shell_stride = 0;
    if (p.v0_mode == HPMC_V0_SHELL) {
        if (p.shape != HPMC_SPHERE) return HPMC_ERR_ARG;
        R.dd = (std::sqrt(3.0) * h.d_max) / 32.0;
        std::vector<double> Fl[kShellLevels];
        for (int k = 1; k <= kShellLevels; ++k) {
            const double t = (double)k * R.dd + 1e-9 * R_s;
            double rin = R_s - t;
            if (rin < 0.0) rin = 0.0;
            R.sh_rin[k - 1] = rin;
            R.sh_h[k - 1] = R_s - rin;
            R.sh_rin32[k - 1] = (float)rin;
            R.sh_h32[k - 1] = (float)R.sh_h[k - 1];
            if (!(lambda > 0.0)) continue;
            const double vs = ((4.0 / 3.0) * kPi) * (((R_s * R_s) * R_s) - ((rin * rin) * rin));
            int rc = build_table(h.n_r * vs, Fl[k - 1]);
            if (rc != HPMC_OK) return rc;
            if ((int)Fl[k - 1].size() > shell_stride) shell_stride = (int)Fl[k - 1].size();
        }
        if (lambda > 0.0) {
            F.clear();
            for (int k = 0; k < kShellLevels; ++k) {
                F.insert(F.end(), Fl[k].begin(), Fl[k].end());
                F.resize((size_t)(k + 1) * (size_t)shell_stride, 2.0);
            }
            R.v0_shell = 1;
        }
    }
    R.n = h.n;
    R.nc = nc;
    R.half_nc = nc / 2;
    R.n_stencil = nc == 2 ? 2 : 3;
    R.nF = R.v0_shell ? shell_stride : (int)F.size();
    // soft colloid-depletant interaction: spheres, no CB, a V_0 that holds
    // the new circumsphere
    if (p.soft_eps > 0.0 && (p.shape != HPMC_SPHERE || h.n_trial != 0 || p.v0_mode == HPMC_V0_SHELL))
        return HPMC_ERR_ARG;
    R.soft_eps = p.soft_eps;
    R.soft32 = (p.soft_eps > 0.0 && c->precision == HPMC_FP32_RECHECK) ? 1 : 0;
    if (R.soft32) {
        // FP32 bands (u = 2^-24).  A point's FP32 coordinates err by <= 6u R_s
        // each and the displacement's FP32 image by u |o|; a difference adds
        // u (R_s + |o|).  Vectors therefore err by Ev <= sqrt(3) (6u R_s +
        // 2u (R_s + |o|)), and a squared length r^2 <= Rm^2 (Rm = R_s + |o|)
        // by 2 Rm Ev + Ev^2 + 3u Rm^2; r_new >= r_old is certain when
        // r2n32 - r2o32 exceeds twice that plus the subtraction's u Rm^2.
        // A length errs by dr <= Ev + 4u Rm (the norm is 1-Lipschitz), so
        // t = 1 - r / s by dt <= dr / s + 4u and u(r) = eps t^(5/2) by
        // du <= eps (5/2 dt + 6u); expf errs by <= 2 ulp (CUDA's bound) and
        // e^-u is 1-Lipschitz for u >= 0, so each e^-u by <= 2^-22 + du, the
        // difference of two by twice that plus u, and u01(w) in FP32 by
        // u + 2^-33: u01 >= e_old - e_new is certain beyond their sum.  The
        // FP64 statements' own rounding is below 1e-12 eps.  A margin set by
        // the caller widens both bands (1 sends every point to FP64).
        const double u = 0x1p-24;
        const double om = std::sqrt(3.0) * h.d_max, Rm = R_s + om;
        // (the displacement's FP32 image is bit-built: <= 6u d_max more)
        const double Ev = std::sqrt(3.0) * (6.0 * u * R_s + 7.0 * u * h.d_max + 2.0 * u * Rm);
        const double r2err = 2.0 * Rm * Ev + Ev * Ev + 3.0 * u * Rm * Rm;
        const double dt = (Ev + 4.0 * u * Rm) / R_s + 4.0 * u;
        const double du = p.soft_eps * (2.5 * dt + 6.0 * u) + 1e-12 * p.soft_eps;
        const double eE = 0x1p-22 + du + 1e-12;
        const double extra = p.margin > 0.0 ? p.margin : 0.0;
        R.soft_eps32 = (float)p.soft_eps;
        R.soft_inv_s32 = (float)(1.0 / R_s);
        R.soft_r2band = (float)(2.0 * (2.0 * r2err + u * Rm * Rm) + extra);
        R.soft_vband = (float)(2.0 * (2.0 * eE + u + u + 0x1p-33) + extra);
        // the colour phases' test u01 < e^-U (e^-u_old - e^-u_new): a
        // neighbour's offset from the point errs by <= sqrt(3) (E + 6u R_s)
        // (E: the cell-relative budget of the certified form), so its energy
        // by du_nb = eps (2.5 dt_nb + 6u); U (n terms in range) by n du_nb plus
        // n u U for the sum, e^-U by 2^-22 plus that; the product with the
        // difference d (its bound above) adds u.  The band is twice the sum
        // (n counted per point), plus the caller's margin.
        const double Enb = std::sqrt(3.0) * (40.0 * u * (w > 1.0 ? w : 1.0) + 6.0 * u * R_s);
        const double dt_nb = (Enb + 4.0 * u * 2.0 * R_s) / R_s + 4.0 * u;
        R.soft_du_nb = (float)(2.0 * (p.soft_eps * (2.5 * dt_nb + 6.0 * u) + 1e-12 * p.soft_eps));
        R.soft_bband = (float)(2.0 * (2.0 * eE + 0x1p-22 + 3.0 * u + 0x1p-33) + extra);
    }
    R.v0_cube = p.v0_mode == HPMC_V0_CUBE ? 1 : 0;
    R.has_dep = lambda > 0.0 ? 1 : 0;
    R.n_trial = h.n_trial;
    R.key0 = (uint32_t)c->seed;
    R.key1 = (uint32_t)(c->seed >> 32) ^ h.replica;
    R.L = h.L;
    R.half_L = 0.5 * h.L;
    R.w = w;
    R.R_s = R_s;
    R.R_s2 = R_s * R_s;
    R.R_s4 = R.R_s2 * R.R_s2;
    R.R_s4_32 = (float)R.R_s4;
    // a margin set by the caller also widens the shell test's band (a margin
    // >= 1 sends every shell decision to FP64)
    R.shell_band = (float)p.margin;
    const double Rd = 0.5 * p.sp[0] + 0.5 * h.q;
    R.R_dep2 = Rd * Rd;
    R.contact2 = p.sp[0] * p.sp[0];
    R.nb_cut2 = cut * cut;
    R.d_max = h.d_max;
    R.shape = p.shape;
    R.R_circ = R_circ;
    R.r_dep = 0.5 * h.q;
    R.sh_R = 0.5 * p.sp[0];
    R.sh_a = p.sp[0];
    R.sh_c = p.shape == HPMC_SPHEROID ? p.sp[1] : p.sp[0];
    R.rot_on = (p.shape != HPMC_SPHERE && h.a_max > 0.0) ? 1 : 0;
    // rotation by 2 atan(alpha |v|) <= a_max, |v| < 1
    R.alpha = h.a_max > 0.0 ? std::tan(0.5 * h.a_max) : 0.0;
    R.p_translate = h.p_translate;
    // FP32 form: thresholds in float and the certified margin.  Every vector a
    // test forms is a difference of cell-relative coordinates; each component
    // carries at most E = 40 u max(w, 1) of FP32 error (rounding of the
    // cell-relative copies, including one FP32 step for a colloid already moved
    // this sweep, of the displacement, of the bit-built depletant coordinate
    // (<= 6 u R) and of the differences).  For |v| near a threshold radius R the
    // squared length then errs by at most 2 sqrt(3) R E + 3 E^2 + 3 u R^2, plus
    // u R^2 for rounding the threshold itself; the margin is twice that, and at
    // least 1e-5.
    const double u = 0x1p-24;
    const double Wc = w > 1.0 ? w : 1.0;
    // (a shell point, built from its direction and radius, errs by <= 16 u R_s
    // per component instead of 6 u R_s)
    const double E = 40.0 * u * Wc + (R.v0_shell ? 12.0 * u * R_s : 0.0);
    const double Rmax = std::sqrt(std::fmax(R.R_s2, R.contact2));
    const double bound = 2.0 * std::sqrt(3.0) * Rmax * E + 3.0 * E * E + 4.0 * u * Rmax * Rmax + 1e-12;
    const double m_r2 = std::fmax(1e-5, 2.0 * bound);
    if (p.margin > 0.0 && p.margin < m_r2) return HPMC_ERR_ARG;
    R.m_r2 = (float)(p.margin > 0.0 ? p.margin : m_r2);
    R.m_cell = (float)(1e-5 * Wc);
    {
        // differences of FP32 images of absolute positions in [0, L): each
        // component errs by <= 4 u max(L, 1) (two roundings of a coordinate,
        // the difference, the periodic shift)
        const double EL = 4.0 * u * std::fmax(h.L, 1.0);
        const double bl = 2.0 * std::sqrt(3.0) * Rmax * EL + 3.0 * EL * EL + 4.0 * u * Rmax * Rmax + 1e-12;
        R.m_box32 = (float)std::fmax(std::fmax(1e-5, 2.0 * bl), p.margin);
    }
    R.w32 = (float)w;
    R.L32 = (float)h.L;
    R.half_L32 = (float)(0.5 * h.L);
    R.R_s32 = (float)R_s;
    R.T_s32 = (float)R.R_s2;
    R.T_dep32 = (float)R.R_dep2;
    R.T_contact32 = (float)R.contact2;
    R.nb_cut2_32 = (float)R.nb_cut2;
    R.d_max32 = (float)h.d_max;
    // anisotropic FP32 form.  A body-frame point errs by at most
    // sqrt(3) E (its lab-frame offset) + 64 u |v| (an FP32 frame built from
    // the FP32 image of the FP64 quaternion rotates v within ~33 u |v|), and
    // the FP32 distance evaluation adds < 32 u max(1, R_circ); m_d is twice
    // that.  A pair certificate involves two bodies: offsets 2 sqrt(3) E, the
    // support value or witness depth 256 u max(1, R_circ), evaluation 64 u.
    R.R_circ32 = (float)R_circ;
    R.r_dep32 = (float)R.r_dep;
    R.sh_R32 = (float)R.sh_R;
    R.sh_a32 = (float)R.sh_a;
    R.sh_c32 = (float)R.sh_c;
    {
        const double Rc = std::fmax(1.0, R_circ);
        const double md = 2.0 * (std::sqrt(3.0) * E + 64.0 * u * (R_circ + R.r_dep + 1e-3) + 32.0 * u * Rc);
        const double mp = 2.0 * (2.0 * std::sqrt(3.0) * E + 256.0 * u * Rc + 64.0 * u);
        R.m_d = (float)std::fmax(1e-5, md);
        R.m_pair = (float)std::fmax(1e-5, mp);
        // the FP32 shortcuts assume the depletant radius is well above the margin
        if (p.shape != HPMC_SPHERE && c->precision == HPMC_FP32_RECHECK && h.n_r > 0.0 &&
            !(R.r_dep > 4.0 * R.m_d))
            return HPMC_ERR_ARG;
        // a larger margin set by the caller widens every FP32 test's band
        if (p.margin > 0.0) {
            R.m_d = (float)std::fmax((double)R.m_d, p.margin);
            R.m_pair = (float)std::fmax((double)R.m_pair, p.margin);
        }
        // spheroid quick tests.  The outer spheroid (A', A', C') contains
        // E + ball(r) iff sqrt(a^2 x + c^2 z) + r <= sqrt(A'^2 x + C'^2 z) for
        // x + z = 1 (support functions); with A' = a + r (oblate) this holds iff
        // C'^2 >= c^2 + r^2 + K, K = max(2 r c, r (a^2 + c^2) / a) (the squared
        // inequality is linear in x, so its end points decide), and symmetrically
        // for a prolate spheroid.
        const double a = R.sh_a, cc = R.sh_c, rr = R.r_dep, md2 = (double)R.m_d;
        double Ao = a + rr, Co = cc + rr;
        if (a >= cc) Co = std::sqrt(cc * cc + rr * rr + std::fmax(2.0 * rr * cc, rr * (a * a + cc * cc) / a));
        else Ao = std::sqrt(a * a + rr * rr + std::fmax(2.0 * rr * a, rr * (a * a + cc * cc) / cc));
        const double kin = 1.0 - md2 / std::fmin(a + rr, cc + rr);
        const double kout = 1.0 + md2 / std::fmin(Ao, Co);
        R.sp_iA2 = (float)(1.0 / (a * a));
        R.sp_iC2 = (float)(1.0 / (cc * cc));
        R.sp_inA = (float)(1.0 / ((a + rr) * (a + rr)));
        R.sp_inC = (float)(1.0 / ((cc + rr) * (cc + rr)));
        R.sp_outA = (float)(1.0 / (Ao * Ao));
        R.sp_outC = (float)(1.0 / (Co * Co));
        R.sp_kin2 = kin > 0.0 ? (float)(kin * kin) : -1.0f;
        R.sp_kout2 = (float)(kout * kout);
    }
    return HPMC_OK;
}

// The persistent colour-phase kernel runs the FP32 sphere form's sweeps with
// one-warp CTAs (warps per colloid = 1) when the schedule selects it.
bool use_persistent(const hpmc_ctx *c)
{
    return c->prm.schedule == HPMC_PHASES_PERSISTENT && c->precision == HPMC_FP32_RECHECK &&
           c->prm.shape == HPMC_SPHERE && c->prm.warps == 1 && c->d_done != nullptr;
}

SimParams make_params(hpmc_ctx *c)
{
    SimParams P;
    std::memset(&P, 0, sizeof P);
    P.n_rep = (int)c->reps.size();
    P.n_total = c->n_total;
    P.cap = c->cap;
    P.lens_cap = c->lens_cap;
    P.reps = c->d_reps;
    P.rep_of = c->d_rep_of;
    P.cta_rep = c->d_cta_rep;
    P.pos = c->d_pos;
    P.quat = c->d_quat;
    P.rel = c->d_rel;
    P.count[0] = c->d_count;
    P.count[1] = c->d_count ? c->d_count + c->n_cells : nullptr;
    P.bins = c->d_bins;
    P.T = c->d_T;
    P.lens = c->d_lens;
    P.prop_pos = c->d_prop_pos;
    P.prop_quat = c->d_prop_quat;
    P.n_cta = c->n_cta;
    P.task = c->d_task;
    P.n_live = c->d_n_live;
    P.gibbs_step = c->d_gibbs_step;
    P.gibbs_cnt = c->d_gibbs_cnt;
    P.pos32 = c->d_gibbs_pos32;
    P.task_ord = c->d_task_ord;
    P.cls_count = c->d_cls_count;
    P.binpos = c->d_binpos;
    P.hdr_bin = c->d_hdr_bin;
    P.mv_bin = c->d_mv_bin;
    P.lens_bin = c->d_lens_bin;
    P.bin_q = c->prm.shape == HPMC_SPHERE ? nullptr : c->d_bin_q;
    P.sched = c->d_sched;
    P.sweep = c->d_sweep;
    P.counters = c->d_counters;
    P.err = c->d_err;
    P.n_cells = c->n_cells;
    P.done = c->d_done;
    P.epoch = c->d_epoch;
    P.ticket = c->d_ticket;
    P.wait_ns = (unsigned long long)(c->wait_s * 1e9);
    P.ticket_chunk = c->ticket_chunk;
    P.persistent = use_persistent(c) ? 1 : 0;
    P.withhold = c->withhold;
    return P;
}



// Enqueue the binned cell lists (and schedules) of the sweep whose index is
// in *d_sweep.  Their count buffer was zeroed by the previous sweep's phase
// kernels (or by check_config).
// tasks = false: bins for a configuration check only (no phase task table,
// no proposals)
int enqueue_cells(hpmc_ctx *c, cudaStream_t s, bool tasks = true)
{
    SimParams P = make_params(c);
    const int threads = (c->d_task && tasks) ? std::max(c->n_total, 8 * c->n_cta) : c->n_total;
    k_cells_bin<<<(threads + 255) / 256, 256, 0, s>>>(P, tasks ? 1 : 0);
    if (c->d_task && tasks) k_task_order<<<(8 * c->n_cta + 255) / 256, 256, 0, s>>>(P);
    CK(cudaGetLastError());
    return HPMC_OK;
}

// Launch with programmatic stream serialization (the kernel may start while
// its predecessor in the stream drains; it orders itself with pdl_wait()).
template <typename K>
void launch_pdl(K kernel, int grid, int block, size_t dyn, cudaStream_t s, const SimParams &P,
                int phase)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, P, phase);
}

template <typename K>
void launch_pdl1(K kernel, int grid, int block, cudaStream_t s, const SimParams &P)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, P);
}

// CTAs of a kernel resident on the whole GPU at once.
template <typename K>
int resident_ctas(K kernel, int threads, size_t dyn)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dyn);
    return sms * std::max(1, per_sm);
}

// Waves of the looping FP32 sphere colour phases (0: a CTA per cell).  Set:
// c->phase_waves; automatic (-1), for hard interactions without CB: two
// waves when a phase has more cells than one wave of the one-CTA-per-cell
// kernel holds (CTA launches are then a large part of a phase), else none.
// (With CB or the soft interaction a cell's work is longer and the looping
// grid measured slower: none.)
template <typename K>
int phase_waves(const hpmc_ctx *c, K single, int threads, size_t dyn, bool long_cells)
{
    if (c->phase_waves >= 0) return c->phase_waves;
    if (long_cells) return 0;
    return c->n_cta > resident_ctas(single, threads, dyn) ? 2 : 0;
}

// One FP32 sphere colour phase of the one-warp kernel: a CTA per cell, or
// waves of looping CTAs (identical results: any grid size is correct).
template <typename K1, typename KL>
void launch_phase_sphere32(const hpmc_ctx *c, K1 single, KL loop, size_t dyn, cudaStream_t s,
                           const SimParams &P, int phase, bool long_cells)
{
    const int w = phase_waves(c, single, 32, dyn, long_cells);
    if (w <= 0) {
        launch_pdl(single, c->n_cta, 32, dyn, s, P, phase);
        return;
    }
    const long long g = (long long)w * resident_ctas(loop, 32, dyn);
    launch_pdl(loop, (int)std::max(1LL, std::min((long long)c->n_cta, g)), 32, dyn, s, P, phase);
}

template <int CAP>
void launch_phase_cap(hpmc_ctx *c, const SimParams &P, int phase, cudaStream_t s)
{
    const int threads = 32 * c->prm.warps;
    bool cb = false;
    for (const RepHost &h : c->reps) cb = cb || h.n_trial > 0;
    // the CB pass's per-thread factor and index slots; none without CB (the
    // one-warp CTA of the 16-slot bins then fits 32 per SM)
    const size_t dyn = cb ? (size_t)threads * (sizeof(double) + sizeof(int)) : 0;
    if (c->precision == HPMC_FP32_RECHECK && c->prm.shape != HPMC_SPHERE) {
        // the anisotropic shapes' packing bound always selects a capacity >= 32
        if constexpr (CAP >= kSmallCellCap) {
            const bool warp = threads == 32;
            if (cb) {
                if (warp) launch_pdl(k_phase_aniso_fp32<true, true, CAP>, c->n_cta, threads, dyn, s, P, phase);
                else launch_pdl(k_phase_aniso_fp32<true, false, CAP>, c->n_cta, threads, dyn, s, P, phase);
            } else {
                if (warp) launch_pdl(k_phase_aniso_fp32<false, true, CAP>, c->n_cta, threads, dyn, s, P, phase);
                else launch_pdl(k_phase_aniso_fp32<false, false, CAP>, c->n_cta, threads, dyn, s, P, phase);
            }
        }
    } else if (c->precision == HPMC_FP32_RECHECK) {
        const bool warp = threads == 32;
        if (cb) {
            if (warp) launch_phase_sphere32(c, k_phase_sphere_fp32<true, true, CAP>,
                                            k_phase_sphere_fp32<true, true, CAP, false, true>, dyn, s, P,
                                            phase, true);
            else launch_pdl(k_phase_sphere_fp32<true, false, CAP>, c->n_cta, threads, dyn, s, P, phase);
        } else if (c->prm.soft_eps > 0.0) {
            if (warp) launch_phase_sphere32(c, k_phase_sphere_fp32<false, true, CAP, true>,
                                            k_phase_sphere_fp32<false, true, CAP, true, true>, dyn, s, P,
                                            phase, true);
            else launch_pdl(k_phase_sphere_fp32<false, false, CAP, true>, c->n_cta, threads, dyn, s, P, phase);
        } else {
            if (warp) launch_phase_sphere32(c, k_phase_sphere_fp32<false, true, CAP>,
                                            k_phase_sphere_fp32<false, true, CAP, false, true>, dyn, s, P,
                                            phase, false);
            else launch_pdl(k_phase_sphere_fp32<false, false, CAP>, c->n_cta, threads, dyn, s, P, phase);
        }
    } else if (c->prm.shape == HPMC_SPHERE) {
        k_phase_sphere_fp64<CAP><<<c->n_cta, threads, 0, s>>>(P, phase);
    } else {
        if constexpr (CAP >= kSmallCellCap)
            k_phase_aniso_fp64<CAP><<<c->n_cta, threads, 0, s>>>(P, phase);
    }
}

// One launch for all eight colour phases: as many one-warp CTAs as fit on
// the GPU at once (any count is correct; more would only wait for a slot).
template <typename K>
void launch_persistent(K kernel, size_t dyn, cudaStream_t s, const SimParams &P)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32, dyn);
    const int grid = std::max(1, sms * std::max(1, per_sm));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(32u);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, P);
}

template <int CAP>
void launch_sweep_cap(hpmc_ctx *c, const SimParams &P, cudaStream_t s)
{
    bool cb = false;
    for (const RepHost &h : c->reps) cb = cb || h.n_trial > 0;
    const size_t dyn = cb ? (size_t)32 * (sizeof(double) + sizeof(int)) : 0;
    if (cb) launch_persistent(k_sweep_sphere_fp32<true, CAP>, dyn, s, P);
    else if (c->prm.soft_eps > 0.0) launch_persistent(k_sweep_sphere_fp32<false, CAP, true>, dyn, s, P);
    else launch_persistent(k_sweep_sphere_fp32<false, CAP>, dyn, s, P);
}

void launch_sweep_phases(hpmc_ctx *c, const SimParams &P, cudaStream_t s)
{
    if (c->cap == kTinyCellCap) launch_sweep_cap<kTinyCellCap>(c, P, s);
    else if (c->cap == kSmallCellCap) launch_sweep_cap<kSmallCellCap>(c, P, s);
    else launch_sweep_cap<kMaxCellCap>(c, P, s);
}

void launch_phase(hpmc_ctx *c, const SimParams &P, int phase, cudaStream_t s)
{
    if (c->cap == kTinyCellCap) launch_phase_cap<kTinyCellCap>(c, P, phase, s);
    else if (c->cap == kSmallCellCap) launch_phase_cap<kSmallCellCap>(c, P, phase, s);
    else launch_phase_cap<kMaxCellCap>(c, P, phase, s);
}

void launch_lens(hpmc_ctx *c, const SimParams &P, cudaStream_t s)
{
    if (c->precision != HPMC_FP32_RECHECK) return;
    if (c->prm.shape == HPMC_SPHERE) {
        if (c->prm.v0_mode == HPMC_V0_SHELL)
            launch_pdl1(k_lens_shell_fp32, (c->n_total + 127) / 128, 128, s, P);
        else if (c->prm.soft_eps > 0.0 && c->prm.v0_mode == HPMC_V0_CUBE)
            launch_pdl1(k_lens_sphere_fp32<2, true>, (c->n_total + 3) / 4, 128, s, P);
        else if (c->prm.soft_eps > 0.0)
            launch_pdl1(k_lens_sphere_fp32<0, true>, (c->n_total + 3) / 4, 128, s, P);
        else if (c->prm.v0_mode == HPMC_V0_CUBE)
            launch_pdl1(k_lens_sphere_fp32<2>, (c->n_total + 3) / 4, 128, s, P);
        else
            launch_pdl1(k_lens_sphere_fp32<0>, (c->n_total + 3) / 4, 128, s, P);
    } else {
        k_propose_aniso<<<(c->n_total + 127) / 128, 128, 0, s>>>(P);
        k_lens_aniso_fp32<<<(c->n_total + 3) / 4, 128, 0, s>>>(P);
    }
}

// One sweep of every replica: binned cell lists, depletant lens lists (FP32
// form), then the 8 colour phases (phase 7 advances the sweep counter).
int enqueue_sweep(hpmc_ctx *c, cudaStream_t s)
{
    int rc = enqueue_cells(c, s);
    if (rc != HPMC_OK) return rc;
    SimParams P = make_params(c);
    launch_lens(c, P, s);
    if (use_persistent(c)) launch_sweep_phases(c, P, s);
    else
        for (int phase = 0; phase < 8; ++phase) launch_phase(c, P, phase, s);
    CK(cudaGetLastError());
    return HPMC_OK;
}

cudaEvent_t pool_event(hpmc_ctx *c)
{
    if (!c->tpool.empty()) {
        cudaEvent_t e = c->tpool.back();
        c->tpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// One sweep launched kernel by kernel with events around the cell lists, the
// lens kernel and each colour-phase kernel.
int enqueue_sweep_timed(hpmc_ctx *c, cudaStream_t s)
{
    cudaEvent_t a = pool_event(c), b = pool_event(c);
    CK(cudaEventRecord(a, s));
    nvtxRangePushA("cell lists");
    int rc = enqueue_cells(c, s);
    nvtxRangePop();
    if (rc != HPMC_OK) return rc;
    CK(cudaEventRecord(b, s));
    c->tev.push_back(a);
    c->tev.push_back(b);
    c->tkind.push_back(0);
    SimParams P = make_params(c);
    if (c->precision == HPMC_FP32_RECHECK) {
        cudaEvent_t x = pool_event(c), y = pool_event(c);
        CK(cudaEventRecord(x, s));
        nvtxRangePushA("depletant lens lists");
        launch_lens(c, P, s);
        nvtxRangePop();
        CK(cudaEventRecord(y, s));
        c->tev.push_back(x);
        c->tev.push_back(y);
        c->tkind.push_back(2);
    }
    if (use_persistent(c)) {
        cudaEvent_t x = pool_event(c), y = pool_event(c);
        CK(cudaEventRecord(x, s));
        nvtxRangePushA("colour phases 0-7 (persistent)");
        launch_sweep_phases(c, P, s);
        nvtxRangePop();
        CK(cudaEventRecord(y, s));
        c->tev.push_back(x);
        c->tev.push_back(y);
        c->tkind.push_back(1);
    } else {
        for (int phase = 0; phase < 8; ++phase) {
            static const char *names[8] = {"colour phase 0", "colour phase 1", "colour phase 2",
                                           "colour phase 3", "colour phase 4", "colour phase 5",
                                           "colour phase 6", "colour phase 7"};
            cudaEvent_t x = pool_event(c), y = pool_event(c);
            CK(cudaEventRecord(x, s));
            nvtxRangePushA(names[phase]);
            launch_phase(c, P, phase, s);
            nvtxRangePop();
            CK(cudaEventRecord(y, s));
            c->tev.push_back(x);
            c->tev.push_back(y);
            c->tkind.push_back(1);
        }
    }
    CK(cudaGetLastError());
    return HPMC_OK;
}

void free_graph(hpmc_ctx *c)
{
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->check_exec) cudaGraphExecDestroy(c->check_exec);
    c->check_exec = nullptr;
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
}

// Configuration check on cell lists of the current sweep index: positions in
// [0, L) and no overlapping colloids, in every replica.  enqueue_check puts
// the device work on stream s (bins of the current sweep, the check kernel,
// the flags to pinned host memory, zeroed populations); check_result reads
// the flags once s has been synchronised.
int enqueue_check(hpmc_ctx *c, cudaStream_t s)
{
    const size_t cbytes = sizeof(int) * 2 * (size_t)c->n_cells;
    CK(cudaMemsetAsync(c->d_count, 0, cbytes, s));
    CK(cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int), s));
    int rc = enqueue_cells(c, s, false);   // (the phase task order is not needed)
    if (rc != HPMC_OK) return rc;
    CK(cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
    SimParams P = make_params(c);
    if (c->prm.shape == HPMC_SPHERE && c->precision == HPMC_FP32_RECHECK)
        k_check_spheres32<<<(unsigned)(((size_t)c->n_total * kCheckStencil + 255) / 256), 256, 0, s>>>(P, c->d_flag);
    else if (c->prm.shape == HPMC_SPHERE)
        k_check_spheres<<<(c->n_total + 255) / 256, 256, 0, s>>>(P, c->d_flag);
    else
        k_check_aniso<<<(c->n_total + 127) / 128, 128, 0, s>>>(P, c->d_flag);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->h_pin + kPinFlag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->h_pin + kPinErr, c->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    // the sweeps start from zeroed populations
    CK(cudaMemsetAsync(c->d_count, 0, cbytes, s));
    return HPMC_OK;
}

int check_result(hpmc_ctx *c)
{
    const int flag = *reinterpret_cast<const int *>(c->h_pin + kPinFlag);
    const int err = *reinterpret_cast<const int *>(c->h_pin + kPinErr);
    if (flag & 2) return HPMC_ERR_ARG;
    if (err == kErrCellCap) return HPMC_ERR_CAP;
    if (flag & 1) return HPMC_ERR_OVERLAP;
    c->state_dirty = false;
    return HPMC_OK;
}

// Synchronous check: on the context's own stream after its pending work, or
// (own = false) on stream s, which the caller has ordered; the recorded
// check graph when one exists.
int check_config(hpmc_ctx *c, cudaStream_t s = nullptr, bool own = true)
{
    if (own) {
        s = c->cap_stream;
        CK(cudaStreamSynchronize(s));
    }
    if (c->check_exec) {
        CK(cudaGraphLaunch(c->check_exec, s));
    } else {
        int rc = enqueue_check(c, s);
        if (rc != HPMC_OK) return rc;
    }
    CK(cudaStreamSynchronize(s));
    return check_result(c);
}

// Validate parameters, derive every replica, upload tables and maps, check
// the configuration, record the sweep graph.
int prepare(hpmc_ctx *c)
{
    const Params &p = c->prm;
    const int n_rep = (int)c->reps.size();
    std::vector<Rep> rd((size_t)n_rep);
    std::vector<unsigned long long> T;
    std::vector<int> rep_of, cta_rep;
    rep_of.reserve((size_t)c->n_total);
    int off = 0, cell_off = 0, cta_off = 0, nF_max = 0;
    std::vector<double> F;
    for (int r = 0; r < n_rep; ++r) {
        int rc = derive_rep(c, c->reps[(size_t)r], rd[(size_t)r], F);
        if (rc != HPMC_OK) return rc;
        Rep &R = rd[(size_t)r];
        R.off = off;
        R.cell_off = cell_off;
        R.cta_off = cta_off;
        R.t_off = (int)T.size();
        // F[k] <= m 2^-53  <=>  m >= ceil(F[k] 2^53): exact integer form of the table
        for (double f : F) T.push_back((unsigned long long)std::ceil(std::ldexp(f, 53)));
        for (int i = 0; i < R.n; ++i) rep_of.push_back(r);
        const int h = R.half_nc;
        for (int a = 0; a < h * h * h; ++a) cta_rep.push_back(r);
        off += R.n;
        cell_off += R.nc * R.nc * R.nc;
        cta_off += h * h * h;
        if (R.nF > nF_max) nF_max = R.nF;
    }
    double bound = 0.0;
    for (const Rep &R : rd) bound = std::fmax(bound, R.pad_cell_bound);
    int cap = bound < (double)kTinyCellCap && p.shape == HPMC_SPHERE ? kTinyCellCap
              : (bound < (double)kSmallCellCap ? kSmallCellCap : kMaxCellCap);
    if (c->precision == HPMC_FP32_RECHECK && p.shape == HPMC_SPHERE)
        for (const Rep &R : rd)
            if (R.pad_nb_bound >= (double)max_nb(cap)) return HPMC_ERR_CAP;
    DeviceGuard g(c->device);
    if (cap != c->cap) c->cells_alloc = -2;  // force re-allocation of the bins
    c->cap = cap;
    if (cell_off != c->cells_alloc) {
        cudaFree(c->d_count);
        cudaFree(c->d_bins);
        c->d_count = nullptr;
        c->d_bins = nullptr;
        c->cells_alloc = -1;
        CK(cudaMalloc(&c->d_count, sizeof(int) * 2 * (size_t)cell_off));
        CK(cudaMalloc(&c->d_bins, sizeof(float4) * (size_t)cell_off * cap));
        c->cells_alloc = cell_off;
    }
    if (cta_off != c->cta_alloc) {
        cudaFree(c->d_cta_rep);
        c->d_cta_rep = nullptr;
        c->cta_alloc = -1;
        CK(cudaMalloc(&c->d_cta_rep, sizeof(int) * (size_t)cta_off));
        c->cta_alloc = cta_off;
    }
    CK(cudaMemcpy(c->d_cta_rep, cta_rep.data(), sizeof(int) * (size_t)cta_off,
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_rep_of, rep_of.data(), sizeof(int) * (size_t)c->n_total,
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_reps, rd.data(), sizeof(Rep) * (size_t)n_rep, cudaMemcpyHostToDevice));
    cudaFree(c->d_T);
    c->d_T = nullptr;
    if (!T.empty()) {
        CK(cudaMalloc(&c->d_T, sizeof(unsigned long long) * T.size()));
        CK(cudaMemcpy(c->d_T, T.data(), sizeof(unsigned long long) * T.size(),
                      cudaMemcpyHostToDevice));
    }
    // lens lists hold at most N_p <= nF points each: capacity nF_max, no overflow
    if (c->precision == HPMC_FP32_RECHECK) {
        // task table, bin positions, per-slot lens headers and displacements
        if (cta_off != c->task_alloc) {
            cudaFree(c->d_task);
            cudaFree(c->d_task_ord);
            c->d_task = nullptr;
            c->d_task_ord = nullptr;
            c->task_alloc = -1;
            CK(cudaMalloc(&c->d_task, sizeof(int4) * 8 * (size_t)cta_off));
            CK(cudaMalloc(&c->d_task_ord, sizeof(int4) * 32 * (size_t)cta_off));
            c->task_alloc = cta_off;
        }
        if (!c->d_cls_count) CK(cudaMalloc(&c->d_cls_count, sizeof(int) * 32));
        // readiness counters of the persistent colour phases (zero: done in
        // no sweep yet; the epoch only grows)
        if (cell_off != c->done_alloc) {
            cudaFree(c->d_done);
            c->d_done = nullptr;
            c->done_alloc = -1;
            CK(cudaMalloc(&c->d_done, sizeof(uint32_t) * (size_t)cell_off));
            CK(cudaMemset(c->d_done, 0, sizeof(uint32_t) * (size_t)cell_off));
            c->done_alloc = cell_off;
        }
        if (!c->d_epoch) {
            CK(cudaMalloc(&c->d_epoch, sizeof(uint32_t)));
            CK(cudaMemset(c->d_epoch, 0, sizeof(uint32_t)));
            CK(cudaMalloc(&c->d_ticket, sizeof(int)));
            CK(cudaMemset(c->d_ticket, 0, sizeof(int)));
        }
        if (!c->d_binpos) CK(cudaMalloc(&c->d_binpos, sizeof(int) * (size_t)c->n_total));
        const long long slots = (long long)cell_off * cap;
        if (slots != c->aux_alloc) {
            cudaFree(c->d_hdr_bin);
            cudaFree(c->d_mv_bin);
            cudaFree(c->d_lens_bin);
            c->d_hdr_bin = nullptr;
            c->d_mv_bin = nullptr;
            c->d_lens_bin = nullptr;
            c->aux_alloc = -1;
            CK(cudaMalloc(&c->d_hdr_bin, sizeof(int4) * (size_t)slots));
            CK(cudaMalloc(&c->d_mv_bin, sizeof(float4) * (size_t)slots));
            CK(cudaMalloc(&c->d_lens_bin, sizeof(float4) * kLensInline * (size_t)slots));
            c->aux_alloc = slots;
        }
        if (p.shape != HPMC_SPHERE && slots != c->binq_alloc) {
            cudaFree(c->d_bin_q);
            c->d_bin_q = nullptr;
            c->binq_alloc = -1;
            CK(cudaMalloc(&c->d_bin_q, sizeof(float4) * (size_t)slots));
            c->binq_alloc = slots;
        }
    } else if (c->d_task) {
        cudaFree(c->d_task);
        cudaFree(c->d_task_ord);
        cudaFree(c->d_cls_count);
        c->d_task = nullptr;
        c->d_task_ord = nullptr;
        c->d_cls_count = nullptr;
        c->task_alloc = -1;
    }
    if (c->precision == HPMC_FP32_RECHECK) {
        if (!c->d_prop_pos) CK(cudaMalloc(&c->d_prop_pos, sizeof(double4) * (size_t)c->n_total));
        if (p.shape != HPMC_SPHERE && !c->d_prop_quat)
            CK(cudaMalloc(&c->d_prop_quat, sizeof(double4) * (size_t)c->n_total));
    }
    if (c->precision == HPMC_FP32_RECHECK) {
        if (nF_max > c->lens_cap) {
            const double bytes = (double)sizeof(float4) * (double)c->n_total * (double)nF_max;
            if (bytes > 64.0 * (1ull << 30)) return HPMC_ERR_CAP;
            cudaFree(c->d_lens);
            c->d_lens = nullptr;
            c->lens_cap = 0;
            CK(cudaMalloc(&c->d_lens, sizeof(float4) * (size_t)c->n_total * (size_t)nF_max));
            c->lens_cap = nF_max;
        }
    }
    c->rdev = rd;
    c->n_cells = cell_off;
    c->n_cta = cta_off;
    c->nF_max = nF_max;

    // (the graphs of the previous parameters go first: the check must not
    // launch a stale one)
    free_graph(c);
    int rc = check_config(c);
    if (rc != HPMC_OK) return rc;

    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_sweep(c, c->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (rc != HPMC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    CK(e);
    c->graph = graph;
    CK(cudaGraphInstantiate(&c->exec, c->graph, 0));
    // the check an upload runs, as one graph launch
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_check(c, c->cap_stream);
    cudaGraph_t cg = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &cg);
    if (rc != HPMC_OK) {
        if (cg) cudaGraphDestroy(cg);
        return rc;
    }
    CK(e);
    e = cudaGraphInstantiate(&c->check_exec, cg, 0);
    cudaGraphDestroy(cg);
    CK(e);
    c->dirty = false;
    return HPMC_OK;
}

// Device address of a host buffer the GPU reaches directly (page-locked and
// mapped, as every pinned allocation is under unified addressing), else
// null: such buffers are read and written in place by the layout kernels,
// with no staging copy.
// read-backs of at least this many bytes take the staging copy (see
// hpmc_get_state)
constexpr size_t kDmaReadBytes = (size_t)4 << 20;

const double *mapped_host(const double *p)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // (an unregistered pointer is not an error here)
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? static_cast<const double *>(a.devicePointer) : nullptr;
}

int copy_in(hpmc_ctx *c, const double *pos, const double *quat, int mem, cudaStream_t s)
{
    const int n = c->n_total;
    const int nb = (n + 255) / 256;
    if (mem == HPMC_DEVICE) {
        k_unpack<<<nb, 256, 0, s>>>(n, pos, quat, c->d_pos, quat ? c->d_quat : nullptr);
        CK(cudaGetLastError());
        return HPMC_OK;
    }
    if (mem != HPMC_HOST) return HPMC_ERR_ARG;
    if (pos) {
        const double *src = mapped_host(pos);
        if (!src) {
            CK(cudaMemcpyAsync(c->d_stage, pos, sizeof(double) * 3 * (size_t)n,
                               cudaMemcpyHostToDevice, s));
            src = c->d_stage;
        }
        k_unpack<<<nb, 256, 0, s>>>(n, src, nullptr, c->d_pos, nullptr);
        CK(cudaGetLastError());
    }
    if (quat) {
        const double *src = mapped_host(quat);
        if (!src) {
            CK(cudaMemcpyAsync(c->d_stage, quat, sizeof(double) * 4 * (size_t)n,
                               cudaMemcpyHostToDevice, s));
            src = c->d_stage;
        }
        k_unpack<<<nb, 256, 0, s>>>(n, nullptr, src, nullptr, c->d_quat);
        CK(cudaGetLastError());
    }
    return HPMC_OK;
}

// Allocate the per-colloid and per-replica buffers of a new context.
int alloc_ctx(hpmc_ctx *c)
{
    const int n = c->n_total, n_rep = (int)c->reps.size();
    CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    CK(cudaMallocHost(&c->h_pin, sizeof(unsigned long long) * (kPinHead + counter_words(c))));
    {
        std::vector<int> live((size_t)n_rep);
        for (int r = 0; r < n_rep; ++r) live[(size_t)r] = c->reps[(size_t)r].n;
        CK(cudaMalloc(&c->d_n_live, sizeof(int) * (size_t)n_rep));
        CK(cudaMemcpy(c->d_n_live, live.data(), sizeof(int) * (size_t)n_rep, cudaMemcpyHostToDevice));
    }
    CK(cudaMalloc(&c->d_pos, sizeof(double4) * (size_t)n));
    CK(cudaMalloc(&c->d_quat, sizeof(double4) * (size_t)n));
    CK(cudaMalloc(&c->d_rel, sizeof(float4) * (size_t)n));
    CK(cudaMalloc(&c->d_stage, sizeof(double) * 4 * (size_t)n));
    CK(cudaMalloc(&c->d_rep_of, sizeof(int) * (size_t)n));
    CK(cudaMalloc(&c->d_reps, sizeof(Rep) * (size_t)n_rep));
    CK(cudaMalloc(&c->d_sched, sizeof(Sched) * (size_t)n_rep));
    CK(cudaMalloc(&c->d_sweep, sizeof(unsigned long long)));
    CK(cudaMalloc(&c->d_counters,
                  sizeof(unsigned long long) * (size_t)n_rep * kRepSlots * kNumCounters));
    CK(cudaMalloc(&c->d_err, 2 * sizeof(int)));   // error code, check id
    CK(cudaMalloc(&c->d_flag, sizeof(int)));
    CK(cudaMemsetAsync(c->d_sweep, 0, sizeof(unsigned long long), c->cap_stream));
    CK(cudaMemsetAsync(c->d_counters, 0,
                       sizeof(unsigned long long) * (size_t)n_rep * kRepSlots * kNumCounters,
                       c->cap_stream));
    CK(cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int), c->cap_stream));
    // identity orientations unless given
    std::vector<double> ident(4 * (size_t)n, 0.0);
    for (int i = 0; i < n; ++i) ident[4 * (size_t)i] = 1.0;
    CK(cudaMemcpy(c->d_stage, ident.data(), sizeof(double) * 4 * (size_t)n,
                  cudaMemcpyHostToDevice));
    k_unpack<<<(n + 255) / 256, 256, 0, c->cap_stream>>>(n, nullptr, c->d_stage, nullptr,
                                                         c->d_quat);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->cap_stream));
    return HPMC_OK;
}

void sum_counters(const unsigned long long *h, int r0, int r1, hpmc_counters *out)
{
    uint64_t tot[kNumCounters] = {0};
    for (int r = r0; r < r1; ++r)
        for (int slot = 0; slot < kRepSlots; ++slot)
            for (int k = 0; k < kNumCounters; ++k)
                tot[k] += h[((size_t)r * kRepSlots + slot) * kNumCounters + k];
    std::memset(out, 0, sizeof *out);
    out->moves = tot[kMoves];
    out->accept = tot[kAccept];
    out->reject_cell = tot[kRejCell];
    out->reject_overlap = tot[kRejOverlap];
    out->reject_depletant = tot[kRejDep];
    out->reject_cb = tot[kRejCb];
    out->dep_drawn = tot[kDepDrawn];
    out->translate = tot[kTranslate];
    out->dep_evaluated = tot[kDepEval];
    out->dep_blocking = tot[kDepBlocking];
    out->cb_fwd_ok = tot[kCbFwdOk];
    out->cb_rev_ok = tot[kCbRevOk];
    out->cap_hits = tot[kCapHits];
    out->rechecks = tot[kRechecks];
}

// Enqueue the copies of the error word and (optionally) the counters into
// the pinned staging block; the caller synchronises once.
int stage_err_counters(hpmc_ctx *c, cudaStream_t s, bool counters)
{
    CK(cudaMemcpyAsync(c->h_pin + kPinErr, c->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    if (counters)
        CK(cudaMemcpyAsync(c->h_pin + kPinHead, c->d_counters,
                           sizeof(unsigned long long) * counter_words(c), cudaMemcpyDeviceToHost, s));
    return HPMC_OK;
}

int staged_err(const hpmc_ctx *c)
{
    const int e = *reinterpret_cast<const int *>(c->h_pin + kPinErr);
    const int detail = reinterpret_cast<const int *>(c->h_pin + kPinErr)[1];
    if (e && getenv("HPMC_VERBOSE"))
        fprintf(stderr, "hpmc: device error %d (%s), detail %d\n", e,
                e == kErrCandCap ? "neighbourhood or lens capacity"
                : e == kErrTimeout ? "a bounded wait ran out"
                : e == kErrCheck ? "a check of the checked build failed" : "cell bin capacity",
                detail);
    if (e == kErrTimeout) return HPMC_ERR_TIMEOUT;
    return e ? HPMC_ERR_DEVICE : HPMC_OK;
}

int read_counters(hpmc_ctx *c, std::vector<unsigned long long> &h, cudaStream_t s)
{
    h.resize(counter_words(c));
    CK(cudaMemcpyAsync(c->h_pin + kPinHead, c->d_counters, sizeof(unsigned long long) * h.size(),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::memcpy(h.data(), c->h_pin + kPinHead, sizeof(unsigned long long) * h.size());
    return HPMC_OK;
}

int read_err(hpmc_ctx *c, cudaStream_t s)
{
    int rc = stage_err_counters(c, s, false);
    if (rc != HPMC_OK) return rc;
    CK(cudaStreamSynchronize(s));
    return staged_err(c);
}

int create_ctx(hpmc_ctx **out, const std::vector<RepHost> &reps, uint64_t seed, int precision,
               int device)
{
    *out = nullptr;
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return HPMC_ERR_ARG;
    hpmc_ctx *c = new (std::nothrow) hpmc_ctx();
    if (!c) return HPMC_ERR_ARG;
    c->device = device;
    c->seed = seed;
    c->precision = precision;
    c->reps = reps;
    long long tot = 0;
    for (const RepHost &h : reps) tot += h.n;
    if (tot > (1ll << 30)) {
        delete c;
        return HPMC_ERR_CAP;
    }
    c->n_total = (int)tot;
    // performance knob of the persistent colour phases (results do not
    // depend on it): work items taken per ticket atomic
    if (const char *e = getenv("HPMC_TICKET_CHUNK")) {
        const int v = atoi(e);
        if (v >= 1 && v <= 1024) c->ticket_chunk = v;
    }
    // and of the FP32 sphere colour phases (hpmc_set_phase_waves)
    if (const char *e = getenv("HPMC_PHASE_WAVES")) {
        const int v = atoi(e);
        if (v >= -1 && v <= 64) c->phase_waves = v;
    }
    DeviceGuard g(device);
    int rc = alloc_ctx(c);
    if (rc != HPMC_OK) {
        hpmc_destroy(c);
        return rc;
    }
    *out = c;
    return HPMC_OK;
}

}  // namespace

extern "C" {

const char *hpmc_strerror(int code)
{
    switch (code) {
    case HPMC_OK: return "ok";
    case HPMC_ERR_ARG: return "invalid argument";
    case HPMC_ERR_OVERLAP: return "overlapping colloids in the configuration";
    case HPMC_ERR_CUDA: return "CUDA runtime error";
    case HPMC_ERR_TIMEOUT: return "device-side wait timed out";
    case HPMC_ERR_STATE: return "call not valid in this state";
    case HPMC_ERR_CAP: return "size exceeds a documented capacity";
    case HPMC_ERR_DEVICE: return "a kernel recorded an error";
    default: return "unknown error";
    }
}

int hpmc_init(hpmc_ctx **out, int n, double box_l, const double *pos, const double *quat,
              int mem, uint64_t seed, uint32_t replica, int precision, int device)
{
    if (!out) return HPMC_ERR_ARG;
    *out = nullptr;
    if (n < 1 || !(box_l > 0.0) || !std::isfinite(box_l) || !pos) return HPMC_ERR_ARG;
    if (mem != HPMC_HOST && mem != HPMC_DEVICE) return HPMC_ERR_ARG;
    if (precision != HPMC_FP64 && precision != HPMC_FP32_RECHECK) return HPMC_ERR_ARG;
    RepHost h;
    h.n = n;
    h.L = box_l;
    h.replica = replica;
    hpmc_ctx *c = nullptr;
    int rc = create_ctx(&c, std::vector<RepHost>(1, h), seed, precision, device);
    if (rc != HPMC_OK) return rc;
    DeviceGuard g(device);
    rc = copy_in(c, pos, quat, mem, c->cap_stream);
    if (rc == HPMC_OK) rc = cuda_fail(cudaStreamSynchronize(c->cap_stream), "sync");
    if (rc != HPMC_OK) {
        hpmc_destroy(c);
        return rc;
    }
    *out = c;
    return HPMC_OK;
}

int hpmc_init_batch(hpmc_ctx **out, int n_rep, const hpmc_replica_desc *desc, int shape,
                    const double *shape_params, int nparams, uint64_t seed, int precision,
                    int device)
{
    if (!out) return HPMC_ERR_ARG;
    *out = nullptr;
    if (n_rep < 1 || !desc) return HPMC_ERR_ARG;
    if (precision != HPMC_FP64 && precision != HPMC_FP32_RECHECK) return HPMC_ERR_ARG;
    std::vector<RepHost> reps((size_t)n_rep);
    for (int r = 0; r < n_rep; ++r) {
        const hpmc_replica_desc &d = desc[r];
        if (d.n < 1 || !(d.box_l > 0.0) || !std::isfinite(d.box_l) || !d.pos) return HPMC_ERR_ARG;
        if (!(d.q >= 0.0) || !(d.n_r >= 0.0) || !std::isfinite(d.n_r) || d.n_trial < 0)
            return HPMC_ERR_ARG;
        if (!(d.d_max >= 0.0) || !(d.a_max >= 0.0) || !(d.p_translate >= 0.0) ||
            d.p_translate > 1.0 || d.n_cell < 0 || (d.n_cell & 1))
            return HPMC_ERR_ARG;
        RepHost &h = reps[(size_t)r];
        h.n = d.n;
        h.L = d.box_l;
        h.q = d.q;
        h.n_r = d.n_r;
        h.n_trial = d.n_trial;
        h.d_max = d.d_max;
        h.a_max = d.a_max;
        h.p_translate = d.p_translate;
        h.replica = d.replica;
        h.nc_req = d.n_cell;
    }
    hpmc_ctx *c = nullptr;
    int rc = create_ctx(&c, reps, seed, precision, device);
    if (rc != HPMC_OK) return rc;
    if (shape_params) rc = hpmc_set_shape(c, shape, shape_params, nparams);
    DeviceGuard g(device);
    // replica positions, one after another
    std::vector<double> pos(3 * (size_t)c->n_total), quat;
    bool any_quat = false;
    for (int r = 0; r < n_rep; ++r) any_quat = any_quat || desc[r].quat;
    if (any_quat) quat.assign(4 * (size_t)c->n_total, 0.0);
    size_t o = 0;
    for (int r = 0; r < n_rep && rc == HPMC_OK; ++r) {
        std::memcpy(pos.data() + 3 * o, desc[r].pos, sizeof(double) * 3 * (size_t)desc[r].n);
        if (any_quat) {
            for (int i = 0; i < desc[r].n; ++i) {
                if (desc[r].quat)
                    std::memcpy(quat.data() + 4 * (o + i), desc[r].quat + 4 * (size_t)i,
                                sizeof(double) * 4);
                else
                    quat[4 * (o + i)] = 1.0;
            }
        }
        o += (size_t)desc[r].n;
    }
    if (rc == HPMC_OK)
        rc = copy_in(c, pos.data(), any_quat ? quat.data() : nullptr, HPMC_HOST, c->cap_stream);
    if (rc == HPMC_OK) rc = cuda_fail(cudaStreamSynchronize(c->cap_stream), "sync");
    if (rc != HPMC_OK) {
        hpmc_destroy(c);
        return rc;
    }
    *out = c;
    return HPMC_OK;
}

int hpmc_set_shape(hpmc_ctx *c, int kind, const double *params, int nparams)
{
    if (!c || !params) return HPMC_ERR_ARG;
    Params p = c->prm;
    if (kind == HPMC_SPHERE || kind == HPMC_HEMISPHERE) {
        if (nparams < 1 || !(params[0] > 0.0)) return HPMC_ERR_ARG;
        p.sp[0] = params[0];
        p.nsp = 1;
    } else if (kind == HPMC_SPHEROID) {
        if (nparams < 2 || !(params[0] > 0.0) || !(params[1] > 0.0)) return HPMC_ERR_ARG;
        p.sp[0] = params[0];
        p.sp[1] = params[1];
        p.nsp = 2;
    } else {
        return HPMC_ERR_ARG;
    }
    p.shape = kind;
    c->prm = p;
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_set_depletant(hpmc_ctx *c, double q, double n_r, int n_trial)
{
    if (!c || !(q >= 0.0) || !(n_r >= 0.0) || !std::isfinite(n_r) || n_trial < 0)
        return HPMC_ERR_ARG;
    for (RepHost &h : c->reps) {
        h.q = q;
        h.n_r = n_r;
        h.n_trial = n_trial;
    }
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_set_moves(hpmc_ctx *c, double d_max, double a_max, double p_translate)
{
    if (!c || !(d_max >= 0.0) || !(a_max >= 0.0) || a_max > 3.0 || !(p_translate >= 0.0) ||
        p_translate > 1.0)
        return HPMC_ERR_ARG;
    for (RepHost &h : c->reps) {
        h.d_max = d_max;
        h.a_max = a_max;
        h.p_translate = p_translate;
    }
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_set_replica_moves(hpmc_ctx *c, int r, double d_max, double a_max, double p_translate)
{
    if (!c || r < 0 || r >= (int)c->reps.size() || !(d_max >= 0.0) || !(a_max >= 0.0) ||
        a_max > 3.0 || !(p_translate >= 0.0) || p_translate > 1.0)
        return HPMC_ERR_ARG;
    RepHost &h = c->reps[(size_t)r];
    h.d_max = d_max;
    h.a_max = a_max;
    h.p_translate = p_translate;
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_set_cells(hpmc_ctx *c, int n_cell)
{
    if (!c || n_cell < 0 || (n_cell & 1) || n_cell == 1) return HPMC_ERR_ARG;
    for (RepHost &h : c->reps) h.nc_req = n_cell;
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_set_launch(hpmc_ctx *c, int warps_per_colloid, int phase_schedule)
{
    if (!c || warps_per_colloid < 1 || warps_per_colloid > kMaxThreads / 32) return HPMC_ERR_ARG;
    if (phase_schedule != HPMC_PHASES_LAUNCHES && phase_schedule != HPMC_PHASES_PERSISTENT)
        return HPMC_ERR_ARG;
    c->prm.warps = warps_per_colloid;
    c->prm.schedule = phase_schedule;
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_set_phase_waves(hpmc_ctx *c, int waves)
{
    if (!c || waves < -1 || waves > 64) return HPMC_ERR_ARG;
    c->phase_waves = waves;
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_set_wait_limit(hpmc_ctx *c, double seconds)
{
    if (!c || !(seconds >= 1e-6) || !(seconds <= 60.0)) return HPMC_ERR_ARG;
    c->wait_s = seconds;
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_debug_withhold_cell(hpmc_ctx *c, int cell)
{
    if (!c || cell < -1) return HPMC_ERR_ARG;
    c->withhold = cell;
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_autotune(hpmc_ctx *c, const int *warps, int nw, const int *cells, int nc, int n_sweeps,
                  int *best_warps, int *best_cells, double *best_ms)
{
    if (!c || !warps || !cells || nw < 1 || nc < 1 || n_sweeps < 1) return HPMC_ERR_ARG;
    for (int a = 0; a < nw; ++a)
        if (warps[a] < 1 || warps[a] > kMaxThreads / 32) return HPMC_ERR_ARG;
    for (int b = 0; b < nc; ++b)
        if (cells[b] < 0 || (cells[b] & 1) || cells[b] == 1) return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    CK(cudaDeviceSynchronize());
    const int n = c->n_total;
    const size_t cnt_bytes = sizeof(unsigned long long) * c->reps.size() * kRepSlots * kNumCounters;
    // saved state: poses, sweep index, counters, configuration
    double4 *sp = nullptr, *sq = nullptr;
    unsigned long long *sc = nullptr, sweep0 = 0;
    CK(cudaMalloc(&sp, sizeof(double4) * (size_t)n));
    cudaError_t e = cudaMalloc(&sq, sizeof(double4) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&sc, cnt_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(sp, c->d_pos, sizeof(double4) * (size_t)n, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sq, c->d_quat, sizeof(double4) * (size_t)n, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(sc, c->d_counters, cnt_bytes, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(&sweep0, c->d_sweep, sizeof sweep0, cudaMemcpyDeviceToHost);
    const Params p0 = c->prm;
    std::vector<int> nc0(c->reps.size());
    for (size_t r = 0; r < c->reps.size(); ++r) nc0[r] = c->reps[r].nc_req;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    int rc = cuda_fail(e, "autotune setup");
    double best = 1e300;
    int bw = -1, bc = -1;
    auto restore = [&]() -> int {
        CK(cudaMemcpy(c->d_pos, sp, sizeof(double4) * (size_t)n, cudaMemcpyDeviceToDevice));
        CK(cudaMemcpy(c->d_quat, sq, sizeof(double4) * (size_t)n, cudaMemcpyDeviceToDevice));
        CK(cudaMemcpy(c->d_counters, sc, cnt_bytes, cudaMemcpyDeviceToDevice));
        CK(cudaMemcpy(c->d_sweep, &sweep0, sizeof sweep0, cudaMemcpyHostToDevice));
        CK(cudaMemset(c->d_err, 0, 2 * sizeof(int)));
        c->state_dirty = true;   // cell populations are rebuilt before the next sweep
        return HPMC_OK;
    };
    for (int b = 0; b < nc && rc == HPMC_OK; ++b) {
        for (int a = 0; a < nw && rc == HPMC_OK; ++a) {
            c->prm.warps = warps[a];
            for (RepHost &h : c->reps) h.nc_req = cells[b];
            c->dirty = true;
            const bool timing = c->timing;
            c->timing = false;
            int rs = hpmc_sweep(c, 1, c->cap_stream);
            if (rs == HPMC_OK) {
                e = cudaEventRecord(t0, c->cap_stream);
                if (e == cudaSuccess) rs = hpmc_sweep(c, n_sweeps, c->cap_stream);
                if (e == cudaSuccess && rs == HPMC_OK) e = cudaEventRecord(t1, c->cap_stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                float ms = 0.0f;
                if (e == cudaSuccess && rs == HPMC_OK) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e != cudaSuccess) rc = cuda_fail(e, "autotune timing");
                else if (rs == HPMC_OK && read_err(c, c->cap_stream) == HPMC_OK &&
                         ms / n_sweeps < best) {
                    best = ms / n_sweeps;
                    bw = warps[a];
                    bc = cells[b];
                }
            } else if (rs == HPMC_ERR_CUDA) {
                rc = rs;
            }
            c->timing = timing;
            if (rc == HPMC_OK) rc = restore();
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(sp);
    cudaFree(sq);
    cudaFree(sc);
    if (rc != HPMC_OK) {
        c->prm = p0;
        for (size_t r = 0; r < c->reps.size(); ++r) c->reps[r].nc_req = nc0[r];
        c->dirty = true;
        return rc;
    }
    if (bw < 0) {
        c->prm = p0;
        for (size_t r = 0; r < c->reps.size(); ++r) c->reps[r].nc_req = nc0[r];
        c->dirty = true;
        return HPMC_ERR_ARG;
    }
    c->prm = p0;
    c->prm.warps = bw;
    for (RepHost &h : c->reps) h.nc_req = bc;
    c->dirty = true;
    if (best_warps) *best_warps = bw;
    if (best_cells) *best_cells = bc;
    if (best_ms) *best_ms = best;
    return HPMC_OK;
}

int hpmc_sweep(hpmc_ctx *c, int n_sweeps, void *stream)
{
    if (!c || n_sweeps < 0) return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (c->dirty || c->state_dirty) {
        // order the preparation after the caller's pending work
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, s));
        CK(cudaStreamWaitEvent(c->cap_stream, ev, 0));
        cudaEventDestroy(ev);
        int rc = c->dirty ? prepare(c) : check_config(c);
        if (rc != HPMC_OK) return rc;
    }
    // NVTX: one range per call, and (timing mode, kernels launched one by
    // one) one per sweep with nested ranges for the cell lists, the lens
    // kernel and each colour phase
    nvtxRangePushA("hpmc_sweep");
    if (c->timing) {
        for (int k = 0; k < n_sweeps; ++k) {
            nvtxRangePushA("sweep");
            int rc = enqueue_sweep_timed(c, s);
            nvtxRangePop();
            if (rc != HPMC_OK) {
                nvtxRangePop();
                return rc;
            }
        }
        nvtxRangePop();
        return HPMC_OK;
    }
    for (int k = 0; k < n_sweeps; ++k) {
        const cudaError_t e = cudaGraphLaunch(c->exec, s);
        if (e != cudaSuccess) {
            nvtxRangePop();
            return cuda_fail(e, "cudaGraphLaunch");
        }
    }
    nvtxRangePop();
    return HPMC_OK;
}

int hpmc_set_fp32_margin(hpmc_ctx *c, double margin)
{
    if (!c || !(margin >= 0.0) || margin > 1e3) return HPMC_ERR_ARG;
    c->prm.margin = margin;
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_set_v0(hpmc_ctx *c, int mode)
{
    if (!c || mode < HPMC_V0_CIRCUMSPHERE || mode > HPMC_V0_CUBE) return HPMC_ERR_ARG;
    if (mode == HPMC_V0_SHELL && c->prm.shape != HPMC_SPHERE) return HPMC_ERR_ARG;
    c->prm.v0_mode = mode;
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_set_soft(hpmc_ctx *c, double eps)
{
    if (!c || !(eps >= 0.0) || !std::isfinite(eps) || eps > 1e6) return HPMC_ERR_ARG;
    c->prm.soft_eps = eps;
    c->dirty = true;
    return HPMC_OK;
}

int hpmc_set_timing(hpmc_ctx *c, int on)
{
    if (!c) return HPMC_ERR_ARG;
    c->timing = on != 0;
    return HPMC_OK;
}

int hpmc_get_timing(hpmc_ctx *c, double *ms, uint64_t *launches, int nkinds)
{
    if (!c || nkinds < 0) return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    CK(cudaDeviceSynchronize());
    double acc[3] = {0.0, 0.0, 0.0};
    uint64_t cnt[3] = {0, 0, 0};
    for (size_t k = 0; k < c->tkind.size(); ++k) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, c->tev[2 * k], c->tev[2 * k + 1]));
        acc[c->tkind[k]] += t;
        cnt[c->tkind[k]] += 1;
    }
    for (cudaEvent_t e : c->tev) c->tpool.push_back(e);
    c->tev.clear();
    c->tkind.clear();
    for (int k = 0; k < nkinds && k < 3; ++k) {
        if (ms) ms[k] = acc[k];
        if (launches) launches[k] = cnt[k];
    }
    return HPMC_OK;
}

int hpmc_get_state(hpmc_ctx *c, double *pos, double *quat, int mem, uint64_t *sweep,
                   hpmc_counters *counters, void *stream)
{
    if (!c || (mem != HPMC_HOST && mem != HPMC_DEVICE)) return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = c->n_total, nb = (n + 255) / 256;
    if (mem == HPMC_DEVICE) {
        if (pos || quat) {
            k_pack<<<nb, 256, 0, s>>>(n, c->d_pos, c->d_quat, pos, quat);
            CK(cudaGetLastError());
        }
    } else {
        bool staged = false;
        if (pos) {
            // a large read-back goes through the staging buffer and one DMA
            // copy (measured faster than the layout kernel's writes across
            // the host link: 0.15 against 0.25 ms for 621 288 positions); a
            // small one is written in place
            double *dst = (size_t)n * 3 * sizeof(double) >= kDmaReadBytes
                              ? nullptr : const_cast<double *>(mapped_host(pos));
            if (dst) {
                k_pack<<<nb, 256, 0, s>>>(n, c->d_pos, nullptr, dst, nullptr);
                CK(cudaGetLastError());
            } else {
                k_pack<<<nb, 256, 0, s>>>(n, c->d_pos, nullptr, c->d_stage, nullptr);
                CK(cudaGetLastError());
                CK(cudaMemcpyAsync(pos, c->d_stage, sizeof(double) * 3 * (size_t)n,
                                   cudaMemcpyDeviceToHost, s));
                staged = true;
            }
        }
        if (quat) {
            double *dst = const_cast<double *>(mapped_host(quat));
            if (dst) {
                k_pack<<<nb, 256, 0, s>>>(n, nullptr, c->d_quat, nullptr, dst);
                CK(cudaGetLastError());
            } else {
                // (the staging buffer is reused: the position copy must finish first)
                if (staged) CK(cudaStreamSynchronize(s));
                k_pack<<<nb, 256, 0, s>>>(n, nullptr, c->d_quat, nullptr, c->d_stage);
                CK(cudaGetLastError());
                CK(cudaMemcpyAsync(quat, c->d_stage, sizeof(double) * 4 * (size_t)n,
                                   cudaMemcpyDeviceToHost, s));
            }
        }
    }
    // the sweep index, the counters and the error word in the same round trip
    if (sweep)
        CK(cudaMemcpyAsync(c->h_pin + kPinSweep, c->d_sweep, sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
    int rc = stage_err_counters(c, s, counters != nullptr);
    if (rc != HPMC_OK) return rc;
    CK(cudaStreamSynchronize(s));
    if (sweep) *sweep = c->h_pin[kPinSweep];
    if (counters) sum_counters(c->h_pin + kPinHead, 0, (int)c->reps.size(), counters);
    return staged_err(c);
}

int hpmc_get_replica(hpmc_ctx *c, int r, double *pos, double *quat, hpmc_counters *counters)
{
    if (!c || r < 0 || r >= (int)c->reps.size()) return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = c->cap_stream;
    CK(cudaDeviceSynchronize());
    size_t off = 0;
    for (int k = 0; k < r; ++k) off += (size_t)c->reps[(size_t)k].n;
    const int n = c->reps[(size_t)r].n;
    const int nb = (n + 255) / 256;
    if (pos) {
        k_pack<<<nb, 256, 0, s>>>(n, c->d_pos + off, nullptr, c->d_stage, nullptr);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(pos, c->d_stage, sizeof(double) * 3 * (size_t)n,
                           cudaMemcpyDeviceToHost, s));
    }
    if (quat) {
        k_pack<<<nb, 256, 0, s>>>(n, nullptr, c->d_quat + off, nullptr, c->d_stage + 3 * (size_t)n);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(quat, c->d_stage + 3 * (size_t)n, sizeof(double) * 4 * (size_t)n,
                           cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    if (counters) {
        std::vector<unsigned long long> h;
        int rc = read_counters(c, h, s);
        if (rc != HPMC_OK) return rc;
        sum_counters(h.data(), r, r + 1, counters);
    }
    return read_err(c, s);
}

int hpmc_set_state(hpmc_ctx *c, const double *pos, const double *quat, int mem, uint64_t sweep,
                   void *stream)
{
    if (!c || (mem != HPMC_HOST && mem != HPMC_DEVICE)) return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = copy_in(c, pos, quat, mem, s);
    if (rc != HPMC_OK) return rc;
    c->h_pin[kPinUp] = sweep;
    CK(cudaMemcpyAsync(c->d_sweep, c->h_pin + kPinUp, sizeof(unsigned long long),
                       cudaMemcpyHostToDevice, s));
    c->state_dirty = true;  // re-validate the new configuration before the next sweep
    if (c->dirty) {
        // (the next sweep prepares the context, the check included)
        CK(cudaStreamSynchronize(s));
        return HPMC_OK;
    }
    // validate now, in the same host round trip as the upload; a failed check
    // leaves the state dirty, so the next sweep repeats it and reports it
    rc = check_config(c, s, false);
    return rc == HPMC_ERR_CUDA ? rc : HPMC_OK;
}

int hpmc_get_size(hpmc_ctx *c, int *n_total, int *n_rep)
{
    if (!c) return HPMC_ERR_ARG;
    if (n_total) *n_total = c->n_total;
    if (n_rep) *n_rep = (int)c->reps.size();
    return HPMC_OK;
}

int hpmc_reset_counters(hpmc_ctx *c)
{
    if (!c) return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    CK(cudaDeviceSynchronize());
    CK(cudaMemset(c->d_counters, 0,
                  sizeof(unsigned long long) * c->reps.size() * kRepSlots * kNumCounters));
    return HPMC_OK;
}

int hpmc_sync(hpmc_ctx *c)
{
    if (!c) return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    CK(cudaDeviceSynchronize());
    return read_err(c, c->cap_stream);
}

int hpmc_cell_list(int n, double box_l, int n_cell, const double *pos_dev, uint64_t seed,
                   uint32_t replica, uint64_t sweep, int *cell_start_dev, int *cell_idx_dev,
                   void *stream)
{
    if (n < 0 || !(box_l > 0.0) || n_cell < 2 || (n_cell & 1) || n_cell > 1024) return HPMC_ERR_ARG;
    if (n > 0 && (!pos_dev || !cell_idx_dev)) return HPMC_ERR_ARG;
    if (!cell_start_dev) return HPMC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int ncell = n_cell * n_cell * n_cell;
    const double w = box_l / (double)n_cell;
    int *count = nullptr, *cell_of = nullptr;
    CK(cudaMallocAsync(&count, sizeof(int) * (size_t)ncell, s));
    cudaError_t e = cudaMallocAsync(&cell_of, sizeof(int) * (size_t)(n > 0 ? n : 1), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(count, s);
        return cuda_fail(e, "cudaMallocAsync");
    }
    int rc = HPMC_OK;
    e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)ncell, s);
    if (e == cudaSuccess) {
        const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ replica;
        if (n > 0)
            k_csr_count<<<(n + 255) / 256, 256, 0, s>>>(n, box_l, w, n_cell, pos_dev, 3, k0, k1,
                                                        (uint32_t)sweep, cell_of, count);
        k_csr_scan<<<1, 1024, 0, s>>>(ncell, count, cell_start_dev);
        if (n > 0) {
            k_csr_scatter<<<(n + 255) / 256, 256, 0, s>>>(n, cell_of, count, cell_idx_dev);
            k_csr_sort<<<(ncell + 255) / 256, 256, 0, s>>>(ncell, cell_start_dev, cell_idx_dev);
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "hpmc_cell_list");
    cudaFreeAsync(cell_of, s);
    cudaFreeAsync(count, s);
    return rc;
}

int hpmc_kernel_arch(int *binary_version, int *ptx_version)
{
    if (!binary_version && !ptx_version) return HPMC_ERR_ARG;
    cudaFuncAttributes a;
    CK(cudaFuncGetAttributes(&a, k_philox));
    if (binary_version) *binary_version = a.binaryVersion;
    if (ptx_version) *ptx_version = a.ptxVersion;
    return HPMC_OK;
}

int hpmc_philox(int n, const uint32_t *ctr_dev, const uint32_t *key_dev, uint32_t *out_dev,
                int variant, void *stream)
{
    if (n < 0 || (variant != 0 && variant != 1)) return HPMC_ERR_ARG;
    if (n == 0) return HPMC_OK;
    if (!ctr_dev || !key_dev || !out_dev) return HPMC_ERR_ARG;
    k_philox<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, ctr_dev, key_dev, out_dev, variant);
    CK(cudaGetLastError());
    return HPMC_OK;
}

int hpmc_set_live(hpmc_ctx *c, int replica, int n_live)
{
    if (!c || replica < 0 || replica >= (int)c->reps.size() || c->prm.shape != HPMC_SPHERE ||
        n_live < 0 || n_live > c->reps[(size_t)replica].n)
        return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(c->d_n_live + replica, &n_live, sizeof(int), cudaMemcpyHostToDevice));
    c->state_dirty = true;   // re-validate the colloids in use at the next sweep
    return HPMC_OK;
}

int hpmc_get_live(hpmc_ctx *c, int *n_live)
{
    if (!c || !n_live) return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(n_live, c->d_n_live, sizeof(int) * c->reps.size(), cudaMemcpyDeviceToHost));
    return HPMC_OK;
}

int hpmc_gibbs_exchange(hpmc_ctx *c, int n_attempts, void *stream)
{
    if (!c || n_attempts < 0) return HPMC_ERR_ARG;
    const int n_rep = (int)c->reps.size();
    if (c->prm.shape != HPMC_SPHERE || (n_rep & 1)) return HPMC_ERR_ARG;
    // (the exchange inserts depletants in the circumsphere, hard interaction)
    if (c->prm.v0_mode != HPMC_V0_CIRCUMSPHERE || c->prm.soft_eps > 0.0) return HPMC_ERR_ARG;
    for (int p = 0; p < n_rep / 2; ++p) {
        const RepHost &a = c->reps[(size_t)(2 * p)], &b = c->reps[(size_t)(2 * p + 1)];
        if (a.q != b.q || a.n_r != b.n_r || a.n_trial != b.n_trial) return HPMC_ERR_ARG;
    }
    DeviceGuard g(c->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (c->dirty || c->state_dirty) {
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, s));
        CK(cudaStreamWaitEvent(c->cap_stream, ev, 0));
        cudaEventDestroy(ev);
        int rc = c->dirty ? prepare(c) : check_config(c);
        if (rc != HPMC_OK) return rc;
    }
    if (!c->d_gibbs_step) {
        const size_t np = (size_t)(n_rep / 2);
        CK(cudaMalloc(&c->d_gibbs_step, sizeof(unsigned long long) * np));
        CK(cudaMalloc(&c->d_gibbs_cnt, sizeof(unsigned long long) * np * kGibbsCounters));
        CK(cudaMemset(c->d_gibbs_step, 0, sizeof(unsigned long long) * np));
        CK(cudaMemset(c->d_gibbs_cnt, 0, sizeof(unsigned long long) * np * kGibbsCounters));
        CK(cudaMalloc(&c->d_gibbs_pos32, sizeof(float4) * (size_t)(c->n_total > 0 ? c->n_total : 1)));
    }
    if (n_attempts == 0 || n_rep == 0) return HPMC_OK;
    SimParams P = make_params(c);
    if (c->precision == HPMC_FP32_RECHECK) k_gibbs_exchange<true><<<n_rep / 2, kMaxThreads, 0, s>>>(P, n_attempts);
    else k_gibbs_exchange<false><<<n_rep / 2, kMaxThreads, 0, s>>>(P, n_attempts);
    CK(cudaGetLastError());
    return HPMC_OK;
}

int hpmc_get_gibbs(hpmc_ctx *c, int pair, uint64_t *step, uint64_t *counters)
{
    if (!c || pair < 0 || pair >= (int)c->reps.size() / 2) return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    CK(cudaDeviceSynchronize());
    unsigned long long st = 0, cnt[kGibbsCounters] = {0};
    if (c->d_gibbs_step) {
        CK(cudaMemcpy(&st, c->d_gibbs_step + pair, sizeof st, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(cnt, c->d_gibbs_cnt + (size_t)pair * kGibbsCounters, sizeof cnt,
                      cudaMemcpyDeviceToHost));
    }
    if (step) *step = st;
    if (counters)
        for (int k = 0; k < kGibbsCounters; ++k) counters[k] = cnt[k];
    return read_err(c, c->cap_stream);
}

int hpmc_free_volume(hpmc_ctx *c, int replica, double q, uint64_t seed, uint32_t sample,
                     uint64_t n_probe, uint64_t *n_free)
{
    if (!c || !n_free || replica < 0 || replica >= (int)c->reps.size() || !(q >= 0.0) ||
        !std::isfinite(q))
        return HPMC_ERR_ARG;
    DeviceGuard g(c->device);
    if (c->dirty || c->state_dirty) {
        CK(cudaDeviceSynchronize());
        const int rc = c->dirty ? prepare(c) : check_config(c);
        if (rc != HPMC_OK) return rc;
    }
    Rep R = c->rdev[(size_t)replica];
    R.r_dep = 0.5 * q;
    const double Rd = 0.5 * c->prm.sp[0] + 0.5 * q;
    R.R_dep2 = Rd * Rd;
    const int nc = R.nc, ncell = nc * nc * nc;
    const double w = R.L / (double)nc;
    cudaStream_t s = c->cap_stream;
    CK(cudaStreamSynchronize(s));
    int n = R.n;   // the colloids in use (slots 0 .. n - 1)
    CK(cudaMemcpy(&n, c->d_n_live + replica, sizeof(int), cudaMemcpyDeviceToHost));
    int *count = nullptr, *cell_of = nullptr, *start = nullptr, *idx = nullptr;
    unsigned long long *d_free = nullptr;
    cudaError_t e = cudaMallocAsync(&count, sizeof(int) * (size_t)ncell, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&cell_of, sizeof(int) * (size_t)std::max(n, 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&start, sizeof(int) * ((size_t)ncell + 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&idx, sizeof(int) * (size_t)std::max(n, 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_free, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)ncell, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_free, 0, sizeof(unsigned long long), s);
    unsigned long long h_free = 0;
    if (e == cudaSuccess) {
        const double *pos = reinterpret_cast<const double *>(c->d_pos + R.off);
        const int nb = std::max(1, (n + 255) / 256);   // (an empty box still has its probes)
        k_csr_count<<<nb, 256, 0, s>>>(n, R.L, w, nc, pos, 4, R.key0, R.key1, 0u, cell_of, count);
        k_csr_scan<<<1, 1024, 0, s>>>(ncell, count, start);
        k_csr_scatter<<<nb, 256, 0, s>>>(n, cell_of, count, idx);
        const unsigned long long want = (n_probe + 255) / 256;
        const int blocks = (int)std::min<unsigned long long>(want > 0 ? want : 1, 152ull * 16);
        k_free_volume<<<blocks, 256, 0, s>>>(R, nc, R.key0, R.key1, 0u, c->d_pos + R.off,
                                             c->d_quat + R.off, start, idx, (uint32_t)seed,
                                             (uint32_t)(seed >> 32), sample, n_probe, d_free);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&h_free, d_free, sizeof h_free, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFreeAsync(count, s);
    cudaFreeAsync(cell_of, s);
    cudaFreeAsync(start, s);
    cudaFreeAsync(idx, s);
    cudaFreeAsync(d_free, s);
    if (e != cudaSuccess) return cuda_fail(e, "hpmc_free_volume");
    *n_free = h_free;
    return HPMC_OK;
}

}  // extern "C"

// --- allocation-free variant of the standalone cell list ------------------------
//
// Some callers cannot allocate device memory when they need a cell list: a
// real-time loop that has a fixed memory budget after start-up, code that
// runs while another component owns the device allocator, or a framework that
// hands out memory only from its own pool.  hpmc_cell_list_noalloc serves them:
// its scratch (the per-cell counts and the per-colloid cell ids) lives in the
// file-scope device array below, which every GPU that loads this library
// holds until the process exits.
namespace {

constexpr int kNoAllocMaxCells = 1 << 16;  // n_cell^3 <= 65536, i.e. n_cell <= 40
constexpr int kNoAllocMaxN = 1 << 18;      // at most 262144 colloids
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) int g_noalloc_scratch[kNoAllocMaxCells + kNoAllocMaxN];

// In host code the symbol above is only a host-side stand-in; the device
// address is looked up once per device, with that device current.
int *g_noalloc_dev[kNoAllocMaxDevices] = {nullptr};
std::mutex g_noalloc_mutex;

int noalloc_scratch(int **out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return HPMC_ERR_CAP;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_dev[dev]) {
        void *ptr = nullptr;
        CK(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        g_noalloc_dev[dev] = (int *)ptr;
    }
    *out = g_noalloc_dev[dev];
    return HPMC_OK;
}

}  // namespace

extern "C" {

int hpmc_cell_list_noalloc(int n, double box_l, int n_cell, const double *pos_dev, uint64_t seed,
                           uint32_t replica, uint64_t sweep, int *cell_start_dev,
                           int *cell_idx_dev, void *stream)
{
    // the same argument rules as hpmc_cell_list (n_cell > 1024 is invalid
    // there too), then this entry point's own capacity
    if (n < 0 || !(box_l > 0.0) || n_cell < 2 || (n_cell & 1) || n_cell > 1024) return HPMC_ERR_ARG;
    if (n > 0 && (!pos_dev || !cell_idx_dev)) return HPMC_ERR_ARG;
    if (!cell_start_dev) return HPMC_ERR_ARG;
    if (n_cell > 40 || n > kNoAllocMaxN) return HPMC_ERR_CAP;
    const int ncell = n_cell * n_cell * n_cell;
    int *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != HPMC_OK) return rc;
    int *count = scratch, *cell_of = scratch + kNoAllocMaxCells;
    cudaStream_t s = (cudaStream_t)stream;
    const double w = box_l / (double)n_cell;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) ^ replica;
    // the array keeps the previous call's contents: the counts must start at zero
    CK(cudaMemsetAsync(count, 0, sizeof(int) * (size_t)ncell, s));
    if (n > 0)
        k_csr_count<<<(n + 255) / 256, 256, 0, s>>>(n, box_l, w, n_cell, pos_dev, 3, k0, k1,
                                                    (uint32_t)sweep, cell_of, count);
    k_csr_scan<<<1, 1024, 0, s>>>(ncell, count, cell_start_dev);
    if (n > 0) {
        k_csr_scatter<<<(n + 255) / 256, 256, 0, s>>>(n, cell_of, count, cell_idx_dev);
        k_csr_sort<<<(ncell + 255) / 256, 256, 0, s>>>(ncell, cell_start_dev, cell_idx_dev);
    }
    CK(cudaGetLastError());
    return HPMC_OK;
}

void hpmc_destroy(hpmc_ctx *c)
{
    if (!c) return;
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    free_graph(c);
    for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->tpool) cudaEventDestroy(e);
    cudaFree(c->d_pos);
    cudaFree(c->d_quat);
    cudaFree(c->d_rel);
    cudaFree(c->d_stage);
    cudaFree(c->d_count);
    cudaFree(c->d_bins);
    cudaFree(c->d_lens);
    cudaFree(c->d_prop_pos);
    cudaFree(c->d_prop_quat);
    cudaFree(c->d_task);
    cudaFree(c->d_task_ord);
    cudaFree(c->d_cls_count);
    cudaFree(c->d_binpos);
    cudaFree(c->d_hdr_bin);
    cudaFree(c->d_mv_bin);
    cudaFree(c->d_lens_bin);
    cudaFree(c->d_bin_q);
    cudaFree(c->d_reps);
    cudaFree(c->d_rep_of);
    cudaFree(c->d_cta_rep);
    cudaFree(c->d_sched);
    cudaFree(c->d_T);
    cudaFree(c->d_sweep);
    cudaFree(c->d_counters);
    cudaFree(c->d_err);
    cudaFree(c->d_flag);
    cudaFree(c->d_done);
    cudaFree(c->d_epoch);
    cudaFree(c->d_ticket);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->h_pin) cudaFreeHost(c->h_pin);
    cudaFree(c->d_n_live);
    cudaFree(c->d_gibbs_step);
    cudaFree(c->d_gibbs_cnt);
    cudaFree(c->d_gibbs_pos32);
    delete c;
}

}  // extern "C"
