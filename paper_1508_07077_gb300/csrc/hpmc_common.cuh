// Common device code of the implicit-depletant HPMC library (sm_103a).
//
// Method: Glaser, Karas & Glotzer, arXiv:1508.07077.
//   Sec. III.E  checkerboard of active cells, random grid shift and colour order
//   Sec. III.B  trial move, Poisson number of depletants, reject on overlap
//   Sec. III.C  depletants sampled in the circumsphere of the NEW pose; those
//               overlapping the old configuration are ignored
//   Sec. III.D  configurational-bias reinsertion, Eq. (12)
//   App. A      the depletants of one move are processed by cooperating threads
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
constexpr int kMaxCellCap = 64;      // colloids per cell bin, largest capacity (checked from the packing bound)
constexpr int kSmallCellCap = 32;    // capacity of the usual cells (width near d_colloid + d_depletant)
constexpr int kTinyCellCap = 16;     // spheres in cells below ~1.24 diameters (packing bound < 16)
// candidate capacity of a 27-cell neighbourhood in the FP32 sphere phase
// kernel: smaller for the smallest cells, to keep more CTAs resident
__host__ __device__ constexpr int cand_cap(int cap) { return cap <= kTinyCellCap ? 192 : kMaxCand; }
constexpr int kRepSlots = 16;        // per replica, counters are spread over slots (fewer hot atomics)
constexpr int kNumCounters = 16;
constexpr int kLensInline = 4;       // lens points kept beside each bin slot (FP32 sphere form)

enum Counter {
    kMoves = 0, kAccept, kRejCell, kRejOverlap, kRejDep, kRejCb, kDepDrawn,
    kTranslate, kDepEval, kDepBlocking, kCbFwdOk, kCbRevOk, kCapHits, kRechecks
};

enum DevError { kErrNone = 0, kErrCandCap = 1, kErrCellCap = 2, kErrTimeout = 3, kErrCheck = 4 };

// Checked build (-DHPMC_CHECKED): the FP32 sphere path bounds-checks its
// cell, bin, neighbour, shared-memory and colloid indices and the
// checkerboard invariant (Sec. III.E: a move reads only colloids of its own
// cell and of cells that are not active in the same phase), and re-takes in
// FP64 every decision that FP32 took as certain on the hard-interaction paths
// of spheres and of the anisotropic shapes (the ball and pose tests of the
// lens kernels, the cell-exit, pair and lens-point tests of the colour
// phases, the CB trials' tests) and compares the two.  A
// failed check records kErrCheck, with the check's number in the second
// error word, and the access is skipped; nothing traps.  In the regular build every check
// compiles away.
#ifdef HPMC_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

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


// Philox4x32-10 with the ten round keys of (k0, k1) computed once: the hot
// depletant loops draw many counters under one key.
struct RoundKeys {
    uint32_t a[10], b[10];
};
__device__ __forceinline__ RoundKeys round_keys(uint32_t k0, uint32_t k1)
{
    RoundKeys K;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        K.a[r] = k0 + (uint32_t)r * 0x9E3779B9u;
        K.b[r] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    return K;
}
__device__ __forceinline__ uint4 philox_rk(uint4 c, const RoundKeys &K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ K.a[r], lo1, hi0 ^ c.w ^ K.b[r], lo0);
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

// word -> real maps, exact in FP64: u01(w) = (w + 1/2) 2^-32 and
// s11(w) = (w + 1/2) 2^-31 - 1 = v 2^-31 + 2^-32 with v = w - 2^31 (the fma
// form: every intermediate is exact, so the value is the specification's).
__device__ __forceinline__ double u01(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }
__device__ __forceinline__ double s11(uint32_t w)
{
    return __fma_rn((double)(int)(w ^ 0x80000000u), 0x1p-31, 0x1p-32);
}
__device__ __forceinline__ double u53(uint32_t a, uint32_t b)
{
    return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * 0x1p-53;
}

// Paired depletant points.  The depletant stream of a trial move with hard
// colloid-depletant interactions and the circumsphere or cube V_0 takes two
// attempts from each Philox call, in blocks of 64 attempts: attempt t is half
// (t >> 5) & 1 of call 32 (t >> 6) + (t & 31), so a warp's 32 lanes draw 32
// calls and take first their first halves, then their second halves.  Half 0
// is the top 21 bits of words 0, 1, 2; half 1 is, for coordinate d, the low
// 11 bits of word d below bits 10d .. 10d + 9 of word 3 (126 bits, each used
// once).  Coordinate d is R_s s21(a_d) with s21(a) = (a + 1/2) 2^-20 - 1,
// exact in FP64 and in FP32.
__host__ __device__ __forceinline__ uint32_t paired_call(uint32_t t) { return 32u * (t >> 6) + (t & 31u); }
__host__ __device__ __forceinline__ uint32_t paired_half(uint32_t t) { return (t >> 5) & 1u; }
__host__ __device__ __forceinline__ uint3 paired_fields(uint4 w, uint32_t h)
{
    if (h == 0u) return make_uint3(w.x >> 11, w.y >> 11, w.z >> 11);
    return make_uint3((w.x & 0x7FFu) | ((w.w & 0x3FFu) << 11),
                      (w.y & 0x7FFu) | (((w.w >> 10) & 0x3FFu) << 11),
                      (w.z & 0x7FFu) | (((w.w >> 20) & 0x3FFu) << 11));
}
// (as one fused multiply-add: a 2^-20 + (2^-21 - 1) is exactly representable,
// so the single rounding is exact and the value is (a + 1/2) 2^-20 - 1)
__device__ __forceinline__ double s21(uint32_t a) { return __fma_rn((double)a, 0x1p-20, 0x1p-21 - 1.0); }
// the same value in FP32: a + 1/2 has at most 22 significant bits, the
// scaling is exact and so is the subtraction (the result is a multiple of
// 2^-21 below 1 in magnitude)
__device__ __forceinline__ float s21f(uint32_t a) { return ((float)a + 0.5f) * 0x1p-20f - 1.0f; }
// The same value without an integer-to-float conversion: f = 1 + a 2^-21 has
// a as its mantissa's top 21 bits, and 2 f + (2^-21 - 3) = (2a + 1 - 2^21)
// 2^-21 is a multiple of 2^-21 below 1 in magnitude, so the fused
// multiply-add is exact.
__device__ __forceinline__ float s21f_bits(uint32_t a)
{
    return __fmaf_rn(__uint_as_float(0x3F800000u | (a << 2)), 2.0f, 0x1p-21f - 3.0f);
}

// FP64 point of attempt t of colloid `tag`'s paired depletant stream.
__device__ __forceinline__ void paired_point64(uint32_t k0, uint32_t k1, double R_s, uint32_t sweep,
                                               uint32_t tag, uint32_t t, double &e0, double &e1,
                                               double &e2)
{
    const uint3 a = paired_fields(draw(k0, k1, sweep, tag, kPDep, 0, paired_call(t)), paired_half(t));
    e0 = R_s * s21(a.x);
    e1 = R_s * s21(a.y);
    e2 = R_s * s21(a.z);
}

// ---------------------------------------------------------------------------
// Parameters.  A context is a batch of independent replica systems (one for a
// single system); every kernel covers all replicas of the batch in one launch.
// ---------------------------------------------------------------------------
struct Sched {
    double sigma[3];
    int perm[8];
    uint32_t sweep;   // sweep index these kernels run
    uint32_t phase_of;  // phase of each colour c in bits 4c..4c+3 (the inverse of perm)
};

// One replica: its system, its parameters and where its data sit in the
// batch-wide arrays.  Colloid arrays are indexed by the global colloid index
// g = off + i (i the colloid's index inside its replica, also its RNG stream).
struct Rep {
    int n, off;            // colloids, first global colloid index
    int nc, half_nc, n_stencil;
    int cell_off;          // first global cell index
    int cta_off;           // first CTA of this replica in a colour-phase grid
    int nF, t_off;         // Poisson table length and offset in the batch table
    int has_dep, n_trial;
    uint32_t key0, key1;
    double L, half_L, w;
    double R_s, R_s2;      // sampling sphere radius (R_circ + q/2) and its square
    double R_dep2;         // sphere-depletant contact distance squared
    double contact2;       // sphere-sphere contact distance squared
    double nb_cut2;        // neighbours farther than this cannot meet a depletant
    double d_max;
    // shape (hpmc_shapes.cuh): kind, circumsphere radius about the reference
    // point, depletant radius q/2, hemisphere radius, spheroid semi-axes
    int shape, rot_on;     // rot_on: rotation moves enabled (anisotropic, a_max > 0)
    double R_circ, r_dep, sh_R, sh_a, sh_c;
    double alpha;          // tan(a_max / 2): rotation proposal scale
    double p_translate;    // probability of a translation when rotations are on
    // FP32 form: thresholds rounded to float, and the certified margins
    float w32, L32, half_L32, R_s32, T_s32, T_dep32, T_contact32, nb_cut2_32, d_max32;
    float m_r2;            // bound on |r2_fp32 - r2_fp64| (+ threshold rounding), doubled
    float m_box32;         // the same for vectors from FP32 absolute positions (error ~ u L)
    float m_cell;          // bound on the error of a cell-relative coordinate
    // FP32 form, anisotropic shapes: the shape in float, and the distance
    // margins of the depletant tests and of the colloid-pair certificates
    float R_circ32, r_dep32, sh_R32, sh_a32, sh_c32, m_d, m_pair;
    // spheroid quick tests: 1/a^2, 1/c^2 of the body, of the inner spheroid
    // (a + r, c + r) and of the outer spheroid, and the squared thresholds
    float sp_iA2, sp_iC2, sp_inA, sp_inC, sp_outA, sp_outC, sp_kin2, sp_kout2;
    double pad_cell_bound; // host: packing bound on a cell's population
    double pad_nb_bound;   // host: packing bound on the colloids within a depletant's reach
    // shell-restricted V_0 (spheres, translations): on when v0_shell; level k
    // (1..kShellLevels) samples R_in <= |e| < R_s with R_in = sh_rin[k-1],
    // thickness sh_h[k-1]; its Poisson table is the (k-1)-th block of nF
    // entries at t_off
    double soft_eps;       // > 0: Hertz colloid-depletant interaction (eps in kT)
    // FP32 form of the soft interaction: each depletant's two early exits
    // (r_new >= r_old; u01(w_3) >= e^-u_old - e^-u_new, in the lens kernel)
    // and its blocking test (in the phases) taken in FP32 when clear of the
    // bands, the full FP64 statement otherwise
    int soft32;
    float soft_eps32, soft_inv_s32, soft_r2band, soft_vband;
    // and the colour phases' blocking test: band soft_bband + U-dependent
    // terms (soft_du_nb per neighbour in range, relative u per term of U)
    float soft_du_nb, soft_bband;
    int v0_shell;
    int v0_cube;           // V_0 is the cube [-R_s, R_s)^3: every attempt is a depletant
    double dd;             // level thickness step sqrt(3) d_max / 32
    double R_s4;           // R_s^4
    float R_s4_32;
    float shell_band;      // extra relative band of the FP32 shell test (caller's margin)
    double sh_rin[32], sh_h[32];
    float sh_rin32[32], sh_h32[32];
};

constexpr int kShellLevels = 32;

// Shell level of a translation from its move words (integer rule).  The
// displacement is D_d = d_max n_d 2^-32 with n_d = 2 w_d + 1 - 2^32 (odd,
// |n_d| < 2^32).  a_d = floor(|n_d| / 2^16) + 1 exceeds |n_d| / 2^16, so with
// S = a_0^2 + a_1^2 + a_2^2 the move length obeys |D| < d_max sqrt(S) 2^-16;
// the level is the smallest k >= 1 with S <= 3 k^2 2^22, which makes
// |D| < k sqrt(3) d_max / 32, the level's thickness.
__host__ __device__ __forceinline__ int shell_level(uint32_t w0, uint32_t w1, uint32_t w2)
{
    const uint32_t w[3] = {w0, w1, w2};
    unsigned long long S = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        // |n_d| >> 16 without 64-bit signed arithmetic: |2 w + 1 - 2^32| is
        // 2 (w - 2^31) + 1 for w >= 2^31 and 2 (2^31 - w) - 1 below
        const unsigned long long n = w[d] >= 0x80000000u
                                         ? 2ull * (unsigned long long)(w[d] - 0x80000000u) + 1ull
                                         : 2ull * (unsigned long long)(0x80000000u - w[d]) - 1ull;
        const unsigned long long a = (n >> 16) + 1ull;
        S += a * a;
    }
    // k = ceil(sqrt(S / (3 2^22))) by a float estimate, fixed up exactly
    int k = (int)ceilf(sqrtf((float)S * (1.0f / 12582912.0f)));
    k = k < 1 ? 1 : (k > kShellLevels ? kShellLevels : k);
    while (k > 1 && S <= ((3ull * (unsigned long long)((k - 1) * (k - 1))) << 22)) --k;
    while (k < kShellLevels && S > ((3ull * (unsigned long long)(k * k)) << 22)) ++k;
    return k;
}

struct SimParams {
    int n_rep, n_total, cap, lens_cap;
    int n_cta;             // CTAs of a colour-phase grid (all replicas)
    const Rep *reps;
    const int *rep_of;     // global colloid index -> replica
    const int *cta_rep;    // CTA of a colour-phase grid -> replica
    double4 *pos;
    double4 *quat;
    float4 *rel;           // FP32 position relative to the origin of its cell (this sweep)
    int *count[2];         // per-cell populations, double-buffered by sweep parity
    float4 *bins;          // [cap][cell] (FP32 offset from the cell origin, global index bits
                           // in .w), unordered within a cell; see bin_at
    const unsigned long long *T;   // Poisson CDF tables as integers ceil(F[k] 2^53)
    // per-colloid depletant "lens" lists of this sweep (FP32 form):
    // lens[g][0..n) = (e, (t << 16) | k) of the depletants that overlap the new
    // pose and not the old one, in depletant order (their header is filed
    // per bin slot, hdr_bin below)
    float4 *lens;
    double4 *prop_pos;     // FP32 forms: exact proposed position of this sweep (anisotropic:
                           // .w = move kind)
    double4 *prop_quat;    // and orientation
    // per-sweep tables written by the cell-list kernel for the FP32 sphere
    // phases: task[phase][cta] = (global cell, replica, cx | cy << 10 | cz << 20);
    // binpos[g] = bin_at(cell, slot) of colloid g; the lens kernel's header
    // (N_p, obtained, n_lens) and displacement of each bin slot
    int4 *task;
    // the same tasks per phase in four classes of the cell's population
    // (>= 3, 2, 1, 0: the longest chains first), class sizes in cls_count
    int4 *task_ord;
    int *cls_count;        // [8][4]
    int *binpos;
    int4 *hdr_bin;
    float4 *mv_bin;
    float4 *lens_bin;      // the first kLensInline lens points of each bin slot
    float4 *bin_q;         // FP32 orientation of each bin slot (anisotropic FP32 form)
    // colloids in use per replica (slots off .. off + n_live - 1; fewer than
    // the replica's slots only in Gibbs-ensemble pairs), and per pair of
    // replicas the exchange step counter and counters
    int *n_live;
    unsigned long long *gibbs_step;
    unsigned long long *gibbs_cnt;
    float4 *pos32;         // FP32 images of the positions, kept by the exchange kernel
    Sched *sched;          // per replica
    unsigned long long *sweep;     // next sweep index (all replicas)
    unsigned long long *counters;  // [n_rep][kRepSlots][kNumCounters]
    int *err;
    // persistent colour phases (FP32 sphere form): readiness counter of every
    // cell (the epoch of the sweep in which it was last done), the epoch
    // (advanced by the cell-list kernel before every sweep), the ticket
    // counter of the work items (reset with it), the bound of every wait in
    // nanoseconds of global time, and a cell whose readiness is never
    // published (-1: none; set only to test the bounded waits)
    int n_cells;
    uint32_t *done;
    uint32_t *epoch;
    int *ticket;
    int ticket_chunk;      // work items a CTA takes per ticket atomic
    int persistent;        // the colour phases run as one persistent launch
    unsigned long long wait_ns;
    int withhold;
};

// True (and the error recorded) when a check of the checked build fails.
__device__ __noinline__ bool check_failed(int *err, int id)
{
    atomicCAS(err, kErrNone, kErrCheck);
    atomicCAS(err + 1, 0, id);
    return true;
}
#define HPMC_CHECK_FAILS(P, cond, id) (kChecked && !(cond) && check_failed((P).err, (id)))

// --- bounded device-side waits ----------------------------------------------

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *flag has reached target (compared modulo 2^32, so epochs may
// wrap), at most limit_ns of global time and a matching number of polls;
// false if the wait ran out.  Polls back off with __nanosleep after the
// first 64.
__device__ __noinline__ bool wait_ready_slow(const uint32_t *flag, uint32_t target,
                                             unsigned long long limit_ns)
{
    const unsigned long long t0 = globaltimer_ns();
    const unsigned long long max_polls = limit_ns / 32ull + 1024ull;
    for (unsigned long long it = 0; it < max_polls; ++it) {
        // the usual wait is about one cell's work: poll at L2 latency first,
        // then back off
        if (it >= 64) __nanosleep(it < 256 ? 64 : 512);
        if ((int)(ld_acquire_u32(flag) - target) >= 0) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

__device__ __forceinline__ bool wait_ready(const uint32_t *flag, uint32_t target,
                                           unsigned long long limit_ns)
{
    if ((int)(ld_acquire_u32(flag) - target) >= 0) return true;
    return wait_ready_slow(flag, target, limit_ns);
}

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

// Attempt w of the shell generator at level lvl, FP64 in the specification's
// operation order: v_d = s11(w_d) uniform in the cube, r = R_in + h u01(w_3)
// uniform in [R_in, R_s); accepted iff |v|^6 R_s^4 < r^4 (that is
// |v|^3 < (r / R_s)^2: for v in the unit ball |v|^3 is uniform and
// independent of the direction, so the accepted r has density ~ r^2 and e is
// uniform in the shell); the point is e = v (r / |v|).
__device__ __forceinline__ bool shell_point64(const Rep &R, int lvl, uint4 w, double &e0, double &e1,
                                              double &e2)
{
    const double v0 = s11(w.x), v1 = s11(w.y), v2 = s11(w.z);
    const double p2 = (v0 * v0 + v1 * v1) + v2 * v2;
    const double r = R.sh_rin[lvl - 1] + R.sh_h[lvl - 1] * u01(w.w);
    const double r2 = r * r;
    const double sc = r / sqrt(p2);
    e0 = v0 * sc;
    e1 = v1 * sc;
    e2 = v2 * sc;
    return ((p2 * p2) * p2) * R.R_s4 < r2 * r2;
}

__device__ __forceinline__ double wrap_box(double x, double L)
{
    if (x < 0.0) x = x + L;
    if (x >= L) x = x - L;
    return x;
}

// ---------------------------------------------------------------------------
// Sweep schedule (Sec. III.E): grid shift and colour order.
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
// Per-CTA set-up of a colour phase: which replica and cell this CTA owns, and
// the zeroing of the other count buffer for the next sweep.
// ---------------------------------------------------------------------------
struct CellTask {
    int r;                 // replica
    int cx, cy, cz;        // cell coordinates inside the replica
    int cell;              // global cell index
    int n_own;
    int *count;            // this sweep's populations (global cell index)
};

__device__ __forceinline__ CellTask cell_task(const SimParams &P, const Rep &R, int r, int phase)
{
    CellTask t;
    t.r = r;
    const int colour = P.sched[r].perm[phase];
    const int h = R.half_nc, nc = R.nc;
    const int a = blockIdx.x - R.cta_off;
    t.cx = 2 * (a % h) + (colour & 1);
    t.cy = 2 * ((a / h) % h) + ((colour >> 1) & 1);
    t.cz = 2 * (a / (h * h)) + ((colour >> 2) & 1);
    t.cell = R.cell_off + t.cx + nc * (t.cy + nc * t.cz);
    t.count = P.count[P.sched[r].sweep & 1u];
    t.n_own = t.count[t.cell];
    return t;
}

// Every cell is owned by exactly one CTA of one phase per sweep: that CTA
// zeroes the cell in the other buffer, which the next sweep fills.
__device__ __forceinline__ void clear_next(const SimParams &P, uint32_t sweep, int cell)
{
    if (threadIdx.x == 0) P.count[(sweep + 1u) & 1u][cell] = 0;
}

// Flat index of slot s of global cell c in the per-slot arrays (bins, bin_q,
// hdr_bin, mv_bin; lens_bin in units of kLensInline points): slot-major, so
// that the first slots of neighbouring cells share cache lines (most cells
// hold one or two colloids; a cell-major layout gave every cell's few used
// slots a cache line of their own in each array).
__device__ __forceinline__ size_t bin_at(const SimParams &P, int c, int s)
{
    return (size_t)s * (size_t)P.n_cells + (size_t)c;
}

// The global cell of a flat slot index.
__device__ __forceinline__ int bin_cell(const SimParams &P, int bp)
{
    return bp % P.n_cells;
}

// Sort the own cell's members into s_own[0..n) ascending (n <= kMaxCellCap).
__device__ __forceinline__ void own_members_sorted(const SimParams &P, int cell, int n, int *s_tmp,
                                                   int *s_own)
{
    const int tid = threadIdx.x;
    for (int t = tid; t < n; t += blockDim.x)
        s_tmp[t] = __float_as_int(P.bins[bin_at(P, cell, t)].w);
    __syncthreads();
    for (int t = tid; t < n; t += blockDim.x) {
        const int v = s_tmp[t];
        int r = 0;
        for (int u = 0; u < n; ++u) r += s_tmp[u] < v ? 1 : 0;
        s_own[r] = v;
    }
    __syncthreads();
}

// Neighbour cell (global index, and geometric offset in cells) number `t` of
// the deduplicated 27-cell stencil of (cx, cy, cz).
__device__ __forceinline__ int stencil_cell(const Rep &R, int t, int cx, int cy, int cz, int &dx,
                                            int &dy, int &dz)
{
    const int ns = R.n_stencil, nc = R.nc;
    const int ox = t % ns, oy = (t / ns) % ns, oz = t / (ns * ns);
    int nx, ny, nz;
    if (nc == 2) {
        nx = ox; ny = oy; nz = oz;
        dx = ox - cx; dy = oy - cy; dz = oz - cz;
    } else {
        nx = (cx + ox - 1 + nc) % nc;
        ny = (cy + oy - 1 + nc) % nc;
        nz = (cz + oz - 1 + nc) % nc;
        dx = ox - 1; dy = oy - 1; dz = oz - 1;
    }
    return R.cell_off + nx + nc * (ny + nc * nz);
}

// Programmatic dependent launch (a kernel launched with programmatic stream
// serialization may start before its predecessor finishes): let the next
// kernel in the stream launch early, and wait for the predecessor's
// completion (and the visibility of its writes) before touching its results.
// --- FP32 helpers of the certified forms ---------------------------------

// R * s11(w) in FP32 without an integer-to-float conversion: the float with
// exponent of 2 and the top 23 bits of w as mantissa lies in [2, 4), so
// f - 3 = -1 + (w >> 9) 2^-22 exactly, within 2^-22 below s11(w); one more
// rounding for the product.  |result - R s11(w)| <= 6 u R (u = 2^-24).
__device__ __forceinline__ float coord32(uint32_t w, float R)
{
    return (__int_as_float(0x40000000u | (w >> 9)) - 3.0f) * R;
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

// (one thread) The factors of a CB pass in ascending slot order, i.e.
// ascending depletant index: bit l of masks[w] marks slot 32 w + l as holding
// a factor; kc[slot] is its depletant index k (factor f[slot], nonzero) or
// -1 - k (a zero factor).  Multiplies the nonzero factors into W up to the
// first zero one and returns that one's k, else -1; *n_fact counts the
// factors walked (the zero one included).  Slots are skipped and zeros found
// by integer tests: a thread's FP64 work is one product per factor.
__device__ __forceinline__ int cb_walk(const unsigned *masks, int nwarps, const int *kc, const double *f,
                                       double &W, int &n_fact)
{
    for (int w = 0; w < nwarps; ++w) {
        unsigned m = masks[w];
        while (m) {
            const int u = (w << 5) + __ffs(m) - 1;
            m &= m - 1u;
            ++n_fact;
            const int c = kc[u];
            if (c < 0) return -1 - c;
            W = W * f[u];
        }
    }
    return -1;
}

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Stencil cell number t of (cx, cy, cz) from the cell count per side and the
// replica's first cell only (no Rep access).
__device__ __forceinline__ int stencil_cell_nc(int nc, int cell_off, int t, int cx, int cy, int cz,
                                               int &dx, int &dy, int &dz)
{
    const int ns = nc == 2 ? 2 : 3;
    const int ox = t % ns, oy = (t / ns) % ns, oz = t / (ns * ns);
    int nx, ny, nz;
    if (nc == 2) {
        nx = ox; ny = oy; nz = oz;
        dx = ox - cx; dy = oy - cy; dz = oz - cz;
    } else {
        nx = (cx + ox - 1 + nc) % nc;
        ny = (cy + oy - 1 + nc) % nc;
        nz = (cz + oz - 1 + nc) % nc;
        dx = ox - 1; dy = oy - 1; dz = oz - 1;
    }
    return cell_off + nx + nc * (ny + nc * nz);
}

__device__ __forceinline__ void flush_counters(const SimParams &P, int r,
                                               const unsigned long long *c)
{
    unsigned long long *cnt =
        P.counters + ((size_t)r * kRepSlots + (blockIdx.x % kRepSlots)) * kNumCounters;
#pragma unroll
    for (int k = 0; k < kNumCounters; ++k)
        if (c[k]) atomicAdd(cnt + k, c[k]);
}

__device__ __forceinline__ void count_one(const SimParams &P, int r, int k,
                                          unsigned long long v)
{
    atomicAdd(P.counters + ((size_t)r * kRepSlots + (blockIdx.x % kRepSlots)) * kNumCounters + k,
              v);
}

}  // namespace hpmc
