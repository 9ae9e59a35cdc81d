// sidm_internal.cuh -- context layout and device helpers shared by the CUDA
// translation units of libsidm (sm_103a).  Nothing here is used by the CPU
// oracle; the two implementations share no code.
#pragma once

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sidm.h"

namespace sidm {

constexpr int kLeaf = 32;            // particles per leaf (one warp of queries)
constexpr int kMortonBits = 17;      // Morton bits per axis
constexpr int kHaloShift = 51;       // halo index sits above the 51 Morton bits
constexpr int kMaxHalos = 1024;
constexpr int kMaxNgb = 128;
constexpr int kMaxLevels = 12;       // tree levels including the leaf level
constexpr int kArityLog = 5;         // tree nodes have 2^kArityLog = 32 children: one per lane
constexpr int kArity = 1 << kArityLog;
constexpr int kStack = 160;          // traversal stack entries per warp
constexpr int kLamNX = 257;          // Lambda table: x = d / (h_i + h_j) in [0, 1]
constexpr int kLamNR = 65;           //               rho = h_min / h_max in [0, 1]
constexpr uint32_t kIdLimit = 1u << 27;

// Per-halo frame of the canonical geometry: cube [O, O + 2^(E+1))^3,
// Morton quantisation with 17 bits per axis.
struct HaloFrame {
    double O[3];
    double qs;         // Morton quantisation scale 2^(17-E-1) (a power of two)
    int E;
    float cube;        // 2^(E+1)
    float margin;      // pruning margin: 2^(E+1) * 2^-20 (canonical vs exact distance)
    float fine;        // finest Morton cell edge 2^(E+1-17)
};

// Internal device counters (one struct, zeroed where each call needs it).
struct DevCounters {
    unsigned long long ev_count;     // events drawn this step
    unsigned long long de_lo;        // 128-bit fixed-point sum of pair dE (2^-80 units)
    unsigned long long de_hi;
    unsigned int work[4];            // persistent work-queue counters; [2], [3]: grid barrier
    unsigned int status;             // sticky SIDM_DEV_* bits (cleared by sidm_status)
    unsigned int pad;
    unsigned int knn_redo[2];        // leaves the warm-started search hands to the exhaustive one; its work counter
    unsigned long long diag[8];      // diagnostics (sidm_diagnostics)
    unsigned long long bbox[kMaxHalos * 6];   // ordered bits of per-halo min/max
};

struct LayoutHost {
    int H = 0;
    int64_t N = 0, Npad = 0;
    int L = 0;                                   // leaves
    int nlev = 1;                                // tree levels incl. leaves
    std::vector<int64_t> halo_off, halo_pad;
    std::vector<int32_t> leaf_off;               // [H+1]
    std::vector<int32_t> lvl_off;                // [nlev][H+1]
    std::vector<int32_t> top;                    // [H] start level of the traversal
    std::vector<int32_t> chunk_halo;             // energy reduction chunks
    std::vector<int64_t> chunk_begin;
    int nchunk = 0;
    std::vector<int32_t> chunk_off, group_off;   // per halo: first chunk, first group of chunks
    int ngroup = 0;
    int sort_passes = 7;
};

}  // namespace sidm

struct sidm_ctx {
    sidm_config cfg{};
    int dev = 0;
    int sm_count = 0;
    std::string err;
    int64_t launches = 0;
    bool has_layout = false, built = false, sized = false, stepped = false;
    sidm::LayoutHost lay;
    std::vector<int32_t> ngb_host;               // cached N_ngb (uploaded when changed)
    int kmax_cur = 0;

    // warm start of the kernel-size search: the last h per particle (in the
    // order of the caller's arrays after that call), and whether the next
    // build may seed P4.w with it / the last build did
    void* d_hprev = nullptr;           // f32|f64 [N]
    bool warm_enabled = true;
    bool hprev_valid = false;
    bool guess_in_p4 = false;
    std::vector<int32_t> ngb_prev;     // N_ngb of the call that wrote d_hprev

    // layout arrays (device)
    int64_t* d_halo_off = nullptr;     // [H+1]
    int64_t* d_halo_pad = nullptr;     // [H+1]
    int32_t* d_leaf_off = nullptr;     // [H+1]
    int32_t* d_lvl_off = nullptr;      // [kMaxLevels][H+1]
    int32_t* d_top = nullptr;          // [H]
    int32_t* d_ngb = nullptr;          // [H]
    int32_t* d_leaf_halo = nullptr;    // [Lmax]
    int32_t* d_knn_redo = nullptr;     // [Lmax] leaves whose warm-started kernel-size search is redone
    int32_t* d_chunk_halo = nullptr;   // [chunks]
    int64_t* d_chunk_begin = nullptr;  // [chunks]
    sidm::HaloFrame* d_frame = nullptr;  // [H]
    int64_t* d_stage = nullptr;        // host-pinned staging for layout uploads
    size_t stage_bytes = 0;

    // sort
    unsigned long long* d_key = nullptr;
    unsigned long long* d_key2 = nullptr;
    uint32_t* d_val = nullptr;
    uint32_t* d_val2 = nullptr;
    unsigned long long* d_sort_status = nullptr;   // radix sort look-back words, [tiles][256]
    uint32_t* d_sort_hist = nullptr;               // digit counts [8][256], then 8 tile tickets
    int64_t sort_tiles_cap = 0;

    // particles (padded per halo to multiples of 32 slots)
    void* d_P4 = nullptr;              // float4 (ox,oy,oz,h) | double4 (x,y,z,h)
    void* d_V4 = nullptr;              // float4 (vx,vy,vz,id) | double4
    uint32_t* d_ID = nullptr;          // ids by slot
    float4* d_cell = nullptr;          // [Lmax] leaf frame origin relative to O
    double4* d_cellb = nullptr;        // [Lmax] RN64(O + origin) per axis (the mixed form's gather)
    float4* d_nlo = nullptr;           // [nodes] bbox lo (w = max h)
    float4* d_nhi = nullptr;           // [nodes] bbox hi
    int64_t node_cap = 0;
    uint32_t* d_perm = nullptr;        // [N] sorted position -> previous index
    double* d_tmp_pos = nullptr;       // [3][N]
    void* d_tmp_vel = nullptr;         // [3][N]
    uint32_t* d_tmp_id = nullptr;      // [N]

    // scatter
    unsigned long long* d_claim = nullptr;  // [N] resolve claims (all ones at rest)
    uint32_t* d_hits = nullptr;             // [N] events per particle (zero at rest)
    uint8_t* d_done = nullptr;              // [event_cap]
    sidm_event* d_ev = nullptr;             // [event_cap]
    float* d_sump = nullptr;                // [N] (SIDM_FLAG_SUM_P)
    double* d_dacc = nullptr;               // [5][N] kernel-weighted moments (SIDM_FLAG_LOCAL_DIAG)
    // forward-dominated halos (SIDM_FLAG_DRAG): per-record G = m_j Lambda dt, and
    // the per-particle interaction lists (2 entries per record, key = particle
    // index << 27 | partner id, sorted), their starts/lengths, round pointers,
    // active lists and counters
    double* d_evg = nullptr;                // [event_cap]
    unsigned long long* d_lkey = nullptr;   // [2][2 event_cap] ping-pong
    uint32_t* d_lval = nullptr;             // [2][2 event_cap]
    uint32_t* d_lstart = nullptr;           // [N]
    uint32_t* d_llen = nullptr;             // [N]
    uint32_t* d_lptr = nullptr;             // [N] (zero at rest)
    uint32_t* d_lact = nullptr;             // [2][N]
    uint32_t* d_lcnt = nullptr;             // [8] active counts, multi-hit count, rounds, status
    double gl8x[8] = {}, gl8w[8] = {};      // 8-point Gauss-Legendre rule (Lambda quadrature on the device)
    unsigned long long* d_halo_ord = nullptr;  // [H] per-halo minima (order-preserving bits)

    // individual time steps of the scatter step in flight (set by
    // sidm_scatter_step_binned for one launch, NULL otherwise)
    const int32_t* step_bins = nullptr;
    int step_nbins = 1, step_sub = 0;
    double step_dtmax = 0.0;
    sidm_step_stats* d_stats_own = nullptr; // used when the caller passes NULL
    sidm::DevCounters* d_cnt = nullptr;

    // energy partials
    double* d_epart = nullptr;         // [chunks][8]
    int32_t* d_chunk_off = nullptr;    // [H+1] first energy chunk of each halo
    int32_t* d_group_off = nullptr;    // [H+1] first group of chunks of each halo
    double* d_gpart = nullptr;         // [groups][8] group sums of the energy reduction
    int64_t chunk_cap = 0;

    // Lambda table (float or double [kLamNR][kLamNX])
    void* d_lam = nullptr;

    int knn_grid = 0, pair_grid = 0, knn_warps = 4, pair_warps = 4;

    // launch configuration cache: (kernel, dynamic smem) -> CTAs per SM, so
    // that repeated calls issue stream operations only
    struct LaunchCfg { const void* fn; size_t smem; int occ; };
    std::vector<LaunchCfg> launch_cache;

    // CUDA-event timing of hot kernels (SIDM_FLAG_TIMING): pairs of events
    std::vector<cudaEvent_t> t_ev;     // [2 * kTimerCap]
    std::vector<int8_t> t_slot;        // [kTimerCap]
    int t_used = 0;
};

namespace sidm {

// ---------------------------------------------------------------- launches
int set_err(sidm_ctx* c, int code, const std::string& msg);
int cuda_check(sidm_ctx* c, cudaError_t e, const char* what);

// event timing (no-ops unless SIDM_FLAG_TIMING): slot 0 build, 1 knn, 2 pairs, 3 resolve
constexpr int kTimerCap = 4096;
int timer_begin(sidm_ctx* c, int slot, cudaStream_t s);
void timer_end(sidm_ctx* c, int idx, cudaStream_t s);

// make the context's device current (no call if it already is)
cudaError_t ensure_device(sidm_ctx* c);

// CTAs per SM of a kernel at a dynamic shared-memory size (cached per context;
// sets the kernel's dynamic shared-memory limit on first use)
int occupancy(sidm_ctx* c, const void* fn, int threads, size_t smem, int* occ);

// kernel entry points implemented in the other translation units
int launch_knn(sidm_ctx* c, void* h_out, uint32_t* nbr, int k_stride, bool use_guess, cudaStream_t s);
int launch_pairs(sidm_ctx* c, uint64_t seed, uint64_t step, const sidm_xs* xs, const double* dt,
                 const double* mass, sidm_step_stats* st, cudaStream_t s);
int launch_pairs_diag(sidm_ctx* c, const sidm_xs* xs, const double* mass, cudaStream_t s);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ void raise_status(DevCounters* cnt, unsigned int bits)
{
    atomicOr(&cnt->status, bits);
}

// Philox4x32-10 block (Salmon et al. 2011): per round the products
// M0*c0 and M1*c2 are split into high/low words and mixed with c1, c3 and the
// key; the key advances by the Weyl constants after each round.
struct Philox4 { uint32_t x[4]; };

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;   // one 32x32->64 product
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        const uint32_t y0 = hi1 ^ c1 ^ k0;
        const uint32_t y2 = hi0 ^ c3 ^ k1;
        c0 = y0; c1 = lo1; c2 = y2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    Philox4 o; o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
    return o;
}

// The same block with the round keys given (rk[2r], rk[2r+1] = key + r * Weyl
// pair, mod 2^32); a launch passes them as kernel parameters, so a round is the
// two products and two three-way xors.
__device__ __forceinline__ Philox4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                    const uint32_t* rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        const uint32_t y0 = hi1 ^ c1 ^ rk[2 * r];
        const uint32_t y2 = hi0 ^ c3 ^ rk[2 * r + 1];
        c0 = y0; c1 = lo1; c2 = y2; c3 = lo0;
    }
    Philox4 o; o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
    return o;
}

// Lagrange cubic weights on nodes 0..3 at parameter t.
template <class R>
__device__ __forceinline__ void lagrange4(R t, R w[4])
{
    const R t1 = t - R(1), t2 = t - R(2), t3 = t - R(3);
    w[0] = -(t1 * t2 * t3) * (R(1) / R(6));
    w[1] = (t * t2 * t3) * R(0.5);
    w[2] = -(t * t1 * t3) * R(0.5);
    w[3] = (t * t1 * t2) * (R(1) / R(6));
}

// Upper bound of the interpolated table value f = h_max^3 Lambda: the exact
// overlap obeys Lambda <= W(0, h_max) and the largest tabulated value is
// h^3 Lambda(0; h, h) = 0.9923; a 4 x 4-point Lagrange interpolant can exceed
// the largest node value by at most the square of the cubic Lebesgue constant
// (1.631^2 = 2.66), so no interpolated f exceeds 2.64 < 4.
constexpr float kLamFUp = 4.0f;

// Lambda(d; h_i, h_j) from the table f(x, rho) = h_max^3 Lambda,
// x = d / (h_i + h_j), rho = h_min / h_max, Lagrange-bicubic on a
// uniform 257 x 65 grid.
template <class R>
__device__ __forceinline__ R lambda_f(const R* __restrict__ T, R d, R hi, R hj)
{
    const R hmax = hi > hj ? hi : hj;
    const R hmin = hi > hj ? hj : hi;
    R x = d / (hi + hj);
    if (!(x < R(1))) return R(0);
    if (x < R(0)) x = R(0);
    const R rho = hmin / hmax;
    const R gx = x * R(kLamNX - 1);
    int ix = (int)floor(gx) - 1;
    ix = ix < 0 ? 0 : (ix > kLamNX - 4 ? kLamNX - 4 : ix);
    const R gr = rho * R(kLamNR - 1);
    int ir = (int)floor(gr) - 1;
    ir = ir < 0 ? 0 : (ir > kLamNR - 4 ? kLamNR - 4 : ir);
    R wx[4], wr[4];
    lagrange4<R>(gx - R(ix), wx);
    lagrange4<R>(gr - R(ir), wr);
    R f = R(0);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const R* row = T + (ir + a) * kLamNX + ix;
        const R s = wx[0] * __ldg(row) + wx[1] * __ldg(row + 1) + wx[2] * __ldg(row + 2) + wx[3] * __ldg(row + 3);
        f += wr[a] * s;
    }
    return f;
}

// Lambda(d; h_i, h_j) = f(x, rho) / h_max^3.
template <class R>
__device__ __forceinline__ R lambda_lookup(const R* __restrict__ T, R d, R hi, R hj)
{
    const R hmax = hi > hj ? hi : hj;
    const R inv = R(1) / hmax;
    return lambda_f<R>(T, d, hi, hj) * inv * inv * inv;
}

// FP32 interpolated f with approximate reciprocals (relative error ~1e-7,
// far below the table's own 1e-6 of the peak); inv = 1/h_max from the caller.
__device__ __forceinline__ float lambda_f_fast(const float* __restrict__ T, float d, float hi, float hj, float inv)
{
    const float hmin = fminf(hi, hj);
    float x = __fdividef(d, hi + hj);
    if (!(x < 1.f)) return 0.f;
    x = fmaxf(x, 0.f);
    const float rho = hmin * inv;
    const float gx = x * (float)(kLamNX - 1);
    int ix = (int)floorf(gx) - 1;
    ix = ix < 0 ? 0 : (ix > kLamNX - 4 ? kLamNX - 4 : ix);
    const float gr = rho * (float)(kLamNR - 1);
    int ir = (int)floorf(gr) - 1;
    ir = ir < 0 ? 0 : (ir > kLamNR - 4 ? kLamNR - 4 : ir);
    float wx[4], wr[4];
    lagrange4<float>(gx - (float)ix, wx);
    lagrange4<float>(gr - (float)ir, wr);
    float f = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const float* row = T + (ir + a) * kLamNX + ix;
        f = fmaf(wr[a], wx[0] * __ldg(row) + wx[1] * __ldg(row + 1) + wx[2] * __ldg(row + 2) + wx[3] * __ldg(row + 3), f);
    }
    return f;
}

__device__ __forceinline__ float lambda_lookup_fast(const float* __restrict__ T, float d, float hi, float hj)
{
    const float inv = __fdividef(1.f, fmaxf(hi, hj));
    return lambda_f_fast(T, d, hi, hj, inv) * inv * inv * inv;
}

// Lambda(d; a, b) by quadrature, for pairs whose result must be accurate
// relative to Lambda itself (the forward-dominated turn, whose sine is the
// square root of a multiple of Lambda): the overlap of spline kernels of
// support a (at the origin) and b (at distance d),
//   Lambda = (2 pi / d) int r W_a(r) [S_b(r + d) - S_b(|r - d|)] dr,
//   S_b(s) = S_1(s/b) / b,  S_1(t) = int_0^t t' W_1(t') dt' (closed form),
// over r in [max(0, d - b), min(a, d + b)], split at the breakpoints of the
// polynomial pieces and integrated with the 8-point Gauss-Legendre rule
// (gx, gw on [-1, 1]), exact for each piece up to rounding.  d = 0 takes the
// limit 4 pi int r^2 W_a W_b dr.
template <class R>
__device__ __forceinline__ R spline_w1_q(R t)
{
    const R c = R(8.0 / 3.14159265358979323846);
    if (!(t < R(1)) || t < R(0)) return R(0);
    if (t < R(0.5)) return c * (R(1) - R(6) * t * t + R(6) * t * t * t);
    const R u = R(1) - t;
    return c * R(2) * u * u * u;
}

template <class R>
__device__ __forceinline__ R spline_s1_q(R t)
{
    const R c = R(8.0 / 3.14159265358979323846);
    auto inner = [&](R q) { return c * (R(0.5) * q * q - R(1.5) * q * q * q * q + R(1.2) * q * q * q * q * q); };
    auto outer = [&](R q) { const R u = R(1) - q; return R(-2) * c * (R(0.25) * u * u * u * u - R(0.2) * u * u * u * u * u); };
    if (!(t > R(0))) return R(0);
    if (t < R(0.5)) return inner(t);
    const R q = t < R(1) ? t : R(1);
    return inner(R(0.5)) + outer(q) - outer(R(0.5));
}

template <class R>
__device__ R lambda_quad(R d, R a, R b, const R* gx, const R* gw)
{
    if (!(d < a + b)) return R(0);
    R br[12];
    int nb = 0;
    R lo, hi;
    if (d == R(0)) {
        lo = R(0); hi = a < b ? a : b;
        br[nb++] = lo; br[nb++] = hi;
        const R c2[2] = {R(0.5) * a, R(0.5) * b};
        for (int k = 0; k < 2; ++k) if (c2[k] > lo && c2[k] < hi) br[nb++] = c2[k];
    } else {
        lo = d - b > R(0) ? d - b : R(0);
        hi = a < d + b ? a : d + b;
        if (!(hi > lo)) return R(0);
        br[nb++] = lo; br[nb++] = hi;
        const R c9[9] = {R(0.5) * a, a, d, d - R(0.5) * b, d + R(0.5) * b, d - b, d + b, R(0.5) * b - d, b - d};
        for (int k = 0; k < 9; ++k) if (c9[k] > lo && c9[k] < hi) br[nb++] = c9[k];
    }
    for (int i = 1; i < nb; ++i) {                       // insertion sort of the breakpoints
        const R v = br[i];
        int j = i - 1;
        while (j >= 0 && br[j] > v) { br[j + 1] = br[j]; --j; }
        br[j + 1] = v;
    }
    const R ia = R(1) / a, ib = R(1) / b;
    R acc = R(0);
    for (int pc = 0; pc + 1 < nb; ++pc) {
        const R m = R(0.5) * (br[pc] + br[pc + 1]), hw = R(0.5) * (br[pc + 1] - br[pc]);
        if (!(hw > R(0))) continue;
        R sum = R(0);
        for (int g = 0; g < 8; ++g) {
            const R r = m + hw * gx[g];
            const R wa = spline_w1_q<R>(r * ia) * ia * ia * ia;
            if (d == R(0)) {
                sum += gw[g] * r * r * wa * spline_w1_q<R>(r * ib) * ib * ib * ib;
            } else {
                const R rd = r - d;
                sum += gw[g] * r * wa * (spline_s1_q<R>((r + d) * ib) - spline_s1_q<R>((rd < R(0) ? -rd : rd) * ib)) * ib;
            }
        }
        acc += hw * sum;
    }
    const R two_pi = R(2.0 * 3.14159265358979323846);
    return d == R(0) ? R(2) * two_pi * acc : two_pi * acc / d;
}

// Lower bound of the squared distance from a point to a box (FP32, rounded down).
__device__ __forceinline__ float point_gap2_rd(float3 p, float4 lo, float4 hi)
{
    float gx = fmaxf(0.f, fmaxf(__fsub_rd(lo.x, p.x), __fsub_rd(p.x, hi.x)));
    float gy = fmaxf(0.f, fmaxf(__fsub_rd(lo.y, p.y), __fsub_rd(p.y, hi.y)));
    float gz = fmaxf(0.f, fmaxf(__fsub_rd(lo.z, p.z), __fsub_rd(p.z, hi.z)));
    return __fadd_rd(__fadd_rd(__fmul_rd(gx, gx), __fmul_rd(gy, gy)), __fmul_rd(gz, gz));
}

// Lower bound of the squared gap between two boxes (FP32, rounded down).
__device__ __forceinline__ float box_gap2_rd(float4 alo, float4 ahi, float4 blo, float4 bhi)
{
    float gx = fmaxf(0.f, fmaxf(__fsub_rd(blo.x, ahi.x), __fsub_rd(alo.x, bhi.x)));
    float gy = fmaxf(0.f, fmaxf(__fsub_rd(blo.y, ahi.y), __fsub_rd(alo.y, bhi.y)));
    float gz = fmaxf(0.f, fmaxf(__fsub_rd(blo.z, ahi.z), __fsub_rd(alo.z, bhi.z)));
    return __fadd_rd(__fadd_rd(__fmul_rd(gx, gx), __fmul_rd(gy, gy)), __fmul_rd(gz, gz));
}

// Order-preserving map of a double to unsigned 64-bit (for atomic min/max).
__device__ __forceinline__ unsigned long long dbl_to_ord(double v)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_to_dbl(unsigned long long u)
{
    u = (u & 0x8000000000000000ull) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
    return __longlong_as_double((long long)u);
}

template <class R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4_16a; };   // 16-byte aligned, as staged

}  // namespace sidm
